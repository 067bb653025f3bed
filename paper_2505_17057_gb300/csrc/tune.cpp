// tune.cpp -- the autotuner: times (temporal depth, work-item height) candidates of a solver's
// step kernel on its own grid and keeps the fastest; optional text cache of earlier choices.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "solver.h"

namespace mmfd {

namespace {

std::string tune_key(const Solver* s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop{};
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ' || c == '|') c = '_';
    std::ostringstream k;
    k << name << ":" << sms << ":lat" << s->r.lat << ":pde" << s->r.pde << ":lev" << s->r.levels << ":st" << s->r.st
      << ":fl" << s->desc.flags << ":n" << s->g.nx << "x" << s->g.ny << "x" << s->g.nz << ":depth"
      << (s->desc.temporal_depth == 0 ? std::string("auto") : std::to_string(s->depth));
    return k.str();
}

// Cache line: key depth height ms
bool cache_lookup(const char* path, const std::string& key, int* depth, int* h, double* ms) {
    std::ifstream in(path);
    if (!in) return false;
    std::string line;
    bool found = false;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string k;
        int d = 0, hh = 0;
        double m = 0;
        if (ls >> k >> d >> hh >> m && k == key && d >= 1 && hh >= 0) {
            *depth = d;
            *h = hh;
            *ms = m;
            found = true;  // the last entry for a key wins
        }
    }
    return found;
}

void cache_append(const char* path, const std::string& key, int depth, int h, double ms) {
    std::ofstream out(path, std::ios::app);
    if (out) out << key << " " << depth << " " << h << " " << ms << "\n";
}

}  // namespace

int solver_autotune(Solver* s, const char* cache_path, mmfd_tune_info* out) {
    const std::string key = tune_key(s);
    const bool auto_depth = s->desc.temporal_depth == 0 && s->max_depth >= 2;
    mmfd_tune_info info{};
    int cd = 0, ch = 0;
    double cms = 0;
    if (cache_path && cache_lookup(cache_path, key, &cd, &ch, &cms) && cd <= (auto_depth ? s->max_depth : s->depth) &&
        (auto_depth || cd == s->depth)) {
        if (auto_depth) solver_use_depth(s, cd);
        s->H = s->use_tma ? ch : 0;
        info.temporal_depth = s->depth;
        info.rows_per_item = s->H;
        info.ms_per_step = cms;
        info.from_cache = 1;
        if (out) *out = info;
        return MMFD_OK;
    }

    std::vector<int> depths;
    if (auto_depth)
        for (int d = 1; d <= s->max_depth; ++d) depths.push_back(d);
    else
        depths.push_back(s->depth);
    std::vector<int> heights = {0};
    if (s->use_tma) {
        if (s->r.dim == 2) heights.insert(heights.end(), {4, 8, 16, 32, 64, 128});
        else heights.insert(heights.end(), {8, 16, 32, 64, 128});
    }

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    const int keep_depth = s->depth;
    const int keep_h = s->H;
    double best = -1.0;
    int best_d = keep_depth, best_h = keep_h;
    int rc = MMFD_OK;
    // one sample = `reps` back-to-back launches; reps is sized from a probe so that a sample
    // lasts about a millisecond, and the median of three samples is kept (single short samples
    // picked different heights from run to run)
    auto sample = [&](LaunchFn fn, const LaunchArgs& a, int reps, float* ms) -> cudaError_t {
        cudaError_t e2 = cudaEventRecord(e0, s->stream);
        for (int r = 0; r < reps && e2 == cudaSuccess; ++r) e2 = fn(a);
        if (e2 == cudaSuccess) e2 = cudaEventRecord(e1, s->stream);
        if (e2 == cudaSuccess) e2 = cudaEventSynchronize(e1);
        if (e2 == cudaSuccess) e2 = cudaEventElapsedTime(ms, e0, e1);
        return e2;
    };
    for (int d : depths) {
        solver_use_depth(s, d);
        LaunchFn fn = d >= 2 ? s->fn_block : s->fn;
        if (!fn || (d >= 2 && s->depth != d)) continue;
        for (int h : heights) {
            LaunchArgs a;
            solver_launch_args(s, a);   // reads the current level(s), writes the spare buffer only
            a.H = h;
            float probe = 0.f;
            e = fn(a);                  // warm-up (the first launch also sets the kernel's attributes)
            if (e == cudaSuccess) e = fn(a);
            if (e == cudaSuccess) e = sample(fn, a, 1, &probe);
            int reps = probe > 0.f ? (int)(1.0f / probe) + 1 : 1;
            if (reps > 50) reps = 50;
            float t[3] = {0.f, 0.f, 0.f};
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = sample(fn, a, reps, &t[k]);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune trial launch");
                break;
            }
            ++info.candidates;
            const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
            const double per_step = (double)med / ((double)reps * d);
            if (best < 0 || per_step < best) {
                best = per_step;
                best_d = d;
                best_h = h;
            }
        }
        if (rc != MMFD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == MMFD_OK) rc = solver_check_flag(s);
    if (rc != MMFD_OK || best < 0) {
        solver_use_depth(s, keep_depth);
        s->H = keep_h;
        return rc != MMFD_OK ? rc : set_error(MMFD_ERR_UNSUPPORTED, "no kernel configuration to tune");
    }
    solver_use_depth(s, best_d);
    s->H = best_h;
    info.temporal_depth = s->depth;
    info.rows_per_item = s->H;
    info.ms_per_step = best;
    if (cache_path) cache_append(cache_path, key, s->depth, s->H, best);
    if (out) *out = info;
    return MMFD_OK;
}

}  // namespace mmfd

extern "C" int mmfd_autotune(mmfd_solver* h, const char* cache_path, mmfd_tune_info* out) {
    using namespace mmfd;
    Solver* s = reinterpret_cast<Solver*>(h);
    if (!s) return set_error(MMFD_ERR_ARG, "null solver");
    return solver_autotune(s, cache_path, out);
}
