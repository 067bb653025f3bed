// serve.cpp -- persistent solve server with continuous batching (mmfd_server_* of mmfd.h).
//
// Scheduler (driven by mmfd_poll / mmfd_server_drain, never blocking in poll):
//   1. reap ticks whose completion event fired; their finishing requests become DONE;
//   2. admit queued requests, in arrival order, while a slot is free and the HBM footprint
//      (level buffers + coefficients) fits the budget; upload their initial level;
//   3. launch one tick: steps_per_tick steps of every active request; per step, one batched
//      grid-stride launch per kernel class (lattice, PDE, levels, storage) covering all of that
//      class's requests -- uneven grids packed into one launch (or, with MMFD_SERVE_QUEUE=1,
//      one launch per class for all the tick's steps: a device work queue of (step, tile) items
//      with bounded waits on each request's previous step); the tick's launches are
//      captured once per batch composition as a CUDA graph and replayed;
//   4. record the tick's event.
// At most two ticks are in flight, so host scheduling overlaps GPU work.  Requests share no
// state: each node's update reads only its own request's buffers and coefficients.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/mmfd.h"
#include "batch.h"
#include "kernels.h"
#include "params.h"
#include "solver.h"

namespace mmfd {

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum ReqState { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Req {
    unsigned long long ticket = 0;
    mmfd_desc desc{};
    Resolved* r = nullptr;
    Geom g{};
    std::vector<unsigned char> init;  // host copy of the initial level (nf x N x esz)
    int dtype = 0;
    long long nsteps = 0;
    long long launched = 0;  // steps covered by launched ticks
    int state = RQ_QUEUED;
    void* lev[3] = {nullptr, nullptr, nullptr};
    int nlev = 2;
    int cur = 0;
    void* d_coef = nullptr;
    size_t footprint = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int status = MMFD_OK;
    int cls = 0;
    // large requests run their own TMA march launches instead of joining a batched launch;
    // two-level 2D ones advance solo_depth steps per launch with the blocked kernel
    LaunchFn solo = nullptr;
    LaunchFn solo_tb = nullptr;
    int solo_depth = 1;
    CUtensorMap tmaps[3][4] = {};   // march solos only (the direct kernel takes none)
};

// A request this large is stepped with its own single-solve launches (the march kernel when it
// is at least 128 columns wide in 2D or 64 in 3D, else the direct kernel); smaller ones are
// packed into the batched kernel of their class.  A 3D grid of 64 .. 127 columns fills only part
// of the GPU with march items, which is why a single solve keeps the direct kernel there; in the
// server the solos of several requests run side by side and fill it.
constexpr long long kSoloNodes = 1ll << 16;

struct ClassTables {
    BatchFn fn = nullptr;
    QueueFn qfn = nullptr;                 // the work-queue kernel of the class (MMFD_SERVE_QUEUE=1)
    unsigned* ctl = nullptr;               // its control words: head, abort, per-request counters
    std::vector<Req*> members;
    BatchItem* h[2] = {nullptr, nullptr};  // pinned host tables (double-buffered)
    BatchItem* d[2] = {nullptr, nullptr};  // device tables
    int cap = 0;
};

struct TickRec {
    cudaEvent_t done = nullptr;
    int parity = 0;
    std::vector<Req*> finishing;
};

int class_of(const Resolved& r) { return ((r.lat * 3 + r.pde) * 2 + (r.levels - 2)) * 3 + r.st; }

}  // namespace

struct Server {
    mmfd_server_desc d{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    std::map<unsigned long long, Req*> reqs;
    std::deque<Req*> queue;
    std::vector<Req*> active;
    std::map<int, ClassTables> classes;
    std::deque<TickRec> inflight;
    mmfd_server_stats st{};
    unsigned long long next_ticket = 1;
    int parity = 0;
    int sms = 152;
    int* d_flag = nullptr;  // device error flag for the kernels' bounded waits
    // MMFD_SERVE_QUEUE=1 at server creation: the batched classes run all steps of a tick as one
    // work-queue launch (k_batch_queue) instead of one k_batch launch per step
    bool use_queue = false;
    unsigned queue_stall = 0;   // MMFD_SERVE_QUEUE_STALL=1: every queue wait runs out (failure-detection test)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // graph cache: composition key -> executable graph
    std::map<std::string, cudaGraphExec_t> graphs;
    std::deque<std::string> graph_lru;
    // side streams: a tick forks its solo requests across them so that their launches overlap
    // on the GPU (each request stays on one stream within the tick; the join at the end of a
    // tick orders it before the next tick's fork)
    static constexpr int kSide = 8;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kSide] = {};
};

namespace {

int srv_alloc(Server* s, size_t bytes, void** p) {
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, s->pool, s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MMFD_ERR_OOM, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
    }
    return MMFD_OK;
}

void srv_free(Server* s, void* p) {
    if (p) cudaFreeAsync(p, s->stream);
}

size_t footprint_of(const Resolved& r, const Geom& g) {
    const size_t level = (size_t)g.fs * g.nf * g.es;
    return level * (size_t)(r.levels == 3 ? 3 : 2) + sizeof(Coef<double>);
}

int ensure_stage(Server* s, size_t need) {
    if (s->stage && s->stage_bytes >= need) return MMFD_OK;
    if (s->stage) srv_free(s, s->stage);
    s->stage = nullptr;
    int rc = srv_alloc(s, need, &s->stage);
    if (rc == MMFD_OK) s->stage_bytes = need;
    return rc;
}

int admit(Server* s, Req* q) {
    const int nl = q->r->levels == 3 ? 3 : 2;
    q->nlev = nl;
    const size_t level = (size_t)q->g.fs * q->g.nf * q->g.es;
    for (int i = 0; i < nl; ++i) {
        int rc = srv_alloc(s, level, &q->lev[i]);
        if (rc != MMFD_OK) return rc;
        cudaError_t e = cudaMemsetAsync(q->lev[i], 0, level, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    int rc = srv_alloc(s, sizeof(Coef<double>), &q->d_coef);
    if (rc != MMFD_OK) return rc;
    const void* coef = q->r->st == ST_F64 ? static_cast<const void*>(&q->r->cd) : static_cast<const void*>(&q->r->cf);
    const size_t cbytes = q->r->st == ST_F64 ? sizeof(Coef<double>) : sizeof(Coef<float>);
    cudaError_t e = cudaMemcpyAsync(q->d_coef, coef, cbytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync coef");
    const long long N = (long long)q->g.nx * q->g.ny * q->g.nz;
    const size_t esz = q->dtype == MMFD_DT_F64 ? 8 : 4;
    rc = ensure_stage(s, (size_t)N * esz);
    if (rc != MMFD_OK) return rc;
    for (int f = 0; f < q->g.nf; ++f) {
        e = cudaMemcpyAsync(s->stage, q->init.data() + (size_t)f * N * esz, (size_t)N * esz, cudaMemcpyHostToDevice,
                            s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync init");
        for (int lv = 0; lv < (nl == 3 ? 2 : 1); ++lv) {
            // three-level requests start from phi^{-1} := phi^0 (level index 2 = prev of cur 0)
            void* dst = q->lev[lv == 0 ? 0 : 2];
            e = launch_pack(q->g, q->r->st, s->stage, q->dtype, dst, f, q->r->ref[f], s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
        }
    }
    q->init.clear();
    q->init.shrink_to_fit();
    q->solo = nullptr;
    const bool large = (long long)q->g.nx * q->g.ny * q->g.nz >= kSoloNodes;
    if (large && q->g.nx >= (q->g.dim == 3 ? 64 : 128)) {
        LaunchFn fn = find_march_lean(q->r->lat, q->r->levels, q->r->st, q->r->lean);
        if (!fn)
            fn = q->g.dim == 2 ? find_march2d(q->r->lat, q->r->pde, q->r->levels, q->r->st)
                               : find_march3d(q->r->lat, q->r->pde, q->r->levels, q->r->st);
        bool ok = fn != nullptr;
        const int boxw = 128 + 2 * (16 / q->g.es);
        const int boxh = q->g.dim == 2 ? march2d_rows_per_stage(q->r->pde) : march3d_tile_rows(q->r->pde) + 2;
        for (int b = 0; ok && b < nl; ++b)
            for (int f = 0; ok && f < q->g.nf; ++f) {
                char* base = static_cast<char*>(q->lev[b]) + (size_t)f * q->g.fs * q->g.es;
                ok = encode_field_map(&q->tmaps[b][f], base, q->r->st, q->g, boxw, boxh, 1) == 0;
            }
        if (ok) q->solo = fn;
        // temporal blocking for two-level 2D solos (the blocked kernel reads the same 2-row maps)
        if (ok && q->g.dim == 2 && nl == 2 && march2d_rows_per_stage(q->r->pde) == 2) {
            int depth = march2d_tb_max_depth(q->r->st);
            const int S = s->d.steps_per_tick > 0 ? s->d.steps_per_tick : 1;
            while (depth >= 2 && (q->g.ny < 2 * depth || depth > S)) --depth;
            if (depth >= 2) {
                q->solo_tb = find_march2d_tb(q->r->lat, q->r->pde, 2, q->r->st, depth);
                q->solo_depth = q->solo_tb ? depth : 1;
            }
        }
    }
    // a large request too narrow for the march kernels runs its own one-node-per-thread
    // launches: they take the coefficients as a kernel parameter, where the batched kernel reads
    // them from its device table at every use
    if (large && !q->solo) q->solo = find_direct(q->r->lat, q->r->pde, q->r->levels, q->r->st);
    q->cur = 0;
    q->state = RQ_ACTIVE;
    q->t_admit = now_s();
    s->st.admitted++;
    return MMFD_OK;
}

void reap(Server* s, bool block) {
    while (!s->inflight.empty()) {
        TickRec& t = s->inflight.front();
        cudaError_t e = block ? cudaEventSynchronize(t.done) : cudaEventQuery(t.done);
        if (e == cudaErrorNotReady) return;
        const double tf = now_s();
        for (Req* q : t.finishing) {
            q->state = (e == cudaSuccess) ? RQ_DONE : RQ_FAILED;
            q->status = (e == cudaSuccess) ? MMFD_OK : MMFD_ERR_CUDA;
            q->t_finish = tf;
            s->st.finished++;
        }
        cudaEventDestroy(t.done);
        s->inflight.pop_front();
        if (e != cudaSuccess && e != cudaErrorNotReady) cudaGetLastError();
        if (block) block = false;  // only wait for the oldest
    }
}

int ensure_tables(Server* s, ClassTables& c, int n) {
    if (c.cap >= n) return MMFD_OK;
    int cap = c.cap ? c.cap : 16;
    while (cap < n) cap *= 2;
    while (!s->inflight.empty()) reap(s, true);  // old tables may still feed in-flight copies
    for (int p = 0; p < 2; ++p) {
        if (c.h[p]) cudaFreeHost(c.h[p]);
        if (c.d[p]) srv_free(s, c.d[p]);
        c.h[p] = nullptr;
        c.d[p] = nullptr;
        if (cudaMallocHost(reinterpret_cast<void**>(&c.h[p]), sizeof(BatchItem) * cap) != cudaSuccess) {
            cudaGetLastError();
            return set_error(MMFD_ERR_OOM, "cudaMallocHost for batch tables failed");
        }
        int rc = srv_alloc(s, sizeof(BatchItem) * cap, reinterpret_cast<void**>(&c.d[p]));
        if (rc != MMFD_OK) return rc;
    }
    if (c.ctl) srv_free(s, c.ctl);
    c.ctl = nullptr;
    int rc = srv_alloc(s, sizeof(unsigned) * (size_t)(cap + 2), reinterpret_cast<void**>(&c.ctl));
    if (rc != MMFD_OK) return rc;
    c.cap = cap;
    return MMFD_OK;
}

int launch_tick(Server* s) {
    const int S = s->d.steps_per_tick > 0 ? s->d.steps_per_tick : 1;
    const int par = s->parity;
    // table buffers of this parity were last used two ticks ago: make sure that tick finished
    while (s->inflight.size() >= 2) reap(s, true);
    for (auto& kv : s->classes) kv.second.members.clear();
    std::vector<Req*> solos;
    for (Req* q : s->active) {
        if (q->state != RQ_ACTIVE || q->launched >= q->nsteps) continue;
        if (q->solo)
            solos.push_back(q);
        else
            s->classes[q->cls].members.push_back(q);
    }
    std::string key;
    struct Launch {
        BatchFn fn;
        const BatchItem* items;
        int n;
        long long total;
        QueueFn qfn;        // set when the class runs as one work-queue launch
        unsigned* ctl;
    };
    std::vector<Launch> launches;
    TickRec tick;
    tick.parity = par;
    long long lu = 0;
    for (auto& kv : s->classes) {
        ClassTables& c = kv.second;
        if (c.members.empty()) continue;
        if (!c.fn) {
            const Resolved& r = *c.members[0]->r;
            c.fn = find_batch(r.lat, r.pde, r.levels, r.st);
            c.qfn = find_batch_queue(r.lat, r.pde, r.levels, r.st);
            if (!c.fn) return set_error(MMFD_ERR_UNSUPPORTED, "no batched kernel for this class");
        }
        int rc = ensure_tables(s, c, (int)c.members.size());
        if (rc != MMFD_OK) return rc;
        long long tile0 = 0;
        int n = 0;
        for (Req* q : c.members) {
            BatchItem& it = c.h[par][n++];
            std::memset(&it, 0, sizeof(it));
            it.g = q->g;
            for (int i = 0; i < 3; ++i) it.lev[i] = q->lev[i];
            it.nlev = q->nlev;
            it.cur = q->cur;
            it.steps_left = q->nsteps - q->launched;
            it.step0 = q->launched;
            it.coef = q->d_coef;
            it.tile0 = tile0;
            tile0 += batch_tiles(q->g, &it.tx, &it.ty, &it.tz);
            it.sr = (q->r->st == ST_BF16 && (q->desc.flags & MMFD_FLAG_STOCHASTIC_ROUND)) ? 1 : 0;
            it.seed = q->desc.seed;
            const long long adv = it.steps_left < S ? it.steps_left : S;
            lu += adv * (long long)q->g.nx * q->g.ny * q->g.nz;
        }
        cudaError_t e = cudaMemcpyAsync(c.d[par], c.h[par], sizeof(BatchItem) * n, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync batch table");
        const bool queued = s->use_queue && c.qfn && tile0 * S < (1ll << 31);
        launches.push_back({c.fn, c.d[par], n, tile0, queued ? c.qfn : nullptr, c.ctl});
        key += std::to_string(kv.first) + (queued ? "q" : "") + ":" + std::to_string(n) + ":" + std::to_string(tile0) + ":" +
               std::to_string(reinterpret_cast<uintptr_t>(c.d[par])) + ";";
    }
    for (Req* q : solos) {
        const long long left = q->nsteps - q->launched;
        const long long adv = left < S ? left : S;
        lu += adv * (long long)q->g.nx * q->g.ny * q->g.nz;
        key += "solo:" + std::to_string(q->ticket) + ":" + std::to_string(q->cur) + ":" + std::to_string(adv) + ";";
    }
    if (launches.empty() && solos.empty()) return MMFD_OK;
    // one solo launch of request q: reads buffer c (and its predecessor for three-level), writes
    // the next buffer, advancing `steps` time levels from step index step0
    auto solo_launch = [&](Req* q, LaunchFn fn, int c, long long step0, int steps, cudaStream_t st) -> cudaError_t {
        const int nl = q->nlev;
        const int prev = nl == 3 ? (c + 2) % 3 : c;
        const int next = nl == 2 ? 1 - c : (c + 1) % 3;
        TmapSet maps;
        for (int f = 0; f < q->g.nf; ++f) {
            maps.m[f] = q->tmaps[c][f];
            if (nl == 3) maps.m[q->g.nf + f] = q->tmaps[prev][f];
        }
        LaunchArgs a;
        a.g = q->g;
        a.in0 = q->lev[c];
        a.in1 = nl == 3 ? q->lev[prev] : nullptr;
        a.out = q->lev[next];
        a.coef = q->r->st == ST_F64 ? static_cast<const void*>(&q->r->cd) : static_cast<const void*>(&q->r->cf);
        a.ex.seed = q->desc.seed;
        a.ex.step = step0 + steps;
        a.ex.sr = (q->r->st == ST_BF16 && (q->desc.flags & MMFD_FLAG_STOCHASTIC_ROUND)) ? 1 : 0;
        a.stream = st;
        a.variant = 0;
        a.maps = &maps;
        a.H = 0;
        a.err = s->d_flag;
        return fn(a);
    };
    // the tick's launches of solo request q: blocked launches while a full block of steps is
    // left, then single steps; returns the buffer index after them through *cur_after
    auto solo_tick = [&](Req* q, cudaStream_t st, int* cur_after) -> cudaError_t {
        const long long left = q->nsteps - q->launched;
        const long long adv = left < S ? left : S;
        int c = q->cur;
        long long done = 0;
        while (done < adv) {
            const bool blocked = q->solo_tb && adv - done >= q->solo_depth;
            const int steps = blocked ? q->solo_depth : 1;
            cudaError_t e = solo_launch(q, blocked ? q->solo_tb : q->solo, c, q->launched + done, steps, st);
            if (e != cudaSuccess) return e;
            s->st.launches++;
            c = q->nlev == 2 ? 1 - c : (c + 1) % 3;
            done += steps;
        }
        *cur_after = c;
        return cudaSuccess;
    };
    auto enqueue = [&]() -> cudaError_t {
        const int nside = solos.empty() ? 0 : (int)std::min<size_t>(solos.size(), Server::kSide);
        if (nside > 0) {
            cudaError_t e = cudaEventRecord(s->fork_ev, s->stream);
            for (int k = 0; k < nside && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s->side[k], s->fork_ev, 0);
            if (e != cudaSuccess) return e;
        }
        for (const Launch& L : launches) {
            if (!L.qfn) continue;
            cudaError_t e = cudaMemsetAsync(L.ctl, 0, sizeof(unsigned) * (size_t)(L.n + 2), s->stream);
            if (e == cudaSuccess) e = L.qfn(L.items, L.n, L.total, S, L.ctl, s->d_flag, s->queue_stall, s->stream);
            if (e != cudaSuccess) return e;
            s->st.launches++;
        }
        for (int j = 0; j < S; ++j) {
            for (const Launch& L : launches) {
                if (L.qfn) continue;
                long long grid = L.total < (long long)s->sms * 8 ? L.total : (long long)s->sms * 8;
                cudaError_t e = L.fn(L.items, L.n, L.total, j, (int)grid, s->stream);
                if (e != cudaSuccess) return e;
                s->st.launches++;
            }
        }
        for (size_t i = 0; i < solos.size(); ++i) {
            int cur_after = 0;
            cudaError_t e = solo_tick(solos[i], s->side[i % Server::kSide], &cur_after);
            if (e != cudaSuccess) return e;
        }
        for (int k = 0; k < nside; ++k) {
            cudaError_t e = cudaEventRecord(s->join_ev[k], s->side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->join_ev[k], 0);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    if (s->d.use_graphs) {
        auto it = s->graphs.find(key);
        if (it == s->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
            cudaError_t le = enqueue();
            e = cudaStreamEndCapture(s->stream, &g);
            if (le != cudaSuccess) return cuda_fail(le, "batched launch (capture)");
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            cudaGraphExec_t ge = nullptr;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            if (s->graph_lru.size() >= 8) {
                auto old = s->graphs.find(s->graph_lru.front());
                if (old != s->graphs.end()) {
                    cudaGraphExecDestroy(old->second);
                    s->graphs.erase(old);
                }
                s->graph_lru.pop_front();
            }
            it = s->graphs.emplace(key, ge).first;
            s->graph_lru.push_back(key);
        }
        cudaError_t e = cudaGraphLaunch(it->second, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        s->st.graph_replays++;
    } else {
        cudaError_t e = enqueue();
        if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    }
    // advance the bookkeeping of every launched request
    auto advance = [&](Req* q) {
        const long long left = q->nsteps - q->launched;
        const long long adv = left < S ? left : S;
        q->cur = (int)((q->cur + adv) % q->nlev);
        q->launched += adv;
        if (q->launched >= q->nsteps) tick.finishing.push_back(q);
    };
    for (auto& kv : s->classes)
        for (Req* q : kv.second.members) advance(q);
    for (Req* q : solos) {
        // one buffer flip per launch: blocked launches while a full block is left, then singles
        const long long left = q->nsteps - q->launched;
        const long long adv = left < S ? left : S;
        const long long flips = q->solo_tb ? adv / q->solo_depth + adv % q->solo_depth : adv;
        q->cur = (int)((q->cur + flips) % q->nlev);
        q->launched += adv;
        if (q->launched >= q->nsteps) tick.finishing.push_back(q);
    }
    cudaError_t e = cudaEventCreateWithFlags(&tick.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    e = cudaEventRecord(tick.done, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    s->inflight.push_back(tick);
    s->parity ^= 1;
    s->st.ticks++;
    s->st.lattice_updates += lu;
    return MMFD_OK;
}

// One scheduler pass.  Non-blocking unless `block` (then waits for the oldest tick when two
// are in flight).
int schedule(Server* s, bool block) {
    reap(s, false);
    // drop finished requests from the active list (their memory stays until release)
    std::vector<Req*> still;
    for (Req* q : s->active)
        if (q->state == RQ_ACTIVE) still.push_back(q);
    s->active.swap(still);
    // admission in arrival order: slots and HBM budget
    while (!s->queue.empty()) {
        Req* q = s->queue.front();
        if ((int)s->active.size() >= s->d.max_slots) break;
        if (s->st.bytes_in_use + q->footprint > s->d.hbm_budget) break;
        s->queue.pop_front();
        s->st.bytes_in_use += q->footprint;
        int rc = admit(s, q);
        if (rc != MMFD_OK) {
            for (int i = 0; i < 3; ++i) {
                srv_free(s, q->lev[i]);
                q->lev[i] = nullptr;
            }
            srv_free(s, q->d_coef);
            q->d_coef = nullptr;
            s->st.bytes_in_use -= q->footprint;
            q->state = RQ_FAILED;
            q->status = rc;
            continue;
        }
        if (q->nsteps == 0) {
            q->state = RQ_DONE;
            q->t_finish = now_s();
            s->st.finished++;
            continue;
        }
        s->active.push_back(q);
    }
    bool work = false;
    for (Req* q : s->active)
        if (q->launched < q->nsteps) work = true;
    if (!work) return MMFD_OK;
    if (s->inflight.size() >= 2) {
        if (!block) return MMFD_OK;
        reap(s, true);
    }
    return launch_tick(s);
}

}  // namespace

}  // namespace mmfd

using namespace mmfd;

extern "C" {

int mmfd_server_create(const mmfd_server_desc* desc, mmfd_server** out) {
    if (!desc || !out) return set_error(MMFD_ERR_ARG, "null argument");
    if (desc->max_slots < 1 || desc->hbm_budget == 0) return set_error(MMFD_ERR_ARG, "bad server budget");
    Server* s = new (std::nothrow) Server();
    if (!s) return set_error(MMFD_ERR_OOM, "host allocation failed");
    s->d = *desc;
    s->stream = static_cast<cudaStream_t>(desc->stream);
    if (!s->stream) {
        // graphs cannot be captured on the legacy default stream: use a private stream
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return set_error(MMFD_ERR_CUDA, "cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (const char* qv = std::getenv("MMFD_SERVE_QUEUE")) s->use_queue = std::strcmp(qv, "1") == 0;
    if (const char* qv = std::getenv("MMFD_SERVE_QUEUE_STALL")) s->queue_stall = std::strcmp(qv, "1") == 0 ? (1u << 30) : 0u;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaMemPoolCreate");
    }
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (srv_alloc(s, 256, reinterpret_cast<void**>(&s->d_flag)) != MMFD_OK ||
        cudaMemsetAsync(s->d_flag, 0, 256, s->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaMemPoolDestroy(s->pool);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return set_error(MMFD_ERR_OOM, "server flag allocation failed");
    }
    e = cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming);
    for (int k = 0; k < Server::kSide && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join_ev[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        mmfd_server_destroy(reinterpret_cast<mmfd_server*>(s));
        return cuda_fail(e, "side streams");
    }
    *out = reinterpret_cast<mmfd_server*>(s);
    return MMFD_OK;
}

int mmfd_submit(mmfd_server* h, const mmfd_desc* d, const void* const* init, int dtype, long long nsteps,
                unsigned long long* ticket) {
    Server* s = reinterpret_cast<Server*>(h);
    if (!s || !d || !init || !ticket || nsteps < 0) return set_error(MMFD_ERR_ARG, "bad argument");
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    Req* q = new (std::nothrow) Req();
    if (!q) return set_error(MMFD_ERR_OOM, "host allocation failed");
    q->r = new (std::nothrow) Resolved;
    if (!q->r) {
        delete q;
        return set_error(MMFD_ERR_OOM, "host allocation failed");
    }
    std::string msg;
    int rc = resolve(*d, *q->r, &msg);
    if (rc != MMFD_OK) {
        delete q->r;
        delete q;
        s->st.rejected++;
        return set_error(rc, msg);
    }
    if (q->r->src || q->r->theta_on || q->r->dirichlet) {
        const char* why = q->r->src ? "the server does not take requests with source terms"
                        : q->r->theta_on ? "the server does not take theta-scheme requests"
                                         : "the server takes periodic requests only";
        delete q->r;
        delete q;
        s->st.rejected++;
        return set_error(MMFD_ERR_UNSUPPORTED, why);
    }
    q->desc = *d;
    q->g = make_geom(*q->r);
    q->footprint = footprint_of(*q->r, q->g);
    if (q->footprint > s->d.hbm_budget) {
        delete q->r;
        delete q;
        s->st.rejected++;
        return set_error(MMFD_ERR_ADMISSION, "request footprint exceeds the server's HBM budget");
    }
    const long long N = (long long)q->g.nx * q->g.ny * q->g.nz;
    const size_t esz = dtype == MMFD_DT_F64 ? 8 : 4;
    q->init.resize((size_t)q->g.nf * N * esz);
    for (int f = 0; f < q->g.nf; ++f) {
        if (!init[f]) {
            delete q->r;
            delete q;
            return set_error(MMFD_ERR_ARG, "null field pointer");
        }
        std::memcpy(q->init.data() + (size_t)f * N * esz, init[f], (size_t)N * esz);
    }
    q->dtype = dtype;
    q->nsteps = nsteps;
    q->cls = class_of(*q->r);
    q->ticket = s->next_ticket++;
    q->t_submit = now_s();
    s->reqs[q->ticket] = q;
    s->queue.push_back(q);
    s->st.submitted++;
    *ticket = q->ticket;
    return MMFD_OK;
}

int mmfd_poll(mmfd_server* h, unsigned long long ticket, mmfd_result* res) {
    Server* s = reinterpret_cast<Server*>(h);
    if (!s) return set_error(MMFD_ERR_ARG, "null server");
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(MMFD_ERR_ARG, "unknown ticket");
    int rc = schedule(s, false);
    if (rc != MMFD_OK) return rc;
    Req* q = it->second;
    if (q->state == RQ_QUEUED || q->state == RQ_ACTIVE) return MMFD_PENDING;
    if (res) {
        res->status = q->status;
        res->steps_done = q->state == RQ_DONE ? q->nsteps : 0;
        res->submit_s = q->t_submit;
        res->admit_s = q->t_admit;
        res->finish_s = q->t_finish;
        res->nf = q->g.nf;
        res->n[0] = q->g.nx;
        res->n[1] = q->g.ny;
        res->n[2] = q->g.nz;
    }
    return q->state == RQ_DONE ? MMFD_OK : q->status;
}

int mmfd_server_drain(mmfd_server* h) {
    Server* s = reinterpret_cast<Server*>(h);
    if (!s) return set_error(MMFD_ERR_ARG, "null server");
    for (;;) {
        int rc = schedule(s, true);
        if (rc != MMFD_OK) return rc;
        bool pending = !s->queue.empty();
        for (Req* q : s->active)
            if (q->state == RQ_ACTIVE) pending = true;
        if (!pending && s->inflight.empty()) break;
        if (!s->inflight.empty() && (s->queue.empty() || (int)s->active.size() >= s->d.max_slots)) reap(s, true);
        if (s->queue.size() && s->active.empty() && s->inflight.empty()) {
            // nothing can run: the head request does not fit although the server is empty
            Req* q = s->queue.front();
            s->queue.pop_front();
            q->state = RQ_FAILED;
            q->status = MMFD_ERR_ADMISSION;
        }
    }
    return MMFD_OK;
}

int mmfd_result_fields(mmfd_server* h, unsigned long long ticket, void* const* out, int where, int dtype) {
    Server* s = reinterpret_cast<Server*>(h);
    if (!s || !out) return set_error(MMFD_ERR_ARG, "null argument");
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(MMFD_ERR_ARG, "unknown ticket");
    Req* q = it->second;
    if (q->state != RQ_DONE) return set_error(MMFD_ERR_STATE, "request not finished");
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    {
        int flag = 0;
        cudaError_t fe = cudaMemcpyAsync(&flag, s->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        if (fe == cudaSuccess) fe = cudaStreamSynchronize(s->stream);
        if (fe != cudaSuccess) return cuda_fail(fe, "reading the server error flag");
        if (flag != 0)
            return set_error(MMFD_ERR_TIMEOUT, flag == KERR_QUEUE_TIMEOUT
                                                   ? "the batched work queue's bounded wait for a request's previous step ran out"
                                                   : "a kernel's bounded wait for its TMA copies ran out");
    }
    const long long N = (long long)q->g.nx * q->g.ny * q->g.nz;
    const size_t esz = dtype == MMFD_DT_F64 ? 8 : 4;
    if (where == MMFD_HOST) {
        int rc = ensure_stage(s, (size_t)N * esz);
        if (rc != MMFD_OK) return rc;
    }
    for (int f = 0; f < q->g.nf; ++f) {
        void* dst = where == MMFD_HOST ? s->stage : out[f];
        cudaError_t e = launch_unpack(q->g, q->r->st, q->lev[q->cur], f, q->r->ref[f], dst, dtype, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "unpack kernel");
        if (where == MMFD_HOST) {
            e = cudaMemcpyAsync(out[f], s->stage, (size_t)N * esz, cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
            e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        }
    }
    return MMFD_OK;
}

int mmfd_release(mmfd_server* h, unsigned long long ticket) {
    Server* s = reinterpret_cast<Server*>(h);
    if (!s) return set_error(MMFD_ERR_ARG, "null server");
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(MMFD_ERR_ARG, "unknown ticket");
    Req* q = it->second;
    if (q->state == RQ_QUEUED || q->state == RQ_ACTIVE) return set_error(MMFD_ERR_STATE, "request still running");
    for (int i = 0; i < 3; ++i) srv_free(s, q->lev[i]);
    srv_free(s, q->d_coef);
    if (q->state == RQ_DONE && q->t_admit > 0) s->st.bytes_in_use -= q->footprint;
    delete q->r;
    delete q;
    s->reqs.erase(it);
    return MMFD_OK;
}

int mmfd_server_get_stats(const mmfd_server* h, mmfd_server_stats* out) {
    const Server* s = reinterpret_cast<const Server*>(h);
    if (!s || !out) return set_error(MMFD_ERR_ARG, "null argument");
    *out = s->st;
    int act = 0;
    for (Req* q : s->active)
        if (q->state == RQ_ACTIVE) ++act;
    out->active = act;
    return MMFD_OK;
}

int mmfd_server_destroy(mmfd_server* h) {
    Server* s = reinterpret_cast<Server*>(h);
    if (!s) return MMFD_OK;
    cudaStreamSynchronize(s->stream);
    for (auto& t : s->inflight) cudaEventDestroy(t.done);
    for (auto& kv : s->reqs) {
        Req* q = kv.second;
        for (int i = 0; i < 3; ++i) srv_free(s, q->lev[i]);
        srv_free(s, q->d_coef);
        delete q->r;
        delete q;
    }
    for (auto& kv : s->classes) {
        for (int p = 0; p < 2; ++p) {
            if (kv.second.h[p]) cudaFreeHost(kv.second.h[p]);
            srv_free(s, kv.second.d[p]);
        }
        srv_free(s, kv.second.ctl);
    }
    for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
    srv_free(s, s->stage);
    srv_free(s, s->d_flag);
    cudaStreamSynchronize(s->stream);
    for (int k = 0; k < Server::kSide; ++k) {
        if (s->side[k]) {
            cudaStreamSynchronize(s->side[k]);
            cudaStreamDestroy(s->side[k]);
        }
        if (s->join_ev[k]) cudaEventDestroy(s->join_ev[k]);
    }
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    cudaMemPoolDestroy(s->pool);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return MMFD_OK;
}

}  // extern "C"
