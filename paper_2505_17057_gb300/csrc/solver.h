// solver.h -- the solver object behind mmfd_solver.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/mmfd.h"
#include "kernels.h"
#include "params.h"

namespace mmfd {

struct Solver {
    mmfd_desc desc{};
    Resolved r{};
    Geom g{};
    cudaStream_t stream = nullptr;
    mmfd_alloc_fn alloc = nullptr;
    mmfd_free_fn free_fn = nullptr;
    void* alloc_ctx = nullptr;
    void* lev[3] = {nullptr, nullptr, nullptr};  // level buffers (nf fields each, ghosted)
    int nlev = 0;                                // 2 (two-level) or 3 (three-level ring)
    int cur = 0;                                 // buffer holding level t_n
    size_t level_bytes = 0;
    void* stage = nullptr;                       // dense staging buffer for host transfers
    size_t stage_bytes = 0;
    double* d_red = nullptr;                     // reduction partials and results
    long long steps_done = 0;
    int depth = 1;                               // steps fused per launch
    int max_depth = 1;                           // deepest blocking this solver's ghosts allow
    LaunchFn fn = nullptr;                       // single-step kernel
    LaunchFn fn_block = nullptr;                 // temporally blocked kernel (depth > 1)
    int variant = 0;
    const char* kernel_name = "k_direct";
    int tile_rows = 0;  // 3D marching kernels: rows of the CTA tile (mmfd_info_t::tile_rows)
    int* d_flag = nullptr;                       // device error flag written by kernels
    bool fields_set = false;
    bool use_tma = false;                        // kernel family consumes tensor maps
    int lean = 0;                                // LEAN_* variant of the marching kernel in use
    CUtensorMap tmaps[3][4];                     // per level buffer, per field
    TmapSet launch_maps;                         // assembled per launch (inputs of this step)
    int H = 0;                                   // rows / planes per CTA
    void* srcbuf[2] = {nullptr, nullptr};        // source levels (compute type, ghosted layout)
    size_t src_bytes = 0;
    int src_i0 = 0, src_i1 = 0;                  // buffers holding the sources at t_n and t_{n-1}
    bool src_fresh = true;                       // no step since creation or set_fields(level 0)
    void* bnd = nullptr;                         // Dirichlet: boundary values (a level in the level layout)
    void* rhs = nullptr;                         // theta-scheme: right-hand side (I + theta L) phi^n
    LaunchFn fn_rhs = nullptr;                   // theta-scheme: kernel writing rhs (plain LCDE step)

    int prev() const { return nlev == 2 ? 1 - cur : (cur + 2) % 3; }
    int next() const { return nlev == 2 ? 1 - cur : (cur + 1) % 3; }
    const void* coef() const { return r.st == ST_F64 ? static_cast<const void*>(&r.cd) : static_cast<const void*>(&r.cf); }
};

int set_error(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
Geom make_geom(const Resolved& r);
int dev_alloc(Solver* s, size_t bytes, void** p);
void dev_free(Solver* s, void* p);

int solver_init_device(Solver* s);
void solver_free_device(Solver* s);
int solver_set_fields(Solver* s, int level, const void* const* fields, int where, int dtype);
int solver_set_source(Solver* s, int level, const void* const* fields, int where, int dtype);
int solver_set_boundary(Solver* s, const void* const* fields, int where, int dtype);
int solver_step(Solver* s, long long nsteps);
int solver_get_fields(Solver* s, int level, void* const* out, int where, int dtype);
int solver_set_rows(Solver* s, int level, long long r0, long long count, const void* const* fields, int where,
                    int dtype);
int solver_get_rows(Solver* s, int level, long long r0, long long count, void* const* out, int where, int dtype);
int solver_reduce(Solver* s, int what, double* out);
int solver_error_norms(Solver* s, int field, const void* ref, int where, int dtype, double* out);
// Pick the kernel family / variant for this solver (autotuner cache or heuristics).
int solver_pick_kernels(Solver* s);
// Read (and clear) the device error flag; MMFD_ERR_TIMEOUT if a kernel gave up a wait.
int solver_check_flag(Solver* s);
// Launch arguments of the next step: inputs the current level(s), output the spare buffer.
void solver_launch_args(Solver* s, LaunchArgs& a);
// Switch to temporal depth `depth` (1 = unblocked; must not exceed max_depth).
void solver_use_depth(Solver* s, int depth);
// Time the candidate configurations and keep the fastest (mmfd_autotune).
int solver_autotune(Solver* s, const char* cache_path, mmfd_tune_info* out);

}  // namespace mmfd
