// solver.cpp -- device side of a solver: level buffers, transfers, stepping, reductions.
#include "solver.h"

#include <cstdlib>
#include <cstring>

namespace mmfd {

namespace {

long long nodes(const Solver* s) { return (long long)s->g.nx * s->g.ny * s->g.nz; }

// The dense staging buffer for host transfers: one FP64 field, or `at_least` bytes if more.
int ensure_stage(Solver* s, size_t at_least = 0) {
    size_t need = (size_t)nodes(s) * sizeof(double);
    if (at_least > need) need = at_least;
    if (s->stage && s->stage_bytes >= need) return MMFD_OK;
    if (s->stage) {
        dev_free(s, s->stage);
        s->stage = nullptr;
    }
    int rc = dev_alloc(s, need, &s->stage);
    if (rc != MMFD_OK) return rc;
    s->stage_bytes = need;
    return MMFD_OK;
}

int level_index(const Solver* s, int level, int* idx) {
    if (level == 0) {
        *idx = s->cur;
        return MMFD_OK;
    }
    if (level == 1 && s->nlev == 3) {
        *idx = s->prev();
        return MMFD_OK;
    }
    return set_error(MMFD_ERR_ARG, "level must be 0 (t_n) or, for three-level solvers, 1 (t_{n-1})");
}

}  // namespace

int solver_init_device(Solver* s) {
    s->nlev = s->r.levels == 3 ? 3 : 2;
    s->level_bytes = (size_t)s->g.fs * s->g.nf * s->g.es;
    for (int i = 0; i < s->nlev; ++i) {
        int rc = dev_alloc(s, s->level_bytes, &s->lev[i]);
        if (rc != MMFD_OK) return rc;
        cudaError_t e = cudaMemsetAsync(s->lev[i], 0, s->level_bytes, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    int rc = dev_alloc(s, (size_t)(reduce_parts_needed() + 64) * sizeof(double), reinterpret_cast<void**>(&s->d_red));
    if (rc != MMFD_OK) return rc;
    if (s->r.src) {
        // two source buffers (levels t_n, t_{n-1}, aliased while equal), zero until set
        s->src_bytes = (size_t)s->g.fs * s->r.nsrc * (s->r.st == ST_F64 ? 8 : 4);
        for (int i = 0; i < 2; ++i) {
            rc = dev_alloc(s, s->src_bytes, &s->srcbuf[i]);
            if (rc != MMFD_OK) return rc;
            cudaError_t e = cudaMemsetAsync(s->srcbuf[i], 0, s->src_bytes, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        }
        s->src_i0 = s->src_i1 = 0;
        s->src_fresh = true;
    }
    if (s->r.dirichlet) {
        // boundary values, in the level layout and storage
        rc = dev_alloc(s, s->level_bytes, &s->bnd);
        if (rc != MMFD_OK) return rc;
        cudaError_t e = cudaMemsetAsync(s->bnd, 0, s->level_bytes, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    if (s->r.theta_on) {
        // same element size and ghosted layout as a level (FP64 / FP32 storage only)
        rc = dev_alloc(s, s->level_bytes, &s->rhs);
        if (rc != MMFD_OK) return rc;
        cudaError_t e = cudaMemsetAsync(s->rhs, 0, s->level_bytes, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    rc = dev_alloc(s, 256, reinterpret_cast<void**>(&s->d_flag));
    if (rc != MMFD_OK) return rc;
    cudaError_t e = cudaMemsetAsync(s->d_flag, 0, 256, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    s->cur = 0;
    return solver_pick_kernels(s);
}

void solver_free_device(Solver* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (int i = 0; i < 3; ++i) {
        dev_free(s, s->lev[i]);
        s->lev[i] = nullptr;
    }
    dev_free(s, s->stage);
    s->stage = nullptr;
    for (int i = 0; i < 2; ++i) {
        dev_free(s, s->srcbuf[i]);
        s->srcbuf[i] = nullptr;
    }
    dev_free(s, s->rhs);
    s->rhs = nullptr;
    dev_free(s, s->bnd);
    s->bnd = nullptr;
    dev_free(s, s->d_red);
    s->d_red = nullptr;
    dev_free(s, s->d_flag);
    s->d_flag = nullptr;
}

int solver_check_flag(Solver* s) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error flag");
    if (h != 0) {
        cudaMemsetAsync(s->d_flag, 0, sizeof(int), s->stream);
        return set_error(MMFD_ERR_TIMEOUT, "a kernel's bounded wait for its TMA copies ran out");
    }
    return MMFD_OK;
}

int solver_set_fields(Solver* s, int level, const void* const* fields, int where, int dtype) {
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (where != MMFD_HOST && where != MMFD_DEVICE) return set_error(MMFD_ERR_ARG, "where must be HOST or DEVICE");
    int idx;
    int rc = level_index(s, level, &idx);
    if (rc != MMFD_OK) return rc;
    const size_t esz = dtype == MMFD_DT_F64 ? 8 : 4;
    const size_t bytes = (size_t)nodes(s) * esz;
    if (where == MMFD_HOST && (rc = ensure_stage(s)) != MMFD_OK) return rc;
    for (int f = 0; f < s->g.nf; ++f) {
        if (!fields[f]) return set_error(MMFD_ERR_ARG, "null field pointer");
        const void* src = fields[f];
        if (where == MMFD_HOST) {
            // page-locked host memory is read by the pack kernel itself, over the host link (one
            // pass instead of a copy into the staging buffer plus a second pass over it)
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, src) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                pa.devicePointer) {
                src = pa.devicePointer;
            } else {
                cudaGetLastError();
                cudaError_t e = cudaMemcpyAsync(s->stage, src, bytes, cudaMemcpyHostToDevice, s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
                src = s->stage;
            }
        }
        cudaError_t e = launch_pack(s->g, s->r.st, src, dtype, s->lev[idx], f, s->r.ref[f], s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
        if (s->nlev == 3 && level == 0) {
            // equilibrium start: level t - dt := level t until set explicitly
            e = launch_pack(s->g, s->r.st, src, dtype, s->lev[s->prev()], f, s->r.ref[f], s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
        }
        if (s->r.dirichlet && level == 0) {
            // Dirichlet: the boundary keeps these values until mmfd_set_boundary replaces them
            e = launch_pack(s->g, s->r.st, src, dtype, s->bnd, f, s->r.ref[f], s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
        }
    }
    s->fields_set = true;
    if (level == 0) s->src_fresh = true;
    return MMFD_OK;
}

int solver_set_source(Solver* s, int level, const void* const* fields, int where, int dtype) {
    if (!s->r.src) return set_error(MMFD_ERR_STATE, "the solver was created without a source");
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (where != MMFD_HOST && where != MMFD_DEVICE) return set_error(MMFD_ERR_ARG, "where must be HOST or DEVICE");
    if (level != 0 && !(level == 1 && s->nlev == 3))
        return set_error(MMFD_ERR_ARG, "level must be 0 (t_n) or, for three-level solvers, 1 (t_{n-1})");
    // Level 0 while the two levels share a buffer: write the other buffer, so that level 1 keeps
    // its values -- except before the first step, where level 1 follows level 0 (the sources'
    // counterpart of the equilibrium start).  Level 1 while shared: split off the other buffer.
    int idx;
    if (level == 0) {
        if (s->src_i0 == s->src_i1 && !s->src_fresh) s->src_i0 = 1 - s->src_i1;
        idx = s->src_i0;
    } else {
        if (s->src_i0 == s->src_i1) s->src_i1 = 1 - s->src_i0;
        idx = s->src_i1;
    }
    Geom gs = s->g;
    gs.es = s->r.st == ST_F64 ? 8 : 4;
    const int sst = s->r.st == ST_F64 ? ST_F64 : ST_F32;
    const size_t esz = dtype == MMFD_DT_F64 ? 8 : 4;
    const size_t bytes = (size_t)nodes(s) * esz;
    int rc;
    if (where == MMFD_HOST && (rc = ensure_stage(s)) != MMFD_OK) return rc;
    for (int f = 0; f < s->r.nsrc; ++f) {
        if (!fields[f]) return set_error(MMFD_ERR_ARG, "null field pointer");
        const void* src = fields[f];
        if (where == MMFD_HOST) {
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, src) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                pa.devicePointer) {
                src = pa.devicePointer;
            } else {
                cudaGetLastError();
                cudaError_t e = cudaMemcpyAsync(s->stage, src, bytes, cudaMemcpyHostToDevice, s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
                src = s->stage;
            }
        }
        cudaError_t e = launch_pack(gs, sst, src, dtype, s->srcbuf[idx], f, 0.0, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
    }
    return MMFD_OK;
}

int solver_set_boundary(Solver* s, const void* const* fields, int where, int dtype) {
    if (!s->r.dirichlet) return set_error(MMFD_ERR_STATE, "the solver has periodic boundaries");
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (where != MMFD_HOST && where != MMFD_DEVICE) return set_error(MMFD_ERR_ARG, "where must be HOST or DEVICE");
    const size_t bytes = (size_t)nodes(s) * (dtype == MMFD_DT_F64 ? 8 : 4);
    int rc;
    if (where == MMFD_HOST && (rc = ensure_stage(s)) != MMFD_OK) return rc;
    for (int f = 0; f < s->g.nf; ++f) {
        if (!fields[f]) return set_error(MMFD_ERR_ARG, "null field pointer");
        const void* src = fields[f];
        if (where == MMFD_HOST) {
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, src) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                pa.devicePointer) {
                src = pa.devicePointer;
            } else {
                cudaGetLastError();
                cudaError_t e = cudaMemcpyAsync(s->stage, src, bytes, cudaMemcpyHostToDevice, s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
                src = s->stage;
            }
        }
        cudaError_t e = launch_pack(s->g, s->r.st, src, dtype, s->bnd, f, s->r.ref[f], s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "pack kernel");
    }
    return MMFD_OK;
}

void solver_launch_args(Solver* s, LaunchArgs& a) {
    a.g = s->g;
    a.in0 = s->lev[s->cur];
    a.in1 = s->nlev == 3 ? s->lev[s->prev()] : nullptr;
    a.out = s->lev[s->next()];
    a.coef = s->coef();
    a.ex.seed = s->desc.seed;
    a.ex.step = s->steps_done + 1;
    a.ex.sr = (s->r.st == ST_BF16 && (s->desc.flags & MMFD_FLAG_STOCHASTIC_ROUND)) ? 1 : 0;
    a.stream = s->stream;
    a.variant = s->variant;
    a.H = s->H;
    a.err = s->d_flag;
    a.maps = nullptr;
    a.src[0] = s->r.src ? s->srcbuf[s->src_i0] : nullptr;
    a.src[1] = s->r.src ? s->srcbuf[s->src_i1] : nullptr;
    a.src_coef = s->r.st == ST_F64 ? static_cast<const void*>(&s->r.sd) : static_cast<const void*>(&s->r.sf);
    if (s->r.theta_on) {
        // theta-scheme: the step kernel fn is the Jacobi sweep (rhs enters as a centre-only source)
        const bool f64 = s->r.st == ST_F64;
        a.coef = f64 ? static_cast<const void*>(&s->r.thj_d) : static_cast<const void*>(&s->r.thj_f);
        a.src[0] = a.src[1] = s->rhs;
        a.src_coef = f64 ? static_cast<const void*>(&s->r.ths_d) : static_cast<const void*>(&s->r.ths_f);
    }
    if (s->use_tma) {
        const int nf = s->g.nf;
        for (int f = 0; f < nf; ++f) {
            s->launch_maps.m[f] = s->tmaps[s->cur][f];
            if (s->nlev == 3) s->launch_maps.m[nf + f] = s->tmaps[s->prev()][f];
        }
        a.maps = &s->launch_maps;
    }
}

int solver_step(Solver* s, long long nsteps) {
    if (!s->fields_set) return set_error(MMFD_ERR_STATE, "set the fields before stepping");
    if (s->r.theta_on) {
        // Eq. (GCN): rhs = ((1 - theta) I + theta E) phi^n, then r.sweeps Jacobi sweeps from
        // x = phi^n, each into the spare level buffer
        const bool f64 = s->r.st == ST_F64;
        for (long long n = 0; n < nsteps; ++n) {
            LaunchArgs a;
            solver_launch_args(s, a);
            a.out = s->rhs;
            a.coef = f64 ? static_cast<const void*>(&s->r.thr_d) : static_cast<const void*>(&s->r.thr_f);
            a.src[0] = a.src[1] = nullptr;
            cudaError_t e = s->fn_rhs(a);
            if (e != cudaSuccess) return cuda_fail(e, "theta-scheme right-hand side kernel");
            // sweeps fused `depth` per launch by the blocked kernel (a shallower blocked launch,
            // with the launcher's own work-item height, or a single sweep for the remainder)
            int left = s->r.sweeps;
            while (left > 0) {
                solver_launch_args(s, a);
                LaunchFn f = s->fn;
                int did = 1;
                if (s->fn_block && s->depth > 1 && left >= 2) {
                    did = left >= s->depth ? s->depth : left;
                    f = did == s->depth ? s->fn_block : find_march2d_tb_jacobi(s->r.lat, s->r.st, did);
                    if (did != s->depth) a.H = 0;
                    if (!f) {
                        f = s->fn;
                        did = 1;
                        a.H = s->H;
                    }
                }
                e = f(a);
                if (e != cudaSuccess) return cuda_fail(e, "theta-scheme sweep kernel");
                s->cur = s->next();
                left -= did;
            }
            s->steps_done += 1;
        }
        return MMFD_OK;
    }
    long long done = 0;
    while (done < nsteps) {
        const long long left = nsteps - done;
        const bool blocked = s->fn_block && s->depth > 1 && left >= s->depth;
        LaunchArgs a;
        solver_launch_args(s, a);
        if (blocked) {
            // the blocked kernel (two-level solvers) writes level t + depth dt into next()
            a.ex.step = s->steps_done + s->depth;
            cudaError_t e = s->fn_block(a);
            if (e != cudaSuccess) return cuda_fail(e, "blocked step kernel");
            s->cur = s->next();
            s->steps_done += s->depth;
            done += s->depth;
        } else {
            cudaError_t e = s->fn(a);
            if (e != cudaSuccess) return cuda_fail(e, "step kernel");
            s->cur = s->next();
            if (s->r.dirichlet) {
                // the new level's boundary nodes take the prescribed values
                e = launch_ring_copy(s->g, s->bnd, s->lev[s->cur], s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "boundary kernel");
            }
            s->steps_done += 1;
            done += 1;
            if (s->r.src) {
                // the source at t_n becomes the one at t_{n-1}; level 0 keeps it until replaced
                s->src_i1 = s->src_i0;
                s->src_fresh = false;
            }
        }
    }
    return MMFD_OK;
}

int solver_get_fields(Solver* s, int level, void* const* out, int where, int dtype) {
    int frc = solver_check_flag(s);
    if (frc != MMFD_OK) return frc;
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (where != MMFD_HOST && where != MMFD_DEVICE) return set_error(MMFD_ERR_ARG, "where must be HOST or DEVICE");
    int idx;
    int rc = level_index(s, level, &idx);
    if (rc != MMFD_OK) return rc;
    const size_t esz = dtype == MMFD_DT_F64 ? 8 : 4;
    const size_t bytes = (size_t)nodes(s) * esz;
    if (where == MMFD_HOST && (rc = ensure_stage(s)) != MMFD_OK) return rc;
    for (int f = 0; f < s->g.nf; ++f) {
        if (!out[f]) return set_error(MMFD_ERR_ARG, "null field pointer");
        void* dst = where == MMFD_HOST ? s->stage : out[f];
        cudaError_t e = launch_unpack(s->g, s->r.st, s->lev[idx], f, s->r.ref[f], dst, dtype, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "unpack kernel");
        if (where == MMFD_HOST) {
            e = cudaMemcpyAsync(out[f], s->stage, bytes, cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
            e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        }
    }
    return MMFD_OK;
}

// Rows [r0, r0 + count) of the slab axis (y in 2D, z in 3D) <-> dense buffers: flat row range
// [r0, r0 + count) * (1 or ny) of the pack / unpack kernels.
static int rows_range(const Solver* s, long long r0, long long count, long long* lo, long long* hi) {
    const long long n = s->g.dim == 3 ? s->g.nz : s->g.ny;
    if (r0 < 0 || count < 1 || r0 + count > n) return set_error(MMFD_ERR_ARG, "row range outside the grid");
    const long long per = s->g.dim == 3 ? s->g.ny : 1;
    *lo = r0 * per;
    *hi = (r0 + count) * per;
    return MMFD_OK;
}

int solver_set_rows(Solver* s, int level, long long r0, long long count, const void* const* fields, int where,
                    int dtype) {
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (where != MMFD_HOST && where != MMFD_DEVICE) return set_error(MMFD_ERR_ARG, "where must be HOST or DEVICE");
    int idx;
    int rc = level_index(s, level, &idx);
    if (rc != MMFD_OK) return rc;
    long long lo, hi;
    if ((rc = rows_range(s, r0, count, &lo, &hi)) != MMFD_OK) return rc;
    for (int f = 0; f < s->g.nf; ++f)
        if (!fields[f]) return set_error(MMFD_ERR_ARG, "null field pointer");
    const size_t bytes = (size_t)(hi - lo) * s->g.nx * (dtype == MMFD_DT_F64 ? 8 : 4);
    const void* src[4] = {fields[0], nullptr, nullptr, nullptr};
    for (int f = 1; f < s->g.nf; ++f) src[f] = fields[f];
    if (where == MMFD_HOST) {
        // staged field after field in the staging buffer
        if ((rc = ensure_stage(s, bytes * s->g.nf)) != MMFD_OK) return rc;
        for (int f = 0; f < s->g.nf; ++f) {
            char* dst = static_cast<char*>(s->stage) + f * bytes;
            cudaError_t e = cudaMemcpyAsync(dst, fields[f], bytes, cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
            src[f] = dst;
        }
    }
    cudaError_t e = launch_rows(s->g, s->r.st, true, src, s->g.nf, dtype, s->lev[idx], s->r.ref, lo, hi, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "row pack kernel");
    if (where == MMFD_HOST) {
        e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return MMFD_OK;
}

int solver_get_rows(Solver* s, int level, long long r0, long long count, void* const* out, int where, int dtype) {
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (where != MMFD_HOST && where != MMFD_DEVICE) return set_error(MMFD_ERR_ARG, "where must be HOST or DEVICE");
    int idx;
    int rc = level_index(s, level, &idx);
    if (rc != MMFD_OK) return rc;
    long long lo, hi;
    if ((rc = rows_range(s, r0, count, &lo, &hi)) != MMFD_OK) return rc;
    for (int f = 0; f < s->g.nf; ++f)
        if (!out[f]) return set_error(MMFD_ERR_ARG, "null field pointer");
    const size_t bytes = (size_t)(hi - lo) * s->g.nx * (dtype == MMFD_DT_F64 ? 8 : 4);
    const void* dst[4] = {out[0], nullptr, nullptr, nullptr};
    for (int f = 1; f < s->g.nf; ++f) dst[f] = out[f];
    if (where == MMFD_HOST) {
        if ((rc = ensure_stage(s, bytes * s->g.nf)) != MMFD_OK) return rc;
        for (int f = 0; f < s->g.nf; ++f) dst[f] = static_cast<char*>(s->stage) + f * bytes;
    }
    cudaError_t e = launch_rows(s->g, s->r.st, false, dst, s->g.nf, dtype, s->lev[idx], s->r.ref, lo, hi, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "row unpack kernel");
    if (where == MMFD_HOST) {
        for (int f = 0; f < s->g.nf; ++f) {
            e = cudaMemcpyAsync(out[f], dst[f], bytes, cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
        }
        e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return MMFD_OK;
}

int solver_reduce(Solver* s, int what, double* out) {
    if (what < MMFD_RED_SUM || what > MMFD_RED_NONFINITE) return set_error(MMFD_ERR_ARG, "unknown reduction");
    int frc = solver_check_flag(s);
    if (frc != MMFD_OK) return frc;
    const int nf = s->g.nf;
    double* d_out = s->d_red + reduce_parts_needed();
    double host[4 * 4];
    for (int f = 0; f < nf; ++f) {
        cudaError_t e = launch_reduce(s->g, s->r.st, s->lev[s->cur], f, s->r.ref[f], what, nullptr, 0, s->d_red,
                                      reduce_parts_needed(), d_out + 4 * f, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "reduce kernel");
    }
    cudaError_t e = cudaMemcpyAsync(host, d_out, sizeof(double) * 4 * nf, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (what == MMFD_RED_NONFINITE) {
        double t = 0;
        for (int f = 0; f < nf; ++f) t += host[4 * f];
        out[0] = t;
    } else {
        for (int f = 0; f < nf; ++f) out[f] = host[4 * f];
    }
    return MMFD_OK;
}

int solver_error_norms(Solver* s, int field, const void* ref, int where, int dtype, double* out) {
    if (field < 0 || field >= s->g.nf) return set_error(MMFD_ERR_ARG, "bad field index");
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    const void* dref = ref;
    if (where == MMFD_HOST) {
        int rc = ensure_stage(s);
        if (rc != MMFD_OK) return rc;
        const size_t bytes = (size_t)nodes(s) * (dtype == MMFD_DT_F64 ? 8 : 4);
        cudaError_t e = cudaMemcpyAsync(s->stage, ref, bytes, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
        dref = s->stage;
    }
    double* d_out = s->d_red + reduce_parts_needed();
    cudaError_t e = launch_reduce(s->g, s->r.st, s->lev[s->cur], field, s->r.ref[field], 3, dref, dtype, s->d_red,
                                  reduce_parts_needed(), d_out, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce kernel");
    double host[4];
    e = cudaMemcpyAsync(host, d_out, sizeof(host), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    out[0] = host[1] > 0 ? host[0] / host[1] : host[0];
    out[1] = host[2];
    out[2] = host[3];
    return MMFD_OK;
}

// Name of a marching kernel family with its lean He-Luo variant: "_nse_s" (streaming momentum),
// "_nse_g" (general momentum), none for the general pair form.
static const char* lean_name(const Solver* s, const char* family) {
    static const char* const names[2][3] = {{"k_march2d", "k_march2d_nse_s", "k_march2d_nse_g"},
                                            {"k_march3d", "k_march3d_nse_s", "k_march3d_nse_g"}};
    const int d = std::strcmp(family, "k_march2d") == 0 ? 0 : 1;
    return names[d][s->lean];
}

// The 2D temporally blocked step kernel of this solver at `depth` levels per launch: the scalar
// blocked kernel (two-level LCDE / NCDE), or the blocked lean NSE kernel (D2Q9 He-Luo NSE with a
// streaming momentum set, two levels); null where neither applies.
static LaunchFn blocked_kernel(const Solver* s, int depth) {
    if (s->r.dim != 2 || depth < 2) return nullptr;
    if (s->r.pde == PDE_NSE)
        return s->lean == LEAN_STREAM && s->r.levels == 2 ? find_march2d_tb_nse(s->r.st, depth) : nullptr;
    return find_march2d_tb(s->r.lat, s->r.pde, s->r.levels, s->r.st, depth);
}

void solver_use_depth(Solver* s, int depth) {
    LaunchFn fb = nullptr;
    if (depth >= 2 && s->r.theta_on)
        fb = s->r.dim == 2 ? find_march2d_tb_jacobi(s->r.lat, s->r.st, depth) : nullptr;
    else if (depth >= 2)
        fb = blocked_kernel(s, depth);
    if (fb) {
        s->fn_block = fb;
        s->depth = depth;
        s->kernel_name = s->r.pde == PDE_NSE && !s->r.theta_on ? "k_march2d_tb_nse" : "k_march2d_tb";
    } else {
        s->fn_block = nullptr;
        s->depth = 1;
        if (s->r.src || s->r.theta_on)
            s->kernel_name = s->use_tma ? (s->r.dim == 2 ? "k_march2d_src" : "k_march3d_src") : "k_direct_src";
        else s->kernel_name = s->use_tma ? lean_name(s, s->r.dim == 2 ? "k_march2d" : "k_march3d") : "k_direct";
    }
}

int solver_pick_kernels(Solver* s) {
    s->fn_block = nullptr;
    s->depth = 1;
    s->max_depth = 1;
    s->variant = 0;
    s->use_tma = false;
    s->fn = nullptr;
    const char* force = std::getenv("MMFD_FORCE_KERNEL");
    const bool want_direct = force && std::strcmp(force, "direct") == 0;
    // source terms: kernel variant 1 (S only, M_1F = 0 or S u folded) or 2 (S and M_1F fields);
    // such solvers run unblocked.  The theta-scheme's Jacobi sweep is variant 1 (its right-hand
    // side enters as a centre-only source) and its right-hand side a plain step.
    const int srcv = s->r.theta_on ? 1 : s->r.src == 0 ? 0 : (s->r.src == MMFD_SRC_SM ? 2 : 1);
    s->fn_rhs = nullptr;
    // the lean He-Luo NSE form where the coefficients allow it (MMFD_FORCE_KERNEL=generic keeps the
    // general pair form, for comparisons; it computes the same update)
    const bool want_generic = force && std::strcmp(force, "generic") == 0;
    const int lean = (!want_generic && !srcv && !s->r.theta_on) ? s->r.lean : LEAN_NONE;
    // 3D lean solvers of large grids run 16-row tiles at one CTA per SM (march3d_lean_tile_rows;
    // MMFD_FORCE_KERNEL=lean3d_rows16 / lean3d_rows4 picks the tile whatever the grid, for
    // comparisons: both compute every node with the same arithmetic in the same order)
    const int force_rows = !force ? 0 : std::strcmp(force, "lean3d_rows16") == 0 ? 1 : std::strcmp(force, "lean3d_rows4") == 0 ? -1 : 0;
    const int lean_rows = s->r.dim == 3 ? march3d_lean_tile_rows(s->g.nx, s->g.ny, s->g.nz, force_rows) : 0;
    LaunchFn fn_lean =
        lean != LEAN_NONE ? find_march_lean(s->r.lat, s->r.levels, s->r.st, lean, s->r.dim == 3 ? lean_rows : 4) : nullptr;
    s->lean = fn_lean ? lean : LEAN_NONE;
    if (s->r.dim == 2 && s->g.nx >= 128 && !want_direct) {
        s->fn = fn_lean ? fn_lean
                : srcv  ? find_march2d_src(s->r.lat, s->r.pde, s->r.levels, s->r.st, srcv)
                        : find_march2d(s->r.lat, s->r.pde, s->r.levels, s->r.st);
        if (s->r.theta_on) {
            s->fn_rhs = find_march2d(s->r.lat, s->r.pde, s->r.levels, s->r.st);
            if (!s->fn_rhs) s->fn = nullptr;
        }
        if (s->fn) {
            const int es = s->g.es;
            const int boxw = 128 + 2 * (16 / es);
            for (int b = 0; b < s->nlev; ++b)
                for (int f = 0; f < s->g.nf; ++f) {
                    char* base = static_cast<char*>(s->lev[b]) + (size_t)f * s->g.fs * es;
                    if (encode_field_map(&s->tmaps[b][f], base, s->r.st, s->g, boxw,
                                         march2d_rows_per_stage(s->r.pde), 1) != 0) {
                        s->fn = nullptr;
                        break;
                    }
                }
        }
        if (s->fn) {
            s->use_tma = true;
            s->kernel_name = srcv ? "k_march2d_src" : lean_name(s, "k_march2d");
            s->H = 0;  // chosen by the launcher from the kernel's occupancy
            // temporal blocking: 0 asks for the deepest blocking the storage allows (the
            // autotuner may then pick a shallower one); the x ghost columns, kept current to
            // their full depth ox by every writer, bound the depth.
            // (The blocked kernel stages two rows per box, as the solver's maps for these PDEs do.)
            int maxd = march2d_tb_max_depth(s->r.st);
            if (s->r.pde == PDE_NSE && maxd > march2d_tb_nse_max_depth()) maxd = march2d_tb_nse_max_depth();
            while (maxd >= 2 && s->g.ny < 2 * maxd) --maxd;
            if (s->r.theta_on && s->desc.temporal_depth != 1 && maxd >= 2 &&
                find_march2d_tb_jacobi(s->r.lat, s->r.st, 2)) {
                // theta-scheme: Jacobi sweeps fused per launch
                s->max_depth = maxd;
                int want = s->desc.temporal_depth == 0 ? maxd : s->desc.temporal_depth;
                if (want > maxd) want = maxd;
                solver_use_depth(s, want);
            }
            if (!srcv && !s->r.dirichlet && s->desc.temporal_depth != 1 && maxd >= 2 && march2d_rows_per_stage(s->r.pde) == 2 &&
                blocked_kernel(s, 2)) {
                s->max_depth = maxd;
                int want = s->desc.temporal_depth == 0 ? maxd : s->desc.temporal_depth;
                if (want > maxd) want = maxd;
                solver_use_depth(s, want);
            }
            return MMFD_OK;
        }
    }
    if (s->r.dim == 3 && s->g.nx >= 128 && !want_direct) {
        s->fn = fn_lean ? fn_lean
                : srcv  ? find_march3d_src(s->r.lat, s->r.pde, s->r.levels, s->r.st, srcv)
                        : find_march3d(s->r.lat, s->r.pde, s->r.levels, s->r.st);
        if (s->r.theta_on) {
            s->fn_rhs = find_march3d(s->r.lat, s->r.pde, s->r.levels, s->r.st);
            if (!s->fn_rhs) s->fn = nullptr;
        }
        if (s->fn) {
            const int es = s->g.es;
            const int boxw = 128 + 2 * (16 / es);
            s->tile_rows = fn_lean ? lean_rows : march3d_tile_rows(s->r.pde);
            const int rows = s->tile_rows + 2;
            // the 16-row BF16 kernel streams balanced per-group ranges (k_march3d.cuh): neighbouring
            // y tiles sit at unrelated planes, so L2 promotion would fetch bytes no neighbour reads
            // in time
            const bool promote = !(fn_lean && s->tile_rows > march3d_tile_rows(s->r.pde) && s->r.st == ST_BF16);
            for (int b = 0; b < s->nlev && s->fn; ++b)
                for (int f = 0; f < s->g.nf; ++f) {
                    char* base = static_cast<char*>(s->lev[b]) + (size_t)f * s->g.fs * es;
                    if (encode_field_map(&s->tmaps[b][f], base, s->r.st, s->g, boxw, rows, 1, promote) != 0) {
                        s->fn = nullptr;
                        break;
                    }
                }
        }
        if (s->fn) {
            s->use_tma = true;
            s->kernel_name = srcv ? "k_march3d_src" : lean_name(s, "k_march3d");
            s->H = 0;
            // 3D solvers run unblocked: a temporally blocked 3D LCDE kernel (shared-memory level
            // planes, T = 2..5) was slower than this one at every depth and has been removed
            return MMFD_OK;
        }
    }
    s->lean = LEAN_NONE;
    s->fn = srcv ? find_direct_src(s->r.lat, s->r.pde, s->r.levels, s->r.st, srcv)
                 : find_direct(s->r.lat, s->r.pde, s->r.levels, s->r.st);
    s->kernel_name = srcv ? "k_direct_src" : "k_direct";
    if (s->r.theta_on) s->fn_rhs = find_direct(s->r.lat, s->r.pde, s->r.levels, s->r.st);
    if (!s->fn || (s->r.theta_on && !s->fn_rhs))
        return set_error(MMFD_ERR_UNSUPPORTED, "no kernel for this lattice/PDE/levels/storage");
    return MMFD_OK;
}

}  // namespace mmfd
