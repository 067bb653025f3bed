// kernels.h -- host-side entry points of the kernel families (type-erased launchers).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "mmfd_internal.h"

namespace mmfd {

// Up to 8 TMA tensor maps (nf fields x input levels), passed to a kernel as a grid constant.
struct TmapSet {
    CUtensorMap m[8];
};

// A launcher advances one (or `depth`) time level(s): reads level t (in0) and level t - dt
// (in1, three-level only) and writes level t + dt (out), all in the ghosted layout `g`.
// coef points at a Coef<double> or Coef<float> matching the storage type.
struct LaunchArgs {
    Geom g;
    const void* in0;
    const void* in1;
    void* out;
    const void* coef;
    StepExtra ex;
    cudaStream_t stream;
    int variant;          // kernel-shape variant chosen by the tuner (family specific)
    const TmapSet* maps;  // TMA descriptors of the input levels (march / blocked kernels)
    int H;                // rows (2D) or planes (3D) per CTA
    int* err;             // device error flag (bounded waits that ran out)
    const void* src[2];   // source levels t, t - dt (solvers with source terms; else null)
    const void* src_coef; // SrcCoef<double> or SrcCoef<float> matching the storage type
};
using LaunchFn = cudaError_t (*)(const LaunchArgs&);

// One node per thread, neighbours read straight from the ghosted layout (any shape).
LaunchFn find_direct(int lat, int pde, int levels, int st);
// The same with source terms: src 1 (a source S, M_1F = 0 or S u folded) or 2 (S and M_1F fields).
LaunchFn find_direct_src(int lat, int pde, int levels, int st, int src);
// Row-marching 2D kernels fed by a TMA (cp.async.bulk.tensor) shared-memory ring.
LaunchFn find_march2d(int lat, int pde, int levels, int st);
// The same with source terms in the store epilogue (src as for find_direct_src; LCDE / NCDE).
LaunchFn find_march2d_src(int lat, int pde, int levels, int st, int src);
// Input rows per TMA box (stage) of the 2D marching kernel for this PDE; its tensor maps use
// boxes of 128 + 2 x 16 bytes by this many rows.
int march2d_rows_per_stage(int pde);
// 3D plane-marching kernels (z march, x-y tile staged in shared memory by TMA).
LaunchFn find_march3d(int lat, int pde, int levels, int st);
// Temporally blocked 2D kernel advancing `depth` levels per launch (two-level LCDE / NCDE;
// nullptr where unsupported) and the largest depth its ghost columns allow for storage st.
// It reads the level through the same 2-row-box tensor maps as k_march2d.
LaunchFn find_march2d_tb(int lat, int pde, int levels, int st, int depth);
int march2d_tb_max_depth(int st);
// The temporally blocked D2Q9 He-Luo NSE step in the lean streaming form (two levels, FP32 /
// BF16 storage; depth 2 .. march2d_tb_nse_max_depth()).
LaunchFn find_march2d_tb_nse(int st, int depth);
int march2d_tb_nse_max_depth();
// The same kernel advancing `depth` Jacobi sweeps of the two-level LCDE theta-scheme per launch
// (FP32 / FP64 levels): the coefficient block is the sweep's stencil, src[0] the right-hand
// side and src_coef's W0[0] its weight.
LaunchFn find_march2d_tb_jacobi(int lat, int st, int depth);
// The same with source terms in the store epilogue (src as for find_direct_src; LCDE / NCDE).
LaunchFn find_march3d_src(int lat, int pde, int levels, int st, int src);
// Rows of the x-y tile a 3D march CTA stages per plane (the TMA box is 128+halo x rows+2 x 1).
int march3d_tile_rows(int pde);
// The 2D (D2Q9) and 3D (D3Q19) marching kernels in the lean He-Luo NSE form (lean = LEAN_STREAM
// or LEAN_GENERAL, see Coef::nA; FP32 / BF16 storage, two or three levels; nullptr elsewhere).
// They take the same tensor maps and launch arguments as find_march2d / find_march3d, except that
// in 3D `rows` picks the CTA tile: march3d_tile_rows(PDE_NSE) rows at four CTAs per SM, or 16 rows
// at one CTA per SM (tensor-map boxes of rows + 2 rows either way; 2D ignores it).
LaunchFn find_march_lean(int lat, int levels, int st, int lean, int rows = 4);
// Tile rows a 3D lean solver of this grid runs with: 16 where the grid has enough 16-row tiles to
// fill the GPU with one CTA per SM, march3d_tile_rows(PDE_NSE) otherwise; force > 0 asks for the
// 16-row tiles and force < 0 for the narrow ones whatever the grid (for comparisons).
int march3d_lean_tile_rows(int nx, int ny, int nz, int force = 0);

// Encode a 2D / 3D tiled TMA descriptor over one field of a ghosted level buffer
// (box = boxw x 1 [x 1] elements).  Returns 0 on success.
// promote_l2 = false: no L2 promotion of the box's requests (only the box's own sectors are
// fetched), for kernels whose neighbouring CTAs do not read the surrounding bytes at about the
// same time.
int encode_field_map(CUtensorMap* m, void* field_base, int st, const Geom& g, int boxw, int boxh, int boxd,
                     bool promote_l2 = true);

// Utility kernels (k_util.cu).
// Rows r (r = y + z ny) in [r_lo, r_hi) only (r_hi < 0: every row); the dense buffer holds those
// rows, x fastest.
cudaError_t launch_pack(const Geom& g, int st, const void* src, int src_dtype, void* dst_level, int field,
                        double ref, cudaStream_t s, long long r_lo = 0, long long r_hi = -1);
cudaError_t launch_unpack(const Geom& g, int st, const void* src_level, int field, double ref, void* dst,
                          int dst_dtype, cudaStream_t s, long long r_lo = 0, long long r_hi = -1);
// Rows [r_lo, r_hi) of all nf fields of a level to (pack) or from (unpack) nf dense buffers of
// element type dtype (MMFD_DT_*), one launch; refs are the fields' storage references.
cudaError_t launch_rows(const Geom& g, int st, bool pack, const void* const* bufs, int nf, int dtype, void* level,
                        const double* refs, long long r_lo, long long r_hi, cudaStream_t s);
// Copy the boundary ring (x = 0 / nx - 1, y = 0 / ny - 1, z = 0 / nz - 1 in 3D) of every field
// from one level buffer to another of the same layout and storage (Dirichlet boundaries).
cudaError_t launch_ring_copy(const Geom& g, const void* src_level, void* dst_level, cudaStream_t s);
// Deterministic FP64 reductions over the interior of one field: op 0 sum, 1 max|v|,
// 2 non-finite count; with ref != NULL: op 3 -> (sum |v - ref|, sum |ref|, max |v - ref|, max |ref|).
cudaError_t launch_reduce(const Geom& g, int st, const void* level, int field, double fref, int op,
                          const void* ref, int ref_dtype, double* d_partials, int nparts, double* d_out,
                          cudaStream_t s);
int reduce_parts_needed();

}  // namespace mmfd
