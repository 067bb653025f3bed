// k_march2d.cu -- instantiations of the 2D row-marching TMA kernels.
#include "k_march2d.cuh"

namespace mmfd {

namespace {

// Rows per stage: two input rows per TMA box halve the per-row waits, copy issues and
// accumulator rotations.  For the NSE it costs registers (128 instead of 96, four CTAs per SM
// instead of five) and still measured faster on 4096^2 (207 vs 191 GLUPS).
constexpr int rows_per_stage(int) { return 2; }

// Ring depth per warp: about 8 KB of stages, between 3 and 12 stages in flight.
template <int LAT, int PDE, int LEVELS, int ST, int LN>
constexpr int march2d_stages() {
    constexpr size_t per = (march2d_smem<ST, LEVELS, pde_nf(PDE, LAT), 1, 1, LN, rows_per_stage(PDE)>() - 256);
    constexpr size_t n = 8192 / per;
    return n < 3 ? 3 : (n > 12 ? 12 : (int)n);
}

template <int LAT, int PDE, int LEVELS, int ST, int LN>
cudaError_t launch_variant(const LaunchArgs& a) {
    return launch_march2d_t<LAT, PDE, LEVELS, ST, 4, march2d_stages<LAT, PDE, LEVELS, ST, LN>(), LN,
                            rows_per_stage(PDE)>(a);
}

// 4 nodes per lane (128-column items: the TMA box of 128 + 2 x 16 bytes stays within the
// 256-element box limit)
template <int LAT, int PDE, int LEVELS, int ST>
cudaError_t launch_any(const LaunchArgs& a) {
    return launch_variant<LAT, PDE, LEVELS, ST, 4>(a);
}

template <int LAT, int PDE, int LEVELS, int ST>
LaunchFn pick() {
    return launch_any<LAT, PDE, LEVELS, ST>;
}

template <int LAT, int PDE>
LaunchFn pick_ls(int levels, int st) {
    if (levels == 2) {
        if (st == ST_F64) return pick<LAT, PDE, 2, ST_F64>();
        if (st == ST_F32) return pick<LAT, PDE, 2, ST_F32>();
        if (st == ST_BF16) return pick<LAT, PDE, 2, ST_BF16>();
    } else if (levels == 3) {
        if (st == ST_F64) return pick<LAT, PDE, 3, ST_F64>();
        if (st == ST_F32) return pick<LAT, PDE, 3, ST_F32>();
        if (st == ST_BF16) return pick<LAT, PDE, 3, ST_BF16>();
    }
    return nullptr;
}

}  // namespace

int march2d_rows_per_stage(int pde) { return rows_per_stage(pde); }

LaunchFn find_march2d(int lat, int pde, int levels, int st) {
    if (lat == LAT_D2Q5) return pde == PDE_LCDE ? pick_ls<LAT_D2Q5, PDE_LCDE>(levels, st) : nullptr;
    if (lat == LAT_D2Q9) {
        if (pde == PDE_LCDE) return pick_ls<LAT_D2Q9, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_ls<LAT_D2Q9, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_ls<LAT_D2Q9, PDE_NSE>(levels, st);
    }
    return nullptr;
}

}  // namespace mmfd
