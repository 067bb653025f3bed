// k_march2d.cu -- instantiations of the 2D row-marching TMA kernels.
#include "k_march2d.cuh"

namespace mmfd {

namespace {

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
