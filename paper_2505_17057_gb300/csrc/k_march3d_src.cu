// k_march3d_src.cu -- the 3D plane-marching TMA kernels with source terms (LCDE on D3Q7 / D3Q19,
// NCDE on D3Q19): the same kernels and tiling as k_march3d.cu, plus the source stencil in the
// store epilogue.
#include "k_march3d.cuh"

namespace mmfd {

namespace {

template <int LAT, int PDE, int LEVELS, int ST, int SRC>
cudaError_t launch_src(const LaunchArgs& a) {
    return launch_march3d_t<LAT, PDE, LEVELS, ST, tile_rows(PDE), march3d_stages<LAT, PDE, LEVELS, ST>(), SRC>(a);
}

template <int LAT, int PDE, int SRC>
LaunchFn pick_ls(int levels, int st) {
    if (levels == 2) {
        if (st == ST_F64) return launch_src<LAT, PDE, 2, ST_F64, SRC>;
        if (st == ST_F32) return launch_src<LAT, PDE, 2, ST_F32, SRC>;
        if (st == ST_BF16) return launch_src<LAT, PDE, 2, ST_BF16, SRC>;
    } else if (levels == 3) {
        if (st == ST_F64) return launch_src<LAT, PDE, 3, ST_F64, SRC>;
        if (st == ST_F32) return launch_src<LAT, PDE, 3, ST_F32, SRC>;
        if (st == ST_BF16) return launch_src<LAT, PDE, 3, ST_BF16, SRC>;
    }
    return nullptr;
}

template <int LAT, int PDE>
LaunchFn pick_src(int levels, int st, int src) {
    if (src == 1) return pick_ls<LAT, PDE, 1>(levels, st);
    if (src == 2) return pick_ls<LAT, PDE, 2>(levels, st);
    return nullptr;
}

}  // namespace

LaunchFn find_march3d_src(int lat, int pde, int levels, int st, int src) {
    if (lat == LAT_D3Q7) return pde == PDE_LCDE ? pick_src<LAT_D3Q7, PDE_LCDE>(levels, st, src) : nullptr;
    if (lat == LAT_D3Q19) {
        if (pde == PDE_LCDE) return pick_src<LAT_D3Q19, PDE_LCDE>(levels, st, src);
        if (pde == PDE_NCDE) return pick_src<LAT_D3Q19, PDE_NCDE>(levels, st, src);
    }
    return nullptr;
}

}  // namespace mmfd
