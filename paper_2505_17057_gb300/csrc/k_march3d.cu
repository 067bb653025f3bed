// k_march3d.cu -- instantiations of the 3D plane-marching TMA kernels.
#include "k_march3d.cuh"

namespace mmfd {

namespace {

template <int LAT, int PDE, int LEVELS, int ST>
LaunchFn pick() {
    return launch_march3d_t<LAT, PDE, LEVELS, ST, tile_rows(PDE), march3d_stages<LAT, PDE, LEVELS, ST>()>;
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

int march3d_tile_rows(int pde) { return tile_rows(pde); }

LaunchFn find_march3d(int lat, int pde, int levels, int st) {
    if (lat == LAT_D3Q7) return pde == PDE_LCDE ? pick_ls<LAT_D3Q7, PDE_LCDE>(levels, st) : nullptr;
    if (lat == LAT_D3Q19) {
        if (pde == PDE_LCDE) return pick_ls<LAT_D3Q19, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_ls<LAT_D3Q19, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_ls<LAT_D3Q19, PDE_NSE>(levels, st);
    }
    return nullptr;
}

}  // namespace mmfd
