// k_direct.cu -- instantiations of the one-node-per-thread kernels for every supported
// (lattice, PDE, levels, storage) combination.
#include "k_direct.cuh"

namespace mmfd {

template <int LAT, int PDE>
static LaunchFn pick_ls(int levels, int st) {
    if (levels == 2) {
        if (st == ST_F64) return launch_direct<LAT, PDE, 2, ST_F64>;
        if (st == ST_F32) return launch_direct<LAT, PDE, 2, ST_F32>;
        if (st == ST_BF16) return launch_direct<LAT, PDE, 2, ST_BF16>;
    } else if (levels == 3) {
        if (st == ST_F64) return launch_direct<LAT, PDE, 3, ST_F64>;
        if (st == ST_F32) return launch_direct<LAT, PDE, 3, ST_F32>;
        if (st == ST_BF16) return launch_direct<LAT, PDE, 3, ST_BF16>;
    }
    return nullptr;
}

LaunchFn find_direct(int lat, int pde, int levels, int st) {
    switch (lat) {
    case LAT_D2Q5:
        return pde == PDE_LCDE ? pick_ls<LAT_D2Q5, PDE_LCDE>(levels, st) : nullptr;
    case LAT_D3Q7:
        return pde == PDE_LCDE ? pick_ls<LAT_D3Q7, PDE_LCDE>(levels, st) : nullptr;
    case LAT_D2Q9:
        if (pde == PDE_LCDE) return pick_ls<LAT_D2Q9, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_ls<LAT_D2Q9, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_ls<LAT_D2Q9, PDE_NSE>(levels, st);
        return nullptr;
    case LAT_D3Q19:
        if (pde == PDE_LCDE) return pick_ls<LAT_D3Q19, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_ls<LAT_D3Q19, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_ls<LAT_D3Q19, PDE_NSE>(levels, st);
        return nullptr;
    }
    return nullptr;
}

}  // namespace mmfd
