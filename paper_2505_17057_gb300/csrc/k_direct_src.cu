// k_direct_src.cu -- instantiations of the one-node-per-thread kernels with source terms
// (LCDE / NCDE; every lattice, level count and storage type).
#include "k_direct.cuh"

namespace mmfd {

template <int LAT, int PDE, int SRC>
static LaunchFn pick_src_ls(int levels, int st) {
    if (levels == 2) {
        if (st == ST_F64) return launch_direct_src<LAT, PDE, 2, ST_F64, SRC>;
        if (st == ST_F32) return launch_direct_src<LAT, PDE, 2, ST_F32, SRC>;
        if (st == ST_BF16) return launch_direct_src<LAT, PDE, 2, ST_BF16, SRC>;
    } else if (levels == 3) {
        if (st == ST_F64) return launch_direct_src<LAT, PDE, 3, ST_F64, SRC>;
        if (st == ST_F32) return launch_direct_src<LAT, PDE, 3, ST_F32, SRC>;
        if (st == ST_BF16) return launch_direct_src<LAT, PDE, 3, ST_BF16, SRC>;
    }
    return nullptr;
}

template <int LAT, int PDE>
static LaunchFn pick_src(int levels, int st, int src) {
    if (src == 1) return pick_src_ls<LAT, PDE, 1>(levels, st);
    if (src == 2) return pick_src_ls<LAT, PDE, 2>(levels, st);
    return nullptr;
}

LaunchFn find_direct_src(int lat, int pde, int levels, int st, int src) {
    switch (lat) {
    case LAT_D2Q5:
        return pde == PDE_LCDE ? pick_src<LAT_D2Q5, PDE_LCDE>(levels, st, src) : nullptr;
    case LAT_D3Q7:
        return pde == PDE_LCDE ? pick_src<LAT_D3Q7, PDE_LCDE>(levels, st, src) : nullptr;
    case LAT_D2Q9:
        if (pde == PDE_LCDE) return pick_src<LAT_D2Q9, PDE_LCDE>(levels, st, src);
        if (pde == PDE_NCDE) return pick_src<LAT_D2Q9, PDE_NCDE>(levels, st, src);
        return nullptr;
    case LAT_D3Q19:
        if (pde == PDE_LCDE) return pick_src<LAT_D3Q19, PDE_LCDE>(levels, st, src);
        if (pde == PDE_NCDE) return pick_src<LAT_D3Q19, PDE_NCDE>(levels, st, src);
        return nullptr;
    }
    return nullptr;
}

}  // namespace mmfd
