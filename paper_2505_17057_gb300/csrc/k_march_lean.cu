// k_march_lean.cu -- instantiations of the 2D and 3D marching kernels in the lean He-Luo NSE form
// (Coef::nA; FP32 and BF16 storage, two and three levels), chosen by the solver when the host
// check in params.cpp accepts the problem's coefficients.
#include "k_march3d.cuh"

namespace mmfd {

namespace {

template <int LEVELS, int ST, int LEAN>
LaunchFn pick2() {
    return launch_march2d_sr<LAT_D2Q9, PDE_NSE, LEVELS, ST, 4, march2d_stages<LAT_D2Q9, PDE_NSE, LEVELS, ST, 4>(), 4,
                            rows_per_stage(PDE_NSE), 0, LEAN>;
}

template <int LEVELS, int ST, int LEAN>
LaunchFn pick3() {
    return launch_march3d_sr<LAT_D3Q19, PDE_NSE, LEVELS, ST, tile_rows(PDE_NSE),
                            march3d_stages<LAT_D3Q19, PDE_NSE, LEVELS, ST>(), 0, LEAN>;
}

template <int LEAN>
LaunchFn pick_dim(int dim, int levels, int st) {
    if (dim == 2) {
        if (levels == 2) return st == ST_F32 ? pick2<2, ST_F32, LEAN>() : st == ST_BF16 ? pick2<2, ST_BF16, LEAN>() : nullptr;
        if (levels == 3) return st == ST_F32 ? pick2<3, ST_F32, LEAN>() : st == ST_BF16 ? pick2<3, ST_BF16, LEAN>() : nullptr;
    } else {
        if (levels == 2) return st == ST_F32 ? pick3<2, ST_F32, LEAN>() : st == ST_BF16 ? pick3<2, ST_BF16, LEAN>() : nullptr;
        if (levels == 3) return st == ST_F32 ? pick3<3, ST_F32, LEAN>() : st == ST_BF16 ? pick3<3, ST_BF16, LEAN>() : nullptr;
    }
    return nullptr;
}

}  // namespace

LaunchFn find_march_lean(int lat, int levels, int st, int lean) {
    const int dim = lat == LAT_D2Q9 ? 2 : lat == LAT_D3Q19 ? 3 : 0;
    if (dim == 0) return nullptr;
    if (lean == LEAN_STREAM) return pick_dim<LEAN_STREAM>(dim, levels, st);
    if (lean == LEAN_GENERAL) return pick_dim<LEAN_GENERAL>(dim, levels, st);
    return nullptr;
}

}  // namespace mmfd
