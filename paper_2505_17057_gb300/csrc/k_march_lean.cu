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
LaunchFn pick3(int rows) {
    if (rows == kLeanWideRows)
        return launch_march3d_sr<LAT_D3Q19, PDE_NSE, LEVELS, ST, kLeanWideRows,
                                 march3d_stages<LAT_D3Q19, PDE_NSE, LEVELS, ST, kLeanWideRows, kLeanWideRing>(), 0, LEAN>;
    if (rows == tile_rows(PDE_NSE))
        return launch_march3d_sr<LAT_D3Q19, PDE_NSE, LEVELS, ST, tile_rows(PDE_NSE),
                                 march3d_stages<LAT_D3Q19, PDE_NSE, LEVELS, ST>(), 0, LEAN>;
    return nullptr;
}

template <int LEAN>
LaunchFn pick_dim(int dim, int levels, int st, int rows) {
    if (dim == 2) {
        if (levels == 2) return st == ST_F32 ? pick2<2, ST_F32, LEAN>() : st == ST_BF16 ? pick2<2, ST_BF16, LEAN>() : nullptr;
        if (levels == 3) return st == ST_F32 ? pick2<3, ST_F32, LEAN>() : st == ST_BF16 ? pick2<3, ST_BF16, LEAN>() : nullptr;
    } else {
        if (levels == 2)
            return st == ST_F32 ? pick3<2, ST_F32, LEAN>(rows) : st == ST_BF16 ? pick3<2, ST_BF16, LEAN>(rows) : nullptr;
        if (levels == 3)
            return st == ST_F32 ? pick3<3, ST_F32, LEAN>(rows) : st == ST_BF16 ? pick3<3, ST_BF16, LEAN>(rows) : nullptr;
    }
    return nullptr;
}

}  // namespace

LaunchFn find_march_lean(int lat, int levels, int st, int lean, int rows) {
    const int dim = lat == LAT_D2Q9 ? 2 : lat == LAT_D3Q19 ? 3 : 0;
    if (dim == 0) return nullptr;
    if (lean == LEAN_STREAM) return pick_dim<LEAN_STREAM>(dim, levels, st, rows);
    if (lean == LEAN_GENERAL) return pick_dim<LEAN_GENERAL>(dim, levels, st, rows);
    return nullptr;
}

// One 16-row tile per SM needs enough tiles to fill the GPU: (nx / 128 strips) x (ny / 16 tiles)
// per z segment of at least 32 planes, and at least 128 columns in x.
int march3d_lean_tile_rows(int nx, int ny, int nz, int force) {
    if (force != 0) return force > 0 ? kLeanWideRows : tile_rows(PDE_NSE);
    const long long strips = (nx + 127) / 128;
    const long long tiles = strips * ((ny + kLeanWideRows - 1) / kLeanWideRows);
    return (nx >= 128 && ny >= 8 * kLeanWideRows && tiles * (nz / 32) >= 256) ? kLeanWideRows : tile_rows(PDE_NSE);
}

}  // namespace mmfd
