// stencil.cuh -- device building blocks of the MMFD update (see mmfd_internal.h for the
// paired central form the kernels evaluate).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mmfd_internal.h"

namespace mmfd {

// ------------------------------------------------------------------ storage traits
// FP32 and BF16 levels hold offsets v - ref[field] from a reference state (FP64 levels hold v).
// load / pack convert between stored offsets and values; raw / pack_raw move the offsets as they
// are (the kernels' offset arithmetic, see kload below).
template <int ST> struct Storage;
template <> struct Storage<ST_F64> {
    using S = double;
    using T = double;
    __device__ static T raw(const S* p) { return *p; }
    __device__ static S pack_raw(T v, unsigned) { return v; }
    __device__ static T load(const S* p, T) { return *p; }
    __device__ static S pack(T v, T, unsigned) { return v; }
};
template <> struct Storage<ST_F32> {
    using S = float;
    using T = float;
    __device__ static T raw(const S* p) { return *p; }
    __device__ static S pack_raw(T v, unsigned) { return v; }
    __device__ static T load(const S* p, T ref) { return ref + *p; }
    __device__ static S pack(T v, T ref, unsigned) { return v - ref; }
};
template <> struct Storage<ST_BF16> {
    using S = __nv_bfloat16;
    using T = float;
    __device__ static T raw(const S* p) { return __bfloat162float(*p); }
    // round-to-nearest-even (rnd == 0), or stochastic rounding with the 16 random low bits
    // `rnd` added before truncation.
    __device__ static S pack_raw(T d, unsigned rnd) {
        if (rnd == 0u) return __float2bfloat16_rn(d);
        unsigned b = __float_as_uint(d);
        if ((b & 0x7f800000u) == 0x7f800000u) return __float2bfloat16_rn(d);  // inf / nan
        b += (rnd & 0xffffu);
        return __ushort_as_bfloat16((unsigned short)(b >> 16));
    }
    __device__ static T load(const S* p, T ref) { return ref + raw(p); }
    __device__ static S pack(T v, T ref, unsigned rnd) { return pack_raw(v - ref, rnd); }
};

// Offset arithmetic.  The LCDE (and wave) update and the He-Luo NSE update are affine in the
// stored scalar / density with coefficients summing to A_00 = 1 (and the momentum sees the
// density only through differences), so they run on the stored offsets directly: the level t+dt
// offset comes out of the same stencil applied to the level-t offsets, with no reference added
// or subtracted and no precision lost to a large common value.  The NCDE update is nonlinear in
// phi and works on values: BF16 levels add the reference on load (FP32 NCDE levels are stored
// without an offset).  NSE velocities have zero reference (checked on the host).
template <int PDE>
__host__ __device__ constexpr bool offset_arith() { return PDE != PDE_NCDE; }

template <int ST, int PDE>
__device__ __forceinline__ typename Storage<ST>::T kload(const typename Storage<ST>::S* p, typename Storage<ST>::T ref) {
    if constexpr (ST == ST_BF16 && !offset_arith<PDE>()) return Storage<ST>::load(p, ref);
    else return Storage<ST>::raw(p);
}
template <int ST, int PDE>
__device__ __forceinline__ typename Storage<ST>::S kpack(typename Storage<ST>::T v, typename Storage<ST>::T ref, unsigned rnd) {
    if constexpr (ST == ST_BF16 && !offset_arith<PDE>()) return Storage<ST>::pack(v, ref, rnd);
    else return Storage<ST>::pack_raw(v, rnd);
}

// Starting value of a fresh accumulator: -0 is the additive identity of IEEE arithmetic (-0 + x == x
// for every x, +0 and -0 included), so the compiler can drop the first addition into it, which it
// may not do for +0 (+0 + -0 is +0).
template <typename T>
__device__ __forceinline__ constexpr T acc_zero() {
    return T(-0.0);
}

// Whether a BF16 store rounds stochastically.  SRM is a kernel's compile-time choice: 0 never, 1
// always (the launcher picks the instantiation from the step's flag, so the rounding-off kernel
// carries no hashing code), 2 decided per store from ex.sr.
template <int SRM>
__device__ __forceinline__ bool sr_on(const StepExtra& ex) {
    return SRM == 1 || (SRM == 2 && ex.sr != 0);
}

// SplitMix64 finaliser as a counter-based hash (stochastic rounding bits).
__device__ __forceinline__ unsigned sr_bits(unsigned long long seed, long long step, long long node, int f) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(step * 8 + f + 1) +
                           0xD1B54A32D192ED03ull * (unsigned long long)node;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (unsigned)(z & 0xffffu) | 1u;  // never 0 (0 selects nearest rounding)
}

// ------------------------------------------------------------------ node basis
// Fields at one node -> E_p, O_p of pair p (PDE-specific arguments of Eq. (3-3)).
template <int LAT, int PDE, typename T>
struct Basis;

// NCDE (Eq. (NCDEfeq)): A = phi, B_a = flux_a(phi), C = (M2(phi) - cs_a^2 phi) I folded into
// E_p = ePhi_p phi + eM2_p M2(phi).
template <int LAT, typename T>
struct Basis<LAT, PDE_NCDE, T> {
    static constexpr int D = lat_dim(LAT);
    T phi, m2, B[3];
    __device__ __forceinline__ void init(const T* f, const Coef<T>& c) {
        phi = f[0];
        m2 = (((c.m2[4] * phi + c.m2[3]) * phi + c.m2[2]) * phi + c.m2[1]) * phi + c.m2[0];
#pragma unroll
        for (int a = 0; a < D; ++a) B[a] = ((c.flux[a][3] * phi + c.flux[a][2]) * phi + c.flux[a][1]) * phi + c.flux[a][0];
    }
    __device__ __forceinline__ T A() const { return phi; }
    __device__ __forceinline__ T rest(const Coef<T>& c) const { return c.rPhi * phi + c.rM2 * m2; }
    template <int P>
    __device__ __forceinline__ void eo(const Coef<T>& c, T& E, T& O) const {
        E = c.ePhi[P] * phi + c.eM2[P] * m2;
        T o = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (pair_e(LAT, P, a) != 0) o += c.oB[P][a] * B[a];
        O = o;
    }
    __device__ __forceinline__ T mom(int) const { return T(0); }
};

// NSE, He-Luo (Remark 4): A = rho, B = rho0 u, C = rho0 u u; rho0 is folded into eC and oB,
// so E_p = eA rho + eC . (u u), O_p = oB . u.
template <int LAT, typename T>
struct Basis<LAT, PDE_NSE, T> {
    static constexpr int D = lat_dim(LAT);
    T rho, u[3];
    T uu[6];   // u_a u_b: (xx, yy, zz, xy, xz, yz), formed once per node and shared by all pairs
    __device__ __forceinline__ void init(const T* f, const Coef<T>&) {
        rho = f[0];
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = f[1 + a];
#pragma unroll
        for (int a = 0; a < D; ++a) uu[a] = u[a] * u[a];
        uu[3] = u[0] * u[1];
        if constexpr (D == 3) {
            uu[4] = u[0] * u[2];
            uu[5] = u[1] * u[2];
        }
    }
    __device__ __forceinline__ T A() const { return rho; }
    __device__ __forceinline__ T rest(const Coef<T>& c) const {
        T r = c.rA * rho;
#pragma unroll
        for (int a = 0; a < D; ++a) r += c.rC[a] * uu[a];
        return r;
    }
    template <int P>
    __device__ __forceinline__ void eo(const Coef<T>& c, T& E, T& O) const {
        T e = c.eA[P] * rho;
#pragma unroll
        for (int a = 0; a < D; ++a) e += c.eC[P][a] * uu[a];
        if (pair_e(LAT, P, 0) * pair_e(LAT, P, 1) != 0) e += c.eC[P][3] * uu[3];
        if (D == 3) {
            if (pair_e(LAT, P, 0) * pair_e(LAT, P, 2) != 0) e += c.eC[P][4] * uu[4];
            if (pair_e(LAT, P, 1) * pair_e(LAT, P, 2) != 0) e += c.eC[P][5] * uu[5];
        }
        T o = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (pair_e(LAT, P, a) != 0) o += c.oB[P][a] * u[a];
        E = e;
        O = o;
    }
    __device__ __forceinline__ T mom(int a) const { return u[a]; }
};

// ------------------------------------------------------------------ lean He-Luo form
// Whether pair p is an axis pair (one nonzero component of e_p) -- class 0 of Coef::nA.
__host__ __device__ constexpr int pair_class(int lat, int p) {
    int n = 0;
    for (int a = 0; a < lat_dim(lat); ++a) n += pair_e(lat, p, a) != 0 ? 1 : 0;
    return n == 1 ? 0 : 1;
}

// e_p . u for a representative direction (unit components, at most two nonzero).
template <int LAT, int P, typename T>
__device__ __forceinline__ T edot(T ux, T uy, T uz) {
    constexpr int ex = pair_e(LAT, P, 0), ey = pair_e(LAT, P, 1), ez = lat_dim(LAT) == 3 ? pair_e(LAT, P, 2) : 0;
    auto term = [](int e, T v) { return e > 0 ? v : -v; };
    if constexpr (ex != 0 && ey != 0) return ey > 0 ? (ex > 0 ? uy + ux : uy - ux) : term(ex, ux) - uy;
    else if constexpr (ex != 0 && ez != 0) return ez > 0 ? (ex > 0 ? uz + ux : uz - ux) : term(ex, ux) - uz;
    else if constexpr (ey != 0 && ez != 0) return ez > 0 ? (ey > 0 ? uz + uy : uz - uy) : term(ey, uy) - uz;
    else if constexpr (ex != 0) return term(ex, ux);
    else if constexpr (ey != 0) return term(ey, uy);
    else return term(ez, uz);
}

// One plus (SIGN = +1: output x - e_p) or minus (SIGN = -1: output x + e_p) contribution of pair P
// in the lean form (Coef::nA) from the input node's E, O.  Streaming momentum: E, O carry a+, a-
// already, the scalar contribution is E +- O and the momentum one +-kappa times it (nsm).
// General: sE = a+ E and mO = abar+ O (formed once per pair and node), the scalar contribution
// a- O +- ... and the momentum abar- E +- ... of Eq. (2-4-1) as in the general pair form.
// acc points at the output node's NF accumulators.
// Arithmetic with its rounding fixed by the source: one rounding per multiply, add or fused
// multiply-add, none left to the compiler's choice of contraction.  Kernels that evaluate the same
// node's contributions in different contexts (a value with one use in one kernel, two in another)
// then round alike.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Streaming momentum: a contribution sv of pair P in direction SIGN into one output node's
// accumulators (scalar sv, momentum +-kappa c_a / rho0 times sv).
template <int LAT, int P, int SIGN, typename T>
__device__ __forceinline__ void lean_push_sv(T* acc, const Coef<T>& cf, int l, T sv) {
    constexpr int D = lat_dim(LAT);
    acc[0] = radd(acc[0], sv);
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (pair_e(LAT, P, a) != 0) acc[1 + a] = rfma(T(SIGN * pair_e(LAT, P, a)) * cf.nsm[l][a], sv, acc[1 + a]);
}

// The streaming contribution of pair P in direction SIGN from its even / odd parts.
template <int SIGN, typename T>
__device__ __forceinline__ T lean_sv(T E, T O) {
    return SIGN > 0 ? E + O : E - O;
}

template <int LAT, int LEAN, int P, int SIGN, int NF, typename T>
__device__ __forceinline__ void lean_push(T* acc, const Coef<T>& cf, int l, T E, T O, T sE, T mO) {
    constexpr int D = lat_dim(LAT);
    if constexpr (LEAN == LEAN_STREAM) {
        lean_push_sv<LAT, P, SIGN>(acc, cf, l, lean_sv<SIGN>(E, O));
    } else {
        const T sv = SIGN > 0 ? cf.am[l] * O + sE : sE - cf.am[l] * O;
        const T mv = SIGN > 0 ? cf.abm[l] * E + mO : mO - cf.abm[l] * E;
        acc[0] += sv;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (pair_e(LAT, P, a) != 0) acc[1 + a] += (T(pair_e(LAT, P, a)) * cf.fmom[a]) * mv;
    }
}

// ------------------------------------------------------------------ ghost write-through
// Write value v of node (x, y, z) to its interior slot and to every periodic ghost image
// (x < gx also lands at x + nx, x >= nx - gx also at x - nx, with gx the ghost depth in x;
// y == 0 also at y = ny, y == ny - 1 at y = -1; likewise z; all combinations).
template <int DIM, typename S>
__device__ __forceinline__ void store_with_ghosts(S* f, const Geom& g, int x, int y, int z, S v) {
    int xs[3], ys[3], zs[3];
    int nxs = 0, nys = 0, nzs = 0;
    xs[nxs++] = x;
    if (x < g.gx) xs[nxs++] = x + g.nx;
    if (x >= g.nx - g.gx) xs[nxs++] = x - g.nx;
    ys[nys++] = y;
    if (y == 0) ys[nys++] = g.ny;
    if (y == g.ny - 1) ys[nys++] = -1;
    zs[nzs++] = z;
    if (DIM == 3) {
        if (z == 0) zs[nzs++] = g.nz;
        if (z == g.nz - 1) zs[nzs++] = -1;
    }
    for (int k = 0; k < nzs; ++k)
        for (int j = 0; j < nys; ++j)
            for (int i = 0; i < nxs; ++i) f[g.at(xs[i], ys[j], zs[k])] = v;
}

template <int LAT>
__device__ __forceinline__ long long pair_offset(const Geom& g, int p) {
    return (long long)pair_e(LAT, p, 0) + (long long)pair_e(LAT, p, 1) * g.py +
           (lat_dim(LAT) == 3 ? (long long)pair_e(LAT, p, 2) * g.pz : 0ll);
}

}  // namespace mmfd
