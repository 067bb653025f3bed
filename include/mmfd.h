/*
 * mmfd.h -- C ABI of the GB300 MMFD library (explicit macroscopic finite-difference
 * form of the EDF-based mesoscopic FD scheme, Shi, Du and Chai, arXiv 2505.17057).
 *
 * Every function returns an int status: MMFD_OK (0), MMFD_PENDING (1, poll only) or a
 * negative MMFD_ERR_* code.  No function throws, aborts or exits.  All device work is
 * enqueued on the CUDA stream given in the descriptor (or the server's stream) and is
 * asynchronous unless stated otherwise.
 *
 * Layout conventions for user-visible fields: a "level" is nf fields; each field is a
 * dense nx*ny*nz array, x fastest (index (z*ny + y)*nx + x).  LCDE/NCDE: nf = 1 (phi).
 * NSE: nf = 1 + dim, in the order (rho, u_x, u_y[, u_z]) (velocity, not momentum).
 * Internally the library keeps each level in a padded, ghost-celled layout that the
 * caller never sees.
 */
#ifndef MMFD_H
#define MMFD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define MMFD_OK 0
#define MMFD_PENDING 1               /* mmfd_poll: request not finished yet */
#define MMFD_ERR_ARG (-1)            /* malformed descriptor or argument */
#define MMFD_ERR_UNSUPPORTED (-2)    /* combination not supported (e.g. NSE on D2Q5) */
#define MMFD_ERR_UNREPRESENTABLE (-3)/* K_xy != 0 on an axis lattice (D2Q5/D3Q7) without MMFD_FLAG_DROP_OFFDIAG */
#define MMFD_ERR_UNSTABLE (-4)       /* max |lambda| > 1 + 1e-12 on the grid's wave numbers */
#define MMFD_ERR_OOM (-5)            /* device allocation failed */
#define MMFD_ERR_ADMISSION (-6)      /* server: footprint exceeds the HBM budget, or no slot */
#define MMFD_ERR_NONFINITE (-7)      /* a non-finite value was found in the fields */
#define MMFD_ERR_TIMEOUT (-8)        /* a bounded device wait ran out */
#define MMFD_ERR_CUDA (-9)           /* CUDA runtime error; text in mmfd_last_error() */
#define MMFD_ERR_STATE (-10)         /* call not valid in the object's current state */

/* ------------------------------------------------------------------ enums */
/* MMFD_LWE: the linear wave equation d_t^2 phi = div(K grad phi) (Eq. (LWE)), three-level. */
typedef enum { MMFD_LCDE = 0, MMFD_NCDE = 1, MMFD_NSE = 2, MMFD_LWE = 3 } mmfd_pde;
typedef enum { MMFD_D2Q5 = 0, MMFD_D2Q9 = 1, MMFD_D3Q7 = 2, MMFD_D3Q19 = 3 } mmfd_lattice;
/* Storage of the level buffers.  FP32 and BF16 levels hold offsets v - ref[field] from a reference
 * state (BF16: bf16(v - ref[field])); values are read back as ref[field] + offset.  The LCDE, wave
 * and NSE updates are affine in the stored scalar / density with coefficients summing to one, so
 * their kernels step the offsets directly in FP32 (no precision spent on the common value); the
 * NCDE's FP32 levels hold values (ref ignored) and its BF16 levels are stepped on values.  FP64:
 * values, arithmetic in FP64. */
typedef enum { MMFD_FP64 = 0, MMFD_FP32 = 1, MMFD_BF16 = 2 } mmfd_storage;
enum { MMFD_HOST = 0, MMFD_DEVICE = 1 };
enum { MMFD_DT_F64 = 0, MMFD_DT_F32 = 1 };          /* element type of user buffers */
enum { MMFD_COEF_EXPLICIT = 0, MMFD_COEF_TARGETS = 1 };
/* Source distribution F_j = g_j^eq(S, M_1F, 0) (Eq. (SourceF)) of the source terms of Eq. (2-1):
 * none; M_1F = 0; M_1F = S u (LCDE, with its u: the F_j of Example 1); or M_1F given as fields. */
enum { MMFD_SRC_NONE = 0, MMFD_SRC_S = 1, MMFD_SRC_SU = 2, MMFD_SRC_SM = 3 };

#define MMFD_FLAG_ALLOW_UNSTABLE 0x1u   /* skip the create-time stability rejection */
#define MMFD_FLAG_DROP_OFFDIAG 0x2u     /* axis lattices: drop K_xy (solve with diag(K)) */
#define MMFD_FLAG_STOCHASTIC_ROUND 0x4u /* BF16 storage: stochastic instead of nearest rounding */
#define MMFD_FLAG_TWO_SETS 0x8u         /* multiple-parameter-set scheme, Eq. (2-2-1b): see mmfd_desc */
#define MMFD_FLAG_THETA 0x10u           /* two-level theta-scheme, Eq. (GCN): see mmfd_desc */

/* Boundary treatment (mmfd_desc.boundary). */
#define MMFD_BC_PERIODIC 0              /* periodic in every direction (the default) */
#define MMFD_BC_DIRICHLET 1             /* prescribed values on the outermost ring of nodes */

typedef int (*mmfd_alloc_fn)(size_t bytes, void** ptr, void* ctx);
typedef void (*mmfd_free_fn)(void* ptr, void* ctx);

/*
 * Problem descriptor: the paper's statement of the problem (Sec. II, Eq. (2-1)-(2-4);
 * Sec. III.D, Eq. (LCDE); App. A lattices).  Start from mmfd_desc_init().
 *
 *  pde, lattice, levels  PDE, rDdQb lattice, 2 (explicit two-level, Eq. (2-2-2)) or
 *                        3 (explicit three-level, Eq. (3layerMMFD-1)).
 *  dim, n[3]             periodic grid (n[2] = 1 in 2D).
 *  dt, dx[3]             time step and grid spacings; c_alpha = dx_alpha / dt.
 *  d0[3]                 lattice free parameters d_0alpha = c_salpha^2 / c_alpha^2 (App. A).
 *                        D2Q9/D3Q19: used as given (mmfd_desc_init sets 1/3).  D2Q5/D3Q7:
 *                        ignored for the LCDE (derived from K, u, the scheme moments).
 *  K[3][3], u[3]         LCDE: diffusion tensor alpha D0 and constant velocity (Eq. (LCDE)).
 *                        LWE: the wave tensor alpha D0 of Eq. (LWE) (u must be zero).  The EDF
 *                        is the linear one of Eq. (TforMMFD-0) with second moment K phi / A_22
 *                        (Eq. (ME-NCDE-W-1)): on D2Q9 / D3Q19 C = K / A_22 - c_s^2 I, on
 *                        D2Q5 / D3Q7 c_salpha^2 = K_alphaalpha / A_22.  The scheme must be
 *                        three-level with A_10 = A_11 = A_21 = 0 and A_20 = -1 (Sec. III.B (3)),
 *                        e.g. mmfd_wave_coefficients; no source terms.
 *  lambda_bar            LCDE quadratic EDF parameter of Eq. (TforMMFD-0) (default 1).
 *  flux[3][4]            NCDE: B_alpha(phi) = sum_p flux[alpha][p] phi^p.
 *  diff[4]               NCDE: isotropic D(phi) = sum_p diff[p] phi^p (div(D grad phi)).
 *  rho0                  NSE: He-Luo reference density (Remark 4).
 *  coef_mode             MMFD_COEF_EXPLICIT: a, ahat (level t - dt), abar, abarhat
 *                        (NSE momentum sets, Eq. (2-4)), each (a_{-1}, a_0, a_1).
 *                        MMFD_COEF_TARGETS: targets = (a_0, A_10, A_11, A_21, A_22) solved by
 *                        Eq. (X) (three-level) or a_{-1} = 1 - a_0/2, a_1 = -a_0/2 (two-level,
 *                        Eq. (LMMFD-2-2); only targets[0] used); targets_bar likewise for the
 *                        NSE momentum set.
 *  d2, d1, bar_d2, bar_d1  with MMFD_FLAG_TWO_SETS: the multiple-parameter-set scheme of
 *                        Eq. (2-2-1b).  a / ahat (abar / abarhat) then give only the zeroth-order
 *                        term sum_k a_k phi(x); the second-difference term on the even parts
 *                        f^eq,+ takes d2, the first-difference term on the odd parts f^eq,- takes
 *                        d1.  The NSE momentum, likewise: bar_d2 on the second difference of
 *                        f^eq,-, bar_d1 on the first difference of f^eq,+.  Index [0] is level t,
 *                        [1] level t - dt (three-level), each (a_{-1}, a_0, a_1).  With a = d2 and
 *                        abar = bar_d2 this is the TRT MesoFD scheme of Eq. (2-1b) (even set d2,
 *                        odd set d1; momentum: even set bar_d1, odd set bar_d2).
 *  storage, ref[4]       storage type; FP32 / BF16 reference state per field (default ref = {rho0
 *                        for the NSE density, 0 otherwise}); NSE velocity references must be 0.
 *  flags                 MMFD_FLAG_*.
 *  temporal_depth        time steps fused per kernel launch (temporal blocking): 1 = none;
 *                        T >= 2 asks for T; 0 asks for the deepest available.  Blocking is
 *                        available for 2D two-level LCDE / NCDE grids with nx >= 128 and
 *                        ny >= 2T, up to T = 2 (FP64), 4 (FP32), 5 (BF16) -- the x ghost
 *                        columns of the padded layout hold that many levels -- and for the
 *                        2D D2Q9 He-Luo NSE in the lean streaming form (two levels, equal
 *                        spacing, a momentum set proportional to the scalar one; FP32 / BF16)
 *                        up to T = 3.  3D grids run unblocked.  Larger requests
 *                        are clamped, other configurations run unblocked; mmfd_get_info reports
 *                        the depth in use.  mmfd_step(n) runs n / T blocked launches and the
 *                        remaining n % T steps unblocked.  With BF16 storage a blocked solver
 *                        rounds the state to BF16 once per T steps (the intermediate levels
 *                        stay in FP32).  For a theta-scheme solver (MMFD_FLAG_THETA) the depth
 *                        counts Jacobi sweeps fused per launch instead (2D grids with nx >= 128,
 *                        up to 2 for FP64 and 4 for FP32); every mmfd_step is one time step.
 *  seed                  BF16 stochastic-rounding seed.
 *  stream                cudaStream_t (NULL = legacy default stream).
 *  alloc/free_fn/ctx     device allocator for the level buffers (NULL = cudaMalloc/cudaFree).
 *  source, b, bhat       source terms of Eq. (2-1) / (3layer-1): the update gains
 *                        dt sum_j sum_k [ b_k F_j(x + k c_j dt, t) + bhat_k F_j(x + k c_j dt, t - dt) ]
 *                        with F_j = g_j^eq(S, M_1F, 0) (Eq. (SourceF)); source = MMFD_SRC_*
 *                        (LCDE / NCDE only; MMFD_SRC_SU: LCDE only).  b, bhat are (b_{-1}, b_0,
 *                        b_1); bhat is for three-level solvers (it must be zero for two-level
 *                        ones).  b = bhat = 0 selects the defaults b = (1, 0, 0) (two-level) and
 *                        b = (3/2, 0, 0), bhat = (-1/2, 0, 0) (three-level, as in Sec. III.C and
 *                        Example 1).  The source fields are set with mmfd_set_source.  A solver
 *                        with sources runs unblocked (temporal_depth 1).
 *  theta                 with MMFD_FLAG_THETA: the two-level theta-scheme of Eq. (GCN), theta in
 *                        [0, 1] (mmfd_desc_init sets 1/2, Crank-Nicolson).  theta weights the
 *                        difference terms of the old level and 1 - theta those of the new one:
 *                        with phi + L phi the explicit update Eq. (2-2-2), every step solves
 *                            (I - (1 - theta) L) phi^{n+1} = (I + theta L) phi^n.
 *                        theta = 1 is Eq. (2-2-2), theta = 0 the implicit Eq. (2-2-3).  LCDE,
 *                        two-level, FP64 or FP32 storage, no source terms.  The system is solved
 *                        by a Jacobi iteration started from phi^n, with a sweep count fixed at
 *                        create time so that the iteration error is below the storage type's
 *                        rounding (mmfd_info_t.sweeps); MMFD_ERR_UNSUPPORTED when the
 *                        iteration would not contract.  The stability check uses Eq. (Tcond1-1).
 *                        temporal_depth fuses sweeps (see there); the server does not take such
 *                        requests.
 *  boundary              MMFD_BC_PERIODIC (0, default) or MMFD_BC_DIRICHLET: the nodes with
 *                        x = 0 or nx - 1, y = 0 or ny - 1 (and z = 0 or nz - 1 in 3D) hold
 *                        prescribed values.  Every step updates the other nodes as usual (their
 *                        stencils reach only nodes of the grid) and then sets the boundary nodes
 *                        of the new level from the boundary values (mmfd_set_boundary; until it
 *                        is called, those of the field given to mmfd_set_fields level 0).  This
 *                        is how Example 3 of Sec. IV is posed (exact values on the boundary).
 *                        Needs at least 3 nodes along every axis; runs unblocked; not with the
 *                        theta-scheme; the server does not take such requests.  The create-time
 *                        stability check still uses the periodic symbol.
 */
typedef struct {
    int pde, lattice, levels;
    int dim;
    long long n[3];
    double dt, dx[3];
    double d0[3];
    double K[3][3];
    double u[3];
    double lambda_bar;
    double flux[3][4];
    double diff[4];
    double rho0;
    int coef_mode;
    double a[3], ahat[3], abar[3], abarhat[3];
    double targets[5], targets_bar[5];
    double d2[2][3], d1[2][3], bar_d2[2][3], bar_d1[2][3];
    int storage;
    unsigned flags;
    double ref[4];
    int temporal_depth;
    unsigned long long seed;
    void* stream;
    mmfd_alloc_fn alloc;
    mmfd_free_fn free_fn;
    void* alloc_ctx;
    int source;
    double b[3], bhat[3];
    double theta;
    int boundary;
} mmfd_desc;

/* Derived constants of a created solver (read-only view, for checking and reporting). */
typedef struct {
    int nf;                      /* fields per level */
    int levels_stored;           /* level buffers held on the device */
    double a[3], ahat[3], abar[3], abarhat[3]; /* resolved coefficients (a_{-1}, a_0, a_1) */
    double A10, A20, A21, A22;   /* scheme moments, Eq. (4-2-0) / (4-2-00) */
    double c[3], d0[3], cs2[3];  /* lattice scaling, App. A */
    double w[19];                /* lattice weights omega_j in App. A order */
    double Cmat[3][3];           /* LCDE: EDF C per unit phi (Eq. (TforMMFD-0)) */
    double m2[5];                /* NCDE: second-moment target polynomial M2(phi) */
    double max_lambda;           /* max |amplification| found by the create-time check (-1: not checked) */
    double bytes_per_lu;         /* compulsory HBM bytes per lattice update (theta-scheme: per step,
                                    the right-hand side and every Jacobi sweep) */
    long long device_bytes;      /* device memory held by the level buffers */
    int temporal_depth;          /* depth in use */
    long long steps_done;        /* time levels advanced so far */
    char kernel[32];             /* name of the step kernel family in use */
    int sweeps;                  /* theta-scheme: Jacobi sweeps per step (0: explicit scheme) */
    int tile_rows;               /* 3D marching kernels: rows of the x-y tile a CTA stages per plane
                                    (16 for the lean NSE kernels on large grids, else 4 or 8); 0 for
                                    the other kernel families */
} mmfd_info_t;

typedef struct mmfd_solver mmfd_solver;

/* Fill a descriptor with defaults (D2Q9 LCDE two-level FP32, d0 = 1/3, lambda_bar = 1,
 * rho0 = 1, targets a_0 = 0).  Host only. */
int mmfd_desc_init(mmfd_desc* d);

/* Validate the descriptor, resolve the scheme coefficients and EDF constants, run the
 * create-time stability check, and allocate the level buffers.  *out owns all device memory.
 * The stability check is exact for the LCDE (the amplification symbol on the grid's wave numbers,
 * Sec. III); NCDE and NSE problems are checked linearised about their reference state (see
 * mmfd_linear_stability; mmfd_check_fields repeats it about the fields' extreme states) -- watch
 * long nonlinear runs with mmfd_reduce(..., MMFD_RED_NONFINITE, ...).
 * The step kernel family is chosen here (mmfd_get_info names it): the TMA marching kernels for
 * grids at least 128 nodes wide, the one-node-per-thread direct kernel otherwise.  For the
 * He-Luo NSE with one speed on every axis on D2Q9, or on D3Q19 with d_0 = 1/3 (FP32 / BF16 storage)
 * the marching kernels run a lean form of the same update: the uu terms of Eq. (3-3) through
 * |u|^2 and (e_p . u)^2, a+ / a- folded into the pair parts, and, when the momentum set is
 * proportional to the scalar one ((abar-, abar+) = kappa (a+, a-), e.g. LBGK tau = 1), the
 * momentum taken from the scalar contributions (kernel names *_nse_s, else *_nse_g).  The 3D lean
 * kernels stage 16-row tiles at one CTA per SM where the grid has enough of them to fill the GPU
 * (x strips x 16-row tiles x 32-plane segments >= 256, ny >= 128), 4-row tiles at four CTAs per
 * SM otherwise; the tile changes only which warp computes a node, not its arithmetic.  Setting
 * the environment variable MMFD_FORCE_KERNEL=direct before mmfd_create selects the direct
 * kernel for any grid, MMFD_FORCE_KERNEL=generic the general pair form,
 * MMFD_FORCE_KERNEL=lean3d_rows16 / lean3d_rows4 the 3D lean tile (for comparisons; all compute
 * the same update). */
int mmfd_create(const mmfd_desc* desc, mmfd_solver** out);

/* Copy one level into the solver.  level 0 = t_n, level 1 = t_{n-1} (three-level only).
 * fields: nf pointers, each to nx*ny*nz values of element type dtype (MMFD_DT_*), on the
 * host (where = MMFD_HOST, pageable or pinned) or device (MMFD_DEVICE).  The data is copied;
 * pointers are not retained.  Copies are asynchronous on the solver's stream: device and
 * page-locked host buffers (the latter are read directly by the packing kernel) must stay
 * unchanged until the stream has passed this call; pageable host buffers are staged first.  Setting level 0 of a three-level solver also sets level 1
 * to the same values (the equilibrium start) unless level 1 is set afterwards. */
int mmfd_set_fields(mmfd_solver* s, int level, const void* const* fields, int where, int dtype);

/* Source fields of a solver created with a source (Eq. (2-1), F_j = g_j^eq(S, M_1F, 0) of
 * Eq. (SourceF)).  level 0 is the source at t_n (the current level), 1 at t_{n-1} (three-level
 * only).  fields: S, then, for MMFD_SRC_SM, the dim components of M_1F; each a dense nx*ny*nz
 * array as in mmfd_set_fields (same transfer rules).  The solver keeps them in FP64 (FP64
 * storage) or FP32 (otherwise).  Time levels: a step uses the sources of levels 0 and 1;
 * afterwards level 1 holds what level 0 held and level 0 keeps its values, so a source stays
 * constant in time until it is replaced -- a time-dependent source is set (level 0) before
 * every step.  Before the first step after creation or after mmfd_set_fields(level 0), setting
 * level 0 also sets level 1 unless level 1 is set explicitly.  Both levels start at zero.
 * MMFD_ERR_STATE if the solver has no source. */
int mmfd_set_source(mmfd_solver* s, int level, const void* const* fields, int where, int dtype);

/* MMFD_BC_DIRICHLET solvers: the boundary values the following steps give the boundary nodes of
 * every new level (set them before each step for time-dependent values).  fields: nf pointers
 * to full nx*ny*nz arrays (x fastest) of type dtype on host or device, of which only the
 * boundary nodes are used; copied, not retained.  MMFD_ERR_STATE if the solver is periodic. */
int mmfd_set_boundary(mmfd_solver* s, const void* const* fields, int where, int dtype);

/* Advance nsteps time levels (Eq. (2-2-2) / Eq. (3layerMMFD-1)), asynchronously on the
 * solver's stream. */
int mmfd_step(mmfd_solver* s, long long nsteps);

/* Copy one level out (level 0 = current t_n, 1 = t_{n-1}).  out: nf pointers to
 * nx*ny*nz values of type dtype on host or device.  Host copies are synchronous. */
int mmfd_fields(mmfd_solver* s, int level, void* const* out, int where, int dtype);

/* Deterministic FP64 reductions of the current level (fixed-order tree, no atomics).
 * what = MMFD_RED_SUM: out[f] = sum of field f (nf values).
 * what = MMFD_RED_MAXABS: out[f] = max |field f|.
 * what = MMFD_RED_NONFINITE: out[0] = number of non-finite values.
 * Synchronous. */
enum { MMFD_RED_SUM = 0, MMFD_RED_MAXABS = 1, MMFD_RED_NONFINITE = 2 };
int mmfd_reduce(mmfd_solver* s, int what, double* out);

/* Error norms of field `field` of the current level against a reference field ref
 * (nx*ny*nz values, type dtype, host or device): out[0] = sum |v - ref| / sum |ref|
 * (the paper's GRE, Sec. IV), out[1] = max |v - ref|, out[2] = max |ref|.  FP64,
 * synchronous. */
int mmfd_error_norms(mmfd_solver* s, int field, const void* ref, int where, int dtype, double* out);

/* Rows (2D: y) or planes (3D: z) [r0, r0 + count) of one level, to or from dense buffers: nf
 * pointers, each to count * nx (2D) or count * nx * ny (3D) values, x fastest, of element type
 * dtype, on the host or the device.  For a slab decomposition of one solve over several solvers
 * (one per GPU): each slab's solver steps its rows plus halo rows as a periodic grid and swaps the
 * halo rows with its neighbours between steps (no counterpart in the paper; paper_2505_17057_gb300
 * /slab.py has the bookkeeping).  mmfd_set_rows keeps the rows' periodic ghost images current and,
 * unlike mmfd_set_fields, leaves level t - dt of a three-level solver alone.  Asynchronous on the
 * solver's stream for device buffers; synchronous for host buffers. */
int mmfd_set_rows(mmfd_solver* s, int level, long long r0, long long count, const void* const* fields, int where,
                  int dtype);
int mmfd_get_rows(mmfd_solver* s, int level, long long r0, long long count, void* const* out, int where, int dtype);

/* Frozen-coefficient stability of the nonlinear schemes (the paper analyses the linear CDE only,
 * Sec. III.D, Theorems 1-3; the NCDE and NSE are checked here linearised about a uniform state).
 * The update is linearised about `state` -- NCDE: (phi); NSE: (rho, u_x, u_y[, u_z]) -- and a
 * Fourier mode of the perturbation is multiplied per level by the scheme's symbol matrix
 * (Eq. (TforMMFD-3) with the EDF's Jacobian; three-level: the companion matrix of Eq. (3-level)).
 * *max_amp = the largest eigenvalue modulus over the grid's wave numbers (all of them up to 96
 * per axis, else a sample).  Returns MMFD_ERR_UNSTABLE when it exceeds 1 + 1e-9 (*max_amp set),
 * MMFD_OK otherwise, MMFD_ERR_UNSUPPORTED for the linear PDEs (mmfd_create checks those exactly).
 * Host only.  mmfd_create runs the same check about the reference state (the NCDE at
 * phi = ref[0], 0 unless given; the NSE at rest, rho0 and u = 0) and refuses an unstable
 * descriptor unless MMFD_FLAG_ALLOW_UNSTABLE is set. */
int mmfd_linear_stability(const mmfd_desc* desc, const double* state, double* max_amp);

/* The same check about the extreme states of the solver's current level: the NCDE at nine values
 * of phi spanning [-max|phi|, max|phi|], the NSE at rho0 with u at the origin and on the corners
 * of the box |u_a| <= max|u_a|.  Synchronous (field reductions on the solver's stream);
 * MMFD_ERR_NONFINITE if the level holds non-finite values. */
int mmfd_check_fields(mmfd_solver* s, double* max_amp);

/* mmfd_reduce_static: the deterministic FP64 reduction of mmfd_reduce (what = MMFD_RED_SUM,
 * MMFD_RED_MAXABS or MMFD_RED_NONFINITE) over one dense device array, for callers that cannot
 * allocate device memory at the point of use (cudaFree synchronises the whole device and both
 * cudaMalloc and cudaFree can block in the driver, which an asynchronous pipeline stage, an
 * allocator's own bookkeeping path or a component held to a fixed memory budget cannot afford).
 * No counterpart in the paper.  It allocates nothing: its per-block partials live in a fixed
 * 8 KB file-scope device array (1024 doubles) that every GPU loading the library holds until
 * the process exits.
 *   field  device pointer to count values of type dtype (MMFD_DT_F64 / MMFD_DT_F32), dense;
 *   count  1 .. 2^27 elements (larger counts return MMFD_ERR_ARG: the scratch has one slot
 *          per 2^17 elements);
 *   out    device pointer to one double, written asynchronously on `stream`.
 * field and out must be device memory of the current device, or managed memory; a host
 * pointer or another device's pointer returns MMFD_ERR_ARG before anything is launched.
 * Outside stream capture every call looks up the scratch array's device address with the
 * current device (so a cudaDeviceReset, after which the array may move, is harmless); a call
 * made while `stream` is capturing reuses the address of the last uncaptured call on that
 * device, so the first call on a device must come before any capture (MMFD_ERR_STATE
 * otherwise).  All calls share the array and each overwrites the slots it uses, so nothing
 * needs clearing; calls that overlap on the GPU (other streams or threads) race on it and must
 * be serialised by the caller. */
int mmfd_reduce_static(const void* field, int dtype, long long count, int what, double* out, void* stream);

int mmfd_get_info(const mmfd_solver* s, mmfd_info_t* out);
int mmfd_set_stream(mmfd_solver* s, void* stream);
int mmfd_destroy(mmfd_solver* s);

/* Host-only helpers (no GPU needed). */
/* Eq. (X): (a_0, A_10, A_11, A_21, A_22) -> a = (a_{-1}, a_0, a_1), ahat likewise. */
int mmfd_solve_three_level(const double targets[5], double a[3], double ahat[3]);
/* Sec. III.C, special case (2): the TRT lattice-Boltzmann model with s+ + s- = 2 as a
 * three-level MMFD scheme.  s_minus (the odd-moment rate, 0 < s_minus < 2) gives, with
 * w = 1 - s_minus, the scalar / density sets a = (1, 0, w), ahat = (0, -w, 0) and the NSE
 * momentum sets abar = (1, 0, -w), abarhat = (0, w, 0) (the momentum pair follows from the same
 * collide-and-stream elimination; it gives the viscosity c_s^2 (1/s+ - 1/2) dt, the scalar pair
 * the diffusivity c_s^2 (1/s- - 1/2) dt).  The scheme reproduces the LB moments from the second
 * step on when level t - dt holds the initial moments and level t one LBGK tau = 1 step of them
 * (a = (1, 0, 0)).  Any output pointer may be NULL.  MMFD_ERR_ARG if s_minus is outside (0, 2). */
int mmfd_trt_coefficients(double s_minus, double a[3], double ahat[3], double abar[3], double abarhat[3]);
/* Sec. III.C, special case (4): the wave-equation scheme a = (gamma, 2 (1 - gamma), gamma),
 * ahat = (0, -1, 0), with A_22 = gamma (so that alpha = gamma beta c_s^2).  MMFD_ERR_ARG if gamma
 * is not finite and positive. */
int mmfd_wave_coefficients(double gamma, double a[3], double ahat[3]);
/* ---- autotuner --------------------------------------------------------------------------
 * Not from the paper: a build choice.  The step kernels take two tuning parameters, the temporal
 * depth (time steps per launch, where blocking is available) and the work-item height (rows in
 * 2D, planes in 3D, streamed per warp or CTA item; 0 = the launcher's occupancy-based choice).
 * mmfd_autotune times candidate pairs on this solver's own grid -- depths 1 .. the deepest the
 * solver allows when it was created with temporal_depth = 0, else the depth in use; heights 0,
 * 4, 8, 16, 32, 64, 128 (2D) or 0, 8, 16, 32, 64, 128 (3D marching kernels) -- and keeps the fastest for
 * later mmfd_step calls.  Trial launches read the current level(s) and write only the spare
 * buffer, so the solver's fields and step count are unchanged; the call synchronises the
 * solver's stream.  Any solver can be tuned, before or after its fields are set.
 * cache_path (NULL = no cache): a text file of earlier choices, one line per key
 * (device name, SM count, lattice, PDE, levels, storage, flags, grid, depth mode).  A hit applies
 * the stored choice without timing; a miss times the candidates and appends the choice.  A
 * cache that cannot be read or written is ignored (the tuning result still applies). */
typedef struct {
    int temporal_depth;     /* depth now in use */
    int rows_per_item;      /* work-item height now in use (0 = launcher's choice) */
    double ms_per_step;     /* measured time per time step of that choice (cached value on a hit) */
    int candidates;         /* configurations timed (0 on a cache hit) */
    int from_cache;         /* 1 if the choice came from cache_path */
} mmfd_tune_info;

int mmfd_autotune(mmfd_solver* s, const char* cache_path, mmfd_tune_info* out);

/* Resolve a descriptor's constants without touching the GPU (info filled as by create; kernel
 * names the step kernel family create would pick for a periodic explicit solver: the marching
 * kernels from 128 columns -- k_march2d / k_march3d, or their lean He-Luo NSE variants *_nse_s
 * (streaming momentum) and *_nse_g (general momentum) for FP32 / BF16 storage with one speed on
 * every axis on D2Q9, or on D3Q19 with d_0 = 1/3 -- and k_direct otherwise). */
int mmfd_describe(const mmfd_desc* desc, mmfd_info_t* out);

/* Diagnostic: launch a kernel whose mbarrier wait can never complete and check that the
 * bounded wait gives up after budget_cycles SM clocks.  Returns MMFD_ERR_TIMEOUT when the
 * failure path works (the expected result), MMFD_OK if the wait unexpectedly completed, or
 * MMFD_ERR_CUDA.  Nothing traps; the CUDA context stays usable.  No counterpart in the paper:
 * it exercises the library's own failure detection. */
int mmfd_selftest_wait_timeout(void* stream, long long budget_cycles);

const char* mmfd_strerror(int status);
/* Text of the last error on this thread (CUDA error string or validation message). */
const char* mmfd_last_error(void);

/* ------------------------------------------------------------------ serving
 * A persistent solve server with continuous batching: requests are admitted while others
 * run, as slots and HBM budget free up; every scheduler tick advances all admitted requests
 * of one kernel class in one batched launch (uneven grids packed together), replayed from
 * captured CUDA graphs.  Requests never share state: each result equals the one the same
 * request gives alone (bit-identical for the same kernel variant).
 */
typedef struct {
    size_t hbm_budget;       /* bytes of device memory the server may hold for fields */
    int max_slots;           /* concurrent requests */
    int steps_per_tick;      /* time steps per scheduler tick */
    int use_graphs;          /* capture and replay each tick's launches as a CUDA graph */
    void* stream;            /* cudaStream_t for all server work */
} mmfd_server_desc;

typedef struct {
    int status;              /* MMFD_OK or an error of this request */
    long long steps_done;
    double submit_s, admit_s, finish_s; /* host monotonic clock, seconds */
    int nf;
    long long n[3];
} mmfd_result;

typedef struct {
    long long submitted, admitted, finished, rejected;
    long long lattice_updates;   /* total node updates done */
    long long ticks, launches, graph_replays;
    size_t bytes_in_use;
    int active;
} mmfd_server_stats;

typedef struct mmfd_server mmfd_server;

/* Create a server.  Environment read at creation (for comparisons and tests):
 *   MMFD_SERVE_QUEUE=1        every batched class runs all steps of a tick as one persistent
 *                             launch: a device-resident work queue of (step, tile) items, each
 *                             tile waiting (bounded, about a second) until its request's
 *                             previous step is complete.  Same results as the per-step launches.
 *   MMFD_SERVE_QUEUE_STALL=1  (with the queue) no wait can be met: every wait runs out and the
 *                             results of the server's requests report MMFD_ERR_TIMEOUT.  Only
 *                             for testing the failure path. */
int mmfd_server_create(const mmfd_server_desc* desc, mmfd_server** out);
/* Queue a solve: the descriptor (stream and allocator fields ignored), the initial level
 * (nf host pointers, MMFD_DT_F64 or F32, copied at submit) and the step count.  Returns
 * MMFD_ERR_ADMISSION at once if the request could never fit the budget. */
int mmfd_submit(mmfd_server* s, const mmfd_desc* d, const void* const* init, int dtype,
                long long nsteps, unsigned long long* ticket);
/* Drive the scheduler (admit, launch one tick) and report the ticket: MMFD_PENDING while it
 * runs, MMFD_OK when done (res filled), <0 on error. */
int mmfd_poll(mmfd_server* s, unsigned long long ticket, mmfd_result* res);
/* Run the scheduler until every queued request is finished. */
int mmfd_server_drain(mmfd_server* s);
/* Copy a finished request's final level (nf pointers, host or device, type dtype).
 * MMFD_ERR_TIMEOUT if a kernel of the server gave up a bounded wait (a TMA copy of a solo
 * launch, or the work queue's wait for a previous step); the server's results are then void. */
int mmfd_result_fields(mmfd_server* s, unsigned long long ticket, void* const* out, int where, int dtype);
/* Forget a finished request and free its memory. */
int mmfd_release(mmfd_server* s, unsigned long long ticket);
int mmfd_server_get_stats(const mmfd_server* s, mmfd_server_stats* out);
int mmfd_server_destroy(mmfd_server* s);

#ifdef __cplusplus
}
#endif

#endif /* MMFD_H */
