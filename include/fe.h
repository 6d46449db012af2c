/*
 * fe.h -- C ABI of libfe.so: compressible fast-Eulerian PISO step on GB300.
 *
 * Method: Cerminara, Berselli, Esposti Ongaro, Salvetti, "Direct numerical
 * simulation of a compressible multiphase flow through the fast Eulerian
 * approach" (arXiv:1404.0959).  Sec. 2 par. 1: PISO pressure-velocity
 * coupling with fourth-order central interpolation and an adaptive time step;
 * Sec. 2 par. 2 and footnotes: Equilibrium-Eulerian dust (first-order Stokes
 * expansion u_p = u - tau_p Du/Dt), Fourier (q = -k grad T) or barotropic
 * (p ~ rho^gamma) closure; Sec. 1: decaying homogeneous isotropic turbulence
 * at r.m.s. Mach 0.2 / 0.5 on a periodic box.  The paper prints no
 * equations; the discrete step implemented here is stated in full in the
 * documentation of fe_step below.
 *
 * Conventions (every entry point):
 *  - Return 0 (FE_OK) on success, a negative FE_ERR_* code on failure;
 *    fe_strerror() gives a message.  FE_ERR_INVALID_ARG leaves the context
 *    unchanged.
 *  - One context = one or more independent periodic boxes ("ensemble"),
 *    all advanced together; every kernel launch covers all boxes.
 *  - Grid: box [0, 2 pi)^3, N^3 cells, h = 2 pi / N; a cell field is N^3
 *    contiguous values, flat index i + N*(j + N*k), x fastest (SoA).  A face
 *    field of direction d holds at cell index c the value on the face
 *    between cell c and its +d neighbour.
 *  - Field precision: FE_FP64 -> double; FE_FP32_MIXED -> float (Krylov dot
 *    products, refinement residuals and conserved totals still in double).
 *  - Device pointers are borrowed: the caller keeps them alive and issues
 *    its own work on the stream given to fe_create (work is ordered on that
 *    stream).  Host pointers are read/written synchronously before return.
 *  - The context owns all of its device memory (allocated in fe_create,
 *    freed in fe_destroy).  Calls on one context must not run concurrently.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FE_OK                  0
#define FE_ERR_INVALID_ARG    -1
#define FE_ERR_CUDA           -2
#define FE_ERR_NOT_CONVERGED  -3
#define FE_ERR_NONFINITE      -4
#define FE_ERR_OOM            -5
#define FE_ERR_UNSUPPORTED    -6
#define FE_ERR_TOO_LARGE      -7   /* grid larger than a fixed static buffer */

/* precision */
#define FE_FP64        0
#define FE_FP32_MIXED  1

/* closure (Sec. 2 footnotes) */
#define FE_BAROTROPIC  0   /* p = rho^gamma / gamma, no energy equation     */
#define FE_FOURIER     1   /* total-energy equation, q = -kappa grad T      */

/* pressure-correction solver */
#define FE_PCG_JACOBI       0   /* SPD operator (transonic = 0)              */
#define FE_BICGSTAB_JACOBI  1   /* any operator (required for transonic = 1) */
#define FE_FCG_LEARNED      2   /* flexible CG, learned preconditioner with  *
                                 * Jacobi fallback (needs fe_load_preconditioner) */
#define FE_FGMRES_LEARNED   3   /* flexible GMRES(20) (Saad 1993), any operator  *
                                 * (transonic included): learned directions when *
                                 * a network is loaded, Jacobi otherwise; one box, *
                                 * N divisible by 4; host-driven (no CUDA graph)  */
#define FE_PCG_POLY         4   /* SPD operator (transonic = 0): CG with the      *
                                 * first-order Neumann polynomial preconditioner *
                                 * P = D^-1 (2 I - M D^-1) (Dubois, Greenbaum and *
                                 * Rodrigue 1979) in FP32 (mixed-precision)       *
                                 * contexts; FP64 contexts run FE_PCG_JACOBI     */

/* field ids for fe_set_field / fe_get_field */
#define FE_RHO   0
#define FE_UX    1
#define FE_UY    2
#define FE_UZ    3
#define FE_P     4
#define FE_T     5   /* temperature, Fourier closure only */
#define FE_PHIX  6   /* face mass flux per unit area, x faces */
#define FE_PHIY  7
#define FE_PHIZ  8
#define FE_Y0    9   /* dust mass fraction of class j is FE_Y0 + j */
#define FE_V0   17   /* two-fluid dust: velocity component m of class j is FE_V0 + 3 j + m */

/* fe_init_state modes */
#define FE_INIT_SPECTRAL 0  /* random solenoidal u from (seed, k0, mach_rms); rho = T = 1, Y = Y0 */
#define FE_INIT_DERIVE   1  /* keep rho, u, Y (and T) already set; derive p (EOS) and phi = I4(rho) I4(u) */

#define FE_MAX_DUST 8

/* dust model (Sec. 2 par. 2) */
#define FE_DUST_EQUILIBRIUM 0  /* Equilibrium-Eulerian: particle velocity u - tau_p Du/Dt    */
#define FE_DUST_TWO_FLUID   1  /* Eulerian two-fluid: each class carries its own momentum */

/* coupling of the dust to the gas (Marble's dusty-gas mixture, the Sec. 2 par. 3 footnote) */
#define FE_COUPLING_ONE_WAY 0  /* the dust does not act on the gas                          */
#define FE_COUPLING_TWO_WAY 1  /* the drag's reaction -rho Ysum Du/Dt loads the gas momentum */

typedef struct fe_ctx fe_ctx;   /* opaque */

typedef struct {
    int32_t n_boxes;            /* >= 1                                          */
    const int32_t* N;           /* [n_boxes] cells per side, 8 <= N <= 512       */
    int32_t precision;          /* FE_FP64 | FE_FP32_MIXED                       */
    int32_t closure;            /* FE_BAROTROPIC | FE_FOURIER                    */
    double gamma;               /* ratio of specific heats (1.4)                 */
    double Pr;                  /* Prandtl number (Fourier)                      */
    const double* nu;           /* [n_boxes] kinematic viscosity; mu = nu        */
    int32_t n_dust;             /* dust classes, 0..FE_MAX_DUST                  */
    const double* tau_p;        /* [n_boxes * n_dust] particle relaxation times  */
    const double* Y0;           /* [n_boxes * n_dust] initial mass fractions     */
    const double* mach_rms;     /* [n_boxes] initial r.m.s. Mach number          */
    const double* k0;           /* [n_boxes] spectrum peak wavenumber            */
    const uint64_t* seed;       /* [n_boxes] RNG seeds                           */
    double cfl;                 /* Courant number of the adaptive step (0.5)     */
    double dt_growth_max;       /* max dt ratio between steps (1.2)              */
    double dt_max;              /* upper bound on dt (use HUGE_VAL for none)     */
    int32_t n_corr;             /* PISO correctors, >= 1 (2 recommended)         */
    int32_t solver;             /* FE_PCG_JACOBI | FE_BICGSTAB_JACOBI | FE_FCG_LEARNED |
                                 * FE_FGMRES_LEARNED | FE_PCG_POLY */
    double p_tol;               /* ||b - M x||_2 <= p_tol ||b||_2                */
    int32_t p_maxit;            /* Krylov iteration cap per solve                */
    int32_t transonic;          /* 1: add the psi-convection term (non-symmetric) */
    int32_t learned_every;      /* FE_FCG_LEARNED, FE_FGMRES_LEARNED: network direction at
                                 * iterations it with it % learned_every == 0 (1 = every
                                 * iteration), Jacobi direction otherwise; 0 = the first
                                 * direction of each corrector's solve only (mixed
                                 * precision: of its first refinement solve; such steps
                                 * are host-driven, not CUDA graphs) */
    int32_t dust_model;         /* FE_DUST_EQUILIBRIUM | FE_DUST_TWO_FLUID (tau_p > 0 required) */
    int32_t coupling;           /* FE_COUPLING_ONE_WAY | FE_COUPLING_TWO_WAY (barotropic closure
                                 * and equilibrium dust only, else FE_ERR_UNSUPPORTED) */
} fe_params;

typedef struct {
    double t;                   /* time after the step                           */
    double dt;                  /* step just taken                               */
    int32_t iters[4];           /* Krylov iterations of correctors 1..4          */
    double rel_res[4];          /* true relative residual of correctors 1..4     */
} fe_step_info;

typedef struct {
    int32_t iters;              /* Krylov iterations                             */
    double rel_res_true;        /* ||b - M x|| / ||b|| recomputed from x         */
} fe_solve_info;

typedef struct {
    double ke;                  /* <rho |u|^2> / 2                               */
    double ke_u;                /* <|u|^2> / 2                                   */
    double enstrophy;           /* <|curl u|^2> / 2 (Gauss-gradient curl)        */
    double taylor;              /* sqrt(sum_d <u_d^2> / sum_d <(d u_d/d x_d)^2>) */
    double rho_rms;             /* sqrt(<(rho - <rho>)^2>)                       */
    double mass;                /* h^3 sum rho                                   */
    double dust_mass[FE_MAX_DUST]; /* h^3 sum rho Y_j                            */
    double energy;              /* h^3 sum rho E (Fourier) or h^3 sum rho|u|^2/2 */
    double t;                   /* current time                                  */
    double dt_prev;             /* last step                                     */
} fe_diag;

/* Allocate a context for prm (arrays are copied).  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  Uses the current device. */
int fe_create(const fe_params* prm, void* cuda_stream, fe_ctx** out);

/* Initial state of one box (box >= 0) or of all boxes (box = -1).
 * FE_INIT_SPECTRAL: decaying-HIT start (Sec. 1): u random solenoidal with
 * E(k) ~ k^4 exp(-2 (k/k0)^2), r.m.s. |u| = mach_rms (sound speed 1);
 * rho = 1, T = 1, Y_j = Y0_j, then as FE_INIT_DERIVE.  The random numbers
 * are SplitMix64 draws 2(3f+c), 2(3f+c)+1 for FFT mode f, component c,
 * through Box-Muller.  FE_INIT_DERIVE: p from the closure, phi = I4(rho)
 * I4(u_d), t = 0, no previous step (growth limit inactive).  Two-fluid dust:
 * both modes also set every class's velocity V = u (set FE_V0 + 3 j + m
 * afterwards for another start). */
int fe_init_state(fe_ctx* ctx, int box, int mode);

/* Copy one field of the current state in (set) or out (get).  src/dst hold
 * N^3 values of the context precision; *_is_device selects device or host
 * memory.  Setting FE_RHO, FE_UX..FE_UZ, FE_T or FE_Y0+j does not update p or phi: call
 * fe_init_state(FE_INIT_DERIVE) or set FE_P and FE_PHI* explicitly
 * (checkpoint restore). */
int fe_set_field(fe_ctx* ctx, int box, int field, const void* src, int src_is_device);
int fe_get_field(fe_ctx* ctx, int box, int field, void* dst, int dst_is_device);

/* The same for n fields at once: fields[q] is copied from src[q] (to
 * dst[q]); all n copies are queued before the one synchronisation at the end
 * (with pinned host memory they run back to back at the host link's rate).
 * Every id and pointer is checked first; on FE_ERR_INVALID_ARG nothing is
 * copied.  The arrays are the caller's and are not kept. */
int fe_set_fields(fe_ctx* ctx, int box, int n, const int* fields, const void* const* src, int src_is_device);
int fe_get_fields(fe_ctx* ctx, int box, int n, const int* fields, void* const* dst, int dst_is_device);

/* Time and previous step of a box (checkpoint restore; dt_prev <= 0 means none). */
int fe_set_clock(fe_ctx* ctx, int box, double t, double dt_prev);

/* Advance every box by nsteps PISO steps (Sec. 2 par. 1).  For each box,
 * with operators I4 (4-point 4th-order face interpolation), G4 (4-point
 * face gradient), G2 (compact face gradient), D (face-to-cell divergence),
 * Gc (Gauss cell gradient from I4 faces), psi = rho^n/(gamma p^n), mu = nu:
 *   dt = min(cfl h / max sum_d|u_d|, dt_growth_max dt_prev, dt_max)
 *   rho0 = rho^n - dt D(phi^n); R^n = L(u^n, phi^n) with
 *   L_m(u, phi) = -D(phi I4(u_m)) + D(tau_.m),
 *   tau_dm = mu (G4_d u_m + I4_d Gc_m u_d - 2/3 delta_dm I4_d div u);
 *   u* = (rho^n u^n + dt (R^n - Gc p^n)) / rho0;
 *   corrector k = 1..n_corr (iterate 0 = (u*, phi^n, p^n, rho0)):
 *     HbyA = (rho^n u^n + dt (R^n + L(u^{k-1}, phi^{k-1}))/2) / rho^{k-1}
 *     phi* = I4(rho^{k-1}) I4(HbyA) - dt G2(p^{k-1})
 *     solve psi p'/dt - dt/2 D(G2 p') [+ D(I4(psi p') I4(HbyA))/2] =
 *           -[(rho^{k-1} - rho^n)/dt + D(phi^n)/2 + D(phi*)/2]
 *     p^k = p^{k-1} + p'; phi^k = phi* - dt G2 p' [+ I4(psi p') I4(HbyA)]
 *     u^k = HbyA - dt Gc(p^k) / rho^{k-1}; rho^k = rho^n - dt/2 D(phi^n + phi^k)
 *     Du/Dt = (-Gc p^k + D tau(u^k)) / rho^k; per dust class
 *     phi_p = phi^k - tau_p I4(rho^k) I4(Du/Dt);
 *     (rho Y)^k = rho^n Y^n - dt/2 [D(phi_p^n I4 Y^n) + D(phi_p^k I4 Y^{k-1})]
 *     Fourier: (rho E)^k likewise with flux phi I4(E + p/rho)
 *              - sum_m tau_dm I4(u_m) - kappa G4(T), kappa = mu c_p / Pr
 *   closure: barotropic p = rho^gamma/gamma; Fourier T = (E - |u|^2/2)/c_v,
 *   p = rho R T with R = 1/gamma, c_v = R/(gamma-1).
 * Two-way coupling (coupling = FE_COUPLING_TWO_WAY): with u_p = u - tau_p a the
 *   drag per unit dust mass is the gas acceleration a, so the gas momentum gains
 *   f = -(rho Ysum) a, Ysum = sum_j Y_j^n (held over the step), and a is taken
 *   with the mixture inertia: a = (D tau - Gc p) / (rho (1 + Ysum)).  R^n above
 *   includes f^n = -(rho^n Ysum) a^n; corrector k adds -(rho^{k-1} Ysum) a to
 *   L(u^{k-1}, phi^{k-1}) with a the latest Du/Dt (a^n in the first corrector,
 *   a^{k-1} after); the pressure operator is unchanged.  For a uniform loading
 *   Y this is Marble's dusty gas: sound speed c / sqrt(1 + Y), kinematic
 *   viscosity nu / (1 + Y).  The reaction lags the implicit pressure by one
 *   corrector, so the loading must stay below 1 (dilute suspensions).
 * Two-fluid dust (dust_model = FE_DUST_TWO_FLUID): the classes' Y are not
 *   updated with u_p as above; after the gas step each class (bulk density
 *   sigma = rho Y, velocity V; pressureless, one-way coupled) is advanced by
 *   the dust face flux phi_v = phi + I4(rho) I4(V - u), mass flux F = phi_v I4(Y),
 *   momentum flux G_m = F I4(V_m): predictor sigma* = sigma^n - dt D(F^n),
 *   m* = sigma^n V^n - dt D(G^n); corrector from the gas at n+1 and the
 *   predicted dust, sigma = sigma^n - dt/2 [D(F^n) + D(F*)], m likewise;
 *   Stokes drag backward Euler after each stage,
 *   V = u^{n+1} + (m/sigma - u^{n+1}) tau_p/(tau_p + dt); Y = sigma/rho^{n+1}.
 * info: NULL or [n_boxes] records of the last step.  On
 * FE_ERR_NOT_CONVERGED / FE_ERR_NONFINITE the failing step is not
 * committed (state stays at the previous step). */
int fe_step(fe_ctx* ctx, int nsteps, fe_step_info* info);

/* Solve the pressure-correction equation M x = b of one box with the psi
 * of its current state and the given dt, the operator, solver and
 * preconditioner of the context (transonic term uses HbyA = u of the current
 * state).  b, x: device arrays (N^3, context precision).  x starts at 0.
 * Stops at ||r|| <= tol ||b|| or maxit; info->rel_res_true is recomputed
 * from x.  Returns FE_ERR_NOT_CONVERGED if maxit was reached. */
int fe_solve_pressure(fe_ctx* ctx, int box, const void* b, void* x, double dt,
                      double tol, int maxit, fe_solve_info* info);

/* Turbulence diagnostics of one box (Sec. 2 par. 1: spectrum, enstrophy,
 * kinetic energy, Taylor microscale; Fig. 1: density r.m.s.).  spectrum:
 * NULL or a host array of nbins doubles, E(k) = sum over modes with
 * round(|k|) = k of |u_hat|^2 / (2 N^6). */
int fe_diagnostics(fe_ctx* ctx, int box, fe_diag* out, double* spectrum, int nbins);

/* Q criterion (|Omega|^2 - |S|^2)/2 of the current velocity of a box into a
 * device array of N^3 context-precision values (Fig. 3 of the paper shows
 * Q iso-surfaces). */
int fe_q_criterion(fe_ctx* ctx, int box, void* q_dev);

/* Iso-surface of a cell field (Fig. 3 of the paper shows iso-surfaces of Q;
 * fe_q_criterion gives that field) by marching tetrahedra, without a
 * graphics API.  field: device array of N^3 values of the context precision
 * for box `box`.  The cube whose corners are cells (i + dx, j + dy, k + dz)
 * (dx, dy, dz in {0, 1}, values with periodic wrap, corner b = dx + 2 dy +
 * 4 dz at unwrapped position ((i + dx + 1/2) h, (j + dy + 1/2) h,
 * (k + dz + 1/2) h)) is split into the six Freudenthal tetrahedra
 * (0,1,3,7) (0,1,5,7) (0,2,3,7) (0,2,6,7) (0,4,5,7) (0,4,6,7); a corner is
 * inside when f > iso; one corner apart a (inside or outside) gives the
 * triangle (P(a,b), P(a,c), P(a,d)) with b, c, d the others in tetrahedron
 * order, two inside (a, b) and two outside (c, d) give (P(a,c), P(a,d),
 * P(b,d)) and (P(a,c), P(b,d), P(b,c)); P is the linear zero of f - iso on
 * the edge, computed from its corner of smaller b as p_lo + t (p_hi - p_lo).
 * Triangles are ordered by flat cube index i + N (j + N k), then tetrahedron.
 * The surface is closed (the split is the same in every cube).  tri: NULL
 * (max_tri = 0) or a device array of 9 * max_tri doubles (x, y, z of the three
 * corners); the first min(total, max_tri) triangles are written.  *ntri
 * receives the total count, *area the total area.  Work memory (16 bytes per
 * cell) is allocated on the first call and kept by the context. */
int fe_isosurface(fe_ctx* ctx, int box, const void* field, double iso, double* tri, long long max_tri,
                  long long* ntri, double* area);
/* Depth image of ntri triangles (device, 9 doubles each) viewed along +z
 * (orthographic) on width x width pixels covering [0, extent)^2, in single
 * precision as rasterisers work: pixel (px, py) has centre c = ((px + 1/2),
 * (py + 1/2)) extent / width (double); per triangle the corners relative to
 * the first one are rounded to FP32 (X_q = f32(x_q - x_0), ..., X_0 = Y_0 =
 * 0, Z_q = f32(z_q)) and per pixel CX = f32(c_x - x_0), CY = f32(c_y - y_0);
 * the pixel is covered when E_12, E_20, E_01, with E_ab = (X_b - X_a)(CY -
 * Y_a) - (Y_b - Y_a)(CX - X_a) in FP32, share a sign (a triangle with
 * X_1 Y_2 - Y_1 X_2 = 0 covers nothing); depth ((E_12 Z_0 + E_20 Z_1) +
 * E_01 Z_2) / ((E_12 + E_20) + E_01) in FP32, the smallest non-negative depth
 * kept, +inf where nothing is covered.  depth: device array of width^2 floats,
 * row py * width + px.  Each step is one correctly rounded operation in this
 * order. */
int fe_raster_depth(fe_ctx* ctx, const double* tri, long long ntri, int width, double extent, float* depth);

/* A-priori analysis for large-eddy simulation (Sec. 1 names LES of the plume
 * as the goal of the DNS; Sec. 2 the a-priori use of the DNS database; the
 * paper names no filter or model).  From the current rho, u of a box:
 * top-hat filter of width Delta = 2 m h per axis by the trapezoidal rule
 * (end points at half weight), tensor product, 1 <= m <= FE_LES_MAX_M and
 * 2 m + 1 <= N; Favre filtering rho_bar = bar(rho), u~ = bar(rho u) /
 * rho_bar; sub-grid stress tau_ij = bar(rho u_i u_j) - bar(rho u_i)
 * bar(rho u_j) / rho_bar; strain S_ij = (Gc_j u~_i + Gc_i u~_j) / 2 from the
 * Gauss cell gradient, |S| = sqrt(2 S:S); Smagorinsky model slot tau^M =
 * Cs^2 B with B_ij = -2 rho_bar Delta^2 |S| S^d_ij (d: deviatoric part).
 * Means over the box: k_sgs = <tau_kk>/2, pi_sgs = -<tau^d:S>, cs2_opt =
 * <tau^d:B>/<B:B> (least-squares Cs^2), corr = <tau^d:B>/sqrt(<tau^d:tau^d>
 * <B:B>), pi_model = -cs^2 <B:S>.  fields: NULL or a device array of 10 N^3
 * values of the context precision receiving rho_bar, u~_0..2 and tau in the
 * order 00 01 02 11 12 22.  Work memory (23 N^3 values) is allocated on the
 * first call and kept by the context (FE_ERR_OOM if it cannot be).  The model
 * is evaluated a priori only; it does not enter fe_step. */
#define FE_LES_MAX_M 8
typedef struct {
    double delta;       /* filter width 2 m h */
    double k_sgs;       /* <tau_kk> / 2 */
    double pi_sgs;      /* -<tau^d_ij S_ij> */
    double cs2_opt;     /* <tau^d:B> / <B:B> */
    double corr;        /* <tau^d:B> / sqrt(<tau^d:tau^d> <B:B>) */
    double pi_model;    /* -cs^2 <B:S> */
} fe_les_stats;
int fe_les_apriori(fe_ctx* ctx, int box, int m, double cs, fe_les_stats* out, void* fields);

/* Learned preconditioner (extension of the paper's pressure solve, Sec. 2
 * par. 1): a 3-level 3D-conv U-Net (16/32/64 channels, 3x3x3 kernels,
 * periodic padding, ReLU; BF16 weights and activations, FP32 accumulation on
 * the tensor cores) that corrects the Jacobi direction of flexible CG
 * (solver FE_FCG_LEARNED; one box, N divisible by 4).  For a residual r of
 * the operator M = diag(psi/dt) - dt/2 D(G2 .), whose Jacobi diagonal is
 * d = psi/dt + 3 dt/h^2, with rms(r) = sqrt(mean r^2) and d0 = 1/(1/dt +
 * 3 dt/h^2) (d at psi = 1):
 *     input channel 0 = (r/d) / (rms(r) d0),  channel 1 = (3 dt/h^2) / d,
 *     direction z = r/d + rms(r) d0 y,  y = network(input).
 * A network whose last layer is zero gives exactly the Jacobi direction.
 * When <z, r> <= 0 the Jacobi direction is used instead, so plain
 * preconditioned CG remains the fallback.  With FE_FGMRES_LEARNED the same
 * direction is formed for each unit Arnoldi vector v_j (right
 * preconditioning, M Z_k = V_{k+1} H_k; x minimises ||b - M x|| over the
 * span of Z_k), which needs no symmetry and so also serves the transonic
 * operator; a network direction that is not finite, is zero, has an image
 * already in the span of the basis (new component below 1e-5 of its norm),
 * or shrinks the least-squares residual by less than 10 % is replaced by the
 * Jacobi direction, and without a loaded network every direction is Jacobi's.
 * Layers, in parameter order: e1a 2->16, e1b 16->16, d1 16->32 (stride 2),
 * e2 32->32, d2 32->64 (stride 2), e3 64->64, u2 [up2(e3), e2] 96->32,
 * u1 [up2(u2), e1b] 48->16, out 16->1 (linear).  Parameter layout (FP32,
 * host): per layer W[27][cin][cout] (tap index (dz+1)*9 + (dy+1)*3 + (dx+1)
 * of a weight applied to x(v + (dx, dy, dz))) followed by b[cout]. */
long fe_preconditioner_size(void);   /* number of floats of the layout above */
/* Copy weights in (Adam state reset).  Allocates the network buffers on first use. */
int fe_load_preconditioner(fe_ctx* ctx, const float* weights, size_t count);
/* Copy the weights (gradients = 0) or the last training step's gradients (1) out. */
int fe_get_preconditioner(fe_ctx* ctx, float* out, size_t count, int gradients);
/* z (device, N^3 FP32) = the direction above for the device residual r
 * (context precision), the operator with time step dt > 0 and psi of the
 * current state.  The raw network output y is activation 8. */
int fe_precond_apply(fe_ctx* ctx, int box, const void* r, double dt, float* z);
/* One training step on a pair (r, e) with M e = r, M the operator with time
 * step dt > 0 and psi of the current state (device arrays, context
 * precision): input as fe_precond_apply, target t = (e - r/d) / (rms(r) d0)
 * (the part of M^{-1} r the Jacobi direction misses), loss ||y - t||^2 /
 * ||t||^2, then Adam (Kingma and Ba 2015) with learning rate lr (lr <= 0:
 * gradients only).  *loss receives the loss before the update.
 * FE_ERR_INVALID_ARG when r = 0 or e = r/d (nothing to learn). */
int fe_precond_train_step(fe_ctx* ctx, int box, const void* r, const void* e, double dt, double lr, double* loss);
/* Activations of the last network pass (inspection): layer 0..7 = e1a, e1b,
 * d1, e2, d2, e3, u2, u1 (after ReLU, channels-last, n_l^3 * C_l floats, n_l
 * = N, N/2 or N/4), 8 = network output y (N^3 floats), 9 = packed input
 * (N^3 * 16). */
int fe_precond_activation(fe_ctx* ctx, int layer, float* out, size_t count);
/* Advance the context by one step with the plain Jacobi-PCG solver and copy
 * (residual, correction) pairs of box 0 into b_out[i], x_out[i] (device
 * arrays of N^3 values of the context precision), per corrector: the
 * residuals r_k and corrections x* - x_k after Krylov iterations 2 and 5 (when
 * the solve is still running there), then the right-hand side b with its
 * converged solution x*.  *npairs = pairs written (<= max_pairs).  These are
 * the training pairs of this run; all pairs of one call belong to operators
 * with the step's dt (fe_diagnostics dt_prev after the call), which
 * fe_precond_train_step takes, with the psi of the then current state. */
int fe_harvest_pressure(fe_ctx* ctx, void* const* b_out, void* const* x_out, int max_pairs, int* npairs);

/* Run each step as one CUDA graph (on = 1): the step's kernels plus the
 * Krylov iterations and the mixed-precision refinement as conditional WHILE
 * nodes evaluated on the device (each loop also stops at its iteration cap),
 * so the host waits once per step instead of once per Krylov iteration.  The
 * graphs are built on first use for each parity of the state set and rebuilt
 * after fe_set_tiling / fe_autotune / fe_load_preconditioner.  Results are
 * identical to the host-driven path (same kernels, same order).  Off by
 * default; not used during fe_harvest_pressure, profiling, or with
 * learned_every > 1. */
int fe_use_graphs(fe_ctx* ctx, int on);

/* Convolution kernels of the learned preconditioner: mode 1 (default) runs
 * the stride-1 layers whose output grid is a multiple of 128 on the
 * fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
 * memory); mode 0 runs every layer on warp-level MMA.  Both accumulate in
 * FP32 from BF16 operands; the order of the partial sums differs.  Not part
 * of the method. */
int fe_precond_kernels(fe_ctx* ctx, int mode);

/* Plane streaming for the fused CG iteration (on by default).  For FP32
 * contexts whose boxes all have N in {64, 128, 256, 512} and the symmetric
 * operator, the kernel that forms the new direction and applies M to it
 * streams whole x-rows of each z-plane into shared memory with bulk
 * asynchronous copies instead of z-marching 32 x 8 column tiles; the
 * arithmetic per cell is the same, the order of the partial sums of
 * <pd, M pd> differs.  (FP64 contexts, bound by the FP64 pipe rather than
 * by memory, always z-march.)  Off: the z-marching kernel for every box.
 * fe_plane_streaming_active returns 1 when the next step streams, 0 when it
 * z-marches, FE_ERR_INVALID_ARG for a null context.  Not part of the method. */
int fe_use_plane_streaming(fe_ctx* ctx, int on);
int fe_plane_streaming_active(const fe_ctx* ctx);

/* Tile depth of the stencil kernels: every kernel launch covers all boxes
 * with 32 x 8-cell column tiles that walk tz z-planes.  fe_set_tiling sets tz
 * for every box, fe_set_box_tiling for one (0 = built-in default: 8 for
 * N >= 128, else 4).  fe_autotune times `trials` trial steps (computed from
 * the current state and discarded: the state and clock are unchanged) for
 * tz in {4, 8, 16, 24, 32, 48, 64} for all boxes, then, when the boxes have several
 * sizes, for each size in turn (largest first) with the other boxes fixed;
 * it keeps the fastest tiling and returns the depth of the largest box in
 * *best_tz (NULL allowed).  The x/y tile (32 x 8) and the copy lookahead of
 * the stencil kernels are compile-time constants, measured at 256^3.  Not
 * part of the method. */
int fe_set_tiling(fe_ctx* ctx, int tz);
int fe_set_box_tiling(fe_ctx* ctx, int box, int tz);
int fe_autotune(fe_ctx* ctx, int trials, int* best_tz);

/* Instrumentation (not part of the method).  fe_profile_start resets the
 * counters of the context and, when kernel_id >= 0, brackets every later
 * launch of that kernel with CUDA events on the context's stream;
 * fe_profile_stop synchronises the stream and reports the number of kernel
 * launches since the start (total and per kernel id) and the summed device
 * time of the bracketed launches.  Kernel ids run 0 .. fe_kernel_count()-1,
 * fe_kernel_name() gives their names. */
#define FE_PROFILE_MAX_KERNELS 64
typedef struct {
    int64_t launches;                          /* all kernels of this context */
    int64_t target_launches;                   /* launches of kernel_id       */
    double target_ms;                          /* their summed event time     */
    int64_t counts[FE_PROFILE_MAX_KERNELS];    /* launches per kernel id      */
} fe_profile_info;
int fe_profile_start(fe_ctx* ctx, int kernel_id);
int fe_profile_stop(fe_ctx* ctx, fe_profile_info* out);
int fe_kernel_count(void);
const char* fe_kernel_name(int kernel_id);

/* Allocation-free pressure solve.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory (for example
 * code running while another framework owns the device allocator, or
 * real-time loops that must not allocate).  It solves, for one box of N^3
 * cells (8 <= N <= FE_NOALLOC_MAX_N), the same equation and with the same
 * Jacobi-PCG as fe_solve_pressure, in FP64:
 *     psi x / dt - dt/2 D(G2 x) = b,   x starts at 0,
 * stopping at ||r|| <= tol ||b|| or maxit.  psi, b, x: device arrays of N^3
 * doubles owned by the caller (flat index i + N*(j + N*k)); stream: a
 * cudaStream_t or NULL.  No context is needed and nothing is allocated: the
 * Krylov vectors and reduction scratch live in one static device array of
 * about 6.3 MB per device (sized for N = 64), held from library load until
 * process exit.  The entry point looks up that array's device address
 * (cudaGetSymbolAddress) in the current CUDA context and caches it per
 * context.  The solve is host-polled: it reads the convergence flag back
 * every four iterations and synchronises the stream, so it cannot be
 * recorded into a CUDA graph; on a stream that is being captured it returns
 * FE_ERR_UNSUPPORTED before enqueueing anything.  All calls on a device
 * share the array and it keeps the previous call's contents (each call
 * clears its counters and flags); calls that overlap on the GPU race with
 * each other.  A launch error left by earlier unrelated work is cleared on
 * entry and not reported by this call.  Returns FE_ERR_TOO_LARGE for
 * N > FE_NOALLOC_MAX_N, FE_ERR_NOT_CONVERGED if maxit was reached,
 * FE_ERR_INVALID_ARG for other bad arguments. */
#define FE_NOALLOC_MAX_N 64
int fe_solve_pressure_noalloc(int N, const double* psi, const double* b, double* x, double dt, double tol,
                              int maxit, void* stream, fe_solve_info* info);

void fe_destroy(fe_ctx* ctx);
const char* fe_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
