/*
 * sib.h -- C ABI of the GB300 Stokes-IB multigrid solver (libsib.so).
 *
 * Solves one semi-implicit immersed-boundary step as the linear system of the paper's
 * Eq. (matrix-impib) (Bhalla, Knepley, Adams, Guy, Griffith, "Scalable smoothing strategies for
 * a geometric multigrid method for the immersed boundary equations", Sec. 2.2):
 *
 *     [ A - dt S K J   G ] [u]   [ g + S K X^n ]
 *     [ -D             0 ] [p] = [ 0           ]
 *
 * on a periodic N x N staggered (MAC) grid of the unit square, h = 1/N, A = (rho/dt) I - mu Lap,
 * with Peskin four-point spreading S and interpolation J (S = J^T / h^2, Appendix), and the
 * stiffness K of zero-rest-length springs between Lagrangian markers (Sec. 5, Eq. F-lin-functional).
 * The solver is flexible GMRES (FP64) preconditioned by one geometric-multigrid V-cycle (Alg. 1)
 * whose smoother is additive Vanka (Alg. 2, per-cell patches) or the Schur-complement smoother
 * (Eq. approx-fact-Stokes-IB), with RT0 prolongation, restriction = its adjoint, and the Galerkin
 * coarse IB operator (Sec. 3.1-3.2).  The V-cycle may run in FP32.
 *
 * Conventions for every call
 *   - Return value: SIB_OK (0) or a negative SIB_ERR_* code; sib_last_error() gives the text.
 *     No C++ exception crosses this boundary.
 *   - Array arguments are DEVICE pointers owned by the caller unless the name ends in _host.
 *     Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream); results are valid once that stream has been synchronised.
 *   - Eulerian vectors hold 3*N*N values laid out [u | v | p], each block row-major [j][i]:
 *     u[j][i] at the x-face (i*h, (j+1/2)*h), v[j][i] at the y-face ((i+1/2)*h, j*h), p[j][i] at
 *     the cell centre.  Level-l vectors (N_l = n_min * 2^l) use the same layout with N_l.
 *   - Marker positions X are float64 (M, 2) interleaved x,y; edges int32 (E, 2); kappa float64 (E).
 *   - The library owns all workspace.  It allocates device memory in sib_create/sib_setup
 *     (and when sizes grow); sib_solve and the level calls do not allocate.
 *   - A context is not thread-safe; different contexts are independent.
 *   - N must be n_min * 2^k with n_min a power of two in [4, 16]; N <= 8192.
 */
#ifndef SIB_H
#define SIB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIB_OK                  0
#define SIB_ERR_ARG            -1  /* invalid argument (size, null pointer, option out of range)    */
#define SIB_ERR_CUDA           -2  /* a CUDA runtime call failed, or a kernel's bounded wait gave up  */
#define SIB_ERR_NONFINITE      -3  /* a non-finite value in inputs or in the Krylov recurrence        */
#define SIB_ERR_NOT_CONVERGED  -4  /* max_it reached; outputs and stats are still written             */
#define SIB_ERR_BREAKDOWN      -5  /* reserved: Arnoldi breakdown that is not a converged solve      */
#define SIB_ERR_UNIMPLEMENTED  -6  /* option combination not implemented                             */
#define SIB_ERR_STATE          -7  /* call out of order (e.g. solve before setup)                    */
#define SIB_ERR_ALLOC          -8  /* device or host allocation failed                               */
#define SIB_ERR_TOO_LARGE      -9  /* sib_spread_noalloc: N or M beyond its fixed scratch            */

#define SIB_SMOOTHER_VANKA 0       /* additive per-cell Vanka (Alg. 2 with one-cell subdomains)     */
#define SIB_SMOOTHER_SC    1       /* Schur-complement smoother (Eq. approx-fact-Stokes-IB)         */
#define SIB_SMOOTHER_RAS   2       /* restricted additive Schwarz over box subdomains (Alg. 2, boxes) */

#define SIB_PREC_FP64 0
#define SIB_PREC_FP32 1

#define SIB_MAX_LEVELS 12

typedef struct sib_ctx sib_ctx;    /* opaque, library-owned */

typedef struct {
    int    smoother;      /* SIB_SMOOTHER_VANKA (default) or SIB_SMOOTHER_SC                       */
    int    nu1, nu2;      /* pre- and post-smoothing sweeps (2, 2)                                   */
    double omega;         /* damping of one sweep: Vanka 0.8, SC 1.0 (a negative value = default)    */
    int    cheb_iters;    /* SC: Chebyshev iterations for the A_IB and Schur-complement solves (2)   */
    double cheb_lo;       /* SC: Chebyshev interval [cheb_lo, cheb_hi] * lambda_max (0.1, 1.1)       */
    double cheb_hi;
    int    power_iters;   /* SC: power iterations for lambda_max estimates at setup (10)             */
    int    vcycle_fp32;   /* 1: V-cycle in FP32 (coarsest solve FP64), 0: all FP64 (default 1)       */
    double rtol;          /* stop when ||b - L x||_2 <= rtol ||b||_2 (1e-8)                          */
    int    max_it;        /* iteration cap (100, the paper's cap)                                    */
    int    restart;       /* FGMRES restart length (100)                                             */
    int    add_SKXn;      /* 1: right-hand side g + S K X^n (paper form), 0: g only (1)              */
    int    use_graphs;    /* 1: replay the V-cycle as a CUDA graph (1)                               */
    int    fuse_small;    /* 1: levels 1 and 0 of the V-cycle run as one single-block kernel when
                             level 1 (at most 16 x 16) fits in shared memory; 0: one kernel per step (1) */
    int    smooth_krylov; /* 1: every pre- and post-smoothing stage of nu sweeps is nu iterations of
                             flexible GMRES on the level's residual equation, each preconditioned by
                             one undamped basic sweep (Sec. 3.3; nu <= 8); 0: nu damped sweeps (0)    */
    int    sc_relax;      /* SC: point relaxation preconditioning both Chebyshev iterations (Sec. 3.3,
                             SC smoothing): SIB_RELAX_JACOBI (diagonal, default) or SIB_RELAX_SGS (one
                             symmetric red-black Gauss-Seidel sweep from zero, colours 0, 1, 1, 0)    */
    int    box;           /* RAS: cells per box side b, 1, 2, 4, 8 or 16 (4)                         */
    int    box_overlap;   /* RAS: overlap o in cells on each side: b + 2 o <= 16 for b <= 8, o <= 4
                             for b = 16 (1).  A level too small for the boxes (b does not divide
                             N_l, or b + 2 o + 1 > N_l: the subdomain would wrap onto itself) is
                             smoothed by its exact level solve, x + omega L_l^+ (b - L_l x), the one
                             box clipped to the periodic level; with b = 16 the IB boxes' subdomain
                             inverses are a low-rank update of the shared one                       */
    int    domain;        /* SIB_DOMAIN_PERIODIC (default) or SIB_DOMAIN_CAVITY (see below)          */
    int    ras_tc;        /* RAS, FP32 levels: the correction of the boxes that share one inverse runs
                             on the tensor cores (tcgen05, three TF32 products per pair for FP32
                             accuracy) (1) or on the FP32 CUDA cores (0) (1).  With 16 x 16 boxes a
                             level of fewer than 1,024 boxes takes the CUDA cores either way        */
    int    l2_persist;    /* the graphs' kernels keep the finest level's FP32 IB windows in the L2
                             cache (an access-policy window, with this process's persisting L2 limit
                             set to their size) (1) or treat them as any other data (0) (0: on the
                             1024^2 differentiated solve the set-aside L2 slows the other passes
                             more than it speeds the window passes, 232 against 220 ms a step)    */
} sib_opts;

/* Domains.  SIB_DOMAIN_CAVITY is the paper's lid-driven cavity (Sec. 5) on the same layout: the seam
 * faces u(0, j) and v(i, 0) are the no-slip walls and hold 0 in every vector; tangential walls use
 * the ghost value 2 q_wall - q_inside.  The solve's right-hand side is g with its wall faces set to 0,
 * plus S K X^n, plus the regularised lid u_lid(x) = (1 - cos 2 pi x) / 2 at y = 1 as its ghost term
 * 2 mu u_lid(x_i) / h^2 on the top row of u faces.  Solves, V-cycles, sweeps and transfers then
 * follow the cavity: Vanka sweeps with the wall rules, the walled RT0 transfers with the pressure
 * prolongation reflected at the walls, coarse IB windows without wall couplings, and a coarsest
 * pseudo-inverse whose kernel is the constant pressure.  The cavity takes the Vanka smoother with
 * damped sweeps (smooth_krylov = 0), and its structure must keep its Peskin support 2.5 h away from
 * the walls; other smoothers return SIB_ERR_UNIMPLEMENTED from sib_set_options. */
#define SIB_DOMAIN_PERIODIC 0
#define SIB_DOMAIN_CAVITY   1

#define SIB_RELAX_JACOBI 0
#define SIB_RELAX_SGS    1

typedef struct {
    int    iterations;          /* FGMRES iterations performed                                       */
    int    converged;           /* 1 if the estimate reached rtol                                    */
    double rel_residual;        /* true ||b - L x|| / ||b|| computed at exit (FP64)                  */
    double rel_residual_est;    /* Givens estimate at exit                                           */
    double bnorm;               /* ||b||_2 of the (projected) right-hand side                        */
    double setup_ms;            /* device time of the last sib_setup                                 */
    double solve_ms;            /* device time of the last solve                                     */
    double history[101];        /* residual estimates, history[0] = ||b||; only the first
                                   min(iterations + 1, 101) entries are written                      */
} sib_stats;

/* ---- lifecycle ----------------------------------------------------------------------------- */
void        sib_default_opts(sib_opts* opts);
/* Creates a context for an N x N periodic grid with coarsest grid n_min x n_min (8 in the paper,
 * Sec. 5).  Allocates the grid-sized workspace.  *out is NULL on failure. */
int         sib_create(sib_ctx** out, int N, int n_min);
void        sib_destroy(sib_ctx* ctx);
const char* sib_last_error(const sib_ctx* ctx);   /* never NULL; "" when no error */

/* ---- problem definition (Sec. 2.2: rho, mu, dt; Appendix: markers and springs) ---------------- */
int sib_set_fluid(sib_ctx* ctx, double rho, double mu, double dt);
/* Copies X (M x 2), edges (E x 2, int32, 0 <= index < M) and kappa (E) from device memory into
 * library-owned buffers; marks the structure dirty.  M = 0 or E = 0 are allowed. */
int sib_set_structure(sib_ctx* ctx, int M, const double* X, int E, const int32_t* edges,
                      const double* kappa, void* stream);
/* Replaces kappa only (same edge list); marks the stiffness-dependent setup dirty. */
int sib_set_stiffness(sib_ctx* ctx, const double* kappa, void* stream);
int sib_set_options(sib_ctx* ctx, const sib_opts* opts);
/* SC smoother: override the per-level lambda_max estimates (arrays of sib_num_levels() values;
 * entry 0, the coarsest level, is ignored).  Pass NULL to return to the power-iteration estimates. */
int sib_set_eigen_estimates(sib_ctx* ctx, const double* lamA, const double* lamM);
int sib_get_eigen_estimates(const sib_ctx* ctx, double* lamA, double* lamM);

/* Builds everything that depends on X and kappa: marker binning (stable Morton-ordered sort of
 * the markers' interpolation stencils), per-level composite stencils J_l = J P (Galerkin coarse IB
 * operator, Sec. 3.1), the IB entries of every Vanka patch and of diag(A_IB), the dense coarsest
 * operator and its pseudo-inverse, and (SC) the lambda_max estimates.  Synchronises `stream`. */
int sib_setup(sib_ctx* ctx, void* stream);

/* ---- the solve (Eq. matrix-impib) -------------------------------------------------------------- */
/* g: 3N^2 right-hand side [g_u | g_v | g_p] (g_p is used as the divergence right-hand side and is
 * 0 in the paper's form).  w: 3N^2 output [u | v | p], gauge-fixed (zero-mean p; zero-mean u and
 * v when rho = 0).  When rho = 0 the velocity means of the right-hand side are removed first.
 * stats may be NULL.  Returns SIB_ERR_NOT_CONVERGED (outputs written) if max_it is reached. */
int sib_solve(sib_ctx* ctx, const double* g, double* w, sib_stats* stats, void* stream);
/* Same with HOST buffers (pageable or pinned): copies g in and w out inside the call. */
int sib_solve_host(sib_ctx* ctx, const double* g_host, double* w_host, sib_stats* stats, void* stream);
/* Solve L w = rhs for an arbitrary right-hand side rhs (3N^2), without adding S K X^n.  L is
 * symmetric, so this is also the transposed (adjoint) solve. */
int sib_solve_rhs(sib_ctx* ctx, const double* rhs, double* w, sib_stats* stats, void* stream);
/* The transposed (adjoint) solve L^T w = rhs, used by the backward pass of a differentiated solve.
 * The eliminated operator of Eq. (matrix-impib) is symmetric: S = J^T / h^2 (Appendix), K is
 * symmetric and -D = G^T on the periodic MAC grid, so L^T = L and this is the same FGMRES and
 * V-cycle as sib_solve_rhs, with the same arguments (rhs, w: 3N^2 device doubles; stats may be
 * NULL; SIB_ERR_NOT_CONVERGED with outputs written if max_it is reached).  It is kept as its own
 * entry point so that callers state which system they solve. */
int sib_solve_transpose(sib_ctx* ctx, const double* rhs, double* w, sib_stats* stats, void* stream);

/* Gradients of a loss l(w) through the solve (discrete adjoint of Eq. matrix-impib): given the
 * forward solution w and the adjoint solution lam (both 3N^2), writes
 *   dkappa[e] = -(Lam_a - Lam_b) . (Y_a - Y_b),   Lam = J lam_u / h^2,  Y = a X^n + dt J u,
 *   dX[l][d]  = sum_c (d_{X_l^d} Lam_l^c) (K Y)_l^c + a (K Lam)_l^d + dt sum_c (K Lam)_l^c d_{X_l^d} U_l^c
 * with a = add_SKXn.  dkappa: E doubles, dX: 2M doubles (M x 2).  Spread weights are recomputed
 * from X (nothing is stored between the solve and this call). */
int sib_grad(sib_ctx* ctx, const double* w, const double* lam, double* dkappa, double* dX, void* stream);

/* ---- level-wise operations (building blocks of the V-cycle, for parity checks) --------------- */
int sib_num_levels(const sib_ctx* ctx);                  /* lmax + 1; level 0 is the coarsest   */
int sib_level_size(const sib_ctx* ctx, int level);       /* N_l                                 */
/* y = L^l x (prec: SIB_PREC_FP64 -> double*, SIB_PREC_FP32 -> float*). */
int sib_apply_operator(sib_ctx* ctx, int level, int prec, const void* x, void* y, void* stream);
/* y = L^l x for the lid-driven cavity (Sec. 5: no-slip walls) instead of the periodic box.  Same
 * layout; the seam faces u(0, j) and v(i, 0) are the wall faces: x must hold 0 there and y gets 0
 * there.  Tangential wall rows use the ghost value -q_inside (the lid enters the right-hand side
 * only); the structure must keep its Peskin support 2.5 h away from the walls. */
int sib_cavity_apply_operator(sib_ctx* ctx, int level, int prec, const void* x, void* y, void* stream);
/* x <- `sweeps` additive Vanka sweeps (Alg. 2, one-cell patches; damping: the Vanka omega of the options,
 * 0.8 by default) for the lid-driven cavity's L^l x = b, in place, level >= 1; wall-face entries stay 0. */
int sib_cavity_smooth(sib_ctx* ctx, int level, int prec, void* x, const void* b, int sweeps, void* stream);
/* f = [S K J]^l u on the velocity faces: u and f hold 2 N_l^2 values [u | v]. */
int sib_apply_ib(sib_ctx* ctx, int level, int prec, const void* u, void* f, void* stream);
/* x <- `sweeps` smoothing sweeps for L^l x = b (in place), level >= 1. */
int sib_smooth(sib_ctx* ctx, int level, int prec, void* x, const void* b, int sweeps, void* stream);
/* rc = R (b - L^l x): residual on level `level` restricted to level-1 (3 N_{l-1}^2 values). */
int sib_residual_restrict(sib_ctx* ctx, int level, int prec, const void* x, const void* b, void* rc,
                          void* stream);
/* xf += P ec, ec on level-1, xf on level `level`. */
int sib_prolong_add(sib_ctx* ctx, int level, int prec, const void* ec, void* xf, void* stream);
/* x = (L^0)^+ b on the coarsest level (computed in FP64 for both precisions). */
int sib_coarse_solve(sib_ctx* ctx, int prec, const void* b, void* x, void* stream);
/* z = one V-cycle (Alg. 1) applied to b on the finest level, from a zero initial guess. */
int sib_vcycle(sib_ctx* ctx, int prec, const void* b, void* z, void* stream);
/* Fine-level interpolation U = J u (u: 2N^2, U: 2M doubles, M x 2) and spreading f = S F
 * (F: 2M doubles, f: 2N^2), FP64. */
int sib_interp(sib_ctx* ctx, const double* u, double* U, void* stream);
int sib_spread(sib_ctx* ctx, const double* F, double* f, void* stream);
/* Structure update of the semi-implicit time step (Sec. 2.2, Eq. imp-X-new):
 * X_next = X^n + dt J^n u^{n+1}.  w: 3N^2 device doubles, the solution [u | v | p] of the step (only
 * u, v are read); J^n is the interpolation at the context's current markers X^n (the lagged
 * configuration the solve used) and dt the context's.  X_next: M x 2 interleaved device doubles,
 * caller-owned (it may not alias the context's own copy of X, which stays X^n until the next
 * sib_set_structure).  Positions are not wrapped into the unit square; the periodic stencils accept
 * any position.  Requires sib_setup since the last change of structure.  A time loop sets X_next as
 * the next structure, sets up and solves again. */
int sib_advance_markers(sib_ctx* ctx, const double* w, double* X_next, void* stream);

/* ---- measurement ----------------------------------------------------------------------------- */
#define SIB_KERNEL_VANKA     0   /* one additive Vanka sweep kernel (residual + patch solves + update) */
#define SIB_KERNEL_RESIDUAL  1   /* Stokes-IB residual r = b - L x                                   */
#define SIB_KERNEL_SPREAD    2   /* spreading gather of the level                                    */
#define SIB_KERNEL_INTERP    3   /* interpolation of the level                                       */
#define SIB_KERNEL_RESTRICT  4   /* restriction of a residual from `level` to level-1                 */
#define SIB_KERNEL_PROLONG   5   /* prolongation-correction from level-1 to `level`                   */
#define SIB_KERNEL_RAS       6   /* box RAS correction from a residual (needs the RAS smoother's setup) */
#define SIB_KERNEL_IB_WINDOW 7   /* the IB force [S K J]^l u through the level's assembled windows      */
#define SIB_KERNEL_RESIDUAL_RESTRICT 8   /* the fused residual r = b - L x and its restriction to level-1 */
#define SIB_TIME_COLD     0x100  /* or-ed into `kernel`: no warm-up launch before the timed ones, so that
                                    a caller who flushes L2 first (and times reps = 1) gets a cold launch */
/* Times `reps` back-to-back launches of one kernel of the V-cycle on `level` (operands: the
 * level's own work buffers, zero-filled first) between two CUDA events recorded on `stream`,
 * and returns the mean device time of one launch (*ms) and the algorithmic DRAM bytes one
 * launch must move (*bytes: every operand word read once and every result word written once;
 * IB data counted only in IB-active tiles; for SIB_KERNEL_IB_WINDOW the bytes of the IB operator
 * applied through the markers, 15 words per marker and 2 words per face of a tile that a marker
 * stencil touches).  Synchronises `stream`.  Requires sib_setup. */
int sib_time_kernel(sib_ctx* ctx, int kernel, int level, int prec, int reps, void* stream, double* ms,
                    double* bytes);

/* ---- spreading without device allocation ----------------------------------------------------- */
/* f = S F on an N x N grid for markers X (M x 2) and forces F (M x 2), written to the caller's
 * f (2 N^2 values [f_u | f_v]); the same result as sib_spread without a solver context.
 * The paper has no counterpart: this is for callers that cannot allocate device memory, such as
 * programs whose device memory is owned by their own pool allocator (a raw cudaMalloc would fail
 * or fragment it) and latency-critical loops that cannot afford the device-wide synchronisation
 * of cudaMalloc/cudaFree.  It calls no cudaMalloc, cudaFree or allocating library routine; its
 * scratch is one static device array of about 4.4 MB that every GPU loading the library holds
 * until exit.
 *   Limits: N a power of two, 8 <= N <= 256; 0 <= M <= 16384.  Larger sizes return
 *   SIB_ERR_TOO_LARGE; other invalid arguments return SIB_ERR_ARG.
 *   Each call outside stream capture looks up the scratch array's device address on the current
 *   device; a call made while `stream` is being captured reuses the address found by the last
 *   uncaptured call on that device.  So make one call on each device before any capture, and one
 *   again after a cudaDeviceReset; a captured call on a device with no earlier call returns
 *   SIB_ERR_STATE.
 *   All calls share the one scratch array: calls that overlap on the GPU (other streams, other
 *   host threads) race and must be serialised by the caller. */
int sib_spread_noalloc(int N, int M, const double* X, const double* F, double* f, void* stream);

/* ---- accounting ---------------------------------------------------------------------------- */
/* Number of kernels this context has launched (graph replays count every kernel node). */
int64_t sib_launch_count(const sib_ctx* ctx);
/* Bytes of device memory this context holds. */
int64_t sib_device_bytes(const sib_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SIB_H */
