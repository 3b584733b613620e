/*
 * gm.h - C ABI of the GB300 library for the partitioned poro-elastic solver with
 * cohesive faults (Gallyamov et al., "A Parallelized 3D Geomechanical Solver for
 * Fluid-induced Fault Slip in Poroelastic Media").
 *
 * Conventions for every call:
 *  - Returns 0 (GM_OK) or a negative gm_status.  gm_last_error(ctx) gives text.
 *    No C++ exception crosses this boundary.
 *  - Pointers named *_host are host memory, read (or written) during the call
 *    only; the caller keeps ownership.  Pointers named *_dev are device memory
 *    on the context's GPU, borrowed for the duration of the call (kernels are
 *    enqueued on `stream`; the call returns after they are enqueued unless the
 *    description says it synchronises).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.
 *  - Grid: nx*ny*nz trilinear hexahedra on an affinely sheared structured grid.
 *    A fault is an index node plane kf (0 < kf < nz), duplicated: extended
 *    plane kf is the lower lip, kf+1 the upper lip, so the node count is
 *    N = (nx+1)(ny+1)(nz+2) with a fault, (nx+1)(ny+1)(nz+1) without.
 *    node id n = i + (nx+1)*(j + (ny+1)*kk);  element id e = ei + nx*(ej + ny*ek).
 *  - Vectors are field-major ("SoA"): a displacement vector is 3*N values
 *    [ux(0..N-1), uy(..), uz(..)], a pressure vector N values, a coupled vector
 *    4*N values [ux, uy, uz, p].  With tied lip pressures (infinite transverse
 *    permeability, Table 1) the upper-lip pressure entries are slaves of the
 *    lower-lip ones: operator outputs hold 0 there and inputs there are ignored.
 *  - Pair id of the fault node pair (i, j) is i + (nx+1)*j.
 *  - dtype: GM_F64 (double) or GM_F32 (float) for device vectors.
 */
#ifndef GM_H
#define GM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_ctx gm_ctx;

typedef enum {
    GM_OK = 0,
    GM_EINVAL = -1,      /* bad argument or call order */
    GM_ECUDA = -2,       /* a CUDA runtime call failed */
    GM_ENOMEM = -3,      /* device allocation failed */
    GM_ENOCONV = -4,     /* an iterative solve hit its iteration limit */
    GM_ENEWTON = -5,     /* Newton did not converge in its iteration limit */
    GM_ENAN = -6,        /* NaN or Inf met in a reduction */
    GM_ESTATE = -7       /* context not ready for this call (missing setup) */
} gm_status;

typedef enum { GM_F64 = 0, GM_F32 = 1 } gm_dtype;

/* Operators for gm_apply_operator (Sec. 3.3, Eq. linear_system):
 *  GM_OP_KB   bulk elasticity K_b (3N -> 3N)                      Sec. 3.2.1
 *  GM_OP_KT   tangent stiffness K_T = K_b + fault tangent (3N->3N) Sec. 3.3.1
 *  GM_OP_A22  S + dt*C, matrix and fracture flow (N -> N)          Sec. 3.2.2-3.2.3
 *  GM_OP_APU  A_pu, bulk (App. A Eq. Apdp) + fault (App. B) (N -> 3N)
 *  GM_OP_AUP  A_up = A_pu^T (App. A Eq. Adpd, App. B Eq. afdpd) (3N -> N)
 *  GM_OP_J    Jacobian [K_T, -A_pu; A_up, S + dt C] (4N -> 4N)
 * dt is the value of the last gm_set_timestep call. */
typedef enum {
    GM_OP_KB = 0, GM_OP_KT = 1, GM_OP_A22 = 2, GM_OP_APU = 3, GM_OP_AUP = 4, GM_OP_J = 5
} gm_operator;

/* Fault states, per node pair (Sec. 2.2.1). */
enum { GM_OPEN = 0, GM_STICK = 1, GM_SLIP = 2 };

/* Cohesive-fault and fracture-flow parameters (Sec. 2.2, Table 1). */
typedef struct {
    double kn;       /* normal penalty stiffness [Pa/m], Eq. normal_traction */
    double ks;       /* shear penalty stiffness [Pa/m], Eq. slip_split */
    double f;        /* friction coefficient, Eq. yield_function */
    double w0;       /* hydraulic aperture of the flow operators [m], Sec. 2.2.2 */
    double wk_par;   /* longitudinal transmissibility w*k_par [m^3], Eq. flux_decompose */
    double k_perp;   /* transverse permeability [m^2]; <= 0: infinite (tied lip pressures) */
    double MF;       /* fracture Biot modulus [Pa], Eq. fluid_content_fracture */
    double tn0;      /* in-situ effective normal traction, compression > 0 [Pa] */
    double tau0[2];  /* in-situ shear traction in the fault frame (t1, t2) [Pa] */
} gm_fault_params;

typedef struct {
    int iterations;          /* iterations performed */
    double rel_residual;     /* final ||r|| / ||r0|| */
    int status;              /* GM_OK or GM_ENOCONV / GM_ENAN */
} gm_solve_report;

typedef struct {
    double newton_rtol;      /* Newton stop: rhat <= rtol * max(rhat0, 1e-3 shat) */
    int newton_maxit;        /* Newton iteration limit */
    double outer_rtol;       /* partitioned CG relative tolerance (defaults: 1e-8 FP64, 1e-1 FP32) */
    int outer_maxit;
    double inner_rtol;       /* inner PCG relative tolerance (K_T and A22 solves; defaults: 1e-10
                                FP64, 1e-2 FP32: the Newton loop refines inexact solves) */
    int inner_maxit;
    int precision;           /* GM_F64, or GM_F32: FP32 operators + preconditioners
                                inside the FP64 Newton/refinement loop */
    int schur_precond;       /* 0: A22^-1 (Sec. 3.3.2); 1: (A22 + sum_e alpha^2/K_dr,e M_e)^-1,
                                the fixed-stress approximation of the Schur complement
                                (same solution, fewer outer iterations under strong coupling) */
} gm_step_opts;

typedef struct {
    int newton;              /* Newton iterations */
    int outer;               /* total partitioned-CG iterations */
    long long inner_k;       /* total inner PCG iterations on K_T */
    long long inner_a;       /* total inner PCG iterations on A22 */
    long long applies;       /* operator applications (bulk kernel launches) */
    double rhat;             /* final scaled residual */
    double rhat0;            /* initial scaled residual */
    int n_open, n_stick, n_slip;
    double min_yield_margin;   /* min |F| / (f t'_n) over contact pairs */
    double min_normal_margin;  /* min |t'_n0 - k_n n.[[u]]| / t'_n0 over pairs */
} gm_step_report;

/* ---- lifetime -------------------------------------------------------- */

/* Create a context on CUDA device `device`.  *ctx receives the handle. */
int gm_create(gm_ctx** ctx, int device);
/* Free all device memory held by ctx and the context itself.  NULL is a no-op. */
int gm_destroy(gm_ctx* ctx);
/* Last error message of ctx ("" if none).  Valid until the next call on ctx. */
const char* gm_last_error(const gm_ctx* ctx);
/* Library version string. */
const char* gm_version(void);

/* ---- set-up (Sec. 3.1) ----------------------------------------------- */

/* Structured grid: node (i, j, k) sits at
 *   x = origin[0] + i h[0],  y = origin[1] + j h[1],
 *   z = origin[2] + k h[2] + shear[0] * i h[0] + shear[1] * j h[1].
 * Every element is the same parallelepiped (affine map), Sec. 3.1. */
int gm_mesh_structured(gm_ctx* ctx, int nx, int ny, int nz, const double origin_host[3],
                       const double h_host[3], const double shear_host[2]);

/* Duplicate node plane kf (0 < kf < nz) into a zero-thickness cohesive fault with
 * double-node flow (Sec. 3.1.1-3.1.2).  Must precede gm_set_materials. */
int gm_fault_plane(gm_ctx* ctx, int kf, const gm_fault_params* params_host);

/* Materials (Sec. 2.1): E and k per element (n = n_el) or broadcast (n = 1);
 * nu, alpha (Biot), M (Biot modulus) uniform; mu_f fluid viscosity. */
int gm_set_materials(gm_ctx* ctx, const double* E_host, const double* k_host, int64_t n,
                     double nu, double alpha, double M, double mu_f);

/* Homogeneous Dirichlet constraints: fixed_host is 4*N bytes, field-major
 * (ux, uy, uz, p); non-zero marks a constrained dof. */
int gm_set_dirichlet(gm_ctx* ctx, const uint8_t* fixed_host, int64_t n);

/* Nodal loads: f^u (3*N, forces [N]) and f^p (N, fluid sources [m^3/s]); either
 * may be NULL (zero).  A source on a tied upper-lip node is added to its
 * lower-lip partner. */
int gm_set_loads(gm_ctx* ctx, const double* fu_host, const double* fp_host);

/* Allocate device state and work vectors, build the reference-cell operators,
 * upload materials, masks and loads, and reset the state to u = p = 0,
 * inelastic slip 0, all pairs STICK.  Matrix-free: nothing global is assembled.
 * Call after the set-up calls above and again after changing any of them. */
int gm_assemble_or_bind(gm_ctx* ctx);

/* Time-step size used by GM_OP_A22 / GM_OP_J and by diagonal preconditioners. */
int gm_set_timestep(gm_ctx* ctx, double dt);

/* ---- operators and fault law ----------------------------------------- */

/* y = P_f A P_f x on the free dofs (constrained entries of y set to 0), for the
 * operator `which` (gm_operator).  x_dev, y_dev are device vectors of type
 * `dtype` with the lengths listed at gm_operator.  GM_OP_KT and GM_OP_J use the
 * fault tangent of the last return map (gm_fault_update or a step). */
int gm_apply_operator(gm_ctx* ctx, int which, const void* x_dev, void* y_dev, int dtype,
                      void* stream);

/* Return map (Sec. 2.2.1, Eqs. normal_traction ... corrector) at every pair for
 * the total displacement u_dev (3*N doubles), using the inelastic slip of the
 * last accepted step; stores the state and tangent in the context.  Optional
 * device outputs (NULL to skip), one entry per pair:
 *   flags_dev (int8) state, tn_dev effective normal traction, ts_dev (2 per
 *   pair, field-major) shear traction, dlie_dev (2 per pair) inelastic slip,
 *   T_dev (3 per pair, field-major) incremental conjugate traction
 *   -(t'_n - t'_n0) n + (t_s - tau0).  Synchronises the stream. */
int gm_fault_update(gm_ctx* ctx, const double* u_dev, int8_t* flags_dev, double* tn_dev,
                    double* ts_dev, double* dlie_dev, double* T_dev, void* stream);

/* ---- solvers (Sec. 3.3) ---------------------------------------------- */

/* Preconditioned CG on GM_OP_KT (3x3 nodal block-Jacobi) or GM_OP_A22 (Jacobi):
 * solves A x = b from the initial guess in x_dev until ||r|| <= rtol ||r0||.
 * FP64 vectors.  Synchronises.  Returns GM_ENOCONV at maxit. */
int gm_pcg_solve(gm_ctx* ctx, int which, const double* b_dev, double* x_dev, double rtol,
                 int maxit, gm_solve_report* report_host, void* stream);

/* Prevost's partitioned CG (Sec. 3.3.2, Eq. schur_system) on the Jacobian with
 * the current fault tangent: b_dev = [b1 (3N); b2 (N)], x_dev receives
 * [x1; x2].  Outer CG on the Schur complement A22 + A_up K_T^-1 A_pu,
 * preconditioned by A22^-1 (inner PCG), inner K_T solves by PCG.  Synchronises. */
int gm_prevost_solve(gm_ctx* ctx, const double* b_dev, double* x_dev, double outer_rtol,
                     int outer_maxit, double inner_rtol, int inner_maxit,
                     gm_solve_report* report_host, void* stream);

/* Residuals of Eq. linear_system's right-hand side at the current state plus the
 * increments du_dev (3N) / dp_dev (N): b1 = f^u - K_b u - F_coh + A_pu p,
 * b2 = dt (f^p - C p) - S dp - A_up du, constrained entries 0.  Runs the return
 * map first.  b_dev receives [b1; b2] (4N doubles); *rhat_host (may be NULL)
 * the Jacobi-scaled norm.  Synchronises. */
int gm_residual(gm_ctx* ctx, const double* du_dev, const double* dp_dev, double* b_dev,
                double* rhat_host, void* stream);

/* gm_residual for callers that cannot allocate device memory during the call
 * (for example code that runs under a fixed memory pool or budget that forbids
 * cudaMalloc).  The paper has no counterpart: this is a property of the library.
 * Same arguments and results as gm_residual; the reduction scratch that
 * gm_residual keeps in the context lives instead in one library-owned device
 * array of about 1 MB (held on every GPU that loads the library until the
 * process exits), so the call allocates nothing.  Limit: at most 16,777,216
 * nodes; larger problems get GM_EINVAL before any GPU work.  Every call looks
 * up the array's device address with the context's device current (the lookup
 * allocates nothing, and a context re-created after cudaDeviceReset gets the
 * new address); the first lookup on a device may load the library's device
 * code, so make the first call on a device before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls whose
 * GPU work overlaps (other streams or contexts on the same device) race and
 * must be serialised by the caller.  Synchronises. */
int gm_residual_noalloc(gm_ctx* ctx, const double* du_dev, const double* dp_dev, double* b_dev,
                        double* rhat_host, void* stream);

/* One backward-Euler step of size dt (Sec. 3.3): Newton with the
 * elastic-predictor / plastic-corrector return map and Prevost's partitioned CG
 * for each Jacobian system; on convergence the state (u, p, inelastic slip,
 * flags) advances.  opts_host may be NULL (defaults).  Synchronises. */
int gm_partitioned_step(gm_ctx* ctx, double dt, const gm_step_opts* opts_host,
                        gm_step_report* report_host, void* stream);

/* ---- parameters and adjoint (gradients) ------------------------------- */

/* Replace the element permeabilities (n = n_el, or 1 to broadcast) without
 * resetting the state; diagonals are refreshed.  Synchronises. */
int gm_set_permeability(gm_ctx* ctx, const double* k_host, int64_t n);

/* Friction coefficient of the fault (Eq. yield_function): n = 1 sets the common
 * value, n = pair count sets one value per pair.  Takes effect at the next
 * return map.  Synchronises. */
int gm_set_friction(gm_ctx* ctx, const double* f_host, int64_t n);

/* Preconditioner of the K_T inner solves, FP32 and FP64 (the paper leaves the
 * inner solvers open, Sec. 3.3.2).  kind 0: block Jacobi, 3x3 nodal blocks and
 * 6x6 blocks for the two lips of each fault pair.  kind 1 (default): one
 * geometric multigrid V-cycle (grids halved within each fault block down to
 * about 10 cells per direction, degree-2 Chebyshev smoothing with that block
 * Jacobi, a degree-24 Chebyshev polynomial on the coarsest grid), built on
 * first use (its set-up synchronises); grids whose cell counts or fault index
 * cannot be halved keep kind 0.  The environment variables GM_MG_MIN_CELLS,
 * GM_MG_SMOOTH_DEG, GM_MG_COARSE_DEG, GM_MG_SMOOTH_LO and GM_MG_COARSE_LO,
 * read at set-up, override these choices (tuning only).  The converged solutions agree to the solver tolerances.  GM_EINVAL
 * for another kind. */
int gm_set_preconditioner(gm_ctx* ctx, int kind);

/* Per-pair in-situ fault tractions, for in-situ stress that varies over the
 * fault (depth gradients, Sec. 5): tn0_host[i] is the effective normal
 * traction t'_n0 of pair i (compression > 0) and tau0_host the shear traction
 * in the fault frame, field-major (tau0_1 of all pairs, then tau0_2); n is the
 * pair count.  They replace the uniform tn0, tau0 of gm_fault_plane in the
 * return map (Sec. 2.2.1: the in-situ tractions are the offsets of the
 * elastic predictor) and in the Newton test's scale; both NULL restores the
 * uniform values.  Valid after gm_assemble_or_bind, which clears them.
 * GM_EINVAL for a wrong n, one NULL array or non-finite values.  Synchronises. */
int gm_set_insitu(gm_ctx* ctx, const double* tn0_host, const double* tau0_host, int64_t n);

/* Adjoint of the last converged implicit step (call it right after
 * gm_partitioned_step, before anything re-runs the return map).  For an
 * objective J(u, p) whose derivatives the caller gives as device vectors
 * dJ_du (3N), dJ_dp (N) and dJ_dslip (2 per pair, field-major: derivative with
 * respect to the slip P_t [[u]] in the fault frame) -- any may be NULL -- it
 * solves (dF/dx)^T lambda = dJ/dx with the consistent Jacobian of the step
 * (Sec. 3.3.1, fault states frozen, slipping pairs with the nonsymmetric
 * tangent) by flexible GMRES preconditioned with the partitioned CG of
 * Sec. 3.3.2, and returns dJ/dtheta = -lambda^T dF/dtheta for
 *   g_logk_dev (n_el): theta = log k_e,   g_f_dev (pairs): theta = f_i,
 *   g_logQ_host (scalar): theta = log of a common factor on the sources.
 * The state before the step is held fixed.  rtol is the relative GMRES
 * tolerance, maxit its iteration limit.  Synchronises. */
int gm_adjoint_step(gm_ctx* ctx, const double* dJ_du_dev, const double* dJ_dp_dev,
                    const double* dJ_dslip_dev, double* g_logk_dev, double* g_f_dev,
                    double* g_logQ_host, double rtol, int maxit, gm_solve_report* report_host,
                    void* stream);

/* One step of the reverse sweep of a multi-step adjoint, for objectives of
 * the state after several implicit steps, with the inelastic slip carried
 * from step to step as history (Eq. plastic_slip_increment).  The context must
 * hold this step's state: accepted u_n, p_n and the inelastic slip h_{n-1}
 * before the step (gm_set_state), its dt (gm_set_timestep), and the return
 * map at u_n (gm_fault_update).  Inputs from the later step n+1 (all NULL at
 * the last step): lam_next_dev (4N) its adjoint, mu_next_dev (2 per pair) its
 * history adjoint, frozen_next_dev (6 per pair) its frozen pair data.  Direct
 * objective terms dJ_* as in gm_adjoint_step (usually only at the last step).
 * Outputs: lam_dev (4N), mu_dev (2 per pair), frozen_dev (6 per pair) for the
 * earlier step, and this step's gradient contributions g_logk_dev, g_f_dev,
 * g_logQ_host (overwritten; the caller sums over steps).  Synchronises. */
int gm_adjoint_sweep_step(gm_ctx* ctx, const double* dJ_du_dev, const double* dJ_dp_dev,
                          const double* dJ_dslip_dev, const double* lam_next_dev,
                          const double* mu_next_dev, const double* frozen_next_dev,
                          double* lam_dev, double* mu_dev, double* frozen_dev,
                          double* g_logk_dev, double* g_f_dev, double* g_logQ_host,
                          double rtol, int maxit, gm_solve_report* report_host, void* stream);

/* Options of the adjoint solves (gm_adjoint_step, gm_adjoint_sweep_step).
 * The Krylov iteration (flexible GMRES(30) on the transposed consistent
 * Jacobian) always applies the operator in FP64; its preconditioner is one
 * partitioned solve (Sec. 3.3.2) of the symmetric Newton system, inexact by
 * design.  precision: GM_F64 (default) or GM_F32 for the preconditioner's
 * inner operators; prec_rtol: relative tolerance of that solve (default 1e-8;
 * values in (0, 1)); schur_precond: 0 or 1 as in gm_step_opts.  Returns
 * GM_EINVAL for values out of range; the previous options are kept then. */
int gm_set_adjoint_options(gm_ctx* ctx, int precision, double prec_rtol, int schur_precond);

/* ---- state I/O (checkpoint / resume) --------------------------------- */

/* Copy the accepted state to host arrays (any may be NULL): u (3N), p (N, tied
 * slaves filled with their partner's value), slip (2 per pair, field-major:
 * P_t [[u]] in the fault frame, relative to the pre-injection state), dlie
 * (2 per pair), flags (1 byte per pair).  Synchronises. */
int gm_get_state(gm_ctx* ctx, double* u_host, double* p_host, double* slip_host,
                 double* dlie_host, int8_t* flags_host);

/* Overwrite the accepted state from host arrays (NULL leaves a field unchanged). */
int gm_set_state(gm_ctx* ctx, const double* u_host, const double* p_host,
                 const double* dlie_host, const int8_t* flags_host);

/* Device pointers of the accepted state (u: 3N doubles, p: N doubles), valid
 * until gm_assemble_or_bind or gm_destroy. */
int gm_state_device(gm_ctx* ctx, double** u_dev, double** p_dev);

/* Number of nodes, elements and fault pairs of the bound problem. */
int gm_sizes(const gm_ctx* ctx, int64_t* n_nodes, int64_t* n_el, int64_t* n_pairs);

/* Counters since gm_assemble_or_bind: kernels launched by the library and bulk
 * operator applications (any may be NULL). */
int gm_counters(const gm_ctx* ctx, int64_t* kernel_launches, int64_t* bulk_applies);

#ifdef __cplusplus
}
#endif

#endif /* GM_H */
