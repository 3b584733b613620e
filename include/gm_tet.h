/*
 * gm_tet.h - operators of the paper's own discretisation on unstructured
 * meshes: linear (P1) tetrahedra for displacement and pressure (Sec. 3.1:
 * linear shape functions on tetrahedra for both fields), used for Cryer's
 * sphere (Sec. 4.1), and a fault of duplicated nodes with interface elements
 * on its triangles (Sec. 3.1.1-3.1.2) stepped by Newton (Sec. 3.3.1).
 *
 * Conventions are those of gm.h (status codes, *_host / *_dev pointers,
 * stream as void*, field-major vectors: u as [ux | uy | uz] of 3*N values,
 * p as N values, coupled as 4*N).  The operators are the assembled ones,
 * with no Dirichlet masking: callers constrain rows themselves.
 */
#ifndef GM_TET_H
#define GM_TET_H

#include <stdint.h>

#include "gm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gm_tet gm_tet;

/* Create / destroy a tetrahedral-mesh context on `device`. */
int gm_tet_create(gm_tet** out, int device);
int gm_tet_destroy(gm_tet* t);

/* Last error message of the context. */
const char* gm_tet_last_error(const gm_tet* t);

/* Mesh: nodes_host holds 3*n_nodes coordinates, point-major (x0 y0 z0 x1 ...);
 * tets_host holds 4*n_tets vertex ids in [0, n_nodes).  Element gradients and
 * volumes are computed here (FP64, FP32 copy); the node-to-element incidence
 * is stored so that each node gathers its elements in a fixed order
 * (deterministic results).  GM_EINVAL for ids out of range, a degenerate
 * tetrahedron, or sizes beyond 2^27 nodes or tetrahedra.  Synchronises. */
int gm_tet_mesh(gm_tet* t, const double* nodes_host, int64_t n_nodes, const int64_t* tets_host,
                int64_t n_tets);

/* Homogeneous materials (Sec. 2.1): Young's modulus E, Poisson ratio nu, Biot
 * coefficient alpha, Biot modulus M, permeability k, fluid viscosity mu_f. */
int gm_tet_materials(gm_tet* t, double E, double nu, double alpha, double M, double k, double mu_f);

/* y = A x for `which` in GM_OP_KB (= GM_OP_KT: no fault), GM_OP_APU, GM_OP_AUP,
 * GM_OP_A22 (S + dt C) and GM_OP_J ([K, -A_pu; A_pu^T, S + dt C]); element
 * operators as in Sec. 3.2 with exact integration on P1 tetrahedra:
 * K_e = V B^T D B, A_e = alpha (V/4) B^T m 1^T, S_e = (V/20M)(1 + delta),
 * C_e = (k/mu) V G G^T.  x_dev, y_dev of `dtype` with the lengths of gm.h's
 * operator list. */
int gm_tet_apply(gm_tet* t, int which, const void* x_dev, void* y_dev, double dt, int dtype,
                 void* stream);

/* Dirichlet constraints for gm_tet_step: 4*N bytes, fixed[c*N + n] = 1 sets
 * component c (ux, uy, uz, p) of node n to zero (homogeneous). */
int gm_tet_dirichlet(gm_tet* t, const uint8_t* fixed_host, int64_t n);

/* Nodal forces of a compressive normal traction sigma0 on surface triangles
 * (3*n_tris vertex ids; the vertex order gives the outward side by the right-
 * hand rule): -sigma0 (A/3) n at each vertex of each triangle, replacing the
 * previous forces.  Used by gm_tet_step. */
int gm_tet_surface_load(gm_tet* t, const int64_t* tris_host, int64_t n_tris, double sigma0);

/* One backward-Euler step of the fault-free poroelastic problem (Sec. 3.3):
 * K u - A p = f,  A^T (u - u_n) + S (p - p_n) + dt C p = 0, with the
 * Dirichlet constraints and loads above.  u_dev (3N) and p_dev (N) hold the
 * previous state on entry and the new one on return (constrained entries 0).
 * Solved by Prevost's partitioned CG (Sec. 3.3.2): CG on the Schur complement
 * (S + dt C) + A^T K^-1 A, preconditioned by the diagonal of S + dt C,
 * relative tolerance rtol; inner K solves by PCG with 3x3 nodal block Jacobi
 * to rtol/100, their scalars kept on the device.  FP64.  report: outer iterations and final relative residual.
 * GM_ENOCONV if an iteration limit (maxit) is reached.  Synchronises. */
int gm_tet_step(gm_tet* t, double dt, double* u_dev, double* p_dev, double rtol, int maxit,
                gm_solve_report* report_host, void* stream);

/* ---- Fault on the tetrahedral mesh (Sec. 3.1.1-3.1.2: interface elements on
 * the triangles of the fault surface) ------------------------------------- */

/* One planar fault of duplicated nodes.  pairs_host holds 2*n_pairs node ids,
 * the minus lips first (pairs_host[i]) then the plus lips (pairs_host[P + i]);
 * a node belongs to at most one pair, and no tetrahedron holds both lips of a
 * pair.  tris_host holds 3*n_tris pair ids, one triangle of the fault surface
 * each, ordered so that the right-hand-rule normal points from the minus to
 * the plus lip.  t1_ref_host (3 values) is the direction whose projection on
 * the fault gives the first tangent t1 (tau0 is given in t1, t2 = n x t1).
 * Computed here from the minus-lip coordinates: the tributary area A_i = sum
 * of area/3 over the pair's triangles (nodal quadrature), the normal = the
 * normalised area-weighted sum of its triangles' normals, and each triangle's
 * longitudinal Laplacian.  k_perp <= 0 ties the two lip pressures (the plus
 * lip's pressure then equals the minus lip's and carries no equation).
 * Resets the fault history (inelastic slip 0).  GM_EINVAL for ids out of
 * range, a node in two pairs, a degenerate triangle, a pair on no triangle,
 * t1_ref normal to the fault, or more than 2^27 triangles.  Synchronises. */
int gm_tet_fault(gm_tet* t, const int64_t* pairs_host, int64_t n_pairs, const int64_t* tris_host,
                 int64_t n_tris, const double* t1_ref_host, const gm_fault_params* params_host);

/* Nodal loads for gm_tet_fault_step: f^u (3*N forces [N]) and f^p (N fluid
 * sources [m^3/s]); either may be NULL (zero).  Replaces the forces of
 * gm_tet_surface_load.  A source on a tied plus-lip node is added to its
 * minus-lip partner. */
int gm_tet_loads(gm_tet* t, const double* fu_host, const double* fp_host);

/* y = A x with the fault terms (Sec. 3.2.3 and App. B: A^f_pu, its transpose
 * A^f_up, fracture storage, longitudinal and transverse flow), FP64, for
 * which = GM_OP_KT (bulk K plus the cohesive tangent of the last return map,
 * Sec. 3.3.1; zero before the first step),
 * GM_OP_APU, GM_OP_AUP or GM_OP_A22 (S + dt C with fault storage, the
 * triangles' longitudinal flow and, untied, the transverse term).  Pressure
 * vectors live in the tied space: the plus-lip entry of a tied pair is an
 * unknown of no equation, ignored on input and 0 on output.  Constrained
 * entries of x are ignored and those of y are 0. */
int gm_tet_fault_apply(gm_tet* t, int which, const double* x_dev, double* y_dev, double dt, void* stream);

/* One implicit step with the fault (Sec. 3.3.1): Newton on the incremental
 * residuals with the contact / Coulomb return map at every pair (Sec. 2.2.1),
 * each correction by Prevost's partitioned CG (Sec. 3.3.2) with inner K_T
 * solves by PCG preconditioned with nodal 3x3 block Jacobi off the fault and,
 * for the two lips of each pair, the inverse of their 6x6 block (bulk blocks
 * plus the cohesive tangent that couples them), and the diagonal of S + dt C
 * as the outer preconditioner.  The inner PCG keeps its scalars on the device
 * (no host round trip per dot product).
 * Stops when the fault states of two successive iterations agree and
 * rhat <= newton_rtol * max(rhat0, 1e-3 shat), with rhat the residual scaled
 * by the diagonals of K and S + dt C.  u_dev (3N) and p_dev (N) hold the
 * accepted state on entry and the new one on return (tied plus lips carry
 * their partner's pressure).  Uses newton_rtol, newton_maxit, outer_rtol,
 * outer_maxit, inner_rtol, inner_maxit and precision of opts: GM_F64, or
 * GM_F32 for inner K_T solves in FP32 (operator, preconditioner blocks and
 * vectors; the residuals, the return map and the outer CG stay FP64, and
 * Newton refines the inexact corrections to newton_rtol).  GM_ENEWTON
 * at the Newton limit, GM_ENOCONV at a CG limit; the state is then unchanged.
 * Synchronises. */
int gm_tet_fault_step(gm_tet* t, double dt, double* u_dev, double* p_dev, const gm_step_opts* opts_host,
                      gm_step_report* report_host, void* stream);

/* Fault state after the last accepted step, any pointer may be NULL:
 * flags (P: GM_OPEN / GM_STICK / GM_SLIP), slip (2P, field-major: the jump
 * [[u]] projected on t1, then on t2), inelastic slip (2P, same layout). */
int gm_tet_fault_state(gm_tet* t, int8_t* flags_host, double* slip_host, double* dlie_host);

#ifdef __cplusplus
}
#endif

#endif /* GM_TET_H */
