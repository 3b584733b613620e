/*
 * gm_tet.h - operators of the paper's own discretisation on unstructured
 * meshes: linear (P1) tetrahedra for displacement and pressure (Sec. 3.1:
 * linear shape functions on tetrahedra for both fields), without fault
 * elements.  Used for Cryer's sphere (Sec. 4.1).
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
 * tetrahedron, or sizes beyond 2^29 nodes or tetrahedra.  Synchronises. */
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

#ifdef __cplusplus
}
#endif

#endif /* GM_TET_H */
