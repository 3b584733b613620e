// Internal declarations shared by the translation units of libgm.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gm.h"

// ---------------------------------------------------------------------------
// Operator block selection for the matrix-free applies
// ---------------------------------------------------------------------------
enum : int {
    GM_M_K = 1,      // bulk elasticity K_b
    GM_M_APU = 2,    // pressure -> force coupling A_pu (bulk + fault lips)
    GM_M_AUP = 4,    // displacement -> fluid-volume coupling A_up = A_pu^T
    GM_M_S = 8,      // storage S (bulk consistent mass / M, fault w/M_F)
    GM_M_C = 16,     // conductivity C (bulk k/mu, fault longitudinal + transverse)
    GM_M_KF = 32     // fault tangent (cohesive stiffness)
};
// Modes used by the solvers (bit sets of the above)
enum : int {
    GM_MODE_K = GM_M_K,                                         // K_b
    GM_MODE_KT = GM_M_K | GM_M_KF,                              // K_T
    GM_MODE_A22 = GM_M_S | GM_M_C,                              // S + dt C
    GM_MODE_APU = GM_M_APU,
    GM_MODE_AUP = GM_M_AUP,
    GM_MODE_J = GM_M_K | GM_M_KF | GM_M_APU | GM_M_AUP | GM_M_S | GM_M_C,
    GM_MODE_RES1 = GM_M_K | GM_M_APU | GM_M_C,                  // K_b u - A_pu p, dt C p
    GM_MODE_RES2 = GM_M_AUP | GM_M_S                            // A_up du + S dp
};

// ---------------------------------------------------------------------------
// Reference-cell operators in the parity (Walsh-Hadamard) basis
//
// The 8 nodal values of a field on a cell are replaced by their parity modes
// x_s = sum_a (-1)^popc(s & a) v_a (node a = ax + 2 ay + 4 az, s = sx + 2 sy +
// 4 sz).  In the trilinear space the modes are the monomials 1, xi_x, xi_y,
// xi_x xi_y, ... and the derivative along reference axis d maps mode s (with
// bit d set) to mode s ^ e_d; 2x2x2 Gauss quadrature keeps distinct modes
// orthogonal.  An entry between modes s and s2 of the element operators can
// therefore be nonzero only if there are reference directions d (a bit of s)
// and d2 (a bit of s2) with s ^ e_d == s2 ^ e_d2, and if the physical
// coefficient that couples (field c, derivative d) with (field c2, derivative
// d2) can be nonzero.  For the affine cell
//   X = (h0 xi0, h1 xi1, h2 xi2 + s0 h0 xi0 + s1 h1 xi1)
// reference derivative d feeds physical derivative i when d == i or when
// d = z and the shear s0 (i = x) or s1 (i = y) is nonzero.  The tables below
// list every entry this rule allows; the host checks at bind that all other
// entries of the actual operators vanish (else the bind fails), and the
// kernels multiply only the allowed entries.  K (elasticity) has 45 / 73 / 109
// allowed entries for a box / a cell sheared in x-z / a general cell, against
// 576 dense; A (Biot) 12 / 16 / 20; M (storage) is diagonal; L (Darcy)
// 7 / 11 / 15.
// ---------------------------------------------------------------------------

// Symmetry classes of the affine cell.
enum : int { GM_CLS_BOX = 0, GM_CLS_MONO = 1, GM_CLS_GEN = 2 };

__host__ __device__ constexpr int gm_popc3(int s) { return (s & 1) + ((s >> 1) & 1) + ((s >> 2) & 1); }

// reference derivative d contributes to physical derivative i
__host__ __device__ constexpr bool gm_jac_feeds(int cls, int d, int i)
{
    return d == i || (d == 2 && ((i == 0 && cls != GM_CLS_BOX) || (i == 1 && cls == GM_CLS_GEN)));
}

// isotropic elasticity couples (field c, reference derivative d) with
// (field c2, reference derivative d2): lambda div u div v + mu (grad u + grad u^T) : grad v
__host__ __device__ constexpr bool gm_elastic_couples(int cls, int c, int d, int c2, int d2)
{
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            if (gm_jac_feeds(cls, d, i) && gm_jac_feeds(cls, d2, k) &&
                ((c == i && c2 == k) || (c == c2 && i == k) || (c == k && c2 == i)))
                return true;
    return false;
}

__host__ __device__ constexpr bool gm_shares_mode(int s, int d, int s2, int d2)
{
    return ((s >> d) & 1) && ((s2 >> d2) & 1) && ((s ^ (1 << d)) == (s2 ^ (1 << d2)));
}

__host__ __device__ constexpr bool gm_kpat(int cls, int c, int s, int c2, int s2)
{
    for (int d = 0; d < 3; ++d)
        for (int d2 = 0; d2 < 3; ++d2)
            if (gm_shares_mode(s, d, s2, d2) && gm_elastic_couples(cls, c, d, c2, d2)) return true;
    return false;
}

// A_pu: divergence of u (physical derivative c of field c) against pressure mode s2
__host__ __device__ constexpr bool gm_apat(int cls, int c, int s, int s2)
{
    for (int d = 0; d < 3; ++d)
        if (((s >> d) & 1) && (s ^ (1 << d)) == s2 && gm_jac_feeds(cls, d, c)) return true;
    return false;
}

__host__ __device__ constexpr bool gm_lpat(int cls, int s, int s2)
{
    for (int d = 0; d < 3; ++d)
        for (int d2 = 0; d2 < 3; ++d2)
            if (gm_shares_mode(s, d, s2, d2))
                for (int i = 0; i < 3; ++i)
                    if (gm_jac_feeds(cls, d, i) && gm_jac_feeds(cls, d2, i)) return true;
    return false;
}

// Packed positions of the allowed entries (row-major), -1 elsewhere.  Rows and
// columns are indexed c * 8 + s for displacement modes and s for pressure modes.
struct ParPat {
    int nk, na, nl;
    signed char k[24][24];
    signed char a[24][8];
    signed char l[8][8];
};

__host__ __device__ constexpr ParPat gm_make_parpat(int cls)
{
    ParPat t{};
    t.nk = t.na = t.nl = 0;
    for (int i = 0; i < 24; ++i) {
        for (int j = 0; j < 24; ++j)
            t.k[i][j] = gm_kpat(cls, i / 8, i % 8, j / 8, j % 8) ? (signed char)(t.nk++) : (signed char)-1;
        for (int j = 0; j < 8; ++j)
            t.a[i][j] = gm_apat(cls, i / 8, i % 8, j) ? (signed char)(t.na++) : (signed char)-1;
    }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) t.l[i][j] = gm_lpat(cls, i, j) ? (signed char)(t.nl++) : (signed char)-1;
    return t;
}

constexpr int GM_PP_MAXK = 112, GM_PP_MAXA = 24, GM_PP_MAXL = 16;
static_assert(gm_make_parpat(GM_CLS_BOX).nk == 45 && gm_make_parpat(GM_CLS_MONO).nk == 73 &&
              gm_make_parpat(GM_CLS_GEN).nk == 109, "elasticity pattern sizes");
static_assert(gm_make_parpat(GM_CLS_GEN).nk <= GM_PP_MAXK && gm_make_parpat(GM_CLS_GEN).na <= GM_PP_MAXA &&
              gm_make_parpat(GM_CLS_GEN).nl <= GM_PP_MAXL, "packed operator sizes");

// Allowed entries of the reference operators (E = 1, alpha = 1, 1/M = 1,
// k/mu = 1), packed in the order of gm_make_parpat(cls); the 1/64 of the
// inverse transform is folded in.  M holds the diagonal.
template <typename T>
struct RefOps {
    T K[GM_PP_MAXK];
    T A[GM_PP_MAXA];
    T M[8];
    T L[GM_PP_MAXL];
};

// The FP32 pattern entries, each duplicated as a pair (lo, hi) so that one
// packed instruction of the FP32 bulk kernel applies it to two elements.
struct RefPairs32 {
    float2 K[GM_PP_MAXK];
    float2 M[8];
    float2 L[GM_PP_MAXL];
};

// Per-node mask bits: 1,2,4 = ux,uy,uz fixed, 8 = p fixed.
// Tied upper-lip pressures are slaves (handled by index, not by this mask).

// ---------------------------------------------------------------------------
// Kernel argument blocks
// ---------------------------------------------------------------------------
struct PcgScalars {
    double rz, pq, alpha, beta, rr, rr0, tol2, pad;
    int it, done, status, pad2;
};

struct GridDesc {
    int nx, ny, nz, nplanes;
    int kf;          // lower-lip extended plane, -1 without fault
    int tied;        // 1: upper-lip pressures slaved to lower lip
    long long N;     // nodes
    long long nb;    // nodes per plane
};

template <typename T>
struct BulkArgs {
    GridDesc g;
    int zchunk;
    const T* xu;     // 3N (or null)
    const T* xp;     // N  (or null)
    T* yu;
    T* yp;
    const T* E;      // per element
    const T* kap;    // per element k / mu_f
    const uint8_t* mask;
    T cK, cApu, cAup, cS, cC;   // alpha and 1/M folded in by the host
    const int* skip; // if non-null and *skip != 0 the kernel returns at once
    // FP32 kernel: per (node plane, 15 x 15 tile) 1 if a node of the tile's
    // staged 17 x 17 region carries a constraint (for a tied upper lip, also of
    // the lower lip it reads); null: every tile-plane is treated as constrained
    const uint8_t* tflag;
    // PCG mode: input p = z + beta * x (x = p_old), p written to p*_new,
    // per-CTA partial of p.(A p) over non-lip nodes written to part[cta]
    const T* zu;
    const T* zp;
    T* pu_new;
    T* pp_new;
    const double* beta;
    double* part;
    // optional per-element extra storage coefficient (fixed-stress term): the
    // storage block uses cS + cFS * fs[e] instead of cS when fs is non-null
    const T* fs;
    T cFS;
};

template <typename T>
struct FaultArgs {
    GridDesc g;
    const T* xu;
    const T* xp;
    T* yu;
    T* yp;
    const T* D;      // 6 per pair, field-major: D00 D01 D02 D11 D12 D22
    const uint8_t* mask;
    T cKf, cApu, cAup, cS, cC;
    T Aq;            // area of one fault quad
    T n[3];          // unit normal, lower -> upper lip
    T stor;          // w0 / M_F
    T lcoef;         // wk_par / mu_f
    T tcoef;         // k_perp / (mu_f w0)
    T Lf[16];        // reference quad Laplacian (coefficient 1)
    const int* skip;
    // PCG mode: add p.(A p) over the lip nodes to the bulk partials and let the
    // last block form p.Ap and alpha = (r.z)/(p.Ap) in *sc
    double* part;        // bulk partials at [0, nbulk), this kernel's at [nbulk, ...)
    int nbulk;
    unsigned* counter;
    PcgScalars* sc;
    // consistent-tangent term of slipping pairs, coef * tau n^T with
    // tauc = (tau_x, tau_y, tau_z, coef) per pair (field-major, 4P):
    // cons 0 ignores it, 1 adds it, 2 adds its transpose coef * n tau^T
    const double* tauc;
    int cons;
};

struct LawArgs {
    GridDesc g;
    const double* un;        // accepted displacement (3N)
    const double* du;        // increment (3N) or null
    const double* dlie_prev; // 2P
    const double* fpair;     // per-pair friction or null
    const double* insitu;    // per-pair t'_n0, tau0_1, tau0_2 (3P, field-major) or null
    double kn, ks, f, tn0, tau0[2];
    double n[3], t1[3], t2[3];
    double Aq;
    int8_t* state;
    double* tn;
    double* ts;              // 2P
    double* dlie;            // 2P
    double* T;               // 3P (incremental conjugate traction)
    double* F;               // P (trial yield value)
    double* dn;              // P (n.[[u]])
    double* gs;              // 2P (P_t [[u]] in the fault frame)
    double* D64;             // 6P
    float* D32;              // 6P (or null)
    double* tauc;            // 4P: slip direction and -f k_n (0 unless slipping)
};


// Inputs of the Newton residual (RHS of Eq. linear_system, Sec. 3.3.1) shared by
// gm_residual and gm_residual_noalloc.
struct ResidualInputs {
    GridDesc g;
    double dt, Aq;
    const double* fu;     // 3N loads
    const double* fp;     // N sources
    const double* y1u;    // 3N: K_b u - A_pu p
    const double* y1p;    // N: dt C p
    const double* y2p;    // N: A_up du + S dp
    const double* ut;     // 3N total displacement
    const double* pt;     // N total pressure
    const double* T;      // 3P incremental cohesive traction
    const double* dK;     // 3N diag(K_b)
    const double* dA;     // N diag(A22)
    const uint8_t* mask;
    double* b;            // 4N output
};

// Residual of node n written to b (0 on constrained and tied-slave dofs);
// v[0] += its terms of sum b1^2/diag(K_b) + sum b2^2/diag(A22), v[1] += its
// terms of sum diag(K_b) u^2 + sum diag(A22) p^2.
__device__ __forceinline__ void gm_residual_node(const ResidualInputs& a, long long n, double (&v)[2])
{
    const long long N = a.g.N;
    const unsigned m = a.mask[n];
    const long long kk = n / a.g.nb;
    const long long pid = n - kk * a.g.nb;
    double lipsign = 0.0;
    if (a.g.kf >= 0) {
        if (kk == a.g.kf) lipsign = -1.0;
        else if (kk == a.g.kf + 1) lipsign = 1.0;
    }
    double Ai = 0.0;
    if (lipsign != 0.0) {
        const int pi = (int)(pid % (a.g.nx + 1)), pj = (int)(pid / (a.g.nx + 1));
        const int nqi = (pi > 0) + (pi < a.g.nx), nqj = (pj > 0) + (pj < a.g.ny);
        Ai = a.Aq * 0.25 * nqi * nqj;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double r = 0.0;
        if (!((m >> c) & 1u)) {
            r = a.fu[c * N + n] - a.y1u[c * N + n];
            if (lipsign != 0.0) r -= lipsign * Ai * a.T[c * a.g.nb + pid];
            const double d = a.dK[c * N + n];
            v[0] += r * r / d;
            const double u = a.ut[c * N + n];
            v[1] += d * u * u;
        }
        a.b[c * N + n] = r;
    }
    const bool slave = a.g.tied && kk == a.g.kf + 1;
    double r = 0.0;
    if (!slave && !((m >> 3) & 1u)) {
        r = a.dt * a.fp[n] - a.y1p[n] - a.y2p[n];
        const double d = a.dA[n];
        v[0] += r * r / d;
        const double p = a.pt[n];
        v[1] += d * p * p;
    }
    a.b[3 * N + n] = r;
}

// ---------------------------------------------------------------------------
// Device buffer
// ---------------------------------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t bytes) {
        release();
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) n = bytes;
        else p = nullptr;
        return e;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct gm_ctx;

// One level of the geometric multigrid hierarchy of the K_T inner solves.
// Level 0 is the context itself (b = PCG residual, x = preconditioned
// residual); coarser levels are child contexts on grids halved within each
// fault block, owning their vectors.
struct MGLevel {
    gm_ctx* cx = nullptr;
    float* b = nullptr;
    float* x = nullptr;
    float* d = nullptr;      // Chebyshev direction
    float* y = nullptr;      // operator output
    double* b64 = nullptr;   // the same vectors for FP64 solves
    double* x64 = nullptr;
    double* d64 = nullptr;
    double* y64 = nullptr;
    double lmax = 0.0;       // largest eigenvalue estimate of M^-1 K_T
    int deg = 2;             // Chebyshev degree of the smoother (of the solve on the coarsest level)
    int coef_off = 0;        // first (c1, c2) pair of this level in mg_coef
};

struct gm_ctx {
    int device = 0;
    std::string err;
    int sm_count = 152;

    // set-up
    bool has_mesh = false, has_fault = false, has_mat = false, bound = false;
    int nx = 0, ny = 0, nz = 0;
    double origin[3] = {0, 0, 0}, h[3] = {1, 1, 1}, shear[2] = {0, 0};
    int kf_orig = -1;
    gm_fault_params fp{};
    std::vector<double> E, kperm;
    double nu = 0.25, alpha = 1.0, M = 1.0, mu_f = 1.0;
    std::vector<uint8_t> fixed;   // 4N
    std::vector<double> fu, fpv;  // 3N, N

    // derived
    GridDesc g{};
    long long N = 0, n_el = 0, P = 0;
    int cls = GM_CLS_BOX;
    RefOps<double> R64{};
    RefOps<float> R32{};
    RefPairs32 R32p{};
    double Kblk_ref[8][9] = {};   // nodal 3x3 diagonal blocks of K_ref (E = 1)
    double Mdiag_ref[8] = {}, Ldiag_ref[8] = {};
    double Aq = 0, nrm[3] = {0, 0, 1}, t1[3] = {1, 0, 0}, t2[3] = {0, 1, 0};
    double Lf[16] = {};
    double dt = 1.0;
    double f0sq = 0.0;            // sum F0^2 / diag(K_b) over free lip dofs

    // device data
    DevBuf dE64, dK64, dE32, dK32, dmask, dfu, dfp;
    DevBuf du_n, dp_n, ddlie_n, dflags_n;              // accepted state
    DevBuf dstate, dtn, dts, ddlie, dT, dF, ddn, dgs, dD64, dD32;   // fault work
    DevBuf dtauc, dfpair;                              // consistent-tangent term, per-pair f
    bool has_fpair = false;
    DevBuf dinsitu;                                    // per-pair in-situ tractions (3P)
    bool has_insitu = false;
    std::vector<double> h_insitu;                      // host copy (3P)
    int fault_cons = 0;                                // tangent variant used by the fault kernel
    double Lref[64] = {};                              // nodal L of the reference cell (k/mu = 1)
    DevBuf adj_V, adj_Z, adj_w, adj_b, adj_x, adj_t;   // adjoint (FGMRES) work, allocated on first use
    DevBuf adj_s, adj_u;                               // row scaling of the adjoint system, scratch
    int adj_m = 0;
    int adj_prec = 0;            // preconditioner precision (GM_F64 / GM_F32)
    double adj_prtol = 1e-8;     // preconditioner tolerance
    int adj_schur = 0;           // preconditioner's Schur preconditioner
    DevBuf ddiagK, ddiagA, dKinv64, dKinv32, dAinv64, dAinv32;
    DevBuf dKinv16;                                    // 6N bf16 copy of the nodal block inverses (multigrid smoother)
    DevBuf dKpair64, dKpair32;                         // 6x6 inverse blocks of the lip pairs (36 per pair)
    bool pair_prec = true;                             // K_T preconditioner: lip pairs as 6x6 blocks
    int precond = 1;                                   // FP32 K_T solves: 0 block Jacobi, 1 multigrid
    std::vector<MGLevel> mg;                           // built on first use
    DevBuf mg_d0, mg_y0, mg_coef;                      // level-0 smoother vectors, Chebyshev coefficients
    DevBuf mg_d0_64, mg_y0_64;                         // level-0 smoother vectors of FP64 solves
    DevBuf dFS64, dFS32, dAfsinv64, dAfsinv32;         // fixed-stress storage term
    DevBuf dscal;                                      // PcgScalars[4] + misc
    DevBuf dpart;                                      // reduction partials
    DevBuf dtflag;                                     // constrained tile-planes of the FP32 bulk kernel
    DevBuf dcount;                                     // last-block counters
    // work vectors (FP64)
    DevBuf w_du, w_dp, w_ut, w_pt, w_b, w_x, w_y1u, w_y1p, w_y2u, w_y2p;
    DevBuf k_r, k_z, k_p, k_p2, k_q, a_r, a_z, a_p, a_p2, a_q;     // inner PCG (FP64)
    DevBuf k_x64, a_x64;                               // FP64 PCG corrections
    DevBuf k_r32, k_z32, k_p32, k_pb32, k_q32, k_x32, k_b32;      // inner PCG (FP32)
    DevBuf a_r32, a_z32, a_p32, a_pb32, a_q32, a_x32, a_b32;
    int bulk_grid = 0;                                 // CTAs of one bulk apply
    int zchunk_override = 0;                           // GM_BULK_ZCHUNK (tuning), 0 = heuristic
    DevBuf o_y1, o_w, o_x1, o_t3, o_r, o_z, o_zold, o_p, o_q, o_x2, o_t1;   // outer CG
    DevBuf o_s32a, o_s32b;                             // FP32 operands / products of the outer CG (3N each)
    DevBuf dprevstate;
    void* hpin = nullptr;                              // pinned host scratch (4 KB)
    // CUDA graphs of two fused PCG iterations, per (operator, precision);
    // captured on a private stream, replayed on the caller's stream
    cudaStream_t cap_stream = nullptr;
    // [which][0: FP64, 1: FP32, 2: FP32 with the multigrid preconditioner, 3: FP64 with it]
    cudaGraphExec_t pcg_graph[3][4] = {};
    double pcg_graph_dt[3][4] = {};
    int pcg_graph_maxit[3][4] = {};
    long long pcg_graph_launches[3][4] = {};
    bool use_graphs = true;
    void drop_graphs() {
        for (auto& row : pcg_graph)
            for (auto& gph : row)
                if (gph) { cudaGraphExecDestroy(gph); gph = nullptr; }
    }
    long long applies = 0;                             // bulk apply launches
    long long launches = 0;                            // all kernel launches

    int set_err(int code, const std::string& msg) {
        err = msg;
        return code;
    }
};

// Count one kernel launch and check it.
#define GM_LAUNCHED(ctx)                                                              \
    do {                                                                              \
        (ctx)->launches++;                                                            \
        cudaError_t _e = cudaGetLastError();                                          \
        if (_e != cudaSuccess)                                                        \
            return (ctx)->set_err(GM_ECUDA, std::string("launch: ") + cudaGetErrorString(_e)); \
    } while (0)

#define GM_CUDA_TRY(ctx, call)                                                        \
    do {                                                                              \
        cudaError_t _e = (call);                                                      \
        if (_e != cudaSuccess)                                                        \
            return (ctx)->set_err(GM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// Matrix-free operator application: bulk kernel then fault kernel.
int gm_launch_apply_f64(gm_ctx* c, int mode, double cK, double cApu, double cAup, double cS,
                        double cC, const double* xu, const double* xp, double* yu, double* yp,
                        cudaStream_t s, const int* skip);
int gm_launch_apply_f32(gm_ctx* c, int mode, double cK, double cApu, double cAup, double cS,
                        double cC, const float* xu, const float* xp, float* yu, float* yp,
                        cudaStream_t s, const int* skip);

// Fault law, residual, preconditioners
int gm_launch_return_map(gm_ctx* c, const double* un, const double* du, cudaStream_t s);
int gm_upload_permeability(gm_ctx* c);                 // kap arrays + diagonals from c->kperm
ResidualInputs gm_residual_inputs(const gm_ctx* c, const double* y1u, const double* y1p, const double* y2p,
                                  const double* ut, const double* pt, double* b);
int gm_launch_residual(gm_ctx* c, const double* y1u, const double* y1p, const double* y2p,
                       const double* ut, const double* pt, double* b, cudaStream_t s,
                       double* out2 /* device: rhat^2, shat^2 */);
int gm_launch_diag(gm_ctx* c, cudaStream_t s);            // dK (bulk), dA (needs dt)
int gm_launch_block_jacobi(gm_ctx* c, cudaStream_t s);    // K_T 3x3 inverse blocks
// multigrid preconditioner of the FP32 K_T solves (gm_mg.cu)
int gm_prepare_bulk32(gm_ctx* c);                     // kernel attributes, at bind
int gm_launch_bulk_k_f32(gm_ctx* c, const float* x, float* y, cudaStream_t s, const int* skip);
int gm_launch_bulk_k_f64(gm_ctx* c, const double* x, double* y, cudaStream_t s, const int* skip);
int gm_mg_prepare(gm_ctx* c, int prec, cudaStream_t s);   // GM_EINVAL: grid not coarsenable (caller falls back)
int gm_mg_vcycle(gm_ctx* c, int prec, const void* r, void* z, const int* skip, cudaStream_t s);
void gm_mg_release(gm_ctx* c);
int gm_launch_pcg_update_noz(gm_ctx* c, int prec, void* x, void* r, const void* p, const void* q,
                             PcgScalars* sc, int maxit, cudaStream_t s);
int gm_launch_pcg_rz(gm_ctx* c, int prec, const void* r, const void* z, PcgScalars* sc, int init,
                     cudaStream_t s);
int gm_launch_count_changes(gm_ctx* c, const int8_t* a, const int8_t* b, int* out, cudaStream_t s);

// Linear algebra
int gm_launch_pcg_init(gm_ctx* c, int which, int prec, const void* b, const void* q, void* r,
                       void* z, void* p, double rtol, PcgScalars* sc, cudaStream_t s);
// One fused PCG operator step: p_new = z + beta p_old, q = A p_new, and
// alpha = (r.z)/(p_new.q) into *sc (which 0: K_T, which 1: A22).
int gm_launch_pcg_apply_f64(gm_ctx* c, int which, const double* z, const double* p_old,
                            double* p_new, double* q, PcgScalars* sc, cudaStream_t s);
int gm_launch_pcg_apply_f32(gm_ctx* c, int which, const float* z, const float* p_old,
                            float* p_new, float* q, PcgScalars* sc, cudaStream_t s);
int gm_launch_pcg_update(gm_ctx* c, int which, int prec, void* x, void* r, void* z,
                         const void* p, const void* q, PcgScalars* sc, int maxit, cudaStream_t s);
// y = a*x + b*y over n doubles; z = x + y etc.
int gm_launch_axpby(gm_ctx* c, long long n, double a, const double* x, double b, double* y,
                    cudaStream_t s);
int gm_launch_copy_cast_d2f(gm_ctx* c, long long n, const double* x, float* y, cudaStream_t s);
int gm_launch_copy_cast_f2d(gm_ctx* c, long long n, const float* x, double* y, cudaStream_t s);
int gm_launch_axpy_f2d(gm_ctx* c, long long n, double a, const float* x, double* y, cudaStream_t s);
// scaled cast for the FP32 correction solves: sc (2 device doubles) receives
// x.x and the power-of-two scale 2^e; y = x / 2^e, later y_64 += 2^e x_32
int gm_launch_cast_scaled_d2f(gm_ctx* c, long long n, const double* x, float* y, double* sc,
                              cudaStream_t s);
int gm_launch_axpy_scaled_f2d(gm_ctx* c, long long n, const double* sc, const float* x, double* y,
                              cudaStream_t s);
// Deterministic dot products: out[0] = x.y (and out[1] = x2.y2 if x2) as doubles
int gm_launch_dot(gm_ctx* c, long long n, const double* x, const double* y, const double* x2,
                  const double* y2, double* out, cudaStream_t s);

// Solvers (gm_solve.cu)
// x_zero: the initial guess is zero (x is overwritten), which skips the
// initial operator application.  An inner solve that reaches maxit returns
// GM_ENOCONV with its current iterate in x.
int gm_pcg(gm_ctx* c, int which, int prec, const double* b, double* x, double rtol, int maxit,
           int* iters, double* relres, cudaStream_t s, bool x_zero = false);
int gm_prevost(gm_ctx* c, int prec, const double* b1, const double* b2, double* x1, double* x2,
               double outer_rtol, int outer_maxit, double inner_rtol, int inner_maxit,
               int* outer_it, long long* inner_k, long long* inner_a, double* relres,
               cudaStream_t s, int schur_precond = 0);

constexpr int GM_RED_BLOCKS = 608;   // fixed grid of the deterministic reductions
constexpr int GM_RED_THREADS = 256;
