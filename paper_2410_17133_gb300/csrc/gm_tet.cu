// Matrix-free operators on unstructured P1 tetrahedra (include/gm_tet.h).
//
// Each element's shape-function gradients G (4 x 3, constant on the element)
// and volume V are computed once on the host.  An apply runs one thread per
// node: the node walks its incident (element, local vertex) list in a fixed
// order, recomputes that element's strain / pressure sums from the element's
// four vertices and adds the element's row for itself.  No atomics, so the
// result does not depend on scheduling.  With constant gradients the element
// rows are short closed expressions:
//   K:    y_a = V B_a^T D (sum_b B_b u_b)             (isotropic D: sigma from the strain)
//   A_pu: y_a = alpha (V/4) g_a sum_b p_b             (B_a^T m = g_a, integral of N_b = V/4)
//   A_up: y_a = alpha (V/4) div u
//   S:    y_a = (V / 20 M) (sum_b p_b + p_a)
//   C:    y_a = (k/mu) V g_a . sum_b g_b p_b
#include <algorithm>
#include <cmath>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gm_tet.h"

namespace {

enum : int { TM_K = 1, TM_APU = 2, TM_AUP = 4, TM_S = 8, TM_C = 16 };

template <typename T>
struct TetCoef {
    T lam, mu, alpha, invM, cond;
    T cK, cApu, cAup, cS, cC;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(128) gm_tet_apply_kernel(int N, const int* rowptr, const int* adj, const int* tets,
                                                           const T* G, const T* V, TetCoef<T> c, const T* xu,
                                                           const T* xp, T* yu, T* yp, const int* skip)
{
    if (skip != nullptr && *skip != 0) return;
    constexpr bool IN_U = (MODE & (TM_K | TM_AUP)) != 0;
    constexpr bool IN_P = (MODE & (TM_APU | TM_S | TM_C)) != 0;
    constexpr bool OUT_U = (MODE & (TM_K | TM_APU)) != 0;
    constexpr bool OUT_P = (MODE & (TM_AUP | TM_S | TM_C)) != 0;
    // one warp per node: lane l takes the node's incident elements l, l + 32, ...
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= N) return;                     // uniform over the warp
    const int n = (int)wid;
    T au[3] = {T(0), T(0), T(0)};
    T ap = T(0);
    for (int q = rowptr[n] + lane; q < rowptr[n + 1]; q += 32) {
        const int code = adj[q];
        const int e = code >> 2, a = code & 3;
        int v[4];
        T g[4][3];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            v[b] = tets[4 * e + b];
#pragma unroll
            for (int d = 0; d < 3; ++d) g[b][d] = G[12 * e + 3 * b + d];
        }
        const T vol = V[e];
        T exx = T(0), eyy = T(0), ezz = T(0), gyz = T(0), gxz = T(0), gxy = T(0);
        if constexpr (IN_U) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const T ux = xu[v[b]], uy = xu[N + v[b]], uz = xu[2 * N + v[b]];
                exx += g[b][0] * ux;
                eyy += g[b][1] * uy;
                ezz += g[b][2] * uz;
                gyz += g[b][2] * uy + g[b][1] * uz;
                gxz += g[b][2] * ux + g[b][0] * uz;
                gxy += g[b][1] * ux + g[b][0] * uy;
            }
        }
        T psum = T(0), gp[3] = {T(0), T(0), T(0)}, pa = T(0);
        if constexpr (IN_P) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const T pb = xp[v[b]];
                psum += pb;
#pragma unroll
                for (int d = 0; d < 3; ++d) gp[d] += g[b][d] * pb;
                if (b == a) pa = pb;
            }
        }
        const T gax = g[a][0], gay = g[a][1], gaz = g[a][2];
        if constexpr ((MODE & TM_K) != 0) {
            const T tr = exx + eyy + ezz;
            const T sxx = c.lam * tr + T(2) * c.mu * exx;
            const T syy = c.lam * tr + T(2) * c.mu * eyy;
            const T szz = c.lam * tr + T(2) * c.mu * ezz;
            const T syz = c.mu * gyz, sxz = c.mu * gxz, sxy = c.mu * gxy;
            const T s = c.cK * vol;
            au[0] += s * (gax * sxx + gaz * sxz + gay * sxy);
            au[1] += s * (gay * syy + gaz * syz + gax * sxy);
            au[2] += s * (gaz * szz + gay * syz + gax * sxz);
        }
        if constexpr ((MODE & TM_APU) != 0) {
            const T s = c.cApu * c.alpha * vol * T(0.25) * psum;
            au[0] += s * gax;
            au[1] += s * gay;
            au[2] += s * gaz;
        }
        if constexpr ((MODE & TM_AUP) != 0) ap += c.cAup * c.alpha * vol * T(0.25) * (exx + eyy + ezz);
        if constexpr ((MODE & TM_S) != 0) ap += c.cS * c.invM * vol * T(0.05) * (psum + pa);
        if constexpr ((MODE & TM_C) != 0) ap += c.cC * c.cond * vol * (gax * gp[0] + gay * gp[1] + gaz * gp[2]);
    }
    // fixed butterfly over the lanes: the same sums in the same order every call
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if constexpr (OUT_U) {
#pragma unroll
            for (int c = 0; c < 3; ++c) au[c] += __shfl_xor_sync(0xffffffffu, au[c], o);
        }
        if constexpr (OUT_P) ap += __shfl_xor_sync(0xffffffffu, ap, o);
    }
    if (lane != 0) return;
    if constexpr (OUT_U) {
        yu[n] = au[0];
        yu[N + n] = au[1];
        yu[2 * N + n] = au[2];
    }
    if constexpr (OUT_P) yp[n] = ap;
}

struct DBuf {
    void* p = nullptr;
    ~DBuf() { if (p) cudaFree(p); }
    cudaError_t put(const void* h, size_t bytes) {
        if (p) { cudaFree(p); p = nullptr; }
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e != cudaSuccess) { p = nullptr; return e; }
        return bytes ? cudaMemcpy(p, h, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    }
    cudaError_t alloc(size_t bytes) {
        if (p) { cudaFree(p); p = nullptr; }
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e != cudaSuccess) p = nullptr;
        return e;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace

#include "gm_tet_pcg.cuh"

// Largest node, tetrahedron or fault-triangle count: all device index arithmetic
// (12 gradients per element, 9 frame entries per pair, 3N field offsets) is in
// 32-bit int, which this bound keeps in range.
constexpr long long kTetMaxEntities = 1LL << 27;
static_assert(12 * kTetMaxEntities < 2147483647LL, "tet index arithmetic must fit in int");

struct gm_tet {
    int device = 0;
    std::string err;
    long long N = 0, M = 0;
    bool has_mesh = false, has_mat = false;
    double E = 0, nu = 0, alpha = 0, Mb = 0, k = 0, mu_f = 0;
    DBuf G64, G32, V64, V32, tets, rowptr, adj;
    // time stepping
    std::vector<double> hG, hV;            // element gradients and volumes (host copy)
    std::vector<double> hX;                // node coordinates (host copy, point-major)
    std::vector<int> htv;                  // element vertices (host copy)
    std::vector<uint8_t> fixed;            // 4N: constrained (ux, uy, uz, p)
    std::vector<double> fu;                // 3N nodal forces
    DBuf mask, dfu, Kinv, Sd, Cd, part;
    DBuf w[15];
    DBuf pcg_st, pcg_part;                  // device-resident PCG: state and reduction partials
    bool prec_ready = false;
    // fault: interface elements on the fault triangles
    bool has_fault = false, tied = false, fault_ready = false;
    long long P = 0, NTRI = 0;
    gm_fault_params fpar{};
    std::vector<int> hpm, hpp, hn2p;        // lips of each pair; node -> pair (-1 off the fault)
    std::vector<double> harea, hfr, hLt;    // A_i; frame (9P, n t1 t2 field-major); 9 per triangle
    std::vector<int> htri;                  // 3 pair ids per triangle
    std::vector<double> fpsrc;              // N fluid sources as given
    DBuf f_pm, f_pp, f_n2p, f_area, f_fr, f_Lt, f_tri, f_prow, f_padj;
    DBuf f_dlie_n, f_dlie, f_state, f_T, f_D, f_tn, f_F, f_dn, f_gs, f_flags_acc, f_gs_acc;
    DBuf f_Kblk, f_Kinv, f_fu, f_fpv, f_Sd, f_Cd, f_dKm, f_invdK, f_dAm, f_invdA, f_mask, f_err;
    DBuf f_Pinv;                            // 36P: inverses of the lip-pair 6x6 blocks of K_T
    DBuf f_Kinv32, f_Pinv32, f_D32;         // FP32 copies for the FP32 inner solves
    DBuf fw[25];
    DBuf fw32[5];                           // 3N floats each: x, r, z, p, q of the FP32 inner solves
    double f0sq = 0.0;
    // captured PCG iterations (0: K solves of gm_tet_step, 1 / 2: K_T solves of
    // the fault step in FP64 / FP32) and the stream they are captured on
    cudaGraphExec_t pcg_graph[3] = {nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    bool use_graphs = true;
    void drop_graphs()
    {
        for (auto& g : pcg_graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    ~gm_tet()
    {
        drop_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
    int set_err(int code, const std::string& m) { err = m; return code; }
};

extern "C" {

int gm_tet_create(gm_tet** out, int device)
{
    if (!out) return GM_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return GM_ECUDA;
    gm_tet* t = new (std::nothrow) gm_tet();
    if (!t) return GM_ENOMEM;
    t->device = device;
    *out = t;
    return GM_OK;
}

int gm_tet_destroy(gm_tet* t)
{
    if (!t) return GM_OK;
    cudaSetDevice(t->device);
    delete t;
    return GM_OK;
}

const char* gm_tet_last_error(const gm_tet* t) { return t ? t->err.c_str() : "null context"; }

int gm_tet_mesh(gm_tet* t, const double* nodes, int64_t n_nodes, const int64_t* tets, int64_t n_tets)
{
    if (!t) return GM_EINVAL;
    if (!nodes || !tets || n_nodes < 4 || n_tets < 1) return t->set_err(GM_EINVAL, "tet mesh: empty mesh");
    // the kernels index element and nodal-block arrays (12 M, 9 N entries) with 32-bit ints
    if (n_nodes > kTetMaxEntities || n_tets > kTetMaxEntities) return t->set_err(GM_EINVAL, "tet mesh: too large");
    const long long N = n_nodes, M = n_tets;
    std::vector<double> G(12 * M), V(M);
    std::vector<int> tv(4 * M);
    std::vector<int> count(N + 1, 0);
    for (long long e = 0; e < M; ++e) {
        double x[4][3];
        for (int b = 0; b < 4; ++b) {
            const int64_t id = tets[4 * e + b];
            if (id < 0 || id >= N) return t->set_err(GM_EINVAL, "tet mesh: vertex id out of range");
            tv[4 * e + b] = (int)id;
            count[id + 1]++;
            for (int d = 0; d < 3; ++d) x[b][d] = nodes[3 * id + d];
        }
        // J: rows are the edges x_b - x_0; gradients of N_b (b >= 1) are the
        // columns of J^-1, that of N_0 minus their sum
        double J[3][3];
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) J[r][d] = x[r + 1][d] - x[0][d];
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        double scale = 1.0;   // product of the three edge lengths from x_0
        for (int r = 0; r < 3; ++r) scale *= std::sqrt(J[r][0] * J[r][0] + J[r][1] * J[r][1] + J[r][2] * J[r][2]);
        if (!(std::fabs(det) > 1e-12 * scale)) return t->set_err(GM_EINVAL, "tet mesh: degenerate tetrahedron");
        double inv[3][3];   // inverse of J
        inv[0][0] = c00 / det;
        inv[1][0] = c01 / det;
        inv[2][0] = c02 / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int b = 1; b < 4; ++b) {
                G[12 * e + 3 * b + d] = inv[d][b - 1];
                s += inv[d][b - 1];
            }
            G[12 * e + d] = -s;
        }
        V[e] = std::fabs(det) / 6.0;
    }
    for (long long n = 0; n < N; ++n) count[n + 1] += count[n];
    std::vector<int> adj(4 * M), fill(count.begin(), count.end() - 1);
    for (long long e = 0; e < M; ++e)
        for (int b = 0; b < 4; ++b) adj[fill[tv[4 * e + b]]++] = (int)(4 * e + b);
    std::vector<float> G32(G.begin(), G.end()), V32(V.begin(), V.end());
    cudaSetDevice(t->device);
    cudaError_t ce;
    if ((ce = t->G64.put(G.data(), G.size() * 8)) != cudaSuccess || (ce = t->G32.put(G32.data(), G32.size() * 4)) != cudaSuccess ||
        (ce = t->V64.put(V.data(), V.size() * 8)) != cudaSuccess || (ce = t->V32.put(V32.data(), V32.size() * 4)) != cudaSuccess ||
        (ce = t->tets.put(tv.data(), tv.size() * 4)) != cudaSuccess ||
        (ce = t->rowptr.put(count.data(), count.size() * 4)) != cudaSuccess ||
        (ce = t->adj.put(adj.data(), adj.size() * 4)) != cudaSuccess)
        return t->set_err(GM_ECUDA, std::string("tet mesh: ") + cudaGetErrorString(ce));
    t->N = N;
    t->M = M;
    t->hX.assign(nodes, nodes + 3 * N);
    t->hG.swap(G);
    t->hV.swap(V);
    t->htv.swap(tv);
    t->fixed.assign(4 * N, 0);
    t->fu.assign(3 * N, 0.0);
    t->fpsrc.assign(N, 0.0);
    t->prec_ready = false;
    t->has_fault = false;
    t->fault_ready = false;
    t->has_mesh = true;
    return GM_OK;
}

int gm_tet_materials(gm_tet* t, double E, double nu, double alpha, double M, double k, double mu_f)
{
    if (!t) return GM_EINVAL;
    if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(M > 0) || !(k >= 0) || !(mu_f > 0))
        return t->set_err(GM_EINVAL, "tet materials: invalid values");
    t->E = E; t->nu = nu; t->alpha = alpha; t->Mb = M; t->k = k; t->mu_f = mu_f;
    t->has_mat = true;
    t->prec_ready = false;
    t->fault_ready = false;
    return GM_OK;
}

}  // extern "C"

namespace {

template <typename T, int MODE>
void launch(gm_tet* t, const TetCoef<T>& c, const T* xu, const T* xp, T* yu, T* yp, cudaStream_t s, const T* G,
            const T* V, const int* skip)
{
    const int N = (int)t->N;
    const unsigned blocks = (unsigned)((32LL * N + 127) / 128);   // one warp per node
    gm_tet_apply_kernel<T, MODE><<<blocks, 128, 0, s>>>(N, t->rowptr.as<int>(), t->adj.as<int>(), t->tets.as<int>(), G,
                                                        V, c, xu, xp, yu, yp, skip);
}

// skip: if non-null, the kernel does nothing while *skip != 0
template <typename T>
int apply_t(gm_tet* t, int which, const void* x, void* y, double dt, cudaStream_t s, const int* skip = nullptr)
{
    const long long N = t->N;
    TetCoef<T> c;
    const double lam = t->E * t->nu / ((1 + t->nu) * (1 - 2 * t->nu));
    c.lam = T(lam);
    c.mu = T(t->E / (2 * (1 + t->nu)));
    c.alpha = T(t->alpha);
    c.invM = T(1.0 / t->Mb);
    c.cond = T(t->k / t->mu_f);
    c.cK = T(1); c.cApu = T(1); c.cAup = T(1); c.cS = T(1); c.cC = T(dt);
    const T* G = sizeof(T) == 8 ? (const T*)t->G64.p : (const T*)t->G32.p;
    const T* V = sizeof(T) == 8 ? (const T*)t->V64.p : (const T*)t->V32.p;
    const T* xu = static_cast<const T*>(x);
    T* yu = static_cast<T*>(y);
    switch (which) {
    case GM_OP_KB:
    case GM_OP_KT: launch<T, TM_K>(t, c, xu, nullptr, yu, nullptr, s, G, V, skip); break;
    case GM_OP_APU: launch<T, TM_APU>(t, c, nullptr, xu, yu, nullptr, s, G, V, skip); break;
    case GM_OP_AUP: launch<T, TM_AUP>(t, c, xu, nullptr, nullptr, yu, s, G, V, skip); break;
    case GM_OP_A22: launch<T, TM_S | TM_C>(t, c, nullptr, xu, nullptr, yu, s, G, V, skip); break;
    case GM_OP_J:
        c.cApu = T(-1);
        launch<T, TM_K | TM_APU | TM_AUP | TM_S | TM_C>(t, c, xu, xu + 3 * N, yu, yu + 3 * N, s, G, V, skip);
        break;
    default: return t->set_err(GM_EINVAL, "tet apply: unknown operator");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return t->set_err(GM_ECUDA, std::string("tet apply: ") + cudaGetErrorString(e));
    return GM_OK;
}

}  // namespace

extern "C" int gm_tet_apply(gm_tet* t, int which, const void* x, void* y, double dt, int dtype, void* stream)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh || !t->has_mat) return t->set_err(GM_ESTATE, "tet apply: mesh and materials required");
    if (!x || !y) return t->set_err(GM_EINVAL, "tet apply: null vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == GM_F64) return apply_t<double>(t, which, x, y, dt, s);
    if (dtype == GM_F32) return apply_t<float>(t, which, x, y, dt, s);
    return t->set_err(GM_EINVAL, "tet apply: bad dtype");
}

// ---------------------------------------------------------------------------
// Time stepping (FP64): the backward-Euler monolithic step of Sec. 3.3 without
// faults, K u - A p = f,  A^T (u - u_n) + S (p - p_n) + dt C p = 0, solved by
// Prevost's partitioned CG (Sec. 3.3.2): CG on the Schur complement
// S~ = (S + dt C) + A^T K^-1 A preconditioned by the diagonal of S + dt C, each
// product with one inner K solve (PCG with 3x3 nodal block-Jacobi).
// ---------------------------------------------------------------------------
namespace {

constexpr int TET_RED_BLOCKS = 256;

__global__ void tet_zero_masked(int N, const uint8_t* mask, double* u, double* p)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const unsigned m = mask[n];
    if (u)
        for (int c = 0; c < 3; ++c)
            if ((m >> c) & 1u) u[c * N + n] = 0.0;
    if (p && ((m >> 3) & 1u)) p[n] = 0.0;
}

__global__ void tet_jac_p(int N, const double* Sd, const double* Cd, double dt, const uint8_t* mask, const double* r,
                          double* z)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    z[n] = ((mask[n] >> 3) & 1u) ? 0.0 : r[n] / (Sd[n] + dt * Cd[n]);
}

__global__ void tet_axpy(long long n, double a, const double* x, double* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void tet_xpby(long long n, const double* x, double b, double* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] + b * y[i];
}

__global__ void __launch_bounds__(256) tet_dot(long long n, const double* x, const double* y, double* part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += x[i] * y[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

struct Stepper {
    gm_tet* t;
    cudaStream_t s;
    int N;
    int blocks() const { return (N + 127) / 128; }

    int apply(int which, const double* x, double* y, double dt) {
        int rc = apply_t<double>(t, which, x, y, dt, s);
        if (rc) return rc;
        const bool out_u = which == GM_OP_KB || which == GM_OP_APU;
        tet_zero_masked<<<blocks(), 128, 0, s>>>(N, t->mask.as<uint8_t>(), out_u ? y : nullptr, out_u ? nullptr : y);
        return GM_OK;
    }
    double dot(long long n, const double* x, const double* y) {
        tet_dot<<<TET_RED_BLOCKS, 256, 0, s>>>(n, x, y, t->part.as<double>());
        double h[TET_RED_BLOCKS];
        cudaMemcpyAsync(h, t->part.p, sizeof(h), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        double acc = 0.0;
        for (double v : h) acc += v;
        return acc;
    }
    void axpy(long long n, double a, const double* x, double* y) { tet_axpy<<<TET_RED_BLOCKS, 256, 0, s>>>(n, a, x, y); }
    void xpby(long long n, const double* x, double b, double* y) { tet_xpby<<<TET_RED_BLOCKS, 256, 0, s>>>(n, x, b, y); }

    // x = K^-1 b (x from 0), PCG with 3x3 nodal block Jacobi to ||r|| <= rtol ||b||,
    // device-resident (scratch 0-3 and 14)
    int solve_k(const double* b, double* x, double rtol, int maxit, long long* its) {
        TetPcg<double> e{N, s, t->w[14].as<double>(), t->w[0].as<double>(), t->w[1].as<double>(),
                         t->w[2].as<double>(), t->w[3].as<double>(), t->pcg_st.as<TetPcgState>(),
                         t->pcg_part.as<double>(),
                         TetPrecT<double>{N, 0, t->Kinv.as<double>(), nullptr, nullptr, nullptr, nullptr},
                         t->mask.as<uint8_t>()};
        const int rc = e.solve(
            b, x, rtol, maxit, its,
            [&](const double* p, double* q, const int* skip, cudaStream_t cs) {
                apply_t<double>(t, GM_OP_KB, p, q, 0.0, cs, skip);
            },
            t->use_graphs ? &t->pcg_graph[0] : nullptr, &t->cap_stream);
        if (rc == 2) return t->set_err(GM_ENAN, "tet step: K not positive on a direction");
        if (rc == 3) return t->set_err(GM_ENOCONV, "tet step: K solve did not converge");
        if (rc < 0) return t->set_err(GM_ECUDA, std::string("tet step: ") + cudaGetErrorString(cudaGetLastError()));
        return GM_OK;
    }
};

// nodal 3x3 blocks of K and the diagonals of S and C (host), uploaded
int tet_prepare(gm_tet* t)
{
    t->drop_graphs();   // the vectors they hold are reallocated below
    const long long N = t->N, M = t->M;
    const double lam = t->E * t->nu / ((1 + t->nu) * (1 - 2 * t->nu)), mu = t->E / (2 * (1 + t->nu));
    std::vector<double> B(9 * N, 0.0), Sd(N, 0.0), Cd(N, 0.0);
    for (long long e = 0; e < M; ++e) {
        const double V = t->hV[e];
        for (int a = 0; a < 4; ++a) {
            const int n = t->htv[4 * e + a];
            const double* g = &t->hG[12 * e + 3 * a];
            const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    B[(3 * i + j) * N + n] += V * ((lam + mu) * g[i] * g[j] + (i == j ? mu * gg : 0.0));
            Sd[n] += V / (10.0 * t->Mb);
            Cd[n] += (t->k / t->mu_f) * V * gg;
        }
    }
    std::vector<double> Kinv(9 * N, 0.0);
    for (long long n = 0; n < N; ++n) {
        double b[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) b[i][j] = B[(3 * i + j) * N + n];
        for (int c = 0; c < 3; ++c)
            if (t->fixed[c * N + n])
                for (int d = 0; d < 3; ++d) { b[c][d] = (c == d) ? 1.0 : 0.0; b[d][c] = (c == d) ? 1.0 : 0.0; }
        const double c00 = b[1][1] * b[2][2] - b[1][2] * b[2][1];
        const double c01 = b[1][2] * b[2][0] - b[1][0] * b[2][2];
        const double c02 = b[1][0] * b[2][1] - b[1][1] * b[2][0];
        const double det = b[0][0] * c00 + b[0][1] * c01 + b[0][2] * c02;
        if (!(det > 0.0)) return t->set_err(GM_EINVAL, "tet step: singular nodal block");
        double inv[3][3] = {{c00 / det, (b[0][2] * b[2][1] - b[0][1] * b[2][2]) / det, (b[0][1] * b[1][2] - b[0][2] * b[1][1]) / det},
                            {c01 / det, (b[0][0] * b[2][2] - b[0][2] * b[2][0]) / det, (b[0][2] * b[1][0] - b[0][0] * b[1][2]) / det},
                            {c02 / det, (b[0][1] * b[2][0] - b[0][0] * b[2][1]) / det, (b[0][0] * b[1][1] - b[0][1] * b[1][0]) / det}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Kinv[(3 * i + j) * N + n] = (t->fixed[i * N + n] || t->fixed[j * N + n]) ? 0.0 : inv[i][j];
    }
    std::vector<uint8_t> mk(N, 0);
    for (long long n = 0; n < N; ++n)
        for (int c = 0; c < 4; ++c)
            if (t->fixed[c * N + n]) mk[n] |= (uint8_t)(1u << c);
    std::vector<double> fu = t->fu;
    for (long long i = 0; i < 3 * N; ++i)
        if (t->fixed[i]) fu[i] = 0.0;
    cudaError_t ce;
    if ((ce = t->Kinv.put(Kinv.data(), Kinv.size() * 8)) != cudaSuccess || (ce = t->Sd.put(Sd.data(), N * 8)) != cudaSuccess ||
        (ce = t->Cd.put(Cd.data(), N * 8)) != cudaSuccess || (ce = t->mask.put(mk.data(), N)) != cudaSuccess ||
        (ce = t->dfu.put(fu.data(), 3 * N * 8)) != cudaSuccess || (ce = t->part.alloc(TET_RED_BLOCKS * 8)) != cudaSuccess ||
        (ce = t->pcg_st.alloc(sizeof(TetPcgState))) != cudaSuccess ||
        (ce = t->pcg_part.alloc(2 * TPCG_BLOCKS * sizeof(double))) != cudaSuccess)
        return t->set_err(GM_ECUDA, std::string("tet step: ") + cudaGetErrorString(ce));
    for (auto& b : t->w)
        if ((ce = b.alloc(3 * N * 8)) != cudaSuccess)
            return t->set_err(GM_ECUDA, std::string("tet step: ") + cudaGetErrorString(ce));
    t->prec_ready = true;
    return GM_OK;
}

}  // namespace

extern "C" int gm_tet_dirichlet(gm_tet* t, const uint8_t* fixed, int64_t n)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh) return t->set_err(GM_ESTATE, "tet dirichlet: no mesh");
    if (!fixed || n != 4 * t->N) return t->set_err(GM_EINVAL, "tet dirichlet: need 4*N bytes");
    t->fixed.assign(fixed, fixed + n);
    t->prec_ready = false;
    t->fault_ready = false;
    return GM_OK;
}

extern "C" int gm_tet_surface_load(gm_tet* t, const int64_t* tris, int64_t n_tris, double sigma0)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh) return t->set_err(GM_ESTATE, "tet load: no mesh");
    if ((!tris && n_tris > 0) || n_tris < 0) return t->set_err(GM_EINVAL, "tet load: bad triangles");
    const long long N = t->N;
    std::vector<double> f(3 * N, 0.0);
    for (long long q = 0; q < n_tris; ++q) {
        long long v[3];
        for (int b = 0; b < 3; ++b) {
            v[b] = tris[3 * q + b];
            if (v[b] < 0 || v[b] >= N) return t->set_err(GM_EINVAL, "tet load: vertex id out of range");
        }
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = t->hX[3 * v[1] + d] - t->hX[3 * v[0] + d];
            e2[d] = t->hX[3 * v[2] + d] - t->hX[3 * v[0] + d];
        }
        // area times normal: half the cross product (the vertex order gives its side)
        const double an[3] = {0.5 * (e1[1] * e2[2] - e1[2] * e2[1]), 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]),
                              0.5 * (e1[0] * e2[1] - e1[1] * e2[0])};
        for (int b = 0; b < 3; ++b)
            for (int d = 0; d < 3; ++d) f[d * N + v[b]] -= sigma0 * an[d] / 3.0;
    }
    t->fu.swap(f);
    t->prec_ready = false;
    t->fault_ready = false;
    return GM_OK;
}

extern "C" int gm_tet_step(gm_tet* t, double dt, double* u, double* p, double rtol, int maxit,
                           gm_solve_report* rep, void* stream)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh || !t->has_mat) return t->set_err(GM_ESTATE, "tet step: mesh and materials required");
    if (!u || !p || !(dt > 0) || !(rtol > 0) || maxit < 1) return t->set_err(GM_EINVAL, "tet step: bad arguments");
    cudaSetDevice(t->device);
    int rc;
    if (!t->prec_ready && (rc = tet_prepare(t))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = (int)t->N;
    const long long n3 = 3LL * N;
    Stepper st{t, s, N};
    double* b1 = t->w[4].as<double>();
    double* y1 = t->w[5].as<double>();
    double* t3 = t->w[6].as<double>();
    double* t3b = t->w[7].as<double>();
    double* r2 = t->w[8].as<double>();
    double* z2 = t->w[9].as<double>();
    double* p2 = t->w[10].as<double>();
    double* q2 = t->w[11].as<double>();
    double* x2 = t->w[12].as<double>();
    double* tp = t->w[13].as<double>();
    const double irtol = rtol * 1e-2;
    long long ik = 0;
    // right-hand sides: b1 = f, b2 = A^T u_n + S p_n
    cudaMemcpyAsync(b1, t->dfu.p, n3 * 8, cudaMemcpyDeviceToDevice, s);
    if ((rc = st.apply(GM_OP_AUP, u, r2, 0.0))) return rc;
    if ((rc = st.apply(GM_OP_A22, p, tp, 0.0))) return rc;        // dt = 0: S p
    st.axpy(N, 1.0, tp, r2);
    // y1 = K^-1 b1;  r2 = b2 - A^T y1
    if ((rc = st.solve_k(b1, y1, irtol, maxit, &ik))) return rc;
    if ((rc = st.apply(GM_OP_AUP, y1, tp, 0.0))) return rc;
    st.axpy(N, -1.0, tp, r2);
    cudaMemsetAsync(x2, 0, (size_t)N * 8, s);
    const double rr0 = st.dot(N, r2, r2);
    int it = 0;
    double rr = rr0;
    if (rr0 > 0.0) {
        tet_jac_p<<<st.blocks(), 128, 0, s>>>(N, t->Sd.as<double>(), t->Cd.as<double>(), dt, t->mask.as<uint8_t>(), r2, z2);
        cudaMemcpyAsync(p2, z2, (size_t)N * 8, cudaMemcpyDeviceToDevice, s);
        double rz = st.dot(N, r2, z2);
        for (it = 1; it <= maxit; ++it) {
            // q2 = (S + dt C) p2 + A^T K^-1 A p2
            if ((rc = st.apply(GM_OP_A22, p2, q2, dt))) return rc;
            if ((rc = st.apply(GM_OP_APU, p2, t3, 0.0))) return rc;
            if ((rc = st.solve_k(t3, t3b, irtol, maxit, &ik))) return rc;
            if ((rc = st.apply(GM_OP_AUP, t3b, tp, 0.0))) return rc;
            st.axpy(N, 1.0, tp, q2);
            const double pq = st.dot(N, p2, q2);
            if (!(pq > 0.0) || !std::isfinite(pq)) return t->set_err(GM_ENAN, "tet step: Schur complement not positive");
            const double a = rz / pq;
            st.axpy(N, a, p2, x2);
            st.axpy(N, -a, q2, r2);
            rr = st.dot(N, r2, r2);
            if (rr <= rtol * rtol * rr0) break;
            tet_jac_p<<<st.blocks(), 128, 0, s>>>(N, t->Sd.as<double>(), t->Cd.as<double>(), dt, t->mask.as<uint8_t>(), r2, z2);
            const double rzn = st.dot(N, r2, z2);
            st.xpby(N, z2, rzn / rz, p2);
            rz = rzn;
        }
    }
    // u = K^-1 (b1 + A x2), p = x2
    if ((rc = st.apply(GM_OP_APU, x2, t3, 0.0))) return rc;
    st.axpy(n3, 1.0, b1, t3);
    if ((rc = st.solve_k(t3, u, irtol, maxit, &ik))) return rc;
    cudaMemcpyAsync(p, x2, (size_t)N * 8, cudaMemcpyDeviceToDevice, s);
    const cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return t->set_err(GM_ECUDA, std::string("tet step: ") + cudaGetErrorString(ce));
    if (rep) {
        rep->iterations = it;
        rep->rel_residual = rr0 > 0 ? std::sqrt(rr / rr0) : 0.0;
        rep->status = (it > maxit) ? GM_ENOCONV : GM_OK;
    }
    if (it > maxit) return t->set_err(GM_ENOCONV, "tet step: partitioned CG did not converge");
    return GM_OK;
}

// ---------------------------------------------------------------------------
// Fault on the tetrahedral mesh (Sec. 3.1.1-3.1.2, 3.3.1): interface elements
// on the fault triangles.  The pair terms run one thread per node pair; each
// pair owns its two lip nodes, so these kernels add into them without atomics
// after the bulk kernel has written them.  The triangle Laplacian is gathered
// by each pair from its incident triangles in a fixed order.  Tied lip
// pressures are handled by expanding the plus-lip entries from the minus lip
// before a product (P x) and folding the plus-lip rows into the minus lip
// after it (P^T y), so every operator is the one of the tied unknowns.
// Frame layout: fr[c*P + i] = n_c, fr[(3+c)*P + i] = t1_c, fr[(6+c)*P + i] = t2_c.
// ---------------------------------------------------------------------------
namespace {

struct PairGeo {
    int P, N;
    const int* pm;
    const int* pp;
    const double* area;
    const double* fr;
};

// contact / Coulomb return map of one pair (Sec. 2.2.1, Eqs. normal_traction,
// yield_function, plastic_slip_increment, corrector): the arithmetic of the
// structured path's return map with a per-pair frame.  T is the incremental
// conjugate traction -(t'_n - t'_n0) n + (t_s - tau0); D the symmetric tangent
// (stick k_n nn + k_s P_t, slip k_n nn + k_s (f t'_n / |t^tr|)(P_t - tau tau),
// open 0), six entries xx xy xz yy yz zz.
__global__ void tetf_return_map(PairGeo g, const double* u, const double* du, const double* dlie_prev, double kn,
                                double ks, double fric, double tn0, double t01, double t02, int8_t* state,
                                double* tn_out, double* dlie, double* T, double* F_out, double* dn_out, double* gs,
                                double* D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    const int P = g.P, N = g.N, a = g.pm[i], b = g.pp[i];
    double j[3], n[3], t1[3], t2[3];
    for (int c = 0; c < 3; ++c) {
        j[c] = (u[c * N + b] + du[c * N + b]) - (u[c * N + a] + du[c * N + a]);
        n[c] = g.fr[c * P + i];
        t1[c] = g.fr[(3 + c) * P + i];
        t2[c] = g.fr[(6 + c) * P + i];
    }
    const double dn = n[0] * j[0] + n[1] * j[1] + n[2] * j[2];
    const double g1 = t1[0] * j[0] + t1[1] * j[1] + t1[2] * j[2];
    const double g2 = t2[0] * j[0] + t2[1] * j[1] + t2[2] * j[2];
    const double tnc = tn0 - kn * dn;
    const bool contact = tnc >= 0.0;
    const double dl1 = dlie_prev[i], dl2 = dlie_prev[P + i];
    const double tr1 = t01 + ks * (g1 - dl1);
    const double tr2 = t02 + ks * (g2 - dl2);
    const double nt = sqrt(tr1 * tr1 + tr2 * tr2);
    const double tn = contact ? tnc : 0.0;
    const double F = nt - fric * tn;
    const bool slip = contact && F > 0.0 && nt > 0.0;
    const bool stick = contact && !slip;
    double l1 = dl1, l2 = dl2, tau1 = 0.0, tau2 = 0.0, ratio = 0.0, Ts1, Ts2;
    if (stick) {
        Ts1 = ks * (g1 - dl1);
        Ts2 = ks * (g2 - dl2);
    } else if (slip) {
        tau1 = tr1 / nt;
        tau2 = tr2 / nt;
        const double dlam = F / ks;
        l1 = dl1 + dlam * tau1;
        l2 = dl2 + dlam * tau2;
        Ts1 = fric * tn * tau1 - t01;
        Ts2 = fric * tn * tau2 - t02;
        ratio = fric * tn / nt;
    } else {
        Ts1 = -t01;
        Ts2 = -t02;
    }
    const double Tn = contact ? kn * dn : tn0;
    state[i] = contact ? (slip ? GM_SLIP : GM_STICK) : GM_OPEN;
    tn_out[i] = tn;
    dlie[i] = l1;
    dlie[P + i] = l2;
    F_out[i] = F;
    dn_out[i] = dn;
    gs[i] = g1;
    gs[P + i] = g2;
    for (int c = 0; c < 3; ++c) T[c * P + i] = Tn * n[c] + Ts1 * t1[c] + Ts2 * t2[c];
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    const double tg[3] = {tau1 * t1[0] + tau2 * t2[0], tau1 * t1[1] + tau2 * t2[1], tau1 * t1[2] + tau2 * t2[2]};
    for (int q = 0; q < 6; ++q) {
        const int x = ia[q], y = ib[q];
        const double pt = t1[x] * t1[y] + t2[x] * t2[y];
        D[q * P + i] = contact ? kn * n[x] * n[y] + (stick ? ks * pt : ks * ratio * (pt - tg[x] * tg[y])) : 0.0;
    }
}

// y(+) += A D [[x]],  y(-) -= A D [[x]]  (nothing while *skip != 0)
template <typename T>
__global__ void tetf_pair_tangent(PairGeo g, const T* D, const T* x, T* y, const int* skip)
{
    if (skip != nullptr && *skip != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    const int P = g.P, N = g.N, a = g.pm[i], b = g.pp[i];
    T j[3];
    for (int c = 0; c < 3; ++c) j[c] = x[c * N + b] - x[c * N + a];
    const T d0 = D[i], d1 = D[P + i], d2 = D[2 * P + i], d3 = D[3 * P + i], d4 = D[4 * P + i], d5 = D[5 * P + i];
    const T A = (T)g.area[i];
    const T v[3] = {A * (d0 * j[0] + d1 * j[1] + d2 * j[2]), A * (d1 * j[0] + d3 * j[1] + d4 * j[2]),
                    A * (d2 * j[0] + d4 * j[1] + d5 * j[2])};
    for (int c = 0; c < 3; ++c) {
        y[c * N + b] += v[c];
        y[c * N + a] -= v[c];
    }
}

// b1 -= cohesive force: A T on the plus lip, -A T on the minus lip
__global__ void tetf_pair_force(PairGeo g, const double* T, double* b1)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    const int P = g.P, N = g.N, a = g.pm[i], b = g.pp[i];
    const double A = g.area[i];
    for (int c = 0; c < 3; ++c) {
        b1[c * N + b] -= A * T[c * P + i];
        b1[c * N + a] += A * T[c * P + i];
    }
}

// A^f_pu: y_u(+/-) += +/- A <p> n, <p> = (p+ + p-) / 2
__global__ void tetf_pair_apu(PairGeo g, const double* xp, double* yu)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    const int P = g.P, N = g.N, a = g.pm[i], b = g.pp[i];
    const double s = g.area[i] * 0.5 * (xp[b] + xp[a]);
    for (int c = 0; c < 3; ++c) {
        const double v = s * g.fr[c * P + i];
        yu[c * N + b] += v;
        yu[c * N + a] -= v;
    }
}

// A^f_up = (A^f_pu)^T: both lips += (A / 2) n . [[u]]
__global__ void tetf_pair_aup(PairGeo g, const double* xu, double* yp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    const int P = g.P, N = g.N, a = g.pm[i], b = g.pp[i];
    double dn = 0.0;
    for (int c = 0; c < 3; ++c) dn += g.fr[c * P + i] * (xu[c * N + b] - xu[c * N + a]);
    const double v = 0.5 * g.area[i] * dn;
    yp[b] += v;
    yp[a] += v;
}

// fracture flow on <p> and [[p]] (Sec. 3.2.3): storage (A w / M_F) <p> / 2 to
// each lip, longitudinal (w k_par / mu) (1/2) sum_t L_t <p> to each lip, and,
// untied, the transverse A k_perp / (mu w) [[p]]; cst, clap, ctr carry the
// coefficients times the storage / flow weights of the product.
__global__ void tetf_pair_flow(PairGeo g, double cst, double clap, double ctr, const int* prow, const int* padj,
                               const int* tri, const double* Lt, const double* x, double* y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    const int a = g.pm[i], b = g.pp[i];
    const double A = g.area[i];
    double acc = 0.5 * cst * A * 0.5 * (x[b] + x[a]);
    double lap = 0.0;
    for (int q = prow[i]; q < prow[i + 1]; ++q) {
        const int code = padj[q];
        const int tt = code / 3, la = code - 3 * tt;
        for (int v = 0; v < 3; ++v) {
            const int pv = tri[3 * tt + v];
            lap += Lt[9 * tt + 3 * la + v] * 0.5 * (x[g.pp[pv]] + x[g.pm[pv]]);
        }
    }
    acc += 0.5 * clap * lap;
    const double tr = ctr * A * (x[b] - x[a]);
    y[b] += acc + tr;
    y[a] += acc - tr;
}

__global__ void tetf_expand(PairGeo g, double* x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.P) x[g.pp[i]] = x[g.pm[i]];
}

__global__ void tetf_fold(PairGeo g, double* y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.P) return;
    y[g.pm[i]] += y[g.pp[i]];
    y[g.pp[i]] = 0.0;
}

// inverse nodal 3x3 blocks of K_T: bulk block plus A D on both lips of a pair
__global__ void tetf_bjac_build(int N, int P, const double* Kblk, const int* n2p, const double* area, const double* D,
                                const uint8_t* mask, double* Kinv, int* err)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double b[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b[i][j] = Kblk[(3 * i + j) * N + n];
    const int q = n2p[n];
    if (q >= 0) {
        const double A = area[q];
        const double d[6] = {D[q], D[P + q], D[2 * P + q], D[3 * P + q], D[4 * P + q], D[5 * P + q]};
        const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) b[i][j] += A * d[idx[i][j]];
    }
    const unsigned m = mask[n];
    for (int c = 0; c < 3; ++c)
        if ((m >> c) & 1u)
            for (int d = 0; d < 3; ++d) { b[c][d] = (c == d) ? 1.0 : 0.0; b[d][c] = (c == d) ? 1.0 : 0.0; }
    const double c00 = b[1][1] * b[2][2] - b[1][2] * b[2][1];
    const double c01 = b[1][2] * b[2][0] - b[1][0] * b[2][2];
    const double c02 = b[1][0] * b[2][1] - b[1][1] * b[2][0];
    const double det = b[0][0] * c00 + b[0][1] * c01 + b[0][2] * c02;
    if (!(det > 0.0)) {
        *err = 1;
        for (int k = 0; k < 9; ++k) Kinv[k * N + n] = 0.0;
        return;
    }
    const double inv[3][3] = {
        {c00 / det, (b[0][2] * b[2][1] - b[0][1] * b[2][2]) / det, (b[0][1] * b[1][2] - b[0][2] * b[1][1]) / det},
        {c01 / det, (b[0][0] * b[2][2] - b[0][2] * b[2][0]) / det, (b[0][2] * b[1][0] - b[0][0] * b[1][2]) / det},
        {c02 / det, (b[0][1] * b[2][0] - b[0][0] * b[2][1]) / det, (b[0][0] * b[1][1] - b[0][1] * b[1][0]) / det}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Kinv[(3 * i + j) * N + n] = (((m >> i) & 1u) || ((m >> j) & 1u)) ? 0.0 : inv[i][j];
}

// diagonal of S + dt C on free pressures (0 elsewhere) and its inverse
__global__ void tetf_diag_a(int N, const double* Sd, const double* Cd, double dt, const uint8_t* mask, double* dAm,
                            double* invdA)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const bool fixed = (mask[n] >> 3) & 1u;
    const double d = Sd[n] + dt * Cd[n];
    dAm[n] = fixed ? 0.0 : d;
    invdA[n] = fixed ? 0.0 : 1.0 / d;
}

// sum_i x_i y_i w_i (w may be null), per-block partials summed on the host in order
__global__ void __launch_bounds__(256) tetf_wdot(long long n, const double* x, const double* y, const double* w,
                                                 double* part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += x[i] * y[i] * (w ? w[i] : 1.0);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// host: nodal blocks of K, diagonals of S and C with the fault terms (folded
// when tied), masks, scaled-norm weights, loads, in-situ floor; uploads
int tetf_prepare(gm_tet* t)
{
    t->drop_graphs();   // the vectors they hold are reallocated below
    const long long N = t->N, M = t->M, P = t->P;
    const double lam = t->E * t->nu / ((1 + t->nu) * (1 - 2 * t->nu)), mu = t->E / (2 * (1 + t->nu));
    const double cond = t->k / t->mu_f;
    const gm_fault_params& fp = t->fpar;
    std::vector<double> B(9 * N, 0.0), Sd(N, 0.0), Cd(N, 0.0);
    for (long long e = 0; e < M; ++e) {
        const double V = t->hV[e];
        for (int a = 0; a < 4; ++a) {
            const int n = t->htv[4 * e + a];
            const double* g = &t->hG[12 * e + 3 * a];
            const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    B[(3 * i + j) * N + n] += V * ((lam + mu) * g[i] * g[j] + (i == j ? mu * gg : 0.0));
            Sd[n] += V / (10.0 * t->Mb);
            Cd[n] += cond * V * gg;
        }
    }
    // fault entries on the lip diagonals and on the (minus, plus) entry of each pair
    std::vector<double> xS(P, 0.0), xC(P, 0.0);
    const double clap = fp.wk_par / t->mu_f;
    for (long long i = 0; i < P; ++i) {
        const double st = t->harea[i] * fp.w0 / fp.MF;
        Sd[t->hpm[i]] += 0.25 * st;
        Sd[t->hpp[i]] += 0.25 * st;
        xS[i] += 0.25 * st;
        if (!t->tied) {
            const double tr = t->harea[i] * fp.k_perp / (t->mu_f * fp.w0);
            Cd[t->hpm[i]] += tr;
            Cd[t->hpp[i]] += tr;
        }
    }
    for (long long q = 0; q < t->NTRI; ++q)
        for (int a = 0; a < 3; ++a) {
            const int i = t->htri[3 * q + a];
            const double l = 0.25 * clap * t->hLt[9 * q + 4 * a];
            Cd[t->hpm[i]] += l;
            Cd[t->hpp[i]] += l;
            xC[i] += l;
        }
    std::vector<uint8_t> fixed = t->fixed;
    if (t->tied)
        for (long long i = 0; i < P; ++i) {
            const int a = t->hpm[i], b = t->hpp[i];
            Sd[a] += Sd[b] + 2.0 * xS[i];
            Cd[a] += Cd[b] + 2.0 * xC[i];
            Sd[b] = 1.0;   // the plus lip carries no equation
            Cd[b] = 0.0;
            fixed[3 * N + b] = 1;
        }
    std::vector<uint8_t> mk(N, 0);
    for (long long n = 0; n < N; ++n)
        for (int c = 0; c < 4; ++c)
            if (fixed[c * N + n]) mk[n] |= (uint8_t)(1u << c);
    std::vector<double> dKm(3 * N), invdK(3 * N), fu = t->fu;
    for (int c = 0; c < 3; ++c)
        for (long long n = 0; n < N; ++n) {
            const long long k = c * N + n;
            const double d = B[(3 * c + c) * N + n];
            const bool fr = fixed[k] != 0;
            dKm[k] = fr ? 0.0 : d;
            invdK[k] = fr ? 0.0 : 1.0 / d;
            if (fr) fu[k] = 0.0;
        }
    std::vector<double> fpv = t->fpsrc;
    if (t->tied)
        for (long long i = 0; i < P; ++i) {
            fpv[t->hpm[i]] += fpv[t->hpp[i]];
            fpv[t->hpp[i]] = 0.0;
        }
    // in-situ floor of the scale: sum over free lip dofs of F0^2 / K_ii,
    // F0 = A (-t'_n0 n + tau0_1 t1 + tau0_2 t2)
    double f0 = 0.0;
    for (long long i = 0; i < P; ++i)
        for (int c = 0; c < 3; ++c) {
            const double F0 = t->harea[i] * (-fp.tn0 * t->hfr[c * P + i] + fp.tau0[0] * t->hfr[(3 + c) * P + i] +
                                             fp.tau0[1] * t->hfr[(6 + c) * P + i]);
            for (int lip = 0; lip < 2; ++lip) {
                const long long k = c * N + (lip ? t->hpp[i] : t->hpm[i]);
                if (!fixed[k]) f0 += F0 * F0 / B[(3 * c + c) * N + (lip ? t->hpp[i] : t->hpm[i])];
            }
        }
    t->f0sq = f0;
    cudaError_t ce;
    if ((ce = t->f_Kblk.put(B.data(), B.size() * 8)) != cudaSuccess || (ce = t->f_Kinv.alloc(9 * N * 8)) != cudaSuccess ||
        (ce = t->f_fu.put(fu.data(), 3 * N * 8)) != cudaSuccess || (ce = t->f_fpv.put(fpv.data(), N * 8)) != cudaSuccess ||
        (ce = t->f_Sd.put(Sd.data(), N * 8)) != cudaSuccess || (ce = t->f_Cd.put(Cd.data(), N * 8)) != cudaSuccess ||
        (ce = t->f_dKm.put(dKm.data(), 3 * N * 8)) != cudaSuccess ||
        (ce = t->f_invdK.put(invdK.data(), 3 * N * 8)) != cudaSuccess || (ce = t->f_dAm.alloc(N * 8)) != cudaSuccess ||
        (ce = t->f_invdA.alloc(N * 8)) != cudaSuccess || (ce = t->f_mask.put(mk.data(), N)) != cudaSuccess ||
        (ce = t->f_err.alloc(sizeof(int))) != cudaSuccess || (ce = t->part.alloc(TET_RED_BLOCKS * 8)) != cudaSuccess ||
        (ce = t->f_Pinv.alloc(36 * P * 8)) != cudaSuccess || (ce = t->f_Pinv32.alloc(36 * P * 4)) != cudaSuccess ||
        (ce = t->f_Kinv32.alloc(9 * N * 4)) != cudaSuccess || (ce = t->f_D32.alloc(6 * P * 4)) != cudaSuccess ||
        (ce = t->pcg_st.alloc(sizeof(TetPcgState))) != cudaSuccess ||
        (ce = t->pcg_part.alloc(2 * TPCG_BLOCKS * sizeof(double))) != cudaSuccess)
        return t->set_err(GM_ECUDA, std::string("tet fault: ") + cudaGetErrorString(ce));
    for (auto& b : t->fw)
        if ((ce = b.alloc(3 * N * 8)) != cudaSuccess)
            return t->set_err(GM_ECUDA, std::string("tet fault: ") + cudaGetErrorString(ce));
    for (auto& b : t->fw32)
        if ((ce = b.alloc(3 * N * 4)) != cudaSuccess)
            return t->set_err(GM_ECUDA, std::string("tet fault: ") + cudaGetErrorString(ce));
    t->fault_ready = true;
    return GM_OK;
}

struct FStepper {
    gm_tet* t;
    cudaStream_t s;
    int N, P;
    bool f32 = false;          // inner K_T solves in FP32
    long long applies = 0;

    PairGeo geo() const
    {
        return PairGeo{P, N, t->f_pm.as<int>(), t->f_pp.as<int>(), t->f_area.as<double>(), t->f_fr.as<double>()};
    }
    int nb() const { return (N + 127) / 128; }
    int pb() const { return (P + 127) / 128; }
    double* w(int k) const { return t->fw[k].as<double>(); }

    void mask_u(double* y) { tet_zero_masked<<<nb(), 128, 0, s>>>(N, t->f_mask.as<uint8_t>(), y, nullptr); }
    void mask_p(double* y) { tet_zero_masked<<<nb(), 128, 0, s>>>(N, t->f_mask.as<uint8_t>(), nullptr, y); }
    void axpy(long long n, double a, const double* x, double* y) { tet_axpy<<<TET_RED_BLOCKS, 256, 0, s>>>(n, a, x, y); }
    void xpby(long long n, const double* x, double b, double* y) { tet_xpby<<<TET_RED_BLOCKS, 256, 0, s>>>(n, x, b, y); }
    void copy(double* y, const double* x, long long n) { cudaMemcpyAsync(y, x, n * 8, cudaMemcpyDeviceToDevice, s); }
    double dot(long long n, const double* x, const double* y, const double* wt = nullptr)
    {
        tetf_wdot<<<TET_RED_BLOCKS, 256, 0, s>>>(n, x, y, wt, t->part.as<double>());
        double h[TET_RED_BLOCKS];
        cudaMemcpyAsync(h, t->part.p, sizeof(h), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        double acc = 0.0;
        for (double v : h) acc += v;
        return acc;
    }
    int bulk(int which, const double* x, double* y, double dt)
    {
        ++applies;
        return apply_t<double>(t, which, x, y, dt, s);
    }
    // pressure input with the plus lips of tied pairs set from the minus lips (scratch 0)
    const double* expanded(const double* xp)
    {
        if (!t->tied) return xp;
        double* e = w(0);
        copy(e, xp, N);
        tetf_expand<<<pb(), 128, 0, s>>>(geo(), e);
        return e;
    }

    // unmasked products in the tied unknowns
    int KT_raw(const double* x, double* y)
    {
        int rc = bulk(GM_OP_KB, x, y, 0.0);
        if (rc) return rc;
        tetf_pair_tangent<double><<<pb(), 128, 0, s>>>(geo(), t->f_D.as<double>(), x, y, nullptr);
        return GM_OK;
    }
    // q = K_T p in the inner-solve precision, unmasked (the PCG masks it)
    template <typename T>
    void KT_inner(const T* p, T* q, const int* skip, cudaStream_t cs)
    {
        apply_t<T>(t, GM_OP_KB, p, q, 0.0, cs, skip);
        const T* D = sizeof(T) == 8 ? (const T*)t->f_D.p : (const T*)t->f_D32.p;
        tetf_pair_tangent<T><<<pb(), 128, 0, cs>>>(geo(), D, p, q, skip);
    }
    int APU_raw(const double* xp, double* yu)
    {
        const double* e = expanded(xp);
        int rc = bulk(GM_OP_APU, e, yu, 0.0);
        if (rc) return rc;
        tetf_pair_apu<<<pb(), 128, 0, s>>>(geo(), e, yu);
        return GM_OK;
    }
    int AUP_raw(const double* xu, double* yp)
    {
        int rc = bulk(GM_OP_AUP, xu, yp, 0.0);
        if (rc) return rc;
        tetf_pair_aup<<<pb(), 128, 0, s>>>(geo(), xu, yp);
        if (t->tied) tetf_fold<<<pb(), 128, 0, s>>>(geo(), yp);
        return GM_OK;
    }
    int A22_raw(const double* xp, double* yp, double dt)
    {
        const gm_fault_params& fp = t->fpar;
        const double* e = expanded(xp);
        int rc = bulk(GM_OP_A22, e, yp, dt);
        if (rc) return rc;
        const double cst = fp.w0 / fp.MF;
        const double clap = dt * fp.wk_par / t->mu_f;
        const double ctr = t->tied ? 0.0 : dt * fp.k_perp / (t->mu_f * fp.w0);
        tetf_pair_flow<<<pb(), 128, 0, s>>>(geo(), cst, clap, ctr, t->f_prow.as<int>(), t->f_padj.as<int>(),
                                            t->f_tri.as<int>(), t->f_Lt.as<double>(), e, yp);
        if (t->tied) tetf_fold<<<pb(), 128, 0, s>>>(geo(), yp);
        return GM_OK;
    }
    int KT(const double* x, double* y) { int rc = KT_raw(x, y); if (!rc) mask_u(y); return rc; }
    int APU(const double* x, double* y) { int rc = APU_raw(x, y); if (!rc) mask_u(y); return rc; }
    int AUP(const double* x, double* y) { int rc = AUP_raw(x, y); if (!rc) mask_p(y); return rc; }
    int A22(const double* x, double* y, double dt) { int rc = A22_raw(x, y, dt); if (!rc) mask_p(y); return rc; }

    // x = K_T^-1 b from x = 0 to ||r|| <= rtol ||b||: device-resident PCG with
    // nodal 3x3 and lip-pair 6x6 block Jacobi, in FP32 (operator, blocks and
    // vectors) when f32 is set  (scratch 1-4 and 24, or the FP32 scratch)
    int solve_kt(const double* b, double* x, double rtol, int maxit, long long* its)
    {
        int rc;
        const long long its0 = *its;
        TetPcgState* ps = t->pcg_st.as<TetPcgState>();
        double* part = t->pcg_part.as<double>();
        const uint8_t* mk = t->f_mask.as<uint8_t>();
        if (f32) {
            float* v[5];
            for (int k = 0; k < 5; ++k) v[k] = t->fw32[k].as<float>();
            TetPcg<float> e{N, s, v[0], v[1], v[2], v[3], v[4], ps, part,
                            TetPrecT<float>{N, P, t->f_Kinv32.as<float>(), t->f_n2p.as<int>(), t->f_pm.as<int>(),
                                            t->f_pp.as<int>(), t->f_Pinv32.as<float>()},
                            mk};
            rc = e.solve(
                b, x, rtol, maxit, its,
                [&](const float* p, float* q, const int* skip, cudaStream_t cs) { KT_inner<float>(p, q, skip, cs); },
                t->use_graphs ? &t->pcg_graph[2] : nullptr, &t->cap_stream);
        } else {
            TetPcg<double> e{N, s, w(24), w(1), w(2), w(3), w(4), ps, part,
                             TetPrecT<double>{N, P, t->f_Kinv.as<double>(), t->f_n2p.as<int>(), t->f_pm.as<int>(),
                                              t->f_pp.as<int>(), t->f_Pinv.as<double>()},
                             mk};
            rc = e.solve(
                b, x, rtol, maxit, its,
                [&](const double* p, double* q, const int* skip, cudaStream_t cs) { KT_inner<double>(p, q, skip, cs); },
                t->use_graphs ? &t->pcg_graph[1] : nullptr, &t->cap_stream);
        }
        applies += *its - its0;
        if (rc == 2) return t->set_err(GM_ENAN, "tet fault: K_T not positive on a direction");
        if (rc == 3) return t->set_err(GM_ENOCONV, "tet fault: K_T solve did not converge");
        if (rc < 0) return t->set_err(GM_ECUDA, std::string("tet fault: ") + cudaGetErrorString(cudaGetLastError()));
        return GM_OK;
    }

    // [K_T, -A_pu; A_up, S + dt C] [x1; x2] = [b1; b2] by Prevost's partitioned
    // CG (Sec. 3.3.2, Eq. schur_system)  (scratch 5-12)
    int prevost(const double* b1, const double* b2, double* x1, double* x2, double dt, const gm_step_opts& o,
                int* outer, long long* inner)
    {
        double *y1 = w(5), *t3 = w(6), *t3b = w(7), *r2 = w(8), *z2 = w(9), *p2 = w(10), *q2 = w(11), *tp = w(12);
        int rc;
        if ((rc = solve_kt(b1, y1, o.inner_rtol, o.inner_maxit, inner))) return rc;
        if ((rc = AUP(y1, tp))) return rc;
        copy(r2, b2, N);
        axpy(N, -1.0, tp, r2);
        cudaMemsetAsync(x2, 0, (size_t)N * 8, s);
        const double rr0 = dot(N, r2, r2);
        if (rr0 > 0.0) {
            tet_jac_p<<<nb(), 128, 0, s>>>(N, t->f_Sd.as<double>(), t->f_Cd.as<double>(), dt, t->f_mask.as<uint8_t>(), r2, z2);
            copy(p2, z2, N);
            double rz = dot(N, r2, z2);
            int it;
            for (it = 1; it <= o.outer_maxit; ++it) {
                if ((rc = A22(p2, q2, dt))) return rc;
                if ((rc = APU(p2, t3))) return rc;
                if ((rc = solve_kt(t3, t3b, o.inner_rtol, o.inner_maxit, inner))) return rc;
                if ((rc = AUP(t3b, tp))) return rc;
                axpy(N, 1.0, tp, q2);
                const double pq = dot(N, p2, q2);
                if (!(pq > 0.0) || !std::isfinite(pq)) return t->set_err(GM_ENAN, "tet fault: Schur complement not positive");
                const double a = rz / pq;
                axpy(N, a, p2, x2);
                axpy(N, -a, q2, r2);
                ++*outer;
                if (dot(N, r2, r2) <= o.outer_rtol * o.outer_rtol * rr0) break;
                tet_jac_p<<<nb(), 128, 0, s>>>(N, t->f_Sd.as<double>(), t->f_Cd.as<double>(), dt, t->f_mask.as<uint8_t>(), r2,
                                               z2);
                const double rzn = dot(N, r2, z2);
                xpby(N, z2, rzn / rz, p2);
                rz = rzn;
            }
            if (it > o.outer_maxit) return t->set_err(GM_ENOCONV, "tet fault: partitioned CG did not converge");
        }
        if ((rc = APU(x2, t3))) return rc;
        axpy(3LL * N, 1.0, b1, t3);
        return solve_kt(t3, x1, o.inner_rtol, o.inner_maxit, inner);
    }

    // b1 = f^u - K (u + du) - F_coh + A_pu (p + dp),
    // b2 = dt f^p - dt C (p + dp) - S dp - A_up du   (Eq. linear_system), masked;
    // ut = u + du, pt = p + dp kept in scratch 17, 18  (scratch 0, 21, 22)
    int residual(const double* u, const double* p, const double* du, const double* dp, double dt, double* b1, double* b2)
    {
        const long long n3 = 3LL * N;
        double *ut = w(17), *pt = w(18), *y = w(21), *yp = w(22);
        int rc;
        copy(ut, u, n3);
        axpy(n3, 1.0, du, ut);
        copy(pt, p, N);
        axpy(N, 1.0, dp, pt);
        copy(b1, t->f_fu.as<double>(), n3);
        if ((rc = bulk(GM_OP_KB, ut, y, 0.0))) return rc;
        axpy(n3, -1.0, y, b1);
        tetf_pair_force<<<pb(), 128, 0, s>>>(geo(), t->f_T.as<double>(), b1);
        if ((rc = APU_raw(pt, y))) return rc;
        axpy(n3, 1.0, y, b1);
        mask_u(b1);
        cudaMemsetAsync(b2, 0, (size_t)N * 8, s);
        axpy(N, dt, t->f_fpv.as<double>(), b2);
        if ((rc = A22_raw(pt, yp, dt))) return rc;     // S pt + dt C pt
        axpy(N, -1.0, yp, b2);
        if ((rc = A22_raw(p, yp, 0.0))) return rc;     // S p
        axpy(N, 1.0, yp, b2);
        if ((rc = AUP_raw(du, yp))) return rc;
        axpy(N, -1.0, yp, b2);
        mask_p(b2);
        return GM_OK;
    }
};

int tetf_launch_check(gm_tet* t, const char* what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return t->set_err(GM_ECUDA, std::string(what) + cudaGetErrorString(e));
    return GM_OK;
}

}  // namespace

extern "C" int gm_tet_fault(gm_tet* t, const int64_t* pairs, int64_t n_pairs, const int64_t* tris, int64_t n_tris,
                            const double* t1_ref, const gm_fault_params* fp)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh) return t->set_err(GM_ESTATE, "tet fault: no mesh");
    if (!pairs || !tris || !t1_ref || !fp || n_pairs < 1 || n_tris < 1 || n_pairs > t->N || n_tris > kTetMaxEntities)
        return t->set_err(GM_EINVAL, "tet fault: bad arguments");
    if (!(fp->kn >= 0) || !(fp->ks > 0) || !(fp->f >= 0) || !(fp->w0 > 0) || !(fp->wk_par >= 0) || !(fp->MF > 0))
        return t->set_err(GM_EINVAL, "tet fault: invalid fault parameters");
    const long long N = t->N, P = n_pairs, NT = n_tris;
    std::vector<int> pm(P), pp(P), n2p(N, -1);
    for (long long i = 0; i < P; ++i) {
        const int64_t a = pairs[i], b = pairs[P + i];
        if (a < 0 || a >= N || b < 0 || b >= N || a == b) return t->set_err(GM_EINVAL, "tet fault: pair node out of range");
        if (n2p[a] >= 0 || n2p[b] >= 0) return t->set_err(GM_EINVAL, "tet fault: node in two pairs");
        pm[i] = (int)a;
        pp[i] = (int)b;
        n2p[a] = n2p[b] = (int)i;
    }
    std::vector<int> tri(3 * NT), cnt(P + 1, 0);
    std::vector<double> area(P, 0.0), nsum(3 * P, 0.0), Lt(9 * NT);
    for (long long q = 0; q < NT; ++q) {
        double x[3][3];
        for (int v = 0; v < 3; ++v) {
            const int64_t id = tris[3 * q + v];
            if (id < 0 || id >= P) return t->set_err(GM_EINVAL, "tet fault: triangle pair id out of range");
            tri[3 * q + v] = (int)id;
            cnt[id + 1]++;
            for (int d = 0; d < 3; ++d) x[v][d] = t->hX[3 * pm[id] + d];
        }
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = x[1][d] - x[0][d];
            e2[d] = x[2][d] - x[0][d];
        }
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double at = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        const double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
        if (!(at > 1e-12 * std::sqrt(l1 * l2))) return t->set_err(GM_EINVAL, "tet fault: degenerate triangle");
        for (int v = 0; v < 3; ++v) {
            const int i = tri[3 * q + v];
            area[i] += at / 3.0;
            for (int d = 0; d < 3; ++d) nsum[3 * i + d] += cr[d] / 6.0;
        }
        // surface gradients from the metric of the edges e1, e2: grad N = [e1 e2] G^-1 dN
        const double g11 = l1, g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2], g22 = l2;
        const double det = g11 * g22 - g12 * g12;
        const double i11 = g22 / det, i12 = -g12 / det, i22 = g11 / det;
        const double dN[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Lt[9 * q + 3 * a + b] = at * (dN[a][0] * (i11 * dN[b][0] + i12 * dN[b][1]) +
                                              dN[a][1] * (i12 * dN[b][0] + i22 * dN[b][1]));
    }
    // Orientation: the pair normal is built from the triangles' vertex order, so
    // that order must agree across the fault (an edge shared by two triangles
    // runs in opposite directions in them) ...
    {
        std::unordered_map<unsigned long long, int> dir;
        dir.reserve((size_t)(3 * NT));
        for (long long q = 0; q < NT; ++q)
            for (int v = 0; v < 3; ++v) {
                const unsigned long long a = (unsigned)tri[3 * q + v], b = (unsigned)tri[3 * q + (v + 1) % 3];
                if (a == b) return t->set_err(GM_EINVAL, "tet fault: triangle repeats a pair");
                if (++dir[a * (unsigned long long)P + b] > 1)
                    return t->set_err(GM_EINVAL, "tet fault: adjacent triangles are ordered inconsistently "
                                                 "(an edge runs the same way in both)");
            }
    }
    std::vector<double> fr(9 * P);
    for (long long i = 0; i < P; ++i) {
        if (!(area[i] > 0.0)) return t->set_err(GM_EINVAL, "tet fault: a pair lies on no triangle");
        const double* ns = &nsum[3 * i];
        const double nl = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
        if (!(nl > 1e-12 * area[i])) return t->set_err(GM_EINVAL, "tet fault: the triangle normals around a pair cancel");
        const double n[3] = {ns[0] / nl, ns[1] / nl, ns[2] / nl};
        const double dr = n[0] * t1_ref[0] + n[1] * t1_ref[1] + n[2] * t1_ref[2];
        double e[3] = {t1_ref[0] - dr * n[0], t1_ref[1] - dr * n[1], t1_ref[2] - dr * n[2]};
        const double el = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        const double rl = std::sqrt(t1_ref[0] * t1_ref[0] + t1_ref[1] * t1_ref[1] + t1_ref[2] * t1_ref[2]);
        if (!(el > 1e-8 * rl)) return t->set_err(GM_EINVAL, "tet fault: t1_ref normal to the fault");
        const double t1[3] = {e[0] / el, e[1] / el, e[2] / el};
        const double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
        for (int c = 0; c < 3; ++c) {
            fr[c * P + i] = n[c];
            fr[(3 + c) * P + i] = t1[c];
            fr[(6 + c) * P + i] = t2[c];
        }
    }
    // ... and the normal must point from the minus lip to the plus lip: every
    // tetrahedron touching a minus-lip node lies on the -n side of it, every one
    // touching a plus-lip node on the +n side, and none holds both lips of a pair.
    for (long long e = 0; e < t->M; ++e) {
        const int* tv = &t->htv[4 * e];
        double cen[3] = {0.0, 0.0, 0.0};
        for (int v = 0; v < 4; ++v)
            for (int d = 0; d < 3; ++d) cen[d] += 0.25 * t->hX[3 * tv[v] + d];
        for (int v = 0; v < 4; ++v) {
            const int q = n2p[tv[v]];
            if (q < 0) continue;
            const bool minus = pm[q] == tv[v];
            for (int w = 0; w < 4; ++w)
                if (w != v && tv[w] == (minus ? pp[q] : pm[q]))
                    return t->set_err(GM_EINVAL, "tet fault: a tetrahedron holds both lips of a pair");
            double side = 0.0;
            for (int d = 0; d < 3; ++d) side += (cen[d] - t->hX[3 * tv[v] + d]) * fr[d * P + q];
            if (minus ? !(side < 0.0) : !(side > 0.0))
                return t->set_err(GM_EINVAL, minus ? "tet fault: a minus-lip tetrahedron lies on the +n side "
                                                     "(triangle order gives a normal from plus to minus)"
                                                   : "tet fault: a plus-lip tetrahedron lies on the -n side "
                                                     "(triangle order gives a normal from plus to minus)");
        }
    }
    for (long long i = 0; i < P; ++i) cnt[i + 1] += cnt[i];
    std::vector<int> padj(3 * NT), fill(cnt.begin(), cnt.end() - 1);
    for (long long q = 0; q < NT; ++q)
        for (int v = 0; v < 3; ++v) padj[fill[tri[3 * q + v]]++] = (int)(3 * q + v);
    cudaSetDevice(t->device);
    std::vector<double> zero2(2 * P, 0.0);
    std::vector<int8_t> stick(P, (int8_t)GM_STICK);
    cudaError_t ce;
    if ((ce = t->f_pm.put(pm.data(), P * 4)) != cudaSuccess || (ce = t->f_pp.put(pp.data(), P * 4)) != cudaSuccess ||
        (ce = t->f_n2p.put(n2p.data(), N * 4)) != cudaSuccess || (ce = t->f_area.put(area.data(), P * 8)) != cudaSuccess ||
        (ce = t->f_fr.put(fr.data(), 9 * P * 8)) != cudaSuccess || (ce = t->f_Lt.put(Lt.data(), 9 * NT * 8)) != cudaSuccess ||
        (ce = t->f_tri.put(tri.data(), 3 * NT * 4)) != cudaSuccess ||
        (ce = t->f_prow.put(cnt.data(), (P + 1) * 4)) != cudaSuccess ||
        (ce = t->f_padj.put(padj.data(), 3 * NT * 4)) != cudaSuccess ||
        (ce = t->f_dlie_n.put(zero2.data(), 2 * P * 8)) != cudaSuccess || (ce = t->f_dlie.alloc(2 * P * 8)) != cudaSuccess ||
        (ce = t->f_state.alloc(P)) != cudaSuccess || (ce = t->f_T.alloc(3 * P * 8)) != cudaSuccess ||
        (ce = t->f_D.put(std::vector<double>(6 * P, 0.0).data(), 6 * P * 8)) != cudaSuccess ||
        (ce = t->f_tn.alloc(P * 8)) != cudaSuccess || (ce = t->f_F.alloc(P * 8)) != cudaSuccess ||
        (ce = t->f_dn.alloc(P * 8)) != cudaSuccess || (ce = t->f_gs.alloc(2 * P * 8)) != cudaSuccess ||
        (ce = t->f_flags_acc.put(stick.data(), P)) != cudaSuccess ||
        (ce = t->f_gs_acc.put(zero2.data(), 2 * P * 8)) != cudaSuccess)
        return t->set_err(GM_ECUDA, std::string("tet fault: ") + cudaGetErrorString(ce));
    t->P = P;
    t->NTRI = NT;
    t->fpar = *fp;
    t->tied = !(fp->k_perp > 0);
    t->hpm.swap(pm);
    t->hpp.swap(pp);
    t->hn2p.swap(n2p);
    t->harea.swap(area);
    t->hfr.swap(fr);
    t->hLt.swap(Lt);
    t->htri.swap(tri);
    t->has_fault = true;
    t->fault_ready = false;
    return GM_OK;
}

extern "C" int gm_tet_loads(gm_tet* t, const double* fu, const double* fp)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh) return t->set_err(GM_ESTATE, "tet loads: no mesh");
    const long long N = t->N;
    if (fu) t->fu.assign(fu, fu + 3 * N);
    else t->fu.assign(3 * N, 0.0);
    if (fp) t->fpsrc.assign(fp, fp + N);
    else t->fpsrc.assign(N, 0.0);
    t->prec_ready = false;
    t->fault_ready = false;
    return GM_OK;
}

extern "C" int gm_tet_fault_apply(gm_tet* t, int which, const double* x, double* y, double dt, void* stream)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh || !t->has_mat || !t->has_fault) return t->set_err(GM_ESTATE, "tet fault apply: mesh, materials and fault required");
    if (!x || !y) return t->set_err(GM_EINVAL, "tet fault apply: null vector");
    cudaSetDevice(t->device);
    int rc;
    if (!t->fault_ready && (rc = tetf_prepare(t))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FStepper st{t, s, (int)t->N, (int)t->P};
    const long long N = t->N;
    double* xu = st.w(21);
    double* xp = st.w(22);
    switch (which) {
    case GM_OP_KT: st.copy(xu, x, 3 * N); st.mask_u(xu); rc = st.KT(xu, y); break;
    case GM_OP_APU: st.copy(xp, x, N); st.mask_p(xp); rc = st.APU(xp, y); break;
    case GM_OP_AUP: st.copy(xu, x, 3 * N); st.mask_u(xu); rc = st.AUP(xu, y); break;
    case GM_OP_A22: st.copy(xp, x, N); st.mask_p(xp); rc = st.A22(xp, y, dt); break;
    default: return t->set_err(GM_EINVAL, "tet fault apply: operator not available");
    }
    if (rc) return rc;
    return tetf_launch_check(t, "tet fault apply: ");
}

extern "C" int gm_tet_fault_step(gm_tet* t, double dt, double* u, double* p, const gm_step_opts* opts,
                                 gm_step_report* rep, void* stream)
{
    if (!t) return GM_EINVAL;
    if (!t->has_mesh || !t->has_mat || !t->has_fault) return t->set_err(GM_ESTATE, "tet fault step: mesh, materials and fault required");
    if (!u || !p || !opts || !(dt > 0) || !(opts->newton_rtol > 0) || opts->newton_maxit < 1 || !(opts->outer_rtol > 0) ||
        opts->outer_maxit < 1 || !(opts->inner_rtol > 0) || opts->inner_maxit < 1 ||
        (opts->precision != GM_F64 && opts->precision != GM_F32))
        return t->set_err(GM_EINVAL, "tet fault step: bad arguments");
    cudaSetDevice(t->device);
    int rc;
    if (!t->fault_ready && (rc = tetf_prepare(t))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = (int)t->N, P = (int)t->P;
    const long long n3 = 3LL * N;
    FStepper st{t, s, N, P};
    st.f32 = opts->precision == GM_F32;
    const gm_fault_params& fp = t->fpar;
    double *du = st.w(13), *dp = st.w(14), *b1 = st.w(15), *b2 = st.w(16), *x1 = st.w(19), *x2 = st.w(20);
    double* pst = st.w(23);
    double *ut = st.w(17), *pt = st.w(18);
    cudaMemsetAsync(du, 0, n3 * 8, s);
    cudaMemsetAsync(dp, 0, (size_t)N * 8, s);
    st.copy(pst, p, N);
    st.mask_p(pst);   // the tied unknowns: plus lips and constrained entries 0
    tetf_diag_a<<<st.nb(), 128, 0, s>>>(N, t->f_Sd.as<double>(), t->f_Cd.as<double>(), dt, t->f_mask.as<uint8_t>(),
                                        t->f_dAm.as<double>(), t->f_invdA.as<double>());
    std::vector<int8_t> prev(P), cur(P);
    bool have_prev = false;
    double rhat0 = -1.0, rhat = 0.0;
    int outer = 0, it = 0;
    long long inner = 0;
    for (it = 0;; ++it) {
        tetf_return_map<<<st.pb(), 128, 0, s>>>(st.geo(), u, du, t->f_dlie_n.as<double>(), fp.kn, fp.ks, fp.f, fp.tn0,
                                                fp.tau0[0], fp.tau0[1], t->f_state.as<int8_t>(), t->f_tn.as<double>(),
                                                t->f_dlie.as<double>(), t->f_T.as<double>(), t->f_F.as<double>(),
                                                t->f_dn.as<double>(), t->f_gs.as<double>(), t->f_D.as<double>());
        if ((rc = st.residual(u, pst, du, dp, dt, b1, b2))) return rc;
        rhat = std::sqrt(st.dot(n3, b1, b1, t->f_invdK.as<double>()) + st.dot(N, b2, b2, t->f_invdA.as<double>()));
        if (rhat0 < 0.0) rhat0 = rhat;
        const double shat = std::sqrt(st.dot(n3, ut, ut, t->f_dKm.as<double>()) + st.dot(N, pt, pt, t->f_dAm.as<double>()) +
                                      t->f0sq);
        cudaMemcpyAsync(cur.data(), t->f_state.p, P, cudaMemcpyDeviceToHost, s);
        const cudaError_t ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return t->set_err(GM_ECUDA, std::string("tet fault step: ") + cudaGetErrorString(ce));
        if (!std::isfinite(rhat)) return t->set_err(GM_ENAN, "tet fault step: non-finite residual");
        const bool same = have_prev && prev == cur;
        if (it > 0 && same && rhat <= opts->newton_rtol * std::max(rhat0, 1e-3 * shat)) break;
        if (it == opts->newton_maxit)
            return t->set_err(GM_ENEWTON, "tet fault step: Newton did not converge (rhat/rhat0=" +
                                              std::to_string(rhat / std::max(rhat0, 1e-300)) + ")");
        cudaMemsetAsync(t->f_err.p, 0, sizeof(int), s);
        tetf_bjac_build<<<st.nb(), 128, 0, s>>>(N, P, t->f_Kblk.as<double>(), t->f_n2p.as<int>(), t->f_area.as<double>(),
                                               t->f_D.as<double>(), t->f_mask.as<uint8_t>(), t->f_Kinv.as<double>(),
                                               t->f_err.as<int>());
        tpcg_pair_inverse<<<st.pb(), 128, 0, s>>>(N, P, t->f_Kblk.as<double>(), t->f_pm.as<int>(), t->f_pp.as<int>(),
                                                  t->f_area.as<double>(), t->f_D.as<double>(), t->f_mask.as<uint8_t>(),
                                                  t->f_Pinv.as<double>(), t->f_err.as<int>());
        if (st.f32) {
            tpcg_cast<float><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(9LL * N, t->f_Kinv.as<double>(), t->f_Kinv32.as<float>());
            tpcg_cast<float><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(36LL * P, t->f_Pinv.as<double>(), t->f_Pinv32.as<float>());
            tpcg_cast<float><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(6LL * P, t->f_D.as<double>(), t->f_D32.as<float>());
        }
        int herr = 0;
        cudaMemcpyAsync(&herr, t->f_err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (herr) return t->set_err(GM_ENAN, "tet fault step: singular nodal or lip-pair block of K_T");
        if ((rc = st.prevost(b1, b2, x1, x2, dt, *opts, &outer, &inner))) return rc;
        st.axpy(n3, 1.0, x1, du);
        st.axpy(N, 1.0, x2, dp);
        prev = cur;
        have_prev = true;
    }
    // accept: u += du, p += dp (plus lips of tied pairs from their partners), history
    st.axpy(n3, 1.0, du, u);
    st.axpy(N, 1.0, dp, pst);
    st.copy(p, pst, N);
    if (t->tied) tetf_expand<<<st.pb(), 128, 0, s>>>(st.geo(), p);
    cudaMemcpyAsync(t->f_dlie_n.p, t->f_dlie.p, 2LL * P * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(t->f_flags_acc.p, t->f_state.p, P, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(t->f_gs_acc.p, t->f_gs.p, 2LL * P * 8, cudaMemcpyDeviceToDevice, s);
    std::vector<double> F(P), tn(P), dn(P);
    cudaMemcpyAsync(F.data(), t->f_F.p, P * 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(tn.data(), t->f_tn.p, P * 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(dn.data(), t->f_dn.p, P * 8, cudaMemcpyDeviceToHost, s);
    const cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return t->set_err(GM_ECUDA, std::string("tet fault step: ") + cudaGetErrorString(ce));
    if (rep) {
        rep->newton = it;
        rep->outer = outer;
        rep->inner_k = inner;
        rep->inner_a = 0;
        rep->applies = st.applies;
        rep->rhat = rhat;
        rep->rhat0 = rhat0;
        rep->n_open = rep->n_stick = rep->n_slip = 0;
        double my = INFINITY, mn = INFINITY;
        for (int i = 0; i < P; ++i) {
            if (cur[i] == GM_OPEN) rep->n_open++;
            else if (cur[i] == GM_STICK) rep->n_stick++;
            else rep->n_slip++;
            if (cur[i] != GM_OPEN && fp.f * tn[i] > 0) my = std::min(my, std::fabs(F[i]) / (fp.f * tn[i]));
            if (fp.tn0 > 0) mn = std::min(mn, std::fabs(fp.tn0 - fp.kn * dn[i]) / fp.tn0);
        }
        rep->min_yield_margin = my;
        rep->min_normal_margin = mn;
    }
    return GM_OK;
}

extern "C" int gm_tet_fault_state(gm_tet* t, int8_t* flags, double* slip, double* dlie)
{
    if (!t) return GM_EINVAL;
    if (!t->has_fault) return t->set_err(GM_ESTATE, "tet fault state: no fault");
    cudaSetDevice(t->device);
    const long long P = t->P;
    cudaError_t ce = cudaSuccess;
    if (flags && ce == cudaSuccess) ce = cudaMemcpy(flags, t->f_flags_acc.p, P, cudaMemcpyDeviceToHost);
    if (slip && ce == cudaSuccess) ce = cudaMemcpy(slip, t->f_gs_acc.p, 2 * P * 8, cudaMemcpyDeviceToHost);
    if (dlie && ce == cudaSuccess) ce = cudaMemcpy(dlie, t->f_dlie_n.p, 2 * P * 8, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return t->set_err(GM_ECUDA, std::string("tet fault state: ") + cudaGetErrorString(ce));
    return GM_OK;
}
