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
#include <cmath>
#include <string>
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
                                                           const T* xp, T* yu, T* yp)
{
    constexpr bool IN_U = (MODE & (TM_K | TM_AUP)) != 0;
    constexpr bool IN_P = (MODE & (TM_APU | TM_S | TM_C)) != 0;
    constexpr bool OUT_U = (MODE & (TM_K | TM_APU)) != 0;
    constexpr bool OUT_P = (MODE & (TM_AUP | TM_S | TM_C)) != 0;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    T au[3] = {T(0), T(0), T(0)};
    T ap = T(0);
    for (int q = rowptr[n]; q < rowptr[n + 1]; ++q) {
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
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace

struct gm_tet {
    int device = 0;
    std::string err;
    long long N = 0, M = 0;
    bool has_mesh = false, has_mat = false;
    double E = 0, nu = 0, alpha = 0, Mb = 0, k = 0, mu_f = 0;
    DBuf G64, G32, V64, V32, tets, rowptr, adj;
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
    if (n_nodes > (1LL << 29) || n_tets > (1LL << 29)) return t->set_err(GM_EINVAL, "tet mesh: too large");
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
    return GM_OK;
}

}  // extern "C"

namespace {

template <typename T, int MODE>
void launch(gm_tet* t, const TetCoef<T>& c, const T* xu, const T* xp, T* yu, T* yp, cudaStream_t s, const T* G,
            const T* V)
{
    const int N = (int)t->N;
    gm_tet_apply_kernel<T, MODE><<<(N + 127) / 128, 128, 0, s>>>(N, t->rowptr.as<int>(), t->adj.as<int>(),
                                                                t->tets.as<int>(), G, V, c, xu, xp, yu, yp);
}

template <typename T>
int apply_t(gm_tet* t, int which, const void* x, void* y, double dt, cudaStream_t s)
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
    case GM_OP_KT: launch<T, TM_K>(t, c, xu, nullptr, yu, nullptr, s, G, V); break;
    case GM_OP_APU: launch<T, TM_APU>(t, c, nullptr, xu, yu, nullptr, s, G, V); break;
    case GM_OP_AUP: launch<T, TM_AUP>(t, c, xu, nullptr, nullptr, yu, s, G, V); break;
    case GM_OP_A22: launch<T, TM_S | TM_C>(t, c, nullptr, xu, nullptr, yu, s, G, V); break;
    case GM_OP_J:
        c.cApu = T(-1);
        launch<T, TM_K | TM_APU | TM_AUP | TM_S | TM_C>(t, c, xu, xu + 3 * N, yu, yu + 3 * N, s, G, V);
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
