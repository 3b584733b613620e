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
    cudaError_t alloc(size_t bytes) {
        if (p) { cudaFree(p); p = nullptr; }
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e != cudaSuccess) p = nullptr;
        return e;
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
    // time stepping
    std::vector<double> hG, hV;            // element gradients and volumes (host copy)
    std::vector<double> hX;                // node coordinates (host copy, point-major)
    std::vector<int> htv;                  // element vertices (host copy)
    std::vector<uint8_t> fixed;            // 4N: constrained (ux, uy, uz, p)
    std::vector<double> fu;                // 3N nodal forces
    DBuf mask, dfu, Kinv, Sd, Cd, part;
    DBuf w[14];
    bool prec_ready = false;
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
    t->hX.assign(nodes, nodes + 3 * N);
    t->hG.swap(G);
    t->hV.swap(V);
    t->htv.swap(tv);
    t->fixed.assign(4 * N, 0);
    t->fu.assign(3 * N, 0.0);
    t->prec_ready = false;
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

__global__ void tet_bjac(int N, const double* Kinv, const double* r, double* z)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double r0 = r[n], r1 = r[N + n], r2 = r[2 * N + n];
    for (int i = 0; i < 3; ++i)
        z[i * N + n] = Kinv[(3 * i) * N + n] * r0 + Kinv[(3 * i + 1) * N + n] * r1 + Kinv[(3 * i + 2) * N + n] * r2;
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

    // x = K^-1 b (x from 0), block-Jacobi PCG to ||r|| <= rtol ||b||
    int solve_k(const double* b, double* x, double rtol, int maxit, long long* its) {
        const long long n = 3LL * N;
        double *r = t->w[0].as<double>(), *z = t->w[1].as<double>(), *p = t->w[2].as<double>(), *q = t->w[3].as<double>();
        cudaMemsetAsync(x, 0, n * 8, s);
        cudaMemcpyAsync(r, b, n * 8, cudaMemcpyDeviceToDevice, s);
        const double rr0 = dot(n, r, r);
        if (rr0 == 0.0) return GM_OK;
        tet_bjac<<<blocks(), 128, 0, s>>>(N, t->Kinv.as<double>(), r, z);
        cudaMemcpyAsync(p, z, n * 8, cudaMemcpyDeviceToDevice, s);
        double rz = dot(n, r, z);
        for (int it = 1; it <= maxit; ++it) {
            int rc = apply(GM_OP_KB, p, q, 0.0);
            if (rc) return rc;
            const double pq = dot(n, p, q);
            if (!(pq > 0.0) || !std::isfinite(pq)) return t->set_err(GM_ENAN, "tet step: K not positive on a direction");
            const double a = rz / pq;
            axpy(n, a, p, x);
            axpy(n, -a, q, r);
            ++*its;
            if (dot(n, r, r) <= rtol * rtol * rr0) return GM_OK;
            tet_bjac<<<blocks(), 128, 0, s>>>(N, t->Kinv.as<double>(), r, z);
            const double rzn = dot(n, r, z);
            xpby(n, z, rzn / rz, p);
            rz = rzn;
        }
        return t->set_err(GM_ENOCONV, "tet step: K solve did not converge");
    }
};

// nodal 3x3 blocks of K and the diagonals of S and C (host), uploaded
int tet_prepare(gm_tet* t)
{
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
        (ce = t->dfu.put(fu.data(), 3 * N * 8)) != cudaSuccess || (ce = t->part.alloc(TET_RED_BLOCKS * 8)) != cudaSuccess)
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
