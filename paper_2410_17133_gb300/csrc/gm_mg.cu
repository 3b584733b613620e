// Geometric multigrid preconditioner for the FP32 K_T inner solves.
//
// The inner solves of the partitioned scheme (Sec. 3.3.2) on K_T take
// thousands of block-Jacobi PCG iterations on the larger grids (their count
// grows with the grid size), so the FP32 K_T solves may use one V-cycle as the
// preconditioner instead.  The structured grid is halved in every direction
// within each of the two fault blocks (the fault node plane kf and the block
// boundaries stay node planes), down to about 10 cells per direction:
//   - coarse operators are rediscretised: each coarse level is a child
//     context with E averaged over the 8 fine elements of a coarse element,
//     the Dirichlet bits and the fault tangent D of the coincident fine node
//     or pair, and the reference cell of twice the spacing;
//   - prolongation is trilinear interpolation inside each block, restriction
//     its transpose (full weighting), so the cycle never couples the lips;
//   - smoothing is a degree-2 Chebyshev polynomial in M^-1 K_T with M the
//     nodal / lip-pair block Jacobi, over [0.15, 1.15] x the largest
//     eigenvalue (power iteration at set-up); the coarsest level runs a
//     degree-24 polynomial (by default) over [0.003, 1.15] x that eigenvalue.
// Pre- and post-smoothing use the same polynomial, so the cycle is a
// symmetric positive definite operator and plain PCG stays valid.
// Everything is enqueued on the caller's stream without host synchronisation
// (except the one-time set-up), so the PCG iterations remain graph-capturable.
#include <cmath>
#include <type_traits>
#include <cstdlib>

#include "gm_internal.cuh"
#include "gm_pcgvec.cuh"

namespace {

constexpr int MG_MAX_LEVELS = 8;
constexpr int MG_SMOOTH_DEG = 2;
constexpr int MG_MAX_COARSE_DEG = 32;
// tuning (environment, read at set-up): coarse grids below the first keep at
// least GM_MG_MIN_CELLS cells per direction (default 10; the first coarse
// grid only needs 2); the coarsest level runs a Chebyshev polynomial of degree
// GM_MG_COARSE_DEG (default 24).  Measured on the 160^3 inclined workload
// (FP32-refined), with the interval ends below: stopping at 10^3 instead of
// 5^3 and a degree-24 coarsest polynomial take the step from 0.81 s to 0.55 s
// (K_T iterations per step about 400 -> 220).
constexpr int MG_MIN_CELLS = 10;
constexpr int MG_COARSE_DEG = 24;
int mg_min_cells()
{
    const char* v = std::getenv("GM_MG_MIN_CELLS");
    const int n = v ? std::atoi(v) : MG_MIN_CELLS;
    return n >= 1 ? n : MG_MIN_CELLS;
}
// smoothing degree of the other levels: GM_MG_SMOOTH_DEG (default 2)
int mg_smooth_deg()
{
    const char* v = std::getenv("GM_MG_SMOOTH_DEG");
    const int n = v ? std::atoi(v) : MG_SMOOTH_DEG;
    return (n >= 1 && n <= MG_MAX_COARSE_DEG) ? n : MG_SMOOTH_DEG;
}
// lower ends of the Chebyshev intervals as fractions of the largest
// eigenvalue: GM_MG_SMOOTH_LO (smoothing, default 0.15) and GM_MG_COARSE_LO
// (coarsest level, default 0.003)
double mg_frac(const char* name, double dflt)
{
    const char* v = std::getenv(name);
    const double f = v ? std::atof(v) : dflt;
    return (f > 0.0 && f < 1.0) ? f : dflt;
}
int mg_coarse_deg()
{
    const char* v = std::getenv("GM_MG_COARSE_DEG");
    const int n = v ? std::atoi(v) : MG_COARSE_DEG;
    return (n >= 1 && n <= MG_MAX_COARSE_DEG) ? n : MG_COARSE_DEG;
}

// grid of a level's vector kernels: one thread per node up to the fixed grid
int mg_blocks(long long N)
{
    const long long b = (N + 255) / 256;
    return (int)(b < GM_RED_BLOCKS ? b : GM_RED_BLOCKS);
}

__device__ inline void mg_plane(const GridDesc& g, int kk, int* o, int* up)
{
    if (g.kf < 0) { *o = kk; *up = 0; return; }
    *up = kk > g.kf ? 1 : 0;
    *o = *up ? kk - 1 : kk;
}
__device__ inline int mg_ext(const GridDesc& g, int o, int up) { return (g.kf >= 0 && up) ? o + 1 : o; }

// b_c = R (b_f - y_f): full weighting inside each block; constrained coarse
// components 0.  y_f may be null (then r_f = b_f).
template <typename T>
__global__ void mg_restrict_kernel(GridDesc F, GridDesc Cg, const T* bf, const T* yf, T* bc,
                                   const uint8_t* maskc, const int* skip)
{
    if (skip && *skip) return;
    const long long nc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (nc >= Cg.N) return;
    const int ic = (int)(nc % (Cg.nx + 1));
    const long long t = nc / (Cg.nx + 1);
    const int jc = (int)(t % (Cg.ny + 1)), kkc = (int)(t / (Cg.ny + 1));
    int oc, up;
    mg_plane(Cg, kkc, &oc, &up);
    const int olo = (F.kf >= 0 && up) ? F.kf : 0;
    const int ohi = (F.kf >= 0 && !up) ? F.kf : F.nz;
    T acc[3] = {T(0), T(0), T(0)};
    for (int dk = -1; dk <= 1; ++dk) {
        const int o = 2 * oc + dk;
        if (o < olo || o > ohi) continue;
        const T wz = dk ? T(0.5) : T(1);
        const long long kk = mg_ext(F, o, up);
        for (int dj = -1; dj <= 1; ++dj) {
            const int j = 2 * jc + dj;
            if (j < 0 || j > F.ny) continue;
            const T wy = dj ? T(0.5) : T(1);
            for (int di = -1; di <= 1; ++di) {
                const int i = 2 * ic + di;
                if (i < 0 || i > F.nx) continue;
                const T w = wz * wy * (di ? T(0.5) : T(1));
                const long long f = i + (long long)(F.nx + 1) * (j + (long long)(F.ny + 1) * kk);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T r = bf[c * F.N + f] - (yf ? yf[c * F.N + f] : T(0));
                    acc[c] = fma(w, r, acc[c]);
                }
            }
        }
    }
    const unsigned m = maskc[nc];
#pragma unroll
    for (int c = 0; c < 3; ++c) bc[c * Cg.N + nc] = ((m >> c) & 1u) ? T(0) : acc[c];
}

// x_f += P x_c: trilinear interpolation inside each block; constrained fine
// components unchanged.
template <typename T>
__global__ void mg_prolong_kernel(GridDesc F, GridDesc Cg, const T* xc, T* xf, const uint8_t* maskf,
                                  const int* skip)
{
    if (skip && *skip) return;
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F.N) return;
    const int i = (int)(f % (F.nx + 1));
    const long long t = f / (F.nx + 1);
    const int j = (int)(t % (F.ny + 1)), kk = (int)(t / (F.ny + 1));
    int o, up;
    mg_plane(F, kk, &o, &up);
    int pi[2], pj[2], po[2];
    T wi[2], wj[2], wo[2];
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, no = (o & 1) ? 2 : 1;
    pi[0] = i >> 1; pi[1] = (i + 1) >> 1; wi[0] = wi[1] = (i & 1) ? T(0.5) : T(1);
    pj[0] = j >> 1; pj[1] = (j + 1) >> 1; wj[0] = wj[1] = (j & 1) ? T(0.5) : T(1);
    po[0] = o >> 1; po[1] = (o + 1) >> 1; wo[0] = wo[1] = (o & 1) ? T(0.5) : T(1);
    T acc[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < no; ++a) {
        const long long kkc = mg_ext(Cg, po[a], up);
        for (int b = 0; b < nj; ++b)
            for (int e = 0; e < ni; ++e) {
                const T w = wo[a] * wj[b] * wi[e];
                const long long nc = pi[e] + (long long)(Cg.nx + 1) * (pj[b] + (long long)(Cg.ny + 1) * kkc);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] = fma(w, xc[c * Cg.N + nc], acc[c]);
            }
    }
    const unsigned m = maskf[f];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (!((m >> c) & 1u)) xf[c * F.N + f] += acc[c];
}

// Fault tangent of the coarse pairs: that of the coincident fine pair.
__global__ void mg_inject_d_kernel(GridDesc F, GridDesc Cg, const double* d64f, double* d64c, float* d32c)
{
    const long long qc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (qc >= Cg.nb) return;
    const int ic = (int)(qc % (Cg.nx + 1)), jc = (int)(qc / (Cg.nx + 1));
    const long long qf = 2LL * ic + (long long)(F.nx + 1) * (2LL * jc);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double v = d64f[q * F.nb + qf];
        d64c[q * Cg.nb + qc] = v;
        d32c[q * Cg.nb + qc] = (float)v;
    }
}

// Cohesive term of K_T for the smoother (FaultK.D null: y already holds it).
template <typename T>
struct FaultK {
    const T* D;            // 6 per pair (symmetric 3x3), or null
    const uint8_t* mask;
    T Aq;                  // area of one fault quad
    int nx, ny;
};

// One Chebyshev step: r = b - y (y null: x = 0, r = b), z = M^-1 r,
// d = c1 d + c2 z (c1 = 0: d = c2 z), x = x + d (xzero: x = d).  With fk.D
// set, y holds the bulk product only and the pair thread adds
// +-A_i D [[x]] to the two lips first (the fault rows of K_T).
// mode bits: CHEB_XZERO (x = 0 before the step), CHEB_D_FROM_X (the previous
// d is x: the step after an x = 0 step, which then need not store d) and
// CHEB_NO_D (the last step of a polynomial: d is not needed afterwards).
// The nodal block inverses are read as MT: bf16 in the FP32 smoother (a
// preconditioner only needs to be fixed and SPD; halving its bytes cuts the
// smoothing step's traffic), T in the FP64 one.
enum : int { CHEB_XZERO = 1, CHEB_D_FROM_X = 2, CHEB_NO_D = 4 };
template <typename T, typename MT>
__device__ inline T mg_ld(const MT* p)
{
    if constexpr (std::is_same<MT, __nv_bfloat16>::value) return (T)__bfloat162float(*p);
    else return (T)*p;
}
template <typename T, typename MT>
__global__ void __launch_bounds__(256) mg_cheb_kernel(long long N, const T* b, const T* y, T* x, T* d,
                                                      const MT* mi, PairPrec<T> pp, const double* coef, int mode,
                                                      const int* skip, FaultK<T> fk)
{
    if (skip && *skip) return;
    const T c1 = (T)coef[0], c2 = (T)coef[1];
    const bool xzero = (mode & CHEB_XZERO) != 0, dfx = (mode & CHEB_D_FROM_X) != 0, keepd = (mode & CHEB_NO_D) == 0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const long long dd = n - pp.lo;
        if (pp.inv != nullptr && dd >= 0 && dd < 2 * pp.nb) {
            if (dd >= pp.nb) continue;                 // upper lip: done with its pair
            const long long nd[2] = {n, n + pp.nb};
            T r6[6], z6[6];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long k = c * N + nd[s];
                    r6[3 * s + c] = b[k] - (y ? y[k] : T(0));
                }
            if (fk.D != nullptr && y != nullptr) {
                const int pi = (int)(dd % (fk.nx + 1)), pj = (int)(dd / (fk.nx + 1));
                const int nqi = (pi > 0) + (pi < fk.nx), nqj = (pj > 0) + (pj < fk.ny);
                const T Ai = fk.Aq * T(0.25) * T(nqi * nqj);
                const unsigned mm = fk.mask[nd[0]], mp = fk.mask[nd[1]];
                T j3[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T up = ((mp >> c) & 1u) ? T(0) : x[c * N + nd[1]];
                    const T um = ((mm >> c) & 1u) ? T(0) : x[c * N + nd[0]];
                    j3[c] = up - um;
                }
                const T* D = fk.D;
                const long long P = pp.nb;
                const T d00 = D[dd], d01 = D[P + dd], d02 = D[2 * P + dd];
                const T d11 = D[3 * P + dd], d12 = D[4 * P + dd], d22 = D[5 * P + dd];
                const T f[3] = {Ai * (d00 * j3[0] + d01 * j3[1] + d02 * j3[2]),
                                Ai * (d01 * j3[0] + d11 * j3[1] + d12 * j3[2]),
                                Ai * (d02 * j3[0] + d12 * j3[1] + d22 * j3[2])};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!((mm >> c) & 1u)) r6[c] += f[c];        // y_- -= f
                    if (!((mp >> c) & 1u)) r6[3 + c] -= f[c];    // y_+ += f
                }
            }
            gm_pair_apply(pp, dd, r6, z6);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long k = c * N + nd[s];
                    const T xv = xzero ? T(0) : x[k];
                    const T dn = c1 == T(0) ? c2 * z6[3 * s + c] : fma(c1, dfx ? xv : d[k], c2 * z6[3 * s + c]);
                    if (keepd) d[k] = dn;
                    x[k] = xv + dn;
                }
            continue;
        }
        T r[3], z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = b[c * N + n] - (y ? y[c * N + n] : T(0));
        {
            const T i0 = mg_ld<T>(mi + n), i1 = mg_ld<T>(mi + N + n), i2 = mg_ld<T>(mi + 2 * N + n);
            const T i3 = mg_ld<T>(mi + 3 * N + n), i4 = mg_ld<T>(mi + 4 * N + n), i5 = mg_ld<T>(mi + 5 * N + n);
            z[0] = i0 * r[0] + i1 * r[1] + i2 * r[2];
            z[1] = i1 * r[0] + i3 * r[1] + i4 * r[2];
            z[2] = i2 * r[0] + i4 * r[1] + i5 * r[2];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long k = c * N + n;
            const T xv = xzero ? T(0) : x[k];
            const T dn = c1 == T(0) ? c2 * z[c] : fma(c1, dfx ? xv : d[k], c2 * z[c]);
            if (keepd) d[k] = dn;
            x[k] = xv + dn;
        }
    }
}

// Per-block partial sums of v.v (set-up only; summed on the host in block order).
__global__ void __launch_bounds__(256) mg_norm2_kernel(long long n, const float* v, double* part)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc += (double)v[i] * (double)v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void mg_scale_kernel(long long n, float* v, float a)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] *= a;
}

// Deterministic start vector of the power iteration (free components only).
__global__ void mg_seed_kernel(long long N, const uint8_t* mask, float* v)
{
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const unsigned m = mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            unsigned h = (unsigned)(n * 3 + c) * 2654435761u;
            h ^= h >> 15;
            h *= 2246822519u;
            h ^= h >> 13;
            v[c * N + n] = ((m >> c) & 1u) ? 0.f : ((float)(h & 0xffffu) / 32768.f - 1.f);
        }
    }
}

template <typename T>
PairPrec<T> level_pairs(gm_ctx* x)
{
    PairPrec<T> pp{nullptr, x->g.nb, -1};
    if (x->g.kf >= 0 && x->pair_prec) {
        if constexpr (sizeof(T) == 8) pp.inv = x->dKpair64.as<T>();
        else pp.inv = x->dKpair32.as<T>();
        pp.lo = (long long)x->g.kf * x->g.nb;
    }
    return pp;
}

// storage type of the smoother's nodal block inverses
template <typename T>
struct MinvType { using type = T; };
template <>
struct MinvType<float> { using type = __nv_bfloat16; };

template <typename T>
const typename MinvType<T>::type* level_inv(gm_ctx* x)
{
    if constexpr (sizeof(T) == 8) return x->dKinv64.as<T>();
    else return x->dKinv16.as<__nv_bfloat16>();
}

// the level's vectors in the solve precision
template <typename T>
struct LV { T* b; T* x; T* d; T* y; };
template <typename T>
LV<T> lv(const MGLevel& L)
{
    if constexpr (sizeof(T) == 8) return LV<T>{L.b64, L.x64, L.d64, L.y64};
    else return LV<T>{L.b, L.x, L.d, L.y};
}

bool coarsenable(const gm_ctx* x, bool first)
{
    if (x->nx % 2 || x->ny % 2 || x->nz % 2) return false;
    const int mc = first ? 2 : mg_min_cells();
    if (x->nx / 2 < mc || x->ny / 2 < mc || x->nz / 2 < mc) return false;
    if (x->has_fault) {
        if (x->kf_orig % 2) return false;
        if (x->kf_orig / 2 < 1 || (x->nz - x->kf_orig) / 2 < 1) return false;
    }
    return true;
}

// Child context one level coarser than x (E, k averaged over the 8 fine
// elements; Dirichlet bits of the coincident fine node).
int make_child(gm_ctx* x, gm_ctx** out)
{
    gm_ctx* ch = nullptr;
    int rc = gm_create(&ch, x->device);
    if (rc) return x->set_err(rc, "multigrid: cannot create a coarse level");
    const int nxc = x->nx / 2, nyc = x->ny / 2, nzc = x->nz / 2;
    const double hc[3] = {2 * x->h[0], 2 * x->h[1], 2 * x->h[2]};
    auto fail = [&](const char* what) {
        const std::string m = std::string("multigrid: ") + what + ": " + gm_last_error(ch);
        gm_destroy(ch);
        return x->set_err(GM_EINVAL, m);
    };
    if (gm_mesh_structured(ch, nxc, nyc, nzc, x->origin, hc, x->shear)) return fail("mesh");
    if (x->has_fault && gm_fault_plane(ch, x->kf_orig / 2, &x->fp)) return fail("fault");
    const long long nelc = (long long)nxc * nyc * nzc;
    std::vector<double> Ec(nelc, 0.0), kc(nelc, 0.0);
    for (int ek = 0; ek < nzc; ++ek)
        for (int ej = 0; ej < nyc; ++ej)
            for (int ei = 0; ei < nxc; ++ei) {
                const long long e = ei + (long long)nxc * (ej + (long long)nyc * ek);
                for (int a = 0; a < 8; ++a) {
                    const long long ef = (2 * ei + (a & 1)) + (long long)x->nx *
                                         ((2 * ej + ((a >> 1) & 1)) + (long long)x->ny * (2 * ek + (a >> 2)));
                    Ec[e] += 0.125 * x->E[ef];
                    kc[e] += 0.125 * x->kperm[ef];
                }
            }
    if (gm_set_materials(ch, Ec.data(), kc.data(), nelc, x->nu, x->alpha, x->M, x->mu_f)) return fail("materials");
    const long long npc = nzc + 1 + (x->has_fault ? 1 : 0);
    const long long nbc = (long long)(nxc + 1) * (nyc + 1), Nc = nbc * npc;
    const long long Nf = x->N;
    const int kff = x->has_fault ? x->kf_orig : -1, kfc = x->has_fault ? x->kf_orig / 2 : -1;
    std::vector<uint8_t> fixc(4 * Nc, 0);
    for (long long kkc = 0; kkc < npc; ++kkc) {
        const bool up = kfc >= 0 && kkc > kfc;
        const long long oc = up ? kkc - 1 : kkc;
        const long long kkf = (kff >= 0 && up) ? 2 * oc + 1 : 2 * oc;
        for (int jc = 0; jc <= nyc; ++jc)
            for (int ic = 0; ic <= nxc; ++ic) {
                const long long nc = ic + (long long)(nxc + 1) * (jc + (long long)(nyc + 1) * kkc);
                const long long nf = 2LL * ic + (long long)(x->nx + 1) * (2LL * jc + (long long)(x->ny + 1) * kkf);
                for (int d = 0; d < 4; ++d) fixc[d * Nc + nc] = x->fixed[d * Nf + nf];
            }
    }
    if (gm_set_dirichlet(ch, fixc.data(), 4 * Nc)) return fail("dirichlet");
    ch->pair_prec = x->pair_prec;
    if (gm_assemble_or_bind(ch)) return fail("bind");
    *out = ch;
    return GM_OK;
}

int apply_kt(gm_ctx* x, const float* v, float* y, const int* skip, cudaStream_t s)
{
    return gm_launch_apply_f32(x, GM_MODE_KT, 1.0, 0.0, 0.0, 0.0, 0.0, v, nullptr, y, nullptr, s, skip);
}
int apply_kt(gm_ctx* x, const double* v, double* y, const int* skip, cudaStream_t s)
{
    return gm_launch_apply_f64(x, GM_MODE_KT, 1.0, 0.0, 0.0, 0.0, 0.0, v, nullptr, y, nullptr, s, skip);
}

int apply_kb(gm_ctx* x, const float* v, float* y, const int* skip, cudaStream_t s)
{
    return gm_launch_bulk_k_f32(x, v, y, s, skip);
}
int apply_kb(gm_ctx* x, const double* v, double* y, const int* skip, cudaStream_t s)
{
    return gm_launch_bulk_k_f64(x, v, y, s, skip);
}

template <typename T>
FaultK<T> level_fault(gm_ctx* x)
{
    FaultK<T> fk{nullptr, x->dmask.as<uint8_t>(), T(x->Aq), x->nx, x->ny};
    // with lip-pair blocks every pair has one thread that can add its rows
    if (x->g.kf >= 0 && x->pair_prec) {
        if constexpr (sizeof(T) == 8) fk.D = x->dD64.as<T>();
        else fk.D = x->dD32.as<T>();
    }
    return fk;
}

template <typename T>
int cheb_step(gm_ctx* c, const MGLevel& L, int k, int mode, bool fused, const int* skip, cudaStream_t s)
{
    gm_ctx* x = L.cx;
    const LV<T> v = lv<T>(L);
    const double* cf = c->mg_coef.as<double>() + 2 * (L.coef_off + k);
    FaultK<T> fk = level_fault<T>(x);
    if (!fused) fk.D = nullptr;
    const bool xzero = (mode & CHEB_XZERO) != 0;
    mg_cheb_kernel<T><<<mg_blocks(x->N), 256, 0, s>>>(x->N, v.b, xzero ? nullptr : v.y, v.x, v.d, level_inv<T>(x),
                                                    level_pairs<T>(x), cf, mode, skip, fk);
    GM_LAUNCHED(c);
    return GM_OK;
}

// deg Chebyshev steps on level L (from x = 0 if xzero).  The operator products
// are bulk-only launches when the smoother adds the fault rows itself.
template <typename T>
int smooth(gm_ctx* c, const MGLevel& L, int deg, bool xzero, const int* skip, cudaStream_t s)
{
    const LV<T> v = lv<T>(L);
    const bool fused = level_fault<T>(L.cx).D != nullptr;
    int rc;
    for (int k = 0; k < deg; ++k) {
        const bool z0 = xzero && k == 0;
        if (!z0) {
            rc = fused ? apply_kb(L.cx, v.x, v.y, skip, s) : apply_kt(L.cx, v.x, v.y, skip, s);
            if (rc) return rc;
        }
        // after an x = 0 step d equals x; the last step's d is never read
        const int mode = (z0 ? CHEB_XZERO : 0) | (xzero && k == 1 ? CHEB_D_FROM_X : 0) |
                         (z0 || k == deg - 1 ? CHEB_NO_D : 0);
        if ((rc = cheb_step<T>(c, L, k, mode, fused, skip, s))) return rc;
    }
    return GM_OK;
}

template <typename T>
int vcycle(gm_ctx* c, size_t l, const int* skip, cudaStream_t s)
{
    const MGLevel& L = c->mg[l];
    const LV<T> v = lv<T>(L);
    int rc;
    if (l + 1 == c->mg.size()) return smooth<T>(c, L, L.deg, true, skip, s);
    if ((rc = smooth<T>(c, L, L.deg, true, skip, s))) return rc;
    if ((rc = apply_kt(L.cx, v.x, v.y, skip, s))) return rc;
    const MGLevel& C = c->mg[l + 1];
    const LV<T> w = lv<T>(C);
    mg_restrict_kernel<T><<<(int)((C.cx->N + 255) / 256), 256, 0, s>>>(L.cx->g, C.cx->g, v.b, v.y, w.b,
                                                                        C.cx->dmask.as<uint8_t>(), skip);
    GM_LAUNCHED(c);
    if ((rc = vcycle<T>(c, l + 1, skip, s))) return rc;
    mg_prolong_kernel<T><<<(int)((L.cx->N + 255) / 256), 256, 0, s>>>(L.cx->g, C.cx->g, w.x, v.x,
                                                                       L.cx->dmask.as<uint8_t>(), skip);
    GM_LAUNCHED(c);
    return smooth<T>(c, L, L.deg, false, skip, s);
}

// Chebyshev coefficients (c1, c2) of step k over [lo, hi] (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 12.1, written as updates of x).
void cheb_coefs(double lo, double hi, int deg, std::vector<double>& out)
{
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    out.push_back(0.0);
    out.push_back(1.0 / theta);
    for (int k = 1; k < deg; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        out.push_back(rn * rho);
        out.push_back(2.0 * rn / delta);
        rho = rn;
    }
}

int norm2(gm_ctx* c, long long n, const float* v, double* out)
{
    double* part = c->dpart.as<double>();
    mg_norm2_kernel<<<GM_RED_BLOCKS, 256>>>(n, v, part);
    GM_LAUNCHED(c);
    std::vector<double> h(GM_RED_BLOCKS);
    GM_CUDA_TRY(c, cudaMemcpy(h.data(), part, GM_RED_BLOCKS * sizeof(double), cudaMemcpyDeviceToHost));
    double t = 0.0;
    for (double x : h) t += x;
    *out = t;
    return GM_OK;
}

// Largest eigenvalue of M^-1 K_T on level L by 12 power iterations.
int estimate_lmax(gm_ctx* c, MGLevel& L)
{
    gm_ctx* x = L.cx;
    const long long n3 = 3 * x->N;
    float* v = L.b;     // scratch during set-up
    mg_seed_kernel<<<GM_RED_BLOCKS, 256>>>(x->N, x->dmask.as<uint8_t>(), v);
    GM_LAUNCHED(c);
    double nv;
    int rc;
    if ((rc = norm2(c, n3, v, &nv))) return rc;
    if (!(nv > 0)) { L.lmax = 1.0; return GM_OK; }
    mg_scale_kernel<<<GM_RED_BLOCKS, 256>>>(n3, v, (float)(1.0 / std::sqrt(nv)));
    GM_LAUNCHED(c);
    const double* unit = c->mg_coef.as<double>();   // (0, 1): z = M^-1 b
    double lam = 0.0;
    for (int it = 0; it < 12; ++it) {
        if ((rc = apply_kt(x, v, L.y, nullptr, 0))) return rc;
        FaultK<float> nofk = level_fault<float>(x);
        nofk.D = nullptr;
        mg_cheb_kernel<float><<<GM_RED_BLOCKS, 256>>>(x->N, L.y, nullptr, L.x, L.d, level_inv<float>(x),
                                                      level_pairs<float>(x), unit, CHEB_XZERO | CHEB_NO_D, nullptr,
                                                      nofk);
        GM_LAUNCHED(c);
        double nw;
        if ((rc = norm2(c, n3, L.x, &nw))) return rc;
        lam = std::sqrt(nw);
        if (!(lam > 0) || !std::isfinite(lam)) return c->set_err(GM_ENAN, "multigrid: eigenvalue estimate failed");
        GM_CUDA_TRY(c, cudaMemcpy(v, L.x, n3 * sizeof(float), cudaMemcpyDeviceToDevice));
        mg_scale_kernel<<<GM_RED_BLOCKS, 256>>>(n3, v, (float)(1.0 / lam));
        GM_LAUNCHED(c);
    }
    L.lmax = lam;
    return GM_OK;
}

int inject_and_refresh(gm_ctx* c, cudaStream_t s)
{
    for (size_t l = 1; l < c->mg.size(); ++l) {
        gm_ctx* f = c->mg[l - 1].cx;
        gm_ctx* x = c->mg[l].cx;
        if (x->g.kf >= 0) {
            mg_inject_d_kernel<<<(int)((x->g.nb + 255) / 256), 256, 0, s>>>(f->g, x->g, f->dD64.as<double>(),
                                                                           x->dD64.as<double>(), x->dD32.as<float>());
            GM_LAUNCHED(c);
        }
        int rc = gm_launch_block_jacobi(x, s);
        if (rc) return c->set_err(rc, std::string("multigrid: ") + gm_last_error(x));
    }
    return GM_OK;
}

int build(gm_ctx* c)
{
    c->mg.clear();
    MGLevel L0;
    L0.cx = c;
    c->mg.push_back(L0);
    gm_ctx* cur = c;
    while (coarsenable(cur, c->mg.size() == 1) && (int)c->mg.size() < MG_MAX_LEVELS) {
        gm_ctx* ch = nullptr;
        int rc = make_child(cur, &ch);
        if (rc) { gm_mg_release(c); return rc; }
        MGLevel L;
        L.cx = ch;
        L.b = ch->k_b32.as<float>();
        L.x = ch->k_x32.as<float>();
        L.d = ch->k_z32.as<float>();
        L.y = ch->k_q32.as<float>();
        L.b64 = ch->k_r.as<double>();
        L.x64 = ch->k_x64.as<double>();
        L.d64 = ch->k_z.as<double>();
        L.y64 = ch->k_q.as<double>();
        c->mg.push_back(L);
        cur = ch;
    }
    if (c->mg.size() < 2) {
        c->mg.clear();
        return c->set_err(GM_EINVAL, "multigrid: grid cannot be coarsened (even cell counts and fault index needed)");
    }
    const long long n3 = 3 * c->N;
    GM_CUDA_TRY(c, c->mg_d0.alloc(n3 * sizeof(float)));
    GM_CUDA_TRY(c, c->mg_y0.alloc(n3 * sizeof(float)));
    c->mg[0].d = c->mg_d0.as<float>();
    c->mg[0].y = c->mg_y0.as<float>();
    // coefficient slot 0 = (0, 1) for the eigenvalue estimate; levels follow
    std::vector<double> coef = {0.0, 1.0};
    GM_CUDA_TRY(c, c->mg_coef.alloc(2 * sizeof(double) * (1 + MG_MAX_LEVELS * MG_MAX_COARSE_DEG)));
    GM_CUDA_TRY(c, cudaMemcpy(c->mg_coef.p, coef.data(), 2 * sizeof(double), cudaMemcpyHostToDevice));
    int rc;
    if ((rc = inject_and_refresh(c, 0))) { gm_mg_release(c); return rc; }
    // level 0 vectors during set-up: PCG scratch of the context
    c->mg[0].b = c->k_b32.as<float>();
    c->mg[0].x = c->k_x32.as<float>();
    for (auto& L : c->mg)
        if ((rc = estimate_lmax(c, L))) { gm_mg_release(c); return rc; }
    c->mg[0].b = nullptr;
    c->mg[0].x = nullptr;
    int off = 1;
    for (size_t l = 0; l < c->mg.size(); ++l) {
        MGLevel& L = c->mg[l];
        const bool last = l + 1 == c->mg.size();
        L.deg = last ? mg_coarse_deg() : mg_smooth_deg();
        L.coef_off = off;
        const double hi = 1.15 * L.lmax;
        const double lo = (last ? mg_frac("GM_MG_COARSE_LO", 0.003) : mg_frac("GM_MG_SMOOTH_LO", 0.15)) * L.lmax;
        cheb_coefs(lo, hi, L.deg, coef);
        off += L.deg;
    }
    GM_CUDA_TRY(c, cudaMemcpy(c->mg_coef.p, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice));
    GM_CUDA_TRY(c, cudaDeviceSynchronize());
    return GM_OK;
}

}  // namespace

void gm_mg_release(gm_ctx* c)
{
    for (size_t l = 1; l < c->mg.size(); ++l) gm_destroy(c->mg[l].cx);
    c->mg.clear();
    c->mg_d0.release();
    c->mg_y0.release();
    c->mg_d0_64.release();
    c->mg_y0_64.release();
    c->mg_coef.release();
}

int gm_mg_prepare(gm_ctx* c, int prec, cudaStream_t s)
{
    if (c->mg.empty()) {
        // the one-time build runs on the default stream and reads the block
        // Jacobi that the caller may still be computing on s
        GM_CUDA_TRY(c, cudaStreamSynchronize(s));
        if (int rc = build(c)) return rc;
    } else if (int rc = inject_and_refresh(c, s)) {
        return rc;
    }
    if (prec == GM_F64 && !c->mg_d0_64.p) {
        GM_CUDA_TRY(c, cudaStreamSynchronize(s));
        GM_CUDA_TRY(c, c->mg_d0_64.alloc(3 * c->N * sizeof(double)));
        GM_CUDA_TRY(c, c->mg_y0_64.alloc(3 * c->N * sizeof(double)));
        c->mg[0].d64 = c->mg_d0_64.as<double>();
        c->mg[0].y64 = c->mg_y0_64.as<double>();
    }
    return GM_OK;
}

int gm_mg_vcycle(gm_ctx* c, int prec, const void* r, void* z, const int* skip, cudaStream_t s)
{
    if (c->mg.empty()) return c->set_err(GM_ESTATE, "multigrid: not prepared");
    if (prec == GM_F64 && !c->mg[0].d64) return c->set_err(GM_ESTATE, "multigrid: FP64 vectors not prepared");
    long long before = 0;
    for (size_t l = 1; l < c->mg.size(); ++l) before += c->mg[l].cx->launches;
    int rc;
    if (prec == GM_F64) {
        c->mg[0].b64 = static_cast<double*>(const_cast<void*>(r));
        c->mg[0].x64 = static_cast<double*>(z);
        rc = vcycle<double>(c, 0, skip, s);
    } else {
        c->mg[0].b = static_cast<float*>(const_cast<void*>(r));
        c->mg[0].x = static_cast<float*>(z);
        rc = vcycle<float>(c, 0, skip, s);
    }
    long long after = 0;
    for (size_t l = 1; l < c->mg.size(); ++l) after += c->mg[l].cx->launches;
    c->launches += after - before;   // the coarse levels' kernels count as this context's
    return rc;
}
