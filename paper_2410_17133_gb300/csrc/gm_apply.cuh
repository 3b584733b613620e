// Fault (interface) part of the operators and the apply launchers.
//
// Per node pair i (lips i-, i+), nodal quadrature with weight A_i:
//   cohesive tangent     y_u+- += +- cKf A_i D_i [[x_u]]                  (Sec. 3.3.1)
//   lip pressure force   y_u+- += +- cApu A_i <p> n                       (App. B, Eq. afpdp read as
//                                                                          the transpose of Eq. afdpd)
//   aperture change      y_p(<p>) += cAup A_i n.[[x_u]]                    (App. B, Eq. afdpd)
//   fracture storage     y_p(<p>) += cS A_i (w/M_F) <p>                    (Sec. 3.2.3)
//   longitudinal flow    y_p(<p>) += cC (w k_par/mu) sum_quads L_q <p>     (Sec. 3.2.3, Eq. flux_decompose_operators)
//   transverse flow      y_p+- += +- cC A_i k_perp/(mu w) [[p]]            (Sec. 3.2.3)
// with <p> = (p+ + p-)/2 and [[.]] = (.)+ - (.)- (Eq. operators).  Terms on <p>
// are distributed half/half to the two lips; with tied lips (k_perp infinite)
// the single pressure lives on the lower lip and the upper-lip bulk row,
// written raw by the bulk kernel, is folded into it here.
//
// In PCG mode this kernel is the last writer of the lip rows, so it also adds
// p.(A p) over the lip nodes to the bulk kernel's per-CTA partials, and its last
// block sums all partials in a fixed order and forms alpha = (r.z)/(p.Ap).
#pragma once

#include <algorithm>
#include <type_traits>

#include "gm_bulk.cuh"
#include "gm_bulk32.cuh"

__device__ inline void gm_pcg_alpha_from(PcgScalars* sc, double pq)
{
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
        sc->status = isfinite(pq) ? GM_ENOCONV : GM_ENAN;
        sc->done = 1;
        sc->alpha = 0.0;
    } else {
        sc->alpha = sc->rz / pq;
    }
}

// Sum n partials in a fixed order with one block (thread-strided, then a tree).
__device__ inline double gm_block_sum_fixed(const double* part, int n)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) acc += ((volatile const double*)part)[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    return tot;
}

template <typename T, int MODE, bool PCG>
__global__ void __launch_bounds__(256)
gm_fault_apply_kernel(const FaultArgs<T> a)
{
    constexpr bool DO_KF = (MODE & GM_M_KF) != 0;
    constexpr bool DO_APU = (MODE & GM_M_APU) != 0;
    constexpr bool DO_AUP = (MODE & GM_M_AUP) != 0;
    constexpr bool DO_S = (MODE & GM_M_S) != 0;
    constexpr bool DO_C = (MODE & GM_M_C) != 0;
    constexpr bool OUT_U = (MODE & (GM_M_K | GM_M_KF | GM_M_APU)) != 0;
    constexpr bool OUT_P = (MODE & (GM_M_AUP | GM_M_S | GM_M_C)) != 0;
    constexpr bool BULK_P = (MODE & (GM_M_AUP | GM_M_S | GM_M_C)) != 0;   // bulk wrote y_p

    if (a.skip != nullptr && *a.skip != 0) return;
    const GridDesc& g = a.g;
    const long long P = g.nb;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = g.N;
    double dot = 0.0;
    if (i < P) {
        const int pi = (int)(i % (g.nx + 1)), pj = (int)(i / (g.nx + 1));
        const long long nm = i + g.nb * g.kf, np = nm + g.nb;
        const unsigned mm = a.mask[nm], mp = a.mask[np];
        const int nqi = (pi > 0) + (pi < g.nx), nqj = (pj > 0) + (pj < g.ny);
        const T Ai = a.Aq * T(0.25) * T(nqi * nqj);

        auto pval = [&](long long node) -> T {   // masked pressure input
            return ((a.mask[node] >> 3) & 1u) ? T(0) : a.xp[node];
        };
        // pressure of the mid-plane <p> at pair id q
        auto pav = [&](long long q) -> T {
            const long long m = q + g.nb * g.kf;
            if (g.tied) return pval(m);
            return T(0.5) * (pval(m) + pval(m + g.nb));
        };

        T jmp[3] = {T(0), T(0), T(0)};
        if constexpr (DO_KF || DO_AUP) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T up = ((mp >> c) & 1u) ? T(0) : a.xu[c * N + np];
                const T um = ((mm >> c) & 1u) ? T(0) : a.xu[c * N + nm];
                jmp[c] = up - um;
            }
        }
        T p_av = T(0);
        if constexpr (DO_APU || DO_S) p_av = pav(i);

        if constexpr (OUT_U) {
            T f[3] = {T(0), T(0), T(0)};
            if constexpr (DO_KF) {
                const T d00 = a.D[i], d01 = a.D[P + i], d02 = a.D[2 * P + i];
                const T d11 = a.D[3 * P + i], d12 = a.D[4 * P + i], d22 = a.D[5 * P + i];
                const T s = a.cKf * Ai;
                f[0] = s * (d00 * jmp[0] + d01 * jmp[1] + d02 * jmp[2]);
                f[1] = s * (d01 * jmp[0] + d11 * jmp[1] + d12 * jmp[2]);
                f[2] = s * (d02 * jmp[0] + d12 * jmp[1] + d22 * jmp[2]);
                if (a.cons != 0) {
                    const T co = (T)a.tauc[3 * P + i];
                    if (co != T(0)) {
                        const T tg[3] = {(T)a.tauc[i], (T)a.tauc[P + i], (T)a.tauc[2 * P + i]};
                        const T* v = a.cons == 1 ? tg : a.n;      // left vector
                        const T* w = a.cons == 1 ? a.n : tg;      // right vector
                        const T sc = s * co * (w[0] * jmp[0] + w[1] * jmp[1] + w[2] * jmp[2]);
#pragma unroll
                        for (int c = 0; c < 3; ++c) f[c] = fma(sc, v[c], f[c]);
                    }
                }
            }
            if constexpr (DO_APU) {
                const T s = a.cApu * Ai * p_av;
#pragma unroll
                for (int c = 0; c < 3; ++c) f[c] = fma(s, a.n[c], f[c]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!((mp >> c) & 1u)) {
                    const T y = a.yu[c * N + np] + f[c];
                    a.yu[c * N + np] = y;
                    if constexpr (PCG) dot += (double)a.xu[c * N + np] * (double)y;
                }
                if (!((mm >> c) & 1u)) {
                    const T y = a.yu[c * N + nm] - f[c];
                    a.yu[c * N + nm] = y;
                    if constexpr (PCG) dot += (double)a.xu[c * N + nm] * (double)y;
                }
            }
        }

        if constexpr (OUT_P) {
            T dav = T(0);    // contribution on the <p> test function
            if constexpr (DO_AUP) dav = a.cAup * Ai * (a.n[0] * jmp[0] + a.n[1] * jmp[1] + a.n[2] * jmp[2]);
            if constexpr (DO_S) dav = fma(a.cS * Ai * a.stor, p_av, dav);
            T dtr = T(0);    // transverse contribution on [[p]]
            if constexpr (DO_C) {
                T lap = T(0);
#pragma unroll
                for (int dq = 0; dq < 4; ++dq) {
                    const int qi = pi - 1 + (dq & 1), qj = pj - 1 + (dq >> 1);
                    if (qi < 0 || qi >= g.nx || qj < 0 || qj >= g.ny) continue;
                    const int b = (pi - qi) + 2 * (pj - qj);
#pragma unroll
                    for (int b2 = 0; b2 < 4; ++b2) {
                        const long long q = (qi + (b2 & 1)) + (long long)(g.nx + 1) * (qj + (b2 >> 1));
                        lap = fma(a.Lf[b * 4 + b2], pav(q), lap);
                    }
                }
                dav = fma(a.cC * a.lcoef, lap, dav);
                if (!g.tied) dtr = a.cC * Ai * a.tcoef * (pval(np) - pval(nm));
            }
            if (g.tied) {
                T v = dav;
                if constexpr (BULK_P) v += a.yp[nm] + a.yp[np];
                const T y = ((mm >> 3) & 1u) ? T(0) : v;
                a.yp[nm] = y;
                a.yp[np] = T(0);
                if constexpr (PCG) dot += (double)pval(nm) * (double)y;
            } else {
                const T vp = T(0.5) * dav + dtr, vm = T(0.5) * dav - dtr;
                if (!((mp >> 3) & 1u)) {
                    const T y = a.yp[np] + vp;
                    a.yp[np] = y;
                    if constexpr (PCG) dot += (double)a.xp[np] * (double)y;
                }
                if (!((mm >> 3) & 1u)) {
                    const T y = a.yp[nm] + vm;
                    a.yp[nm] = y;
                    if constexpr (PCG) dot += (double)a.xp[nm] * (double)y;
                }
            }
        }
    }

    if constexpr (PCG) {
        __shared__ double sh[8];
        __shared__ bool last;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) s += sh[w];
            a.part[a.nbulk + blockIdx.x] = s;
            __threadfence();
            last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
        }
        __syncthreads();
        if (!last) return;
        __threadfence();
        const double pq = gm_block_sum_fixed(a.part, a.nbulk + (int)gridDim.x);
        if (threadIdx.x == 0) {
            gm_pcg_alpha_from(a.sc, pq);
            *a.counter = 0u;
        }
    }
}

// Without a fault, one block closes the p.Ap reduction of the bulk partials.
static __global__ void __launch_bounds__(256)
gm_pcg_alpha_finalize_kernel(const double* part, int n, PcgScalars* sc)
{
    if (sc->done) return;
    const double pq = gm_block_sum_fixed(part, n);
    if (threadIdx.x == 0) gm_pcg_alpha_from(sc, pq);
}

inline void gm_bulk_geometry(const gm_ctx* c, int* gx, int* gy, int* gz, int* zchunk)
{
    // chunk of node planes per CTA: aim for >= 4 CTAs per SM on the xy tiling
    *gx = (c->nx + 1 + 14) / 15;
    *gy = (c->ny + 1 + 14) / 15;
    const long long xy = (long long)(*gx) * (*gy);
    int nzc = (int)((4LL * c->sm_count + xy - 1) / xy);
    if (nzc < 1) nzc = 1;
    int zc = (c->g.nplanes + nzc - 1) / nzc;
    if (zc < 4) zc = 4;
    if (c->zchunk_override > 0) zc = c->zchunk_override;
    *zchunk = zc;
    *gz = (c->g.nplanes + zc - 1) / zc;
}

// Plane-chunk length of a bulk launch: the chunk count is chosen so that the
// CTAs fill whole waves of the resident slots, each CTA's march costing its
// planes plus the halo layer and the pipeline fill.
inline int gm_pick_zchunk(const gm_ctx* c, long long xy, int resident)
{
    const int np = c->g.nplanes;
    if (c->zchunk_override > 0) return std::max(2, c->zchunk_override);
    const long long slots = (long long)c->sm_count * std::max(resident, 1);
    int best = np;
    long long bestc = -1;
    for (int zc = 2; zc <= np; ++zc) {
        const long long chunks = (np + zc - 1) / zc;
        const long long waves = (xy * chunks + slots - 1) / slots;
        const long long cost = waves * (zc + 3);
        if (bestc < 0 || cost < bestc) { bestc = cost; best = zc; }
    }
    return best;
}

// FP32 bulk kernel (gm_bulk32.cuh): dynamic shared memory opt-in and resident
// CTAs per SM, set once per device (at bind, outside any stream capture).
template <int CLS, int MODE, bool PCG>
static int& gm_bulk32_resident(int dev)
{
    static int resident[64] = {};
    return resident[dev & 63];
}

template <int CLS, int MODE, bool PCG>
static int gm_bulk32_setup(int dev)
{
    constexpr size_t SMEM = gm32::smem_bytes<MODE, PCG>();
    int& r = gm_bulk32_resident<CLS, MODE, PCG>(dev);
    if (r > 0) return 0;
    cudaError_t e = cudaFuncSetAttribute(gm_bulk32_kernel<CLS, MODE, PCG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return (int)e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gm_bulk32_kernel<CLS, MODE, PCG>, gm32::NT, SMEM);
    if (e != cudaSuccess) return (int)e;
    r = std::max(n, 1);
    return 0;
}

// Launch; returns the number of CTAs.
template <int CLS, int MODE, bool PCG>
static int gm_bulk32_launch(gm_ctx* c, BulkArgs<float>& b, cudaStream_t s)
{
    constexpr size_t SMEM = gm32::smem_bytes<MODE, PCG>();
    const int dev = c->device;
    gm_bulk32_setup<CLS, MODE, PCG>(dev);
    const int resident = gm_bulk32_resident<CLS, MODE, PCG>(dev);
    const int gx = (c->nx + 1 + 14) / 15, gy = (c->ny + 1 + 14) / 15;
    const int zc = std::min(gm_pick_zchunk(c, (long long)gx * gy, resident), gm32::MAXPL - 2);
    const int gz = (c->g.nplanes + zc - 1) / zc;
    b.zchunk = zc;
#if GM32_PACKED_PRODUCTS
    gm_bulk32_kernel<CLS, MODE, PCG><<<dim3(gx, gy, gz), gm32::NT, SMEM, s>>>(b, c->R32p);
#else
    gm_bulk32_kernel<CLS, MODE, PCG><<<dim3(gx, gy, gz), gm32::NT, SMEM, s>>>(b, c->R32);
#endif
    return gx * gy * gz;
}

template <int MODE, bool PCG>
static int gm_bulk32_dispatch(gm_ctx* c, BulkArgs<float>& b, cudaStream_t s)
{
    switch (c->cls) {
    case GM_CLS_BOX: return gm_bulk32_launch<GM_CLS_BOX, MODE, PCG>(c, b, s);
    case GM_CLS_MONO: return gm_bulk32_launch<GM_CLS_MONO, MODE, PCG>(c, b, s);
    default: return gm_bulk32_launch<GM_CLS_GEN, MODE, PCG>(c, b, s);
    }
}

template <typename T>
inline FaultArgs<T> gm_fault_args(gm_ctx* c, double cK, double cApu, double cAup, double cS, double cC,
                                  bool kf_on)
{
    FaultArgs<T> f;
    f.g = c->g;
    f.cKf = T(kf_on ? cK : 0.0);
    f.cApu = T(cApu);
    f.cAup = T(cAup);
    f.cS = T(cS);
    f.cC = T(cC);
    f.Aq = T(c->Aq);
    for (int d = 0; d < 3; ++d) f.n[d] = T(c->nrm[d]);
    f.stor = T(c->fp.w0 / c->fp.MF);
    f.lcoef = T(c->fp.wk_par / c->mu_f);
    f.tcoef = T(c->fp.k_perp > 0 ? c->fp.k_perp / (c->mu_f * c->fp.w0) : 0.0);
    for (int q = 0; q < 16; ++q) f.Lf[q] = T(c->Lf[q]);
    f.mask = c->dmask.as<uint8_t>();
    f.skip = nullptr;
    f.tauc = c->dtauc.as<double>();
    f.cons = c->fault_cons;
    f.part = nullptr;
    f.nbulk = 0;
    f.counter = nullptr;
    f.sc = nullptr;
    return f;
}

template <typename T>
inline BulkArgs<T> gm_bulk_args(gm_ctx* c, double cK, double cApu, double cAup, double cS, double cC,
                                const T* E, const T* kap)
{
    BulkArgs<T> b;
    b.g = c->g;
    b.E = E;
    b.kap = kap;
    b.mask = c->dmask.as<uint8_t>();
    b.cK = T(cK);
    b.cApu = T(cApu * c->alpha);
    b.cAup = T(cAup * c->alpha);
    b.cS = T(cS / c->M);
    b.cC = T(cC);
    b.skip = nullptr;
    b.tflag = c->dtflag.as<uint8_t>();
    b.zu = nullptr; b.zp = nullptr; b.pu_new = nullptr; b.pp_new = nullptr;
    b.beta = nullptr; b.part = nullptr;
    b.fs = nullptr; b.cFS = T(0);
    return b;
}

template <typename T, int CLS, int MODE>
static void gm_apply_launch_t(gm_ctx* c, const RefOps<T>& R, double cK, double cApu, double cAup,
                              double cS, double cC, const T* xu, const T* xp, T* yu, T* yp,
                              const T* E, const T* kap, const T* D, cudaStream_t s, const int* skip)
{
    int gx, gy, gz, zchunk;
    gm_bulk_geometry(c, &gx, &gy, &gz, &zchunk);
    BulkArgs<T> b = gm_bulk_args<T>(c, cK, cApu, cAup, cS, cC, E, kap);
    b.zchunk = zchunk;
    b.xu = xu; b.xp = xp; b.yu = yu; b.yp = yp;
    b.skip = skip;
    constexpr int BULK = MODE & (GM_M_K | GM_M_APU | GM_M_AUP | GM_M_S | GM_M_C);
    if constexpr (std::is_same<T, float>::value && (BULK == GM_M_K || BULK == (GM_M_S | GM_M_C)))
        gm_bulk32_launch<CLS, BULK, false>(c, b, s);
    else
        gm_bulk_apply_kernel<T, CLS, BULK, false><<<dim3(gx, gy, gz), 256, 0, s>>>(b, R);
    c->applies++;
    c->launches++;
    // K_b alone has no fault term: the bulk kernel's product is complete
    constexpr bool FAULT_TERMS = (MODE & (GM_M_KF | GM_M_APU | GM_M_AUP | GM_M_S | GM_M_C)) != 0;
    if (FAULT_TERMS && c->g.kf >= 0) {
        FaultArgs<T> f = gm_fault_args<T>(c, cK, cApu, cAup, cS, cC, (MODE & GM_M_KF) != 0);
        f.xu = xu; f.xp = xp; f.yu = yu; f.yp = yp;
        f.D = D;
        f.skip = skip;
        const int nblk = (int)((c->g.nb + 255) / 256);
        gm_fault_apply_kernel<T, MODE, false><<<nblk, 256, 0, s>>>(f);
        c->launches++;
    }
}

template <typename T, int MODE>
static void gm_apply_dispatch_cls(gm_ctx* c, const RefOps<T>& R, double cK, double cApu, double cAup,
                                  double cS, double cC, const T* xu, const T* xp, T* yu, T* yp,
                                  const T* E, const T* kap, const T* D, cudaStream_t s,
                                  const int* skip)
{
    switch (c->cls) {
    case GM_CLS_BOX:
        gm_apply_launch_t<T, GM_CLS_BOX, MODE>(c, R, cK, cApu, cAup, cS, cC, xu, xp, yu, yp, E, kap, D, s, skip);
        break;
    case GM_CLS_MONO:
        gm_apply_launch_t<T, GM_CLS_MONO, MODE>(c, R, cK, cApu, cAup, cS, cC, xu, xp, yu, yp, E, kap, D, s, skip);
        break;
    default:
        gm_apply_launch_t<T, GM_CLS_GEN, MODE>(c, R, cK, cApu, cAup, cS, cC, xu, xp, yu, yp, E, kap, D, s, skip);
        break;
    }
}

// Fused PCG operator step for K_T (which 0) or A22 (which 1).
template <typename T, int CLS, int MODE>
static void gm_pcg_apply_t(gm_ctx* c, const RefOps<T>& R, const T* z, const T* p_old, T* p_new, T* q,
                           const T* E, const T* kap, const T* D, PcgScalars* sc, cudaStream_t s,
                           const T* fs)
{
    constexpr bool U = (MODE & GM_M_K) != 0;
    const double cK = U ? 1.0 : 0.0, cS = U ? 0.0 : 1.0, cC = U ? 0.0 : c->dt;
    int gx, gy, gz, zchunk;
    gm_bulk_geometry(c, &gx, &gy, &gz, &zchunk);
    int nbulk = gx * gy * gz;
    double* part = c->dpart.as<double>();
    BulkArgs<T> b = gm_bulk_args<T>(c, cK, 0, 0, cS, cC, E, kap);
    b.zchunk = zchunk;
    b.skip = &sc->done;
    b.beta = &sc->beta;
    b.part = part;
    b.fs = fs;
    b.cFS = T(1);
    if (U) { b.xu = p_old; b.zu = z; b.pu_new = p_new; b.yu = q; b.xp = nullptr; b.yp = nullptr; }
    else { b.xp = p_old; b.zp = z; b.pp_new = p_new; b.yp = q; b.xu = nullptr; b.yu = nullptr; }
    constexpr int BULK = MODE & (GM_M_K | GM_M_S | GM_M_C);
    if constexpr (std::is_same<T, float>::value)
        nbulk = gm_bulk32_launch<CLS, BULK, true>(c, b, s);
    else
        gm_bulk_apply_kernel<T, CLS, BULK, true><<<dim3(gx, gy, gz), 256, 0, s>>>(b, R);
    c->applies++;
    c->launches++;
    if (c->g.kf >= 0) {
        FaultArgs<T> f = gm_fault_args<T>(c, cK, 0, 0, cS, cC, U);
        if (U) { f.xu = p_new; f.yu = q; f.xp = nullptr; f.yp = nullptr; }
        else { f.xp = p_new; f.yp = q; f.xu = nullptr; f.yu = nullptr; }
        f.D = D;
        f.skip = &sc->done;
        f.part = part;
        f.nbulk = nbulk;
        f.counter = c->dcount.as<unsigned>();
        f.sc = sc;
        const int nblk = (int)((c->g.nb + 255) / 256);
        gm_fault_apply_kernel<T, MODE, true><<<nblk, 256, 0, s>>>(f);
        c->launches++;
    } else {
        gm_pcg_alpha_finalize_kernel<<<1, 256, 0, s>>>(part, nbulk, sc);
        c->launches++;
    }
}

template <typename T, int MODE>
static void gm_pcg_apply_dispatch(gm_ctx* c, const RefOps<T>& R, const T* z, const T* p_old, T* p_new,
                                  T* q, const T* E, const T* kap, const T* D, PcgScalars* sc,
                                  cudaStream_t s, const T* fs)
{
    switch (c->cls) {
    case GM_CLS_BOX: gm_pcg_apply_t<T, GM_CLS_BOX, MODE>(c, R, z, p_old, p_new, q, E, kap, D, sc, s, fs); break;
    case GM_CLS_MONO: gm_pcg_apply_t<T, GM_CLS_MONO, MODE>(c, R, z, p_old, p_new, q, E, kap, D, sc, s, fs); break;
    default: gm_pcg_apply_t<T, GM_CLS_GEN, MODE>(c, R, z, p_old, p_new, q, E, kap, D, sc, s, fs); break;
    }
}
