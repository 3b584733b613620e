// Fault (interface) part of the operators and the apply launcher.
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
#pragma once

#include "gm_bulk.cuh"

template <typename T, int MODE>
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
    if (i >= P) return;
    const int pi = (int)(i % (g.nx + 1)), pj = (int)(i / (g.nx + 1));
    const long long N = g.N;
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
        }
        if constexpr (DO_APU) {
            const T s = a.cApu * Ai * p_av;
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] = fma(s, a.n[c], f[c]);
        }
        if constexpr (DO_KF || DO_APU) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!((mp >> c) & 1u)) a.yu[c * N + np] += f[c];
                if (!((mm >> c) & 1u)) a.yu[c * N + nm] -= f[c];
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
            a.yp[nm] = ((mm >> 3) & 1u) ? T(0) : v;
            a.yp[np] = T(0);
        } else {
            const T vp = T(0.5) * dav + dtr, vm = T(0.5) * dav - dtr;
            if (!((mp >> 3) & 1u)) a.yp[np] += vp;
            if (!((mm >> 3) & 1u)) a.yp[nm] += vm;
        }
    }
}

template <typename T, int CLS, int MODE>
static void gm_apply_launch_t(gm_ctx* c, const RefOps<T>& R, double cK, double cApu, double cAup,
                              double cS, double cC, const T* xu, const T* xp, T* yu, T* yp,
                              const T* E, const T* kap, const T* D, cudaStream_t s, const int* skip)
{
    BulkArgs<T> b;
    b.g = c->g;
    // chunk of node planes per CTA: aim for >= 4 CTAs per SM on the xy tiling
    const int gx = (c->nx + 1 + 14) / 15, gy = (c->ny + 1 + 14) / 15;
    const long long xy = (long long)gx * gy;
    int nzc = (int)((4LL * c->sm_count + xy - 1) / xy);
    if (nzc < 1) nzc = 1;
    int zchunk = (c->g.nplanes + nzc - 1) / nzc;
    if (zchunk < 4) zchunk = 4;
    const int gz = (c->g.nplanes + zchunk - 1) / zchunk;
    b.zchunk = zchunk;
    b.xu = xu; b.xp = xp; b.yu = yu; b.yp = yp;
    b.E = E; b.kap = kap;
    b.mask = c->dmask.as<uint8_t>();
    b.cK = T(cK);
    b.cApu = T(cApu * c->alpha);
    b.cAup = T(cAup * c->alpha);
    b.cS = T(cS / c->M);
    b.cC = T(cC);
    b.skip = skip;
    constexpr int BULK = MODE & (GM_M_K | GM_M_APU | GM_M_AUP | GM_M_S | GM_M_C);
    gm_bulk_apply_kernel<T, CLS, BULK><<<dim3(gx, gy, gz), 256, 0, s>>>(b, R);
    c->applies++;
    c->launches++;
    if (c->g.kf >= 0) {
        FaultArgs<T> f;
        f.g = c->g;
        f.xu = xu; f.xp = xp; f.yu = yu; f.yp = yp;
        f.D = D;
        f.mask = c->dmask.as<uint8_t>();
        f.cKf = T((MODE & GM_M_KF) ? cK : 0.0);
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
        f.skip = skip;
        const int nblk = (int)((c->g.nb + 255) / 256);
        gm_fault_apply_kernel<T, MODE><<<nblk, 256, 0, s>>>(f);
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
