// FP32 bulk kernel of the inner-solve operators: K_b (elasticity, 3 fields)
// and S + dt C (storage + Darcy, 1 field), plain (y = A x) or fused with the
// PCG direction update (p = z + beta p_old, q = A p, per-CTA partials of p.q).
//
// Same operator as gm_bulk.cuh (Sec. 3.2.1-3.2.2; the element products of the
// Ap-type applications of Sec. 3.3.2) and the same tiling of the grid into
// CTAs (15 x 15 owned node columns plus a halo, a chunk of node planes
// marched upwards), organised for issue throughput:
//  - a thread owns one face column and two face rows (faces lo and hi); the
//    two faces run in lock step as packed FP32 pairs (add/sub/mul/fma .f32x2),
//    so each arithmetic instruction serves two elements, and the shared node
//    row between them is transformed once per plane;
//  - each element multiplies only the entries of the parity-basis operators
//    that the cell's pattern allows (gm_make_parpat), with coefficients
//    duplicated in the kernel parameters so a pair instruction reads them
//    directly;
//  - node planes are staged into a 4-deep shared-memory ring with cp.async,
//    three planes ahead of the march; each thread stages the nodes it later
//    fixes up (masks, z + beta p_old), so a plane needs one barrier;
//  - face sums are combined across the x neighbour with warp shuffles and
//    across the y neighbour through one shared word per field.
// No atomics; results are deterministic.
#pragma once

#include "gm_internal.cuh"

namespace gm32 {

constexpr int TXN = 16;                // threads per tile row (face columns)
constexpr int TYB = 8;                 // thread rows (two face rows each)
constexpr int NT = TXN * TYB;          // 128 threads
constexpr int TN = 17;                 // tile nodes per row and column
constexpr int TILE = TN * TN;          // 289 staged nodes per plane
constexpr int RS = 24;                 // shared row stride (conflict-free pair reads)
constexpr int PLANE = TN * RS;         // floats per staged field plane
constexpr int NS = 4;                  // ring stages
constexpr int DA = 3;                  // planes staged ahead of the march
constexpr int NSLOT = (TILE + NT - 1) / NT;
constexpr int MAXPL = 512;             // staged planes per CTA at most (chunk + 2 halo planes)

#ifndef GM32_PACKED
#define GM32_PACKED 0
#endif
#if GM32_PACKED
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
#else
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c)
{
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#endif
// products with a duplicated constant coefficient: packed, or two scalar FMAs
// that read the coefficient from the parameter bank
#ifndef GM32_PACKED_PRODUCTS
#define GM32_PACKED_PRODUCTS GM32_PACKED
#endif
__device__ __forceinline__ float2 pcfma(float2 k, float2 b, float2 c)
{
#if GM32_PACKED_PRODUCTS
    return pfma(k, b, c);
#else
    return make_float2(fmaf(k.x, b.x, c.x), fmaf(k.x, b.y, c.y));
#endif
}
__device__ __forceinline__ float2 pcmul(float2 k, float2 b)
{
#if GM32_PACKED_PRODUCTS
    return pmul(k, b);
#else
    return make_float2(k.x * b.x, k.x * b.y);
#endif
}
// scalar coefficient (the FP32 parameter block without duplication)
__device__ __forceinline__ float2 pcfma(float k, float2 b, float2 c)
{
    return make_float2(fmaf(k, b.x, c.x), fmaf(k, b.y, c.y));
}
__device__ __forceinline__ float2 pcmul(float k, float2 b) { return make_float2(k * b.x, k * b.y); }
__device__ __forceinline__ float2 dup(float k) { return make_float2(k, k); }
__device__ __forceinline__ float2 dup(float2 k) { return k; }

// kernel parameter block of the pattern coefficients
#if GM32_PACKED_PRODUCTS
using Ref32 = RefPairs32;
#else
using Ref32 = RefOps<float>;
#endif

__device__ __forceinline__ void cp4(unsigned dst, const void* src, int bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int MODE, bool PCG>
constexpr size_t smem_bytes()
{
    constexpr int NF = MODE == GM_M_K ? 3 : 1;
    constexpr int NIN = PCG ? 2 * NF : NF;
    return sizeof(float) * (size_t)NS * NIN * PLANE + sizeof(unsigned) * (size_t)NS * TILE +
           sizeof(float) * 2 * NF * NT + sizeof(double) * 4 + MAXPL;
}

}  // namespace gm32

// CTAs per SM the register budget is sized for: the elasticity product that
// also writes the PCG direction gets the budget of 2 CTAs, where it runs
// without spills (at 3 it spilled and ran about 3x slower than the plain one)
template <int MODE, bool PCG>
constexpr int gm32_min_blocks() { return MODE == GM_M_K ? (PCG ? 2 : 3) : 4; }

template <int CLS, int MODE, bool PCG>
__global__ void __launch_bounds__(gm32::NT, gm32_min_blocks<MODE, PCG>())
gm_bulk32_kernel(const BulkArgs<float> a, const __grid_constant__ gm32::Ref32 R)
{
    using namespace gm32;
    constexpr bool DO_K = MODE == GM_M_K;
    static_assert(MODE == GM_M_K || MODE == (GM_M_S | GM_M_C), "K or S + dt C");
    constexpr int NF = DO_K ? 3 : 1;
    constexpr int NIN = PCG ? 2 * NF : NF;
    constexpr unsigned MBITS = DO_K ? 7u : 8u;
    constexpr ParPat PP = gm_make_parpat(CLS);

    if (a.skip != nullptr && *a.skip != 0) return;

    extern __shared__ __align__(16) unsigned char gm32_smem[];
    float* s_in = reinterpret_cast<float*>(gm32_smem);                   // [NS][NIN][PLANE]
    unsigned* s_mw = reinterpret_cast<unsigned*>(s_in + NS * NIN * PLANE); // [NS][TILE] mask words
    float* s_x = reinterpret_cast<float*>(s_mw + NS * TILE);              // [2][NF][NT]
    double* s_red = reinterpret_cast<double*>(s_x + 2 * NF * NT);         // [4]
    uint8_t* s_flag = reinterpret_cast<uint8_t*>(s_red + 4);               // [MAXPL] constrained tile-planes

    const GridDesc& g = a.g;
    const int tid = threadIdx.x;
    const int tx = tid & 15, tyb = tid >> 4;
    const int x0 = blockIdx.x * 15, y0 = blockIdx.y * 15;
    const int r0 = 2 * tyb;                       // tile row of the lo face's bottom nodes
    const int N = (int)g.N, nb = (int)g.nb, rowlen = g.nx + 1;
    const int fi = x0 - 1 + tx, fj0 = y0 - 1 + r0;
    const bool fx = fi >= 0 && fi < g.nx;
    const bool vlo = fx && fj0 >= 0 && fj0 < g.ny;
    const bool vhi = fx && fj0 + 1 >= 0 && fj0 + 1 < g.ny;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nplanes);
    const float* xin = DO_K ? (PCG ? a.zu : a.xu) : (PCG ? a.zp : a.xp);     // staged array 0
    const float* pin = DO_K ? a.xu : a.xp;                                   // PCG: p_old
    float* yout = DO_K ? a.yu : a.yp;
    float* pnew = DO_K ? a.pu_new : a.pp_new;
    const float beta = PCG ? (float)(*a.beta) : 0.f;

    auto layer_exists = [&](int kb) -> bool { return kb >= 0 && kb + 1 < g.nplanes && kb != g.kf; };
    auto layer_index = [&](int kb) -> int { return (g.kf >= 0 && kb > g.kf) ? kb - 1 : kb; };

    const int kbeg = (z0 > 0 && layer_exists(z0 - 1)) ? z0 - 1 : z0;
    const int klast = (z1 < g.nplanes && layer_exists(z1 - 1)) ? z1 : z1 - 1;
    for (int i = tid; i <= klast - kbeg; i += NT)
        s_flag[i] = a.tflag != nullptr ? a.tflag[((kbeg + i) * (int)gridDim.y + (int)blockIdx.y) * (int)gridDim.x +
                                                 (int)blockIdx.x]
                                       : (uint8_t)1;
    __syncthreads();

    // staged nodes of this thread: tile index tid + NT s
    int s_off[NSLOT], s_pos[NSLOT];
    bool s_in_grid[NSLOT];
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        const int idx = tid + NT * s;
        const int ni = idx % TN, nj = idx / TN;
        const int gi = x0 - 1 + ni, gj = y0 - 1 + nj;
        s_in_grid[s] = idx < TILE && gi >= 0 && gi <= g.nx && gj >= 0 && gj <= g.ny;
        s_off[s] = gi + rowlen * gj;
        s_pos[s] = idx < TILE ? nj * RS + ni : -1;
    }
    const unsigned s_in_u = (unsigned)__cvta_generic_to_shared(s_in);
    const unsigned s_mw_u = (unsigned)__cvta_generic_to_shared(s_mw);

    // cp.async of plane k into ring slot k % NS (values of every staged array,
    // and for each node the aligned mask word holding its byte)
    auto stage = [&](int k) {
        const int st = k & (NS - 1);
        const bool fl = s_flag[k - kbeg] != 0;
        const int pb = k * nb;
        // a tied upper lip reads the pressure (and its constraint) of the lower lip
        const int pbp = (!DO_K && g.tied && k == g.kf + 1) ? pb - nb : pb;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (s_pos[s] < 0) continue;
            const bool ok = s_in_grid[s];
            const int node = pbp + s_off[s];
            const int nodec = ok ? node : 0;
            const int bytes = ok ? 4 : 0;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                cp4(s_in_u + 4u * (unsigned)((st * NIN + f) * PLANE + s_pos[s]), xin + f * N + nodec, bytes);
                if constexpr (PCG)
                    cp4(s_in_u + 4u * (unsigned)((st * NIN + NF + f) * PLANE + s_pos[s]), pin + f * N + nodec, bytes);
            }
            if (fl) cp4(s_mw_u + 4u * (unsigned)(st * TILE + tid + NT * s), a.mask + (nodec & ~3), bytes);
        }
    };
    // after the thread's own copies of plane k landed: constrained inputs to
    // zero, PCG mode forms z + beta p_old in place
    auto fixup = [&](int k) {
        const int st = k & (NS - 1);
        const bool fl = s_flag[k - kbeg] != 0;
        if (!PCG && !fl) return;
        const int pbp = (!DO_K && g.tied && k == g.kf + 1) ? (k - 1) * nb : k * nb;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (s_pos[s] < 0 || !s_in_grid[s]) continue;
            const int node = pbp + s_off[s];
            const unsigned m = fl ? (s_mw[st * TILE + tid + NT * s] >> (8 * (node & 3))) & 0xffu : 0u;
            float* v = s_in + st * NIN * PLANE + s_pos[s];
            if constexpr (PCG) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const unsigned bit = DO_K ? (1u << f) : 8u;
                    const float t = fmaf(beta, v[(NF + f) * PLANE], v[f * PLANE]);
                    v[f * PLANE] = (m & bit) ? 0.f : t;
                }
            } else {
                if (m & MBITS) {
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const unsigned bit = DO_K ? (1u << f) : 8u;
                        if (m & bit) v[f * PLANE] = 0.f;
                    }
                }
            }
        }
    };

    // xy part of the forward transform of plane k for the faces lo and hi:
    // t[q], q = sx + 2 sy, as pairs (lo, hi); own values of the tile nodes
    // (tx, r0) and (tx, r0 + 1) and their mask bytes
    float2 tb[NF][4], tt[NF][4];
    float2 own_cur[NF], own_prev[NF];
    unsigned m_cur = 0, m_prev = 0;
    auto fwd = [&](int k) {
        const int st = k & (NS - 1);
        const float* base = s_in + st * NIN * PLANE + r0 * RS + tx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float* b = base + f * PLANE;
            const float a0 = b[0], a1 = b[1], c0 = b[RS], c1 = b[RS + 1], e0 = b[2 * RS], e1 = b[2 * RS + 1];
            const float2 B0 = make_float2(a0, c0), B1 = make_float2(a1, c1);   // bottom rows of lo, hi
            const float2 T0 = make_float2(c0, e0), T1 = make_float2(c1, e1);   // top rows
            const float2 bp = padd(B0, B1), bm = psub(B0, B1), tp = padd(T0, T1), tm = psub(T0, T1);
            tt[f][0] = padd(bp, tp);
            tt[f][1] = padd(bm, tm);
            tt[f][2] = psub(bp, tp);
            tt[f][3] = psub(bm, tm);
            own_cur[f] = B0;
        }
        m_cur = 0;
        if (s_flag[k - kbeg] == 0) return;
        const int pb = k * nb + (y0 - 1 + r0) * rowlen + x0 - 1 + tx;
        const unsigned w0 = s_mw[st * TILE + r0 * TN + tx], w1 = s_mw[st * TILE + (r0 + 1) * TN + tx];
        // own mask words were staged by other threads at tile positions of
        // rows r0 and r0 + 1; their byte position follows the node index
        const int mb = (!DO_K && g.tied && k == g.kf + 1) ? pb - nb : pb;
        m_cur = ((w0 >> (8 * (mb & 3))) & 0xffu) | (((w1 >> (8 * ((mb + rowlen) & 3))) & 0xffu) << 8);
    };

    // Element layer between the planes of tb and tt for both faces: parity
    // values (xv), then per output field the pattern products, whose bottom
    // part is added into o and top part written to ot.
    constexpr int NXV = DO_K ? 24 : 8;
    auto parity = [&](float2 (&xv)[NXV]) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                if (DO_K && s == 0) continue;   // the constant displacement mode carries no force
                xv[f * 8 + s] = (s & 4) ? psub(tb[f][s & 3], tt[f][s & 3]) : padd(tb[f][s & 3], tt[f][s & 3]);
            }
    };
    auto outputs = [&](const float2 (&xv)[NXV], int c, float2 (&o)[4], float2 (&ot)[4], float2 ce, float2 cs) {
        if constexpr (DO_K) {
            auto row = [&](int s) -> float2 {
                float2 acc = make_float2(0.f, 0.f);
                bool first = true;
#pragma unroll
                for (int j = 0; j < 24; ++j)
                    if (PP.k[c * 8 + s][j] >= 0 && (j & 7) != 0) {
                        acc = first ? pcmul(R.K[PP.k[c * 8 + s][j]], xv[j])
                                    : pcfma(R.K[PP.k[c * 8 + s][j]], xv[j], acc);
                        first = false;
                    }
                return acc;
            };
            const float2 h0 = row(4);
            o[0] = pfma(ce, h0, o[0]);
            ot[0] = pmul(make_float2(-ce.x, -ce.y), h0);
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                const float2 lo = row(q), hi = row(q | 4);
                o[q] = pfma(ce, padd(lo, hi), o[q]);
                ot[q] = pmul(ce, psub(lo, hi));
            }
        } else {
            // ce = dt k/mu of the two elements, cs = their storage coefficient
            auto row = [&](int s) -> float2 {
                float2 acc = make_float2(0.f, 0.f);
                bool first = true;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (PP.l[s][j] >= 0) {
                        acc = first ? pcmul(R.L[PP.l[s][j]], xv[j]) : pcfma(R.L[PP.l[s][j]], xv[j], acc);
                        first = false;
                    }
                acc = pmul(ce, acc);
                return pfma(pmul(cs, dup(R.M[s])), xv[s], acc);
            };
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 lo = row(q), hi = row(q | 4);
                o[q] = padd(o[q], padd(lo, hi));
                ot[q] = psub(lo, hi);
            }
        }
    };

    // pending node stage: the two owned node rows of one plane
    float pn0[NF], pn1[NF];
    float2 pown[NF];
    unsigned pm = 0;
    int pplane = -1;
    double dot = 0.0;

    auto node_stage = [&]() {
        if (pplane < 0) return;
        const int m = pplane;
        const bool lip = g.kf >= 0 && (m == g.kf || m == g.kf + 1);
        const bool slave = !DO_K && g.tied && m == g.kf + 1;
        const int gi = x0 - 1 + tx, gj0 = y0 - 1 + r0;
        const int node0 = m * nb + gj0 * rowlen + gi;
        const float* below = s_x + (m & 1) * NF * NT;
        const bool colok = tx >= 1 && gi <= g.nx;
        const bool ok0 = colok && tyb >= 1 && gj0 <= g.ny;
        const bool ok1 = colok && gj0 + 1 <= g.ny;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const unsigned bit = DO_K ? (1u << f) : 8u;
            if (ok0) {
                const float v = pn0[f] + below[f * NT + tid - 16];
                const float y = (!slave && (pm & bit)) ? 0.f : v;
                yout[f * N + node0] = y;
                if constexpr (PCG) {
                    const float p = slave ? 0.f : pown[f].x;
                    pnew[f * N + node0] = p;
                    if (!lip) dot += (double)p * (double)y;
                }
            }
            if (ok1) {
                const float v = pn1[f];
                const float y = (!slave && (pm & (bit << 8))) ? 0.f : v;
                yout[f * N + node0 + rowlen] = y;
                if constexpr (PCG) {
                    const float p = slave ? 0.f : pown[f].y;
                    pnew[f * N + node0 + rowlen] = p;
                    if (!lip) dot += (double)p * (double)y;
                }
            }
        }
        pplane = -1;
    };

#pragma unroll
    for (int i = 0; i < DA; ++i) {
        if (kbeg + i <= klast) stage(kbeg + i);
        cp_commit();
    }
    float2 carry[NF][4];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int q = 0; q < 4; ++q) carry[f][q] = make_float2(0.f, 0.f);
    // element coefficients of the next layer (prefetched one plane ahead)
    const float* coef = DO_K ? a.E : a.kap;
    auto load_coef = [&](int kb) -> float2 {
        if (!layer_exists(kb)) return make_float2(0.f, 0.f);
        const int e = fi + g.nx * (fj0 + g.ny * layer_index(kb));
        return make_float2(vlo ? coef[e] : 0.f, vhi ? coef[e + g.nx] : 0.f);
    };
    auto load_fs = [&](int kb) -> float2 {
        if (a.fs == nullptr || !layer_exists(kb)) return make_float2(0.f, 0.f);
        const int e = fi + g.nx * (fj0 + g.ny * layer_index(kb));
        return make_float2(vlo ? a.fs[e] : 0.f, vhi ? a.fs[e + g.nx] : 0.f);
    };
    float2 cnext = load_coef(kbeg);
    float2 fnext = DO_K ? make_float2(0.f, 0.f) : load_fs(kbeg);

    for (int k = kbeg; k <= klast + 1; ++k) {
        if (k <= klast) {
            cp_wait<DA - 1>();
            fixup(k);
        }
        __syncthreads();
        if (k + DA <= klast) stage(k + DA);
        cp_commit();
        node_stage();
        const float2 ccur = cnext, fcur = fnext;
        if (k <= klast) {
            fwd(k);
            cnext = load_coef(k);
            if constexpr (!DO_K) fnext = load_fs(k);
        }
        if (k - 1 >= kbeg) {
            // complete plane k - 1 field by field: the bottom contributions of
            // layer k - 1 are added to the carry (top contributions of layer
            // k - 2), the sums go through the inverse xy transform into the
            // pending node rows, and the layer's top contributions become the
            // next carry
            const int m = k - 1;
            const bool lay = k <= klast && layer_exists(m);
            const bool owned = m >= z0 && m < z1;
            float2 ce = make_float2(0.f, 0.f), cs = make_float2(0.f, 0.f);
            float2 xv[NXV];
            if (lay) {
                if constexpr (DO_K) {
                    ce = pmul(make_float2(a.cK, a.cK), ccur);
                } else {
                    ce = pmul(make_float2(a.cC, a.cC), ccur);
                    const float2 fsok = make_float2(vlo ? 1.f : 0.f, vhi ? 1.f : 0.f);
                    cs = pfma(make_float2(a.cFS, a.cFS), fcur, pmul(make_float2(a.cS, a.cS), fsok));
                }
                parity(xv);
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                float2 ot[4];
                if (lay) {
                    outputs(xv, f, carry[f], ot, ce, cs);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) ot[q] = make_float2(0.f, 0.f);
                }
                if (owned) {
                    const float2 o0 = carry[f][0], o1 = carry[f][1], o2 = carry[f][2], o3 = carry[f][3];
                    const float2 c0 = padd(o0, o1), c1 = psub(o0, o1), d0 = padd(o2, o3), d1 = psub(o2, o3);
                    const float2 P00 = padd(c0, d0), P10 = padd(c1, d1), P01 = psub(c0, d0), P11 = psub(c1, d1);
                    // node values of column tx (this thread) and tx + 1 (right neighbour)
                    const float l0 = P00.x, l1 = P01.x + P00.y, l2 = P01.y;
                    const float q0 = P10.x, q1 = P11.x + P10.y, q2 = P11.y;
                    const float u0 = __shfl_up_sync(0xffffffffu, q0, 1, 16);
                    const float u1 = __shfl_up_sync(0xffffffffu, q1, 1, 16);
                    const float u2 = __shfl_up_sync(0xffffffffu, q2, 1, 16);
                    pn0[f] = l0 + u0;
                    pn1[f] = l1 + u1;
                    s_x[(m & 1) * NF * NT + f * NT + tid] = l2 + u2;
                    pown[f] = own_prev[f];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) carry[f][q] = ot[q];
            }
            if (owned) {
                pm = m_prev;
                pplane = m;
            }
        }
        if (k <= klast) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
#pragma unroll
                for (int q = 0; q < 4; ++q) tb[f][q] = tt[f][q];
                own_prev[f] = own_cur[f];
            }
            m_prev = m_cur;
        }
    }
    __syncthreads();
    node_stage();

    if constexpr (PCG) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = dot;
        __syncthreads();
        if (tid == 0) {
            const double sacc = ((s_red[0] + s_red[1]) + s_red[2]) + s_red[3];
            const int cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            a.part[cta] = sacc;
        }
    }
}
