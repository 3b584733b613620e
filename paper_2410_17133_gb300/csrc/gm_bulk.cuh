// Matrix-free bulk operator kernel (Q1 hexahedra on an affine structured grid).
//
// Computes, for the operator blocks selected by MODE,
//   y_u = cK E_e K_e u - cApu A_e p            (Sec. 3.2.1; App. A Eq. Apdp)
//   y_p = cAup A_e^T u + cS S_e p + cC k_e L_e p   (Sec. 3.2.2; App. A Eq. Adpd)
// summed over elements, the Ap-type products evaluated element by element and
// gathered into the nodal vectors (Sec. 3.3.2).  All elements are the same
// parallelepiped, so the element matrices are those of one reference cell
// scaled by the element's E and k.  In the parity basis of the cell (the 8-point
// Walsh-Hadamard transform of the nodal values, one per field) the reference
// operators are sparse (gm_make_parpat); the kernel transforms, multiplies the
// allowed entries and transforms back.
//
// Work decomposition: a CTA of 16x16 threads owns 15x15 node columns and a
// chunk of node planes; it marches up the planes.  Thread (tx, ty) handles the
// element column (face) whose lower-left node is tile node (tx, ty), so each
// element is computed once inside the CTA, plus one halo column/row and one halo
// layer that the neighbour also computes.  The transform is split: the xy part
// is done once per node plane per face and reused by the element layers below
// and above the plane; the z part per element.  Element results are accumulated
// per face in registers across the plane, then each node sums its four faces
// from shared memory.  No atomics; results are deterministic.
//
// Pipelining: the node plane two levels up is fetched from global memory into
// registers while the current element layer is computed, and stored to the
// second of two shared plane buffers afterwards, so each plane step has two
// barriers and its global-load latency overlaps the arithmetic.
//
// PCG mode (inner solves, one field group): the input is the new search
// direction p = z + beta p_old formed while loading; the owner of each node
// writes p to a second buffer (p is double-buffered across iterations because
// neighbouring CTAs read p_old as halo), and the kernel leaves a per-CTA
// partial of p . (A p) over the nodes that are not on a fault lip.
#pragma once

#include "gm_internal.cuh"

// Resident CTAs per SM the register allocation must allow: FP64 is bound by
// the FP64 pipe at one CTA; the FP32 single-field-group box kernels fit three.
template <typename T, int CLS, int MODE>
constexpr int gm_bulk_min_blocks()
{
    return sizeof(T) == 8 ? 1
         : (CLS == GM_CLS_BOX && (MODE == GM_M_K || MODE == (GM_M_S | GM_M_C))) ? 3 : 2;
}

template <typename T, int CLS, int MODE, bool PCG>
__global__ void __launch_bounds__(256, gm_bulk_min_blocks<T, CLS, MODE>())
gm_bulk_apply_kernel(const BulkArgs<T> a, const __grid_constant__ RefOps<T> R)
{
    constexpr bool DO_K = (MODE & GM_M_K) != 0;
    constexpr bool DO_APU = (MODE & GM_M_APU) != 0;
    constexpr bool DO_AUP = (MODE & GM_M_AUP) != 0;
    constexpr bool DO_S = (MODE & GM_M_S) != 0;
    constexpr bool DO_C = (MODE & GM_M_C) != 0;
    constexpr bool IN_U = DO_K || DO_AUP;
    constexpr bool IN_P = DO_APU || DO_S || DO_C;
    constexpr bool OUT_U = DO_K || DO_APU;
    constexpr bool OUT_P = DO_AUP || DO_S || DO_C;
    constexpr int NI = (IN_U ? 3 : 0) + (IN_P ? 1 : 0);
    constexpr int NO = (OUT_U ? 3 : 0) + (OUT_P ? 1 : 0);
    constexpr int IPI = IN_U ? 3 : 0;   // slot of p among the input fields
    constexpr int OPI = OUT_U ? 3 : 0;  // slot of p among the output fields
    constexpr ParPat PP = gm_make_parpat(CLS);
    static_assert(!PCG || (NI == NO && (NI == 3 || NI == 1)), "PCG mode needs a square single-field-group operator");

    if (a.skip != nullptr && *a.skip != 0) return;

    __shared__ T s_plane[2][NI][17 * 17];
    __shared__ T s_face[NO][4][256];

    const GridDesc& g = a.g;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int x0 = blockIdx.x * 15, y0 = blockIdx.y * 15;
    const int fi = x0 - 1 + tx, fj = y0 - 1 + ty;
    const bool fval = fi >= 0 && fi < g.nx && fj >= 0 && fj < g.ny;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nplanes);
    const long long N = g.N;
    const long long rowlen = g.nx + 1;
    T beta = T(0);
    if constexpr (PCG) beta = (T)(*a.beta);

    auto layer_exists = [&](int kb) -> bool {
        return kb >= 0 && kb + 1 < g.nplanes && kb != g.kf;
    };
    auto layer_index = [&](int kb) -> int { return (g.kf >= 0 && kb > g.kf) ? kb - 1 : kb; };

    // input value of field f at a node (masked; PCG mode forms z + beta p_old)
    auto in_u = [&](int c, long long node) -> T {
        if constexpr (PCG) return a.zu[c * N + node] + beta * a.xu[c * N + node];
        else return a.xu[c * N + node];
    };
    auto in_p = [&](long long node) -> T {
        if constexpr (PCG) return a.zp[node] + beta * a.xp[node];
        else return a.xp[node];
    };

    // fetch one node plane (tile + halo) into registers: slots tid and tid + 256
    T pf[2][NI];
    auto fetch = [&](int kk) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            const int idx = tid + sl * 256;
#pragma unroll
            for (int f = 0; f < NI; ++f) pf[sl][f] = T(0);
            if (idx >= 17 * 17) continue;
            const int ni = idx % 17, nj = idx / 17;
            const int gi = x0 - 1 + ni, gj = y0 - 1 + nj;
            if (gi < 0 || gi > g.nx || gj < 0 || gj > g.ny) continue;
            const long long node = gi + rowlen * (gj + (long long)(g.ny + 1) * kk);
            const unsigned m = a.mask[node];
            if constexpr (IN_U) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (!((m >> c) & 1u)) pf[sl][c] = in_u(c, node);
            }
            if constexpr (IN_P) {
                long long pn = node;
                unsigned pm = m;
                if (g.tied && kk == g.kf + 1) {   // slave lip reads its master
                    pn = node - g.nb;
                    pm = a.mask[pn];
                }
                if (!((pm >> 3) & 1u)) pf[sl][IPI] = in_p(pn);
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            const int idx = tid + sl * 256;
            if (idx < 17 * 17)
#pragma unroll
                for (int f = 0; f < NI; ++f) s_plane[buf][f][idx] = pf[sl][f];
        }
    };

    // xy part of the forward transform for this thread's face:
    // t[sx + 2 sy] = sum_{ax,ay} (-1)^(sx ax + sy ay) v[ax, ay]
    // own_next: this thread's own node (tile node (tx, ty)) of the plane last
    // transformed; in PCG mode it is the node's new direction value p
    T own_next[NI];
    auto fwd_xy = [&](int buf, T (&t)[NI][4]) {
#pragma unroll
        for (int f = 0; f < NI; ++f) {
            const T v00 = s_plane[buf][f][ty * 17 + tx], v10 = s_plane[buf][f][ty * 17 + tx + 1];
            own_next[f] = v00;
            const T v01 = s_plane[buf][f][(ty + 1) * 17 + tx], v11 = s_plane[buf][f][(ty + 1) * 17 + tx + 1];
            const T a0 = v00 + v10, a1 = v00 - v10, b0 = v01 + v11, b1 = v01 - v11;
            t[f][0] = a0 + b0;
            t[f][1] = a1 + b1;
            t[f][2] = a0 - b0;
            t[f][3] = a1 - b1;
        }
    };

    // One element: z part of the transform, products with the allowed entries
    // of the parity-basis operators, inverse z part.  ob receives the
    // xy-parity tuples of the bottom node set (added), ot those of the top set.
    auto element = [&](const T (&tb)[NI][4], const T (&tt)[NI][4], int kb, T (&ob)[NO][4],
                       T (&ot)[NO][4]) {
        const long long e = fi + (long long)g.nx * (fj + (long long)g.ny * layer_index(kb));
        T kE = T(0), kC = T(0), kS = T(0);
        if constexpr (DO_K) kE = a.cK * a.E[e];
        if constexpr (DO_C) kC = a.cC * a.kap[e];
        if constexpr (DO_S) kS = a.fs != nullptr ? a.cS + a.cFS * a.fs[e] : a.cS;
        // parity values x[f][s] = tb[f][s & 3] +- tt[f][s & 3]
        T xu[3][8], xp[8];
        if constexpr (IN_U) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int s = 1; s < 8; ++s)
                    xu[c][s] = (s & 4) ? (tb[c][s & 3] - tt[c][s & 3]) : (tb[c][s & 3] + tt[c][s & 3]);
        }
        if constexpr (IN_P) {
#pragma unroll
            for (int s = 0; s < 8; ++s)
                xp[s] = (s & 4) ? (tb[IPI][s & 3] - tt[IPI][s & 3]) : (tb[IPI][s & 3] + tt[IPI][s & 3]);
        }
        // output parity value of field f, mode s (the constant displacement mode
        // carries no force: its row of K and A_pu is empty)
        auto out_u = [&](int c, int s) -> T {
            T acc = T(0);
            if constexpr (DO_K) {
                T t = T(0);
#pragma unroll
                for (int j = 0; j < 24; ++j)
                    if (PP.k[c * 8 + s][j] >= 0 && (j & 7) != 0) t = fma(R.K[PP.k[c * 8 + s][j]], xu[j >> 3][j & 7], t);
                acc = kE * t;
            }
            if constexpr (DO_APU) {
                T t = T(0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (PP.a[c * 8 + s][j] >= 0) t = fma(R.A[PP.a[c * 8 + s][j]], xp[j], t);
                acc = fma(a.cApu, t, acc);
            }
            return acc;
        };
        auto out_p = [&](int s) -> T {
            T acc = T(0);
            if constexpr (DO_AUP) {
                T t = T(0);
#pragma unroll
                for (int i = 0; i < 24; ++i)
                    if (PP.a[i][s] >= 0 && (i & 7) != 0) t = fma(R.A[PP.a[i][s]], xu[i >> 3][i & 7], t);
                acc = a.cAup * t;
            }
            if constexpr (DO_S) acc = fma(kS * R.M[s], xp[s], acc);
            if constexpr (DO_C) {
                T t = T(0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (PP.l[s][j] >= 0) t = fma(R.L[PP.l[s][j]], xp[j], t);
                acc = fma(kC, t, acc);
            }
            return acc;
        };
        if constexpr (OUT_U) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T hi0 = out_u(c, 4);
                ob[c][0] += hi0;
                ot[c][0] = -hi0;
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    const T lo = out_u(c, q), hi = out_u(c, q | 4);
                    ob[c][q] += lo + hi;
                    ot[c][q] = lo - hi;
                }
            }
        }
        if constexpr (OUT_P) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T lo = out_p(q), hi = out_p(q | 4);
                ob[OPI][q] += lo + hi;
                ot[OPI][q] = lo - hi;
            }
        }
    };

    T tb[NI][4], tt[NI][4];
    T carry[NO][4];
#pragma unroll
    for (int f = 0; f < NO; ++f)
#pragma unroll
        for (int q = 0; q < 4; ++q) carry[f][q] = T(0);

    // prologue: the halo layer below the chunk (its top contributions complete
    // plane z0), the bottom tuples of plane z0, and plane z0 + 1 in buffer 0
    int buf = 0;
    if (layer_exists(z0 - 1)) {
        fetch(z0 - 1);
        store(1);
        __syncthreads();
        fwd_xy(1, tb);
        fetch(z0);
        store(0);
        __syncthreads();
        fwd_xy(0, tt);
        if (fval) {
            T ob[NO][4] = {};
            element(tb, tt, z0 - 1, ob, carry);
        }
#pragma unroll
        for (int f = 0; f < NI; ++f)
#pragma unroll
            for (int q = 0; q < 4; ++q) tb[f][q] = tt[f][q];
    } else {
        fetch(z0);
        store(0);
        __syncthreads();
        fwd_xy(0, tb);
    }
    __syncthreads();
    if (z0 + 1 < g.nplanes) fetch(z0 + 1);
    store(buf);

    double dot = 0.0;
    T own_cur[NI];
#pragma unroll
    for (int f = 0; f < NI; ++f) own_cur[f] = own_next[f];   // plane z0
    for (int kk = z0; kk < z1; ++kk) {
        // buffer `buf` holds plane kk + 1 (if it exists); fetch plane kk + 2
        const bool need_next = kk + 2 < g.nplanes && kk + 2 <= z1;
        if (need_next) fetch(kk + 2);
        __syncthreads();
        T ob[NO][4], ot[NO][4];
#pragma unroll
        for (int f = 0; f < NO; ++f)
#pragma unroll
            for (int q = 0; q < 4; ++q) { ob[f][q] = T(0); ot[f][q] = T(0); }
        const bool up = layer_exists(kk);
        if (up) {
            fwd_xy(buf, tt);
            if (fval) element(tb, tt, kk, ob, ot);
#pragma unroll
            for (int f = 0; f < NI; ++f)
#pragma unroll
                for (int q = 0; q < 4; ++q) tb[f][q] = tt[f][q];
        } else if (kk + 1 < z1) {
            // fault gap: the next plane starts a new block of elements
            fwd_xy(buf, tb);
        }
        // complete face tuples of plane kk, inverse xy transform to corner values
#pragma unroll
        for (int f = 0; f < NO; ++f) {
            const T o0 = carry[f][0] + ob[f][0], o1 = carry[f][1] + ob[f][1];
            const T o2 = carry[f][2] + ob[f][2], o3 = carry[f][3] + ob[f][3];
            const T c0 = o0 + o1, c1 = o0 - o1, d0 = o2 + o3, d1 = o2 - o3;
            s_face[f][0][tid] = c0 + d0;   // corner (0,0)
            s_face[f][1][tid] = c1 + d1;   // corner (1,0)
            s_face[f][2][tid] = c0 - d0;   // corner (0,1)
            s_face[f][3][tid] = c1 - d1;   // corner (1,1)
#pragma unroll
            for (int q = 0; q < 4; ++q) carry[f][q] = up ? ot[f][q] : T(0);
        }
        if (need_next) store(buf ^ 1);
        __syncthreads();
        // own values of plane kk (for its node stage below) were stashed when plane kk
        // was transformed; own_next now holds plane kk + 1 (transformed this iteration)
        // node stage: node (tx, ty) of the tile sums its four faces
        if (tx >= 1 && ty >= 1) {
            const int gi = x0 - 1 + tx, gj = y0 - 1 + ty;
            if (gi <= g.nx && gj <= g.ny) {
                const long long node = gi + rowlen * (gj + (long long)(g.ny + 1) * kk);
                const unsigned m = a.mask[node];
                const bool lip = g.kf >= 0 && (kk == g.kf || kk == g.kf + 1);
                T ndot = T(0);
#pragma unroll
                for (int f = 0; f < NO; ++f) {
                    const T v = s_face[f][0][tid] + s_face[f][1][tid - 1] +
                                s_face[f][2][tid - 16] + s_face[f][3][tid - 17];
                    if (OUT_U && f < 3) {
                        const T y = ((m >> f) & 1u) ? T(0) : v;
                        a.yu[f * N + node] = y;
                        if constexpr (PCG) {
                            // own_cur holds z + beta p_old of this node, masked at load
                            a.pu_new[f * N + node] = own_cur[f];
                            if (!lip) ndot = fma(own_cur[f], y, ndot);
                        }
                    } else {
                        // raw value on a tied slave lip: the fault kernel folds it
                        const bool slave = g.tied && kk == g.kf + 1;
                        const T y = (!slave && ((m >> 3) & 1u)) ? T(0) : v;
                        a.yp[node] = y;
                        if constexpr (PCG) {
                            const T pn = slave ? T(0) : own_cur[IPI];
                            a.pp_new[node] = pn;
                            // pressure-system products in FP64 (FP32 squares of flow
                            // quantities can underflow)
                            if (!lip) dot += (double)pn * (double)y;
                        }
                    }
                }
                dot += (double)ndot;
            }
        }
        buf ^= 1;
#pragma unroll
        for (int f = 0; f < NI; ++f) own_cur[f] = own_next[f];
    }

    if constexpr (PCG) {
        // per-CTA partial of p . Ap (fixed order: warp shuffles, then warps)
        __shared__ double sh[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if ((tid & 31) == 0) sh[tid >> 5] = dot;
        __syncthreads();
        if (tid == 0) {
            double sacc = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) sacc += sh[w];
            const int cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            a.part[cta] = sacc;
        }
    }
}
