// Per-node pieces of the preconditioned-CG vector work (nodal and lip-pair
// block-Jacobi application, node-wise dot accumulation), shared by the PCG
// kernels and the multigrid smoother.
#pragma once

#include "gm_internal.cuh"

// Preconditioner application for one node, in the vector precision T.
// WHICH 0: 3 components, 3x3 symmetric block inverse (6 per node);
// WHICH 1: 1 component, diagonal inverse.
template <typename T, int WHICH>
struct Prec;
template <typename T>
struct Prec<T, 0> {
    static constexpr int NC = 3;
    __device__ static void apply(const T* mi, long long N, long long n, const T (&r)[3], T (&z)[3]) {
        const T i0 = mi[n], i1 = mi[N + n], i2 = mi[2 * N + n];
        const T i3 = mi[3 * N + n], i4 = mi[4 * N + n], i5 = mi[5 * N + n];
        z[0] = i0 * r[0] + i1 * r[1] + i2 * r[2];
        z[1] = i1 * r[0] + i3 * r[1] + i4 * r[2];
        z[2] = i2 * r[0] + i4 * r[1] + i5 * r[2];
    }
};
template <typename T>
struct Prec<T, 1> {
    static constexpr int NC = 1;
    __device__ static void apply(const T* mi, long long, long long n, const T (&r)[1], T (&z)[1]) {
        z[0] = mi[n] * r[0];
    }
};

// Add r.z and r.r of one node to the FP64 accumulators v.  Displacement
// vectors (3 components, force-scale residuals) sum the node's components in
// the vector precision first; pressure vectors (flow residuals of order
// 1e-15..1e-20 m^3, whose squares would underflow in FP32) multiply in FP64,
// where the product of two floats is exact.
template <typename T, int NC>
__device__ inline void gm_dot_node(const T (&r)[NC], const T (&z)[NC], double (&v)[2])
{
    if constexpr (NC == 3) {
        T a = T(0), b = T(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            a = fma(r[c], z[c], a);
            b = fma(r[c], r[c], b);
        }
        v[0] += (double)a;
        v[1] += (double)b;
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            v[0] += (double)r[c] * (double)z[c];
            v[1] += (double)r[c] * (double)r[c];
        }
    }
}

// K_T preconditioner blocks of the fault pairs: the thread of a lower-lip node
// applies the 6x6 inverse to both lips of its pair (and updates both), the
// thread of an upper-lip node skips it, so no two threads touch one node.
template <typename T>
struct PairPrec {
    const T* inv;     // 36 per pair, field-major, row-major 6x6 (lower lip 0-2, upper 3-5); null: off
    long long nb;     // pairs (= nodes per plane)
    long long lo;     // first lower-lip node
};

template <typename T>
__device__ inline void gm_pair_apply(const PairPrec<T>& pp, long long d, const T (&r6)[6], T (&z6)[6])
{
    // three rows at a time: the pair path is taken by one thread per fault
    // pair; fully unrolled it would raise the register budget of the node
    // path, one row at a time it waits for six memory round trips in a row
#pragma unroll 3
    for (int a = 0; a < 6; ++a) {
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 6; ++b) acc = fma(pp.inv[(a * 6 + b) * pp.nb + d], r6[b], acc);
        z6[a] = acc;
    }
}

template <typename T>
__device__ inline void gm_dot_pair(const T (&r6)[6], const T (&z6)[6], double (&v)[2])
{
    const T r0[3] = {r6[0], r6[1], r6[2]}, r1[3] = {r6[3], r6[4], r6[5]};
    const T z0[3] = {z6[0], z6[1], z6[2]}, z1[3] = {z6[3], z6[4], z6[5]};
    gm_dot_node<T, 3>(r0, z0, v);
    gm_dot_node<T, 3>(r1, z1, v);
}
