// Device-resident PCG for the K and K_T solves of the tetrahedral path (the
// inner solves of Prevost's partitioned CG, Sec. 3.3.2).  Every scalar of the
// recurrence (r.z, p.q, alpha, beta, the stopping test) stays on the device:
// each reduction ends in the last block of its kernel, which sums the
// per-block partials in a fixed assignment and tree (deterministic) and
// updates the solve's state.  The host launches iterations in chunks and reads the state once per
// chunk; once the state says done, every later kernel of the chunk (the
// operator's included, through the skip flag) returns at once.
//
// Preconditioner: nodal 3x3 block Jacobi, and for the two lips of each fault
// pair the inverse of their 6x6 block [K_-- + A D, -A D; -A D, K_++ + A D]
// (bulk blocks of the two lips plus the cohesive tangent, which couples them).
// Included by gm_tet.cu only.
#pragma once

namespace {

constexpr int TPCG_BLOCKS = 304;   // 2 per SM on a 152-SM part; fixed, so sums are reproducible
constexpr int TPCG_NT = 256;

struct TetPcgState {
    double rz, rr0, tol2, alpha, beta, rr;
    int done;        // 0 running, 1 converged, 2 breakdown (p.q <= 0 or non-finite), 3 iteration limit
    int its, maxit;
    unsigned ticket;
};

template <typename T>
struct TetPrecT {
    int N, P;
    const T* Kinv;      // 9N, (3i + j) * N + n; constrained rows / columns 0
    const int* n2p;     // N: pair of a lip node, -1 elsewhere (null: no fault)
    const int* pm;      // P minus lips
    const int* pp;      // P plus lips
    const T* Pinv;      // 36P, (6 r + c) * P + i; constrained rows / columns 0
};

// Block sum of (a, b) in a fixed tree (warp butterfly, then the warps in order)
__device__ inline void tpcg_block_sum2(double& a, double& b)
{
    __shared__ double sa[TPCG_NT / 32], sb[TPCG_NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    __syncthreads();                       // the shared words may still be read by a previous call
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int w = 0; w < TPCG_NT / 32; ++w) {
        a += sa[w];
        b += sb[w];
    }
}

// Grid sum of (a, b): each block writes its partials; the last block to finish
// (ticket counter) sums all partials, thread t taking blocks t, t + 256, ...,
// then the block tree, so the order is fixed.  Returns true on thread 0 of the
// last block, which holds the sums in (A, B).
__device__ inline bool tpcg_reduce2(double a, double b, double* part, unsigned* ticket, double& A, double& B)
{
    __shared__ bool last;
    tpcg_block_sum2(a, b);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double pa = 0.0, pb = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        pa += __ldcg(part + 2 * k);
        pb += __ldcg(part + 2 * k + 1);
    }
    tpcg_block_sum2(pa, pb);
    if (threadIdx.x != 0) return false;
    A = pa;
    B = pb;
    *ticket = 0u;
    return true;
}

// r = b (cast to T), x = 0; state reset
template <typename T>
__global__ void __launch_bounds__(TPCG_NT) tpcg_start(long long n, const double* b, T* r, T* x, TetPcgState* st,
                                                      double tol2, int maxit)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        r[i] = (T)b[i];
        x[i] = T(0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->tol2 = tol2;
        st->maxit = maxit;
        st->its = 0;
        st->done = 0;
        st->ticket = 0u;
    }
}

// z = M^-1 r on the nodes of one pair (both lips) or one node
template <typename T>
__device__ inline void tpcg_prec_pair(const TetPrecT<T>& M, int i, const T (&r6)[6], T (&z6)[6])
{
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < 6; ++b) acc += M.Pinv[(6 * a + b) * M.P + i] * r6[b];
        z6[a] = acc;
    }
}

// One PCG step after alpha is known (START: the initial preconditioning):
// x += alpha p, r -= alpha q, z = M^-1 r, then r.z and r.r; the last block
// sets beta = (r.z)_new / (r.z)_old and the stopping state.
template <typename T, bool START>
__global__ void __launch_bounds__(TPCG_NT) tpcg_step(TetPrecT<T> M, T* x, T* r, T* z, const T* p, const T* q,
                                                     TetPcgState* st, double* part)
{
    if (!START && st->done) return;
    const int N = M.N;
    const T al = START ? T(0) : (T)st->alpha;
    double rz = 0.0, rr = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int pi = M.n2p ? M.n2p[n] : -1;
        if (pi >= 0) {
            if (M.pm[pi] != n) continue;                 // plus lip: done with its pair
            const int nd[2] = {n, M.pp[pi]};
            T r6[6], z6[6];
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long k = (long long)c * N + nd[s];
                    T rv = r[k];
                    if (!START) {
                        rv -= al * q[k];
                        x[k] += al * p[k];
                        r[k] = rv;
                    }
                    r6[3 * s + c] = rv;
                }
            tpcg_prec_pair(M, pi, r6, z6);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long k = (long long)c * N + nd[s];
                    z[k] = z6[3 * s + c];
                    rz += (double)r6[3 * s + c] * (double)z6[3 * s + c];
                    rr += (double)r6[3 * s + c] * (double)r6[3 * s + c];
                }
            continue;
        }
        T r3[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long k = (long long)c * N + n;
            T rv = r[k];
            if (!START) {
                rv -= al * q[k];
                x[k] += al * p[k];
                r[k] = rv;
            }
            r3[c] = rv;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T za = M.Kinv[(3 * a) * N + n] * r3[0] + M.Kinv[(3 * a + 1) * N + n] * r3[1] +
                         M.Kinv[(3 * a + 2) * N + n] * r3[2];
            z[(long long)a * N + n] = za;
            rz += (double)r3[a] * (double)za;
            rr += (double)r3[a] * (double)r3[a];
        }
    }
    double RZ, RR;
    if (tpcg_reduce2(rz, rr, part, &st->ticket, RZ, RR)) {
        st->rr = RR;
        if (START) {
            st->rr0 = RR;
            st->rz = RZ;
            st->beta = 0.0;
            st->done = RR > 0.0 ? (isfinite(RR) ? 0 : 2) : 1;
        } else {
            st->its += 1;
            st->beta = RZ / st->rz;
            st->rz = RZ;
            if (!isfinite(RR) || !isfinite(RZ)) st->done = 2;
            else if (RR <= st->tol2 * st->rr0) st->done = 1;
            else if (st->its >= st->maxit) st->done = 3;
        }
    }
}

// constrained entries of q set to 0, then p.q; the last block sets alpha
template <typename T>
__global__ void __launch_bounds__(TPCG_NT) tpcg_pq(int N, const uint8_t* mask, const T* p, T* q, TetPcgState* st,
                                                   double* part)
{
    if (st->done) return;
    double acc = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const unsigned m = mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long k = (long long)c * N + n;
            T qv = q[k];
            if ((m >> c) & 1u) {
                qv = T(0);
                q[k] = qv;
            }
            acc += (double)p[k] * (double)qv;
        }
    }
    double PQ, unused;
    if (tpcg_reduce2(acc, 0.0, part, &st->ticket, PQ, unused)) {
        if (!(PQ > 0.0) || !isfinite(PQ)) st->done = 2;
        else st->alpha = st->rz / PQ;
    }
}

// p = z + beta p (START: p = z)
template <typename T, bool START>
__global__ void __launch_bounds__(TPCG_NT) tpcg_dir(long long n, const T* z, T* p, const TetPcgState* st)
{
    if (st->done) return;
    const T b = START ? T(0) : (T)st->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = START ? z[i] : z[i] + b * p[i];
}

template <typename T>
__global__ void __launch_bounds__(TPCG_NT) tpcg_out(long long n, const T* x, double* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

template <typename T>
__global__ void __launch_bounds__(TPCG_NT) tpcg_cast(long long n, const double* x, T* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)x[i];
}

// Inverse of the 6x6 block of each fault pair's two lips (FP64, Gauss-Jordan
// with partial pivoting): [K_-- + A D, -A D; -A D, K_++ + A D], constrained
// components replaced by identity rows and columns before and zeroed after.
__global__ void tpcg_pair_inverse(int N, int P, const double* Kblk, const int* pm, const int* pp, const double* area,
                                  const double* D, const uint8_t* mask, double* Pinv, int* err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int nd[2] = {pm[i], pp[i]};
    const double Ai = area[i];
    const double d[6] = {D[i], D[P + i], D[2 * P + i], D[3 * P + i], D[4 * P + i], D[5 * P + i]};
    const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double a[6][12];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 12; ++c) a[r][c] = (c - 6 == r) ? 1.0 : 0.0;
    for (int s = 0; s < 2; ++s)
        for (int u = 0; u < 2; ++u)
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) {
                    double v = (s == u ? 1.0 : -1.0) * Ai * d[idx[x][y]];
                    if (s == u) v += Kblk[(3 * x + y) * N + nd[s]];
                    a[3 * s + x][3 * u + y] = v;
                }
    bool fixd[6];
    for (int s = 0; s < 2; ++s) {
        const unsigned m = mask[nd[s]];
        for (int c = 0; c < 3; ++c) fixd[3 * s + c] = (m >> c) & 1u;
    }
    for (int r = 0; r < 6; ++r)
        if (fixd[r])
            for (int c = 0; c < 6; ++c) {
                a[r][c] = (r == c) ? 1.0 : 0.0;
                a[c][r] = (r == c) ? 1.0 : 0.0;
            }
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        for (int r = col + 1; r < 6; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        const double pv = a[piv][col];
        if (!(fabs(pv) > 0.0) || !isfinite(pv)) {
            *err = 1;
            for (int k = 0; k < 36; ++k) Pinv[k * P + i] = 0.0;
            return;
        }
        if (piv != col)
            for (int c = 0; c < 12; ++c) {
                const double tmp = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = tmp;
            }
        const double inv = 1.0 / pv;
        for (int c = 0; c < 12; ++c) a[col][c] *= inv;
        for (int r = 0; r < 6; ++r)
            if (r != col) {
                const double f = a[r][col];
                if (f != 0.0)
                    for (int c = 0; c < 12; ++c) a[r][c] -= f * a[col][c];
            }
    }
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) Pinv[(6 * r + c) * P + i] = (fixd[r] || fixd[c]) ? 0.0 : a[r][6 + c];
}

// Device-resident PCG over the fixed vectors x, r, z, p, q (3N each, type T).
template <typename T>
struct TetPcg {
    int N;
    cudaStream_t s;
    T *x, *r, *z, *p, *q;
    TetPcgState* st;
    double* part;
    TetPrecT<T> M;
    const uint8_t* mask;

    static constexpr int GRAPH_ITS = 8;    // iterations per captured graph

    // k iterations on stream cs: q = A p, alpha, x / r / z update, beta, p
    template <class Op>
    void iterate(cudaStream_t cs, int k, Op& op)
    {
        const long long n = 3LL * N;
        for (int i = 0; i < k; ++i) {
            op(p, q, &st->done, cs);
            tpcg_pq<T><<<TPCG_BLOCKS, TPCG_NT, 0, cs>>>(N, mask, p, q, st, part);
            tpcg_step<T, false><<<TPCG_BLOCKS, TPCG_NT, 0, cs>>>(M, x, r, z, p, q, st, part);
            tpcg_dir<T, false><<<TPCG_BLOCKS, TPCG_NT, 0, cs>>>(n, z, p, st);
        }
    }

    // x_out = A^-1 b by PCG from x = 0 to ||r|| <= rtol ||b||; op(p, q, skip,
    // stream) launches q = A p (unmasked) on the stream and skips its work
    // while *skip != 0.  With slot non-null, GRAPH_ITS iterations are captured
    // once (on the non-blocking stream *cap, created on first use) into *slot
    // and replayed; every pointer the graph holds is fixed for the buffers'
    // lifetime and the tolerance and limit sit in the device state, so the
    // owner destroys the graph only when it reallocates the vectors.
    // Returns 0, 2 / 3 (breakdown / iteration limit) or -1 (CUDA error);
    // *its += iterations.
    template <class Op>
    int solve(const double* b, double* x_out, double rtol, int maxit, long long* its, Op&& op,
              cudaGraphExec_t* slot = nullptr, cudaStream_t* cap = nullptr)
    {
        const long long n = 3LL * N;
        if (slot && !*slot) {
            if (!*cap && cudaStreamCreateWithFlags(cap, cudaStreamNonBlocking) != cudaSuccess) return -1;
            if (cudaStreamBeginCapture(*cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
            iterate(*cap, GRAPH_ITS, op);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(*cap, &g);
            if (ec != cudaSuccess) return -1;
            const cudaError_t ei = cudaGraphInstantiate(slot, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                *slot = nullptr;
                return -1;
            }
        }
        tpcg_start<T><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(n, b, r, x, st, rtol * rtol, maxit);
        tpcg_step<T, true><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(M, x, r, z, p, q, st, part);
        tpcg_dir<T, true><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(n, z, p, st);
        int reps = 1;
        int hs[2] = {0, 0};
        for (;;) {
            for (int k = 0; k < reps; ++k) {
                if (slot) {
                    if (cudaGraphLaunch(*slot, s) != cudaSuccess) return -1;
                } else {
                    iterate(s, GRAPH_ITS, op);
                }
            }
            cudaMemcpyAsync(hs, &st->done, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
            if (hs[0] != 0) break;
            reps = std::min(2 * reps, 8);
        }
        *its += hs[1];
        if (hs[0] == 2 || hs[0] == 3) return hs[0];
        tpcg_out<T><<<TPCG_BLOCKS, TPCG_NT, 0, s>>>(n, x, x_out);
        return 0;
    }
};

}  // namespace
