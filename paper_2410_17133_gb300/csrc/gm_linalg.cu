// Preconditioned-CG vector kernels with fused, deterministic FP64 reductions.
//
// One PCG iteration (Hestenes-Stiefel, as used inside the partitioned scheme of
// Sec. 3.3.2) takes two fused passes: the operator kernels form the direction
// p = z + beta p_old, q = A p and alpha = (r.z)/(p.q) (gm_apply.cuh); then
// x += alpha p, r -= alpha q, z = M^-1 r with the new r.z and r.r in one pass
// here, whose last block sets beta = (r.z)_new/(r.z).  The scalars live on the
// device (PcgScalars) so iterations can be enqueued back to back; every kernel
// returns at once when `done` is set, so the host only checks now and then.
// Vectors may be FP32 (mixed precision) or FP64; dots always accumulate in FP64.
#include "gm_internal.cuh"
#include "gm_pcgvec.cuh"

template <int NV>
__device__ void gm_block_sum_l(double (&v)[NV], double* sh)
{
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + w] = v[k];
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v[k] = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
}

template <int NV>
__device__ bool gm_grid_sum_l(double (&v)[NV], double* part, unsigned* counter)
{
    __shared__ double sh[NV * 32];
    __shared__ bool last;
    gm_block_sum_l<NV>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        acc[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            acc[k] += ((volatile double*)part)[k * gridDim.x + b];
    }
    __syncthreads();
    gm_block_sum_l<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = acc[k];
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

struct RedCtx {
    double* part;
    unsigned* counter;
};

template <typename T, int WHICH>
__global__ void __launch_bounds__(256)
gm_pcg_init_kernel(long long N, const T* b, const T* q, T* r, T* z, T* p, const T* mi, double rtol,
                   PcgScalars* sc, RedCtx rc, PairPrec<T> pp)
{
    constexpr int NC = Prec<T, WHICH>::NC;
    double v[2] = {0.0, 0.0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        if constexpr (WHICH == 0) {
            const long long d = n - pp.lo;
            if (pp.inv != nullptr && d >= 0 && d < 2 * pp.nb) {
                if (d >= pp.nb) continue;              // upper lip: done with its pair
                const long long nd[2] = {n, n + pp.nb};
                T r6[6], z6[6];
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const long long k = c * N + nd[s];
                        r6[3 * s + c] = q ? b[k] - q[k] : b[k];
                    }
                gm_pair_apply(pp, d, r6, z6);
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const long long k = c * N + nd[s];
                        r[k] = r6[3 * s + c];
                        z[k] = z6[3 * s + c];
                        p[k] = T(0);
                    }
                gm_dot_pair(r6, z6, v);
                continue;
            }
        }
        T rr[NC], zz[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) rr[c] = q ? b[c * N + n] - q[c * N + n] : b[c * N + n];
        Prec<T, WHICH>::apply(mi, N, n, rr, zz);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            r[c * N + n] = rr[c];
            z[c * N + n] = zz[c];
            p[c * N + n] = T(0);   // previous direction: the first step is p = z
        }
        gm_dot_node<T, NC>(rr, zz, v);
    }
    if (gm_grid_sum_l<2>(v, rc.part, rc.counter)) {
        sc->rz = v[0];
        sc->rr = v[1];
        sc->rr0 = v[1];
        sc->tol2 = rtol * rtol * v[1];
        sc->it = 0;
        sc->status = (isfinite(v[0]) && isfinite(v[1])) ? GM_OK : GM_ENAN;
        sc->done = (v[1] == 0.0 || sc->status != GM_OK) ? 1 : 0;
        sc->alpha = 0.0;
        sc->beta = 0.0;
    }
}

template <typename T, int WHICH>
__global__ void __launch_bounds__(256)
gm_pcg_update_kernel(long long N, T* x, T* r, T* z, const T* p, const T* q, const T* mi,
                     PcgScalars* sc, int maxit, RedCtx rc, PairPrec<T> pp)
{
    constexpr int NC = Prec<T, WHICH>::NC;
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    double v[2] = {0.0, 0.0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        if constexpr (WHICH == 0) {
            const long long d = n - pp.lo;
            if (pp.inv != nullptr && d >= 0 && d < 2 * pp.nb) {
                if (d >= pp.nb) continue;              // upper lip: done with its pair
                const long long nd[2] = {n, n + pp.nb};
                T r6[6], z6[6];
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const long long k = c * N + nd[s];
                        x[k] = fma(alpha, p[k], x[k]);
                        r6[3 * s + c] = fma(-alpha, q[k], r[k]);
                        r[k] = r6[3 * s + c];
                    }
                gm_pair_apply(pp, d, r6, z6);
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) z[c * N + nd[s]] = z6[3 * s + c];
                gm_dot_pair(r6, z6, v);
                continue;
            }
        }
        T rr[NC], zz[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long k = c * N + n;
            x[k] = fma(alpha, p[k], x[k]);
            rr[c] = fma(-alpha, q[k], r[k]);
            r[k] = rr[c];
        }
        Prec<T, WHICH>::apply(mi, N, n, rr, zz);
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c * N + n] = zz[c];
        gm_dot_node<T, NC>(rr, zz, v);
    }
    if (gm_grid_sum_l<2>(v, rc.part, rc.counter)) {
        sc->it += 1;
        sc->rr = v[1];
        if (!isfinite(v[0]) || !isfinite(v[1])) {
            sc->status = GM_ENAN;
            sc->done = 1;
        } else if (v[1] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= maxit) {
            sc->status = GM_ENOCONV;
            sc->done = 1;
        } else {
            sc->beta = v[0] / sc->rz;
            sc->rz = v[0];
        }
    }
}

static RedCtx redctx(gm_ctx* c)
{
    return RedCtx{c->dpart.as<double>(), c->dcount.as<unsigned>()};
}

template <typename T>
static PairPrec<T> pairprec(gm_ctx* c, int which)
{
    PairPrec<T> pp{nullptr, c->g.nb, -1};
    if (which == 0 && c->g.kf >= 0 && c->pair_prec) {
        if constexpr (sizeof(T) == 8) pp.inv = c->dKpair64.as<T>();
        else pp.inv = c->dKpair32.as<T>();
        pp.lo = (long long)c->g.kf * c->g.nb;
    }
    return pp;
}

// which 0: K_T block-Jacobi; 1: A22 Jacobi; 2: Jacobi of A22 plus the fixed-stress term
template <typename T>
static const T* prec_ptr(gm_ctx* c, int which)
{
    if constexpr (sizeof(T) == 8)
        return which == 0 ? c->dKinv64.as<T>() : (which == 1 ? c->dAinv64.as<T>() : c->dAfsinv64.as<T>());
    else
        return which == 0 ? c->dKinv32.as<T>() : (which == 1 ? c->dAinv32.as<T>() : c->dAfsinv32.as<T>());
}

int gm_launch_pcg_init(gm_ctx* c, int which, int prec, const void* b, const void* q, void* r,
                       void* z, void* p, double rtol, PcgScalars* sc, cudaStream_t s)
{
    const long long N = c->N;
    RedCtx rc = redctx(c);
    if (prec == GM_F64) {
        if (which == 0)
            gm_pcg_init_kernel<double, 0><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (const double*)b, (const double*)q, (double*)r, (double*)z, (double*)p,
                prec_ptr<double>(c, 0), rtol, sc, rc, pairprec<double>(c, 0));
        else
            gm_pcg_init_kernel<double, 1><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (const double*)b, (const double*)q, (double*)r, (double*)z, (double*)p,
                prec_ptr<double>(c, which), rtol, sc, rc, pairprec<double>(c, which));
    } else {
        if (which == 0)
            gm_pcg_init_kernel<float, 0><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (const float*)b, (const float*)q, (float*)r, (float*)z, (float*)p,
                prec_ptr<float>(c, 0), rtol, sc, rc, pairprec<float>(c, 0));
        else
            gm_pcg_init_kernel<float, 1><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (const float*)b, (const float*)q, (float*)r, (float*)z, (float*)p,
                prec_ptr<float>(c, which), rtol, sc, rc, pairprec<float>(c, which));
    }
    GM_LAUNCHED(c);
    return GM_OK;
}

int gm_launch_pcg_update(gm_ctx* c, int which, int prec, void* x, void* r, void* z, const void* p,
                         const void* q, PcgScalars* sc, int maxit, cudaStream_t s)
{
    const long long N = c->N;
    RedCtx rc = redctx(c);
    if (prec == GM_F64) {
        if (which == 0)
            gm_pcg_update_kernel<double, 0><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (double*)x, (double*)r, (double*)z, (const double*)p, (const double*)q,
                prec_ptr<double>(c, 0), sc, maxit, rc, pairprec<double>(c, 0));
        else
            gm_pcg_update_kernel<double, 1><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (double*)x, (double*)r, (double*)z, (const double*)p, (const double*)q,
                prec_ptr<double>(c, which), sc, maxit, rc, pairprec<double>(c, which));
    } else {
        if (which == 0)
            gm_pcg_update_kernel<float, 0><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (float*)x, (float*)r, (float*)z, (const float*)p, (const float*)q,
                prec_ptr<float>(c, 0), sc, maxit, rc, pairprec<float>(c, 0));
        else
            gm_pcg_update_kernel<float, 1><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
                N, (float*)x, (float*)r, (float*)z, (const float*)p, (const float*)q,
                prec_ptr<float>(c, which), sc, maxit, rc, pairprec<float>(c, which));
    }
    GM_LAUNCHED(c);
    return GM_OK;
}

// ---------------------------------------------------------------------------
// Generic vector kernels
// ---------------------------------------------------------------------------
__global__ void gm_axpby_kernel(long long n, double a, const double* x, double b, double* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

int gm_launch_axpby(gm_ctx* c, long long n, double a, const double* x, double b, double* y,
                    cudaStream_t s)
{
    gm_axpby_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n, a, x, b, y);
    GM_LAUNCHED(c);
    return GM_OK;
}

__global__ void gm_d2f_kernel(long long n, const double* x, float* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
__global__ void gm_f2d_kernel(long long n, const float* x, double* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}
__global__ void gm_axpy_f2d_kernel(long long n, double a, const float* x, double* y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] += a * (double)x[i];
}

// y = x / 2^e in FP32, with 2^e the power of two at or below the RMS of x read
// from sc[0] = x.x (e = 0 when x is zero or not finite); sc[1] = 2^e.  The FP32
// correction solves then work on values of order one however small the Newton
// residual has become, away from FP32 subnormals; the scale is exact.
__global__ void gm_d2f_scaled_kernel(long long n, const double* x, float* y, double* sc)
{
    const double ms = sc[0] / (double)n;
    const int e = (ms > 0.0 && isfinite(ms)) ? ilogb(sqrt(ms)) : 0;
    const double inv = ldexp(1.0, -e);
    if (blockIdx.x == 0 && threadIdx.x == 0) sc[1] = ldexp(1.0, e);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)(x[i] * inv);
}
__global__ void gm_axpy_f2d_scaled_kernel(long long n, const double* sc, const float* x, double* y)
{
    const double a = sc[1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] += a * (double)x[i];
}

int gm_launch_cast_scaled_d2f(gm_ctx* c, long long n, const double* x, float* y, double* sc,
                              cudaStream_t s)
{
    int rc = gm_launch_dot(c, n, x, x, nullptr, nullptr, sc, s);
    if (rc) return rc;
    gm_d2f_scaled_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n, x, y, sc);
    GM_LAUNCHED(c);
    return GM_OK;
}
int gm_launch_axpy_scaled_f2d(gm_ctx* c, long long n, const double* sc, const float* x, double* y,
                              cudaStream_t s)
{
    gm_axpy_f2d_scaled_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n, sc, x, y);
    GM_LAUNCHED(c);
    return GM_OK;
}

int gm_launch_copy_cast_d2f(gm_ctx* c, long long n, const double* x, float* y, cudaStream_t s)
{
    gm_d2f_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n, x, y);
    GM_LAUNCHED(c);
    return GM_OK;
}
int gm_launch_copy_cast_f2d(gm_ctx* c, long long n, const float* x, double* y, cudaStream_t s)
{
    gm_f2d_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n, x, y);
    GM_LAUNCHED(c);
    return GM_OK;
}
int gm_launch_axpy_f2d(gm_ctx* c, long long n, double a, const float* x, double* y, cudaStream_t s)
{
    gm_axpy_f2d_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n, a, x, y);
    GM_LAUNCHED(c);
    return GM_OK;
}

__global__ void __launch_bounds__(256)
gm_dot_kernel(long long n, const double* x, const double* y, const double* x2, const double* y2,
              double* out, RedCtx rc)
{
    double v[2] = {0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        v[0] += x[i] * y[i];
        if (x2) v[1] += x2[i] * y2[i];
    }
    if (gm_grid_sum_l<2>(v, rc.part, rc.counter)) {
        out[0] = v[0];
        out[1] = v[1];
    }
}

int gm_launch_dot(gm_ctx* c, long long n, const double* x, const double* y, const double* x2,
                  const double* y2, double* out, cudaStream_t s)
{
    gm_dot_kernel<<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(n, x, y, x2, y2, out, redctx(c));
    GM_LAUNCHED(c);
    return GM_OK;
}


// ---------------------------------------------------------------------------
// PCG steps around the multigrid preconditioner (FP32 K_T solves): the update
// pass leaves z to the V-cycle, and a second pass forms r.z and beta.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
gm_pcg_update_noz_kernel(long long n, T* x, T* r, const T* p, const T* q, PcgScalars* sc, int maxit,
                         RedCtx rc)
{
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        v[0] += (double)ri * (double)ri;
    }
    if (gm_grid_sum_l<1>(v, rc.part, rc.counter)) {
        sc->it += 1;
        sc->rr = v[0];
        if (!isfinite(v[0])) {
            sc->status = GM_ENAN;
            sc->done = 1;
        } else if (v[0] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->it >= maxit) {
            sc->status = GM_ENOCONV;
            sc->done = 1;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
gm_pcg_rz_kernel(long long n, const T* r, const T* z, PcgScalars* sc, int init, RedCtx rc)
{
    if (sc->done) return;
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[0] += (double)r[i] * (double)z[i];
    if (gm_grid_sum_l<1>(v, rc.part, rc.counter)) {
        if (!isfinite(v[0]) || !(v[0] > 0.0)) {
            sc->status = isfinite(v[0]) ? GM_ENOCONV : GM_ENAN;
            sc->done = 1;
        } else if (init) {
            sc->rz = v[0];
        } else {
            sc->beta = v[0] / sc->rz;
            sc->rz = v[0];
        }
    }
}

int gm_launch_pcg_update_noz(gm_ctx* c, int prec, void* x, void* r, const void* p, const void* q,
                             PcgScalars* sc, int maxit, cudaStream_t s)
{
    if (prec == GM_F64)
        gm_pcg_update_noz_kernel<double><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
            3 * c->N, (double*)x, (double*)r, (const double*)p, (const double*)q, sc, maxit, redctx(c));
    else
        gm_pcg_update_noz_kernel<float><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(
            3 * c->N, (float*)x, (float*)r, (const float*)p, (const float*)q, sc, maxit, redctx(c));
    GM_LAUNCHED(c);
    return GM_OK;
}

int gm_launch_pcg_rz(gm_ctx* c, int prec, const void* r, const void* z, PcgScalars* sc, int init,
                     cudaStream_t s)
{
    if (prec == GM_F64)
        gm_pcg_rz_kernel<double><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(3 * c->N, (const double*)r,
                                                                        (const double*)z, sc, init, redctx(c));
    else
        gm_pcg_rz_kernel<float><<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(3 * c->N, (const float*)r,
                                                                       (const float*)z, sc, init, redctx(c));
    GM_LAUNCHED(c);
    return GM_OK;
}
