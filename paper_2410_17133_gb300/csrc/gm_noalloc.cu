// gm_residual_noalloc: the Newton residual of gm_residual, for callers that must
// not allocate device memory during the call (code running under an external
// memory budget or pool that forbids cudaMalloc, real-time loops, plug-ins that
// only hand out pre-allocated pointers).  The reduction scratch that
// gm_residual keeps in context memory lives here in one file-scope device array
// of fixed size instead; the call itself allocates nothing.
//
// The array (about 1 MB) is part of the library image: every GPU that loads the
// library holds it until the process exits.  All calls share it and it keeps the
// last call's contents, so calls whose GPU work overlaps (on different streams
// or different contexts on the same device) race on it and must be serialised by
// the caller.
#include <cmath>
#include <string>

#include "gm_internal.cuh"

namespace {

// One reduction block per 256 nodes, so the node count bounds the scratch size.
constexpr long long kMaxNodes = 1LL << 24;                 // 16,777,216 nodes
constexpr int kThreads = 256;
constexpr int kMaxBlocks = (int)(kMaxNodes / kThreads);    // 65,536 blocks
// layout (doubles): [0, 2*kMaxBlocks) block partials, then 2 result slots, then
// one slot whose first 4 bytes are the last-block counter
constexpr int kResultSlot = 2 * kMaxBlocks;
constexpr int kCounterSlot = 2 * kMaxBlocks + 2;
constexpr int kScratchDoubles = 2 * kMaxBlocks + 4;

}  // namespace

static __device__ __align__(256) double gm_noalloc_scratch[kScratchDoubles];

namespace {

struct NoAllocArgs {
    ResidualInputs in;
    double* scratch;   // device address of gm_noalloc_scratch
};

__device__ void na_block_sum(double (&v)[2], double* sh)
{
    for (int k = 0; k < 2; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh[w] = v[0]; sh[32 + w] = v[1]; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < 2; ++k) {
            v[k] = lane < nw ? sh[k * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
}

// b = [f^u - y1u - F_coh ; dt f^p - y1p - y2p] on free dofs (0 elsewhere), and
// sum b1^2/diag(K_b) + sum b2^2/diag(A22), sum diag(K_b) u^2 + sum diag(A22) p^2,
// one node per thread; block partials and the last-block total go to scratch.
__global__ void __launch_bounds__(kThreads) gm_residual_noalloc_kernel(const NoAllocArgs a)
{
    __shared__ double sh[64];
    __shared__ bool last;
    const long long n = (long long)blockIdx.x * kThreads + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (n < a.in.g.N) gm_residual_node(a.in, n, v);
    na_block_sum(v, sh);
    double* part = a.scratch;
    unsigned* counter = reinterpret_cast<unsigned*>(a.scratch + kCounterSlot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = v[0];
        part[kMaxBlocks + blockIdx.x] = v[1];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[2] = {0.0, 0.0};
    for (int bk = threadIdx.x; bk < (int)gridDim.x; bk += kThreads) {
        acc[0] += ((volatile double*)part)[bk];
        acc[1] += ((volatile double*)part)[kMaxBlocks + bk];
    }
    __syncthreads();
    na_block_sum(acc, sh);
    if (threadIdx.x == 0) {
        a.scratch[kResultSlot] = acc[0];
        a.scratch[kResultSlot + 1] = acc[1];
        *counter = 0u;
    }
}

// Device address of the scratch array in the context's device, looked up on
// every call with that device current (the lookup allocates nothing), so a
// context re-created after cudaDeviceReset or a different current context never
// sees a stale address.
int scratch_address(gm_ctx* c, double** out)
{
    int cur = -1;
    GM_CUDA_TRY(c, cudaGetDevice(&cur));
    if (cur != c->device) GM_CUDA_TRY(c, cudaSetDevice(c->device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, gm_noalloc_scratch);
    if (cur != c->device) cudaSetDevice(cur);
    if (e != cudaSuccess || p == nullptr)
        return c->set_err(GM_ECUDA, std::string("residual_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = static_cast<double*>(p);
    return GM_OK;
}

}  // namespace

extern "C" int gm_residual_noalloc(gm_ctx* c, const double* du, const double* dp, double* b,
                                   double* rhat, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "residual_noalloc: not bound");
    if (!du || !dp || !b) return c->set_err(GM_EINVAL, "residual_noalloc: null vector");
    if (c->N > kMaxNodes)
        return c->set_err(GM_EINVAL, "residual_noalloc: " + std::to_string(c->N) +
                                         " nodes exceed the fixed scratch limit of " +
                                         std::to_string(kMaxNodes) + " nodes; use gm_residual");
    double* scratch = nullptr;
    int rc = scratch_address(c, &scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = c->N, N3 = 3 * N;
    double* ut = c->w_ut.as<double>();
    double* pt = c->w_pt.as<double>();
    GM_CUDA_TRY(c, cudaMemcpyAsync(ut, c->du_n.p, N3 * 8, cudaMemcpyDeviceToDevice, s));
    GM_CUDA_TRY(c, cudaMemcpyAsync(pt, c->dp_n.p, N * 8, cudaMemcpyDeviceToDevice, s));
    if ((rc = gm_launch_axpby(c, N3, 1.0, du, 1.0, ut, s))) return rc;
    if ((rc = gm_launch_axpby(c, N, 1.0, dp, 1.0, pt, s))) return rc;
    if ((rc = gm_launch_return_map(c, c->du_n.as<double>(), du, s))) return rc;
    double* y1u = c->w_y1u.as<double>();
    double* y1p = c->w_y1p.as<double>();
    double* y2p = c->w_y2p.as<double>();
    if ((rc = gm_launch_apply_f64(c, GM_MODE_RES1, 1, -1, 0, 0, c->dt, ut, pt, y1u, y1p, s, nullptr))) return rc;
    if ((rc = gm_launch_apply_f64(c, GM_MODE_RES2, 0, 0, 1, 1, 0, du, dp, nullptr, y2p, s, nullptr))) return rc;
    // the counter must start at zero whatever an earlier call left behind
    GM_CUDA_TRY(c, cudaMemsetAsync(scratch + kCounterSlot, 0, sizeof(double), s));
    NoAllocArgs a;
    a.in = gm_residual_inputs(c, y1u, y1p, y2p, ut, pt, b);
    a.scratch = scratch;
    const int nblk = (int)((N + kThreads - 1) / kThreads);
    gm_residual_noalloc_kernel<<<nblk, kThreads, 0, s>>>(a);
    GM_LAUNCHED(c);
    double* h = reinterpret_cast<double*>(static_cast<char*>(c->hpin) + 3072);
    GM_CUDA_TRY(c, cudaMemcpyAsync(h, scratch + kResultSlot, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (rhat) *rhat = std::sqrt(h[0]);
    return GM_OK;
}
