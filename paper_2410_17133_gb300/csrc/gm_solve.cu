// Solvers: inner PCG (device-resident scalars, host checks in batches) and
// Prevost's partitioned CG (Sec. 3.3.2, Eq. schur_system).
#include <cmath>

#include "gm_internal.cuh"

static PcgScalars* scal(gm_ctx* c, int slot) { return c->dscal.as<PcgScalars>() + slot; }

static int apply_inner(gm_ctx* c, int which, int prec, const void* x, void* y, cudaStream_t s,
                       const int* skip)
{
    if (prec == GM_F64) {
        if (which == 0)
            return gm_launch_apply_f64(c, GM_MODE_KT, 1, 0, 0, 0, 0, (const double*)x, nullptr,
                                       (double*)y, nullptr, s, skip);
        return gm_launch_apply_f64(c, GM_MODE_A22, 0, 0, 0, 1, c->dt, nullptr, (const double*)x,
                                   nullptr, (double*)y, s, skip);
    }
    if (which == 0)
        return gm_launch_apply_f32(c, GM_MODE_KT, 1, 0, 0, 0, 0, (const float*)x, nullptr,
                                   (float*)y, nullptr, s, skip);
    return gm_launch_apply_f32(c, GM_MODE_A22, 0, 0, 0, 1, c->dt, nullptr, (const float*)x,
                               nullptr, (float*)y, s, skip);
}

// Solve A x = b (A = K_T for which 0, A22 for which 1) by PCG to ||r|| <= rtol ||r0||.
// b, x are FP64 device vectors; x holds the initial guess.  With prec GM_F32 the
// iteration runs on FP32 vectors and FP32 operators for the correction
// d = A^-1 (b - A x), added to x in FP64.
int gm_pcg(gm_ctx* c, int which, int prec, const double* b, double* x, double rtol, int maxit,
           int* iters, double* relres, cudaStream_t s, bool x_zero)
{
    const long long n = (which == 0 ? 3 : 1) * c->N;
    PcgScalars* sc = scal(c, which);
    // which 2 (A22 plus the fixed-stress term) is only used as a preconditioner
    // solve from a zero initial guess
    if (which == 2 && !x_zero) return c->set_err(GM_EINVAL, "PCG: fixed-stress operator needs x0 = 0");
    int rc;
    void *r, *z, *p, *p2, *q, *xx;
    const void* bb;
    // K_T solves may be preconditioned by a multigrid V-cycle; a grid that
    // cannot be coarsened keeps the block-Jacobi preconditioner
    bool use_mg = which == 0 && c->precond == 1;
    if (use_mg) {
        rc = gm_mg_prepare(c, prec, s);
        if (rc == GM_EINVAL) use_mg = false;
        else if (rc) return rc;
    }
    // Both precisions iterate on a correction d from d = 0 in an internal buffer
    // (so the captured graphs see fixed pointers); x += d at the end.
    if (prec == GM_F64) {
        r = (which == 0 ? c->k_r : c->a_r).p;
        z = (which == 0 ? c->k_z : c->a_z).p;
        p = (which == 0 ? c->k_p : c->a_p).p;
        p2 = (which == 0 ? c->k_p2 : c->a_p2).p;
        q = (which == 0 ? c->k_q : c->a_q).p;
        xx = (which == 0 ? c->k_x64 : c->a_x64).p;
        GM_CUDA_TRY(c, cudaMemsetAsync(xx, 0, n * sizeof(double), s));
        bb = b;
        if (x_zero) {
            GM_CUDA_TRY(c, cudaMemsetAsync(x, 0, n * sizeof(double), s));
            if ((rc = gm_launch_pcg_init(c, which, GM_F64, bb, nullptr, r, z, p, rtol, sc, s))) return rc;
        } else {
            // q = A x for the initial residual
            if ((rc = apply_inner(c, which, GM_F64, x, q, s, nullptr))) return rc;
            if ((rc = gm_launch_pcg_init(c, which, GM_F64, bb, q, r, z, p, rtol, sc, s))) return rc;
        }
    } else {
        r = (which == 0 ? c->k_r32 : c->a_r32).p;
        z = (which == 0 ? c->k_z32 : c->a_z32).p;
        p = (which == 0 ? c->k_p32 : c->a_p32).p;
        p2 = (which == 0 ? c->k_pb32 : c->a_pb32).p;
        q = (which == 0 ? c->k_q32 : c->a_q32).p;
        xx = (which == 0 ? c->k_x32 : c->a_x32).p;
        float* b32 = (which == 0 ? c->k_b32 : c->a_b32).as<float>();
        double* bsc = reinterpret_cast<double*>(c->dscal.as<PcgScalars>() + 8 + which);
        // FP64 residual of the initial guess, then FP32 correction solve from 0
        if (x_zero) {
            GM_CUDA_TRY(c, cudaMemsetAsync(x, 0, n * sizeof(double), s));
            if ((rc = gm_launch_cast_scaled_d2f(c, n, b, b32, bsc, s))) return rc;
        } else {
            double* q64 = (which == 0 ? c->k_q : c->a_q).as<double>();
            if ((rc = apply_inner(c, which, GM_F64, x, q64, s, nullptr))) return rc;
            double* r64 = (which == 0 ? c->k_r : c->a_r).as<double>();
            GM_CUDA_TRY(c, cudaMemcpyAsync(r64, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            if ((rc = gm_launch_axpby(c, n, -1.0, q64, 1.0, r64, s))) return rc;
            if ((rc = gm_launch_cast_scaled_d2f(c, n, r64, b32, bsc, s))) return rc;
        }
        GM_CUDA_TRY(c, cudaMemsetAsync(xx, 0, n * sizeof(float), s));
        bb = b32;
        if ((rc = gm_launch_pcg_init(c, which, GM_F32, bb, nullptr, r, z, p, rtol, sc, s))) return rc;
    }
    if (use_mg) {
        // z = V(r) replaces the block-Jacobi z of the init pass
        if ((rc = gm_mg_vcycle(c, prec, r, z, &sc->done, s))) return rc;
        if ((rc = gm_launch_pcg_rz(c, prec, r, z, sc, 1, s))) return rc;
    }
    PcgScalars* hs = static_cast<PcgScalars*>(c->hpin);
    int batch = 4;
    void* pp[2] = {p, p2};   // search direction, double-buffered across iterations
    // two iterations (one per direction buffer): enqueue directly or as a graph
    auto two_iterations = [&](cudaStream_t st) -> int {
        int e;
        for (int k = 0; k < 2; ++k) {
            void* pold = pp[k];
            void* pnew = pp[k ^ 1];
            if (prec == GM_F64)
                e = gm_launch_pcg_apply_f64(c, which, (const double*)z, (const double*)pold,
                                            (double*)pnew, (double*)q, sc, st);
            else
                e = gm_launch_pcg_apply_f32(c, which, (const float*)z, (const float*)pold,
                                            (float*)pnew, (float*)q, sc, st);
            if (e) return e;
            if (use_mg) {
                if ((e = gm_launch_pcg_update_noz(c, prec, xx, r, pnew, q, sc, maxit, st))) return e;
                if ((e = gm_mg_vcycle(c, prec, r, z, &sc->done, st))) return e;
                if ((e = gm_launch_pcg_rz(c, prec, r, z, sc, 0, st))) return e;
                continue;
            }
            if ((e = gm_launch_pcg_update(c, which, prec, xx, r, z, pnew, q, sc, maxit, st))) return e;
        }
        return GM_OK;
    };
    cudaGraphExec_t gexec = nullptr;
    const int pi = prec == GM_F64 ? (use_mg ? 3 : 0) : (use_mg ? 2 : 1);
    if (c->use_graphs) {
        // the graph bakes in the kernel parameters: dt (A22 operators), maxit and
        // the solution pointer; rebuild when any of them changes
        cudaGraphExec_t& slot = c->pcg_graph[which][pi];
        const double gdt = which == 0 ? 0.0 : c->dt;
        if (slot && (c->pcg_graph_dt[which][pi] != gdt || c->pcg_graph_maxit[which][pi] != maxit)) {
            cudaGraphExecDestroy(slot);
            slot = nullptr;
        }
        if (!slot) {
            if (!c->cap_stream)
                GM_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            const long long l0 = c->launches, a0 = c->applies;
            GM_CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = two_iterations(c->cap_stream);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
            if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
            if (ec != cudaSuccess) return c->set_err(GM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
            const cudaError_t ei = cudaGraphInstantiate(&slot, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) { slot = nullptr; return c->set_err(GM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei)); }
            c->pcg_graph_dt[which][pi] = gdt;
            c->pcg_graph_maxit[which][pi] = maxit;
            c->pcg_graph_launches[which][pi] = c->launches - l0;
            c->launches = l0;
            c->applies = a0;
        }
        gexec = slot;
    }
    for (;;) {
        for (int k = 0; k < batch; k += 2) {
            if (gexec) {
                GM_CUDA_TRY(c, cudaGraphLaunch(gexec, s));
                c->launches += c->pcg_graph_launches[which][pi];
                c->applies += 2;
            } else if ((rc = two_iterations(s))) {
                return rc;
            }
        }
        GM_CUDA_TRY(c, cudaMemcpyAsync(hs, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(c, cudaStreamSynchronize(s));
        if (hs->done) break;
        if (batch < 32) batch *= 2;
    }
    if (prec != GM_F64) {
        const double* bsc = reinterpret_cast<const double*>(c->dscal.as<PcgScalars>() + 8 + which);
        if ((rc = gm_launch_axpy_scaled_f2d(c, n, bsc, (const float*)xx, x, s))) return rc;
    } else {
        if ((rc = gm_launch_axpby(c, n, 1.0, (const double*)xx, 1.0, x, s))) return rc;
    }
    if (iters) *iters = hs->it;
    if (relres) *relres = hs->rr0 > 0 ? std::sqrt(hs->rr / hs->rr0) : 0.0;
    if (hs->status == GM_ENAN) return c->set_err(GM_ENAN, "PCG: non-finite value");
    if (hs->status == GM_ENOCONV)
        return c->set_err(GM_ENOCONV, "PCG: iteration limit or breakdown (which=" + std::to_string(which) + ")");
    return GM_OK;
}

static int dot2(gm_ctx* c, long long n, const double* x, const double* y, const double* x2,
                const double* y2, double* out, cudaStream_t s)
{
    double* dout = reinterpret_cast<double*>(c->dscal.as<PcgScalars>() + 4);
    int rc = gm_launch_dot(c, n, x, y, x2, y2, dout, s);
    if (rc) return rc;
    double* h = reinterpret_cast<double*>(static_cast<char*>(c->hpin) + 512);
    GM_CUDA_TRY(c, cudaMemcpyAsync(h, dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    out[0] = h[0];
    out[1] = h[1];
    return GM_OK;
}

// Products of the outer iteration.  In FP32-refined solves (prec GM_F32) the
// outer CG only has to reach its loose tolerance before the FP64 Newton
// residual refines, so its operator products run in FP32 (operands cast to FP32
// once, products cast back); dot products and vector updates stay FP64.
namespace {
struct OuterOps {
    gm_ctx* c;
    int prec;
    cudaStream_t s;
    float* a32;
    float* b32;
    // t3 (3N) = A_pu p ; the FP32 copy of p stays in a32[0, N) for a22()
    int apu(const double* p, double* t3) {
        if (prec == GM_F64) return gm_launch_apply_f64(c, GM_MODE_APU, 0, 1, 0, 0, 0, nullptr, p, t3, nullptr, s, nullptr);
        int rc = gm_launch_copy_cast_d2f(c, c->N, p, a32, s);
        if (!rc) rc = gm_launch_apply_f32(c, GM_MODE_APU, 0, 1, 0, 0, 0, nullptr, a32, b32, nullptr, s, nullptr);
        if (!rc) rc = gm_launch_copy_cast_f2d(c, 3 * c->N, b32, t3, s);
        return rc;
    }
    // q (N) = A22 p, p as given to the last apu() call
    int a22(const double* p, double* q) {
        if (prec == GM_F64) return gm_launch_apply_f64(c, GM_MODE_A22, 0, 0, 0, 1, c->dt, nullptr, p, nullptr, q, s, nullptr);
        int rc = gm_launch_apply_f32(c, GM_MODE_A22, 0, 0, 0, 1, c->dt, nullptr, a32, nullptr, b32, s, nullptr);
        if (!rc) rc = gm_launch_copy_cast_f2d(c, c->N, b32, q, s);
        return rc;
    }
    // t1 (N) = A_up w
    int aup(const double* w, double* t1) {
        if (prec == GM_F64) return gm_launch_apply_f64(c, GM_MODE_AUP, 0, 0, 1, 0, 0, w, nullptr, nullptr, t1, s, nullptr);
        int rc = gm_launch_copy_cast_d2f(c, 3 * c->N, w, a32, s);
        if (!rc) rc = gm_launch_apply_f32(c, GM_MODE_AUP, 0, 0, 1, 0, 0, a32, nullptr, nullptr, b32, s, nullptr);
        if (!rc) rc = gm_launch_copy_cast_f2d(c, c->N, b32, t1, s);
        return rc;
    }
};
}  // namespace

// Prevost's partitioned CG on [K_T, -A_pu; A_up, A22] [x1; x2] = [b1; b2]:
//   y1 = K_T^-1 b1,  r = b2 - A_up y1          (right side of Eq. schur_system)
//   CG on S~ = A22 + A_up K_T^-1 A_pu, preconditioned by A22^-1, from x2 = 0
//   x1 = K_T^-1 (b1 + A_pu x2) = y1 + sum_k alpha_k K_T^-1 A_pu p_k  (accumulated)
// The preconditioner and the Schur products use inner PCG solves, so the outer
// iteration uses the flexible (Polak-Ribiere) beta, which equals the
// Fletcher-Reeves one when the inner solves are exact.
int gm_prevost(gm_ctx* c, int prec, const double* b1, const double* b2, double* x1, double* x2,
               double outer_rtol, int outer_maxit, double inner_rtol, int inner_maxit,
               int* outer_it, long long* inner_k, long long* inner_a, double* relres,
               cudaStream_t s, int schur_precond)
{
    const int pw = schur_precond == 1 ? 2 : 1;   // preconditioner operator
    const long long N = c->N, N3 = 3 * N;
    int rc, it_in;
    double* y1 = c->o_y1.as<double>();
    double* w = c->o_w.as<double>();
    double* t3 = c->o_t3.as<double>();
    double* r = c->o_r.as<double>();
    double* z = c->o_z.as<double>();
    double* zold = c->o_zold.as<double>();
    double* p = c->o_p.as<double>();
    double* q = c->o_q.as<double>();
    double* t1 = c->o_t1.as<double>();
    long long ik = 0, ia = 0;
    OuterOps ops{c, prec == GM_F64 ? GM_F64 : GM_F32, s, c->o_s32a.as<float>(), c->o_s32b.as<float>()};

    rc = gm_pcg(c, 0, prec, b1, y1, inner_rtol, inner_maxit, &it_in, nullptr, s, true);
    if (rc && rc != GM_ENOCONV) return rc;
    ik += it_in;
    if ((rc = ops.aup(y1, t1))) return rc;
    GM_CUDA_TRY(c, cudaMemcpyAsync(r, b2, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if ((rc = gm_launch_axpby(c, N, -1.0, t1, 1.0, r, s))) return rc;
    GM_CUDA_TRY(c, cudaMemsetAsync(x2, 0, N * sizeof(double), s));
    GM_CUDA_TRY(c, cudaMemcpyAsync(x1, y1, N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rc = gm_pcg(c, pw, prec, r, z, inner_rtol, inner_maxit, &it_in, nullptr, s, true);
    if (rc && rc != GM_ENOCONV) return rc;
    ia += it_in;
    GM_CUDA_TRY(c, cudaMemcpyAsync(p, z, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double d[2];
    if ((rc = dot2(c, N, r, z, r, r, d, s))) return rc;
    double rz = d[0];
    const double rr0 = d[1];
    double rr = rr0;
    int it = 0;
    while (rr0 > 0.0 && rr > outer_rtol * outer_rtol * rr0) {
        if (it >= outer_maxit) {
            if (outer_it) *outer_it = it;
            return c->set_err(GM_ENOCONV, "partitioned CG: iteration limit");
        }
        // w = K_T^-1 A_pu p ;  q = A22 p + A_up w
        if ((rc = ops.apu(p, t3))) return rc;
        rc = gm_pcg(c, 0, prec, t3, w, inner_rtol, inner_maxit, &it_in, nullptr, s, true);
        if (rc && rc != GM_ENOCONV) return rc;
        ik += it_in;
        if ((rc = ops.a22(p, q))) return rc;
        if ((rc = ops.aup(w, t1))) return rc;
        if ((rc = gm_launch_axpby(c, N, 1.0, t1, 1.0, q, s))) return rc;
        if ((rc = dot2(c, N, p, q, nullptr, nullptr, d, s))) return rc;
        const double pq = d[0];
        if (!(pq > 0.0) || !std::isfinite(pq)) return c->set_err(GM_ENAN, "partitioned CG: breakdown (p.S p <= 0)");
        const double alpha = rz / pq;
        if ((rc = gm_launch_axpby(c, N, alpha, p, 1.0, x2, s))) return rc;
        if ((rc = gm_launch_axpby(c, N3, alpha, w, 1.0, x1, s))) return rc;
        if ((rc = gm_launch_axpby(c, N, -alpha, q, 1.0, r, s))) return rc;
        GM_CUDA_TRY(c, cudaMemcpyAsync(zold, z, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        rc = gm_pcg(c, pw, prec, r, z, inner_rtol, inner_maxit, &it_in, nullptr, s, true);
        if (rc && rc != GM_ENOCONV) return rc;
        ia += it_in;
        if ((rc = dot2(c, N, r, z, r, zold, d, s))) return rc;
        const double rz_new = d[0];
        const double beta = (rz_new - d[1]) / rz;
        if ((rc = dot2(c, N, r, r, nullptr, nullptr, d, s))) return rc;
        rr = d[0];
        if (!std::isfinite(rr)) return c->set_err(GM_ENAN, "partitioned CG: non-finite residual");
        if ((rc = gm_launch_axpby(c, N, 1.0, z, beta, p, s))) return rc;
        rz = rz_new;
        ++it;
    }
    if (outer_it) *outer_it = it;
    if (inner_k) *inner_k += ik;
    if (inner_a) *inner_a += ia;
    if (relres) *relres = rr0 > 0 ? std::sqrt(rr / rr0) : 0.0;
    return GM_OK;
}
