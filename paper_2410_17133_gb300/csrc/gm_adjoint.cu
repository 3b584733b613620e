// Adjoint of the last converged implicit step, and the parameter set-up calls
// it needs (per-element permeability, per-pair friction without a rebind).
//
// For the converged step F(x; theta) = 0 (Sec. 3.3.1, residuals of Eq.
// nonlinear_system, x = (u, p) at the end of the step, previous state fixed) and
// an objective J(x):  dJ/dtheta = -lambda^T dF/dtheta  with
// (dF/dx)^T lambda = (dJ/dx)^T on the free dofs.  dF/dx is the consistent
// Jacobian with the fault states frozen; for slipping pairs its cohesive block
// is the symmetric Newton tangent minus f k_n tau n^T (Sec. 2.2.1, Eq. corrector
// differentiated at fixed state).  The transposed system
//     [K_b + K_coh^T   A_pu ] [l_u]   [g_u]
//     [   -A_up        A22  ] [l_p] = [g_p]
// is solved by flexible GMRES, right-preconditioned by Prevost's partitioned CG
// on the symmetric Newton Jacobian (Sec. 3.3.2) applied to (r_u, -r_p), whose
// p-part is negated back.
//   d F_f / d log k_e = dt (k_e/mu) L_e p_e        -> g_logk[e] = -dt l_p,e . (k_e/mu) L_e p_e
//   d F_m / d f_i     = +- A_i t'_n tau  (slipping) -> g_f[i] = -A_i t'_n tau . [[l_u]]_i
//   d F_f / d log Q   = -dt f^p                     -> g_logQ = dt l_p . f^p
#include <cmath>
#include <string>
#include <vector>

#include "gm_internal.cuh"

namespace {

// g = dJ/dx on the free dofs: dJ/du, plus the lip terms of dJ/dslip
// (slip = P_t [[u]] in the fault frame), plus dJ/dp folded onto tied masters.
__global__ void adj_rhs_kernel(GridDesc g, const double* dJu, const double* dJp, const double* dJs,
                               const uint8_t* mask, double t1x, double t1y, double t1z, double t2x,
                               double t2y, double t2z, double* out)
{
    const long long N = g.N;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const unsigned m = mask[n];
    const long long kk = n / g.nb, pid = n - kk * g.nb;
    double gu[3] = {0, 0, 0};
    if (dJu)
        for (int c = 0; c < 3; ++c) gu[c] = dJu[c * N + n];
    if (dJs && g.kf >= 0 && (kk == g.kf || kk == g.kf + 1)) {
        const double sg = kk == g.kf + 1 ? 1.0 : -1.0;
        const long long P = g.nb;
        const double a = dJs[pid], b = dJs[P + pid];
        gu[0] += sg * (a * t1x + b * t2x);
        gu[1] += sg * (a * t1y + b * t2y);
        gu[2] += sg * (a * t1z + b * t2z);
    }
    for (int c = 0; c < 3; ++c) out[c * N + n] = ((m >> c) & 1u) ? 0.0 : gu[c];
    double gp = dJp ? dJp[n] : 0.0;
    const bool slave = g.tied && kk == g.kf + 1;
    if (g.tied && kk == g.kf && dJp) gp += dJp[n + g.nb];
    out[3 * N + n] = (slave || ((m >> 3) & 1u)) ? 0.0 : gp;
}

__global__ void adj_flip_p_kernel(long long N, const double* in, double* out)
{
    // out = (in_u, -in_p)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 4 * N;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = i < 3 * N ? in[i] : -in[i];
}

struct GradArgs {
    GridDesc g;
    const double* lp;    // lambda_p (N)
    const double* p;     // accepted pressure (N)
    const double* kap;   // k/mu per element
    double L[64];
    double dt;
    double* gk;          // per element
};

__global__ void adj_grad_logk_kernel(const GradArgs a)
{
    const long long nel = (long long)a.g.nx * a.g.ny * a.g.nz;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nel) return;
    const int ei = (int)(e % a.g.nx), ej = (int)((e / a.g.nx) % a.g.ny), ek = (int)(e / ((long long)a.g.nx * a.g.ny));
    const int kb = ek + ((a.g.kf >= 0 && ek >= a.g.kf) ? 1 : 0);
    double lv[8], pv[8];
    for (int loc = 0; loc < 8; ++loc) {
        const int ax = loc & 1, ay = (loc >> 1) & 1, az = (loc >> 2) & 1;
        long long node = (ei + ax) + (long long)(a.g.nx + 1) * ((ej + ay) + (long long)(a.g.ny + 1) * (kb + az));
        if (a.g.tied && kb + az == a.g.kf + 1) node -= a.g.nb;   // slave lip -> master dof
        lv[loc] = a.lp[node];
        pv[loc] = a.p[node];
    }
    double s = 0.0;
    for (int i = 0; i < 8; ++i) {
        double t = 0.0;
        for (int j = 0; j < 8; ++j) t += a.L[8 * i + j] * pv[j];
        s += lv[i] * t;
    }
    a.gk[e] = -a.dt * a.kap[e] * s;
}

__global__ void adj_grad_f_kernel(GridDesc g, const double* lu, const double* tn, const double* tauc,
                                  double Aq, double* gf)
{
    const long long P = g.nb;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const long long N = g.N;
    const long long nm = i + g.nb * g.kf, np = nm + g.nb;
    if (tauc[3 * P + i] == 0.0) { gf[i] = 0.0; return; }
    const int pi = (int)(i % (g.nx + 1)), pj = (int)(i / (g.nx + 1));
    const int nqi = (pi > 0) + (pi < g.nx), nqj = (pj > 0) + (pj < g.ny);
    const double Ai = Aq * 0.25 * nqi * nqj;
    double d = 0.0;
    for (int c = 0; c < 3; ++c) d += tauc[c * P + i] * (lu[c * N + np] - lu[c * N + nm]);
    gf[i] = -Ai * tn[i] * d;
}

// Frozen pair data of the current return map, 6 per pair (field-major):
// state, t'_n, |t^tr|, F, tau_1, tau_2 (slip direction in the fault frame).
__global__ void adj_frozen_kernel(long long P, const int8_t* st, const double* tn, const double* F,
                                  const double* tauc, const double* fpair, double fs, double t1x,
                                  double t1y, double t1z, double t2x, double t2y, double t2z, double* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const double f = fpair ? fpair[i] : fs;
    const double tx = tauc[i], ty = tauc[P + i], tz = tauc[2 * P + i];
    out[i] = (double)st[i];
    out[P + i] = tn[i];
    out[2 * P + i] = F[i] + f * tn[i];                // |t^tr|
    out[3 * P + i] = F[i];
    out[4 * P + i] = tx * t1x + ty * t1y + tz * t1z;
    out[5 * P + i] = tx * t2x + ty * t2y + tz * t2z;
}

// mu_n = -(dF_{n+1}/dh_n)^T lambda_{n+1} + (dH_{n+1}/dh_n)^T mu_{n+1}, with the
// later step's frozen data fz (see the multi-step reverse sweep).
__global__ void adj_mu_kernel(GridDesc g, const double* fz, const double* lam_u, const double* mu_next,
                              const double* fpair, double fs, double ks, double Aq, double t1x, double t1y,
                              double t1z, double t2x, double t2y, double t2z, double* mu)
{
    const long long P = g.nb;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const long long N = g.N;
    const long long nm = i + g.nb * g.kf, np = nm + g.nb;
    const int pi = (int)(i % (g.nx + 1)), pj = (int)(i / (g.nx + 1));
    const int nqi = (pi > 0) + (pi < g.nx), nqj = (pj > 0) + (pj < g.ny);
    const double Ai = Aq * 0.25 * nqi * nqj;
    const double dx = lam_u[np] - lam_u[nm], dy = lam_u[N + np] - lam_u[N + nm];
    const double dz = lam_u[2 * N + np] - lam_u[2 * N + nm];
    const double d1 = dx * t1x + dy * t1y + dz * t1z, d2 = dx * t2x + dy * t2y + dz * t2z;
    const int st = (int)fz[i];
    const double m1 = mu_next ? mu_next[i] : 0.0, m2 = mu_next ? mu_next[P + i] : 0.0;
    double o1 = 0.0, o2 = 0.0;
    if (st == GM_STICK) {
        o1 = Ai * ks * d1 + m1;
        o2 = Ai * ks * d2 + m2;
    } else if (st == GM_SLIP) {
        const double f = fpair ? fpair[i] : fs;
        const double tn = fz[P + i], nt = fz[2 * P + i], F = fz[3 * P + i];
        const double a = fz[4 * P + i], b = fz[5 * P + i];
        const double r = f * tn / nt;
        const double dp = a * d1 + b * d2, mp = a * m1 + b * m2;
        const double c1 = 1.0 - F / nt;
        o1 = Ai * ks * r * (d1 - a * dp) + c1 * (m1 - a * mp);
        o2 = Ai * ks * r * (d2 - b * dp) + c1 * (m2 - b * mp);
    } else {
        o1 = m1;
        o2 = m2;
    }
    mu[i] = o1;
    mu[P + i] = o2;
}

// (dH_n/dx_n)^T mu_n added on the lips of b (this step's frozen data fz), and
// mu^T dH/df into gf (added).
__global__ void adj_hist_rhs_kernel(GridDesc g, const double* fz, const double* mu, const double* fpair,
                                    double fs, double kn, double ks, double t1x, double t1y, double t1z,
                                    double t2x, double t2y, double t2z, double nx_, double ny_, double nz_,
                                    const uint8_t* mask, double* b, double* gf)
{
    const long long P = g.nb;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    if ((int)fz[i] != GM_SLIP) return;
    const long long N = g.N;
    const long long nm = i + g.nb * g.kf, np = nm + g.nb;
    const double f = fpair ? fpair[i] : fs;
    const double tn = fz[P + i], nt = fz[2 * P + i], F = fz[3 * P + i];
    const double a = fz[4 * P + i], bb = fz[5 * P + i];
    const double m1 = mu[i], m2 = mu[P + i];
    const double tm = a * m1 + bb * m2;
    const double ratio = F / nt;
    const double g1 = a * tm + ratio * (m1 - a * tm), g2 = bb * tm + ratio * (m2 - bb * tm);
    const double gn = f * kn / ks * tm;
    const double v[3] = {g1 * t1x + g2 * t2x + gn * nx_, g1 * t1y + g2 * t2y + gn * ny_,
                         g1 * t1z + g2 * t2z + gn * nz_};
    const unsigned mp = mask[np], mm = mask[nm];
    for (int c = 0; c < 3; ++c) {
        if (!((mp >> c) & 1u)) b[c * N + np] += v[c];
        if (!((mm >> c) & 1u)) b[c * N + nm] -= v[c];
    }
    if (gf) gf[i] += -(tn / ks) * tm;
}

int ensure_adjoint_buffers(gm_ctx* c, int m)
{
    if (c->adj_m >= m) return GM_OK;
    const size_t v = (size_t)4 * c->N * sizeof(double);
    cudaError_t e;
    if ((e = c->adj_V.alloc(v * (m + 1))) != cudaSuccess ||
        (e = c->adj_Z.alloc(v * m)) != cudaSuccess || (e = c->adj_w.alloc(v)) != cudaSuccess ||
        (e = c->adj_b.alloc(v)) != cudaSuccess || (e = c->adj_x.alloc(v)) != cudaSuccess ||
        (e = c->adj_t.alloc(v)) != cudaSuccess || (e = c->adj_s.alloc(v)) != cudaSuccess ||
        (e = c->adj_u.alloc(v)) != cudaSuccess)
        return c->set_err(GM_ENOMEM, std::string("adjoint: cudaMalloc: ") + cudaGetErrorString(e));
    c->adj_m = m;
    return GM_OK;
}

int dot(gm_ctx* c, long long n, const double* x, const double* y, double* out, cudaStream_t s)
{
    double* d = reinterpret_cast<double*>(c->dscal.as<PcgScalars>() + 7);
    int rc = gm_launch_dot(c, n, x, y, nullptr, nullptr, d, s);
    if (rc) return rc;
    double* h = reinterpret_cast<double*>(static_cast<char*>(c->hpin) + 3584);
    GM_CUDA_TRY(c, cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    *out = h[0];
    return GM_OK;
}

// Row/column scaling of the adjoint system: S = diag(K_b, A22)^(-1/2) (1 on
// rows without a positive diagonal).  GMRES runs on S J^T S, so that force and
// flow rows, whose units differ by many orders of magnitude on layered
// problems, weigh alike in its residual norm.
__global__ void adj_make_scale_kernel(long long N, const double* dK, const double* dA, double* S)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 4 * N;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = i < 3 * N ? dK[i] : dA[i - 3 * N];
        S[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    }
}
// y = S x (inv = 0) or y = x / S (inv = 1); y may alias x
__global__ void adj_scale_kernel(long long n, const double* S, const double* x, double* y, int inv)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = inv ? x[i] / S[i] : x[i] * S[i];
}

// y = J_cons^T x (free dofs)
int apply_adjoint_operator(gm_ctx* c, const double* x, double* y, cudaStream_t s)
{
    const long long N = c->N;
    c->fault_cons = 2;
    const int rc = gm_launch_apply_f64(c, GM_MODE_J, 1, 1, -1, 1, c->dt, x, x + 3 * N, y, y + 3 * N, s, nullptr);
    c->fault_cons = 0;
    return rc;
}

// z = flip(Prevost_sym(flip(v)))
int apply_preconditioner(gm_ctx* c, const double* v, double* z, double prtol, int pmaxit,
                         cudaStream_t s, long long* inner_k)
{
    const long long N = c->N;
    double* t = c->adj_t.as<double>();
    adj_flip_p_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(N, v, t);
    GM_LAUNCHED(c);
    int oit = 0;
    long long ia = 0;
    double rr = 0;
    int rc = gm_prevost(c, c->adj_prec, t, t + 3 * N, z, z + 3 * N, prtol, pmaxit, prtol * 1e-2, 20000, &oit,
                        inner_k, &ia, &rr, s, c->adj_schur);
    if (rc && rc != GM_ENOCONV) return rc;
    adj_flip_p_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(N, z, z);
    GM_LAUNCHED(c);
    return GM_OK;
}

}  // namespace

extern "C" int gm_set_permeability(gm_ctx* c, const double* k, int64_t n)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "set_permeability: not bound");
    if (!k || (n != 1 && n != c->n_el)) return c->set_err(GM_EINVAL, "set_permeability: n must be 1 or n_el");
    for (long long e = 0; e < c->n_el; ++e) {
        const double v = k[n == 1 ? 0 : e];
        if (!(v >= 0)) return c->set_err(GM_EINVAL, "set_permeability: k >= 0");
        c->kperm[e] = v;
    }
    return gm_upload_permeability(c);
}

extern "C" int gm_set_adjoint_options(gm_ctx* c, int precision, double prec_rtol, int schur_precond)
{
    if (!c) return GM_EINVAL;
    if (precision != GM_F64 && precision != GM_F32)
        return c->set_err(GM_EINVAL, "set_adjoint_options: precision must be GM_F64 or GM_F32");
    if (!(prec_rtol > 0 && prec_rtol < 1))
        return c->set_err(GM_EINVAL, "set_adjoint_options: prec_rtol must lie in (0, 1)");
    if (schur_precond != 0 && schur_precond != 1)
        return c->set_err(GM_EINVAL, "set_adjoint_options: schur_precond must be 0 or 1");
    c->adj_prec = precision;
    c->adj_prtol = prec_rtol;
    c->adj_schur = schur_precond;
    return GM_OK;
}

extern "C" int gm_set_friction(gm_ctx* c, const double* f, int64_t n)
{
    if (!c) return GM_EINVAL;
    if (!c->bound || !c->has_fault) return c->set_err(GM_ESTATE, "set_friction: needs a bound fault");
    if (!f || (n != 1 && n != c->P)) return c->set_err(GM_EINVAL, "set_friction: n must be 1 or the pair count");
    if (n == 1) {
        if (!(f[0] >= 0)) return c->set_err(GM_EINVAL, "set_friction: f >= 0");
        c->fp.f = f[0];
        c->has_fpair = false;
        return GM_OK;
    }
    for (long long i = 0; i < n; ++i)
        if (!(f[i] >= 0)) return c->set_err(GM_EINVAL, "set_friction: f >= 0");
    GM_CUDA_TRY(c, cudaMemcpy(c->dfpair.p, f, n * sizeof(double), cudaMemcpyHostToDevice));
    c->has_fpair = true;
    return GM_OK;
}

// FGMRES solve of J_cons^T x = b (b in adj_b, x in adj_x), run on the scaled
// system (S J^T S) y = S b, x = S y.
static int adj_solve(gm_ctx* c, double rtol, int maxit, gm_solve_report* rep, cudaStream_t s)
{
    const long long N = c->N, n4 = 4 * N;
    const int m = 30;
    double* V = c->adj_V.as<double>();
    double* Z = c->adj_Z.as<double>();
    double* w = c->adj_w.as<double>();
    double* b = c->adj_b.as<double>();
    double* x = c->adj_x.as<double>();
    double* S = c->adj_s.as<double>();
    double* u = c->adj_u.as<double>();
    int rc;
    if ((rc = gm_launch_block_jacobi(c, s))) return rc;   // symmetric Newton tangent of the frozen state
    adj_make_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(N, c->ddiagK.as<double>(), c->ddiagA.as<double>(), S);
    GM_LAUNCHED(c);
    adj_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n4, S, b, b, 0);
    GM_LAUNCHED(c);
    // scaled operator and preconditioner
    auto op = [&](const double* v, double* y) -> int {
        adj_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n4, S, v, u, 0);
        GM_LAUNCHED(c);
        int e = apply_adjoint_operator(c, u, y, s);
        if (e) return e;
        adj_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n4, S, y, y, 0);
        GM_LAUNCHED(c);
        return GM_OK;
    };
    auto prec = [&](const double* v, double* z, double prt, long long* ikp) -> int {
        adj_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n4, S, v, u, 1);
        GM_LAUNCHED(c);
        int e = apply_preconditioner(c, u, z, prt, 500, s, ikp);
        if (e) return e;
        adj_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n4, S, z, z, 1);
        GM_LAUNCHED(c);
        return GM_OK;
    };
    GM_CUDA_TRY(c, cudaMemsetAsync(x, 0, n4 * sizeof(double), s));
    double beta0;
    if ((rc = dot(c, n4, b, b, &beta0, s))) return rc;
    beta0 = std::sqrt(beta0);
    long long ik = 0;
    int it = 0;
    double res = beta0;
    const double prtol = c->adj_prtol;
    // flexible GMRES(m), right preconditioned; restart from r = b - A x
    while (beta0 > 0 && res > rtol * beta0 && it < maxit) {
        double* r = V;   // V[0]
        if ((rc = op(x, w))) return rc;
        GM_CUDA_TRY(c, cudaMemcpyAsync(r, b, n4 * 8, cudaMemcpyDeviceToDevice, s));
        if ((rc = gm_launch_axpby(c, n4, -1.0, w, 1.0, r, s))) return rc;
        double beta;
        if ((rc = dot(c, n4, r, r, &beta, s))) return rc;
        beta = std::sqrt(beta);
        res = beta;
        if (!(beta > rtol * beta0)) break;
        if ((rc = gm_launch_axpby(c, n4, 1.0 / beta, r, 0.0, r, s))) return rc;
        std::vector<double> H((m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), gv(m + 1, 0.0);
        gv[0] = beta;
        int j;
        for (j = 0; j < m && it < maxit; ++j, ++it) {
            double* vj = V + (size_t)j * n4;
            double* zj = Z + (size_t)j * n4;
            if ((rc = prec(vj, zj, prtol, &ik))) return rc;
            if ((rc = op(zj, w))) return rc;
            for (int i = 0; i <= j; ++i) {
                double h;
                if ((rc = dot(c, n4, w, V + (size_t)i * n4, &h, s))) return rc;
                H[i * m + j] = h;
                if ((rc = gm_launch_axpby(c, n4, -h, V + (size_t)i * n4, 1.0, w, s))) return rc;
            }
            double hn;
            if ((rc = dot(c, n4, w, w, &hn, s))) return rc;
            hn = std::sqrt(hn);
            H[(j + 1) * m + j] = hn;
            if (hn > 0)
                if ((rc = gm_launch_axpby(c, n4, 1.0 / hn, w, 0.0, V + (size_t)(j + 1) * n4, s))) return rc;
            for (int i = 0; i < j; ++i) {
                const double a = H[i * m + j], bb = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * bb;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            const double a = H[j * m + j], bb = H[(j + 1) * m + j];
            const double rr = std::sqrt(a * a + bb * bb);
            cs[j] = rr > 0 ? a / rr : 1.0;
            sn[j] = rr > 0 ? bb / rr : 0.0;
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            res = std::fabs(gv[j + 1]);
            if (!std::isfinite(res)) return c->set_err(GM_ENAN, "adjoint: non-finite GMRES residual");
            if (res <= rtol * beta0 || hn == 0) { ++j; ++it; break; }
        }
        // x += Z y,  H y = g (upper triangular j x j)
        std::vector<double> y(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double t = gv[i];
            for (int k = i + 1; k < j; ++k) t -= H[i * m + k] * y[k];
            y[i] = t / H[i * m + i];
        }
        for (int i = 0; i < j; ++i)
            if ((rc = gm_launch_axpby(c, n4, y[i], Z + (size_t)i * n4, 1.0, x, s))) return rc;
    }
    // true residual (scaled), then x = S y
    if ((rc = op(x, w))) return rc;
    if ((rc = gm_launch_axpby(c, n4, 1.0, b, -1.0, w, s))) return rc;
    double rfin;
    if ((rc = dot(c, n4, w, w, &rfin, s))) return rc;
    rfin = std::sqrt(rfin);
    adj_scale_kernel<<<GM_RED_BLOCKS, 256, 0, s>>>(n4, S, x, x, 0);
    GM_LAUNCHED(c);
    if (rep) {
        rep->iterations = it;
        rep->rel_residual = beta0 > 0 ? rfin / beta0 : 0.0;
        rep->status = GM_OK;
    }
    if (beta0 > 0 && rfin > 10 * rtol * beta0)
        return c->set_err(GM_ENOCONV, "adjoint: GMRES did not reach the tolerance (" + std::to_string(rfin / beta0) + ")");
    return GM_OK;
}

// gradients of this step from lambda (adj_x): -lambda^T dF/dtheta
static int adj_gradients(gm_ctx* c, double* g_logk, double* g_f, double* g_logQ, cudaStream_t s)
{
    const long long N = c->N;
    const double* lu = c->adj_x.as<double>();
    const double* lp = lu + 3 * N;
    int rc;
    if (g_logk) {
        GradArgs ga;
        ga.g = c->g;
        ga.lp = lp;
        ga.p = c->dp_n.as<double>();
        ga.kap = c->dK64.as<double>();
        for (int q = 0; q < 64; ++q) ga.L[q] = c->Lref[q];
        ga.dt = c->dt;
        ga.gk = g_logk;
        adj_grad_logk_kernel<<<(int)((c->n_el + 255) / 256), 256, 0, s>>>(ga);
        GM_LAUNCHED(c);
    }
    if (g_f && c->has_fault) {
        adj_grad_f_kernel<<<(int)((c->P + 255) / 256), 256, 0, s>>>(c->g, lu, c->dtn.as<double>(),
                                                                     c->dtauc.as<double>(), c->Aq, g_f);
        GM_LAUNCHED(c);
    }
    if (g_logQ) {
        double d;
        if ((rc = dot(c, N, lp, c->dfp.as<double>(), &d, s))) return rc;
        *g_logQ = c->dt * d;
    }
    return GM_OK;
}

static int adj_rhs(gm_ctx* c, const double* dJ_du, const double* dJ_dp, const double* dJ_dslip,
                   cudaStream_t s)
{
    const int nb = (int)((c->N + 255) / 256);
    adj_rhs_kernel<<<nb, 256, 0, s>>>(c->g, dJ_du, dJ_dp, dJ_dslip, c->dmask.as<uint8_t>(), c->t1[0],
                                      c->t1[1], c->t1[2], c->t2[0], c->t2[1], c->t2[2], c->adj_b.as<double>());
    GM_LAUNCHED(c);
    return GM_OK;
}

extern "C" int gm_adjoint_step(gm_ctx* c, const double* dJ_du, const double* dJ_dp, const double* dJ_dslip,
                               double* g_logk, double* g_f, double* g_logQ, double rtol, int maxit,
                               gm_solve_report* rep, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "adjoint: not bound");
    if (!(rtol > 0) || maxit < 1) return c->set_err(GM_EINVAL, "adjoint: bad tolerance or maxit");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_adjoint_buffers(c, 30);
    if (rc) return rc;
    if ((rc = adj_rhs(c, dJ_du, dJ_dp, dJ_dslip, s))) return rc;
    const int rs = adj_solve(c, rtol, maxit, rep, s);
    if (rs && rs != GM_ENOCONV) return rs;
    if ((rc = adj_gradients(c, g_logk, g_f, g_logQ, s))) return rc;
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    return rs;
}

extern "C" int gm_adjoint_sweep_step(gm_ctx* c, const double* dJ_du, const double* dJ_dp,
                                     const double* dJ_dslip, const double* lam_next, const double* mu_next,
                                     const double* frozen_next, double* lam, double* mu, double* frozen,
                                     double* g_logk, double* g_f, double* g_logQ, double rtol, int maxit,
                                     gm_solve_report* rep, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound || !c->has_fault) return c->set_err(GM_ESTATE, "adjoint sweep: needs a bound fault");
    if (!lam || !mu || !frozen) return c->set_err(GM_EINVAL, "adjoint sweep: null output");
    if ((lam_next == nullptr) != (frozen_next == nullptr))
        return c->set_err(GM_EINVAL, "adjoint sweep: lam_next and frozen_next go together");
    if (!(rtol > 0) || maxit < 1) return c->set_err(GM_EINVAL, "adjoint: bad tolerance or maxit");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_adjoint_buffers(c, 30);
    if (rc) return rc;
    const long long N = c->N, P = c->P;
    const int pb = (int)((P + 255) / 256);
    const double* fpair = c->has_fpair ? c->dfpair.as<double>() : nullptr;
    // this step's frozen pair data
    adj_frozen_kernel<<<pb, 256, 0, s>>>(P, c->dstate.as<int8_t>(), c->dtn.as<double>(), c->dF.as<double>(),
                                         c->dtauc.as<double>(), fpair, c->fp.f, c->t1[0], c->t1[1], c->t1[2],
                                         c->t2[0], c->t2[1], c->t2[2], frozen);
    GM_LAUNCHED(c);
    // mu_n from the later step
    if (lam_next) {
        adj_mu_kernel<<<pb, 256, 0, s>>>(c->g, frozen_next, lam_next, mu_next, fpair, c->fp.f, c->fp.ks, c->Aq,
                                         c->t1[0], c->t1[1], c->t1[2], c->t2[0], c->t2[1], c->t2[2], mu);
        GM_LAUNCHED(c);
    } else if (mu_next) {
        GM_CUDA_TRY(c, cudaMemcpyAsync(mu, mu_next, 2 * P * 8, cudaMemcpyDeviceToDevice, s));
    } else {
        GM_CUDA_TRY(c, cudaMemsetAsync(mu, 0, 2 * P * 8, s));
    }
    // right-hand side: direct terms + [A_pu l_p ; S l_p]_{n+1} + (dH_n/dx_n)^T mu_n
    if ((rc = adj_rhs(c, dJ_du, dJ_dp, dJ_dslip, s))) return rc;
    double* b = c->adj_b.as<double>();
    double* t = c->adj_t.as<double>();
    if (lam_next) {
        if ((rc = gm_launch_apply_f64(c, GM_MODE_APU, 0, 1, 0, 0, 0, nullptr, lam_next + 3 * N, t, nullptr, s, nullptr))) return rc;
        if ((rc = gm_launch_axpby(c, 3 * N, 1.0, t, 1.0, b, s))) return rc;
        if ((rc = gm_launch_apply_f64(c, GM_MODE_A22, 0, 0, 0, 1, 0, nullptr, lam_next + 3 * N, nullptr, t + 3 * N, s, nullptr))) return rc;
        if ((rc = gm_launch_axpby(c, N, 1.0, t + 3 * N, 1.0, b + 3 * N, s))) return rc;
    }
    if (g_f) GM_CUDA_TRY(c, cudaMemsetAsync(g_f, 0, P * 8, s));
    double* hist_gf = c->adj_w.as<double>();      // mu^T dH/df, reused below
    GM_CUDA_TRY(c, cudaMemsetAsync(hist_gf, 0, P * 8, s));
    adj_hist_rhs_kernel<<<pb, 256, 0, s>>>(c->g, frozen, mu, fpair, c->fp.f, c->fp.kn, c->fp.ks, c->t1[0], c->t1[1],
                                           c->t1[2], c->t2[0], c->t2[1], c->t2[2], c->nrm[0], c->nrm[1], c->nrm[2],
                                           c->dmask.as<uint8_t>(), b, hist_gf);
    GM_LAUNCHED(c);
    std::vector<double> hgf(P);
    GM_CUDA_TRY(c, cudaMemcpyAsync(hgf.data(), hist_gf, P * 8, cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    const int rs = adj_solve(c, rtol, maxit, rep, s);
    if (rs && rs != GM_ENOCONV) return rs;
    if ((rc = adj_gradients(c, g_logk, g_f, g_logQ, s))) return rc;
    if (g_f) {
        GM_CUDA_TRY(c, cudaMemcpyAsync(hist_gf, hgf.data(), P * 8, cudaMemcpyHostToDevice, s));
        if ((rc = gm_launch_axpby(c, P, 1.0, hist_gf, 1.0, g_f, s))) return rc;
    }
    GM_CUDA_TRY(c, cudaMemcpyAsync(lam, c->adj_x.p, 4 * N * 8, cudaMemcpyDeviceToDevice, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    return rs;
}
