// Fault return map, Newton residual, diagonal / block-diagonal preconditioners.
#include "gm_internal.cuh"

// ---------------------------------------------------------------------------
// Deterministic block reductions (fixed grid, last block sums the partials)
// ---------------------------------------------------------------------------
template <int NV>
__device__ void gm_block_sum(double (&v)[NV], double* sh /* NV * 32 */)
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

// Writes this block's partials; returns true in the (single) last block, whose
// thread 0 then holds the grand totals in v (summed in block order).
template <int NV>
__device__ bool gm_grid_sum(double (&v)[NV], double* part, unsigned* counter)
{
    __shared__ double sh[NV * 32];
    __shared__ bool last;
    gm_block_sum<NV>(v, sh);
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
    gm_block_sum<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = acc[k];
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

// ---------------------------------------------------------------------------
// Return map (Sec. 2.2.1).  Per pair i with jump [[u]] = u+ - u-:
//   delta_n = n.[[u]],  g_s = (t1.[[u]], t2.[[u]])
//   contact if t'_n0 - k_n delta_n >= 0 (total opening <= 0), then
//     t'_n = t'_n0 - k_n delta_n                      (Eq. normal_traction)
//   trial shear t^tr = tau0 + k_s (g_s - delta_ie_n)   (Eq. slip_split, elastic predictor)
//   F = |t^tr| - f t'_n                                (Eq. yield_function)
//   F > 0: d lambda = F / k_s, tau = t^tr/|t^tr|, t_s = f t'_n tau,
//          delta_ie = delta_ie_n + d lambda tau       (Eqs. plastic_slip_increment, corrector)
//   else stick: t_s = t^tr;  open: t' = 0.
// Incremental conjugate traction T = -(t'_n - t'_n0) n + (t_s - tau0), written
// without cancelling the in-situ values where the algebra allows.
// Tangent: stick k_n nn + k_s P_t; slip k_n nn + k_s (f t'_n/|t^tr|)(P_t - tau tau);
// open 0 (symmetric reading, so the Jacobian stays SPD for CG).
// ---------------------------------------------------------------------------
__global__ void gm_return_map_kernel(const LawArgs a)
{
    const long long P = a.g.nb;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const long long N = a.g.N;
    const long long nm = i + a.g.nb * a.g.kf, np = nm + a.g.nb;
    double j[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double up = a.un[c * N + np], um = a.un[c * N + nm];
        if (a.du) { up += a.du[c * N + np]; um += a.du[c * N + nm]; }
        j[c] = up - um;
    }
    const double dn = a.n[0] * j[0] + a.n[1] * j[1] + a.n[2] * j[2];
    const double g1 = a.t1[0] * j[0] + a.t1[1] * j[1] + a.t1[2] * j[2];
    const double g2 = a.t2[0] * j[0] + a.t2[1] * j[1] + a.t2[2] * j[2];
    const double fr = a.fpair ? a.fpair[i] : a.f;
    const double tn0 = a.insitu ? a.insitu[i] : a.tn0;
    const double t01 = a.insitu ? a.insitu[P + i] : a.tau0[0];
    const double t02 = a.insitu ? a.insitu[2 * P + i] : a.tau0[1];
    const double tnc = tn0 - a.kn * dn;
    const bool contact = tnc >= 0.0;
    const double dl1 = a.dlie_prev[i], dl2 = a.dlie_prev[P + i];
    const double tr1 = t01 + a.ks * (g1 - dl1);
    const double tr2 = t02 + a.ks * (g2 - dl2);
    const double nt = sqrt(tr1 * tr1 + tr2 * tr2);
    const double tn = contact ? tnc : 0.0;
    const double F = nt - fr * tn;
    const bool slip = contact && F > 0.0 && nt > 0.0;
    const bool stick = contact && !slip;
    double ts1 = 0.0, ts2 = 0.0, l1 = dl1, l2 = dl2, tau1 = 0.0, tau2 = 0.0, ratio = 0.0;
    double Ts1, Ts2;
    if (stick) {
        ts1 = tr1; ts2 = tr2;
        Ts1 = a.ks * (g1 - dl1);
        Ts2 = a.ks * (g2 - dl2);
    } else if (slip) {
        tau1 = tr1 / nt; tau2 = tr2 / nt;
        const double dlam = F / a.ks;
        ts1 = fr * tn * tau1; ts2 = fr * tn * tau2;
        l1 = dl1 + dlam * tau1; l2 = dl2 + dlam * tau2;
        Ts1 = ts1 - t01;
        Ts2 = ts2 - t02;
        ratio = fr * tn / nt;
    } else {
        Ts1 = -t01;
        Ts2 = -t02;
    }
    const double Tn = contact ? a.kn * dn : tn0;
    a.state[i] = contact ? (slip ? GM_SLIP : GM_STICK) : GM_OPEN;
    a.tn[i] = tn;
    a.ts[i] = ts1; a.ts[P + i] = ts2;
    a.dlie[i] = l1; a.dlie[P + i] = l2;
    a.F[i] = F;
    a.dn[i] = dn;
    a.gs[i] = g1; a.gs[P + i] = g2;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.T[c * P + i] = Tn * a.n[c] + Ts1 * a.t1[c] + Ts2 * a.t2[c];
    // tangent
    double D[6] = {0, 0, 0, 0, 0, 0};
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    if (contact) {
        const double tg[3] = {tau1 * a.t1[0] + tau2 * a.t2[0], tau1 * a.t1[1] + tau2 * a.t2[1],
                              tau1 * a.t1[2] + tau2 * a.t2[2]};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int x = ia[q], y = ib[q];
            const double nn = a.n[x] * a.n[y];
            const double pt = a.t1[x] * a.t1[y] + a.t2[x] * a.t2[y];
            D[q] = a.kn * nn + (stick ? a.ks * pt : a.ks * ratio * (pt - tg[x] * tg[y]));
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        a.D64[q * P + i] = D[q];
        if (a.D32) a.D32[q * P + i] = (float)D[q];
    }
    // consistent tangent of a slipping pair = D - f k_n tau n^T (frozen state)
    const double tgx = tau1 * a.t1[0] + tau2 * a.t2[0];
    const double tgy = tau1 * a.t1[1] + tau2 * a.t2[1];
    const double tgz = tau1 * a.t1[2] + tau2 * a.t2[2];
    a.tauc[i] = tgx;
    a.tauc[P + i] = tgy;
    a.tauc[2 * P + i] = tgz;
    a.tauc[3 * P + i] = slip ? -fr * a.kn : 0.0;
}

int gm_launch_return_map(gm_ctx* c, const double* un, const double* du, cudaStream_t s)
{
    if (c->g.kf < 0) return GM_OK;
    LawArgs a;
    a.g = c->g;
    a.un = un;
    a.du = du;
    a.dlie_prev = c->ddlie_n.as<double>();
    a.fpair = c->has_fpair ? c->dfpair.as<double>() : nullptr;
    a.insitu = c->has_insitu ? c->dinsitu.as<double>() : nullptr;
    a.tauc = c->dtauc.as<double>();
    a.kn = c->fp.kn; a.ks = c->fp.ks; a.f = c->fp.f; a.tn0 = c->fp.tn0;
    a.tau0[0] = c->fp.tau0[0]; a.tau0[1] = c->fp.tau0[1];
    for (int d = 0; d < 3; ++d) { a.n[d] = c->nrm[d]; a.t1[d] = c->t1[d]; a.t2[d] = c->t2[d]; }
    a.Aq = c->Aq;
    a.state = c->dstate.as<int8_t>();
    a.tn = c->dtn.as<double>();
    a.ts = c->dts.as<double>();
    a.dlie = c->ddlie.as<double>();
    a.T = c->dT.as<double>();
    a.F = c->dF.as<double>();
    a.dn = c->ddn.as<double>();
    a.gs = c->dgs.as<double>();
    a.D64 = c->dD64.as<double>();
    a.D32 = c->dD32.as<float>();
    const int nblk = (int)((c->P + 255) / 256);
    gm_return_map_kernel<<<nblk, 256, 0, s>>>(a);
    GM_LAUNCHED(c);
    return GM_OK;
}

// ---------------------------------------------------------------------------
// Newton residual, Eq. linear_system right-hand side:
//   b1 = f^u - (K_b u - A_pu p) - F_coh,    b2 = dt f^p - dt C p - (A_up du + S dp)
// y1 = RES1 apply on (u, p), y2p = RES2 apply on (du, dp).  Also the scaled norms
//   rhat^2 = sum b1^2/diag(K_b) + sum b2^2/diag(A22),
//   shat^2 = sum diag(K_b) u^2 + sum diag(A22) p^2      (free dofs)
// ---------------------------------------------------------------------------
struct ResArgs {
    ResidualInputs in;
    double* part;
    unsigned* counter;
    double* out;           // rhat^2, shat^2
};

__global__ void __launch_bounds__(256) gm_residual_kernel(const ResArgs a)
{
    const long long N = a.in.g.N;
    double v[2] = {0.0, 0.0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x)
        gm_residual_node(a.in, n, v);
    if (gm_grid_sum<2>(v, a.part, a.counter)) {
        a.out[0] = v[0];
        a.out[1] = v[1];
    }
}

ResidualInputs gm_residual_inputs(const gm_ctx* c, const double* y1u, const double* y1p, const double* y2p,
                                  const double* ut, const double* pt, double* b)
{
    ResidualInputs a;
    a.g = c->g;
    a.dt = c->dt;
    a.Aq = c->Aq;
    a.fu = c->dfu.as<double>();
    a.fp = c->dfp.as<double>();
    a.y1u = y1u; a.y1p = y1p; a.y2p = y2p; a.ut = ut; a.pt = pt;
    a.T = c->dT.as<double>();
    a.dK = c->ddiagK.as<double>();
    a.dA = c->ddiagA.as<double>();
    a.mask = c->dmask.as<uint8_t>();
    a.b = b;
    return a;
}

int gm_launch_residual(gm_ctx* c, const double* y1u, const double* y1p, const double* y2p,
                       const double* ut, const double* pt, double* b, cudaStream_t s, double* out2)
{
    ResArgs a;
    a.in = gm_residual_inputs(c, y1u, y1p, y2p, ut, pt, b);
    a.part = c->dpart.as<double>();
    a.counter = c->dcount.as<unsigned>();
    a.out = out2;
    gm_residual_kernel<<<GM_RED_BLOCKS, GM_RED_THREADS, 0, s>>>(a);
    GM_LAUNCHED(c);
    return GM_OK;
}

// ---------------------------------------------------------------------------
// Diagonals.  Bulk nodal 3x3 blocks of K_b and diag(A22) = diag(S + dt C),
// summed over the elements around each node (for a tied lower lip, also over
// the elements of its upper-lip slave), plus the fault storage / flow terms.
// ---------------------------------------------------------------------------
struct DiagArgs {
    GridDesc g;
    double Kblk[8][9];
    double Md[8], Ld[8];
    double invM, dt;
    const double* E;
    const double* kap;
    const uint8_t* mask;
    // fault
    double Aq, stor, lcoef, tcoef, Lfd[4];
    double* Kb6;      // 6N bulk blocks (upper triangle)
    double* dK;       // 3N
    double* dA;       // N
    double* Ainv64;   // N
    float* Ainv32;    // N
    const double* fs;     // per-element fixed-stress storage coefficient
    double* Afsinv64;     // N, Jacobi of A22 + fixed-stress term
    float* Afsinv32;
};

__global__ void __launch_bounds__(256) gm_diag_kernel(const DiagArgs a)
{
    const long long N = a.g.N;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const long long kk = n / a.g.nb;
    const long long pid = n - kk * a.g.nb;
    const int i = (int)(pid % (a.g.nx + 1)), j = (int)(pid / (a.g.nx + 1));
    double K9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double dA = 0.0, dfs = 0.0;
    const bool slave = a.g.tied && kk == a.g.kf + 1;
    auto add_layer = [&](int kb, int az, bool mech) {
        if (kb < 0 || kb + 1 >= a.g.nplanes || kb == a.g.kf) return;
        const int ek = (a.g.kf >= 0 && kb > a.g.kf) ? kb - 1 : kb;
        for (int ay = 0; ay < 2; ++ay)
            for (int ax = 0; ax < 2; ++ax) {
                const int ei = i - ax, ej = j - ay;
                if (ei < 0 || ei >= a.g.nx || ej < 0 || ej >= a.g.ny) continue;
                const long long e = ei + (long long)a.g.nx * (ej + (long long)a.g.ny * ek);
                const int loc = ax + 2 * ay + 4 * az;
                if (mech) {
                    const double E = a.E[e];
                    for (int q = 0; q < 9; ++q) K9[q] += E * a.Kblk[loc][q];
                }
                dA += a.invM * a.Md[loc] + a.dt * a.kap[e] * a.Ld[loc];
                dfs += a.fs[e] * a.Md[loc];
            }
    };
    add_layer((int)kk - 1, 1, true);
    add_layer((int)kk, 0, true);
    if (a.g.tied && kk == a.g.kf) {          // elements of the slave lip share this dof
        add_layer(a.g.kf + 1, 0, false);
    }
    if (a.g.kf >= 0 && (kk == a.g.kf || kk == a.g.kf + 1)) {
        const int nqi = (i > 0) + (i < a.g.nx), nqj = (j > 0) + (j < a.g.ny);
        const double Ai = a.Aq * 0.25 * nqi * nqj;
        double lap = 0.0;
        for (int dq = 0; dq < 4; ++dq) {
            const int qi = i - 1 + (dq & 1), qj = j - 1 + (dq >> 1);
            if (qi < 0 || qi >= a.g.nx || qj < 0 || qj >= a.g.ny) continue;
            const int b = (i - qi) + 2 * (j - qj);
            lap += a.Lfd[b];
        }
        if (a.g.tied) {
            if (kk == a.g.kf) dA += Ai * a.stor + a.dt * a.lcoef * lap;
        } else {
            dA += 0.25 * Ai * a.stor + 0.25 * a.dt * a.lcoef * lap + a.dt * Ai * a.tcoef;
        }
    }
    const int up[6] = {0, 1, 2, 4, 5, 8};
    for (int q = 0; q < 6; ++q) a.Kb6[q * N + n] = K9[up[q]];
    for (int c = 0; c < 3; ++c) a.dK[c * N + n] = K9[4 * c];
    const unsigned m = a.mask[n];
    const bool pfree = !slave && !((m >> 3) & 1u);
    a.dA[n] = pfree ? dA : 1.0;
    a.Ainv64[n] = pfree ? 1.0 / dA : 0.0;
    a.Ainv32[n] = pfree ? (float)(1.0 / dA) : 0.0f;
    a.Afsinv64[n] = pfree ? 1.0 / (dA + dfs) : 0.0;
    a.Afsinv32[n] = pfree ? (float)(1.0 / (dA + dfs)) : 0.0f;
}

int gm_launch_diag(gm_ctx* c, cudaStream_t s)
{
    DiagArgs a;
    a.g = c->g;
    for (int l = 0; l < 8; ++l) {
        for (int q = 0; q < 9; ++q) a.Kblk[l][q] = c->Kblk_ref[l][q];
        a.Md[l] = c->Mdiag_ref[l];
        a.Ld[l] = c->Ldiag_ref[l];
    }
    a.invM = 1.0 / c->M;
    a.dt = c->dt;
    a.E = c->dE64.as<double>();
    a.kap = c->dK64.as<double>();
    a.mask = c->dmask.as<uint8_t>();
    a.Aq = c->Aq;
    a.stor = c->has_fault ? c->fp.w0 / c->fp.MF : 0.0;
    a.lcoef = c->has_fault ? c->fp.wk_par / c->mu_f : 0.0;
    a.tcoef = (c->has_fault && c->fp.k_perp > 0) ? c->fp.k_perp / (c->mu_f * c->fp.w0) : 0.0;
    for (int b = 0; b < 4; ++b) a.Lfd[b] = c->Lf[b * 4 + b];
    a.Kb6 = c->dKinv64.as<double>() + 6 * c->N;   // second half of the buffer holds bulk blocks
    a.dK = c->ddiagK.as<double>();
    a.dA = c->ddiagA.as<double>();
    a.Ainv64 = c->dAinv64.as<double>();
    a.Ainv32 = c->dAinv32.as<float>();
    a.fs = c->dFS64.as<double>();
    a.Afsinv64 = c->dAfsinv64.as<double>();
    a.Afsinv32 = c->dAfsinv32.as<float>();
    const int nblk = (int)((c->N + 255) / 256);
    gm_diag_kernel<<<nblk, 256, 0, s>>>(a);
    GM_LAUNCHED(c);
    return GM_OK;
}

// 3x3 block-Jacobi of K_T: bulk block + A_i D at both lips; constrained
// components get zero rows/columns (z = 0 there).
struct BJArgs {
    GridDesc g;
    const double* Kb6;
    const double* D;     // 6P
    const uint8_t* mask;
    double Aq;
    double* inv64;       // 6N
    float* inv32;        // 6N
    __nv_bfloat16* inv16;   // 6N (the multigrid smoother's copy), or null
};

__global__ void __launch_bounds__(256) gm_block_jacobi_kernel(const BJArgs a)
{
    const long long N = a.g.N;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double B[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) B[q] = a.Kb6[q * N + n];
    const long long kk = n / a.g.nb;
    if (a.g.kf >= 0 && (kk == a.g.kf || kk == a.g.kf + 1)) {
        const long long pid = n - kk * a.g.nb;
        const int i = (int)(pid % (a.g.nx + 1)), j = (int)(pid / (a.g.nx + 1));
        const int nqi = (i > 0) + (i < a.g.nx), nqj = (j > 0) + (j < a.g.ny);
        const double Ai = a.Aq * 0.25 * nqi * nqj;
#pragma unroll
        for (int q = 0; q < 6; ++q) B[q] += Ai * a.D[q * a.g.nb + pid];
    }
    const unsigned m = a.mask[n];
    // symmetric 3x3 [b0 b1 b2; b1 b3 b4; b2 b4 b5]; constrained comps -> identity
    double b00 = B[0], b01 = B[1], b02 = B[2], b11 = B[3], b12 = B[4], b22 = B[5];
    if (m & 1u) { b00 = 1.0; b01 = 0.0; b02 = 0.0; }
    if (m & 2u) { b11 = 1.0; b01 = 0.0; b12 = 0.0; }
    if (m & 4u) { b22 = 1.0; b02 = 0.0; b12 = 0.0; }
    const double c00 = b11 * b22 - b12 * b12;
    const double c01 = b02 * b12 - b01 * b22;
    const double c02 = b01 * b12 - b02 * b11;
    const double c11 = b00 * b22 - b02 * b02;
    const double c12 = b01 * b02 - b00 * b12;
    const double c22 = b00 * b11 - b01 * b01;
    const double det = b00 * c00 + b01 * c01 + b02 * c02;
    const double id = 1.0 / det;
    double I[6] = {c00 * id, c01 * id, c02 * id, c11 * id, c12 * id, c22 * id};
    if (m & 1u) { I[0] = 0.0; I[1] = 0.0; I[2] = 0.0; }
    if (m & 2u) { I[3] = 0.0; I[1] = 0.0; I[4] = 0.0; }
    if (m & 4u) { I[5] = 0.0; I[2] = 0.0; I[4] = 0.0; }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        a.inv64[q * N + n] = I[q];
        a.inv32[q * N + n] = (float)I[q];
        if (a.inv16) a.inv16[q * N + n] = __float2bfloat16_rn((float)I[q]);
    }
}

// 6x6 block of a fault pair: both lips' 3x3 blocks (bulk + A_i D) and the
// coupling -A_i D between them.  The cohesive springs are stiff (k_n h / E of
// order 10-1000), so the two lips move nearly together and a preconditioner
// that inverts only nodal blocks cannot see that; the pair block does.
// Constrained components: zero row and column (z = 0 there).  The block is
// symmetric positive definite, so Gauss-Jordan without pivoting is stable.
__global__ void __launch_bounds__(128) gm_pair_block_kernel(const BJArgs a, double* pinv64, float* pinv32)
{
    const long long P = a.g.nb;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const long long N = a.g.N;
    const long long nm = q + P * a.g.kf, np = nm + P;
    const int i = (int)(q % (a.g.nx + 1)), j = (int)(q / (a.g.nx + 1));
    const int nqi = (i > 0) + (i < a.g.nx), nqj = (j > 0) + (j < a.g.ny);
    const double Ai = a.Aq * 0.25 * nqi * nqj;
    double M[6][6];
    const int sr[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};   // symmetric 3x3 storage
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double C = Ai * a.D[sr[r][c] * P + q];
            M[r][c] = a.Kb6[sr[r][c] * N + nm] + C;
            M[3 + r][3 + c] = a.Kb6[sr[r][c] * N + np] + C;
            M[r][3 + c] = -C;
            M[3 + r][c] = -C;
        }
    const unsigned mk = (a.mask[nm] & 7u) | ((a.mask[np] & 7u) << 3);
#pragma unroll
    for (int r = 0; r < 6; ++r)
        if ((mk >> r) & 1u)
#pragma unroll
            for (int c = 0; c < 6; ++c) { M[r][c] = (r == c) ? 1.0 : 0.0; M[c][r] = (r == c) ? 1.0 : 0.0; }
    double I[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) I[r][c] = (r == c) ? 1.0 : 0.0;
    for (int k = 0; k < 6; ++k) {
        const double piv = 1.0 / M[k][k];
        for (int c = 0; c < 6; ++c) { M[k][c] *= piv; I[k][c] *= piv; }
        for (int r = 0; r < 6; ++r) {
            if (r == k) continue;
            const double f = M[r][k];
            for (int c = 0; c < 6; ++c) { M[r][c] -= f * M[k][c]; I[r][c] -= f * I[k][c]; }
        }
    }
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
            const double v = (((mk >> r) | (mk >> c)) & 1u) ? 0.0 : I[r][c];
            pinv64[(r * 6 + c) * P + q] = v;
            pinv32[(r * 6 + c) * P + q] = (float)v;
        }
}

int gm_launch_block_jacobi(gm_ctx* c, cudaStream_t s)
{
    BJArgs a;
    a.g = c->g;
    a.Kb6 = c->dKinv64.as<double>() + 6 * c->N;
    a.D = c->dD64.as<double>();
    a.mask = c->dmask.as<uint8_t>();
    a.Aq = c->Aq;
    a.inv64 = c->dKinv64.as<double>();
    a.inv32 = c->dKinv32.as<float>();
    a.inv16 = c->dKinv16.as<__nv_bfloat16>();
    const int nblk = (int)((c->N + 255) / 256);
    gm_block_jacobi_kernel<<<nblk, 256, 0, s>>>(a);
    GM_LAUNCHED(c);
    if (c->g.kf >= 0 && c->pair_prec) {
        gm_pair_block_kernel<<<(int)((c->g.nb + 127) / 128), 128, 0, s>>>(a, c->dKpair64.as<double>(),
                                                                           c->dKpair32.as<float>());
        GM_LAUNCHED(c);
    }
    return GM_OK;
}

__global__ void gm_count_changes_kernel(const int8_t* a, const int8_t* b, long long n, int* out)
{
    int local = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        local += (a[i] != b[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(out, local);
}

int gm_launch_count_changes(gm_ctx* c, const int8_t* a, const int8_t* b, int* out, cudaStream_t s)
{
    GM_CUDA_TRY(c, cudaMemsetAsync(out, 0, sizeof(int), s));
    if (c->P == 0) return GM_OK;
    gm_count_changes_kernel<<<64, 256, 0, s>>>(a, b, c->P, out);
    GM_LAUNCHED(c);
    return GM_OK;
}
