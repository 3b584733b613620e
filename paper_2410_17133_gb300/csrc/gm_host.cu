// Context, set-up, reference-cell operators, Newton driver and the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "gm_internal.cuh"

#define GM_VERSION "gm-gb300 0.1"

// ---------------------------------------------------------------------------
// Reference cell (host, FP64).  Trilinear shape functions on [-1,1]^3, exact
// 2x2x2 Gauss quadrature (the cell is affine, so the integrands are
// polynomials of degree <= 2 per reference coordinate).
// Local node a = ax + 2 ay + 4 az; element dof index 3a + c.
// ---------------------------------------------------------------------------
namespace {

void q1(const double xi[3], double N[8], double dN[8][3])
{
    for (int a = 0; a < 8; ++a) {
        const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
        const double f[3] = {0.5 * (1 + s[0] * xi[0]), 0.5 * (1 + s[1] * xi[1]), 0.5 * (1 + s[2] * xi[2])};
        N[a] = f[0] * f[1] * f[2];
        dN[a][0] = 0.5 * s[0] * f[1] * f[2];
        dN[a][1] = 0.5 * s[1] * f[0] * f[2];
        dN[a][2] = 0.5 * s[2] * f[0] * f[1];
    }
}

bool inv3(const double A[3][3], double I[3][3], double* det)
{
    const double d = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(std::fabs(d) > 0)) return false;
    I[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
    I[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
    I[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
    I[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
    I[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
    I[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
    I[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
    I[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
    I[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
    *det = d;
    return true;
}

// Element operators of the reference cell for E = 1, alpha = 1, 1/M = 1, k/mu = 1.
bool ref_cell(const double h[3], const double sh[2], double nu, double K[24][24], double A[24][8],
              double M[8][8], double L[8][8])
{
    double X[8][3];
    for (int a = 0; a < 8; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        X[a][0] = ax * h[0];
        X[a][1] = ay * h[1];
        X[a][2] = az * h[2] + sh[0] * ax * h[0] + sh[1] * ay * h[1];
    }
    const double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 1.0 / (2 * (1 + nu));
    double D[6][6] = {};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) D[i][j] = lam;
        D[i][i] += 2 * mu;
        D[i + 3][i + 3] = mu;
    }
    std::memset(K, 0, sizeof(double) * 24 * 24);
    std::memset(A, 0, sizeof(double) * 24 * 8);
    std::memset(M, 0, sizeof(double) * 64);
    std::memset(L, 0, sizeof(double) * 64);
    const double g = 1.0 / std::sqrt(3.0);
    for (int q = 0; q < 8; ++q) {
        const double xi[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
        double N[8], dN[8][3];
        q1(xi, N, dN);
        double J[3][3] = {};
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 8; ++a) J[d][k] += X[a][d] * dN[a][k];
        double Ji[3][3], det;
        if (!inv3(J, Ji, &det) || det <= 0) return false;
        double G[8][3];   // dN_a/dX_d = sum_k dN_a/dxi_k (J^-1)_{k d}
        for (int a = 0; a < 8; ++a)
            for (int d = 0; d < 3; ++d) {
                G[a][d] = 0;
                for (int k = 0; k < 3; ++k) G[a][d] += dN[a][k] * Ji[k][d];
            }
        double B[6][24] = {};
        for (int a = 0; a < 8; ++a) {
            const int c = 3 * a;
            B[0][c] = G[a][0];
            B[1][c + 1] = G[a][1];
            B[2][c + 2] = G[a][2];
            B[3][c + 1] = G[a][2]; B[3][c + 2] = G[a][1];
            B[4][c] = G[a][2];     B[4][c + 2] = G[a][0];
            B[5][c] = G[a][1];     B[5][c + 1] = G[a][0];
        }
        double DB[6][24];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 24; ++j) {
                DB[i][j] = 0;
                for (int k = 0; k < 6; ++k) DB[i][j] += D[i][k] * B[k][j];
            }
        for (int i = 0; i < 24; ++i)
            for (int j = 0; j < 24; ++j) {
                double s = 0;
                for (int k = 0; k < 6; ++k) s += B[k][i] * DB[k][j];
                K[i][j] += det * s;
            }
        for (int i = 0; i < 24; ++i) {
            const double divi = B[0][i] + B[1][i] + B[2][i];
            for (int b = 0; b < 8; ++b) A[i][b] += det * divi * N[b];
        }
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
                M[a][b] += det * N[a] * N[b];
                L[a][b] += det * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
            }
    }
    return true;
}

inline double hsgn(int s, int a) { return (gm_popc3(s & a) & 1) ? -1.0 : 1.0; }

// Parity transform and packing of the entries the class's pattern allows;
// returns false if an entry outside the pattern is not negligible (the cell
// does not belong to the class, or the pattern rule does not hold).
template <int CLS>
bool pack_ref(const double K[24][24], const double A[24][8], const double M[8][8],
              const double L[8][8], RefOps<double>& R)
{
    constexpr ParPat PP = gm_make_parpat(CLS);
    static double Kt[24][24], At[24][8], Mt[8][8], Lt[8][8];   // index (c*8+s)
    for (int c = 0; c < 3; ++c)
        for (int s = 0; s < 8; ++s) {
            for (int c2 = 0; c2 < 3; ++c2)
                for (int s2 = 0; s2 < 8; ++s2) {
                    double v = 0;
                    for (int a = 0; a < 8; ++a)
                        for (int a2 = 0; a2 < 8; ++a2) v += hsgn(s, a) * K[3 * a + c][3 * a2 + c2] * hsgn(s2, a2);
                    Kt[c * 8 + s][c2 * 8 + s2] = v / 64.0;
                }
            for (int s2 = 0; s2 < 8; ++s2) {
                double v = 0;
                for (int a = 0; a < 8; ++a)
                    for (int a2 = 0; a2 < 8; ++a2) v += hsgn(s, a) * A[3 * a + c][a2] * hsgn(s2, a2);
                At[c * 8 + s][s2] = v / 64.0;
            }
        }
    for (int s = 0; s < 8; ++s)
        for (int s2 = 0; s2 < 8; ++s2) {
            double vm = 0, vl = 0;
            for (int a = 0; a < 8; ++a)
                for (int a2 = 0; a2 < 8; ++a2) {
                    vm += hsgn(s, a) * M[a][a2] * hsgn(s2, a2);
                    vl += hsgn(s, a) * L[a][a2] * hsgn(s2, a2);
                }
            Mt[s][s2] = vm / 64.0;
            Lt[s][s2] = vl / 64.0;
        }
    double kmax = 0, amax = 0, mmax = 0, lmax = 0;
    for (int i = 0; i < 24; ++i) {
        for (int j = 0; j < 24; ++j) kmax = std::max(kmax, std::fabs(Kt[i][j]));
        for (int j = 0; j < 8; ++j) amax = std::max(amax, std::fabs(At[i][j]));
    }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            mmax = std::max(mmax, std::fabs(Mt[i][j]));
            lmax = std::max(lmax, std::fabs(Lt[i][j]));
        }
    const double tol = 1e-12;
    std::memset(&R, 0, sizeof(R));
    for (int i = 0; i < 24; ++i) {
        for (int j = 0; j < 24; ++j) {
            if (PP.k[i][j] >= 0) R.K[PP.k[i][j]] = Kt[i][j];
            else if (std::fabs(Kt[i][j]) > tol * kmax) return false;
        }
        for (int j = 0; j < 8; ++j) {
            if (PP.a[i][j] >= 0) R.A[PP.a[i][j]] = At[i][j];
            else if (std::fabs(At[i][j]) > tol * amax) return false;
        }
    }
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            if (i == j) R.M[i] = Mt[i][i];
            else if (std::fabs(Mt[i][j]) > tol * mmax) return false;
            if (PP.l[i][j] >= 0) R.L[PP.l[i][j]] = Lt[i][j];
            else if (std::fabs(Lt[i][j]) > tol * lmax) return false;
        }
    return true;
}

template <typename D, typename S>
void cast_ref(const RefOps<S>& a, RefOps<D>& b)
{
    for (int i = 0; i < GM_PP_MAXK; ++i) b.K[i] = (D)a.K[i];
    for (int i = 0; i < GM_PP_MAXA; ++i) b.A[i] = (D)a.A[i];
    for (int i = 0; i < 8; ++i) b.M[i] = (D)a.M[i];
    for (int i = 0; i < GM_PP_MAXL; ++i) b.L[i] = (D)a.L[i];
}

int bind_impl(gm_ctx* c);

}  // namespace

// per-element k/mu arrays (FP64, FP32) and the diagonals that depend on them
int gm_upload_permeability(gm_ctx* c)
{
    const long long nel = c->n_el;
    std::vector<double> kap(nel);
    std::vector<float> f32(nel);
    for (long long e = 0; e < nel; ++e) {
        kap[e] = c->kperm[e] / c->mu_f;
        f32[e] = (float)kap[e];
    }
    GM_CUDA_TRY(c, cudaMemcpy(c->dK64.p, kap.data(), nel * 8, cudaMemcpyHostToDevice));
    GM_CUDA_TRY(c, cudaMemcpy(c->dK32.p, f32.data(), nel * 4, cudaMemcpyHostToDevice));
    int rc = gm_launch_diag(c, 0);
    if (rc) return rc;
    GM_CUDA_TRY(c, cudaDeviceSynchronize());
    return GM_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* gm_version(void) { return GM_VERSION; }

int gm_create(gm_ctx** out, int device)
{
    if (!out) return GM_EINVAL;
    *out = nullptr;
    gm_ctx* c = new (std::nothrow) gm_ctx();
    if (!c) return GM_ENOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete c; return GM_ECUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
        c->sm_count = sms;
    if (cudaMallocHost(&c->hpin, 4096) != cudaSuccess) { delete c; return GM_ECUDA; }
    *out = c;
    return GM_OK;
}

int gm_destroy(gm_ctx* c)
{
    if (!c) return GM_OK;
    cudaSetDevice(c->device);
    c->drop_graphs();
    gm_mg_release(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->hpin) cudaFreeHost(c->hpin);
    delete c;
    return GM_OK;
}

const char* gm_last_error(const gm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int gm_mesh_structured(gm_ctx* c, int nx, int ny, int nz, const double* origin, const double* h,
                       const double* shear)
{
    if (!c) return GM_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || !h) return c->set_err(GM_EINVAL, "mesh: bad sizes");
    if ((long long)(nx + 1) * (ny + 1) * (nz + 2) > (1LL << 31) / 4)
        return c->set_err(GM_EINVAL, "mesh: too many nodes for 32-bit element counts");
    for (int d = 0; d < 3; ++d)
        if (!(h[d] > 0)) return c->set_err(GM_EINVAL, "mesh: spacing must be positive");
    c->nx = nx; c->ny = ny; c->nz = nz;
    for (int d = 0; d < 3; ++d) { c->origin[d] = origin ? origin[d] : 0.0; c->h[d] = h[d]; }
    c->shear[0] = shear ? shear[0] : 0.0;
    c->shear[1] = shear ? shear[1] : 0.0;
    c->has_mesh = true;
    c->has_fault = false;
    c->kf_orig = -1;
    c->has_mat = false;
    c->bound = false;
    c->fixed.clear(); c->fu.clear(); c->fpv.clear();
    return GM_OK;
}

// Floor of the Newton test from the in-situ fault forces: sum of F0^2 / diag(K_b)
// over free lip dofs, F0 = A_i (-t'_n0 n + tau0) with per-pair values if set.
static int gm_insitu_floor(gm_ctx* c)
{
    c->f0sq = 0.0;
    if (!c->has_fault) return GM_OK;
    const long long N = c->N, N3 = 3 * N;
    std::vector<double> dK(N3);
    GM_CUDA_TRY(c, cudaMemcpy(dK.data(), c->ddiagK.p, N3 * 8, cudaMemcpyDeviceToHost));
    const long long nb = c->g.nb;
    for (long long q = 0; q < nb; ++q) {
        const int pi = (int)(q % (c->nx + 1)), pj = (int)(q / (c->nx + 1));
        const int nqi = (pi > 0) + (pi < c->nx), nqj = (pj > 0) + (pj < c->ny);
        const double Ai = c->Aq * 0.25 * nqi * nqj;
        const double tn0 = c->has_insitu ? c->h_insitu[q] : c->fp.tn0;
        const double t01 = c->has_insitu ? c->h_insitu[nb + q] : c->fp.tau0[0];
        const double t02 = c->has_insitu ? c->h_insitu[2 * nb + q] : c->fp.tau0[1];
        for (int lip = 0; lip < 2; ++lip) {
            const long long n = q + nb * (c->g.kf + lip);
            for (int d = 0; d < 3; ++d) {
                if (c->fixed[d * N + n]) continue;
                const double F0 = Ai * (-tn0 * c->nrm[d] + t01 * c->t1[d] + t02 * c->t2[d]);
                c->f0sq += F0 * F0 / dK[d * N + n];
            }
        }
    }
    return GM_OK;
}

int gm_set_preconditioner(gm_ctx* c, int kind)
{
    if (!c) return GM_EINVAL;
    if (kind != 0 && kind != 1) return c->set_err(GM_EINVAL, "set_preconditioner: kind must be 0 or 1");
    if (kind != c->precond) c->drop_graphs();
    c->precond = kind;
    return GM_OK;
}

int gm_set_insitu(gm_ctx* c, const double* tn0, const double* tau0, int64_t n)
{
    if (!c) return GM_EINVAL;
    if (!c->bound || !c->has_fault) return c->set_err(GM_ESTATE, "set_insitu: needs a bound fault");
    if (!tn0 && !tau0) {
        c->has_insitu = false;
        c->h_insitu.clear();
        return gm_insitu_floor(c);
    }
    if (!tn0 || !tau0) return c->set_err(GM_EINVAL, "set_insitu: give both arrays, or neither");
    if (n != c->P) return c->set_err(GM_EINVAL, "set_insitu: n must be the pair count");
    std::vector<double> h((size_t)3 * n);
    for (long long i = 0; i < n; ++i) {
        if (!std::isfinite(tn0[i]) || !std::isfinite(tau0[i]) || !std::isfinite(tau0[n + i]))
            return c->set_err(GM_EINVAL, "set_insitu: values must be finite");
        h[i] = tn0[i];
        h[n + i] = tau0[i];
        h[2 * n + i] = tau0[n + i];
    }
    GM_CUDA_TRY(c, cudaMemcpy(c->dinsitu.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    c->h_insitu.swap(h);
    c->has_insitu = true;
    return gm_insitu_floor(c);
}

int gm_fault_plane(gm_ctx* c, int kf, const gm_fault_params* p)
{
    if (!c) return GM_EINVAL;
    if (!c->has_mesh) return c->set_err(GM_ESTATE, "fault: call gm_mesh_structured first");
    if (kf <= 0 || kf >= c->nz || !p) return c->set_err(GM_EINVAL, "fault: need 0 < kf < nz");
    if (!(p->kn > 0) || !(p->ks > 0) || !(p->f >= 0) || !(p->w0 > 0) || !(p->MF > 0) || !(p->wk_par >= 0))
        return c->set_err(GM_EINVAL, "fault: invalid parameters");
    c->kf_orig = kf;
    c->fp = *p;
    c->has_fault = true;
    c->bound = false;
    c->fixed.clear(); c->fu.clear(); c->fpv.clear();
    return GM_OK;
}

static long long n_nodes_of(const gm_ctx* c)
{
    return (long long)(c->nx + 1) * (c->ny + 1) * (c->nz + 1 + (c->has_fault ? 1 : 0));
}

int gm_set_materials(gm_ctx* c, const double* E, const double* k, int64_t n, double nu, double alpha,
                     double M, double mu_f)
{
    if (!c) return GM_EINVAL;
    if (!c->has_mesh) return c->set_err(GM_ESTATE, "materials: no mesh");
    const long long nel = (long long)c->nx * c->ny * c->nz;
    if (!E || !k || (n != 1 && n != nel)) return c->set_err(GM_EINVAL, "materials: n must be 1 or n_el");
    if (!(nu > -1.0 && nu < 0.5) || !(M > 0) || !(mu_f > 0))
        return c->set_err(GM_EINVAL, "materials: invalid nu, M or mu_f");
    c->E.assign(nel, 0.0);
    c->kperm.assign(nel, 0.0);
    for (long long e = 0; e < nel; ++e) {
        c->E[e] = E[n == 1 ? 0 : e];
        c->kperm[e] = k[n == 1 ? 0 : e];
        if (!(c->E[e] > 0) || !(c->kperm[e] >= 0)) return c->set_err(GM_EINVAL, "materials: E > 0, k >= 0");
    }
    c->nu = nu; c->alpha = alpha; c->M = M; c->mu_f = mu_f;
    c->has_mat = true;
    c->bound = false;
    return GM_OK;
}

int gm_set_dirichlet(gm_ctx* c, const uint8_t* fixed, int64_t n)
{
    if (!c) return GM_EINVAL;
    if (!c->has_mesh) return c->set_err(GM_ESTATE, "dirichlet: no mesh");
    const long long N = n_nodes_of(c);
    if (!fixed || n != 4 * N) return c->set_err(GM_EINVAL, "dirichlet: need 4*N bytes");
    c->fixed.assign(fixed, fixed + n);
    c->bound = false;
    return GM_OK;
}

static int upload_loads(gm_ctx* c)
{
    const long long N = c->N;
    {
        std::vector<double> fpm = c->fpv;
        if (c->has_fault && !(c->fp.k_perp > 0)) {
            for (long long q = 0; q < c->g.nb; ++q) {
                const long long m = q + c->g.nb * c->g.kf;
                fpm[m] += fpm[m + c->g.nb];
                fpm[m + c->g.nb] = 0.0;
            }
        }
        GM_CUDA_TRY(c, cudaMemcpy(c->dfu.p, c->fu.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice));
        GM_CUDA_TRY(c, cudaMemcpy(c->dfp.p, fpm.data(), N * sizeof(double), cudaMemcpyHostToDevice));
    }
    return GM_OK;
}

int gm_set_loads(gm_ctx* c, const double* fu, const double* fp)
{
    if (!c) return GM_EINVAL;
    if (!c->has_mesh) return c->set_err(GM_ESTATE, "loads: no mesh");
    const long long N = n_nodes_of(c);
    std::vector<double> a(3 * N, 0.0), b(N, 0.0);
    if (fu) std::copy(fu, fu + 3 * N, a.begin());
    if (fp) std::copy(fp, fp + N, b.begin());
    c->fu.swap(a);
    c->fpv.swap(b);
    // loads can change between steps without rebinding
    if (c->bound) return upload_loads(c);
    return GM_OK;
}

int gm_assemble_or_bind(gm_ctx* c)
{
    if (!c) return GM_EINVAL;
    GM_CUDA_TRY(c, cudaSetDevice(c->device));
    return bind_impl(c);
}

int gm_set_timestep(gm_ctx* c, double dt)
{
    if (!c) return GM_EINVAL;
    if (!(dt > 0)) return c->set_err(GM_EINVAL, "dt must be positive");
    c->dt = dt;
    if (c->bound) {
        int rc = gm_launch_diag(c, 0);
        if (rc) return rc;
        GM_CUDA_TRY(c, cudaDeviceSynchronize());
    }
    return GM_OK;
}

int gm_sizes(const gm_ctx* c, int64_t* nn, int64_t* ne, int64_t* np)
{
    if (!c || !c->has_mesh) return GM_EINVAL;
    const long long N = n_nodes_of(c);
    if (nn) *nn = N;
    if (ne) *ne = (long long)c->nx * c->ny * c->nz;
    if (np) *np = c->has_fault ? (long long)(c->nx + 1) * (c->ny + 1) : 0;
    return GM_OK;
}

int gm_counters(const gm_ctx* c, int64_t* launches, int64_t* applies)
{
    if (!c) return GM_EINVAL;
    if (launches) *launches = c->launches;
    if (applies) *applies = c->applies;
    return GM_OK;
}

int gm_apply_operator(gm_ctx* c, int which, const void* x, void* y, int dtype, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "apply: call gm_assemble_or_bind first");
    if (!x || !y) return c->set_err(GM_EINVAL, "apply: null vector");
    if (dtype != GM_F64 && dtype != GM_F32) return c->set_err(GM_EINVAL, "apply: bad dtype");
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = c->N;
    const size_t es = dtype == GM_F64 ? 8 : 4;
    const char* xb = (const char*)x;
    char* yb = (char*)y;
    int mode;
    double cK = 0, cApu = 0, cAup = 0, cS = 0, cC = 0;
    const void *xu = nullptr, *xp = nullptr;
    void *yu = nullptr, *yp = nullptr;
    switch (which) {
    case GM_OP_KB: mode = GM_MODE_K; cK = 1; xu = x; yu = y; break;
    case GM_OP_KT: mode = GM_MODE_KT; cK = 1; xu = x; yu = y; break;
    case GM_OP_A22: mode = GM_MODE_A22; cS = 1; cC = c->dt; xp = x; yp = y; break;
    case GM_OP_APU: mode = GM_MODE_APU; cApu = 1; xp = x; yu = y; break;
    case GM_OP_AUP: mode = GM_MODE_AUP; cAup = 1; xu = x; yp = y; break;
    case GM_OP_J:
        mode = GM_MODE_J; cK = 1; cApu = -1; cAup = 1; cS = 1; cC = c->dt;
        xu = x; xp = xb + 3 * N * es; yu = y; yp = yb + 3 * N * es;
        break;
    default: return c->set_err(GM_EINVAL, "apply: unknown operator");
    }
    if (dtype == GM_F64)
        return gm_launch_apply_f64(c, mode, cK, cApu, cAup, cS, cC, (const double*)xu, (const double*)xp,
                                   (double*)yu, (double*)yp, s, nullptr);
    return gm_launch_apply_f32(c, mode, cK, cApu, cAup, cS, cC, (const float*)xu, (const float*)xp,
                               (float*)yu, (float*)yp, s, nullptr);
}

int gm_fault_update(gm_ctx* c, const double* u, int8_t* flags, double* tn, double* ts, double* dlie,
                    double* T, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "fault_update: not bound");
    if (!c->has_fault) return c->set_err(GM_ESTATE, "fault_update: no fault");
    if (!u) return c->set_err(GM_EINVAL, "fault_update: null u");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = gm_launch_return_map(c, u, nullptr, s);
    if (rc) return rc;
    if ((rc = gm_launch_block_jacobi(c, s))) return rc;
    const long long P = c->P;
    if (flags) GM_CUDA_TRY(c, cudaMemcpyAsync(flags, c->dstate.p, P, cudaMemcpyDeviceToDevice, s));
    if (tn) GM_CUDA_TRY(c, cudaMemcpyAsync(tn, c->dtn.p, P * 8, cudaMemcpyDeviceToDevice, s));
    if (ts) GM_CUDA_TRY(c, cudaMemcpyAsync(ts, c->dts.p, 2 * P * 8, cudaMemcpyDeviceToDevice, s));
    if (dlie) GM_CUDA_TRY(c, cudaMemcpyAsync(dlie, c->ddlie.p, 2 * P * 8, cudaMemcpyDeviceToDevice, s));
    if (T) GM_CUDA_TRY(c, cudaMemcpyAsync(T, c->dT.p, 3 * P * 8, cudaMemcpyDeviceToDevice, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    return GM_OK;
}

int gm_pcg_solve(gm_ctx* c, int which, const double* b, double* x, double rtol, int maxit,
                 gm_solve_report* rep, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "pcg: not bound");
    if (which != GM_OP_KT && which != GM_OP_A22) return c->set_err(GM_EINVAL, "pcg: which must be KT or A22");
    if (!b || !x || !(rtol > 0) || maxit < 1) return c->set_err(GM_EINVAL, "pcg: bad arguments");
    int it = 0;
    double rr = 0;
    int rc = gm_pcg(c, which == GM_OP_KT ? 0 : 1, GM_F64, b, x, rtol, maxit, &it, &rr, (cudaStream_t)stream);
    if (rep) { rep->iterations = it; rep->rel_residual = rr; rep->status = rc; }
    return rc;
}

int gm_prevost_solve(gm_ctx* c, const double* b, double* x, double outer_rtol, int outer_maxit,
                     double inner_rtol, int inner_maxit, gm_solve_report* rep, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "prevost: not bound");
    if (!b || !x) return c->set_err(GM_EINVAL, "prevost: null vector");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = gm_launch_block_jacobi(c, s);
    if (rc) return rc;
    const long long N = c->N;
    int it = 0;
    double rr = 0;
    long long ik = 0, ia = 0;
    rc = gm_prevost(c, GM_F64, b, b + 3 * N, x, x + 3 * N, outer_rtol, outer_maxit, inner_rtol,
                    inner_maxit, &it, &ik, &ia, &rr, s);
    if (rep) { rep->iterations = it; rep->rel_residual = rr; rep->status = rc; }
    if (rc == GM_OK) {
        GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Newton
// ---------------------------------------------------------------------------
static int residual_impl(gm_ctx* c, const double* du, const double* dp, double* b, double* rhat2,
                         double* shat2, cudaStream_t s)
{
    const long long N = c->N, N3 = 3 * N;
    double* ut = c->w_ut.as<double>();
    double* pt = c->w_pt.as<double>();
    int rc;
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
    double* out2 = reinterpret_cast<double*>(c->dscal.as<PcgScalars>() + 5);
    if ((rc = gm_launch_residual(c, y1u, y1p, y2p, ut, pt, b, s, out2))) return rc;
    double* h = reinterpret_cast<double*>(static_cast<char*>(c->hpin) + 1024);
    GM_CUDA_TRY(c, cudaMemcpyAsync(h, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    *rhat2 = h[0];
    *shat2 = h[1];
    return GM_OK;
}

extern "C" int gm_residual(gm_ctx* c, const double* du, const double* dp, double* b, double* rhat,
                           void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "residual: not bound");
    if (!du || !dp || !b) return c->set_err(GM_EINVAL, "residual: null vector");
    double r2, s2;
    int rc = residual_impl(c, du, dp, b, &r2, &s2, (cudaStream_t)stream);
    if (rc) return rc;
    if (rhat) *rhat = std::sqrt(r2);
    return GM_OK;
}

extern "C" int gm_partitioned_step(gm_ctx* c, double dt, const gm_step_opts* opts,
                                   gm_step_report* rep, void* stream)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "step: not bound");
    if (!(dt > 0)) return c->set_err(GM_EINVAL, "step: dt must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    gm_step_opts o;
    o.newton_rtol = 1e-10; o.newton_maxit = 50;
    o.outer_rtol = 1e-8; o.outer_maxit = 500;
    o.inner_rtol = 1e-10; o.inner_maxit = 20000;
    o.precision = GM_F64;
    o.schur_precond = 0;
    if (opts) o = *opts;
    // FP32-refined defaults: inexact inner solves, the FP64 Newton loop refines
    // (the Newton iteration count is set by the fault nonlinearity, not by these)
    if (o.precision == GM_F32 && !opts) { o.inner_rtol = 1e-2; o.outer_rtol = 1e-1; }
    int rc;
    if (dt != c->dt) {
        c->dt = dt;
        if ((rc = gm_launch_diag(c, s))) return rc;
    }
    const long long N = c->N, N3 = 3 * N;
    double* du = c->w_du.as<double>();
    double* dp = c->w_dp.as<double>();
    double* b = c->w_b.as<double>();
    double* x = c->w_x.as<double>();
    GM_CUDA_TRY(c, cudaMemsetAsync(du, 0, N3 * 8, s));
    GM_CUDA_TRY(c, cudaMemsetAsync(dp, 0, N * 8, s));
    int* dchg = reinterpret_cast<int*>(c->dscal.as<PcgScalars>() + 6);
    int* hchg = reinterpret_cast<int*>(static_cast<char*>(c->hpin) + 2048);
    gm_step_report R{};
    const long long app0 = c->applies;
    double rhat0 = 0, rhat = 0;
    bool converged = false;
    int it;
    for (it = 0; it <= o.newton_maxit; ++it) {
        double r2, s2;
        if ((rc = residual_impl(c, du, dp, b, &r2, &s2, s))) return rc;
        rhat = std::sqrt(r2);
        if (!std::isfinite(rhat)) return c->set_err(GM_ENAN, "step: non-finite residual");
        if (it == 0) rhat0 = rhat;
        bool same = true;
        if (c->has_fault) {
            if (it == 0) {
                same = false;
            } else {
                if ((rc = gm_launch_count_changes(c, c->dstate.as<int8_t>(), c->dprevstate.as<int8_t>(), dchg, s))) return rc;
                GM_CUDA_TRY(c, cudaMemcpyAsync(hchg, dchg, sizeof(int), cudaMemcpyDeviceToHost, s));
                GM_CUDA_TRY(c, cudaStreamSynchronize(s));
                same = (*hchg == 0);
            }
        }
        const double shat = std::sqrt(s2 + c->f0sq);
        if (it > 0 && same && rhat <= o.newton_rtol * std::max(rhat0, 1e-3 * shat)) {
            converged = true;
            break;
        }
        if (it == o.newton_maxit) break;
        if (c->has_fault)
            GM_CUDA_TRY(c, cudaMemcpyAsync(c->dprevstate.p, c->dstate.p, c->P, cudaMemcpyDeviceToDevice, s));
        if ((rc = gm_launch_block_jacobi(c, s))) return rc;
        int oit = 0;
        double orr = 0;
        rc = gm_prevost(c, o.precision, b, b + N3, x, x + N3, o.outer_rtol, o.outer_maxit, o.inner_rtol,
                        o.inner_maxit, &oit, &R.inner_k, &R.inner_a, &orr, s, o.schur_precond);
        if (rc == GM_ENAN) return rc;
        R.outer += oit;
        if ((rc = gm_launch_axpby(c, N3, 1.0, x, 1.0, du, s))) return rc;
        if ((rc = gm_launch_axpby(c, N, 1.0, x + N3, 1.0, dp, s))) return rc;
    }
    R.newton = it;
    R.rhat = rhat;
    R.rhat0 = rhat0;
    R.applies = c->applies - app0;
    if (!converged) {
        if (rep) *rep = R;
        return c->set_err(GM_ENEWTON, "step: Newton did not converge (rhat/rhat0=" +
                                          std::to_string(rhat / std::max(rhat0, 1e-300)) + ")");
    }
    // accept
    if ((rc = gm_launch_axpby(c, N3, 1.0, du, 1.0, c->du_n.as<double>(), s))) return rc;
    if ((rc = gm_launch_axpby(c, N, 1.0, dp, 1.0, c->dp_n.as<double>(), s))) return rc;
    const long long P = c->P;
    if (c->has_fault) {
        GM_CUDA_TRY(c, cudaMemcpyAsync(c->ddlie_n.p, c->ddlie.p, 2 * P * 8, cudaMemcpyDeviceToDevice, s));
        GM_CUDA_TRY(c, cudaMemcpyAsync(c->dflags_n.p, c->dstate.p, P, cudaMemcpyDeviceToDevice, s));
        std::vector<int8_t> st(P);
        std::vector<double> F(P), tn(P), dn(P);
        GM_CUDA_TRY(c, cudaMemcpyAsync(st.data(), c->dstate.p, P, cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(c, cudaMemcpyAsync(F.data(), c->dF.p, P * 8, cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(c, cudaMemcpyAsync(tn.data(), c->dtn.p, P * 8, cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(c, cudaMemcpyAsync(dn.data(), c->ddn.p, P * 8, cudaMemcpyDeviceToHost, s));
        GM_CUDA_TRY(c, cudaStreamSynchronize(s));
        double ym = INFINITY, nm = INFINITY;
        for (long long i = 0; i < P; ++i) {
            if (st[i] == GM_OPEN) R.n_open++;
            else if (st[i] == GM_STICK) R.n_stick++;
            else R.n_slip++;
            if (tn[i] > 0) ym = std::min(ym, std::fabs(F[i]) / (c->fp.f * tn[i]));
            const double tn0 = c->has_insitu ? c->h_insitu[i] : c->fp.tn0;
            nm = std::min(nm, std::fabs(tn0 - c->fp.kn * dn[i]) / tn0);
        }
        R.min_yield_margin = ym;
        R.min_normal_margin = nm;
    } else {
        GM_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    if (rep) *rep = R;
    return GM_OK;
}

// ---------------------------------------------------------------------------
// State I/O
// ---------------------------------------------------------------------------
extern "C" int gm_get_state(gm_ctx* c, double* u, double* p, double* slip, double* dlie, int8_t* flags)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "get_state: not bound");
    GM_CUDA_TRY(c, cudaSetDevice(c->device));
    GM_CUDA_TRY(c, cudaDeviceSynchronize());
    const long long N = c->N, P = c->P, nb = c->g.nb;
    // u straight into the caller's array; the slip needs only the two lip planes
    std::vector<double> lips;
    const double* ul = nullptr;     // lip planes: (component, lip, pair)
    if (u) GM_CUDA_TRY(c, cudaMemcpy(u, c->du_n.p, 3 * N * 8, cudaMemcpyDeviceToHost));
    if (slip && c->has_fault) {
        lips.resize(6 * nb);
        for (int d = 0; d < 3; ++d)
            for (int s = 0; s < 2; ++s) {
                const long long off = d * N + nb * (c->g.kf + s);
                if (u) std::copy(u + off, u + off + nb, lips.begin() + (2 * d + s) * nb);
                else GM_CUDA_TRY(c, cudaMemcpy(lips.data() + (2 * d + s) * nb, c->du_n.as<double>() + off, nb * 8,
                                               cudaMemcpyDeviceToHost));
            }
        ul = lips.data();
    }
    if (p) {
        GM_CUDA_TRY(c, cudaMemcpy(p, c->dp_n.p, N * 8, cudaMemcpyDeviceToHost));
        if (c->has_fault && c->g.tied)
            for (long long q = 0; q < nb; ++q) p[q + nb * (c->g.kf + 1)] = p[q + nb * c->g.kf];
    }
    if (slip && c->has_fault) {
        for (long long q = 0; q < P; ++q) {
            double j[3];
            for (int d = 0; d < 3; ++d) j[d] = ul[(2 * d + 1) * nb + q] - ul[(2 * d) * nb + q];
            slip[q] = c->t1[0] * j[0] + c->t1[1] * j[1] + c->t1[2] * j[2];
            slip[P + q] = c->t2[0] * j[0] + c->t2[1] * j[1] + c->t2[2] * j[2];
        }
    }
    if (dlie && c->has_fault) GM_CUDA_TRY(c, cudaMemcpy(dlie, c->ddlie_n.p, 2 * P * 8, cudaMemcpyDeviceToHost));
    if (flags && c->has_fault) GM_CUDA_TRY(c, cudaMemcpy(flags, c->dflags_n.p, P, cudaMemcpyDeviceToHost));
    return GM_OK;
}

extern "C" int gm_set_state(gm_ctx* c, const double* u, const double* p, const double* dlie,
                            const int8_t* flags)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "set_state: not bound");
    GM_CUDA_TRY(c, cudaSetDevice(c->device));
    const long long N = c->N, P = c->P;
    if (u) GM_CUDA_TRY(c, cudaMemcpy(c->du_n.p, u, 3 * N * 8, cudaMemcpyHostToDevice));
    if (p) {
        GM_CUDA_TRY(c, cudaMemcpy(c->dp_n.p, p, N * 8, cudaMemcpyHostToDevice));
        // a tied upper lip carries no unknown: its slot is 0 on the device
        if (c->has_fault && c->g.tied)
            GM_CUDA_TRY(c, cudaMemset(c->dp_n.as<double>() + c->g.nb * (c->g.kf + 1), 0, c->g.nb * 8));
    }
    if (dlie && c->has_fault) GM_CUDA_TRY(c, cudaMemcpy(c->ddlie_n.p, dlie, 2 * P * 8, cudaMemcpyHostToDevice));
    if (flags && c->has_fault) GM_CUDA_TRY(c, cudaMemcpy(c->dflags_n.p, flags, P, cudaMemcpyHostToDevice));
    GM_CUDA_TRY(c, cudaDeviceSynchronize());
    return GM_OK;
}

extern "C" int gm_state_device(gm_ctx* c, double** u, double** p)
{
    if (!c) return GM_EINVAL;
    if (!c->bound) return c->set_err(GM_ESTATE, "state_device: not bound");
    if (u) *u = c->du_n.as<double>();
    if (p) *p = c->dp_n.as<double>();
    return GM_OK;
}

// ---------------------------------------------------------------------------
// Bind: derived data, reference operators, device allocation and upload
// ---------------------------------------------------------------------------
namespace {

int bind_impl(gm_ctx* c)
{
    (void)cudaGetLastError();   // start from a clean runtime error state
    c->drop_graphs();           // graphs hold pointers into the buffers freed below
    gm_mg_release(c);           // coarse levels are rebuilt from the new set-up on first use
    if (!c->has_mesh || !c->has_mat) return c->set_err(GM_ESTATE, "bind: mesh and materials required");
    const long long N = n_nodes_of(c);
    const long long nel = (long long)c->nx * c->ny * c->nz;
    c->N = N;
    c->n_el = nel;
    c->g.nx = c->nx; c->g.ny = c->ny; c->g.nz = c->nz;
    c->g.nplanes = c->nz + 1 + (c->has_fault ? 1 : 0);
    c->g.kf = c->has_fault ? c->kf_orig : -1;
    c->g.tied = (c->has_fault && !(c->fp.k_perp > 0)) ? 1 : 0;
    c->g.N = N;
    c->g.nb = (long long)(c->nx + 1) * (c->ny + 1);
    c->P = c->has_fault ? c->g.nb : 0;
    if (3 * N >= (1LL << 31)) return c->set_err(GM_EINVAL, "bind: more than 715,827,882 nodes (32-bit vector offsets)");
    if (c->fixed.empty()) c->fixed.assign(4 * N, 0);
    if (c->fu.empty()) c->fu.assign(3 * N, 0.0);
    if (c->fpv.empty()) c->fpv.assign(N, 0.0);
    if ((long long)c->fixed.size() != 4 * N || (long long)c->fu.size() != 3 * N)
        return c->set_err(GM_ESTATE, "bind: constraint/load sizes do not match the mesh (set them after the fault)");

    // symmetry class and reference operators
    c->cls = (c->shear[0] == 0.0 && c->shear[1] == 0.0) ? GM_CLS_BOX
           : (c->shear[1] == 0.0 ? GM_CLS_MONO : GM_CLS_GEN);
    static double K[24][24], A[24][8], M[8][8], L[8][8];
    if (!ref_cell(c->h, c->shear, c->nu, K, A, M, L)) return c->set_err(GM_EINVAL, "bind: degenerate cell");
    bool ok = c->cls == GM_CLS_BOX ? pack_ref<GM_CLS_BOX>(K, A, M, L, c->R64)
            : c->cls == GM_CLS_MONO ? pack_ref<GM_CLS_MONO>(K, A, M, L, c->R64)
                                    : pack_ref<GM_CLS_GEN>(K, A, M, L, c->R64);
    if (!ok) return c->set_err(GM_EINVAL, "bind: cell operators break the expected parity pattern");
    cast_ref(c->R64, c->R32);
    for (int i = 0; i < GM_PP_MAXK; ++i) c->R32p.K[i] = make_float2(c->R32.K[i], c->R32.K[i]);
    for (int i = 0; i < 8; ++i) c->R32p.M[i] = make_float2(c->R32.M[i], c->R32.M[i]);
    for (int i = 0; i < GM_PP_MAXL; ++i) c->R32p.L[i] = make_float2(c->R32.L[i], c->R32.L[i]);
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) c->Lref[8 * a + b] = L[a][b];
    c->has_fpair = false;
    c->has_insitu = false;
    c->h_insitu.clear();
    c->fault_cons = 0;
    c->adj_m = 0;
    for (DevBuf* bf : {&c->adj_V, &c->adj_Z, &c->adj_w, &c->adj_b, &c->adj_x, &c->adj_t}) bf->release();
    for (int a = 0; a < 8; ++a) {
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) c->Kblk_ref[a][3 * x + y] = K[3 * a + x][3 * a + y];
        c->Mdiag_ref[a] = M[a][a];
        c->Ldiag_ref[a] = L[a][a];
    }
    // fault quad geometry: edges e1 = dX/di, e2 = dX/dj of the index plane
    {
        const double e1[3] = {c->h[0], 0.0, c->shear[0] * c->h[0]};
        const double e2[3] = {0.0, c->h[1], c->shear[1] * c->h[1]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        const double a = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        c->Aq = a;
        for (int d = 0; d < 3; ++d) c->nrm[d] = cr[d] / a;
        const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int d = 0; d < 3; ++d) c->t1[d] = e1[d] / l1;
        c->t2[0] = c->nrm[1] * c->t1[2] - c->nrm[2] * c->t1[1];
        c->t2[1] = c->nrm[2] * c->t1[0] - c->nrm[0] * c->t1[2];
        c->t2[2] = c->nrm[0] * c->t1[1] - c->nrm[1] * c->t1[0];
        // surface Laplacian of one bilinear quad, 2x2 Gauss; dX/dxi = e1/2, dX/deta = e2/2
        double G[2][2];
        G[0][0] = 0.25 * (e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        G[1][1] = 0.25 * (e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        G[0][1] = G[1][0] = 0.25 * (e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2]);
        const double dG = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        const double Gi[2][2] = {{G[1][1] / dG, -G[0][1] / dG}, {-G[1][0] / dG, G[0][0] / dG}};
        const double jac = std::sqrt(dG);
        const double g = 1.0 / std::sqrt(3.0);
        std::memset(c->Lf, 0, sizeof(c->Lf));
        for (int q = 0; q < 4; ++q) {
            const double xi = (q & 1) ? g : -g, et = (q & 2) ? g : -g;
            double dN[4][2];
            for (int b = 0; b < 4; ++b) {
                const double sx = (b & 1) ? 1.0 : -1.0, sy = (b & 2) ? 1.0 : -1.0;
                dN[b][0] = 0.25 * sx * (1 + sy * et);
                dN[b][1] = 0.25 * sy * (1 + sx * xi);
            }
            for (int b = 0; b < 4; ++b)
                for (int b2 = 0; b2 < 4; ++b2) {
                    double v = 0;
                    for (int k = 0; k < 2; ++k)
                        for (int l = 0; l < 2; ++l) v += dN[b][k] * Gi[k][l] * dN[b2][l];
                    c->Lf[b * 4 + b2] += jac * v;
                }
        }
    }

    // device allocation
    const long long P = c->P;
    const long long N3 = 3 * N;
    // optional tuning override of the bulk kernel's plane-chunk length
    if (const char* zc = std::getenv("GM_BULK_ZCHUNK")) c->zchunk_override = std::max(0, std::atoi(zc));
    // K_T preconditioner: 6x6 lip-pair blocks (default) or 3x3 nodal blocks only (0)
    if (const char* pp = std::getenv("GM_PAIR_PREC")) c->pair_prec = std::atoi(pp) != 0;
    // reduction partials: the fixed-grid reductions use 2 * GM_RED_BLOCKS slots,
    // a fused PCG step one per bulk CTA plus one per fault block
    // (bulk kernels: at most one CTA per 15 x 15 tile and pair of node planes)
    const int gxp = (c->nx + 1 + 14) / 15, gyp = (c->ny + 1 + 14) / 15;
    const long long xyp = (long long)gxp * gyp;
    const long long zcp = c->zchunk_override > 0 ? std::min<long long>(2, c->zchunk_override) : 2LL;
    c->bulk_grid = (int)(xyp * ((c->g.nplanes + zcp - 1) / zcp));
    const size_t part_bytes = (size_t)8 * std::max<long long>(4LL * GM_RED_BLOCKS,
                                                              c->bulk_grid + (c->g.nb + 255) / 256 + 64);
    struct A_ { DevBuf* b; size_t bytes; } allocs[] = {
        {&c->dE64, (size_t)nel * 8}, {&c->dK64, (size_t)nel * 8},
        {&c->dE32, (size_t)nel * 4}, {&c->dK32, (size_t)nel * 4},
        {&c->dmask, (size_t)N + 64}, {&c->dfu, (size_t)N3 * 8}, {&c->dfp, (size_t)N * 8},
        {&c->du_n, (size_t)N3 * 8}, {&c->dp_n, (size_t)N * 8},
        {&c->ddlie_n, (size_t)2 * P * 8}, {&c->dflags_n, (size_t)P},
        {&c->dstate, (size_t)P}, {&c->dprevstate, (size_t)P}, {&c->dtn, (size_t)P * 8},
        {&c->dts, (size_t)2 * P * 8}, {&c->ddlie, (size_t)2 * P * 8}, {&c->dT, (size_t)3 * P * 8},
        {&c->dF, (size_t)P * 8}, {&c->ddn, (size_t)P * 8}, {&c->dgs, (size_t)2 * P * 8},
        {&c->dD64, (size_t)6 * P * 8}, {&c->dD32, (size_t)6 * P * 4},
        {&c->dtauc, (size_t)4 * P * 8}, {&c->dfpair, (size_t)P * 8},
        {&c->dinsitu, (size_t)3 * P * 8},
        {&c->ddiagK, (size_t)N3 * 8}, {&c->ddiagA, (size_t)N * 8},
        {&c->dKinv64, (size_t)12 * N * 8}, {&c->dKinv32, (size_t)6 * N * 4}, {&c->dKinv16, (size_t)6 * N * 2},
        {&c->dKpair64, (size_t)36 * std::max<long long>(P, 1) * 8}, {&c->dKpair32, (size_t)36 * std::max<long long>(P, 1) * 4},
        {&c->dAinv64, (size_t)N * 8}, {&c->dAinv32, (size_t)N * 4},
        {&c->dFS64, (size_t)nel * 8}, {&c->dFS32, (size_t)nel * 4},
        {&c->dAfsinv64, (size_t)N * 8}, {&c->dAfsinv32, (size_t)N * 4},
        {&c->dscal, (size_t)16 * sizeof(PcgScalars)}, {&c->dpart, part_bytes},
        {&c->dcount, (size_t)64},
        {&c->w_du, (size_t)N3 * 8}, {&c->w_dp, (size_t)N * 8}, {&c->w_ut, (size_t)N3 * 8},
        {&c->w_pt, (size_t)N * 8}, {&c->w_b, (size_t)4 * N * 8}, {&c->w_x, (size_t)4 * N * 8},
        {&c->w_y1u, (size_t)N3 * 8}, {&c->w_y1p, (size_t)N * 8}, {&c->w_y2p, (size_t)N * 8},
        {&c->k_r, (size_t)N3 * 8}, {&c->k_z, (size_t)N3 * 8}, {&c->k_p, (size_t)N3 * 8},
        {&c->k_p2, (size_t)N3 * 8}, {&c->k_x64, (size_t)N3 * 8}, {&c->a_x64, (size_t)N * 8},
        {&c->k_q, (size_t)N3 * 8}, {&c->a_r, (size_t)N * 8}, {&c->a_z, (size_t)N * 8},
        {&c->a_p, (size_t)N * 8}, {&c->a_p2, (size_t)N * 8}, {&c->a_q, (size_t)N * 8},
        {&c->k_r32, (size_t)N3 * 4}, {&c->k_z32, (size_t)N3 * 4}, {&c->k_p32, (size_t)N3 * 4},
        {&c->k_pb32, (size_t)N3 * 4},
        {&c->k_q32, (size_t)N3 * 4}, {&c->k_x32, (size_t)N3 * 4}, {&c->k_b32, (size_t)N3 * 4},
        {&c->a_r32, (size_t)N * 4}, {&c->a_z32, (size_t)N * 4}, {&c->a_p32, (size_t)N * 4},
        {&c->a_pb32, (size_t)N * 4},
        {&c->a_q32, (size_t)N * 4}, {&c->a_x32, (size_t)N * 4}, {&c->a_b32, (size_t)N * 4},
        {&c->o_y1, (size_t)N3 * 8}, {&c->o_w, (size_t)N3 * 8}, {&c->o_t3, (size_t)N3 * 8},
        {&c->o_s32a, (size_t)N3 * 4}, {&c->o_s32b, (size_t)N3 * 4},
        {&c->o_r, (size_t)N * 8}, {&c->o_z, (size_t)N * 8}, {&c->o_zold, (size_t)N * 8},
        {&c->o_p, (size_t)N * 8}, {&c->o_q, (size_t)N * 8}, {&c->o_t1, (size_t)N * 8},
    };
    for (auto& al : allocs) {
        cudaError_t e = al.b->alloc(al.bytes);
        if (e != cudaSuccess) return c->set_err(GM_ENOMEM, std::string("bind: cudaMalloc: ") + cudaGetErrorString(e));
    }
    // upload
    std::vector<float> f32(nel);
    GM_CUDA_TRY(c, cudaMemcpy(c->dE64.p, c->E.data(), nel * 8, cudaMemcpyHostToDevice));
    for (long long e = 0; e < nel; ++e) f32[e] = (float)c->E[e];
    GM_CUDA_TRY(c, cudaMemcpy(c->dE32.p, f32.data(), nel * 4, cudaMemcpyHostToDevice));
    {
        std::vector<double> kap(nel);
        for (long long e = 0; e < nel; ++e) kap[e] = c->kperm[e] / c->mu_f;
        GM_CUDA_TRY(c, cudaMemcpy(c->dK64.p, kap.data(), nel * 8, cudaMemcpyHostToDevice));
        for (long long e = 0; e < nel; ++e) f32[e] = (float)kap[e];
        GM_CUDA_TRY(c, cudaMemcpy(c->dK32.p, f32.data(), nel * 4, cudaMemcpyHostToDevice));
    }
    // fixed-stress storage coefficient alpha^2 / K_dr with the drained bulk
    // modulus K_dr = E / (3 (1 - 2 nu)) of each element
    {
        std::vector<double> fs(nel);
        for (long long e = 0; e < nel; ++e) fs[e] = c->alpha * c->alpha * 3.0 * (1.0 - 2.0 * c->nu) / c->E[e];
        GM_CUDA_TRY(c, cudaMemcpy(c->dFS64.p, fs.data(), nel * 8, cudaMemcpyHostToDevice));
        for (long long e = 0; e < nel; ++e) f32[e] = (float)fs[e];
        GM_CUDA_TRY(c, cudaMemcpy(c->dFS32.p, f32.data(), nel * 4, cudaMemcpyHostToDevice));
    }
    std::vector<uint8_t> mask(N, 0);
    for (long long n = 0; n < N; ++n)
        for (int f = 0; f < 4; ++f)
            if (c->fixed[f * N + n]) mask[n] |= (uint8_t)(1u << f);
    GM_CUDA_TRY(c, cudaMemcpy(c->dmask.p, mask.data(), N, cudaMemcpyHostToDevice));
    GM_CUDA_TRY(c, cudaMemset(static_cast<uint8_t*>(c->dmask.p) + N, 0, 64));
    {
        // constrained tile-planes of the FP32 bulk kernel (15 x 15 tiles, 17 x 17
        // staged nodes; a tied upper lip also reads the lower lip's constraints)
        const int gx = (c->nx + 1 + 14) / 15, gy = (c->ny + 1 + 14) / 15, np = c->g.nplanes;
        const long long rl = c->nx + 1, nbp = c->g.nb;
        std::vector<uint8_t> any(nbp * np, 0), tf((size_t)np * gx * gy, 0);
        for (long long n = 0; n < N; ++n) any[n] = mask[n] != 0;
        for (int k = 0; k < np; ++k)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) {
                    uint8_t f = 0;
                    for (int j = by * 15 - 1; j <= by * 15 + 15 && !f; ++j) {
                        if (j < 0 || j > c->ny) continue;
                        for (int i = bx * 15 - 1; i <= bx * 15 + 15; ++i) {
                            if (i < 0 || i > c->nx) continue;
                            const long long q = i + rl * j;
                            if (any[q + nbp * k] || (c->g.tied && k == c->g.kf + 1 && any[q + nbp * c->g.kf])) {
                                f = 1;
                                break;
                            }
                        }
                    }
                    tf[((size_t)k * gy + by) * gx + bx] = f;
                }
        GM_CUDA_TRY(c, c->dtflag.alloc(tf.size()));
        GM_CUDA_TRY(c, cudaMemcpy(c->dtflag.p, tf.data(), tf.size(), cudaMemcpyHostToDevice));
    }
    c->bound = true;   // loads upload below needs the grid
    int rc = gm_prepare_bulk32(c);
    if (rc) { c->bound = false; return rc; }
    rc = upload_loads(c);
    if (rc) { c->bound = false; return rc; }
    GM_CUDA_TRY(c, cudaMemset(c->du_n.p, 0, N3 * 8));
    GM_CUDA_TRY(c, cudaMemset(c->dp_n.p, 0, N * 8));
    if (P > 0) {
        GM_CUDA_TRY(c, cudaMemset(c->ddlie_n.p, 0, 2 * P * 8));
        GM_CUDA_TRY(c, cudaMemset(c->dflags_n.p, GM_STICK, P));
        GM_CUDA_TRY(c, cudaMemset(c->dD64.p, 0, 6 * P * 8));
        GM_CUDA_TRY(c, cudaMemset(c->dD32.p, 0, 6 * P * 4));
    }
    GM_CUDA_TRY(c, cudaMemset(c->dscal.p, 0, 16 * sizeof(PcgScalars)));
    GM_CUDA_TRY(c, cudaMemset(c->dcount.p, 0, 64));
    if ((rc = gm_launch_diag(c, 0))) { c->bound = false; return rc; }
    if (c->has_fault) {
        if ((rc = gm_launch_return_map(c, c->du_n.as<double>(), nullptr, 0))) { c->bound = false; return rc; }
    }
    if ((rc = gm_launch_block_jacobi(c, 0))) { c->bound = false; return rc; }
    GM_CUDA_TRY(c, cudaDeviceSynchronize());
    // in-situ fault force floor for the Newton test
    if (int rc = gm_insitu_floor(c)) return rc;
    c->applies = 0;
    c->launches = 0;
    return GM_OK;
}

}  // namespace
