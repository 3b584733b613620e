// FP64 instantiations of the matrix-free operator applies.
#include "gm_apply.cuh"

int gm_launch_apply_f64(gm_ctx* c, int mode, double cK, double cApu, double cAup, double cS,
                        double cC, const double* xu, const double* xp, double* yu, double* yp,
                        cudaStream_t s, const int* skip)
{
    const double* E = c->dE64.as<double>();
    const double* kap = c->dK64.as<double>();
    const double* D = c->dD64.as<double>();
    const RefOps<double>& R = c->R64;
#define GM_CASE(MD) \
    case MD: gm_apply_dispatch_cls<double, MD>(c, R, cK, cApu, cAup, cS, cC, xu, xp, yu, yp, E, kap, D, s, skip); break;
    switch (mode) {
        GM_CASE(GM_MODE_K)
        GM_CASE(GM_MODE_KT)
        GM_CASE(GM_MODE_A22)
        GM_CASE(GM_MODE_APU)
        GM_CASE(GM_MODE_AUP)
        GM_CASE(GM_MODE_J)
        GM_CASE(GM_MODE_RES1)
        GM_CASE(GM_MODE_RES2)
    default:
        return c->set_err(GM_EINVAL, "unsupported operator mode");
    }
#undef GM_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->set_err(GM_ECUDA, std::string("apply launch: ") + cudaGetErrorString(e));
    return GM_OK;
}

int gm_launch_pcg_apply_f64(gm_ctx* c, int which, const double* z, const double* p_old, double* p_new, double* q,
                            PcgScalars* sc, cudaStream_t s)
{
    const double* E = c->dE64.as<double>();
    const double* kap = c->dK64.as<double>();
    const double* D = c->dD64.as<double>();
    // which 0: K_T; 1: A22; 2: A22 plus the fixed-stress storage term
    if (which == 0)
        gm_pcg_apply_dispatch<double, GM_MODE_KT>(c, c->R64, z, p_old, p_new, q, E, kap, D, sc, s, nullptr);
    else
        gm_pcg_apply_dispatch<double, GM_MODE_A22>(c, c->R64, z, p_old, p_new, q, E, kap, D, sc, s,
                                                  which == 2 ? c->dFS64.as<double>() : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->set_err(GM_ECUDA, std::string("pcg apply launch: ") + cudaGetErrorString(e));
    return GM_OK;
}

// Bulk part of K_T alone (no fault-kernel launch): y = K_b x.  The multigrid
// smoother adds the cohesive term of the lip pairs itself.
int gm_launch_bulk_k_f64(gm_ctx* c, const double* x, double* y, cudaStream_t s, const int* skip)
{
    int gx, gy, gz, zchunk;
    gm_bulk_geometry(c, &gx, &gy, &gz, &zchunk);
    BulkArgs<double> b = gm_bulk_args<double>(c, 1.0, 0.0, 0.0, 0.0, 0.0, c->dE64.as<double>(), c->dK64.as<double>());
    b.zchunk = zchunk;
    b.xu = x; b.xp = nullptr; b.yu = y; b.yp = nullptr;
    b.skip = skip;
    const dim3 grid(gx, gy, gz);
    switch (c->cls) {
    case GM_CLS_BOX: gm_bulk_apply_kernel<double, GM_CLS_BOX, GM_M_K, false><<<grid, 256, 0, s>>>(b, c->R64); break;
    case GM_CLS_MONO: gm_bulk_apply_kernel<double, GM_CLS_MONO, GM_M_K, false><<<grid, 256, 0, s>>>(b, c->R64); break;
    default: gm_bulk_apply_kernel<double, GM_CLS_GEN, GM_M_K, false><<<grid, 256, 0, s>>>(b, c->R64); break;
    }
    c->applies++;
    GM_LAUNCHED(c);
    return GM_OK;
}
