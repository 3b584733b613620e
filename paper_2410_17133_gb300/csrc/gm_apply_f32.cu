// FP32 instantiations of the matrix-free operator applies (mixed-precision path:
// FP32 operator data, FP32 accumulation inside each element and node).
#include "gm_apply.cuh"

int gm_launch_apply_f32(gm_ctx* c, int mode, double cK, double cApu, double cAup, double cS,
                        double cC, const float* xu, const float* xp, float* yu, float* yp,
                        cudaStream_t s, const int* skip)
{
    const float* E = c->dE32.as<float>();
    const float* kap = c->dK32.as<float>();
    const float* D = c->dD32.as<float>();
    const RefOps<float>& R = c->R32;
#define GM_CASE(MD) \
    case MD: gm_apply_dispatch_cls<float, MD>(c, R, cK, cApu, cAup, cS, cC, xu, xp, yu, yp, E, kap, D, s, skip); break;
    switch (mode) {
        GM_CASE(GM_MODE_K)
        GM_CASE(GM_MODE_KT)
        GM_CASE(GM_MODE_A22)
        GM_CASE(GM_MODE_APU)
        GM_CASE(GM_MODE_AUP)
        GM_CASE(GM_MODE_J)
    default:
        return c->set_err(GM_EINVAL, "unsupported operator mode (fp32)");
    }
#undef GM_CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->set_err(GM_ECUDA, std::string("apply launch: ") + cudaGetErrorString(e));
    return GM_OK;
}

int gm_launch_pcg_apply_f32(gm_ctx* c, int which, const float* z, const float* p_old, float* p_new, float* q,
                            PcgScalars* sc, cudaStream_t s)
{
    const float* E = c->dE32.as<float>();
    const float* kap = c->dK32.as<float>();
    const float* D = c->dD32.as<float>();
    // which 0: K_T; 1: A22; 2: A22 plus the fixed-stress storage term
    if (which == 0)
        gm_pcg_apply_dispatch<float, GM_MODE_KT>(c, c->R32, z, p_old, p_new, q, E, kap, D, sc, s, nullptr);
    else
        gm_pcg_apply_dispatch<float, GM_MODE_A22>(c, c->R32, z, p_old, p_new, q, E, kap, D, sc, s,
                                                  which == 2 ? c->dFS32.as<float>() : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->set_err(GM_ECUDA, std::string("pcg apply launch: ") + cudaGetErrorString(e));
    return GM_OK;
}

// Bulk part of K_T alone (no fault-kernel launch): y = K_b x.  The multigrid
// smoother adds the cohesive term of the lip pairs itself.
int gm_launch_bulk_k_f32(gm_ctx* c, const float* x, float* y, cudaStream_t s, const int* skip)
{
    int gx, gy, gz, zchunk;
    gm_bulk_geometry(c, &gx, &gy, &gz, &zchunk);
    BulkArgs<float> b = gm_bulk_args<float>(c, 1.0, 0.0, 0.0, 0.0, 0.0, c->dE32.as<float>(), c->dK32.as<float>());
    b.zchunk = zchunk;
    b.xu = x; b.xp = nullptr; b.yu = y; b.yp = nullptr;
    b.skip = skip;
    gm_bulk32_dispatch<GM_M_K, false>(c, b, s);
    c->applies++;
    GM_LAUNCHED(c);
    return GM_OK;
}

// Kernel attributes of the FP32 bulk kernels of the context's cell class (called
// at bind, so no attribute call happens inside a later stream capture).
template <int CLS>
static int gm_bulk32_setup_cls(int dev)
{
    int e = gm_bulk32_setup<CLS, GM_M_K, false>(dev);
    if (!e) e = gm_bulk32_setup<CLS, GM_M_K, true>(dev);
    if (!e) e = gm_bulk32_setup<CLS, GM_M_S | GM_M_C, false>(dev);
    if (!e) e = gm_bulk32_setup<CLS, GM_M_S | GM_M_C, true>(dev);
    return e;
}

int gm_prepare_bulk32(gm_ctx* c)
{
    const int e = c->cls == GM_CLS_BOX ? gm_bulk32_setup_cls<GM_CLS_BOX>(c->device)
                : c->cls == GM_CLS_MONO ? gm_bulk32_setup_cls<GM_CLS_MONO>(c->device)
                                        : gm_bulk32_setup_cls<GM_CLS_GEN>(c->device);
    if (e) return c->set_err(GM_ECUDA, std::string("bulk kernel set-up: ") + cudaGetErrorString((cudaError_t)e));
    return GM_OK;
}
