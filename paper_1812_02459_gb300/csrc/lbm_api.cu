// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// A handle owns one device arena holding every plane of the state and the
// scratch planes of one step.  A step is a fixed sequence of tile kernels on
// the handle's stream (see lbm_kernels.cuh):
//   collide+stream (both lattices) -> RK3 stage x3 -> Picard sweep xK -> filter.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

constexpr int CS_TX = 30, CS_TY = 14;    // collide+stream tile: its ring-1 region is 32 x 16 = one node per thread
constexpr int RK_TX = 64, RK_TY = 32, RK_NT = 512;   // RK3 stage tile, threads
constexpr int RS_NT = 256, RS_VR1 = 8, RS_VR2 = 6, RS_VR3 = 4;   // FP32 strips: threads, rows per strip
constexpr int PS_TX = 128, PS_TY = 16, PS_NT = 256, PS_VR1 = 6, PS_VR2 = 4;   // FP32 Picard strips
constexpr int PC_TX = 64, PC_TY = 16, PC_NT = 512;   // Picard sweep tile, threads
constexpr int FL_TX = 64, FL_TY = 16, FL_NT = 512;   // filter tile, threads
constexpr int FS_TX = 64, FS_TY = 64, FS_VR = 8;     // FP32 filter: tile, rows per thread
// TMA-staged FP32 kernels (nx a multiple of 4): tiles, threads, rows per
// strip, resident CTAs per SM the registers are sized for
constexpr int RT_NT = 256, RT_MINB = 4;
constexpr int PT_TX = 64, PT_TY = 16, PT_NT = 128, PT_VR1 = 6, PT_VR2 = 4, PT_MINB = 5;
constexpr int FT_TX = 64, FT_TY = 32, FT_VR = 4, FT_MINB = 4;
constexpr int CP_TX = 60, CP_TY = 14, CP_VR1 = 2;   // collide+stream on node pairs
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_MAX_BLOCKS = 304;     // 2 x 152 SMs (the diagnostics kernel's resident blocks)

thread_local std::string g_create_error;

// Explicit centred selective-filter coefficients d_0..d_5 (App. B table).
void filter_table(int order, double d[6])
{
    for (int k = 0; k < 6; ++k) d[k] = 0.0;
    if (order == 5) {
        d[0] = 6.0 / 16.0; d[1] = -4.0 / 16.0; d[2] = 1.0 / 16.0;
    } else if (order == 7) {
        d[0] = 5.0 / 16.0; d[1] = -15.0 / 64.0; d[2] = 3.0 / 32.0; d[3] = -1.0 / 64.0;
    } else if (order == 9) {
        d[0] = 0.243527493120; d[1] = -0.204788880640; d[2] = 0.120007591680;
        d[3] = -0.045211119360; d[4] = 0.008228661760;
    } else if (order == 11) {
        d[0] = 0.215044884112; d[1] = -0.187772883589; d[2] = 0.123755948787;
        d[3] = -0.059227575576; d[4] = 0.018721609157; d[5] = -0.002999540835;
    }
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace



namespace {

lbm_status fail(lbm_handle *h, lbm_status st, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return st;
}

lbm_status cuda_fail(lbm_handle *h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define CK(h, call, what)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, (what));  \
    } while (0)

template <typename T> KP<T> &kp_of(lbm_handle *h);
template <> KP<double> &kp_of<double>(lbm_handle *h) { return h->kpd; }
template <> KP<float> &kp_of<float>(lbm_handle *h) { return h->kpf; }

// Calls fn(T*, S*) with null pointers typed by the arithmetic type T and
// the population storage type S of a precision.
template <typename F>
lbm_status dispatch(int precision, F &&fn)
{
    switch (precision) {
    case LBM_FP64: return fn((double *)nullptr, (double *)nullptr);
    case LBM_FP32: return fn((float *)nullptr, (float *)nullptr);
    case LBM_MIX_BF16: return fn((float *)nullptr, (__nv_bfloat16 *)nullptr);
    default: return fn((float *)nullptr, (__half *)nullptr);
    }
}
#define TS_TYPES(tp, sp)                                \
    using T = std::remove_pointer_t<decltype(tp)>;      \
    using S = std::remove_pointer_t<decltype(sp)>;

template <typename T>
void build_kp(const lbm_grid &gr, const lbm_params &p, KP<T> &k)
{
    k.nx = gr.nx; k.ny = gr.ny; k.px = gr.periodic_x ? 1 : 0; k.py = gr.periodic_y ? 1 : 0;
    k.N = (long long)gr.nx * gr.ny;
    k.N32 = (unsigned)k.N;
    k.kappa = (T)(3.0 * p.sigma * p.W / 8.0);          // Sec. II.A, below Eq. (free_energy)
    k.beta = (T)(3.0 * p.sigma / (4.0 * p.W));
    k.eta = (T)p.eta; k.M = (T)p.M; k.lambda = (T)p.lambda; k.W = (T)p.W;
    k.flux_corr = p.flux_correction ? 1 : 0;
    k.rhoH = (T)p.rho_H; k.rhoL = (T)p.rho_L;
    k.muH = (T)(p.rho_H * p.nu_H); k.muL = (T)(p.rho_L * p.nu_L);
    k.drho = (T)((p.rho_H - p.rho_L) / 2.0);
    const double tau_f = 0.5 + p.M / (p.eta / 3.0);    // Eq. (mobility): M = eta cs^2 (tau_f - 1/2)
    for (int q = 0; q < 9; ++q) { k.sf[q] = (T)p.s_f[q]; k.sg[q] = (T)p.s_g[q]; }
    k.sf[3] = k.sf[5] = (T)(1.0 / tau_f);
    k.gx = (T)p.gx; k.gy = (T)p.gy;
    k.g_rho_ref = (T)p.g_rho_ref;
    k.eps2 = (T)(p.grad_eps * p.grad_eps);
    k.two_over_W = (T)(2.0 / p.W);
    double d[6];
    filter_table(p.filter_order, d);
    for (int m = 0; m < 6; ++m) k.fd[m] = (T)d[m];
    k.fa = (T)p.filter_a;
    k.fR = p.filter_order / 2;
}

lbm_status validate(const lbm_grid *gr, const lbm_params *p)
{
    char buf[256];
    if (!gr || !p) return fail(nullptr, LBM_ERR_ARG, "grid and params must be non-NULL");
    if (gr->nx < LBM_MIN_EXTENT || gr->ny < LBM_MIN_EXTENT) {
        snprintf(buf, sizeof buf, "nx, ny must be >= %d (got %d x %d)", LBM_MIN_EXTENT, gr->nx, gr->ny);
        return fail(nullptr, LBM_ERR_ARG, buf);
    }
    if ((long long)gr->nx * gr->ny > (1LL << 28))
        return fail(nullptr, LBM_ERR_ARG, "nx*ny must be <= 2^28 (16384^2)");
    if (gr->precision < LBM_FP64 || gr->precision > LBM_MIX_FP16)
        return fail(nullptr, LBM_ERR_ARG, "precision must be LBM_FP64, LBM_FP32, LBM_MIX_BF16 or LBM_MIX_FP16");
    if (!(p->M > 0) || !(p->eta > 0)) return fail(nullptr, LBM_ERR_ARG, "M and eta must be > 0 (tau_f > 1/2)");
    if (!(p->W > 0)) return fail(nullptr, LBM_ERR_ARG, "W must be > 0");
    if (!(p->sigma >= 0) || !(p->lambda >= 0)) return fail(nullptr, LBM_ERR_ARG, "sigma, lambda must be >= 0");
    if (!(p->rho_H > 0) || !(p->rho_L > 0)) return fail(nullptr, LBM_ERR_ARG, "densities must be > 0");
    if (!(p->nu_H > 0) || !(p->nu_L > 0)) return fail(nullptr, LBM_ERR_ARG, "viscosities must be > 0 (tau_g > 1/2)");
    for (int q = 0; q < 9; ++q)
        if (!(p->s_f[q] >= 0 && p->s_f[q] <= 2) || !(p->s_g[q] >= 0 && p->s_g[q] <= 2))
            return fail(nullptr, LBM_ERR_ARG, "relaxation rates must lie in [0, 2]");
    const double tau_f = 0.5 + p->M / (p->eta / 3.0);
    if (!(1.0 / tau_f <= 2.0)) return fail(nullptr, LBM_ERR_ARG, "1/tau_f must be <= 2");
    int fo = p->filter_order;
    if (fo != 0 && fo != 5 && fo != 7 && fo != 9 && fo != 11)
        return fail(nullptr, LBM_ERR_ARG, "filter_order must be 0, 5, 7, 9 or 11");
    if (fo && !(p->filter_a > 0 && p->filter_a <= 1)) return fail(nullptr, LBM_ERR_ARG, "filter_a must be in (0, 1]");
    if (p->picard_iters < 1 || p->picard_iters > 64) return fail(nullptr, LBM_ERR_ARG, "picard_iters must be in [1, 64]");
    if (p->picard_zeta != 0.0) return fail(nullptr, LBM_ERR_ARG, "picard_zeta must be 0 (fixed sweep count)");
    if (!(p->grad_eps > 0)) return fail(nullptr, LBM_ERR_ARG, "grad_eps must be > 0");
    if (p->flags & ~(unsigned)LBM_FLAG_STRAIN_MOMENTS)
        return fail(nullptr, LBM_ERR_ARG, "flags: only LBM_FLAG_STRAIN_MOMENTS is defined");
    if ((p->flags & LBM_FLAG_STRAIN_MOMENTS) && gr->precision != LBM_FP64 && gr->precision != LBM_FP32)
        return fail(nullptr, LBM_ERR_ARG, "LBM_FLAG_STRAIN_MOMENTS needs FP64 or FP32 populations");
    if (!std::isfinite(p->gx) || !std::isfinite(p->gy)) return fail(nullptr, LBM_ERR_ARG, "gravity must be finite");
    if (!(p->g_rho_ref >= 0) || !std::isfinite(p->g_rho_ref)) return fail(nullptr, LBM_ERR_ARG, "g_rho_ref must be >= 0");
    return LBM_OK;
}

template <typename T> size_t smem_cs() { return sizeof(T) * CSGeom<CS_TX, CS_TY>::NSCALAR; }
template <typename T> size_t smem_rk() { return sizeof(T) * RKGeom<RK_TX, RK_TY>::NSCALAR; }
template <typename T> size_t smem_pc() { return sizeof(T) * PCGeom<PC_TX, PC_TY>::NSCALAR; }
template <typename T, int R> size_t smem_fl() { return sizeof(T) * FLGeom<FL_TX, FL_TY, R>::NSCALAR; }

// The default relaxation rates (s_f = 1 except s_f[3], s_f[5]; s_g[0..3] =
// s_g[5] = 1) select the collide kernel that skips the rate-1 relaxations.
bool default_rates(const lbm_params &p)
{
    for (int k : {0, 1, 2, 4, 6, 7, 8})
        if (p.s_f[k] != 1.0) return false;
    for (int k : {0, 1, 2, 3, 5})
        if (p.s_g[k] != 1.0) return false;
    return true;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependence on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

// The tensor map of an FP32 plane of the handle for bw x bh windows.
lbm_status tmap(lbm_handle *h, const void *plane, int bw, int bh, CUtensorMap *out)
{
    for (const auto &e : h->tmaps)
        if (e.ptr == plane && e.bw == bw && e.bh == bh) {
            *out = e.map;
            return LBM_OK;
        }
    auto fn = encode_tiled();
    if (!fn) return fail(h, LBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    lbm_handle::TmaEntry e{plane, bw, bh, {}};
    const cuuint64_t dims[2] = {(cuuint64_t)h->grid.nx, (cuuint64_t)h->grid.ny};
    const cuuint64_t strides[1] = {(cuuint64_t)h->grid.nx * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(&e.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(plane), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, LBM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    h->tmaps.push_back(e);
    *out = e.map;
    return LBM_OK;
}

// Dynamic shared memory of a TMA-staged kernel above the 48 KB default.
template <typename K> lbm_status setup_tma_kernel(lbm_handle *h, K kern, size_t bytes)
{
    CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
       "cudaFuncSetAttribute(tma kernel)");
    return LBM_OK;
}

template <int R> lbm_status setup_filter_tma(lbm_handle *h)
{
    return setup_tma_kernel(h, k_filter_tma<FT_TX, FT_TY, R, FT_VR, FT_MINB>, FLTGeom<FT_TX, FT_TY, R, FT_VR>::Tile::BYTES);
}

template <int R> lbm_status set_strip_smem(lbm_handle *h)
{
    CK(h, cudaFuncSetAttribute(k_filter_strips<FS_TX, FS_TY, R, FS_VR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(float) * FLSGeom<FS_TX, FS_TY, R, FS_VR>::NSCALAR)),
       "cudaFuncSetAttribute(filter_strips)");
    return LBM_OK;
}

template <typename T, typename S>
lbm_status set_smem_limits(lbm_handle *h)
{
    CK(h, cudaFuncSetAttribute(k_collide_stream<T, S, CS_TX, CS_TY, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cs<T>()),
       "cudaFuncSetAttribute(collide_stream)");
    CK(h, cudaFuncSetAttribute(k_collide_stream<T, S, CS_TX, CS_TY, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cs<T>()),
       "cudaFuncSetAttribute(collide_stream)");
    CK(h, cudaFuncSetAttribute(k_collide_ch<T, CS_TX, CS_TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(T) * CHGeom<CS_TX, CS_TY>::NSCALAR)),
       "cudaFuncSetAttribute(collide_ch)");
    CK(h, cudaFuncSetAttribute(k_rk_stage<T, RK_TX, RK_TY, RK_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_rk<T>()),
       "cudaFuncSetAttribute(rk_stage)");
    CK(h, cudaFuncSetAttribute(k_picard<T, PC_TX, PC_TY, PC_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_pc<T>()),
       "cudaFuncSetAttribute(picard)");
    CK(h, cudaFuncSetAttribute(k_filter<T, FL_TX, FL_TY, 5, FL_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_fl<T, 5>()),
       "cudaFuncSetAttribute(filter)");
    if constexpr (std::is_same<T, float>::value) {
        CK(h, cudaFuncSetAttribute(k_rk_strips<RK_TX, RK_TY, RS_NT, RS_VR1, RS_VR2, RS_VR3>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rk<float>()),
           "cudaFuncSetAttribute(rk_strips)");
        CK(h, cudaFuncSetAttribute(k_picard_strips<PS_TX, PS_TY, PS_NT, PS_VR1, PS_VR2>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(float) * PSGeom<PS_TX, PS_TY>::NSCALAR)),
           "cudaFuncSetAttribute(picard_strips)");
        lbm_status st = set_strip_smem<2>(h);
        if (st == LBM_OK) st = set_strip_smem<3>(h);
        if (st == LBM_OK) st = set_strip_smem<4>(h);
        if (st == LBM_OK) st = set_strip_smem<5>(h);
        if (st != LBM_OK) return st;
        if (h->tma) {
            st = setup_tma_kernel(h, k_collide_pairs<S, CP_TX, CP_TY, CP_VR1>, CPGeom<CP_TX, CP_TY>::Tile::BYTES);
            if (st == LBM_OK)
                st = setup_tma_kernel(h, k_rk_tma<RK_TX, RK_TY, RT_NT, RS_VR1, RS_VR2, RS_VR3, RT_MINB>,
                                  RKTGeom<RK_TX, RK_TY>::Tile::BYTES);
            if (st == LBM_OK)
                st = setup_tma_kernel(h, k_picard_tma<PT_TX, PT_TY, PT_NT, PT_VR1, PT_VR2, PT_MINB>,
                                      PCTGeom<PT_TX, PT_TY>::Tile::BYTES);
            if (st == LBM_OK) {
                switch (h->kpf.fR) {
                case 2: st = setup_filter_tma<2>(h); break;
                case 3: st = setup_filter_tma<3>(h); break;
                case 4: st = setup_filter_tma<4>(h); break;
                case 5: st = setup_filter_tma<5>(h); break;
                default: break;
                }
            }
            if (st != LBM_OK) return st;
        }
    }
    return LBM_OK;
}

cudaEvent_t take_event(lbm_handle *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one kernel launch with events when per-kernel timing is on.
// Every pass of a step is launched inside a Timed: an NVTX range named for
// the pass's kind (seen by a profiler that records NVTX; free otherwise)
// and, while lbm_profile is on, CUDA events around the launch.
struct Timed {
    lbm_handle *h;
    int kind;
    cudaEvent_t a = nullptr;
    bool own = true;
    Timed(lbm_handle *h_, int k) : h(h_), kind(k)
    {
        nvtxRangePushA(lbm_kernel_name(k));
        if (h->prof) {
            if (h->chain_ok && h->chain) {
                a = h->chain;
                own = false;
            } else {
                a = take_event(h);
                cudaEventRecord(a, h->stream);
            }
        }
    }
    ~Timed()
    {
        if (h->prof && a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, h->stream);
            h->marks.push_back({kind, a, b, own});
            h->chain = b;
        }
        nvtxRangePop();
    }
};

template <typename T, int R>
lbm_status launch_filter_r(lbm_handle *h, const T *pin, const T *uxi, const T *uyi, T *po, T *uxo, T *uyo)
{
    const KP<T> &P = kp_of<T>(h);
    dim3 grid((P.nx + FL_TX - 1) / FL_TX, (P.ny + FL_TY - 1) / FL_TY);
    Timed tm(h, 3);
    if constexpr (std::is_same<T, float>::value) {
        if (h->tma) {   // TMA-staged windows, one CTA per tile
            using GT = FLTGeom<FT_TX, FT_TY, R, FT_VR>;
            TmaMaps maps{};
            const void *planes[3] = {pin, uxi, uyi};
            for (int f = 0; f < 3; ++f) {
                lbm_status r = tmap(h, planes[f], GT::BW, GT::BH, &maps.m[f]);
                if (r) return r;
            }
            const int ntiles = ((P.nx + FT_TX - 1) / FT_TX) * ((P.ny + FT_TY - 1) / FT_TY);
            k_filter_tma<FT_TX, FT_TY, R, FT_VR, FT_MINB><<<ntiles, GT::NT, GT::Tile::BYTES, h->stream>>>(
                maps, P, pin, uxi, uyi, po, uxo, uyo, h->dev_err);
            return LBM_OK;
        }
        if (P.nx % 2 == 0) {   // 2 x 8 node blocks, register reuse, paired FP32 arithmetic
            using GS = FLSGeom<FS_TX, FS_TY, R, FS_VR>;
            dim3 gs((P.nx + FS_TX - 1) / FS_TX, (P.ny + FS_TY - 1) / FS_TY);
            k_filter_strips<FS_TX, FS_TY, R, FS_VR><<<gs, GS::NT, sizeof(float) * GS::NSCALAR, h->stream>>>(
                P, pin, uxi, uyi, po, uxo, uyo);
            return LBM_OK;
        }
    }
    k_filter<T, FL_TX, FL_TY, R, FL_NT><<<grid, FL_NT, smem_fl<T, R>(), h->stream>>>(P, pin, uxi, uyi, po, uxo, uyo);
    return LBM_OK;
}

// TVD-RK3 finite-difference correction (Sec. III.A Eq. TVD-3order) in
// increments over phi^n: dbar -> d1 -> d2 -> phi^{n+1} = phi^n + d3 (written
// to phin, with phi_lo updated for FP32 handles).
template <typename T>
lbm_status rk3_impl(lbm_handle *h, T *phi, T *phin, T *dbar, T *philo)
{
    const KP<T> &P = kp_of<T>(h);
    cudaStream_t st = h->stream;
    dim3 grid((P.nx + RK_TX - 1) / RK_TX, (P.ny + RK_TY - 1) / RK_TY);
    const size_t sm = smem_rk<T>();
    const T *src[3] = {dbar, (const T *)h->s1, (const T *)h->s2};
    T *dst[3] = {(T *)h->s1, (T *)h->s2, phin};
    const T ca[3] = {T(0), T(0.75), T(1.0 / 3.0)}, cb[3] = {T(1), T(0.25), T(2.0 / 3.0)};
    for (int k = 0; k < 3; ++k) {
        Timed tm(h, 1);
        const int last = k == 2;
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
            if (h->tma) {   // TMA-staged windows, one CTA per tile
                using GT = RKTGeom<RK_TX, RK_TY>;
                TmaMaps maps{};
                lbm_status r = tmap(h, phi, GT::BW, GT::BH, &maps.m[0]);
                if (!r) r = tmap(h, src[k], GT::BW, GT::BH, &maps.m[1]);
                if (r) return r;
                k_rk_tma<RK_TX, RK_TY, RT_NT, RS_VR1, RS_VR2, RS_VR3, RT_MINB>
                    <<<grid.x * grid.y, RT_NT, GT::Tile::BYTES, st>>>(maps, P, phi, src[k], dbar, dst[k],
                                                                     ca[k], cb[k], last, philo, h->dev_err);
                done = true;
            } else if (P.nx % 2 == 0) {   // column-pair strips, paired FP32 arithmetic
                k_rk_strips<RK_TX, RK_TY, RS_NT, RS_VR1, RS_VR2, RS_VR3><<<grid, RS_NT, sm, st>>>(
                    P, phi, src[k], dbar, dst[k], ca[k], cb[k], last, philo);
                done = true;
            }
        }
        if (!done)
            k_rk_stage<T, RK_TX, RK_TY, RK_NT><<<grid, RK_NT, sm, st>>>(P, phi, src[k], dbar, dst[k], ca[k],
                                                                      cb[k], last, philo);
    }
    return LBM_OK;
}

template <typename T, typename S>
lbm_status step_impl(lbm_handle *h)
{
    const KP<T> &P = kp_of<T>(h);
    cudaStream_t st = h->stream;
    const int c = h->cur, u = h->ucur;
    // phi^n; the other phi slot holds phi^{n-1} (the phi the stored
    // populations were collided with) and receives phi^{n+1}
    T *phi = (T *)h->phi[h->pcur], *phin = (T *)h->phi[1 - h->pcur], *pf = (T *)h->pf;
    T *uxc = (T *)h->ux[u], *uyc = (T *)h->uy[u], *uxp = (T *)h->ux[1 - u], *uyp = (T *)h->uy[1 - u];
    T *uhx = (T *)h->uhx, *uhy = (T *)h->uhy;
    const T *dbar_old = (const T *)h->dbar[h->acur], *phat_old = (const T *)h->phat[h->acur];
    T *dbar = (T *)h->dbar[1 - h->acur], *phat = (T *)h->phat[1 - h->acur];
    T *philo = sizeof(T) == sizeof(float) ? (T *)h->philo : nullptr;   // low part of phi (FP32)
    T *jx = (T *)h->jx, *jy = (T *)h->jy;

    {   // fields, forces, collision of f and g, pull streaming, post-stream moments
        dim3 grid((P.nx + CS_TX - 1) / CS_TX, (P.ny + CS_TY - 1) / CS_TY);
        Timed tm(h, 0);
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
            if (h->tma && P.px && default_rates(h->prm)) {   // node pairs, TMA-staged windows
                using GC = CPGeom<CP_TX, CP_TY>;
                TmaMaps maps{};
                const void *planes[4] = {phi, pf, uxc, uyc};
                for (int f = 0; f < 4; ++f) {
                    lbm_status r = tmap(h, planes[f], GC::BW, GC::BH, &maps.m[f]);
                    if (r) return r;
                }
                const int ntiles = ((P.nx + CP_TX - 1) / CP_TX) * ((P.ny + CP_TY - 1) / CP_TY);
                k_collide_pairs<S, CP_TX, CP_TY, CP_VR1><<<ntiles, GC::NT, GC::Tile::BYTES, st>>>(
                    maps, P, (const S *)h->f[c], (const S *)h->g[c], (S *)h->f[1 - c], (S *)h->g[1 - c], phi, pf,
                    uxc, uyc, uxp, uyp, uhx, uhy, (const float *)philo, dbar, phat, jx, jy, h->dev_err);
                done = true;
            }
        }
        if (!done) {
            auto kern = default_rates(h->prm) ? k_collide_stream<T, S, CS_TX, CS_TY, true>
                                              : k_collide_stream<T, S, CS_TX, CS_TY, false>;
            kern<<<grid, (CS_TX + 2) * (CS_TY + 2), smem_cs<T>(), st>>>(
                P, (const S *)h->f[c], (const S *)h->g[c], (S *)h->f[1 - c], (S *)h->g[1 - c], phi, pf, uxc, uyc,
                uxp, uyp, uhx, uhy, phin, dbar_old, phat_old, philo, dbar, phat, jx, jy);
        }
    }
    {   // TVD-RK3 finite-difference correction: phi^n + dbar -> phi^{n+1}
        lbm_status r = rk3_impl<T>(h, phi, phin, dbar, philo);
        if (r) return r;
    }
    {   // implicit velocity by Picard sweeps; the last sweep lands in u_hat
        dim3 grid((P.nx + PC_TX - 1) / PC_TX, (P.ny + PC_TY - 1) / PC_TY);
        const int K = h->prm.picard_iters;
        // F_nu's strain rate from the step's post-stream NS populations (flags bit 0)
        const T *gpop = (h->prm.flags & LBM_FLAG_STRAIN_MOMENTS) ? (const T *)h->g[1 - c] : nullptr;
        for (int k = 0; k < K; ++k) {
            const T *ix = k == 0 ? uxc : (const T *)h->tk[(k - 1) & 1][0];
            const T *iy = k == 0 ? uyc : (const T *)h->tk[(k - 1) & 1][1];
            T *ox = k == K - 1 ? uhx : (T *)h->tk[k & 1][0];
            T *oy = k == K - 1 ? uhy : (T *)h->tk[k & 1][1];
            Timed tm(h, 2);
            if constexpr (std::is_same<T, float>::value) {
                if (h->tma && !gpop) {   // TMA-staged windows, one CTA per tile
                    using GT = PCTGeom<PT_TX, PT_TY>;
                    TmaMaps maps{};
                    const void *planes[4] = {phin, phat, ix, iy};
                    for (int f = 0; f < 4; ++f) {
                        lbm_status r = tmap(h, planes[f], GT::BW, GT::BH, &maps.m[f]);
                        if (r) return r;
                    }
                    const int ntiles = ((P.nx + PT_TX - 1) / PT_TX) * ((P.ny + PT_TY - 1) / PT_TY);
                    k_picard_tma<PT_TX, PT_TY, PT_NT, PT_VR1, PT_VR2, PT_MINB>
                        <<<ntiles, PT_NT, GT::Tile::BYTES, st>>>(maps, P, phin, phat, jx, jy, ix, iy, ox, oy,
                                                                 h->dev_err);
                    continue;
                }
                if (P.nx % 2 == 0 && !gpop) {   // column-pair strips, paired FP32 arithmetic
                    dim3 gs((P.nx + PS_TX - 1) / PS_TX, (P.ny + PS_TY - 1) / PS_TY);
                    k_picard_strips<PS_TX, PS_TY, PS_NT, PS_VR1, PS_VR2>
                        <<<gs, PS_NT, sizeof(float) * PSGeom<PS_TX, PS_TY>::NSCALAR, st>>>(P, phin, phat, jx, jy, ix, iy,
                                                                                         ox, oy);
                    continue;
                }
            }
            k_picard<T, PC_TX, PC_TY, PC_NT><<<grid, PC_NT, smem_pc<T>(), st>>>(P, phin, phat, jx, jy, ix, iy, ox, oy,
                                                                              gpop);
        }
    }
    // selective filter of (p_hat, u_hat) -> (p_f, u_f^{n+1}); u^{n-1} slot is reused
    switch (P.fR) {
    case 2: {
        lbm_status r = launch_filter_r<T, 2>(h, phat, uhx, uhy, pf, uxp, uyp);
        if (r) return r;
        break;
    }
    case 3: {
        lbm_status r = launch_filter_r<T, 3>(h, phat, uhx, uhy, pf, uxp, uyp);
        if (r) return r;
        break;
    }
    case 4: {
        lbm_status r = launch_filter_r<T, 4>(h, phat, uhx, uhy, pf, uxp, uyp);
        if (r) return r;
        break;
    }
    case 5: {
        lbm_status r = launch_filter_r<T, 5>(h, phat, uhx, uhy, pf, uxp, uyp);
        if (r) return r;
        break;
    }
    default: {
        const size_t b = sizeof(T) * (size_t)P.N;
        CK(h, cudaMemcpyAsync(pf, phat, b, cudaMemcpyDeviceToDevice, st), "copy p");
        CK(h, cudaMemcpyAsync(uxp, uhx, b, cudaMemcpyDeviceToDevice, st), "copy ux");
        CK(h, cudaMemcpyAsync(uyp, uhy, b, cudaMemcpyDeviceToDevice, st), "copy uy");
        h->chain = nullptr;   // the next launch does not directly follow a timed one
    }
    }
    CK(h, cudaGetLastError(), "kernel launch");
    h->cur ^= 1;
    h->ucur ^= 1;
    h->acur ^= 1;
    h->pcur ^= 1;
    return LBM_OK;
}

// The two RK stage planes are adjacent in the arena; between steps they
// serve as an N-double staging area for field transfers.
double *staging(lbm_handle *h) { return (double *)h->s1; }

// Host double field -> device plane of T (converted on the device).
template <typename T>
lbm_status upload_plane(lbm_handle *h, void *dst, const double *src)
{
    const size_t n = (size_t)h->N;
    if constexpr (sizeof(T) == sizeof(double)) {
        CK(h, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
    } else {
        CK(h, cudaMemcpyAsync(staging(h), src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
        k_cast<double, T><<<(int)std::min<long long>((h->N + 255) / 256, 4096), 256, 0, h->stream>>>(
            staging(h), (T *)dst, h->N);
        CK(h, cudaGetLastError(), "upload cast");
    }
    return LBM_OK;
}

// Device plane of T -> host double field (converted on the device).
template <typename T>
lbm_status download_plane(lbm_handle *h, double *dst, const void *src)
{
    if (!dst) return LBM_OK;
    const size_t n = (size_t)h->N;
    const void *from = src;
    if (sizeof(T) != sizeof(double)) {
        k_cast<T, double><<<(int)std::min<long long>((h->N + 255) / 256, 4096), 256, 0, h->stream>>>(
            (const T *)src, staging(h), h->N);
        CK(h, cudaGetLastError(), "download cast");
        from = staging(h);
    }
    CK(h, cudaMemcpyAsync(dst, from, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "download");
    CK(h, cudaStreamSynchronize(h->stream), "download sync");
    return LBM_OK;
}

// n steps of the Cahn-Hilliard part alone under u = tfac[k] (ux, uy) at
// step k (tfac NULL: 1); the NS lattice, p and u_hat are left as they are.
template <typename T>
lbm_status step_ch_impl(lbm_handle *h, int n, const double *ux, const double *uy, const double *tfac)
{
    if (n == 0) return LBM_OK;
    const KP<T> &P = kp_of<T>(h);
    cudaStream_t st = h->stream;
    const size_t b = sizeof(T) * (size_t)h->N;
    T *u0x = (T *)h->tk[0][0], *u0y = (T *)h->tk[0][1];   // the prescribed field (Picard scratch)
    lbm_status r;
    if ((r = upload_plane<T>(h, u0x, ux))) return r;
    if ((r = upload_plane<T>(h, u0y, uy))) return r;
    // g stays put: both population buffers hold it, so the buffer flips below are harmless
    CK(h, cudaMemcpyAsync(h->g[1 - h->cur], h->g[h->cur], 9 * b, cudaMemcpyDeviceToDevice, st), "ch copy g");
    CK(h, cudaMemcpyAsync(h->phat[1 - h->acur], h->phat[h->acur], b, cudaMemcpyDeviceToDevice, st), "ch copy p");
    T *philo = sizeof(T) == sizeof(float) ? (T *)h->philo : nullptr;
    using G = CHGeom<CS_TX, CS_TY>;
    dim3 grid((P.nx + CS_TX - 1) / CS_TX, (P.ny + CS_TY - 1) / CS_TY);
    for (int k = 0; k < n; ++k) {
        const T us = tfac ? (T)tfac[k] : T(1);
        // u of the previous step: the state's at the first step, then the prescribed one
        const T *upx = k == 0 ? (const T *)h->ux[1 - h->ucur] : u0x;
        const T *upy = k == 0 ? (const T *)h->uy[1 - h->ucur] : u0y;
        const T ups = k == 0 ? T(1) : (tfac ? (T)tfac[k - 1] : T(1));
        T *phi = (T *)h->phi[h->pcur], *phin = (T *)h->phi[1 - h->pcur];
        T *dbar = (T *)h->dbar[1 - h->acur];
        {
            Timed tm(h, 0);
            k_collide_ch<T, CS_TX, CS_TY><<<grid, (CS_TX + 2) * (CS_TY + 2), sizeof(T) * G::NSCALAR, st>>>(
                P, (const T *)h->f[h->cur], (T *)h->f[1 - h->cur], phi, philo, u0x, u0y, us, upx, upy, ups, dbar);
        }
        if ((r = rk3_impl<T>(h, phi, phin, dbar, philo))) return r;
        CK(h, cudaGetLastError(), "kernel launch");
        h->cur ^= 1;
        h->acur ^= 1;
        h->pcur ^= 1;
    }
    // u of the last step becomes the state's velocity and its previous one
    const T ul = tfac ? (T)tfac[n - 1] : T(1);
    const int blocks = (int)std::min<long long>((h->N + 255) / 256, 4096);
    for (int s2 = 0; s2 < 2; ++s2) {
        k_scale<T><<<blocks, 256, 0, st>>>(u0x, ul, (T *)h->ux[s2], h->N);
        k_scale<T><<<blocks, 256, 0, st>>>(u0y, ul, (T *)h->uy[s2], h->N);
    }
    CK(h, cudaGetLastError(), "kernel launch");
    return LBM_OK;
}

// phi^n from host doubles: FP32 handles keep it as phi_hi + phi_lo.
template <typename T>
lbm_status upload_phi(lbm_handle *h, const double *src)
{
    if constexpr (sizeof(T) == sizeof(double)) {
        return upload_plane<T>(h, h->phi[h->pcur], src);
    } else {
        const size_t n = (size_t)h->N;
        CK(h, cudaMemcpyAsync(staging(h), src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
        k_split<<<(int)std::min<long long>((h->N + 255) / 256, 4096), 256, 0, h->stream>>>(
            staging(h), (float *)h->phi[h->pcur], (float *)h->philo, h->N);
        CK(h, cudaGetLastError(), "upload split");
        return LBM_OK;
    }
}

// phi^n to host doubles (phi_hi + phi_lo for FP32 handles).
template <typename T>
lbm_status download_phi(lbm_handle *h, double *dst)
{
    if (!dst) return LBM_OK;
    if constexpr (sizeof(T) == sizeof(double)) {
        return download_plane<T>(h, dst, phi_cur(h));
    } else {
        const size_t n = (size_t)h->N;
        k_join<<<(int)std::min<long long>((h->N + 255) / 256, 4096), 256, 0, h->stream>>>(
            (const float *)phi_cur(h), (const float *)h->philo, staging(h), h->N);
        CK(h, cudaGetLastError(), "download join");
        CK(h, cudaMemcpyAsync(dst, staging(h), n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "download");
        CK(h, cudaStreamSynchronize(h->stream), "download sync");
        return LBM_OK;
    }
}

// Dynamic pressure p' = rho(phi) p at every node (Sec. II.B: the state's p is
// the kinematic pressure p'/rho), with rho(phi) of Eq. (rho) and phi clamped
// to [-1, 1] as in the step.  The reconstruction runs in FP64 from phi (the
// float pair phi_hi + phi_lo of FP32 handles, lo NULL otherwise) and p.
template <typename T>
static __global__ void k_dynamic_pressure(const T *__restrict__ phi, const float *__restrict__ lo,
                                          const T *__restrict__ p, double rhoH, double rhoL,
                                          double *__restrict__ out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double c = (double)phi[k] + (lo ? (double)lo[k] : 0.0);
        c = c < -1.0 ? -1.0 : (c > 1.0 ? 1.0 : c);
        out[k] = (rhoH * (1.0 + c) * 0.5 + rhoL * (1.0 - c) * 0.5) * (double)p[k];
    }
}

template <typename T>
lbm_status dynamic_pressure_impl(lbm_handle *h, double *dst)
{
    const size_t n = (size_t)h->N;
    const float *lo = sizeof(T) == sizeof(float) ? (const float *)h->philo : nullptr;
    k_dynamic_pressure<T><<<(int)std::min<long long>((h->N + 255) / 256, 4096), 256, 0, h->stream>>>(
        (const T *)phi_cur(h), lo, (const T *)h->pf, h->prm.rho_H, h->prm.rho_L, staging(h), h->N);
    CK(h, cudaGetLastError(), "dynamic pressure");
    CK(h, cudaMemcpyAsync(dst, staging(h), n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "download");
    CK(h, cudaStreamSynchronize(h->stream), "download sync");
    return LBM_OK;
}

template <typename T>
lbm_status upload_field(lbm_handle *h, void *dst, const double *src)
{
    const size_t n = (size_t)h->N;
    if (sizeof(T) == sizeof(double)) {
        CK(h, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
        return LBM_OK;
    }
    std::vector<T> tmp(n);
    for (size_t k = 0; k < n; ++k) tmp[k] = (T)src[k];
    CK(h, cudaMemcpyAsync(dst, tmp.data(), n * sizeof(T), cudaMemcpyHostToDevice, h->stream), "upload");
    CK(h, cudaStreamSynchronize(h->stream), "upload sync");
    return LBM_OK;
}

template <typename T>
lbm_status download_field(lbm_handle *h, double *dst, const void *src, size_t count)
{
    if (!dst) return LBM_OK;
    if (sizeof(T) == sizeof(double)) {
        CK(h, cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "download");
        CK(h, cudaStreamSynchronize(h->stream), "download sync");
        return LBM_OK;
    }
    std::vector<T> tmp(count);
    CK(h, cudaMemcpyAsync(tmp.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, h->stream), "download");
    CK(h, cudaStreamSynchronize(h->stream), "download sync");
    for (size_t k = 0; k < count; ++k) dst[k] = (double)tmp[k];
    return LBM_OK;
}

template <typename T, typename S>
lbm_status init_impl(lbm_handle *h, const double *phi0, const double *p0, const double *ux0, const double *uy0)
{
    lbm_status st;
    h->pcur = 0;
    if ((st = upload_phi<T>(h, phi0))) return st;
    if ((st = upload_plane<T>(h, h->pf, p0))) return st;
    if ((st = upload_plane<T>(h, h->ux[0], ux0))) return st;
    if ((st = upload_plane<T>(h, h->uy[0], uy0))) return st;
    const size_t b = sizeof(T) * (size_t)h->N;
    h->cur = 0;
    h->ucur = 0;
    // u^{n-1} = u_hat = u0 at the start
    CK(h, cudaMemcpyAsync(h->ux[1], h->ux[0], b, cudaMemcpyDeviceToDevice, h->stream), "init copy");
    CK(h, cudaMemcpyAsync(h->uy[1], h->uy[0], b, cudaMemcpyDeviceToDevice, h->stream), "init copy");
    CK(h, cudaMemcpyAsync(h->uhx, h->ux[0], b, cudaMemcpyDeviceToDevice, h->stream), "init copy");
    CK(h, cudaMemcpyAsync(h->uhy, h->uy[0], b, cudaMemcpyDeviceToDevice, h->stream), "init copy");
    // the previous-step slot of phi equals phi: the stored populations sum to it
    CK(h, cudaMemcpyAsync(h->phi[1], h->phi[0], b, cudaMemcpyDeviceToDevice, h->stream), "init copy");
    h->acur = 0;
    const KP<T> &P = kp_of<T>(h);
    int blocks = (int)std::min<long long>((P.N + 255) / 256, 4096);
    k_init<T, S><<<blocks, 256, 0, h->stream>>>(P, (const T *)h->phi[0], (const T *)h->pf, (const T *)h->ux[0],
                                                 (const T *)h->uy[0], (S *)h->f[0], (S *)h->g[0],
                                                 (T *)h->dbar[0], (T *)h->phat[0]);
    CK(h, cudaGetLastError(), "init kernel");
    CK(h, cudaStreamSynchronize(h->stream), "init sync");
    h->fresh_init = true;
    h->chk_pending = false;
    h->chk_status = LBM_OK;
    h->chk_count = 0;
    return LBM_OK;
}

template <typename T>
lbm_status diag_impl(lbm_handle *h, double *out, bool sync = true)
{
    const KP<T> &P = kp_of<T>(h);
    k_diag_partial<T><<<h->diag_blocks, DIAG_THREADS, 0, h->stream>>>(
        P.nx, P.ny, (const T *)phi_cur(h), (const T *)h->pf, (const T *)h->ux[h->ucur], (const T *)h->uy[h->ucur],
        h->diag_part);
    k_diag_final<<<1, 32 * NDIAG, 0, h->stream>>>(h->diag_blocks, h->diag_part, h->diag_out);
    CK(h, cudaGetLastError(), "diagnostics launch");
    CK(h, cudaMemcpyAsync(out, h->diag_out, sizeof(double) * NDIAG, cudaMemcpyDeviceToHost, h->stream),
       "diagnostics copy");
    if (sync) CK(h, cudaStreamSynchronize(h->stream), "diagnostics sync");
    return LBM_OK;
}

template <typename T>
lbm_status fields_impl(lbm_handle *h, double *phi, double *p, double *ux, double *uy)
{
    lbm_status st;
    if ((st = download_phi<T>(h, phi))) return st;
    if ((st = download_plane<T>(h, p, h->pf))) return st;
    if ((st = download_plane<T>(h, ux, h->ux[h->ucur]))) return st;
    if ((st = download_plane<T>(h, uy, h->uy[h->ucur]))) return st;
    return LBM_OK;
}

constexpr double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

// Host side of the reduced-precision codecs (same scaling as the device Codec).
template <typename S> float host_load(S v) { return (float)v; }
template <> float host_load<__half>(__half v) { return __half2float(v) * (1.0f / 16384.0f); }
template <typename S> S host_store(float v) { return S(v); }
template <> __half host_store<__half>(float v) { return __float2half_rn(v * 16384.0f); }

// Rebuild full population sets on the host from reduced-precision storage:
// f_q and g_q - w_q (3 p_hat + s_q(u^n)) stored for q = 1..8, u^n in the
// u^{n-1} slot; f_0, g_0 from the moments (phi_bar = phi of the previous
// step + dbar).
template <typename T, typename S>
lbm_status decode_mixed(lbm_handle *h, double *f, double *g)
{
    const size_t n = (size_t)h->N;
    std::vector<S> fs(9 * n), gs(9 * n);
    std::vector<T> pb(n), db(n), ph(n), u0(n), u1(n);
    CK(h, cudaMemcpyAsync(u0.data(), h->ux[1 - h->ucur], n * sizeof(T), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaMemcpyAsync(u1.data(), h->uy[1 - h->ucur], n * sizeof(T), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaMemcpyAsync(fs.data(), h->f[h->cur], 9 * n * sizeof(S), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaMemcpyAsync(gs.data(), h->g[h->cur], 9 * n * sizeof(S), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaMemcpyAsync(pb.data(), h->phi[1 - h->pcur], n * sizeof(T), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaMemcpyAsync(db.data(), h->dbar[h->acur], n * sizeof(T), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaMemcpyAsync(ph.data(), h->phat[h->acur], n * sizeof(T), cudaMemcpyDeviceToHost, h->stream), "state");
    CK(h, cudaStreamSynchronize(h->stream), "state sync");
    for (size_t k = 0; k < n; ++k) pb[k] += db[k];
    for (size_t k = 0; k < n; ++k) {
        T sf = T(0), sg = T(0);
        for (int q = 1; q < 9; ++q) {
            const T fq = (T)host_load<S>(fs[q * n + k]);
            const T gq = (T)host_load<S>(gs[q * n + k]) + (T)(float)kW[q] * (T(3) * ph[k] + s_eq(q, u0[k], u1[k]));
            if (f) f[q * n + k] = fq;
            if (g) g[q * n + k] = gq;
            sf += fq;
            sg += gq;
        }
        if (f) f[k] = pb[k] - sf;
        if (g) g[k] = T(3) * ph[k] - sg;
    }
    return LBM_OK;
}

// The stored populations are collided next against phi (given to both phi
// slots), so their sum enters as dbar = sum f - phi; g is stored less its
// equilibrium at (p_hat, u^{n-1} of the state), the velocity the next step
// adds back.
template <typename T, typename S>
lbm_status encode_mixed(lbm_handle *h, const double *f, const double *g, const double *phi, const double *upx,
                        const double *upy)
{
    const size_t n = (size_t)h->N;
    std::vector<S> fs(9 * n), gs(9 * n);
    std::vector<T> pb(n), ph(n);
    for (size_t k = 0; k < n; ++k) {
        T sf = T(0), sg = T(0);
        for (int q = 0; q < 9; ++q) {
            sf += (T)f[q * n + k];
            sg += (T)g[q * n + k];
        }
        pb[k] = sf - (T)phi[k];
        ph[k] = sg * T(1.0 / 3.0);
        fs[k] = host_store<S>(0.0f);
        gs[k] = host_store<S>(0.0f);
        for (int q = 1; q < 9; ++q) {
            fs[q * n + k] = host_store<S>((float)f[q * n + k]);
            gs[q * n + k] = host_store<S>(
                (float)((T)g[q * n + k] - (T)(float)kW[q] * (T(3) * ph[k] + s_eq(q, (T)upx[k], (T)upy[k]))));
        }
    }
    CK(h, cudaMemcpyAsync(h->f[0], fs.data(), 9 * n * sizeof(S), cudaMemcpyHostToDevice, h->stream), "state");
    CK(h, cudaMemcpyAsync(h->g[0], gs.data(), 9 * n * sizeof(S), cudaMemcpyHostToDevice, h->stream), "state");
    CK(h, cudaMemcpyAsync(h->dbar[0], pb.data(), n * sizeof(T), cudaMemcpyHostToDevice, h->stream), "state");
    CK(h, cudaMemcpyAsync(h->phat[0], ph.data(), n * sizeof(T), cudaMemcpyHostToDevice, h->stream), "state");
    CK(h, cudaStreamSynchronize(h->stream), "state sync");
    return LBM_OK;
}

template <typename T, typename S>
lbm_status get_state_impl(lbm_handle *h, double *f, double *g, double *phi, double *p, double *ux, double *uy,
                          double *uhx, double *uhy, double *upx, double *upy)
{
    lbm_status st;
    const size_t n = (size_t)h->N;
    if (Mixed<T, S>::on) {
        if ((st = decode_mixed<T, S>(h, f, g))) return st;
    } else {
        if ((st = download_field<S>(h, f, h->f[h->cur], 9 * n))) return st;
        if ((st = download_field<S>(h, g, h->g[h->cur], 9 * n))) return st;
    }
    if ((st = fields_impl<T>(h, phi, p, ux, uy))) return st;
    if ((st = download_field<T>(h, uhx, h->uhx, n))) return st;
    if ((st = download_field<T>(h, uhy, h->uhy, n))) return st;
    if ((st = download_field<T>(h, upx, h->ux[1 - h->ucur], n))) return st;
    if ((st = download_field<T>(h, upy, h->uy[1 - h->ucur], n))) return st;
    return LBM_OK;
}

template <typename T, typename S>
lbm_status set_state_impl(lbm_handle *h, const double *f, const double *g, const double *phi, const double *p,
                          const double *ux, const double *uy, const double *uhx, const double *uhy,
                          const double *upx, const double *upy)
{
    lbm_status st;
    const size_t n = (size_t)h->N;
    h->cur = 0;
    h->ucur = 0;
    h->acur = 0;
    if (Mixed<T, S>::on) {
        if ((st = encode_mixed<T, S>(h, f, g, phi, upx, upy))) return st;
    } else {
        for (int q = 0; q < 9; ++q) {
            if ((st = upload_field<S>(h, (S *)h->f[0] + q * n, f + q * n))) return st;
            if ((st = upload_field<S>(h, (S *)h->g[0] + q * n, g + q * n))) return st;
        }
    }
    h->pcur = 0;
    if constexpr (sizeof(T) == sizeof(double)) {
        if ((st = upload_field<T>(h, h->phi[0], phi))) return st;
    } else {   // phi_hi + phi_lo
        std::vector<float> hi(n), lo(n);
        for (size_t k = 0; k < n; ++k) {
            hi[k] = (float)phi[k];
            lo[k] = (float)(phi[k] - (double)hi[k]);
        }
        CK(h, cudaMemcpyAsync(h->phi[0], hi.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream), "upload");
        CK(h, cudaMemcpyAsync(h->philo, lo.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream), "upload");
        CK(h, cudaStreamSynchronize(h->stream), "upload sync");
    }
    CK(h, cudaMemcpyAsync(h->phi[1], h->phi[0], sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream), "set_state copy");
    if ((st = upload_field<T>(h, h->pf, p))) return st;
    if ((st = upload_field<T>(h, h->ux[0], ux))) return st;
    if ((st = upload_field<T>(h, h->uy[0], uy))) return st;
    if ((st = upload_field<T>(h, h->uhx, uhx))) return st;
    if ((st = upload_field<T>(h, h->uhy, uhy))) return st;
    if ((st = upload_field<T>(h, h->ux[1], upx))) return st;
    if ((st = upload_field<T>(h, h->uy[1], upy))) return st;
    CK(h, cudaStreamSynchronize(h->stream), "set_state sync");
    h->chk_pending = false;
    h->chk_status = LBM_OK;
    h->chk_count = 0;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_internal_poll_device_error(lbm_handle *h)
{
    unsigned derr = 0;
    CK(h, cudaMemcpy(&derr, h->dev_err, sizeof derr, cudaMemcpyDeviceToHost), "read device error word");
    if (derr) h->failed = true;
    if (h->failed)
        return fail(h, LBM_ERR_CUDA, "a kernel gave up a bounded wait for a TMA tile copy; its tile was not "
                                     "updated and a late copy may still write shared memory: destroy the handle");
    return LBM_OK;
}

lbm_status lbm_internal_step(lbm_handle *h)
{
    if (h->failed) return fail(h, LBM_ERR_STATE, "an earlier step gave up a tile-copy wait: destroy the handle");
    h->fresh_init = false;
    return dispatch(h->grid.precision, [&](auto tp, auto sp) {
        TS_TYPES(tp, sp);
        return step_impl<T, S>(h);
    });
}

extern "C" {

lbm_status lbm_create(const lbm_grid *grid, const lbm_params *params, const double *phi0, const double *p0,
                      const double *ux0, const double *uy0, void *stream, lbm_handle **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out must be non-NULL");
    *out = nullptr;
    lbm_status st = validate(grid, params);
    if (st) return st;
    if (!phi0 || !p0 || !ux0 || !uy0) return fail(nullptr, LBM_ERR_ARG, "initial fields must be non-NULL");
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    h->grid = *grid;
    h->prm = *params;
    h->stream = (cudaStream_t)stream;
    h->N = (long long)grid->nx * grid->ny;
    const bool dbl = grid->precision == LBM_FP64;
    h->elem = dbl ? sizeof(double) : sizeof(float);
    h->pop_elem = grid->precision >= LBM_MIX_BF16 ? 2 : h->elem;
    if (dbl) build_kp<double>(*grid, *params, h->kpd);
    else build_kp<float>(*grid, *params, h->kpf);

    // one arena: 2x9 f planes, 2x9 g planes, then the scalar planes, 256-byte aligned each
    const size_t plane = round_up((size_t)h->N * h->elem, 256);
    const size_t pplane = round_up((size_t)h->N * 9 * h->pop_elem, 256);
    const int nscalar = 22;   // phi[2], philo, pf, ux[2], uy[2], uhx, uhy, dbar[2], phat[2], jx, jy, s1, s2, tk[2][2]
    h->diag_blocks = std::min(grid->ny, DIAG_MAX_BLOCKS);   // blocks of the diagnostics sums; the partials they write
    const size_t diag_bytes = round_up(sizeof(double) * (size_t)(h->diag_blocks + 1) * NDIAG, 256);
    h->arena_bytes = 4 * pplane + nscalar * plane + diag_bytes + 256;   // + the device error word
    cudaError_t e = cudaMalloc((void **)&h->arena, h->arena_bytes);
    if (e != cudaSuccess) {
        std::string m = std::string("cudaMalloc arena: ") + cudaGetErrorString(e);
        delete h;
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
    }
    unsigned char *a = h->arena;
    h->f[0] = a; a += pplane;
    h->f[1] = a; a += pplane;
    h->g[0] = a; a += pplane;
    h->g[1] = a; a += pplane;
    void **sc[] = {&h->phi[0], &h->phi[1], &h->philo, &h->pf, &h->ux[0], &h->ux[1], &h->uy[0], &h->uy[1], &h->uhx, &h->uhy,
                   &h->dbar[0], &h->dbar[1], &h->phat[0], &h->phat[1], &h->jx, &h->jy, &h->s1, &h->s2,
                   &h->tk[0][0], &h->tk[0][1], &h->tk[1][0], &h->tk[1][1]};
    static_assert(sizeof(sc) / sizeof(sc[0]) == 22, "one plane per scalar field of the arena");
    for (void **pp : sc) { *pp = a; a += plane; }
    h->diag_part = (double *)a;
    h->diag_out = h->diag_part + (size_t)h->diag_blocks * NDIAG;
    h->dev_err = (unsigned *)(h->arena + h->arena_bytes - 256);
    h->tma = grid->precision != LBM_FP64 && grid->nx % 4 == 0;
    e = cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned), h->stream);
    if (e != cudaSuccess) {
        std::string m = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
        cudaFree(h->arena);
        delete h;
        cudaGetLastError();
        return fail(nullptr, LBM_ERR_CUDA, m);
    }

    st = dispatch(grid->precision, [&](auto tp, auto sp) {
        TS_TYPES(tp, sp);
        lbm_status r = set_smem_limits<T, S>(h);
        return r ? r : init_impl<T, S>(h, phi0, p0, ux0, uy0);
    });
    if (st) {
        g_create_error = h->err;
        lbm_destroy(h);
        return st;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle *h, int n)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (n < 0) return fail(h, LBM_ERR_ARG, "n must be >= 0");
    if (h->failed) return fail(h, LBM_ERR_STATE, "an earlier step gave up a tile-copy wait: destroy the handle");
    if (h->chk_pending && cudaEventQuery(h->chk_ev) == cudaSuccess) {   // never waits
        h->chk_pending = false;
        const double *d = h->chk_host;
        if (d[10] > 0) h->chk_status = LBM_ERR_NONFINITE;
        else if (d[8] > 1.0 + h->chk_delta || d[9] < -1.0 - h->chk_delta) h->chk_status = LBM_ERR_RANGE;
    }
    if (h->chk_status == LBM_ERR_NONFINITE) return fail(h, h->chk_status, "periodic check: non-finite field value");
    if (h->chk_status == LBM_ERR_RANGE) return fail(h, h->chk_status, "periodic check: phi outside [-1-delta, 1+delta]");
    if (n > 0) h->fresh_init = false;
    struct Chain {   // timed launches share boundary events only inside this call
        lbm_handle *h;
        explicit Chain(lbm_handle *h_) : h(h_) { h->chain = nullptr; h->chain_ok = true; }
        ~Chain() { h->chain = nullptr; h->chain_ok = false; }
    } chain(h);
    return dispatch(h->grid.precision, [&](auto tp, auto sp) {
        TS_TYPES(tp, sp);
        for (int t = 0; t < n; ++t) {
            lbm_status st = step_impl<T, S>(h);
            if (st) return st;
            if (h->chk_every > 0 && ++h->chk_count % h->chk_every == 0 && !h->chk_pending) {
                st = diag_impl<T>(h, h->chk_host, false);
                if (st) return st;
                CK(h, cudaEventRecord(h->chk_ev, h->stream), "check event");
                h->chk_pending = true;
                h->chain = nullptr;
            }
        }
        return LBM_OK;
    });
}

lbm_status lbm_step_ch(lbm_handle *h, int n, const double *ux, const double *uy, const double *tfac)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (n < 0) return fail(h, LBM_ERR_ARG, "n must be >= 0");
    if (!ux || !uy) return fail(h, LBM_ERR_ARG, "ux, uy must be non-NULL");
    if (h->grid.precision != LBM_FP64 && h->grid.precision != LBM_FP32)
        return fail(h, LBM_ERR_ARG, "the Cahn-Hilliard-only step needs FP64 or FP32 populations");
    if (h->failed) return fail(h, LBM_ERR_STATE, "an earlier step gave up a tile-copy wait: destroy the handle");
    if (n > 0) h->fresh_init = false;
    return h->grid.precision == LBM_FP64 ? step_ch_impl<double>(h, n, ux, uy, tfac)
                                         : step_ch_impl<float>(h, n, ux, uy, tfac);
}

lbm_status lbm_set_check(lbm_handle *h, int every, double delta)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (every < 0 || !(delta >= 0)) return fail(h, LBM_ERR_ARG, "every must be >= 0 and delta >= 0");
    if (every > 0 && !h->chk_host) {
        CK(h, cudaMallocHost((void **)&h->chk_host, sizeof(double) * NDIAG), "cudaMallocHost(check)");
        CK(h, cudaEventCreateWithFlags(&h->chk_ev, cudaEventDisableTiming), "cudaEventCreate(check)");
    }
    h->chk_every = every;
    h->chk_delta = delta;
    h->chk_count = 0;
    return LBM_OK;
}

lbm_status lbm_fields(lbm_handle *h, double *phi, double *p, double *ux, double *uy)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    lbm_status st =
        h->grid.precision == LBM_FP64 ? fields_impl<double>(h, phi, p, ux, uy) : fields_impl<float>(h, phi, p, ux, uy);
    return st ? st : lbm_internal_poll_device_error(h);
}

lbm_status lbm_dynamic_pressure(lbm_handle *h, double *pd)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!pd) return fail(h, LBM_ERR_ARG, "pd must be non-NULL");
    lbm_status st = h->grid.precision == LBM_FP64 ? dynamic_pressure_impl<double>(h, pd)
                                                  : dynamic_pressure_impl<float>(h, pd);
    return st ? st : lbm_internal_poll_device_error(h);
}

lbm_status lbm_fields_device(lbm_handle *h, void *phi, void *p, void *ux, void *uy, int dtype)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    const bool dbl = h->grid.precision == LBM_FP64;
    if (dtype != (dbl ? 0 : 1))
        return fail(h, LBM_ERR_ARG, "dtype must match the handle's arithmetic type (0 double, 1 float)");
    const size_t b = h->elem * (size_t)h->N;
    void *dst[4] = {phi, p, ux, uy};
    const void *src[4] = {phi_cur(h), h->pf, h->ux[h->ucur], h->uy[h->ucur]};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) CK(h, cudaMemcpyAsync(dst[k], src[k], b, cudaMemcpyDeviceToDevice, h->stream), "fields_device");
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_handle *h, const double *phi0, const double *p0, const double *ux0, const double *uy0)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!phi0 || !p0 || !ux0 || !uy0) return fail(h, LBM_ERR_ARG, "fields must be non-NULL");
    return dispatch(h->grid.precision, [&](auto tp, auto sp) {
        TS_TYPES(tp, sp);
        return init_impl<T, S>(h, phi0, p0, ux0, uy0);
    });
}

lbm_status lbm_diagnostics(lbm_handle *h, double *out)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!out) return fail(h, LBM_ERR_ARG, "out must be non-NULL");
    lbm_status st = h->grid.precision == LBM_FP64 ? diag_impl<double>(h, out) : diag_impl<float>(h, out);
    return st ? st : lbm_internal_poll_device_error(h);
}

lbm_status lbm_diagnostics_async(lbm_handle *h, double *out)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (!out) return fail(h, LBM_ERR_ARG, "out must be non-NULL");
    return h->grid.precision == LBM_FP64 ? diag_impl<double>(h, out, false) : diag_impl<float>(h, out, false);
}

lbm_status lbm_check(lbm_handle *h, double delta)
{
    double d[NDIAG];
    lbm_status st = lbm_diagnostics(h, d);   // includes the device error word
    if (st) return st;
    if (d[10] > 0) return fail(h, LBM_ERR_NONFINITE, "non-finite field value");
    if (d[8] > 1.0 + delta || d[9] < -1.0 - delta) return fail(h, LBM_ERR_RANGE, "phi outside [-1-delta, 1+delta]");
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_handle *h, double *f, double *g, double *phi, double *p, double *ux, double *uy,
                         double *uhx, double *uhy, double *upx, double *upy)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    lbm_status st = dispatch(h->grid.precision, [&](auto tp, auto sp) {
        TS_TYPES(tp, sp);
        return get_state_impl<T, S>(h, f, g, phi, p, ux, uy, uhx, uhy, upx, upy);
    });
    return st ? st : lbm_internal_poll_device_error(h);
}

lbm_status lbm_set_state(lbm_handle *h, const double *f, const double *g, const double *phi, const double *p,
                         const double *ux, const double *uy, const double *uhx, const double *uhy,
                         const double *upx, const double *upy)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    const double *all[10] = {f, g, phi, p, ux, uy, uhx, uhy, upx, upy};
    for (const double *q : all)
        if (!q) return fail(h, LBM_ERR_ARG, "every state array must be non-NULL");
    h->fresh_init = false;
    return dispatch(h->grid.precision, [&](auto tp, auto sp) {
        TS_TYPES(tp, sp);
        return set_state_impl<T, S>(h, f, g, phi, p, ux, uy, uhx, uhy, upx, upy);
    });
}

lbm_status lbm_profile(lbm_handle *h, int on)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    if (on) {
        CK(h, cudaStreamSynchronize(h->stream), "profile sync");
        for (auto &m : h->marks) {
            if (m.own_a) h->pool.push_back(m.a);
            h->pool.push_back(m.b);
        }
        h->marks.clear();
        h->chain = nullptr;
        for (int k = 0; k < LBM_NKERNELS; ++k) { h->prof_ms[k] = 0.0; h->prof_n[k] = 0; }
    }
    h->prof = on != 0;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_handle *h, double *ms, long long *launches)
{
    if (!h) return fail(nullptr, LBM_ERR_ARG, "NULL handle");
    CK(h, cudaStreamSynchronize(h->stream), "profile sync");
    for (auto &m : h->marks) {
        float t = 0.f;
        CK(h, cudaEventElapsedTime(&t, m.a, m.b), "cudaEventElapsedTime");
        h->prof_ms[m.kind] += t;
        h->prof_n[m.kind] += 1;
        if (m.own_a) h->pool.push_back(m.a);
        h->pool.push_back(m.b);
    }
    h->marks.clear();
    h->chain = nullptr;
    for (int k = 0; k < LBM_NKERNELS; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->prof_n[k];
    }
    return LBM_OK;
}

unsigned long long lbm_debug_violations(void)
{
#ifdef LBM_DEBUG
    unsigned long long v = 0, z = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return ~0ull;
    if (cudaMemcpyFromSymbol(&v, g_lbm_debug, sizeof v) != cudaSuccess) return ~0ull;
    cudaMemcpyToSymbol(g_lbm_debug, &z, sizeof z);
    return v;
#else
    return 0;
#endif
}

const char *lbm_kernel_name(int kind)
{
    static const char *names[LBM_NKERNELS] = {"k_collide_stream", "k_rk_stage", "k_picard", "k_filter"};
    return (kind >= 0 && kind < LBM_NKERNELS) ? names[kind] : "unknown";
}

const char *lbm_kernel_variant(const lbm_handle *h, int kind)
{
    if (!h || kind < 0 || kind >= LBM_NKERNELS) return "unknown";
    const bool f32 = h->grid.precision != LBM_FP64, even = h->grid.nx % 2 == 0;
    switch (kind) {
    case 0:
        return (f32 && h->tma && h->grid.periodic_x && default_rates(h->prm)) ? "k_collide_pairs" : "k_collide_stream";
    case 1: return f32 && h->tma ? "k_rk_tma" : (f32 && even ? "k_rk_strips" : "k_rk_stage");
    case 2:
        if (h->prm.flags & LBM_FLAG_STRAIN_MOMENTS) return "k_picard";
        return f32 && h->tma ? "k_picard_tma" : (f32 && even ? "k_picard_strips" : "k_picard");
    default:
        if (h->prm.filter_order == 0) return "none";
        return f32 && h->tma ? "k_filter_tma" : (f32 && even ? "k_filter_strips" : "k_filter");
    }
}

size_t lbm_device_bytes(const lbm_handle *h) { return h ? h->arena_bytes : 0; }

void lbm_destroy(lbm_handle *h)
{
    if (!h) return;
    lbm_internal_adjoint_free(h);
    for (auto &m : h->marks) {
        if (m.own_a) cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    if (h->chk_ev) cudaEventDestroy(h->chk_ev);
    if (h->chk_host) cudaFreeHost(h->chk_host);
    if (h->arena) cudaFree(h->arena);
    delete h;
}

const char *lbm_last_error(const lbm_handle *h)
{
    if (h) return h->err.c_str();
    return g_create_error.c_str();
}

}  // extern "C"
