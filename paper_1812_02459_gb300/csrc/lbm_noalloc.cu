// lbm_noalloc.cu -- field sums that allocate no device memory.
//
// lbm_field_sums_noalloc computes the same FP64 node sums as lbm_diagnostics
// (volume, bubble centroid and rise-velocity sums, extrema, non-finite
// count) for fields the caller already holds on the device, without any
// cudaMalloc/cudaFree.  It exists for callers that cannot allocate: code
// whose device memory is owned by a host framework's own pool, loops that
// cannot afford the device-wide synchronisation cudaMalloc and cudaFree
// imply, and monitors that must keep reporting after device memory has run
// out.  Its block partial sums live in a file-scope static device array of
// fixed size, which every GPU that loads this library holds until exit.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 256LL * 64;   // nodes reduced by one block
constexpr int NA_MAX_BLOCKS = LBM_NOALLOC_MAX_NODES / (int)NA_CHUNK;

static_assert((long long)NA_MAX_BLOCKS * NA_CHUNK == LBM_NOALLOC_MAX_NODES, "chunking");

// Block partials: NA_MAX_BLOCKS x LBM_NDIAG doubles (4096 x 11 x 8 B = 352 KiB).
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS * lbm::NDIAG];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double *g_partials_ptr[MAX_DEVICES] = {};

// Each block reduces its own fixed chunk of nodes, so the summation order
// depends on nx*ny only, never on the GPU.
template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
k_sums_chunks(int nx, long long N, const T *__restrict__ phi, const T *__restrict__ p,
              const T *__restrict__ ux, const T *__restrict__ uy, double *__restrict__ part)
{
    using namespace lbm;
    double acc[NDIAG];
#pragma unroll
    for (int k = 0; k < NDIAG; ++k) acc[k] = 0.0;
    acc[8] = -INFINITY;
    acc[9] = INFINITY;
    const long long lo = blockIdx.x * NA_CHUNK;
    const long long hi = lo + NA_CHUNK < N ? lo + NA_CHUNK : N;
    for (long long k = lo + threadIdx.x; k < hi; k += NA_THREADS) {
        const double ph = (double)phi[k], v = (double)uy[k];
        const double y = (double)(k / nx);
        const double w = (1.0 - ph) * 0.5;
        acc[0] += ph;
        if (ph > 0) acc[1] += 1.0;
        if (ph < 0) { acc[2] += 1.0; acc[3] += y; acc[4] += v; }
        acc[5] += w;
        acc[6] += w * y;
        acc[7] += w * v;
        acc[8] = fmax(acc[8], ph);
        acc[9] = fmin(acc[9], ph);
        acc[10] += (double)(!isfinite(ph)) + (double)(!isfinite((double)p[k])) +
                   (double)(!isfinite((double)ux[k])) + (double)(!isfinite(v));
    }
    __shared__ double red[NDIAG][NA_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NDIAG; ++k) {
        double v = k == 8 ? warp_max(acc[k]) : (k == 9 ? warp_min(acc[k]) : warp_sum(acc[k]));
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NDIAG) {
        const int k = threadIdx.x;
        double v = red[k][0];
        for (int w = 1; w < NA_THREADS / 32; ++w)
            v = k == 8 ? fmax(v, red[k][w]) : (k == 9 ? fmin(v, red[k][w]) : v + red[k][w]);
        part[blockIdx.x * NDIAG + k] = v;   // every used slot is written before it is read
    }
}

// Address of the static partials array on the current device, looked up once.
cudaError_t partials_on_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_ptr[dev] = (double *)ptr;
    }
    *out = g_partials_ptr[dev];
    return cudaSuccess;
}

thread_local char g_err[256];

lbm_status na_fail(lbm_status st, const char *msg, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess) snprintf(g_err, sizeof g_err, "%s: %s", msg, cudaGetErrorString(e));
    else snprintf(g_err, sizeof g_err, "%s", msg);
    return st;
}

}  // namespace

extern "C" {

lbm_status lbm_field_sums_noalloc(const void *phi, const void *p, const void *ux, const void *uy,
                                  int nx, int ny, int dtype, double *out, void *stream)
{
    if (!phi || !p || !ux || !uy || !out) return na_fail(LBM_ERR_ARG, "pointers must be non-NULL");
    if (nx < 1 || ny < 1) return na_fail(LBM_ERR_ARG, "nx and ny must be >= 1");
    const long long N = (long long)nx * ny;
    if (N > LBM_NOALLOC_MAX_NODES)
        return na_fail(LBM_ERR_ARG, "nx*ny exceeds LBM_NOALLOC_MAX_NODES (67108864): the static "
                                    "scratch holds 4096 block partials of 16384 nodes");
    if (dtype != 0 && dtype != 1) return na_fail(LBM_ERR_ARG, "dtype must be 0 (double) or 1 (float)");
    double *part = nullptr;
    cudaError_t e = partials_on_current_device(&part);
    if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, "cudaGetSymbolAddress(static partials)", e);
    const int blocks = (int)((N + NA_CHUNK - 1) / NA_CHUNK);
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == 0)
        k_sums_chunks<double><<<blocks, NA_THREADS, 0, st>>>(nx, N, (const double *)phi, (const double *)p,
                                                             (const double *)ux, (const double *)uy, part);
    else
        k_sums_chunks<float><<<blocks, NA_THREADS, 0, st>>>(nx, N, (const float *)phi, (const float *)p,
                                                            (const float *)ux, (const float *)uy, part);
    lbm::k_diag_final<<<1, 32 * lbm::NDIAG, 0, st>>>(blocks, part, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, "kernel launch", e);
    return LBM_OK;
}

const char *lbm_noalloc_last_error(void) { return g_err; }

}  // extern "C"
