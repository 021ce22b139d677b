// reduce_static.cu -- allocation-free variant of the diagnostics reduction.
//
// Some callers cannot call cudaMalloc: code that hands all device memory out of its own
// pool (a framework's caching allocator, a fixed arena sized at start-up), or code on a
// path where an allocation is not allowed because cudaMalloc/cudaFree may synchronise the
// device or fail mid-run.  lbm_reduce_noalloc gives them the same diagnostics as
// lbm_reduce for a PDF field they own, without any allocation: the per-CTA partial sums
// live in a fixed, file-scope device array of LBM_REDUCE_NOALLOC_MAX_CELLS / 4096 records
// (2 MiB), which every GPU that loads this library keeps until the process exits.
//
// Kernels: the same per-cell FP64 moments as the context's reduction (sum f, sum c f - F/2,
// kinetic energy, max speed, non-finite count), 4096 cells per CTA (256 threads x 16 cells,
// coalesced), warp-shuffle + shared-memory block sums into one record per CTA, then one CTA
// sums the records in a fixed order: the result is deterministic.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"
#include "kernels.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int64_t kCellsPerCta = (int64_t)kThreads * kCellsPerThread;
constexpr int kMaxCtas = (int)(LBM_REDUCE_NOALLOC_MAX_CELLS / kCellsPerCta);  // 32768 records
constexpr int kMaxDevices = 64;

static_assert((int64_t)kMaxCtas * kCellsPerCta == LBM_REDUCE_NOALLOC_MAX_CELLS, "limit must be a whole number of CTAs");

// Scratch: 8 doubles per CTA record.  Shared by every call; each call writes every record it
// reads before reading it, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[kMaxCtas * 8];

// Device address of g_noalloc_partials per device, looked up once with that device current.
std::mutex g_mutex;
double *g_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double wsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double wmax(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int Q, class T>
__global__ void __launch_bounds__(kThreads) k_noalloc_cells(const T *__restrict__ f, int64_t N, double Fx, double Fy,
                                                            double Fz, double *__restrict__ partials)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const double F[3] = {Fx, Fy, Fz};
    const int64_t base = (int64_t)blockIdx.x * kCellsPerCta + threadIdx.x;
    for (int k = 0; k < kCellsPerThread; ++k) {
        const int64_t n = base + (int64_t)k * kThreads;
        if (n >= N) break;
        double v[Q];
        bool finite = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            v[i] = (double)f[(int64_t)i * N + n];
            finite = finite && isfinite(v[i]);
        }
        double rho, j[3];
        lbm::moments_post<Q>(v, F, rho, j);
        const double j2 = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
        acc[0] += rho;
        acc[1] += j[0];
        acc[2] += j[1];
        acc[3] += j[2];
        acc[4] += 0.5 * j2 / rho;
        acc[5] = fmax(acc[5], sqrt(j2) / rho);
        acc[6] += finite ? 0.0 : 1.0;
        acc[7] += 1.0;
    }
    __shared__ double sh[kThreads / 32][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const double r = c == 5 ? wmax(acc[c]) : wsum(acc[c]);
        if (lane == 0) sh[warp][c] = r;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int c = threadIdx.x;
        double r = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) r = c == 5 ? fmax(r, sh[w][c]) : r + sh[w][c];
        partials[(int64_t)blockIdx.x * 8 + c] = r;
    }
}

__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double *__restrict__ partials, int n,
                                                            double *__restrict__ out)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < n; p += kThreads)
        for (int c = 0; c < 8; ++c) acc[c] = c == 5 ? fmax(acc[c], partials[(int64_t)p * 8 + c]) : acc[c] + partials[(int64_t)p * 8 + c];
    __shared__ double sh[kThreads / 32][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const double r = c == 5 ? wmax(acc[c]) : wsum(acc[c]);
        if (lane == 0) sh[warp][c] = r;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int c = threadIdx.x;
        double r = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) r = c == 5 ? fmax(r, sh[w][c]) : r + sh[w][c];
        out[c] = r;
    }
}

// Device address of the scratch array on the current device (first call per device looks
// it up with cudaGetSymbolAddress).
cudaError_t scratch_address(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

template <int Q, class T>
cudaError_t launch(const void *f, int64_t n, const double F[3], double *scratch, double *out, cudaStream_t s)
{
    const int ctas = (int)((n + kCellsPerCta - 1) / kCellsPerCta);
    k_noalloc_cells<Q, T><<<ctas, kThreads, 0, s>>>((const T *)f, n, F[0], F[1], F[2], scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_noalloc_final<<<1, kThreads, 0, s>>>(scratch, ctas, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" lbm_status lbm_reduce_noalloc(const void *f_dev, int32_t stencil, int32_t storage, int64_t ncells,
                                         const double force[3], double *out_dev, void *cuda_stream)
{
    if (!f_dev || !out_dev) return LBM_ERR_ARG;
    if (stencil != LBM_D3Q19 && stencil != LBM_D3Q27) return LBM_ERR_ARG;
    if (storage != LBM_FP64 && storage != LBM_FP32) return LBM_ERR_UNSUPPORTED;
    if (ncells <= 0) return LBM_ERR_ARG;
    if (ncells > LBM_REDUCE_NOALLOC_MAX_CELLS) return LBM_ERR_UNSUPPORTED;
    double F[3] = {0.0, 0.0, 0.0};
    if (force)
        for (int a = 0; a < 3; ++a) F[a] = force[a];
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LBM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (stencil == LBM_D3Q19)
        e = storage == LBM_FP64 ? launch<19, double>(f_dev, ncells, F, scratch, out_dev, s)
                                : launch<19, float>(f_dev, ncells, F, scratch, out_dev, s);
    else
        e = storage == LBM_FP64 ? launch<27, double>(f_dev, ncells, F, scratch, out_dev, s)
                                : launch<27, float>(f_dev, ncells, F, scratch, out_dev, s);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
