// diag.cu -- second pass of the step diagnostics and of the per-block reduction: the sweep
// (or k_reduce_tiles) writes one record of 8 partial sums per CTA (tile); one CTA adds up the
// records of the whole domain, or one CTA per block those of its tiles, in a fixed order, so
// the result is the same from run to run.  Record: mass, momentum x/y/z, kinetic energy, max |u| (max, not sum),
// non-finite cells, fluid cells.
#include "launch.hpp"
#include "mlp_tc.cuh"

namespace lbm {
namespace {

__device__ __forceinline__ double dsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double dmax(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Fixed-order sum of n records into out[8] by the calling CTA (at most 256 threads): each
// thread sums its records, then warp 0 alone sums the threads' sums (lane j takes threads j,
// j + 32, ...) and shuffles.  The FP64 pipe of this GPU retires 2 lanes per clock per SM, so
// warp-wide FP64 shuffles in every warp would cost more than the sums themselves.
__device__ __forceinline__ void final_sum(const double *__restrict__ partials, int64_t n, double *__restrict__ out)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x)
        for (int c = 0; c < 8; ++c) acc[c] = c == 5 ? fmax(acc[c], partials[p * 8 + c]) : acc[c] + partials[p * 8 + c];
    __shared__ double sh[8][256];
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, nt = (int)blockDim.x;
        for (int c = 0; c < 8; ++c) {
            double v = 0.0;
            for (int j = lane; j < nt; j += 32) v = c == 5 ? fmax(v, sh[c][j]) : v + sh[c][j];
            v = c == 5 ? dmax(v) : dsum(v);
            if (lane == 0) out[c] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_diag_final(const double *__restrict__ partials, int64_t n, double *__restrict__ out)
{
    final_sum(partials, n, out);
}

// The same sum written straight into a page-locked host slot (its device address), with the
// bounded-wait status flags beside it, so that reading a step's record needs no copy.
__global__ void __launch_bounds__(256) k_diag_final_slot(const double *__restrict__ partials, int64_t n,
                                                         double *__restrict__ slot, int *__restrict__ slot_err,
                                                         const int *__restrict__ err0, const int *__restrict__ err1)
{
    __shared__ double res[8];
    final_sum(partials, n, res);
    __syncthreads();
    if (threadIdx.x < 8) slot[threadIdx.x] = res[threadIdx.x];
    if (threadIdx.x == 8) slot_err[0] = err0 ? *(const volatile int *)err0 : 0;
    if (threadIdx.x == 9) slot_err[1] = err1 ? *(const volatile int *)err1 : 0;
}

// Per block: CTA b sums the records of tiles start[b] .. start[b+1] - 1 into out[8 b ..].
__global__ void __launch_bounds__(256) k_block_final(const double *__restrict__ partials,
                                                     const int64_t *__restrict__ start, double *__restrict__ out)
{
    const int64_t b = blockIdx.x;
    final_sum(partials + start[b] * 8, start[b + 1] - start[b], out + b * 8);
}

}  // namespace

// Records per CTA of the first level of the two-level sum (a fixed partition of the records).
constexpr int64_t kChunk = 256;

__global__ void __launch_bounds__(256) k_diag_chunks(const double *__restrict__ partials, int64_t n,
                                                     double *__restrict__ out)
{
    const int64_t c0 = (int64_t)blockIdx.x * kChunk;
    final_sum(partials + c0 * 8, min(kChunk, n - c0), out + (int64_t)blockIdx.x * 8);
}

cudaError_t launch_reduce_final(const double *partials, int64_t n, double *out, cudaStream_t s)
{
    // up to kChunk records: one CTA; more: one CTA per chunk of kChunk records into a scratch
    // area after the output (out[8 ..]), then one CTA over the chunk records.  The partition
    // depends on n only, so the result is the same from run to run.
    if (n <= kChunk) {
        k_diag_final<<<1, 256, 0, s>>>(partials, n, out);
        return cudaGetLastError();
    }
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    if (chunks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_diag_chunks<<<(unsigned)chunks, 256, 0, s>>>(partials, n, out + 8);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, 256, 0, s>>>(out + 8, chunks, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_final_slot(const double *partials, int64_t n, double *scratch, double *slot, int *slot_err,
                                     const int *err0, const int *err1, cudaStream_t s)
{
    // the partition of launch_reduce_final: the same result bits
    if (n <= kChunk) {
        k_diag_final_slot<<<1, 256, 0, s>>>(partials, n, slot, slot_err, err0, err1);
        return cudaGetLastError();
    }
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    if (chunks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_diag_chunks<<<(unsigned)chunks, 256, 0, s>>>(partials, n, scratch + 8);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final_slot<<<1, 256, 0, s>>>(scratch + 8, chunks, slot, slot_err, err0, err1);
    return cudaGetLastError();
}

int64_t reduce_final_scratch(int64_t n) { return n <= kChunk ? 8 : 8 + 8 * ((n + kChunk - 1) / kChunk); }

cudaError_t launch_block_final(const double *partials, const int64_t *start, int64_t nblocks, double *out,
                               cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_block_final<<<(unsigned)nblocks, 256, 0, s>>>(partials, start, out);
    return cudaGetLastError();
}

namespace {
// One thread waits, at most `polls` polls, on an mbarrier nothing arrives on (phase 0 of a
// barrier initialised for one arrival), gives up and records value 2 in *err: the path a
// staged sweep takes when its bounded wait runs out, without any copy in flight.
__global__ void k_wait_selfcheck(int *err, uint32_t polls)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!tc::mbar_wait(&bar, 0, polls)) atomicExch(err, 2);
}
}  // namespace

cudaError_t launch_wait_selfcheck(int *err, uint32_t polls, cudaStream_t s)
{
    k_wait_selfcheck<<<1, 32, 0, s>>>(err, polls);
    return cudaGetLastError();
}

}  // namespace lbm
