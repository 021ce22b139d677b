// mlp_tc.cuh -- the closure network on the fifth-generation tensor cores: tcgen05.mma with
// operands in shared memory (no-swizzle K-major core-matrix layout) and FP32 accumulators in
// tensor memory (TMEM), read back with tcgen05.ld.  One tile = 128 cells (rows): the MMA has
// M = 128 and row m of the accumulator is TMEM lane m, so the warp w of a 128-thread group
// owns TMEM lanes 32 w .. 32 w + 31, the accumulators of its own 32 cells.
//   layer 1: D1[128 x 32] = X[128 x 16] W1h^T      (one MMA, K = 16)
//   layer 2: D2[128 x 32] = H1[128 x 32] W2h^T     (two MMAs, K = 2 x 16)
//   output : y = b3 + w3 . H2 on the CUDA cores (32 FP32 FMAs per cell)
// with W1h, W2h, b1h, b2h the halved weights of MlpDev (the SiLU is taken from z/2).
// Every wait on an mbarrier is bounded; a wait that gives up sets *err and the caller skips
// the rest of the tile (its outputs are then undefined, the status tells the host).
#pragma once

#include <cstdint>

namespace lbm {
namespace tc {

// ---- PTX wrappers -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Allocate `ncols` TMEM columns for the CTA (one full warp executes it); the address lands in *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait for phase `parity` of the mbarrier to complete, at most `limit` polls.  False: gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Generic-proxy writes to shared memory become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[taddr] (+)= A B, A and B from shared-memory descriptors, BF16 x BF16 -> FP32 (kind::f16).
__device__ __forceinline__ void mma_f16(uint32_t d_taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_taddr),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier when all tcgen05.mma issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- descriptors --------------------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle: start address, LBO = byte stride between core
// matrices adjacent along K, SBO = byte stride between adjacent 8-row groups (M or N); bits
// 46-47 hold the descriptor version (1).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t m, uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major BF16 operand in the no-swizzle core-matrix
// layout with `kchunks` chunks of 8 elements along K: 8-row groups are kchunks x 128 B apart,
// core matrices adjacent along K 128 B apart, rows of a core matrix 16 B apart.
__host__ __device__ constexpr uint32_t core_off(uint32_t row, uint32_t k, uint32_t kchunks)
{
    return ((row >> 3) * kchunks + (k >> 3)) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

#ifndef LBM_TC_LBO_IS_K
#define LBM_TC_LBO_IS_K 1
#endif
// (LBO, SBO) of an operand with `kchunks` K-chunks.
__device__ __forceinline__ uint64_t operand_desc(uint32_t saddr, uint32_t kchunks)
{
#if LBM_TC_LBO_IS_K
    return sdesc(saddr, 128u, kchunks * 128u);
#else
    return sdesc(saddr, kchunks * 128u, 128u);
#endif
}

// Shared memory of one 128-row tile of the tensor-core network.
struct __align__(1024) TcSmem {
    unsigned char a1[128 * 16 * 2];  // X, 128 x 16 BF16 (2 K-chunks)
    unsigned char a2[128 * 32 * 2];  // H1, 128 x 32 BF16 (4 K-chunks)
    unsigned char b1[32 * 16 * 2];   // W1h, 32 x 16 BF16
    unsigned char b2[32 * 32 * 2];   // W2h, 32 x 32 BF16
    float bias1[32], bias2[32], w3[32];
    uint64_t bar;
    uint32_t tmem;
};

// Shared memory of a 256-row tile (two M = 128 halves; TMEM columns 0-31 / 32-63 hold the
// layer-1 accumulators of rows 0-127 / 128-255, columns 64-95 / 96-127 those of layer 2).
struct __align__(1024) TcSmem256 {
    unsigned char a1[256 * 16 * 2];
    unsigned char a2[256 * 32 * 2];
    unsigned char b1[32 * 16 * 2];
    unsigned char b2[32 * 32 * 2];
    float bias1[32], bias2[32], w3[32];
    uint64_t bar;
    uint32_t tmem;
};

// Stage the weights of the device-form network P into the tile's operand layout (all threads
// of the CTA; caller syncs).
template <class SM, class MLP>
__device__ __forceinline__ void stage_weights(SM &S, const MLP &P)
{
    for (int e = threadIdx.x; e < 32 * 16; e += blockDim.x) {
        const int n = e >> 4, k = e & 15;
        *reinterpret_cast<__nv_bfloat16 *>(S.b1 + core_off(n, k, 2)) = P.w1[n][k];
    }
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int n = e >> 5, k = e & 31;
        *reinterpret_cast<__nv_bfloat16 *>(S.b2 + core_off(n, k, 4)) = P.w2[n][k];
    }
    for (int j = threadIdx.x; j < 32; j += blockDim.x) {
        S.bias1[j] = P.b1[j];
        S.bias2[j] = P.b2[j];
        S.w3[j] = __bfloat162float(P.w3[0][j]);
    }
}

}  // namespace tc
}  // namespace lbm
