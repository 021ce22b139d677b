// closure.cu -- locally varying relaxation for the sweep (D3Q19, FP32 storage): the
// Smagorinsky model and the learned closure, whose 7-32-32-1 SiLU network runs on the
// tensor cores (BF16 mma.sync, FP32 accumulation) fused into the collision; plus the
// network's training kernels (forward, backward, Adam) and a standalone inference entry.
//
// The paper lets the relaxation rate vary per cell from a local fluid property, read from a
// field (Sec. 5.1.1; turbulence models after Yu et al. 2005, cited there).  Here the closure
// computes omega+ of each cell from its pre-collision state inside the sweep:
//   Pi_neq_ab = sum_i c_ia c_ib f_i - rho (delta_ab / 3 + u_a u_b)
//   Smagorinsky: tau = (tau0 + sqrt(tau0^2 + 18 cs^2 sqrt(2 Pi:Pi) / rho)) / 2
//   network:     tau = tau0 + s_tau softplus(y), y = MLP((rho - 1) s_rho, s_pi Pi_neq)
// and omega- follows from the same Lambda.  Network parameters (packed FP32, 1348 values):
//   W1[32][7], b1[32], W2[32][32], b2[32], w3[32], b3, s_rho, s_pi, s_tau
// Inference rounds the features and both hidden layers to BF16 before each product (the
// weights are BF16, sums FP32); training runs in FP32.
#define LBM_Q 19
#define LBM_ST 1
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <cstring>
#include <vector>

#include "cell.cuh"
#include "closure.hpp"
#include "lbm.h"
#include "mlp_tc.cuh"

namespace lbm {
namespace {

constexpr int kH = 32, kIn = 7, kParams = 1348;
constexpr int kOffW1 = 0, kOffB1 = kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH,
              kOffB3 = kOffW3 + kH, kOffScale = kOffB3 + 1;
static_assert(kOffScale + 3 == kParams, "packed layout");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// D (16x8, FP32) += A (16x16, BF16, row) * B (16x8, BF16, col): one warp-wide tensor-core MMA.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU of the inference path.  The device form of the network holds W1, b1, W2, b2 halved
// (exact in BF16 / FP32), so each layer's accumulator is h = z/2 and
//   SiLU(z) = z sigmoid(z) = h tanh(h) + h,
// one tanh.approx.f32 (relative error below 2^-10.9) and one FMA per unit, then the BF16
// rounding of the A fragment.  Measured on the 256^3 box against z / (1 + __expf(-z)) with
// __fdividef: 0.71 vs 0.93 ms per two-grid step; a packed tanh.approx.bf16x2 form was no
// faster (0.71 ms) and less accurate.
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float softplus(float y) { return y > 30.0f ? y : log1pf(expf(y)); }
// The sweep's softplus from the fast exponential and logarithm: its error (a few 1e-7 of the
// value, at most 2^-24 absolute where exp(y) vanishes next to 1) is far below the network's
// own (tanh.approx.f32, BF16 operands) and reaches tau scaled by s_tau.
__device__ __forceinline__ float softplus_fast(float y) { return y > 30.0f ? y : __logf(1.0f + __expf(y)); }

// SiLU of two units from their halved pre-activations h0, h1, packed as BF16 (lo = h0).
__device__ __forceinline__ uint32_t silu_pair(float h0, float h1)
{
    return pack_bf16(fmaf(h0, tanh_approx(h0), h0), fmaf(h1, tanh_approx(h1), h1));
}

// Per-warp MLP on 32 cells (one per lane): the features of all lanes form A = X (32 x 16,
// two 16-row tiles; 7 features padded with zeros); each layer is a few m16n8k16 MMAs whose
// FP32 accumulators, after bias and SiLU, are repacked in registers as the next layer's A
// fragments (the accumulator layout of two adjacent 8-column tiles is the A layout of one
// 16-column k-step).  Returns y of the lane's own cell.  xs: this warp's 32 x 16 BF16
// staging area (256 words) in shared memory.
__device__ float warp_mlp(const MlpDev &P, const float (&feat)[kIn], uint32_t *xs)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t *row = xs + lane * 8;
    row[0] = pack_bf16(feat[0], feat[1]);
    row[1] = pack_bf16(feat[2], feat[3]);
    row[2] = pack_bf16(feat[4], feat[5]);
    row[3] = pack_bf16(feat[6], 0.f);
    row[4] = row[5] = row[6] = row[7] = 0u;
    __syncwarp();
    const uint32_t *w1 = reinterpret_cast<const uint32_t *>(P.w1);  // [32][16] bf16 = [32][8] words
    const uint32_t *w2 = reinterpret_cast<const uint32_t *>(P.w2);  // [32][32] bf16 = [32][16] words
    const uint32_t *w3 = reinterpret_cast<const uint32_t *>(P.w3);  // [8][32] bf16 = [8][16] words
    // Both 16-row tiles (mt) go through each hidden-unit tile (nt) together, so every weight
    // fragment and bias is loaded from shared memory once per warp and z step.
    uint32_t a[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        a[mt][0] = xs[(mt * 16 + g) * 8 + t];
        a[mt][1] = xs[(mt * 16 + g + 8) * 8 + t];
        a[mt][2] = xs[(mt * 16 + g) * 8 + t + 4];
        a[mt][3] = xs[(mt * 16 + g + 8) * 8 + t + 4];
    }
    // layer 1: 4 tiles of 8 hidden units; tile nt is half (nt & 1) of k-step nt / 2 of the next
    // layer's A fragment (registers 0/1 or 2/3)
    uint32_t h1[2][2][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + 2 * t;
        const float b0 = P.b1[c], b1 = P.b1[c + 1];
        const uint32_t wa = w1[(nt * 8 + g) * 8 + t], wb = w1[(nt * 8 + g) * 8 + t + 4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float d[4] = {b0, b1, b0, b1};  // bias as the initial accumulator
            mma_bf16(d, a[mt], wa, wb);
            h1[mt][nt >> 1][(nt & 1) * 2 + 0] = silu_pair(d[0], d[1]);
            h1[mt][nt >> 1][(nt & 1) * 2 + 1] = silu_pair(d[2], d[3]);
        }
    }
    // layer 2
    uint32_t h2[2][2][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + 2 * t;
        const float b0 = P.b2[c], b1 = P.b2[c + 1];
        uint32_t wk[2][2];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            wk[ks][0] = w2[(nt * 8 + g) * 16 + ks * 8 + t];
            wk[ks][1] = w2[(nt * 8 + g) * 16 + ks * 8 + t + 4];
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float d[4] = {b0, b1, b0, b1};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) mma_bf16(d, h1[mt][ks], wk[ks][0], wk[ks][1]);
            h2[mt][nt >> 1][(nt & 1) * 2 + 0] = silu_pair(d[0], d[1]);
            h2[mt][nt >> 1][(nt & 1) * 2 + 1] = silu_pair(d[2], d[3]);
        }
    }
    // layer 3: w3 as column 0 of an 8-column B
    uint32_t w3k[2][2];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        w3k[ks][0] = w3[g * 16 + ks * 8 + t];
        w3k[ks][1] = w3[g * 16 + ks * 8 + t + 4];
    }
    float y = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) mma_bf16(d, h2[mt][ks], w3k[ks][0], w3k[ks][1]);
        // column 0 sits in lanes with t == 0: d[0] for row g, d[2] for row g + 8
        const int r = (lane - mt * 16) & 15;
        const float ylo = __shfl_sync(0xffffffffu, d[0], 4 * (r & 7));
        const float yhi = __shfl_sync(0xffffffffu, d[2], 4 * (r & 7));
        if ((lane >> 4) == mt) y = (r < 8 ? ylo : yhi) + P.b3;
    }
    __syncwarp();
    return y;
}

// Pre-collision moments and non-equilibrium stress of one cell (no body force).
__device__ __forceinline__ void cell_stress(const float (&f)[kQ], float &rho, float (&u)[3], float (&pi)[6])
{
    using L = Lattice<kQ>;
    float m0 = 0.f, j[3] = {0.f, 0.f, 0.f}, s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const float cx = (float)L::cx(i), cy = (float)L::cy(i), cz = (float)L::cz(i);
        m0 += f[i];
        j[0] += cx * f[i];
        j[1] += cy * f[i];
        j[2] += cz * f[i];
        s[0] += cx * cx * f[i];
        s[1] += cy * cy * f[i];
        s[2] += cz * cz * f[i];
        s[3] += cx * cy * f[i];
        s[4] += cx * cz * f[i];
        s[5] += cy * cz * f[i];
    }
    rho = m0;
    const float inv = 1.f / m0;
    u[0] = j[0] * inv;
    u[1] = j[1] * inv;
    u[2] = j[2] * inv;
    pi[0] = s[0] - rho * (1.f / 3.f + u[0] * u[0]);
    pi[1] = s[1] - rho * (1.f / 3.f + u[1] * u[1]);
    pi[2] = s[2] - rho * (1.f / 3.f + u[2] * u[2]);
    pi[3] = s[3] - rho * u[0] * u[1];
    pi[4] = s[4] - rho * u[0] * u[2];
    pi[5] = s[5] - rho * u[1] * u[2];
}

struct ClosureArgsDev {
    float tau0, cs, lambda;
    int trt;
    int *err;  // set to 1 when a bounded wait of the tensor-core network gives up
};

constexpr uint32_t kTcWaitLimit = 1u << 22;

// The network of 256 cells (one per thread of the CTA) on the fifth-generation tensor cores:
// see mlp_tc.cuh.  Every thread of the CTA calls it (CTA barriers inside); ok: false once a
// wait has given up (the outputs are then undefined and *err is set by the caller).
__device__ __forceinline__ float tc_mlp_256(tc::TcSmem256 &S, float b3, const float (&feat)[kIn], uint32_t tmem,
                                            bool &ok)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    *reinterpret_cast<uint4 *>(S.a1 + tc::core_off(tid, 0, 2)) =
        make_uint4(pack_bf16(feat[0], feat[1]), pack_bf16(feat[2], feat[3]), pack_bf16(feat[4], feat[5]),
                   pack_bf16(feat[6], 0.f));
    *reinterpret_cast<uint4 *>(S.a1 + tc::core_off(tid, 8, 2)) = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_async_smem();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
    const uint32_t a1 = tc::smem_u32(S.a1), a2 = tc::smem_u32(S.a2), b1 = tc::smem_u32(S.b1),
                   b2 = tc::smem_u32(S.b2);
    if (tid == 0 && ok) {
        tc::mma_f16(tmem, tc::operand_desc(a1, 2), tc::operand_desc(b1, 2), idesc, 0);
        tc::mma_f16(tmem + 32, tc::operand_desc(a1 + 4096, 2), tc::operand_desc(b1, 2), idesc, 0);
        tc::mma_commit(&S.bar);
    }
    if (ok) ok = tc::mbar_wait(&S.bar, 0, kTcWaitLimit);
    // warp w reads TMEM lanes 32 (w % 4) .., the half w / 4 of the tile
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16, half = 32u * (uint32_t)(warp >> 2);
    if (ok) {
        tc::fence_after_sync();
        float v[32];
        tc::tmem_ld32(tmem + lane_off + half, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint4 q;
            q.x = silu_pair(v[8 * c + 0] + S.bias1[8 * c + 0], v[8 * c + 1] + S.bias1[8 * c + 1]);
            q.y = silu_pair(v[8 * c + 2] + S.bias1[8 * c + 2], v[8 * c + 3] + S.bias1[8 * c + 3]);
            q.z = silu_pair(v[8 * c + 4] + S.bias1[8 * c + 4], v[8 * c + 5] + S.bias1[8 * c + 5]);
            q.w = silu_pair(v[8 * c + 6] + S.bias1[8 * c + 6], v[8 * c + 7] + S.bias1[8 * c + 7]);
            *reinterpret_cast<uint4 *>(S.a2 + tc::core_off(tid, 8 * c, 4)) = q;
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (tid == 0 && ok) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            tc::mma_f16(tmem + 64 + 32 * h, tc::operand_desc(a2 + 8192 * h, 4), tc::operand_desc(b2, 4), idesc, 0);
            tc::mma_f16(tmem + 64 + 32 * h, tc::operand_desc(a2 + 8192 * h + 256, 4), tc::operand_desc(b2 + 256, 4),
                        idesc, 1);
        }
        tc::mma_commit(&S.bar);
    }
    if (ok) ok = tc::mbar_wait(&S.bar, 1, kTcWaitLimit);
    float y = b3;
    if (ok) {
        tc::fence_after_sync();
        float v[32];
        tc::tmem_ld32(tmem + lane_off + 64 + half, v);
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const uint32_t h = silu_pair(v[j] + S.bias2[j], v[j + 1] + S.bias2[j + 1]);
            y = fmaf(S.w3[j], __uint_as_float(h << 16), y);
            y = fmaf(S.w3[j + 1], __uint_as_float(h & 0xffff0000u), y);
        }
    }
    tc::fence_before_sync();
    return y;
}

// Closure sweep: like the plain sweep, but every lane stays in the z loop (the network's
// MMAs need the whole warp); lanes without a fluid cell feed zero features and skip the
// loads and stores.
// Tensor-core form of the network (mlp_tc.cuh): in the closure sweep (measured slower: its CTA
// barriers per z-step serialize the gathers of the CTA's warps) and in the standalone
// batched inference.
#ifndef LBM_MLP_TC_SWEEP
#define LBM_MLP_TC_SWEEP 0
#endif
#ifndef LBM_MLP_TC_INFER
#define LBM_MLP_TC_INFER 1
#endif

// Minimum resident CTAs of 256 threads per SM (register cap) per closure kind, measured on a
// 256^3 periodic box (two-grid, ms per step): Smagorinsky 0.46 at 4 (64 registers), 0.50 at 3,
// 0.61 at 2; network 0.89 at 3 (80 registers), 1.00 at 2.
#ifndef LBM_CLOSURE_MINB_SMAG
#define LBM_CLOSURE_MINB_SMAG 4
#endif
#ifndef LBM_CLOSURE_MINB_MLP
#define LBM_CLOSURE_MINB_MLP 3
#endif

template <int KIND, int CLOSURE, bool DIAG, int THROUGH, bool I32>
__global__ void __launch_bounds__(256, CLOSURE == 1 ? LBM_CLOSURE_MINB_SMAG : LBM_CLOSURE_MINB_MLP)
    k_closure_sweep(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock *__restrict__ blocks,
                    const DevTile *__restrict__ tiles, int tz, Coll<float> k, const MlpDev *__restrict__ mlp,
                    ClosureArgsDev ca, double *__restrict__ partials)
{
    __shared__ MlpDev P;
#if LBM_MLP_TC_SWEEP
    __shared__ tc::TcSmem256 S;
    uint32_t tmem = 0;
    bool tc_ok = true;
    if (CLOSURE == 2) {
        if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&S.tmem, 128);
        if (threadIdx.x == 0) {
            tc::mbar_init(&S.bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        tc::stage_weights(S, *mlp);
    }
#else
    __shared__ uint32_t xs[8][256];
#endif
    if (CLOSURE == 2) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(mlp);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
        for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 4); i += blockDim.x) dst[i] = src[i];
    }
    const DevTile t = tiles[blockIdx.x];
    const DevBlock *Bp = blocks + t.block;
    const DevBlock B = block_geo(Bp);
    constexpr bool kThr = THROUGH != 0 && KIND != SWEEP_AA_LOCAL;
    constexpr bool kTable = THROUGH == 2 && KIND != SWEEP_AA_LOCAL;
    constexpr int kFace = kTable ? 2 : 1;
    __shared__ NbrGeo nb[kTable ? 27 : 1];
    if (kTable) stage_neighbours(nb, blocks, Bp);
    __syncthreads();
    const int ttx = (int)t.width_m1 + 1;
    const int rows = blockDim.x / ttx;
    const int lx = threadIdx.x % ttx, ly = threadIdx.x / ttx;
    const int x = t.x0 + lx, y = t.y0 + ly;
    const bool active = ly < rows && x < B.nx && y < B.ny;
    const int zend = min((int)t.z0 + tz, B.nz);
    const bool masked = (t.flags & 1) != 0;
    const bool thr = kThr && B.through && active;
    const int axes = kTable ? 7 : B.wrap;
    Face fc{0, 0};
    if (thr) {
        fc.lo = ((x == 0 ? 1 : 0) | (y == 0 ? 2 : 0)) & axes;
        fc.hi = ((x == B.nx - 1 ? 1 : 0) | (y == B.ny - 1 ? 2 : 0)) & axes;
    }
    Diag<DIAG> dg;
#if LBM_MLP_TC_SWEEP
    if (CLOSURE == 2) {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = S.tmem;
    }
#else
    uint32_t *wx = xs[threadIdx.x >> 5];
#endif
    for (int z = t.z0; z < zend; ++z) {
        const int64_t cell = B.cell(active ? x : 0, active ? y : 0, z);
        const uint32_t m = (active && masked) ? B.mask[cell] : 0u;
        const bool live = active && !(m & kMaskSolid);
        Face f2 = fc;
        if (thr) {
            f2.lo |= (z == 0 ? 4 : 0) & axes;
            f2.hi |= (z == B.nz - 1 ? 4 : 0) & axes;
        }
        const bool face = live && (f2.lo | f2.hi) != 0;
        float f[kQ];
        const bool any_face = __any_sync(0xffffffffu, face);
        if (live) {
            if (kThr && any_face) {
                if (masked)
                    gather_cell<KIND, kFace, true, I32>(f, A, B, nb, f2, x, y, z, cell, m, k.base);
                else
                    gather_cell<KIND, kFace, false, I32>(f, A, B, nb, f2, x, y, z, cell, 0u, k.base);
            } else {
                if (masked && KIND != SWEEP_AA_LOCAL)
                    gather_cell<KIND, 0, true, I32>(f, A, B, nb, f2, x, y, z, cell, m, k.base);
                else
                    gather_cell<KIND, 0, false, I32>(f, A, B, nb, f2, x, y, z, cell, 0u, k.base);
            }
        } else {
#pragma unroll
            for (int i = 0; i < kQ; ++i) f[i] = (float)Lattice<kQ>::w(i);
        }
        float rho, u[3], pi[6];
        cell_stress(f, rho, u, pi);
        float tau;
        if (CLOSURE == 1) {
            const float q = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] + 2.f * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5]);
            tau = 0.5f * (ca.tau0 + sqrtf(ca.tau0 * ca.tau0 + 18.f * ca.cs * ca.cs * sqrtf(2.f * q) / rho));
        } else {
            float feat[kIn] = {(rho - 1.f) * P.s_rho, pi[0] * P.s_pi, pi[1] * P.s_pi, pi[2] * P.s_pi,
                               pi[3] * P.s_pi,        pi[4] * P.s_pi, pi[5] * P.s_pi};
            if (!live)
                for (int kk = 0; kk < kIn; ++kk) feat[kk] = 0.f;
#if LBM_MLP_TC_SWEEP
            tau = ca.tau0 + P.s_tau * softplus_fast(tc_mlp_256(S, P.b3, feat, tmem, tc_ok));
#else
            tau = ca.tau0 + P.s_tau * softplus_fast(warp_mlp(P, feat, wx));
#endif
        }
        if (live) {
            const float wp = 1.f / tau;
            const float wm = ca.trt ? 1.f / (ca.lambda / (tau - 0.5f) + 0.5f) : wp;
            constexpr float wc[4] = {1.f / 3.f, 1.f / 18.f, 1.f / 36.f, 0.f};  // D3Q19 weight classes
            const Rates<float> rt = rates_of<float>(wp, wm, wc);
            float r2, ux, uy, uz;
            collide<kQ, false, float, true>(f, k, rt, 0.f, r2, ux, uy, uz);
            dg.add(f, 0.f, r2, ux, uy, uz);
            if (kThr && any_face) {
                if (masked)
                    scatter_cell<KIND, kFace, true, I32>(f, A, Bout, B, nb, f2, x, y, z, cell, m, k.base);
                else
                    scatter_cell<KIND, kFace, false, I32>(f, A, Bout, B, nb, f2, x, y, z, cell, 0u, k.base);
            } else {
                if (masked && KIND != SWEEP_AA_LOCAL)
                    scatter_cell<KIND, 0, true, I32>(f, A, Bout, B, nb, f2, x, y, z, cell, m, k.base);
                else
                    scatter_cell<KIND, 0, false, I32>(f, A, Bout, B, nb, f2, x, y, z, cell, 0u, k.base);
            }
        }
    }
#if LBM_MLP_TC_SWEEP
    if (CLOSURE == 2) {
        if (!tc_ok && threadIdx.x == 0 && ca.err) atomicExch(ca.err, 1);
        tc::fence_before_sync();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tmem, 128);
    }
#endif
    dg.tile_record(partials);
}

template <int KIND, int CLOSURE, bool DIAG, bool I32>
cudaError_t go3(const ClosureLaunch &s)
{
    dim3 grid((unsigned)s.sw.ntiles), block((unsigned)(s.sw.tx * s.sw.ty));
    const ClosureArgsDev ca{s.tau0, s.cs, s.lambda, s.trt, s.err};
    if (s.sw.through == 2)
        k_closure_sweep<KIND, CLOSURE, DIAG, 2, I32><<<grid, block, 0, s.sw.stream>>>(
            (StoreT *)s.sw.a, (StoreT *)s.sw.b, s.sw.blocks, s.sw.tiles, s.sw.tz, s.sw.cf, s.mlp, ca, s.sw.partials);
    else if (s.sw.through)
        k_closure_sweep<KIND, CLOSURE, DIAG, 1, I32><<<grid, block, 0, s.sw.stream>>>(
            (StoreT *)s.sw.a, (StoreT *)s.sw.b, s.sw.blocks, s.sw.tiles, s.sw.tz, s.sw.cf, s.mlp, ca, s.sw.partials);
    else
        k_closure_sweep<KIND, CLOSURE, DIAG, 0, I32><<<grid, block, 0, s.sw.stream>>>(
            (StoreT *)s.sw.a, (StoreT *)s.sw.b, s.sw.blocks, s.sw.tiles, s.sw.tz, s.sw.cf, s.mlp, ca, s.sw.partials);
    return cudaGetLastError();
}

template <int KIND, int CLOSURE>
cudaError_t go2(const ClosureLaunch &s)
{
    // 32-bit neighbour indices in the AA neighbour sweep where the arena allows it (as the
    // plain sweeps)
    if constexpr (KIND == SWEEP_AA_NBR) {
        if (s.sw.idx32) return s.sw.partials ? go3<KIND, CLOSURE, true, true>(s) : go3<KIND, CLOSURE, false, true>(s);
    }
    return s.sw.partials ? go3<KIND, CLOSURE, true, false>(s) : go3<KIND, CLOSURE, false, false>(s);
}

template <int KIND>
cudaError_t go1(const ClosureLaunch &s)
{
    return s.closure == 1 ? go2<KIND, 1>(s) : go2<KIND, 2>(s);
}

// ---------------------------------------------------------------------------------------
// Standalone inference (the same warp MMA routine) and training kernels (FP32).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mlp_infer(const MlpDev *__restrict__ mlp, const float *__restrict__ X, int64_t n,
                                                   float *__restrict__ y)
{
    __shared__ MlpDev P;
    __shared__ uint32_t xs[8][256];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(mlp);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float feat[kIn];
    for (int k = 0; k < kIn; ++k) feat[k] = s < n ? X[s * kIn + k] : 0.f;
    const float out = warp_mlp(P, feat, xs[threadIdx.x >> 5]);
    if (s < n) y[s] = out;
}

// Inference on the fifth-generation tensor cores (mlp_tc.cuh): one CTA of 128 threads per
// tile of 128 samples; thread t owns sample (row) t.  Same rounding points as warp_mlp: BF16
// features, weights and hidden activations, FP32 sums; the output layer in FP32 on the CUDA
// cores.  err: set to 1 when a bounded wait on the MMA completion gives up.
__global__ void __launch_bounds__(128) k_mlp_infer_tc(const MlpDev *__restrict__ mlp, const float *__restrict__ X,
                                                      int64_t n, float *__restrict__ y, int *__restrict__ err)
{
    // persistent: TMEM, barrier and weights set up once; the CTA walks tiles of 128 samples
    extern __shared__ unsigned char smem_raw[];
    tc::TcSmem &S = *reinterpret_cast<tc::TcSmem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc::tmem_alloc(&S.tmem, 64);
    if (tid == 0) {
        tc::mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::stage_weights(S, *mlp);
    const float b3 = mlp->b3;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
    const uint32_t a1 = tc::smem_u32(S.a1), a2 = tc::smem_u32(S.a2), b1 = tc::smem_u32(S.b1),
                   b2 = tc::smem_u32(S.b2);
    const int64_t tiles = (n + 127) / 128;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        // features of sample `tid` of the tile -> row tid of A1 (K chunks 0 and 1)
        const int64_t s = tile * 128 + tid;
        float f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = (s < n && k < kIn) ? X[s * kIn + k] : 0.f;
        *reinterpret_cast<uint4 *>(S.a1 + tc::core_off(tid, 0, 2)) =
            make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
        *reinterpret_cast<uint4 *>(S.a1 + tc::core_off(tid, 8, 2)) = make_uint4(0u, 0u, 0u, 0u);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            tc::mma_f16(tmem, tc::operand_desc(a1, 2), tc::operand_desc(b1, 2), idesc, 0);
            tc::mma_commit(&S.bar);
        }
        ok = tc::mbar_wait(&S.bar, 0, kTcWaitLimit);
        if (ok) {
            tc::fence_after_sync();
            float v[32];
            tc::tmem_ld32(tmem + lane_off, v);  // D1 row tid: halved pre-activations of the 32 units
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint4 q;
                q.x = silu_pair(v[8 * c + 0] + S.bias1[8 * c + 0], v[8 * c + 1] + S.bias1[8 * c + 1]);
                q.y = silu_pair(v[8 * c + 2] + S.bias1[8 * c + 2], v[8 * c + 3] + S.bias1[8 * c + 3]);
                q.z = silu_pair(v[8 * c + 4] + S.bias1[8 * c + 4], v[8 * c + 5] + S.bias1[8 * c + 5]);
                q.w = silu_pair(v[8 * c + 6] + S.bias1[8 * c + 6], v[8 * c + 7] + S.bias1[8 * c + 7]);
                *reinterpret_cast<uint4 *>(S.a2 + tc::core_off(tid, 8 * c, 4)) = q;
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        tc::fence_after_sync();
        if (!ok) break;
        if (tid == 0) {
            tc::mma_f16(tmem + 32, tc::operand_desc(a2, 4), tc::operand_desc(b2, 4), idesc, 0);
            tc::mma_f16(tmem + 32, tc::operand_desc(a2 + 256, 4), tc::operand_desc(b2 + 256, 4), idesc, 1);
            tc::mma_commit(&S.bar);
        }
        ok = tc::mbar_wait(&S.bar, 1, kTcWaitLimit);
        float out = 0.f;
        if (ok) {
            tc::fence_after_sync();
            float v[32];
            tc::tmem_ld32(tmem + lane_off + 32, v);
            out = b3;
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const uint32_t h = silu_pair(v[j] + S.bias2[j], v[j + 1] + S.bias2[j + 1]);
                out = fmaf(S.w3[j], __uint_as_float(h << 16), out);
                out = fmaf(S.w3[j + 1], __uint_as_float(h & 0xffff0000u), out);
            }
        }
        if (s < n) y[s] = out;
        // the next tile overwrites A1, A2 and the accumulators: every thread is done with them
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        tc::fence_after_sync();
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// Network in FP32 (training): forward and backward of one sample.  Parameters in global
// memory (read through the cache).  Gradient of L = mean (softplus(y) - t)^2 over n_total.
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Gradient kernel: CTAs of kGradThreads threads, each CTA a run of `per_cta` consecutive
// samples taken kGradThreads at a time.  Per chunk, thread s runs sample s forward and
// backward and leaves x, h1, h2, dz1 = dL/dz1, dz2 = dL/dz2 and dy = dL/dy in shared memory;
// then each thread sums the gradient entries it owns over the chunk (W2 entries e = t +
// kGradThreads k, the other 321 entries as one list) in registers.  One partial record
// (kParams gradient entries + the loss sum) per CTA; all sums in a fixed order.
constexpr int kGradThreads = 128;
constexpr int kRow = kH + 1;  // padded row of the per-sample arrays (no bank conflicts)
constexpr int kW2PerThread = kH * kH / kGradThreads;
constexpr int kRest = kH * kIn + 3 * kH + 1;  // W1, b1, b2, w3, b3
constexpr int kRestPerThread = (kRest + kGradThreads - 1) / kGradThreads;
struct GradSmem {
    float w[kOffScale];  // W1, b1, W2, b2, w3, b3
    float x[kGradThreads][8];
    float h1[kGradThreads][kRow], h2[kGradThreads][kRow], dz1[kGradThreads][kRow], dz2[kGradThreads][kRow];
    float dy[kGradThreads];
    float red[kGradThreads / 32];
};

__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const float *__restrict__ Pg, const float *__restrict__ X,
                                                           const float *__restrict__ T, int64_t n, int64_t per_cta,
                                                           float inv_n, float *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem &sm = *reinterpret_cast<GradSmem *>(smem_raw);
    const int tid = threadIdx.x;
    for (int p = tid; p < kOffScale; p += kGradThreads) sm.w[p] = Pg[p];
    const float *W1 = sm.w + kOffW1, *b1 = sm.w + kOffB1, *W2 = sm.w + kOffW2, *b2 = sm.w + kOffB2,
                *w3 = sm.w + kOffW3;
    float aw2[kW2PerThread], arest[kRestPerThread], aloss = 0.f;
    for (int k = 0; k < kW2PerThread; ++k) aw2[k] = 0.f;
    for (int k = 0; k < kRestPerThread; ++k) arest[k] = 0.f;
    __syncthreads();
    const int64_t s0 = (int64_t)blockIdx.x * per_cta;
    const int64_t s1 = min(s0 + per_cta, n);
    for (int64_t base = s0; base < s1; base += kGradThreads) {
        const int64_t s = base + tid;
        const bool ok = s < s1;
        float x[kIn];
        for (int m = 0; m < kIn; ++m) {
            x[m] = ok ? X[s * kIn + m] : 0.f;
            sm.x[tid][m] = x[m];
        }
        // forward; dz1 / dz2 first hold the SiLU derivatives at z1 / z2
        float *h1 = sm.h1[tid], *h2 = sm.h2[tid], *d1 = sm.dz1[tid], *d2 = sm.dz2[tid];
#pragma unroll 4
        for (int j = 0; j < kH; ++j) {
            float z = b1[j];
#pragma unroll
            for (int m = 0; m < kIn; ++m) z += W1[j * kIn + m] * x[m];
            h1[j] = z / (1.f + expf(-z));
            d1[j] = dsilu(z);
        }
        float yv = sm.w[kOffB3];
#pragma unroll 2
        for (int j = 0; j < kH; ++j) {
            float z = b2[j];
#pragma unroll
            for (int l = 0; l < kH; ++l) z += W2[j * kH + l] * h1[l];
            const float h = z / (1.f + expf(-z));
            h2[j] = h;
            d2[j] = dsilu(z);
            yv += w3[j] * h;
        }
        const float sp = yv > 30.f ? yv : log1pf(expf(yv));
        const float r = ok ? sp - T[s] : 0.f;
        aloss += r * r;
        const float dy = 2.f * r / (1.f + expf(-yv)) * inv_n;
        sm.dy[tid] = dy;
        // backward: dz2 = dy w3 silu'(z2); dz1 = (W2^T dz2) silu'(z1)
#pragma unroll 4
        for (int j = 0; j < kH; ++j) d2[j] *= dy * w3[j];
#pragma unroll 2
        for (int l = 0; l < kH; ++l) {
            float dh = 0.f;
#pragma unroll
            for (int j = 0; j < kH; ++j) dh += W2[j * kH + l] * d2[j];
            d1[l] *= dh;
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kGradThreads, s1 - base);
#pragma unroll
        for (int k = 0; k < kW2PerThread; ++k) {
            const int e = tid + kGradThreads * k, j = e / kH, l = e % kH;
            float acc = 0.f;
            for (int q = 0; q < cnt; ++q) acc += sm.dz2[q][j] * sm.h1[q][l];
            aw2[k] += acc;
        }
#pragma unroll
        for (int k = 0; k < kRestPerThread; ++k) {
            const int e = tid + kGradThreads * k;
            if (e >= kRest) break;
            float acc = 0.f;
            if (e < kH * kIn) {
                const int l = e / kIn, m = e % kIn;
                for (int q = 0; q < cnt; ++q) acc += sm.dz1[q][l] * sm.x[q][m];
            } else if (e < kH * kIn + kH) {
                const int l = e - kH * kIn;
                for (int q = 0; q < cnt; ++q) acc += sm.dz1[q][l];
            } else if (e < kH * kIn + 2 * kH) {
                const int j = e - kH * kIn - kH;
                for (int q = 0; q < cnt; ++q) acc += sm.dz2[q][j];
            } else if (e < kH * kIn + 3 * kH) {
                const int j = e - kH * kIn - 2 * kH;
                for (int q = 0; q < cnt; ++q) acc += sm.dy[q] * sm.h2[q][j];
            } else {
                for (int q = 0; q < cnt; ++q) acc += sm.dy[q];
            }
            arest[k] += acc;
        }
        __syncthreads();
    }
    float *out = partials + (int64_t)blockIdx.x * (kParams + 1);
#pragma unroll
    for (int k = 0; k < kW2PerThread; ++k) out[kOffW2 + tid + kGradThreads * k] = aw2[k];
#pragma unroll
    for (int k = 0; k < kRestPerThread; ++k) {
        const int e = tid + kGradThreads * k;
        if (e >= kRest) break;
        // rest list order W1, b1 | b2, w3, b3 -> packed offsets (W2 sits between b1 and b2)
        out[e < kOffW2 ? e : e + kH * kH] = arest[k];
    }
    if (tid < 3) out[kOffScale + tid] = 0.f;
    for (int o = 16; o > 0; o >>= 1) aloss += __shfl_xor_sync(0xffffffffu, aloss, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = aloss;
    __syncthreads();
    if (tid == 0) {
        float l = 0.f;
        for (int w = 0; w < kGradThreads / 32; ++w) l += sm.red[w];
        out[kParams] = l;
    }
}

// Sum the per-CTA records in a fixed order (deterministic); loss = mean squared residual.
__global__ void k_mlp_reduce(const float *__restrict__ partials, int nrec, float inv_n, float *__restrict__ grad,
                             double *__restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kParams) return;
    double acc = 0.0;
    for (int r = 0; r < nrec; ++r) acc += partials[(int64_t)r * (kParams + 1) + p];
    if (p < kParams)
        grad[p] = (float)acc;
    else
        *loss = acc * inv_n;
}

// Adam on the packed parameters (the three scales are held fixed).
__global__ void k_adam(float *__restrict__ Pg, const float *__restrict__ grad, float *__restrict__ m1,
                       float *__restrict__ m2, float lr, float b1t, float b2t)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kOffScale) return;
    const float g = grad[p];
    m1[p] = 0.9f * m1[p] + 0.1f * g;
    m2[p] = 0.999f * m2[p] + 0.001f * g * g;
    const float mh = m1[p] / (1.f - b1t), vh = m2[p] / (1.f - b2t);
    Pg[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// Device form of packed parameters P on the device (the same values as mlp_device_form).
__global__ void __launch_bounds__(256) k_mlp_device_form(const float *__restrict__ P, MlpDev *__restrict__ d)
{
    for (int e = threadIdx.x; e < kH * 16; e += blockDim.x) {
        const int j = e >> 4, l = e & 15;
        d->w1[j][l] = __float2bfloat16_rn(l < kIn ? 0.5f * P[kOffW1 + j * kIn + l] : 0.f);
    }
    for (int e = threadIdx.x; e < kH * kH; e += blockDim.x)
        d->w2[e / kH][e % kH] = __float2bfloat16_rn(0.5f * P[kOffW2 + e]);
    for (int e = threadIdx.x; e < 8 * kH; e += blockDim.x) {
        const int r = e / kH, j = e % kH;
        d->w3[r][j] = __float2bfloat16_rn(r == 0 ? P[kOffW3 + j] : 0.f);
    }
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
        d->b1[j] = 0.5f * P[kOffB1 + j];
        d->b2[j] = 0.5f * P[kOffB2 + j];
    }
    if (threadIdx.x == 0) {
        d->b3 = P[kOffB3];
        d->s_rho = P[kOffScale];
        d->s_pi = P[kOffScale + 1];
        d->s_tau = P[kOffScale + 2];
    }
}

}  // namespace

MlpDev mlp_device_form(const float *P)
{
    MlpDev d;
    memset(&d, 0, sizeof d);
    auto bf = [](float v) { return __float2bfloat16_rn(v); };
    // hidden layers halved (exact: a power of two), so the accumulators hold z/2 (see silu_pair)
    for (int j = 0; j < kH; ++j) {
        for (int l = 0; l < kIn; ++l) d.w1[j][l] = bf(0.5f * P[kOffW1 + j * kIn + l]);
        for (int l = kIn; l < 16; ++l) d.w1[j][l] = bf(0.f);
        for (int l = 0; l < kH; ++l) d.w2[j][l] = bf(0.5f * P[kOffW2 + j * kH + l]);
        d.w3[0][j] = bf(P[kOffW3 + j]);
        for (int r = 1; r < 8; ++r) d.w3[r][j] = bf(0.f);
        d.b1[j] = 0.5f * P[kOffB1 + j];
        d.b2[j] = 0.5f * P[kOffB2 + j];
    }
    d.b3 = P[kOffB3];
    d.s_rho = P[kOffScale];
    d.s_pi = P[kOffScale + 1];
    d.s_tau = P[kOffScale + 2];
    return d;
}

cudaError_t launch_closure_sweep(const ClosureLaunch &s)
{
    if (s.sw.ntiles <= 0) return cudaSuccess;
    if (s.sw.force || s.sw.tx * s.sw.ty > 256 || s.sw.tx % 32 != 0) return cudaErrorNotSupported;
#if LBM_MLP_TC_SWEEP
    if (s.closure == CLOSURE_MLP && s.sw.tx * s.sw.ty != 256) return cudaErrorNotSupported;  // 256-row MMA tile
#endif
    switch (s.sw.kind) {
        case SWEEP_PULL: return go1<SWEEP_PULL>(s);
        case SWEEP_AA_LOCAL: return go1<SWEEP_AA_LOCAL>(s);
        case SWEEP_AA_NBR: return go1<SWEEP_AA_NBR>(s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm

using namespace lbm;

// ---------------------------------------------------------------------------------------
// C ABI of the network (inference and training); see include/lbm.h.
// ---------------------------------------------------------------------------------------
struct lbm_mlp {
    float *P = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *partials = nullptr;
    double *loss = nullptr;
    MlpDev *dev = nullptr;  // device form of P (refreshed on the device after training)
    int *err = nullptr;     // tensor-core inference status
    int64_t max_batch = 0, nrec_cap = 0, adam_t = 0;
    cudaStream_t stream = nullptr;
};

namespace {
constexpr int64_t kPerCta = 1024;  // samples per gradient CTA (a multiple of kGradThreads)

lbm_status mlp_ck(cudaError_t e) { return e == cudaSuccess ? LBM_OK : (e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA); }
}  // namespace

extern "C" {

lbm_status lbm_mlp_create(const float *params, int64_t max_batch, void *cuda_stream, lbm_mlp **out)
{
    if (!out || !params || max_batch < 1) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_mlp *m = new (std::nothrow) lbm_mlp();
    if (!m) return LBM_ERR_OOM;
    m->stream = (cudaStream_t)cuda_stream;
    m->max_batch = max_batch;
    m->nrec_cap = (max_batch + kPerCta - 1) / kPerCta;
    lbm_status s = LBM_OK;
    if ((s = mlp_ck(cudaMalloc(&m->P, kParams * sizeof(float)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->grad, kParams * sizeof(float)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->m1, kParams * sizeof(float)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->m2, kParams * sizeof(float)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->partials, m->nrec_cap * (kParams + 1) * sizeof(float)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->loss, sizeof(double)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->dev, sizeof(MlpDev)))) != LBM_OK ||
        (s = mlp_ck(cudaMalloc(&m->err, sizeof(int)))) != LBM_OK) {
        lbm_mlp_destroy(m);
        return s;
    }
    cudaMemsetAsync(m->m1, 0, kParams * sizeof(float), m->stream);
    cudaMemsetAsync(m->m2, 0, kParams * sizeof(float), m->stream);
    cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
    if ((s = lbm_mlp_set_params(m, params)) != LBM_OK) {
        lbm_mlp_destroy(m);
        return s;
    }
    *out = m;
    return LBM_OK;
}

lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *params)
{
    if (!m || !params) return LBM_ERR_ARG;
    lbm_status s = mlp_ck(cudaMemcpyAsync(m->P, params, kParams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    if (s != LBM_OK) return s;
    MlpDev d = mlp_device_form(params);
    s = mlp_ck(cudaMemcpyAsync(m->dev, &d, sizeof d, cudaMemcpyHostToDevice, m->stream));
    if (s != LBM_OK) return s;
    m->adam_t = 0;
    cudaMemsetAsync(m->m1, 0, kParams * sizeof(float), m->stream);
    cudaMemsetAsync(m->m2, 0, kParams * sizeof(float), m->stream);
    return mlp_ck(cudaStreamSynchronize(m->stream));
}

lbm_status lbm_mlp_get_params(lbm_mlp *m, float *params)
{
    if (!m || !params) return LBM_ERR_ARG;
    int e = 0;
    lbm_status s = mlp_ck(cudaMemcpyAsync(params, m->P, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (s == LBM_OK) s = mlp_ck(cudaMemcpyAsync(&e, m->err, sizeof e, cudaMemcpyDeviceToHost, m->stream));
    if (s == LBM_OK) s = mlp_ck(cudaStreamSynchronize(m->stream));
    if (s != LBM_OK) return s;
    if (e) {
        cudaMemset(m->err, 0, sizeof e);
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

lbm_status lbm_mlp_infer(lbm_mlp *m, const float *X_dev, int64_t n, float *y_dev)
{
    if (!m || !X_dev || !y_dev || n < 0) return LBM_ERR_ARG;
    if (n == 0) return LBM_OK;
#if LBM_MLP_TC_INFER
    // persistent CTAs: 8 per SM (8 x 64 = 512 TMEM columns, 8 x 17 KB of shared memory)
    const int64_t tiles = (n + 127) / 128;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)sms * 8);
    k_mlp_infer_tc<<<(unsigned)grid, 128, sizeof(tc::TcSmem) + 1024, m->stream>>>(m->dev, X_dev, n, y_dev, m->err);
#else
    const int64_t ctas = (n + 255) / 256;
    if (ctas > 0x7fffffffLL) return LBM_ERR_ARG;
    k_mlp_infer<<<(unsigned)ctas, 256, 0, m->stream>>>(m->dev, X_dev, n, y_dev);
#endif
    return mlp_ck(cudaGetLastError());
}

lbm_status lbm_mlp_loss_grad(lbm_mlp *m, const float *X_dev, const float *T_dev, int64_t n, double *loss_host,
                             float *grad_host)
{
    if (!m || !X_dev || !T_dev || n < 1 || n > m->max_batch) return LBM_ERR_ARG;
    const int64_t nrec = (n + kPerCta - 1) / kPerCta;
    static_assert(kPerCta % kGradThreads == 0, "whole chunks per CTA");
    const size_t smem = sizeof(GradSmem);
    lbm_status s = mlp_ck(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (s != LBM_OK) return s;
    k_mlp_grad<<<(unsigned)nrec, kGradThreads, smem, m->stream>>>(m->P, X_dev, T_dev, n, kPerCta, 1.f / (float)n,
                                                                  m->partials);
    if ((s = mlp_ck(cudaGetLastError())) != LBM_OK) return s;
    if (s != LBM_OK) return s;
    k_mlp_reduce<<<(kParams + 1 + 255) / 256, 256, 0, m->stream>>>(m->partials, (int)nrec, 1.f / (float)n, m->grad,
                                                                   m->loss);
    if ((s = mlp_ck(cudaGetLastError())) != LBM_OK) return s;
    if (grad_host &&
        (s = mlp_ck(cudaMemcpyAsync(grad_host, m->grad, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream))) !=
            LBM_OK)
        return s;
    if (loss_host &&
        (s = mlp_ck(cudaMemcpyAsync(loss_host, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream))) != LBM_OK)
        return s;
    if (grad_host || loss_host) return mlp_ck(cudaStreamSynchronize(m->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp *m, const float *X_dev, const float *T_dev, int64_t n, int64_t batch, int64_t iters,
                         float lr, double *loss_history)
{
    if (!m || !X_dev || !T_dev || n < 1 || batch < 1 || batch > m->max_batch || iters < 0) return LBM_ERR_ARG;
    int64_t start = 0;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t nb = std::min(batch, n - start);
        lbm_status s = lbm_mlp_loss_grad(m, X_dev + start * kIn, T_dev + start, nb, nullptr, nullptr);
        if (s != LBM_OK) return s;
        m->adam_t++;
        const float b1t = std::pow(0.9f, (float)m->adam_t), b2t = std::pow(0.999f, (float)m->adam_t);
        k_adam<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->P, m->grad, m->m1, m->m2, lr, b1t, b2t);
        if ((s = mlp_ck(cudaGetLastError())) != LBM_OK) return s;
        if (loss_history &&
            (s = mlp_ck(cudaMemcpyAsync(loss_history + it, m->loss, sizeof(double), cudaMemcpyDeviceToHost,
                                        m->stream))) != LBM_OK)
            return s;
        start += nb;
        if (start >= n) start = 0;
    }
    k_mlp_device_form<<<1, 256, 0, m->stream>>>(m->P, m->dev);  // inference follows the trained P
    lbm_status s2 = mlp_ck(cudaGetLastError());
    if (s2 != LBM_OK) return s2;
    return mlp_ck(cudaStreamSynchronize(m->stream));
}

void lbm_mlp_destroy(lbm_mlp *m)
{
    if (!m) return;
    cudaFree(m->P);
    cudaFree(m->grad);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->partials);
    cudaFree(m->loss);
    cudaFree(m->dev);
    cudaFree(m->err);
    delete m;
}

}  // extern "C"
