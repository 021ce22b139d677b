// sweep.cu -- fused stream-collide sweeps (two-grid pull, AA local, AA neighbour).
//
// Compiled once per (stencil, storage) pair: -DLBM_Q=19|27 -DLBM_ST=0..3 (fp64, fp32,
// bf16-deviation, fp16-deviation).  Each object defines launch_sweep_<Q>_<ST>.
//
// Method: Eq. 2 of the paper with the stream and collision steps fused into one pass over
// the cells (Sec. 5.1.2), pull form: each cell gathers the PDFs streaming into it, collides
// them (SRT/TRT with Guo force, kernels.cuh) and writes its post-collision PDFs.
//   two-grid pull : f_i <- src[x - c_i][i];  collide;  dst[x][i] <- f*_i
//   AA local      : f_i <- A[x][i];          collide;  A[x][opp i] <- f*_i
//   AA neighbour  : f_i <- A[x - c_i][opp i]; collide; A[x + c_i][i] <- f*_i
// Along an axis where the block is its own periodic neighbour (one block spanning a periodic
// axis), x -+ c_i is wrapped back into the block instead of going through a ghost copy.
// Every PDF value is read once and written once per cell update: 2 Q values per update.
//
// Mapping: one CTA per tile of tx x ty x tz cells of one block; a thread owns one (x, y)
// column of the tile and walks tz cells along z.  A warp covers 32 consecutive x cells,
// so every direction's load and store is one contiguous 32-element row segment
// (coalesced; c_x = +-1 directions are shifted by one element).
#include "select.cuh"

// Occupancy: minimum resident CTAs of 256 threads per SM.  For 4- and 2-byte storage, 4
// caps the sweeps at 64 registers (1024 threads per SM); measured on the 256^3 channel it
// beats the uncapped build by 6 % (two-grid) and 23 % (AA neighbour sweep).  The FP64 sweep
// is bound by the FP64 pipe, not by memory parallelism: 2 CTAs per SM avoid spilling.
#ifndef LBM_SWEEP_MINB
#if LBM_ST == 0
#define LBM_SWEEP_MINB 2
#else
#define LBM_SWEEP_MINB 4
#endif
#endif

namespace lbm {

namespace {

constexpr int kQ = LBM_Q;
using S = Storage<StoreT>;
using R = typename S::R;

// The diagnostics variant (DIAG) keeps eight running sums in registers; one CTA fewer per
// SM leaves it room for them without spilling.
constexpr int kMinB = LBM_SWEEP_MINB;
constexpr int kMinBDiag = LBM_SWEEP_MINB > 3 ? 3 : (LBM_SWEEP_MINB > 1 ? 1 : LBM_SWEEP_MINB);

// Per-CTA diagnostics record of the cells this CTA updated (DIAG): sums accumulated per
// thread and per warp in the sweep's arithmetic type, across warps in FP64:
// mass, momentum (rho u, half-force corrected), kinetic energy, max |u|, non-finite
// cells, fluid cells.
template <bool DIAG>
struct Diag {
    R m = R(0), jx = R(0), jy = R(0), jz = R(0), e = R(0), umax = R(0), bad = R(0), n = R(0);
    __device__ __forceinline__ void add(R rho, R ux, R uy, R uz)
    {
        if (!DIAG) return;
        const R u2 = ux * ux + uy * uy + uz * uz;
        const bool ok = isfinite(rho) && isfinite(u2);
        m += rho;
        jx += rho * ux;
        jy += rho * uy;
        jz += rho * uz;
        e += R(0.5) * rho * u2;
        umax = fmax(umax, sqrt(u2));
        bad += ok ? R(0) : R(1);
        n += R(1);
    }
};

template <class T>
__device__ __forceinline__ T wsum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class T>
__device__ __forceinline__ T wmax(T v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One cell: gather, collide, scatter (see the file header).  FACE: the cell lies on a face
// of an axis the block wraps on, so neighbour indices are wrapped.
template <bool FORCE, int KIND, bool DIAG, bool FACE>
__device__ __forceinline__ void update_cell(StoreT *__restrict__ a, StoreT *__restrict__ b, const DevBlock &B, int x,
                                            int y, int z, int64_t cell, const Coll<R> &k, Diag<DIAG> &dg)
{
    using L = Lattice<kQ>;
    R f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
        if (KIND == SWEEP_PULL) {
            const int64_t w = FACE ? wrap_shift(B, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i)) : 0;
            f[i] = S::ld(a + (int64_t)i * B.slab + cell - off + w, k.base[i]);
        } else if (KIND == SWEEP_AA_LOCAL) {
            f[i] = S::ld_rw(a + (int64_t)i * B.slab + cell, k.base[i]);
        } else {
            const int o = L::opp(i);
            const int64_t w = FACE ? wrap_shift(B, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i)) : 0;
            f[i] = S::ld_rw(a + (int64_t)o * B.slab + cell - off + w, k.base[i]);
        }
    }
    R rho, ux, uy, uz;
    collide<kQ, FORCE, R>(f, k, rho, ux, uy, uz);
    // The neighbour sweep's store offsets equal its load offsets of the opposite directions;
    // hide the coordinates from the optimiser so it recomputes them here instead of keeping
    // 19 offsets live across the collision.
    int xs = x, ys = y, zs = z;
    if (KIND == SWEEP_AA_NBR) asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs));
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
        if (KIND == SWEEP_PULL) {
            S::st(b + (int64_t)i * B.slab + cell, f[i], k.base[i]);
        } else if (KIND == SWEEP_AA_LOCAL) {
            const int o = L::opp(i);
            S::st(a + (int64_t)o * B.slab + cell, f[i], k.base[i]);
        } else {
            const int64_t w = FACE ? wrap_shift(B, xs, ys, zs, L::cx(i), L::cy(i), L::cz(i)) : 0;
            const int64_t c2 = (int64_t)(zs + 1) * B.plane + (int64_t)(ys + 1) * B.pitch + B.xo + xs;
            S::st(a + (int64_t)i * B.slab + c2 + off + w, f[i], k.base[i]);
        }
    }
    dg.add(rho, ux, uy, uz);
}

// The cells of one tile.  A thread owns one (x, y) column and walks the tile's z range; a
// warp whose cells include a face of a wrapped axis takes the wrapped-index path, all other
// warps the plain one (the test is warp-uniform, so neither path diverges).
template <bool FORCE, int KIND, bool DIAG, bool WRAP>
__device__ __forceinline__ void sweep_cells(StoreT *__restrict__ A, StoreT *__restrict__ Bout,
                                            const DevBlock *__restrict__ blocks, const DevTile *__restrict__ tiles,
                                            int tz, const Coll<R> &k, Diag<DIAG> &dg)
{
    const DevTile t = tiles[blockIdx.x];
    const DevBlock B = blocks[t.block];
    const int ttx = 32 * t.tx32;            // this tile's width (<= the CTA's for narrow blocks)
    const int rows = blockDim.x / ttx;      // the tile's height; leftover threads stay idle
    const int lx = threadIdx.x % ttx, ly = threadIdx.x / ttx;
    if (ly >= rows) return;
    const int x = t.x0 + lx, y = t.y0 + ly;
    if (x >= B.nx || y >= B.ny) return;
    const int zend = min((int)t.z0 + tz, B.nz);
    StoreT *a = A + B.offset;
    StoreT *b = (KIND == SWEEP_PULL) ? Bout + B.offset : a;
    const bool masked = (t.flags & 1) != 0;
    const bool xyface = WRAP && (((B.wrap & 1) && (x == 0 || x == B.nx - 1)) || ((B.wrap & 2) && (y == 0 || y == B.ny - 1)));
    for (int z = t.z0; z < zend; ++z) {
        const int64_t cell = (int64_t)(z + 1) * B.plane + (int64_t)(y + 1) * B.pitch + B.xo + x;
        if (masked && B.mask[cell] != 0) continue;
        if (KIND == SWEEP_AA_LOCAL || !WRAP) {
            update_cell<FORCE, KIND, DIAG, false>(a, b, B, x, y, z, cell, k, dg);
        } else {
            const bool face = xyface || ((B.wrap & 4) && (z == 0 || z == B.nz - 1));
            if (__any_sync(__activemask(), face))
                update_cell<FORCE, KIND, DIAG, true>(a, b, B, x, y, z, cell, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, false>(a, b, B, x, y, z, cell, k, dg);
        }
    }
}

template <bool FORCE, int KIND, bool DIAG, bool WRAP>
__global__ void __launch_bounds__(256, DIAG ? kMinBDiag : kMinB)
    k_sweep(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock *__restrict__ blocks,
            const DevTile *__restrict__ tiles, int tx, int tz, Coll<R> k, double *__restrict__ partials)
{
    Diag<DIAG> dg;
    // every thread takes part in the block reduction, including those without cells
    sweep_cells<FORCE, KIND, DIAG, WRAP>(A, Bout, blocks, tiles, tz, k, dg);
    if (DIAG) {
        __shared__ double sh[8][8];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const R v[8] = {wsum(dg.m), wsum(dg.jx), wsum(dg.jy), wsum(dg.jz),
                        wsum(dg.e), wmax(dg.umax), wsum(dg.bad), wsum(dg.n)};
        if (lane == 0)
            for (int c = 0; c < 8; ++c) sh[warp][c] = (double)v[c];
        __syncthreads();
        if (threadIdx.x < 8) {
            const int c = threadIdx.x;
            double r = 0.0;
            for (int w = 0; w < nw; ++w) r = c == 5 ? fmax(r, sh[w][c]) : r + sh[w][c];
            partials[(int64_t)blockIdx.x * 8 + c] = r;
        }
    }
}

template <bool FORCE, int KIND, bool WRAP>
cudaError_t go(const SweepArgs &s, const Coll<R> &k)
{
    if (s.ntiles <= 0) return cudaSuccess;
    if (s.ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)s.ntiles), block((unsigned)(s.tx * s.ty));
    if (s.partials)
        k_sweep<FORCE, KIND, true, WRAP><<<grid, block, 0, s.stream>>>((StoreT *)s.a, (StoreT *)s.b, s.blocks,
                                                                       s.tiles, s.tx, s.tz, k, s.partials);
    else
        k_sweep<FORCE, KIND, false, WRAP><<<grid, block, 0, s.stream>>>((StoreT *)s.a, (StoreT *)s.b, s.blocks,
                                                                        s.tiles, s.tx, s.tz, k, nullptr);
    return cudaGetLastError();
}

template <bool FORCE>
cudaError_t go_kind(const SweepArgs &s, const Coll<R> &k)
{
    switch (s.kind) {
        case SWEEP_PULL: return s.wrap ? go<FORCE, SWEEP_PULL, true>(s, k) : go<FORCE, SWEEP_PULL, false>(s, k);
        case SWEEP_AA_LOCAL: return go<FORCE, SWEEP_AA_LOCAL, false>(s, k);
        case SWEEP_AA_NBR: return s.wrap ? go<FORCE, SWEEP_AA_NBR, true>(s, k) : go<FORCE, SWEEP_AA_NBR, false>(s, k);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t LBM_CAT(launch_sweep_, LBM_Q, LBM_ST)(const SweepArgs &s)
{
    if (s.tx * s.ty > 256 || s.tx % 32 != 0) return cudaErrorInvalidConfiguration;
    const Coll<R> &k = coll_of(s.cd, s.cf, (R *)nullptr);
    return s.force ? go_kind<true>(s, k) : go_kind<false>(s, k);
}

}  // namespace lbm
