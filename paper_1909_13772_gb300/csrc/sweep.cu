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
// Every PDF value is read once and written once per cell update: 2 Q values per update.
//
// Mapping: one CTA per tile of tx x ty x tz cells of one block; a thread owns one (x, y)
// column of the tile and walks tz cells along z.  A warp covers 32 consecutive x cells,
// so every direction's load and store is one contiguous 32-element row segment
// (coalesced; c_x = +-1 directions are shifted by one element).
#include "select.cuh"

namespace lbm {

namespace {

constexpr int kQ = LBM_Q;
using S = Storage<StoreT>;
using R = typename S::R;

template <bool FORCE, int KIND>
__global__ void __launch_bounds__(256) k_sweep(StoreT *__restrict__ A, StoreT *__restrict__ Bout,
                                               const DevBlock *__restrict__ blocks, const DevTile *__restrict__ tiles,
                                               int tx, int tz, Coll<R> k)
{
    const DevTile t = tiles[blockIdx.x];
    const DevBlock B = blocks[t.block];
    const int lx = threadIdx.x % tx, ly = threadIdx.x / tx;
    const int x = t.x0 + lx, y = t.y0 + ly;
    if (x >= B.nx || y >= B.ny) return;
    const int zend = min((int)t.z0 + tz, B.nz);
    StoreT *a = A + B.offset;
    StoreT *b = (KIND == SWEEP_PULL) ? Bout + B.offset : a;
    const bool masked = (t.flags & 1) != 0;
    for (int z = t.z0; z < zend; ++z) {
        const int64_t cell = (int64_t)(z + 1) * B.plane + (int64_t)(y + 1) * B.pitch + B.xo + x;
        if (masked && B.mask[cell] != 0) continue;
        R f[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
            if (KIND == SWEEP_PULL) {
                f[i] = S::ld(a + (int64_t)i * B.slab + cell - off, k.base[i]);
            } else if (KIND == SWEEP_AA_LOCAL) {
                f[i] = S::ld_rw(a + (int64_t)i * B.slab + cell, k.base[i]);
            } else {
                const int o = Lattice<kQ>::opp(i);
                f[i] = S::ld_rw(a + (int64_t)o * B.slab + cell - off, k.base[i]);
            }
        }
        collide<kQ, FORCE, R>(f, k);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
            if (KIND == SWEEP_PULL) {
                S::st(b + (int64_t)i * B.slab + cell, f[i], k.base[i]);
            } else if (KIND == SWEEP_AA_LOCAL) {
                const int o = Lattice<kQ>::opp(i);
                S::st(a + (int64_t)o * B.slab + cell, f[i], k.base[i]);
            } else {
                S::st(a + (int64_t)i * B.slab + cell + off, f[i], k.base[i]);
            }
        }
    }
}

template <bool FORCE, int KIND>
cudaError_t go(const SweepArgs &s, const Coll<R> &k)
{
    if (s.ntiles <= 0) return cudaSuccess;
    if (s.ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)s.ntiles), block((unsigned)(s.tx * s.ty));
    k_sweep<FORCE, KIND><<<grid, block, 0, s.stream>>>((StoreT *)s.a, (StoreT *)s.b, s.blocks, s.tiles, s.tx, s.tz, k);
    return cudaGetLastError();
}

template <bool FORCE>
cudaError_t go_kind(const SweepArgs &s, const Coll<R> &k)
{
    switch (s.kind) {
        case SWEEP_PULL: return go<FORCE, SWEEP_PULL>(s, k);
        case SWEEP_AA_LOCAL: return go<FORCE, SWEEP_AA_LOCAL>(s, k);
        case SWEEP_AA_NBR: return go<FORCE, SWEEP_AA_NBR>(s, k);
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
