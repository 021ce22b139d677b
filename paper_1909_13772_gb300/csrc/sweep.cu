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
// Neighbours outside the block are read (and, for the AA neighbour sweep, written) in place
// in the neighbour block when the block's faces match its neighbours exactly -- a block
// spanning a periodic axis alone is its own neighbour there -- instead of going through a
// ghost copy.
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

// Geometry of a neighbour block read in place (one per ghost-shell region), staged in
// shared memory once per CTA.
struct NbrGeo {
    int64_t offset, slab, plane;
    int32_t pitch, xo, nx, ny, nz, valid;
};

// Per-thread face flags: lo/hi bit a set when the cell is on the low/high face of axis a
// of a block that reads its neighbours in place.
struct Face {
    int lo, hi;
};

// Arena offset of slot `q` of the neighbour (x, y, z) + (DX, DY, DZ) when it may lie in a
// neighbour block (shared-memory table nb); otherwise (inside the block, or a boundary
// region) `own` = the plain own-layout offset.
// (DX, DY, DZ are compile-time constants after the direction loops unroll.)
__device__ __forceinline__ int64_t nbr_addr(const NbrGeo *nb, Face fc, int x, int y, int z, int DX, int DY, int DZ,
                                            int q, int64_t own)
{
    const int rx = DX > 0 ? ((fc.hi & 1) ? 1 : 0) : (DX < 0 ? ((fc.lo & 1) ? -1 : 0) : 0);
    const int ry = DY > 0 ? ((fc.hi & 2) ? 1 : 0) : (DY < 0 ? ((fc.lo & 2) ? -1 : 0) : 0);
    const int rz = DZ > 0 ? ((fc.hi & 4) ? 1 : 0) : (DZ < 0 ? ((fc.lo & 4) ? -1 : 0) : 0);
    if ((rx | ry | rz) == 0) return own;
    const NbrGeo &N = nb[(rx + 1) + 3 * (ry + 1) + 9 * (rz + 1)];
    if (!N.valid) return own;
    const int sx = rx > 0 ? 0 : (rx < 0 ? N.nx - 1 : x + DX);
    const int sy = ry > 0 ? 0 : (ry < 0 ? N.ny - 1 : y + DY);
    const int sz = rz > 0 ? 0 : (rz < 0 ? N.nz - 1 : z + DZ);
    return N.offset + (int64_t)q * N.slab + (int64_t)(sz + 1) * N.plane + (int64_t)(sy + 1) * N.pitch + N.xo + sx;
}

// One cell: gather, collide, scatter (see the file header).  FACE: the warp has cells on a
// face of a block that reads its neighbours in place; directions that leave the block there
// are wrapped (FACE 1: the block is its own neighbour) or resolved through the
// shared-memory neighbour table (FACE 2).  m: the cell's bounce-back
// bits (bit i: the source x - c_i is a no-slip cell; halfway bounce-back then supplies
// f_i(x, t+1) = f*_opp(i)(x, t), read from the cell's own slot).
//   pull: bounce source src[opp i][x]
//   AA neighbour: bounce source A[i][x] (where the E layout keeps f*_opp(i)(x)); the value
//   f*_i(x) whose target x + c_i is no-slip (bit opp(i)) goes to A[opp i][x], where the next
//   local sweep reads it as f_opp(i)(x, t+1).
template <bool FORCE, int KIND, bool DIAG, int FACE, bool MASK>
__device__ __forceinline__ void update_cell(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock &B,
                                            const NbrGeo *nb, Face fc, int x, int y, int z, int64_t cell, uint32_t m,
                                            const Coll<R> &k, Diag<DIAG> &dg)
{
    using L = Lattice<kQ>;
    StoreT *a = A + B.offset;
    R f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
        const bool bounce = MASK && i > 0 && ((m >> i) & 1u);
        if (KIND == SWEEP_AA_LOCAL) {
            f[i] = S::ld_rw(a + (int64_t)i * B.slab + cell, k.base[i]);
            continue;
        }
        const int sl = KIND == SWEEP_PULL ? i : L::opp(i);  // slot read from the source cell
        const int bs = KIND == SWEEP_PULL ? L::opp(i) : i;  // own slot read on bounce-back
        int64_t o = bounce ? (int64_t)bs * B.slab + cell : (int64_t)sl * B.slab + cell - off;
        if (FACE == 1 && !bounce) o += wrap_shift(B, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i));
        if (FACE == 2 && !bounce)
            o = nbr_addr(nb, fc, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i), sl, o + B.offset) - B.offset;
        f[i] = KIND == SWEEP_PULL ? S::ld(a + o, k.base[i]) : S::ld_rw(a + o, k.base[i]);
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
            S::st(Bout + B.offset + (int64_t)i * B.slab + cell, f[i], k.base[i]);
        } else if (KIND == SWEEP_AA_LOCAL) {
            const int o = L::opp(i);
            S::st(a + (int64_t)o * B.slab + cell, f[i], k.base[i]);
        } else {
            const int o = L::opp(i);
            const bool bounce = MASK && i > 0 && ((m >> o) & 1u);
            const int64_t c2 = B.cell(xs, ys, zs);
            int64_t d = bounce ? (int64_t)o * B.slab + c2 : (int64_t)i * B.slab + c2 + off;
            if (FACE == 1 && !bounce) d += wrap_shift(B, xs, ys, zs, L::cx(i), L::cy(i), L::cz(i));
            if (FACE == 2 && !bounce)
                d = nbr_addr(nb, fc, xs, ys, zs, L::cx(i), L::cy(i), L::cz(i), i, d + B.offset) - B.offset;
            S::st(a + d, f[i], k.base[i]);
        }
    }
    dg.add(rho, ux, uy, uz);
}

// The cells of one tile.  A thread owns one (x, y) column and walks the tile's z range.  A
// warp with a cell on a face of a block that reads its neighbours in place takes the
// resolving path, all other warps the plain one (the test is warp-uniform, so neither path
// diverges); THROUGH = some block of the launch reads its neighbours in place.
template <bool FORCE, int KIND, bool DIAG, int THROUGH>
__device__ __forceinline__ void sweep_cells(StoreT *__restrict__ A, StoreT *__restrict__ Bout,
                                            const DevBlock *__restrict__ blocks, const DevTile *__restrict__ tiles,
                                            int tz, const Coll<R> &k, Diag<DIAG> &dg)
{
    const DevTile t = tiles[blockIdx.x];
    const DevBlock *Bp = blocks + t.block;
    // scalar geometry in registers (the neighbour table stays out of them)
    DevBlock B;
    B.nx = Bp->nx;
    B.ny = Bp->ny;
    B.nz = Bp->nz;
    B.pitch = Bp->pitch;
    B.plane = Bp->plane;
    B.slab = Bp->slab;
    B.offset = Bp->offset;
    B.mask = Bp->mask;
    B.xo = Bp->xo;
    B.through = Bp->through;
    B.wrap = Bp->wrap;
    constexpr bool kThr = THROUGH != 0 && KIND != SWEEP_AA_LOCAL;
    constexpr bool kTable = THROUGH == 2 && KIND != SWEEP_AA_LOCAL;
    __shared__ NbrGeo nb[kTable ? 27 : 1];
    if (kTable) {
        if (threadIdx.x < 27) {
            const int r = threadIdx.x;
            const int n = (B.through && r != 13) ? Bp->nbr[r] : -1;
            NbrGeo g{};
            if (n >= 0) {
                const DevBlock *N = blocks + n;
                g = NbrGeo{N->offset, N->slab, N->plane, N->pitch, N->xo, N->nx, N->ny, N->nz, 1};
            }
            nb[r] = g;
        }
        __syncthreads();
    }
    const int ttx = (int)t.width_m1 + 1;  // this tile's width (the block's own if narrower)
    const int rows = blockDim.x / ttx;    // the tile's height; leftover threads stay idle
    const int lx = threadIdx.x % ttx, ly = threadIdx.x / ttx;
    if (ly >= rows) return;
    const int x = t.x0 + lx, y = t.y0 + ly;
    if (x >= B.nx || y >= B.ny) return;
    const int zend = min((int)t.z0 + tz, B.nz);
    const bool masked = (t.flags & 1) != 0;
    const bool thr = kThr && B.through;
    // faces that matter: every face for the table path, the wrapped axes for the wrap path
    const int axes = kTable ? 7 : B.wrap;
    Face fc{0, 0};
    if (thr) {
        fc.lo = ((x == 0 ? 1 : 0) | (y == 0 ? 2 : 0)) & axes;
        fc.hi = ((x == B.nx - 1 ? 1 : 0) | (y == B.ny - 1 ? 2 : 0)) & axes;
    }
    for (int z = t.z0; z < zend; ++z) {
        const int64_t cell = B.cell(x, y, z);
        const uint32_t m = masked ? B.mask[cell] : 0u;
        if (m & kMaskSolid) continue;
        Face f2 = fc;
        if (thr) {
            f2.lo |= (z == 0 ? 4 : 0) & axes;
            f2.hi |= (z == B.nz - 1 ? 4 : 0) & axes;
        }
        const bool face = (f2.lo | f2.hi) != 0;
        if (!kThr) {
            if (masked && KIND != SWEEP_AA_LOCAL)
                update_cell<FORCE, KIND, DIAG, 0, true>(A, Bout, B, nb, f2, x, y, z, cell, m, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, 0, false>(A, Bout, B, nb, f2, x, y, z, cell, 0u, k, dg);
        } else if (__any_sync(__activemask(), face)) {
            constexpr int kFace = kTable ? 2 : 1;
            if (masked)
                update_cell<FORCE, KIND, DIAG, kFace, true>(A, Bout, B, nb, f2, x, y, z, cell, m, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, kFace, false>(A, Bout, B, nb, f2, x, y, z, cell, 0u, k, dg);
        } else {
            if (masked)
                update_cell<FORCE, KIND, DIAG, 0, true>(A, Bout, B, nb, f2, x, y, z, cell, m, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, 0, false>(A, Bout, B, nb, f2, x, y, z, cell, 0u, k, dg);
        }
    }
}

template <bool FORCE, int KIND, bool DIAG, int THROUGH>
__global__ void __launch_bounds__(256, DIAG ? kMinBDiag : kMinB)
    k_sweep(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock *__restrict__ blocks,
            const DevTile *__restrict__ tiles, int tx, int tz, Coll<R> k, double *__restrict__ partials)
{
    Diag<DIAG> dg;
    // every thread takes part in the block reduction, including those without cells
    sweep_cells<FORCE, KIND, DIAG, THROUGH>(A, Bout, blocks, tiles, tz, k, dg);
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

template <bool FORCE, int KIND, int THROUGH>
cudaError_t go(const SweepArgs &s, const Coll<R> &k)
{
    if (s.ntiles <= 0) return cudaSuccess;
    if (s.ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)s.ntiles), block((unsigned)(s.tx * s.ty));
    if (s.partials)
        k_sweep<FORCE, KIND, true, THROUGH><<<grid, block, 0, s.stream>>>((StoreT *)s.a, (StoreT *)s.b, s.blocks,
                                                                       s.tiles, s.tx, s.tz, k, s.partials);
    else
        k_sweep<FORCE, KIND, false, THROUGH><<<grid, block, 0, s.stream>>>((StoreT *)s.a, (StoreT *)s.b, s.blocks,
                                                                        s.tiles, s.tx, s.tz, k, nullptr);
    return cudaGetLastError();
}

template <bool FORCE>
cudaError_t go_kind(const SweepArgs &s, const Coll<R> &k)
{
    switch (s.kind) {
        case SWEEP_PULL:
            return s.through == 2 ? go<FORCE, SWEEP_PULL, 2>(s, k)
                                  : (s.through ? go<FORCE, SWEEP_PULL, 1>(s, k) : go<FORCE, SWEEP_PULL, 0>(s, k));
        case SWEEP_AA_LOCAL: return go<FORCE, SWEEP_AA_LOCAL, 0>(s, k);
        case SWEEP_AA_NBR:
            return s.through == 2 ? go<FORCE, SWEEP_AA_NBR, 2>(s, k)
                                  : (s.through ? go<FORCE, SWEEP_AA_NBR, 1>(s, k) : go<FORCE, SWEEP_AA_NBR, 0>(s, k));
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
