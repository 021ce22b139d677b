// sweep.cu -- fused stream-collide sweeps (two-grid pull, AA local, AA neighbour).
//
// Compiled once per (stencil, storage) pair: -DLBM_Q=19|27 -DLBM_ST=0..3 (fp64, fp32,
// bf16-deviation, fp16-deviation).  Each object defines launch_sweep_<Q>_<ST>; with -DLBM_MRT_SWEEP=1
// (FP64 and FP32 storage) the same sweeps with the MRT collision, launch_sweep_mrt_<Q>_<ST>;
// with -DLBM_CUMULANT_SWEEP=1 (D3Q27, FP64 and FP32 storage) with the cumulant collision,
// launch_sweep_cum_27_<ST>.
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
#include "cell.cuh"

// Occupancy: minimum resident CTAs of 256 threads per SM.  For 4- and 2-byte storage, 4
// caps the sweeps at 64 registers (1024 threads per SM); measured on the 256^3 channel it
// beats the uncapped build by 6 % (two-grid) and 23 % (AA neighbour sweep).  D3Q27 with FP32
// storage needs 80 registers (3: 21 % faster than 4 on the 512^3 AA turbulence box, 2 slower).
// The FP64 sweep is bound by the FP64 pipe, not by memory parallelism: 2 CTAs per SM avoid
// spilling.
#ifndef LBM_SWEEP_MINB
#if LBM_ST == 0
#define LBM_SWEEP_MINB 2
#elif LBM_Q == 27 && LBM_ST == 1
#define LBM_SWEEP_MINB 3
#else
#define LBM_SWEEP_MINB 4
#endif
#endif

namespace lbm {

namespace {

// The diagnostics variant (DIAG) keeps its running sums in shared memory (Diag), so it runs
// at the occupancy of the plain sweep.
constexpr int kMinB = LBM_SWEEP_MINB;
#ifdef LBM_SWEEP_MINB_DIAG
constexpr int kMinBDiag = LBM_SWEEP_MINB_DIAG;
#else
constexpr int kMinBDiag = LBM_SWEEP_MINB;
#endif

// Staged tile of the two-grid pull sweep (DevTile flag bit 1, set by the host only for 16-bit
// storage and for tiles that span their block's full width in at most two rows, carry no
// masks, belong to a block whose in-place neighbours are only itself, and whose rows
// x = -8 .. nx + 7 lie inside the padded row with 16-byte aligned start and length).  For every
// z step the 19 (27) source rows (y - c_y, z - c_z) of the tile's rows are brought into shared
// memory by bulk copies, one step ahead, double-buffered on two mbarriers (a CTA barrier per
// step frees a buffer: waiting warps are parked, where polling an "empty" mbarrier instead
// costs issue slots this issue-bound sweep does not have).  A thread reads its populations
// there (x - c_x, wrapped within the row when the block is its own x neighbour).  Wrapped y
// and z rows are mapped when the copies are issued.
// Failure path: a wait that gives up (stage_wait, limit in time) is made CTA-wide at the
// step's barrier; the CTA then issues no further copies and skips the remaining steps, thread
// 0 waits (bounded again) for the copies still in flight into its shared memory, and *err is
// set to 1.  A CTA that starts after another one gave up (*err == 1) does nothing.  The state
// is invalid after a give-up and the host reports it as such.
constexpr int kStages = kSweepStages;

// Two x-adjacent cells per thread in staged tiles that pair two rows (DevTile flag bit 2, set
// by the host when LBM_STAGED_TWO is on): the pair's loads along c_x = 0 are one 32-bit
// shared-memory load, its 19 (27) stores are packed 32-bit stores (two 16-bit values, one
// conversion instruction), and one store address serves both cells.  Measured on the 256^3
// channel: 0.2764 vs 0.2865 ms per FP16 step (packing the first cell's results into 16-bit
// pairs while the second collides, to save registers, gave 0.2865; three CTAs per SM instead of
// four, 0.2942).
template <class T>
struct Pair16 {  // generic form (the staged path is only taken for 16-bit storage)
    static __device__ __forceinline__ void ld(const T *p, R &a, R &b)
    {
        a = Storage<T>::raw_rw(p);
        b = Storage<T>::raw_rw(p + 1);
    }
    static __device__ __forceinline__ void st(T *p, R a, R b)
    {
        Storage<T>::st_raw(p, a);
        Storage<T>::st_raw(p + 1, b);
    }
};
template <>
struct Pair16<__half> {
    static __device__ __forceinline__ void ld(const __half *p, R &a, R &b)
    {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st(__half *p, R a, R b)
    {
        __stcs(reinterpret_cast<__half2 *>(p), __floats2half2_rn(a, b));
    }
};
template <>
struct Pair16<__nv_bfloat16> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, R &a, R &b)
    {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, R a, R b)
    {
        __stcs(reinterpret_cast<__nv_bfloat162 *>(p), __floats2bfloat162_rn(a, b));
    }
};

template <bool FORCE, bool DIAG>
__device__ __forceinline__ void sweep_staged(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock &B,
                                             const DevTile &t, int tz, const Coll<R> &k, Diag<DIAG> &dg,
                                             unsigned char *smem, int *err)
{
    using L = Lattice<kQ>;
    constexpr int NS = kStages;
    const int nx = B.nx, RW = nx + 16;
    const bool two = LBM_STAGED_TWO && (t.flags & 4) != 0;  // two cells per thread, two rows per tile
    const int tpr = two ? nx / 2 : nx;            // threads per row
    const int rows = two ? 2 : blockDim.x / nx;
    const int nrows = min(rows, B.ny - (int)t.y0);  // rows of the tile inside the block
    const uint32_t rowbytes = (uint32_t)nx * (uint32_t)sizeof(StoreT);  // x = 0 .. nx - 1, 128-byte aligned
    constexpr uint32_t kHalo = 8 * sizeof(StoreT);                        // x = -8 .. -1 or nx .. nx + 7
    StoreT *buf = reinterpret_cast<StoreT *>(smem);
    // full[s]: the copies of the step in stage s have landed
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)NS * kQ * rows * RW * sizeof(StoreT));
    const int tid = threadIdx.x;
    const int lx = tid % tpr, ly = tid / tpr;
    const bool active = ly < nrows;
    const int x = two ? 2 * lx : lx, y = t.y0 + ly;
    const int z0 = t.z0, zend = min(z0 + tz, B.nz);
    const bool wx = (B.wrap & 1) && B.through, wy = (B.wrap & 2) && B.through, wz = (B.wrap & 4) && B.through;
    int qx = 0;  // directions with c_x != 0: they read one element beyond the row
#pragma unroll
    for (int i = 0; i < kQ; ++i) qx += L::cx(i) != 0;
    const uint32_t stepbytes = (uint32_t)nrows * ((uint32_t)kQ * rowbytes + (wx ? 0u : (uint32_t)qx * kHalo));
    if (tid == 0) {
        for (int b = 0; b < NS; ++b) stage_init(&full[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // skip the tile when an earlier CTA of this launch (or of an earlier one) already gave up
    const bool healthy = tid != 0 || !err || *(volatile int *)err != 1;
    if (!__syncthreads_and(healthy)) return;
    const StoreT *a = A + B.offset;
    const int lane = tid & 31;
    // The copies of one step, issued by the lanes of warp 0 (one row each).  Only the row's own
    // 128-byte lines are copied: with the x wrap in place the row is its own neighbour; otherwise
    // the one ghost element a direction reads comes with a 16-byte copy on that side only.
    auto issue = [&](int zz, int st) {
        if (lane == 0) stage_expect(&full[st], stepbytes);
        __syncwarp();
        for (int c = lane; c < kQ * nrows; c += 32) {
            const int i = c / nrows, r = c - i * nrows;
            int yy = t.y0 + r - L::cy(i), zs = zz - L::cz(i);
            if (wy) yy = yy < 0 ? yy + B.ny : (yy >= B.ny ? yy - B.ny : yy);
            if (wz) zs = zs < 0 ? zs + B.nz : (zs >= B.nz ? zs - B.nz : zs);
            const StoreT *src = a + (int64_t)i * B.slab + (int64_t)(zs + 1) * B.plane + (int64_t)(yy + 1) * B.pitch + B.xo;
            StoreT *dst = buf + ((size_t)(st * kQ + i) * rows + r) * RW + 8;
            stage_copy(dst, src, rowbytes, &full[st]);
            if (!wx && L::cx(i) != 0) {
                const int h = L::cx(i) > 0 ? -8 : nx;
                stage_copy(dst + h, src + h, kHalo, &full[st]);
            }
        }
    };
    if (tid < 32)
        for (int j = 0; j < NS && z0 + j < zend; ++j) issue(z0 + j, j);
    int z = z0;
    bool ok = true;  // CTA-wide: the same in every thread after each step's barrier
    for (; z < zend; ++z) {
        const int st = (z - z0) % NS;
        const bool landed = stage_wait(&full[st], ((z - z0) / NS) & 1);
#if LBM_STAGED_TWO
        if (active && landed && two) {
            // cells x and x + 1 (x even: the pair's slots are 4-byte aligned in shared memory
            // and in the arena)
            R fa[kQ], fb[kQ];
            const StoreT *row0 = buf + (size_t)st * kQ * rows * RW + (size_t)ly * RW + 8;
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                const StoreT *row = row0 + (size_t)i * rows * RW;
                if (L::cx(i) == 0) {
                    Pair16<StoreT>::ld(row + x, fa[i], fb[i]);
                } else {
                    int ea = x - L::cx(i), eb = ea + 1;
                    if (wx) {
                        ea = ea < 0 ? ea + nx : (ea >= nx ? ea - nx : ea);
                        eb = eb < 0 ? eb + nx : (eb >= nx ? eb - nx : eb);
                    }
                    fa[i] = S::raw_rw(row + ea);
                    fb[i] = S::raw_rw(row + eb);
                }
            }
            R rho, ux, uy, uz;
            collide_cell<FORCE, true>(fa, k, rho, ux, uy, uz);
            dg.add(fa, k.rho0, rho, ux, uy, uz);
            collide_cell<FORCE, true>(fb, k, rho, ux, uy, uz);
            dg.add(fb, k.rho0, rho, ux, uy, uz);
            StoreT *o = Bout + B.offset + B.cell(x, y, z);
#pragma unroll
            for (int i = 0; i < kQ; ++i) Pair16<StoreT>::st(o + (int64_t)i * B.slab, fa[i], fb[i]);
        } else
#endif
        if (active && landed) {
            R f[kQ];
            const StoreT *row0 = buf + (size_t)st * kQ * rows * RW + (size_t)ly * RW + 8;
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                int e = x - L::cx(i);
                if (L::cx(i) != 0 && wx) e = e < 0 ? e + nx : (e >= nx ? e - nx : e);
                f[i] = S::raw_rw(row0 + (size_t)i * rows * RW + e);
            }
            R rho, ux, uy, uz;
            collide_cell<FORCE, true>(f, k, rho, ux, uy, uz);
            dg.add(f, k.rho0, rho, ux, uy, uz);
            const int64_t cell = B.cell(x, y, z);
#pragma unroll
            for (int i = 0; i < kQ; ++i) S::st_raw(Bout + B.offset + (int64_t)i * B.slab + cell, f[i]);
        }
        ok = __syncthreads_and(landed);  // every thread is done with stage st
        if (!ok) break;
        if (tid < 32 && z + NS < zend) issue(z + NS, st);
    }
    if (!ok) {
        // steps z .. z + NS - 1 have copies issued that may not have landed; thread 0 keeps the
        // CTA (and its shared memory) alive until they do, within the same bounded wait
        if (tid == 0) {
            for (int j = 0; j < NS && z + j < zend; ++j)
                stage_wait(&full[(z + j - z0) % NS], ((z + j - z0) / NS) & 1);
            if (err) atomicExch(err, 1);
        }
    }
}

// The cells of one tile.  A thread owns one (x, y) column and walks the tile's z range.  A
// warp with a cell on a face of a block that reads its neighbours in place takes the
// resolving path, all other warps the plain one (the test is warp-uniform, so neither path
// diverges); THROUGH = some block of the launch reads its neighbours in place.
template <bool FORCE, int KIND, bool DIAG, int THROUGH, bool I32>
__device__ __forceinline__ void sweep_cells(StoreT *__restrict__ A, StoreT *__restrict__ Bout,
                                            const DevBlock *__restrict__ blocks, const DevTile *__restrict__ tiles,
                                            int tz, const Coll<R> &k, Diag<DIAG> &dg, unsigned char *smem, int *err)
{
    const DevTile t = tiles[blockIdx.x];
    const DevBlock *Bp = blocks + t.block;
    const DevBlock B = block_geo(Bp);  // scalar geometry in registers
    if (KIND == SWEEP_PULL && THROUGH != 2 && LBM_ST >= 2 && (t.flags & 2)) {
        // bit 3: the tile's row is swept by the two-row tile before it (two cells per thread)
        if (!(t.flags & 8)) sweep_staged<FORCE, DIAG>(A, Bout, B, t, tz, k, dg, smem, err);
        return;
    }
    constexpr bool kThr = THROUGH != 0 && KIND != SWEEP_AA_LOCAL;
    constexpr bool kTable = THROUGH == 2 && KIND != SWEEP_AA_LOCAL;
    __shared__ NbrGeo nb[kTable ? 27 : 1];
    if (kTable) {
        stage_neighbours(nb, blocks, Bp);
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
                update_cell<FORCE, KIND, DIAG, 0, true, I32>(A, Bout, B, nb, f2, x, y, z, cell, m, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, 0, false, I32>(A, Bout, B, nb, f2, x, y, z, cell, 0u, k, dg);
        } else if (__any_sync(__activemask(), face)) {
            constexpr int kFace = kTable ? 2 : 1;
            if (masked)
                update_cell<FORCE, KIND, DIAG, kFace, true, I32>(A, Bout, B, nb, f2, x, y, z, cell, m, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, kFace, false, I32>(A, Bout, B, nb, f2, x, y, z, cell, 0u, k, dg);
        } else {
            if (masked)
                update_cell<FORCE, KIND, DIAG, 0, true, I32>(A, Bout, B, nb, f2, x, y, z, cell, m, k, dg);
            else
                update_cell<FORCE, KIND, DIAG, 0, false, I32>(A, Bout, B, nb, f2, x, y, z, cell, 0u, k, dg);
        }
    }
}

template <bool FORCE, int KIND, bool DIAG, int THROUGH, bool I32>
__global__ void __launch_bounds__(256, DIAG ? kMinBDiag : kMinB)
    k_sweep(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock *__restrict__ blocks,
            const DevTile *__restrict__ tiles, int tx, int tz, Coll<R> k, double *__restrict__ partials,
            int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char stage_smem[];
    Diag<DIAG> dg;
    // every thread takes part in the block reduction, including those without cells
    sweep_cells<FORCE, KIND, DIAG, THROUGH, I32>(A, Bout, blocks, tiles, tz, k, dg, stage_smem, err);
    dg.tile_record(partials);
}

template <bool FORCE, int KIND, bool DIAG, int THROUGH, bool I32 = false>
cudaError_t go1(const SweepArgs &s, const Coll<R> &k, size_t smem)
{
    dim3 grid((unsigned)s.ntiles), block((unsigned)(s.tx * s.ty));
    // static shared memory (diagnostics sums, neighbour table) counts against the 48 KB that
    // need no opt-in, so larger staging buffers opt in with a margin for it
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<FORCE, KIND, DIAG, THROUGH, I32>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_sweep<FORCE, KIND, DIAG, THROUGH, I32><<<grid, block, smem, s.stream>>>((StoreT *)s.a, (StoreT *)s.b, s.blocks,
                                                                        s.tiles, s.tx, s.tz, k, s.partials, s.err);
    return cudaGetLastError();
}

template <bool FORCE, int KIND, int THROUGH>
cudaError_t go(const SweepArgs &s, const Coll<R> &k)
{
    if (s.ntiles <= 0) return cudaSuccess;
    if (s.ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    // shared memory of the staged tiles (pull sweep only)
    const size_t smem = (KIND == SWEEP_PULL && THROUGH != 2 && LBM_ST >= 2) ? s.stage_bytes : 0;
    // the neighbour sweep spends its issue slots on 38 neighbour addresses per cell: 32-bit
    // index arithmetic where the arena allows it (measured on the 256^3 channel: FP32 AA
    // 0.890 -> 0.903 of HBM, FP16 AA 0.573 -> 0.616)
    // (and the pull sweep's gather where the collision, not memory, bounds the sweep: MRT and
    // cumulant objects)
    if constexpr (KIND == SWEEP_AA_NBR || (KIND == SWEEP_PULL && (kMrt || kCum))) {
        if (s.idx32 && smem == 0)
            return s.partials ? go1<FORCE, KIND, true, THROUGH, true>(s, k, smem)
                              : go1<FORCE, KIND, false, THROUGH, true>(s, k, smem);
    }
    return s.partials ? go1<FORCE, KIND, true, THROUGH>(s, k, smem) : go1<FORCE, KIND, false, THROUGH>(s, k, smem);
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

#if LBM_MRT_SWEEP
cudaError_t LBM_CAT(launch_sweep_mrt_, LBM_Q, LBM_ST)(const SweepArgs &s)
#elif LBM_CUMULANT_SWEEP
cudaError_t LBM_CAT(launch_sweep_cum_, LBM_Q, LBM_ST)(const SweepArgs &s)
#else
cudaError_t LBM_CAT(launch_sweep_, LBM_Q, LBM_ST)(const SweepArgs &s)
#endif
{
    if (s.tx * s.ty > 256 || s.tx % 32 != 0) return cudaErrorInvalidConfiguration;
    const Coll<R> &k = coll_of(s.cd, s.cf, (R *)nullptr);
    return s.force ? go_kind<true>(s, k) : go_kind<false>(s, k);
}

}  // namespace lbm
