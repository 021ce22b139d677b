// cell.cuh -- cell-level pieces shared by the sweep and the closure sweep: gather and
// scatter of one cell in the two-grid / AA layouts (in-place neighbours, wrap, bounce-back
// bits), the per-CTA diagnostics record and the neighbour table staging.  Included after
// select.cuh by translation units compiled for one (stencil, storage) pair.
#pragma once

#include "cumulant.cuh"
#include "select.cuh"

namespace lbm {
namespace {

constexpr int kQ = LBM_Q;
using S = Storage<StoreT>;
using R = typename S::R;
// the collision relaxes the non-equilibrium parts first for full populations in FP32 (see
// collide in kernels.cuh); FP64 and the deviation storages take the pair form
constexpr bool kAccurate = LBM_ST == 1;
// MRT collision (group corrections on top of TRT) in this object's sweeps
constexpr bool kMrt = LBM_MRT_SWEEP != 0;
// cumulant collision in this object's sweeps (D3Q27, FP64 and FP32 storage)
constexpr bool kCum = LBM_CUMULANT_SWEEP != 0;
static_assert(!kCum || (kQ == 27 && LBM_ST <= 1), "cumulant sweeps are D3Q27 with FP64 or FP32 storage");

// The collision of this object's sweeps on the gathered values of one cell.
template <bool FORCE, bool RCP, int Q>
__device__ __forceinline__ void collide_cell(R (&f)[Q], const Coll<R> &k, R &rho, R &ux, R &uy, R &uz)
{
    if constexpr (kCum && Q == 27)
        collide_cumulant<FORCE, true>(f, k, rho, ux, uy, uz);
    else
        collide<Q, FORCE, R, kAccurate, kMrt, RCP>(f, k, k.r, k.rho0, rho, ux, uy, uz);
}

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

// Per-CTA diagnostics record of the cells this CTA updated (DIAG): mass, momentum (rho u,
// half-force corrected), kinetic energy, max |u|, non-finite cells, fluid cells.
//   Mass is the sum of the values the sweep stores (post-collision, after rounding to the
//   storage format), so it matches an FP64 sum over the stored field.  With FP32 arithmetic
//   each cell's values are summed without rounding error as a float-float pair: along the
//   cell's values by Fast2Sum (Dekker 1971: t = s + x, e = x - (t - s) gives s + x = t + e
//   exactly when the exponent of s is at least that of x -- the chain starts at rho0 for the
//   deviation storages, whose |x| stay far below it, and at the rest population for full
//   populations, which is at least every other population: w_0 >= 6 w_i), the error terms in
//   FP32; the cells of a thread by TwoSum (Knuth: b = t - s, e = (s - (t - b)) + (x - b), exact
//   whatever the magnitudes -- consecutive cell masses straddle powers of two).  A cell
//   contributes at most Q^2 u^2 rho of error (u = 2^-24).  The thread adds each cell's error
//   terms and its TwoSum error to its low part in FP32: with n cells those 2n additions round
//   by at most u/2 of a low part below (k + Q) u/2 of the running mass at cell k, at most
//   (2 Q n + n^2) u^2 of the thread's mass in all.
//   Momentum and kinetic energy come from the collision's moments and are accumulated per
//   thread with Kahan's compensated sum (error at most 2u of the sum of magnitudes, whatever
//   the number of cells).  With FP64 arithmetic the sums are plain FP64.  A cell counts as
//   non-finite when rho + |u|^2 is.
// The CTA's record with FP32 arithmetic stays in FP32 until its 8 results: the FP64 pipe of
// this GPU retires 2 lanes per clock per SM, so FP64 warp shuffles of 8 sums per tile of 4
// cells per thread cost more than the rest of the diagnostics.  Mass: the threads' float-float
// pairs are added pairwise (butterfly over the warp, then the warps in order), high parts by
// TwoSum, low parts in FP32 -- 12 additions on every path, each rounding the low part by at
// most u/2 of the low parts' magnitudes (<= (Q + n) u/2 of the mass), 3 (Q + n) u^2 more: the
// record's mass is within (Q + n + 3)^2 u^2 of the exact sum of the stored values (2.4e-12
// for D3Q19 at n = 4).  Momentum and energy: each thread's Kahan pair
// s - c rounded once (u of the magnitudes), then the same 12 plain FP32 additions (6 u);
// counts are integers below 2^24, exact; the maximum exact.  Then FP64.
// The running sums of a thread live in shared memory, column threadIdx.x of a [13][256]
// array (CTAs of at most 256 threads), not in registers: there they would stay live across
// the thread's whole z loop next to the cell's populations, which costs the sweep a CTA per SM
// or spills.  Each thread touches only its own column.
template <bool DIAG>
struct Diag {
    // slots: 0/1 mass (sum, error terms), 2-4 momentum, 5-7 their compensations, 8 sum rho
    // |u|^2, 9 its compensation, 10 max |u|^2, 11 non-finite cells, 12 cells
    static constexpr int kSlots = 13;
    static constexpr bool kComp = sizeof(R) == 4;
    static __device__ __forceinline__ R *home()
    {
        __shared__ R h[DIAG ? kSlots * 256 : 1];
        return h + threadIdx.x;
    }
    // s + x = t + e exactly (TwoSum)
    static __device__ __forceinline__ R two_sum(R s, R x, R &e)
    {
        const R t = s + x;
        const R b = t - s;
        e = (s - (t - b)) + (x - b);
        return t;
    }
    static __device__ __forceinline__ void kahan(R *s, R *c, R x)
    {
        const R y = x - *c;
        const R t = *s + y;
        *c = (t - *s) - y;
        *s = t;
    }
    __device__ __forceinline__ Diag()
    {
        if (!DIAG) return;
        R *h = home();
#pragma unroll
        for (int c = 0; c < kSlots; ++c) h[c * 256] = R(0);
    }
    // f: the cell's post-collision values as the sweep is about to store them (deviations
    // for the *_DEV storages), rho0: the deviation base (0 otherwise); rho, u: the collision's
    // moments.
    __device__ __forceinline__ void add(const R (&f)[kQ], R rho0, R rho, R ux, R uy, R uz)
    {
        if (!DIAG) return;
        R *h = home();
        const R u2 = ux * ux + uy * uy + uz * uz;
        if (kComp) {
            R m = rho0, e = R(0);
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                const R x = S::stored(f[i]);
                const R t = m + x;
                e += x - (t - m);  // Fast2Sum
                m = t;
            }
            R eh;
            h[0] = two_sum(h[0], m, eh);
            h[256] += eh + e;
            kahan(h + 512, h + 1280, rho * ux);
            kahan(h + 768, h + 1536, rho * uy);
            kahan(h + 1024, h + 1792, rho * uz);
            kahan(h + 2048, h + 2304, rho * u2);
        } else {
            h[0] += rho;
            h[512] = fma(rho, ux, h[512]);
            h[768] = fma(rho, uy, h[768]);
            h[1024] = fma(rho, uz, h[1024]);
            h[2048] = fma(rho, u2, h[2048]);
        }
        h[2560] = fmax(h[2560], u2);
        h[2816] += isfinite(rho + u2) ? R(0) : R(1);
        h[3072] += R(1);
    }
    // the thread's record in FP64: mass, momentum x/y/z, kinetic energy, max |u|, non-finite,
    // cells
    __device__ __forceinline__ void record(double (&v)[8]) const
    {
        if (!DIAG) return;
        const R *h = home();
        v[0] = (double)h[0] + (double)h[256];
        v[1] = (double)h[512] - (double)h[1280];
        v[2] = (double)h[768] - (double)h[1536];
        v[3] = (double)h[1024] - (double)h[1792];
        v[4] = 0.5 * ((double)h[2048] - (double)h[2304]);
        v[5] = sqrt((double)h[2560]);
        v[6] = (double)h[2816];
        v[7] = (double)h[3072];
    }
    // The CTA's record (every thread of the CTA calls this): warp shuffles, then the warps in
    // order; partials[blockIdx.x * 8 + c].
    __device__ __forceinline__ void tile_record(double *__restrict__ partials) const
    {
        if (!DIAG) return;
        if constexpr (kComp) {
            tile_record_f32(partials);
            return;
        }
        __shared__ double sh[8][8];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        double v[8];
        record(v);
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = c == 5 ? wmax(v[c]) : wsum(v[c]);
        if (lane == 0)
            for (int c = 0; c < 8; ++c) sh[warp][c] = v[c];
        __syncthreads();
        if (threadIdx.x < 8) {
            const int c = threadIdx.x;
            double r = 0.0;
            for (int w = 0; w < nw; ++w) r = c == 5 ? fmax(r, sh[w][c]) : r + sh[w][c];
            partials[(int64_t)blockIdx.x * 8 + c] = r;
        }
    }
    // FP32 form of the CTA's record (see above): slots 0 mass high, 1 mass low, 2-4 momentum,
    // 5 energy (x 2), 6 max |u|^2, 7 non-finite cells, 8 cells.
    static __device__ __forceinline__ float two_sum_f(float s, float x, float &e)
    {
        const float t = s + x;
        const float b = t - s;
        e = (s - (t - b)) + (x - b);
        return t;
    }
    __device__ __forceinline__ void tile_record_f32(double *__restrict__ partials) const
    {
        __shared__ float sf[8][9];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const R *h = home();
        float mh = h[0], ml = h[256];
        float v[7] = {h[512] - h[1280], h[768] - h[1536], h[1024] - h[1792], h[2048] - h[2304],
                      h[2560], h[2816], h[3072]};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, mh, o), bl = __shfl_xor_sync(0xffffffffu, ml, o);
            float e;
            mh = two_sum_f(mh, bh, e);
            ml = (ml + bl) + e;
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const float w = __shfl_xor_sync(0xffffffffu, v[c], o);
                v[c] = c == 4 ? fmaxf(v[c], w) : v[c] + w;
            }
        }
        if (lane == 0) {
            sf[warp][0] = mh;
            sf[warp][1] = ml;
#pragma unroll
            for (int c = 0; c < 7; ++c) sf[warp][2 + c] = v[c];
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            const int c = threadIdx.x;
            double r;
            if (c == 0) {
                float th = sf[0][0], tl = sf[0][1];
                for (int w = 1; w < nw; ++w) {
                    float e;
                    th = two_sum_f(th, sf[w][0], e);
                    tl = (tl + sf[w][1]) + e;
                }
                r = (double)th + (double)tl;
            } else {
                const int j = c + 1;  // slot of output c: momentum 2-4, energy 5, max 6, counts 7-8
                float t = sf[0][j];
                for (int w = 1; w < nw; ++w) t = c == 5 ? fmaxf(t, sf[w][j]) : t + sf[w][j];
                r = c == 4 ? 0.5 * (double)t : (c == 5 ? sqrt((double)t) : (double)t);
            }
            partials[(int64_t)blockIdx.x * 8 + c] = r;
        }
    }
};

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

// Index shifts that bring a neighbour across a wrapped face back into the block, per axis and
// side (lo: the cell is on the low face, the neighbour is at -1, shift +n stride; hi: -n
// stride), zero where the cell is not on that face.  Taken once per cell from its face flags.
struct WrapD {
    int32_t xl, xh, yl, yh;
    int64_t zl, zh;
};

__device__ __forceinline__ WrapD wrap_deltas(const DevBlock &B, Face f)
{
    WrapD w;
    w.xl = (f.lo & 1) ? B.nx : 0;
    w.xh = (f.hi & 1) ? -B.nx : 0;
    w.yl = (f.lo & 2) ? B.ny * B.pitch : 0;
    w.yh = (f.hi & 2) ? -B.ny * B.pitch : 0;
    w.zl = (f.lo & 4) ? (int64_t)B.nz * B.plane : 0;
    w.zh = (f.hi & 4) ? -(int64_t)B.nz * B.plane : 0;
    return w;
}

// Shift of the neighbour (x, y, z) + (DX, DY, DZ) (compile-time after unrolling).
__device__ __forceinline__ int64_t wrap_of(const WrapD &w, int DX, int DY, int DZ)
{
    const int32_t s = (DX < 0 ? w.xl : (DX > 0 ? w.xh : 0)) + (DY < 0 ? w.yl : (DY > 0 ? w.yh : 0));
    return (int64_t)s + (DZ < 0 ? w.zl : (DZ > 0 ? w.zh : 0));
}

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
// Gather the populations streaming into cell (x, y, z) (see the file header of sweep.cu), as
// stored: deviations f_i - w_i rho0 for the *_DEV storages (the collision works on them).
// I32: element indices in 32-bit arithmetic from the arena base, for arenas of at most 2^32
// elements per array (the host checks): every true index is then below 2^32, so the
// arithmetic modulo 2^32 gives it exactly, and one wide multiply-add forms the address.
template <int KIND, int FACE, bool MASK, bool I32 = false>
__device__ __forceinline__ void gather_cell(R (&f)[kQ], StoreT *__restrict__ A, const DevBlock &B, const NbrGeo *nb,
                                            Face fc, int x, int y, int z, int64_t cell, uint32_t m, const R *base)
{
    using L = Lattice<kQ>;
    StoreT *a = A + B.offset;
    const WrapD wd = FACE == 1 ? wrap_deltas(B, fc) : WrapD{};
    if constexpr (I32 && KIND != SWEEP_AA_LOCAL) {
        const uint32_t pitch = (uint32_t)B.pitch, plane = (uint32_t)B.plane, slab = (uint32_t)B.slab;
        const uint32_t own = (uint32_t)B.offset + (uint32_t)cell;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const bool bounce = MASK && i > 0 && ((m >> i) & 1u);
            const int sl = KIND == SWEEP_PULL ? i : L::opp(i);
            const int bs = KIND == SWEEP_PULL ? L::opp(i) : i;
            const uint32_t off = (uint32_t)L::cx(i) + (uint32_t)L::cy(i) * pitch + (uint32_t)L::cz(i) * plane;
            uint32_t o = bounce ? (uint32_t)bs * slab + own : (uint32_t)sl * slab + own - off;
            if (FACE == 1 && !bounce) o += (uint32_t)wrap_of(wd, -L::cx(i), -L::cy(i), -L::cz(i));
            if (FACE == 2 && !bounce)
                o = (uint32_t)nbr_addr(nb, fc, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i), sl, (int64_t)o);
            f[i] = KIND == SWEEP_PULL ? S::raw(A + o) : S::raw_rw(A + o);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
        const bool bounce = MASK && i > 0 && ((m >> i) & 1u);
        if (KIND == SWEEP_AA_LOCAL) {
            f[i] = S::raw_rw(a + (int64_t)i * B.slab + cell);
            continue;
        }
        const int sl = KIND == SWEEP_PULL ? i : L::opp(i);  // slot read from the source cell
        const int bs = KIND == SWEEP_PULL ? L::opp(i) : i;  // own slot read on bounce-back
        int64_t o = bounce ? (int64_t)bs * B.slab + cell : (int64_t)sl * B.slab + cell - off;
        if (FACE == 1 && !bounce) o += wrap_of(wd, -L::cx(i), -L::cy(i), -L::cz(i));
        if (FACE == 2 && !bounce)
            o = nbr_addr(nb, fc, x, y, z, -L::cx(i), -L::cy(i), -L::cz(i), sl, o + B.offset) - B.offset;
        f[i] = KIND == SWEEP_PULL ? S::raw(a + o) : S::raw_rw(a + o);
    }
}

// Scatter the post-collision populations of cell (x, y, z).
template <int KIND, int FACE, bool MASK, bool I32 = false>
__device__ __forceinline__ void scatter_cell(const R (&f)[kQ], StoreT *__restrict__ A, StoreT *__restrict__ Bout,
                                             const DevBlock &B, const NbrGeo *nb, Face fc, int x, int y, int z,
                                             int64_t cell, uint32_t m, const R *base)
{
    using L = Lattice<kQ>;
    StoreT *a = A + B.offset;
    // The neighbour sweep's store offsets equal its load offsets of the opposite directions;
    // hide the coordinates from the optimiser so it recomputes them here instead of keeping
    // 19 offsets live across the collision.
    int xs = x, ys = y, zs = z;
    Face fs = fc;
    if (KIND == SWEEP_AA_NBR) asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs), "+r"(fs.lo), "+r"(fs.hi));
    const WrapD wd = (FACE == 1 && KIND == SWEEP_AA_NBR) ? wrap_deltas(B, fs) : WrapD{};
    if constexpr (I32 && KIND == SWEEP_AA_NBR) {
        const uint32_t pitch = (uint32_t)B.pitch, plane = (uint32_t)B.plane, slab = (uint32_t)B.slab;
        const uint32_t own = (uint32_t)B.offset + (uint32_t)B.cell(xs, ys, zs);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const int o = L::opp(i);
            const bool bounce = MASK && i > 0 && ((m >> o) & 1u);
            const uint32_t off = (uint32_t)L::cx(i) + (uint32_t)L::cy(i) * pitch + (uint32_t)L::cz(i) * plane;
            uint32_t d = bounce ? (uint32_t)o * slab + own : (uint32_t)i * slab + own + off;
            if (FACE == 1 && !bounce) d += (uint32_t)wrap_of(wd, L::cx(i), L::cy(i), L::cz(i));
            if (FACE == 2 && !bounce)
                d = (uint32_t)nbr_addr(nb, fs, xs, ys, zs, L::cx(i), L::cy(i), L::cz(i), i, (int64_t)d);
            S::st_raw(A + d, f[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int64_t off = dir_offset<kQ>(i, B.pitch, B.plane);
        if (KIND == SWEEP_PULL) {
            S::st_raw(Bout + B.offset + (int64_t)i * B.slab + cell, f[i]);
        } else if (KIND == SWEEP_AA_LOCAL) {
            const int o = L::opp(i);
            S::st_raw(a + (int64_t)o * B.slab + cell, f[i]);
        } else {
            const int o = L::opp(i);
            const bool bounce = MASK && i > 0 && ((m >> o) & 1u);
            const int64_t c2 = B.cell(xs, ys, zs);
            int64_t d = bounce ? (int64_t)o * B.slab + c2 : (int64_t)i * B.slab + c2 + off;
            if (FACE == 1 && !bounce) d += wrap_of(wd, L::cx(i), L::cy(i), L::cz(i));
            if (FACE == 2 && !bounce)
                d = nbr_addr(nb, fs, xs, ys, zs, L::cx(i), L::cy(i), L::cz(i), i, d + B.offset) - B.offset;
            S::st_raw(a + d, f[i]);
        }
    }
}

// One cell: gather, collide, scatter.  FACE: the warp has cells on a face of a block that
// reads its neighbours in place; directions that leave the block there are wrapped (FACE 1:
// the block is its own neighbour) or resolved through the shared-memory neighbour table
// (FACE 2).  m: the cell's bounce-back bits (bit i: the source x - c_i is a no-slip cell;
// halfway bounce-back then supplies f_i(x, t+1) = f*_opp(i)(x, t), read from the cell's own
// slot).
//   pull: bounce source src[opp i][x]
//   AA neighbour: bounce source A[i][x] (where the E layout keeps f*_opp(i)(x)); the value
//   f*_i(x) whose target x + c_i is no-slip (bit opp(i)) goes to A[opp i][x], where the next
//   local sweep reads it as f_opp(i)(x, t+1).
template <bool FORCE, int KIND, bool DIAG, int FACE, bool MASK, bool I32 = false>
__device__ __forceinline__ void update_cell(StoreT *__restrict__ A, StoreT *__restrict__ Bout, const DevBlock &B,
                                            const NbrGeo *nb, Face fc, int x, int y, int z, int64_t cell, uint32_t m,
                                            const Coll<R> &k, Diag<DIAG> &dg)
{
    R f[kQ];
    gather_cell<KIND, FACE, MASK, I32>(f, A, B, nb, fc, x, y, z, cell, m, k.base);
    R rho, ux, uy, uz;
    constexpr bool kRcp = !(KIND == SWEEP_AA_NBR && sizeof(R) == 4);
    collide_cell<FORCE, kRcp>(f, k, rho, ux, uy, uz);
    dg.add(f, k.rho0, rho, ux, uy, uz);
    scatter_cell<KIND, FACE, MASK, I32>(f, A, Bout, B, nb, fc, x, y, z, cell, m, k.base);
}

// Copy the scalar geometry of a block into registers (its neighbour table stays out).
__device__ __forceinline__ DevBlock block_geo(const DevBlock *Bp)
{
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
    return B;
}

// ---- bulk-copy staging of source rows (two-grid pull sweep) ---------------------------------
// Limit of one bounded wait on a staging mbarrier, in nanoseconds of the global timer.  A bulk
// copy of a few kilobytes lands in microseconds; a wait that reaches this limit is a fault.
constexpr uint64_t kStageWaitNs = 1000000000ull;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of an mbarrier: polls until the phase completes or
// kStageWaitNs have passed since the first poll; false when it gave up.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kStageWaitNs) return false;
    }
}

__device__ __forceinline__ void stage_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void stage_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy (TMA, non-tensor) of `bytes` from global to shared memory, completing on *bar.
// Both addresses 16-byte aligned, bytes a multiple of 16 (the plan only stages such rows).
__device__ __forceinline__ void stage_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(dst)),
        "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
        : "memory");
}

// Fill the shared-memory neighbour table of block *Bp (threads 0..26; caller syncs).
__device__ __forceinline__ void stage_neighbours(NbrGeo *nb, const DevBlock *__restrict__ blocks, const DevBlock *Bp)
{
    if (threadIdx.x < 27) {
        const int r = threadIdx.x;
        const int n = (Bp->through && r != 13) ? Bp->nbr[r] : -1;
        NbrGeo g{};
        if (n >= 0) {
            const DevBlock *N = blocks + n;
            g = NbrGeo{N->offset, N->slab, N->plane, N->pitch, N->xo, N->nx, N->ny, N->nz, 1};
        }
        nb[r] = g;
    }
}

}  // namespace
}  // namespace lbm
