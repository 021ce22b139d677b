// launch.hpp -- host-side launch interface between the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace lbm {

enum SweepKind { SWEEP_PULL = 0, SWEEP_AA_LOCAL = 1, SWEEP_AA_NBR = 2 };
enum FillMode { FILL_PULL = 0, FILL_AA_E = 1, FILL_AA_O = 2 };
enum Layout { LAYOUT_PULL = 0, LAYOUT_AA_E = 1, LAYOUT_AA_O = 2 };

// Shared-memory buffers (one z step of source rows each) of a staged sweep tile; the sweep and
// the host's shared-memory size both take it from here
constexpr int kSweepStages = 2;
// staged 16-bit tiles: two x-adjacent cells per thread over pairs of one-row tiles
#ifndef LBM_STAGED_TWO
#define LBM_STAGED_TWO 1
#endif

struct SweepArgs {
    void *a;  // two-grid source / AA array
    void *b;  // two-grid destination (unused for AA)
    const DevBlock *blocks;
    const DevTile *tiles;
    int64_t ntiles;
    int tx, ty, tz;
    int kind;   // SweepKind
    int force;  // body force non-zero
    double *partials;  // non-null: write per-CTA diagnostics records (8 doubles per tile)
    int through;       // in-place neighbours: 0 none, 1 only the block itself (wrap), 2 other blocks
    size_t stage_bytes;  // dynamic shared memory of the staged tiles (DevTile flag bit 1), 0: none
    int *err;            // device flag: a bounded wait gave up
    int idx32;           // every element index of a PDF array is below 2^32 (32-bit index arithmetic)
    Coll<double> cd;
    Coll<float> cf;
    cudaStream_t stream;
};

struct FillArgs {
    void *a;  // array holding the state the next sweep reads
    const DevBlock *blocks;
    const uint64_t *links;
    int64_t nlinks;
    const DevRun *runs;
    int64_t nruns;
    const double *params;  // wall table: (ux, uy, uz, rho) per entry (the six faces first)
    int mode;              // FillMode
    const uint64_t *zouhe;  // wet-node entries (plan.hpp pack_zouhe), two-grid only
    int64_t nzouhe;
    int zouhe_pressure;     // bit f: face f is a wet-node pressure face (else velocity)
    double F[3];
    double base[27];
    cudaStream_t stream;
};

// Halo pack / unpack of a partitioned run (halo.cu): element moves between the PDF array and a
// caller-owned buffer along runs (the device copy of plan.hpp HaloRun).
struct HaloDevRun {
    int64_t arena;
    int64_t buf;
    int32_t len;
    int32_t astride;
};
struct HaloArgs {
    void *arena;  // the PDF array the next sweep reads
    void *buf;    // device buffer of the exchange with one peer
    const HaloDevRun *runs;
    int64_t nruns;
    int to_buf;      // 1: pack (arena -> buffer), 0: unpack
    int elem_bytes;  // 8, 4 or 2
    cudaStream_t stream;
};
cudaError_t launch_halo(const HaloArgs &h);

// The fluid-cell list layout of the two-grid sweep (sweep_sparse.cu, plan.hpp SparsePlan).
enum SparseOp { SPARSE_SWEEP = 0, SPARSE_FILL = 1, SPARSE_TO_LIST = 2, SPARSE_TO_DENSE = 3 };
// table entry of a no-slip source: halfway bounce-back from the cell's own opposite slot
// (the same value as plan.hpp kSparseBounce)
constexpr int32_t kListBounce = (int32_t)0x80000000u;
struct SparseArgs {
    int op;
    const void *src;  // sweep: source list array
    void *dst;        // sweep: destination list array; fill: the array the next sweep reads
    void *dense;      // copies: a dense PDF array
    void *list;       // copies: a list array
    const int32_t *nbr;       // (Q - 1) x nfluid pull sources
    const uint64_t *links;    // link words (fill)
    int64_t nlinks;
    const double *params;     // wall table (fill)
    const DevBlock *blocks;   // copies
    const int32_t *block_of;  // copies
    const int64_t *cell_of;   // copies
    int64_t nfluid;
    int64_t stride;   // entries per direction (>= nfluid + links, padded)
    int force;
    double *partials;  // sweep: per-CTA diagnostics records or null
    Coll<double> cd;
    Coll<float> cf;
    cudaStream_t stream;
};

// Per-cell kernels over the interior cells of one block (get/set/macroscopic/init).
struct CellArgs {
    void *a;
    const DevBlock *blocks;  // device block table
    int block;               // this block's index in it
    DevBlock blk;
    int layout;  // Layout of the stored state
    double *f64;        // get: out f[Q*N]; set: in
    double *rho, *u;    // macroscopic out; init: in (rho[N], u[3N])
    const uint32_t *mask;
    int ratio;  // coarse: edge of the coarse cell in interior cells
    int r0[3], rn[3];  // get: box origin and size in interior cells (rn[0] == 0: the whole block)
    double F[3];
    double base[27];
    Coll<double> cd;
    Coll<float> cf;
    cudaStream_t stream;
};

struct ReduceArgs {
    const void *a;
    const DevBlock *blocks;
    const DevTile *tiles;
    int64_t ntiles;
    int tx, ty, tz;
    int layout;
    double F[3];
    double base[27];
    double *partials;  // ntiles * 8 doubles
    double *out;       // reduce_final_scratch(ntiles) doubles (device); results in out[0..7]
    cudaStream_t stream;
};

inline const Coll<double> &coll_of(const Coll<double> &d, const Coll<float> &, double *) { return d; }
inline const Coll<float> &coll_of(const Coll<double> &, const Coll<float> &f, float *) { return f; }

// Cell-kernel operations of launch_cells.
enum CellOp { CELL_INIT = 0, CELL_GET = 1, CELL_SET = 2, CELL_MACRO = 3, CELL_COARSE = 4 };

// Entry points of the per-(stencil, storage) objects; storage 0 fp64, 1 fp32, 2 bf16-dev,
// 3 fp16-dev.  sweep.cu defines launch_sweep_<Q>_<ST>; aux.cu the other three.
// Second pass of the diagnostics: fixed-order sum of n per-CTA records into out[8].
// out must hold reduce_final_scratch(n) doubles: the 8 results, then the first-level records.
cudaError_t launch_reduce_final(const double *partials, int64_t n, double *out, cudaStream_t s);
// One thread waits `polls` polls on an mbarrier that never completes and sets *err = 2.
cudaError_t launch_wait_selfcheck(int *err, uint32_t polls, cudaStream_t s);
int64_t reduce_final_scratch(int64_t n);
// The same sum written to slot[0..7] (device address of page-locked host memory), with *err0
// and *err1 (device flags, either may be null: 0) copied to slot_err[0..1]; scratch as out above.
cudaError_t launch_reduce_final_slot(const double *partials, int64_t n, double *scratch, double *slot, int *slot_err,
                                     const int *err0, const int *err1, cudaStream_t s);
// Per-block second pass: block b sums the records of tiles start[b] .. start[b+1] - 1 (tiles
// are stored block by block) into out[8 b .. 8 b + 7].
cudaError_t launch_block_final(const double *partials, const int64_t *start, int64_t nblocks, double *out,
                               cudaStream_t s);

#define LBM_DECLARE(Q, ST)                                                  \
    cudaError_t launch_sweep_##Q##_##ST(const SweepArgs &s);                \
    cudaError_t launch_fill_##Q##_##ST(const FillArgs &s);                  \
    cudaError_t launch_zouhe_##Q##_##ST(const FillArgs &s);                 \
    cudaError_t launch_cells_##Q##_##ST(int op, int force, const CellArgs &s); \
    cudaError_t launch_reduce_##Q##_##ST(const ReduceArgs &s);
LBM_DECLARE(19, 0)
LBM_DECLARE(19, 1)
LBM_DECLARE(19, 2)
LBM_DECLARE(19, 3)
LBM_DECLARE(27, 0)
LBM_DECLARE(27, 1)
LBM_DECLARE(27, 2)
LBM_DECLARE(27, 3)
#undef LBM_DECLARE
#define LBM_DECLARE_SPARSE(Q, ST) cudaError_t launch_sparse_##Q##_##ST(const SparseArgs &s);
LBM_DECLARE_SPARSE(19, 0)
LBM_DECLARE_SPARSE(19, 1)
LBM_DECLARE_SPARSE(19, 2)
LBM_DECLARE_SPARSE(19, 3)
LBM_DECLARE_SPARSE(27, 0)
LBM_DECLARE_SPARSE(27, 1)
LBM_DECLARE_SPARSE(27, 2)
LBM_DECLARE_SPARSE(27, 3)
#undef LBM_DECLARE_SPARSE
// MRT sweeps (FP64 and FP32 storage)
cudaError_t launch_sweep_mrt_19_0(const SweepArgs &s);
cudaError_t launch_sweep_mrt_19_1(const SweepArgs &s);
cudaError_t launch_sweep_mrt_27_0(const SweepArgs &s);
cudaError_t launch_sweep_mrt_27_1(const SweepArgs &s);
// cumulant sweeps (D3Q27, FP64 and FP32 storage)
cudaError_t launch_sweep_cum_27_0(const SweepArgs &s);
cudaError_t launch_sweep_cum_27_1(const SweepArgs &s);

// Static 2:1 refinement coupling of a coarse and a fine context (refine.cu), FP64 or FP32
// storage (elem_bytes 8 or 4).  Offsets are elements relative to the arrays' bases.
//   explode:  dst[e[3k]] = src[e[3k + sub]]            (sub 1 or 2; src the coarse state)
//   coalesce: dst[e[9k]] = (sum_{j=1..4} src[e[9k + j]] + sum_{j=5..8} src2[e[9k + j]]) / 8
//             (src the fine state after the first of the two fine steps, src2 the one before it)
struct RefineArgs {
    void *dst;
    const void *src, *src2;
    const int64_t *ent;
    int64_t n;
    int elem_bytes;
    int sub;
    cudaStream_t stream;
};
cudaError_t launch_refine_explode(const RefineArgs &a);
cudaError_t launch_refine_coalesce(const RefineArgs &a);

}  // namespace lbm
