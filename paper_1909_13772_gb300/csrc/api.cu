// api.cu -- the C ABI (include/lbm.h): context, device memory, list upload and the step
// scheduler.  Every step runs on the context's stream as two launches:
//   two-grid:  fill(links + ghost runs into src) -> pull sweep src -> dst, swap
//   AA:        fill(E) -> neighbour sweep  |  fill(O) -> local sweep   (alternating)
// (Sec. 4.2: ghost layers of neighbouring blocks are brought up to date around each sweep;
// Sec. 4.4: each boundary list is handled by its own kernel; Sec. 5.1.2: one fused
// stream-collide sweep.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "closure.hpp"
#include "lbm.h"
#include "launch.hpp"
#include "plan.hpp"

using namespace lbm;

struct lbm_ctx {
    lbm_params p{};
    int q = 19, storage = 1, pattern = 0, bpp = 4;
    bool force = false;
    std::vector<BlockLayout> blocks;
    std::vector<std::vector<uint8_t>> flags;
    std::vector<WallParam> block_param;
    int face_kind[6];
    WallParam face_param[6];
    int tile[3] = {256, 1, 4};
    int in_place = 1;  // read matching neighbour blocks in place (else ghost copies)
    int64_t arena_elems = 0;
    cudaStream_t stream = nullptr;
    // partitioned run (lbm_create_partition): owner rank of every block, this context's rank;
    // empty owner: the context owns every block
    std::vector<int32_t> owner;
    int rank = 0, nranks = 1;
    std::vector<HaloDevRun *> d_halo;  // per peer, 4 lists: send pull, recv pull, send AA, recv AA
    // fluid-cell list layout of the two-grid sweep (lbm_set_sparse): two list arrays (state in
    // sarr[cur]), the pull table, links, cell maps; which of the layouts holds the state
    bool sparse = false;
    bool list_valid = false, dense_valid = true;
    void *sarr_raw = nullptr;
    void *sarr[2] = {nullptr, nullptr};
    int64_t s_stride = 0;
    int32_t *d_snbr = nullptr, *d_sblock = nullptr;
    int64_t *d_scell = nullptr;
    uint64_t *d_slinks = nullptr;

    // device state
    bool dev_ready = false;
    void *arena_raw = nullptr;
    bool arena_owned = false;
    size_t arena_bytes = 0;
    void *arr[2] = {nullptr, nullptr};
    int cur = 0;                 // two-grid: index of the array holding the state
    int aa_layout = LAYOUT_AA_E;  // AA: layout of the stored state

    Plan plan;
    bool plan_built = false, plan_uploaded = false;
    DevBlock *d_blocks = nullptr;
    uint64_t *d_links = nullptr;
    uint64_t *d_zouhe = nullptr;  // wet-node entries
    DevRun *d_runs_pull = nullptr, *d_runs_aa = nullptr;
    DevTile *d_tiles = nullptr;
    double *d_params = nullptr;
    uint32_t *d_masks = nullptr;
    std::vector<const uint32_t *> mask_ptr;
    double *d_partials = nullptr;
    int64_t partials_cap = 0;
    double *d_step_partials = nullptr;  // per-tile diagnostics written by the last sweep
    bool step_diag_valid = false;       // d_step_partials describe the stored state
    double *d_out = nullptr;
    double *d_scratch = nullptr;
    int64_t scratch_cap = 0;
    size_t list_bytes = 0;

    Coll<double> cd{};
    Coll<float> cf{};
    double base[27] = {0};

    int64_t launches = 0;
    int64_t steps_done = 0;
    std::string err;

    // per-block launches (one sweep launch per block instead of one batched launch)
    bool per_block = false;
    std::vector<int64_t> tile_start;  // first tile of each block (+ total at the end)

    // CUDA-graph replay of step pairs (graph mode): one executable graph per starting parity
    bool wide_index = false;  // lbm_set_index_bits(64): no 32-bit index arithmetic in the sweeps
    bool graph_mode = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_epoch[2] = {-1, -1};
    int64_t list_epoch = 0;  // bumped whenever device lists are (re)uploaded

    // locally varying relaxation (closure.cu): kind, Smagorinsky constant, network
    int closure = CLOSURE_NONE;
    double closure_cs = 0.0;
    MlpDev *d_mlp = nullptr;
    int *d_tc_err = nullptr;  // set by the tensor-core network when a bounded wait gives up
    size_t stage_bytes = 0;   // shared memory of the staged sweep tiles (0: none)
    int *d_sweep_err = nullptr;  // set by the staged sweep when a bounded wait gives up
    // pinned host landing zone of the per-step reads (diagnostics record, wait-status flags), so
    // their copies are asynchronous and one stream synchronisation covers them
    struct HostIO {
        double diag[8];
        int wait_err[2];
        // pipelined reads (lbm_step_diagnostics_post/take): one record and its flags per slot
        struct Slot {
            double diag[8];
            int wait_err[2];
        } slot[LBM_DIAG_SLOTS];
    } *h_io = nullptr;
    HostIO *h_io_dev = nullptr;  // its device address (kernels write the pipelined slots directly)
    cudaEvent_t slot_done[LBM_DIAG_SLOTS] = {};      // recorded after each slot's copies
    int64_t slot_ticket[LBM_DIAG_SLOTS] = {-1, -1, -1, -1};  // untaken ticket per slot (-1: free)
    int64_t next_ticket = 0;

    // tracing: events around fill and sweep launches (pairs of [start, end])
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_marks[2];  // per kernel kind: (start idx, end idx)
    size_t ev_used = 0;
};

namespace {

lbm_status fail(lbm_ctx *c, lbm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <class T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// ---- dispatch to the per-(stencil, storage) objects --------------------------------------
#define LBM_SWITCH(q, st, NAME, ...)                              \
    do {                                                          \
        if (q == 19) {                                            \
            switch (st) {                                         \
                case 0: return NAME##19_0(__VA_ARGS__);           \
                case 1: return NAME##19_1(__VA_ARGS__);           \
                case 2: return NAME##19_2(__VA_ARGS__);           \
                case 3: return NAME##19_3(__VA_ARGS__);           \
            }                                                     \
        } else {                                                  \
            switch (st) {                                         \
                case 0: return NAME##27_0(__VA_ARGS__);           \
                case 1: return NAME##27_1(__VA_ARGS__);           \
                case 2: return NAME##27_2(__VA_ARGS__);           \
                case 3: return NAME##27_3(__VA_ARGS__);           \
            }                                                     \
        }                                                         \
        return cudaErrorInvalidValue;                             \
    } while (0)

cudaError_t do_sweep(int q, int st, const SweepArgs &s) { LBM_SWITCH(q, st, launch_sweep_, s); }
// MRT sweeps exist for FP64 and FP32 storage (lbm_create_blocks refuses the others)
cudaError_t do_sweep_mrt(int q, int st, const SweepArgs &s)
{
    if (q == 19) return st == 0 ? launch_sweep_mrt_19_0(s) : launch_sweep_mrt_19_1(s);
    return st == 0 ? launch_sweep_mrt_27_0(s) : launch_sweep_mrt_27_1(s);
}

// Cumulant sweeps: D3Q27 with FP64 or FP32 storage (lbm_create_blocks refuses the others)
cudaError_t do_sweep_cum(int st, const SweepArgs &s)
{
    return st == 0 ? launch_sweep_cum_27_0(s) : launch_sweep_cum_27_1(s);
}

// The step's sweep: the plain sweep, or the closure sweep when a closure is set.
cudaError_t sweep_of(const lbm_ctx *c, const SweepArgs &s)
{
    if (c->closure == CLOSURE_NONE) {
        if (c->p.collision == LBM_CUMULANT) return do_sweep_cum(c->storage, s);
        return c->p.collision == LBM_MRT ? do_sweep_mrt(c->q, c->storage, s) : do_sweep(c->q, c->storage, s);
    }
    ClosureLaunch cl;
    cl.sw = s;
    cl.closure = c->closure;
    cl.trt = c->p.collision == LBM_TRT ? 1 : 0;
    cl.tau0 = (float)(1.0 / c->p.omega);
    cl.cs = (float)c->closure_cs;
    cl.lambda = (float)c->p.magic_lambda;
    cl.mlp = c->d_mlp;
    cl.err = c->d_tc_err;
    return launch_closure_sweep(cl);
}
cudaError_t do_fill(int q, int st, const FillArgs &s) { LBM_SWITCH(q, st, launch_fill_, s); }
cudaError_t do_zouhe(int q, int st, const FillArgs &s) { LBM_SWITCH(q, st, launch_zouhe_, s); }
cudaError_t do_cells(int q, int st, int op, int force, const CellArgs &s) { LBM_SWITCH(q, st, launch_cells_, op, force, s); }
cudaError_t do_reduce(int q, int st, const ReduceArgs &s) { LBM_SWITCH(q, st, launch_reduce_, s); }

int bytes_of(int storage) { return storage == LBM_FP64 ? 8 : (storage == LBM_FP32 ? 4 : 2); }

lbm_status build_lists(lbm_ctx *c)
{
    if (c->plan_built) return LBM_OK;
    PlanInput in;
    in.q = c->q;
    in.bytes_per_pdf = c->bpp;
    for (int a = 0; a < 3; ++a) in.periodic[a] = c->p.periodic[a] != 0;
    for (int f = 0; f < 6; ++f) {
        in.face_kind[f] = c->face_kind[f];
        in.face_param[f] = c->face_param[f];
    }
    for (int a = 0; a < 3; ++a) in.tile[a] = c->tile[a];
    in.in_place = c->in_place;
    in.blocks = &c->blocks;
    in.flags = &c->flags;
    in.block_param = &c->block_param;
    in.owner = c->owner.empty() ? nullptr : &c->owner;
    in.rank = c->rank;
    in.sparse = c->sparse ? 1 : 0;
    std::string e = build_plan(in, c->plan);
    if (!e.empty()) return fail(c, LBM_ERR_UNSUPPORTED, "%s", e.c_str());
    if ((int64_t)c->plan.tiles.size() > 0x7fffffffLL) return fail(c, LBM_ERR_UNSUPPORTED, "too many tiles");
    c->plan_built = true;
    c->plan_uploaded = false;
    return LBM_OK;
}

template <class T>
lbm_status upload(lbm_ctx *c, T *&dst, const std::vector<T> &v, const char *what)
{
    dfree(dst);
    if (v.empty()) return LBM_OK;
    CK(cudaMalloc((void **)&dst, v.size() * sizeof(T)), what);
    CK(cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    c->list_bytes += v.size() * sizeof(T);
    return LBM_OK;
}

lbm_status ensure_arena(lbm_ctx *c)
{
    if (c->dev_ready) return LBM_OK;
    const int narr = c->pattern == LBM_TWO_GRID ? 2 : 1;
    const size_t bytes1 = (size_t)c->arena_elems * c->bpp;
    const size_t need = lbm_required_bytes(c);
    if (!c->arena_raw) {
        CK(cudaMalloc(&c->arena_raw, need), "cudaMalloc(PDF arrays)");
        c->arena_owned = true;
        c->arena_bytes = need;
    }
    uintptr_t b = ((uintptr_t)c->arena_raw + 255) & ~(uintptr_t)255;
    c->arr[0] = (void *)b;
    c->arr[1] = narr == 2 ? (void *)((b + bytes1 + 255) & ~(uintptr_t)255) : nullptr;
    CK(cudaMemsetAsync(c->arr[0], 0, bytes1, c->stream), "clear PDF array");
    if (narr == 2) CK(cudaMemsetAsync(c->arr[1], 0, bytes1, c->stream), "clear PDF array");
    CK(cudaMalloc((void **)&c->d_sweep_err, sizeof(int)), "cudaMalloc(sweep status)");
    CK(cudaMemsetAsync(c->d_sweep_err, 0, sizeof(int), c->stream), "clear sweep status");
    CK(cudaMallocHost((void **)&c->h_io, sizeof(lbm_ctx::HostIO)), "cudaMallocHost(status)");
    CK(cudaHostGetDevicePointer((void **)&c->h_io_dev, c->h_io, 0), "device address of the host landing zone");
    c->dev_ready = true;
    return LBM_OK;
}

DevBlock dev_block(const lbm_ctx *c, int b)
{
    const BlockLayout &L = c->blocks[b];
    DevBlock d{};
    d.nx = L.n[0];
    d.ny = L.n[1];
    d.nz = L.n[2];
    d.pitch = L.pitch;
    d.plane = L.plane;
    d.slab = L.slab;
    d.offset = L.offset;
    d.mask = c->mask_ptr.empty() ? nullptr : c->mask_ptr[b];
    d.xo = L.xo;
    d.through = c->plan.through.empty() ? 0 : c->plan.through[b];
    for (int r = 0; r < 27; ++r) d.nbr[r] = c->plan.nbr.empty() ? -1 : c->plan.nbr[b][r];
    d.wrap = 0;
    if (d.through)
        for (int a = 0; a < 3; ++a) {
            const int lo = a == 0 ? 12 : (a == 1 ? 10 : 4), hi = a == 0 ? 14 : (a == 1 ? 16 : 22);
            if (d.nbr[lo] == b && d.nbr[hi] == b) d.wrap |= 1 << a;
        }
    return d;
}

// Tiles of the two-grid sweep whose source rows are staged in shared memory by bulk copies
// (see sweep_staged): 16-bit storage (the issue-bound case: staging takes the per-direction
// address arithmetic off the threads; with FP32 storage the sweep is at the HBM roofline
// without it and the staged form measured slower), full block width in at most two rows, no
// masks, in-place neighbours only the block itself, rows x = -8 .. nx + 7 inside the padded
// row, 16-byte aligned.  Sets flag bit 1 of those tiles when `tiles` is given, counts them in
// *count, and returns the dynamic shared memory a staged CTA needs (0: none staged).
size_t stage_tiles(const lbm_ctx *c, const Plan &P, DevTile *tiles, int64_t *count = nullptr)
{
    size_t bytes = 0;
    int64_t n = 0;
    if (c->pattern == LBM_TWO_GRID && c->storage >= LBM_BF16_DEV) {
        const int threads = c->tile[0] * c->tile[1];
        std::vector<uint8_t> ok_block(c->blocks.size(), 0);
        for (size_t b = 0; b < c->blocks.size(); ++b) {
            const BlockLayout &L = c->blocks[b];
            const int nx = L.n[0];
            bool ok = nx <= threads && 2 * nx >= threads && (nx * c->bpp) % 16 == 0 &&
                      ((L.xo - 8) * c->bpp) % 16 == 0 && L.xo >= 8 && L.pitch - L.xo - nx >= 8 &&
                      (L.offset * c->bpp) % 16 == 0;
            if (ok && !P.through.empty() && P.through[b])
                for (int r = 0; r < 27; ++r)
                    if (P.nbr[b][r] >= 0 && P.nbr[b][r] != (int)b) ok = false;
            ok_block[b] = ok;
        }
        auto staged = [&](size_t i) {
            const Tile &t = P.tiles[i];
            const int nx = c->blocks[t.block].n[0];
            return ok_block[t.block] && !(t.flags & 1) && t.x0 == 0 && t.width_m1 + 1 == nx;
        };
        for (size_t i = 0; i < P.tiles.size(); ++i) {
            const Tile &t = P.tiles[i];
            const int nx = c->blocks[t.block].n[0];
            if (!staged(i)) continue;
            ++n;
            if (tiles) tiles[i].flags |= 2;
            size_t rows = (size_t)threads / nx;
#if LBM_STAGED_TWO
            // one-row tiles in pairs (rows y0, y0 + 1 of the same block and z range, y0 even):
            // the first sweeps both rows with two cells per thread, the second is skipped
            if (rows == 1 && t.y0 % 2 == 0 && i + 1 < P.tiles.size() && staged(i + 1)) {
                const Tile &u = P.tiles[i + 1];
                if (u.block == t.block && u.z0 == t.z0 && u.y0 == t.y0 + 1) {
                    if (tiles) {
                        tiles[i].flags |= 4;
                        tiles[i + 1].flags |= 2 | 8;
                    }
                    ++n;
                    ++i;
                    rows = 2;
                }
            }
#endif
            bytes = std::max(bytes, kSweepStages * ((size_t)c->q * rows * (nx + 16) * c->bpp + 16));
        }
    }
    if (count) *count = n;
    return bytes;
}

lbm_status ensure_lists(lbm_ctx *c)
{
    lbm_status s = build_lists(c);
    if (s != LBM_OK) return s;
    if (c->plan_uploaded) return LBM_OK;
    CK(cudaStreamSynchronize(c->stream), "synchronise before list upload");
    c->list_bytes = 0;
    const Plan &P = c->plan;
    // masks: one buffer, per-block offsets
    dfree(c->d_masks);
    size_t mbytes = 0;
    // element counts rounded to 64 (256 bytes) so each block's mask starts aligned
    for (const auto &m : P.masks) mbytes += (m.size() + 63) / 64 * 64;
    c->mask_ptr.assign(c->blocks.size(), nullptr);
    if (mbytes) {
        CK(cudaMalloc((void **)&c->d_masks, mbytes * sizeof(uint32_t)), "cudaMalloc(masks)");
        c->list_bytes += mbytes * sizeof(uint32_t);
        size_t off = 0;
        for (size_t b = 0; b < P.masks.size(); ++b) {
            if (P.masks[b].empty()) continue;
            CK(cudaMemcpy(c->d_masks + off, P.masks[b].data(), P.masks[b].size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice),
               "upload mask");
            c->mask_ptr[b] = c->d_masks + off;
            off += (P.masks[b].size() + 63) / 64 * 64;
        }
    }
    std::vector<DevBlock> db(c->blocks.size());
    for (size_t b = 0; b < db.size(); ++b) db[b] = dev_block(c, (int)b);
    lbm_status s2;
    if ((s2 = upload(c, c->d_blocks, db, "upload blocks")) != LBM_OK) return s2;
    if ((s2 = upload(c, c->d_links, P.links, "upload links")) != LBM_OK) return s2;
    if ((s2 = upload(c, c->d_zouhe, P.zouhe, "upload wet-node entries")) != LBM_OK) return s2;
    static_assert(sizeof(GhostRun) == sizeof(DevRun), "run layout");
    static_assert(sizeof(Tile) == sizeof(DevTile), "tile layout");
    std::vector<DevRun> rp(P.runs_pull.size()), ra(P.runs_aa.size());
    if (!rp.empty()) memcpy(rp.data(), P.runs_pull.data(), rp.size() * sizeof(DevRun));
    if (!ra.empty()) memcpy(ra.data(), P.runs_aa.data(), ra.size() * sizeof(DevRun));
    if ((s2 = upload(c, c->d_runs_pull, rp, "upload runs")) != LBM_OK) return s2;
    if ((s2 = upload(c, c->d_runs_aa, ra, "upload runs")) != LBM_OK) return s2;
    static_assert(sizeof(HaloRun) == sizeof(HaloDevRun), "halo run layout");
    for (HaloDevRun *&h : c->d_halo) dfree(h);
    c->d_halo.assign(4 * P.halo.size(), nullptr);
    for (size_t p = 0; p < P.halo.size(); ++p) {
        const std::vector<HaloRun> *lists[4] = {&P.halo[p].send_pull, &P.halo[p].recv_pull, &P.halo[p].send_aa,
                                                &P.halo[p].recv_aa};
        for (int k = 0; k < 4; ++k) {
            std::vector<HaloDevRun> hv(lists[k]->size());
            if (!hv.empty()) memcpy(hv.data(), lists[k]->data(), hv.size() * sizeof(HaloDevRun));
            if ((s2 = upload(c, c->d_halo[4 * p + k], hv, "upload halo runs")) != LBM_OK) return s2;
        }
    }
    std::vector<DevTile> dt(P.tiles.size());
    if (!dt.empty()) memcpy(dt.data(), P.tiles.data(), dt.size() * sizeof(DevTile));
    c->stage_bytes = stage_tiles(c, P, dt.data());
    if ((s2 = upload(c, c->d_tiles, dt, "upload tiles")) != LBM_OK) return s2;
    std::vector<double> par;
    for (const auto &w : P.params) {
        par.push_back(w.u[0]);
        par.push_back(w.u[1]);
        par.push_back(w.u[2]);
        par.push_back(w.rho);
    }
    if ((s2 = upload(c, c->d_params, par, "upload params")) != LBM_OK) return s2;
    // the list layout: tables, links, cell maps and its two arrays
    dfree(c->d_snbr);
    dfree(c->d_sblock);
    dfree(c->d_scell);
    dfree(c->d_slinks);
    if (c->sarr_raw) cudaFree(c->sarr_raw);
    c->sarr_raw = c->sarr[0] = c->sarr[1] = nullptr;
    c->list_valid = false;
    if (c->sparse) {
        const SparsePlan &SP = P.sparse;
        if ((s2 = upload(c, c->d_snbr, SP.nbr, "upload list table")) != LBM_OK) return s2;
        if ((s2 = upload(c, c->d_sblock, SP.block_of, "upload list cell map")) != LBM_OK) return s2;
        if ((s2 = upload(c, c->d_scell, SP.cell_of, "upload list cell map")) != LBM_OK) return s2;
        if ((s2 = upload(c, c->d_slinks, SP.links, "upload list links")) != LBM_OK) return s2;
        // entries per direction rounded to 256 bytes, so every direction starts aligned
        const int64_t per = 256 / c->bpp;
        c->s_stride = std::max<int64_t>(per, (SP.nslots + per - 1) / per * per);
        const size_t one = (size_t)c->s_stride * c->q * c->bpp;
        CK(cudaMalloc(&c->sarr_raw, 2 * one + 256), "cudaMalloc(list arrays)");
        CK(cudaMemsetAsync(c->sarr_raw, 0, 2 * one + 256, c->stream), "clear list arrays");
        c->list_bytes += 2 * one + 256;
        const uintptr_t b0 = ((uintptr_t)c->sarr_raw + 255) & ~(uintptr_t)255;
        c->sarr[0] = (void *)b0;
        c->sarr[1] = (void *)(b0 + one);
    }
    const int64_t list_ctas = c->sparse ? (P.sparse.nfluid + 255) / 256 : 0;
    const int64_t need = std::max<int64_t>(1, std::max<int64_t>((int64_t)P.tiles.size(), list_ctas)) * 8;
    if (need > c->partials_cap) {
        dfree(c->d_partials);
        dfree(c->d_step_partials);
        dfree(c->d_out);
        CK(cudaMalloc((void **)&c->d_partials, need * sizeof(double)), "cudaMalloc(reduction partials)");
        CK(cudaMalloc((void **)&c->d_step_partials, need * sizeof(double)), "cudaMalloc(step diagnostics)");
        // the 8 results of the fixed-order sum plus its first-level records
        CK(cudaMalloc((void **)&c->d_out, reduce_final_scratch(need / 8) * sizeof(double)),
           "cudaMalloc(reduction output)");
        c->partials_cap = need;
    }
    c->step_diag_valid = false;
    c->tile_start.assign(c->blocks.size() + 1, 0);
    for (const Tile &t : P.tiles) c->tile_start[t.block + 1]++;
    for (size_t b = 0; b < c->blocks.size(); ++b) c->tile_start[b + 1] += c->tile_start[b];
    c->plan_uploaded = true;
    c->list_epoch++;
    return LBM_OK;
}

// Device address of a page-locked (cudaHostAlloc'd or cudaHostRegister'ed) host buffer, which
// kernels can read and write over the host link directly; nullptr for any other pointer
// (pageable host memory goes through a device staging copy).
double *device_view(const void *host)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return static_cast<double *>(at.devicePointer);
}

lbm_status ensure_scratch(lbm_ctx *c, int64_t doubles)
{
    if (doubles <= c->scratch_cap) return LBM_OK;
    dfree(c->d_scratch);
    CK(cudaMalloc((void **)&c->d_scratch, doubles * sizeof(double)), "cudaMalloc(transfer buffer)");
    c->scratch_cap = doubles;
    return LBM_OK;
}

int state_layout(const lbm_ctx *c) { return c->pattern == LBM_TWO_GRID ? LAYOUT_PULL : c->aa_layout; }

CellArgs cell_args(lbm_ctx *c, int block)
{
    CellArgs a{};
    const BlockLayout &L = c->blocks[block];
    a.a = c->pattern == LBM_TWO_GRID ? c->arr[c->cur] : c->arr[0];
    a.blocks = c->d_blocks;
    a.block = block;
    a.blk = dev_block(c, block);
    a.layout = state_layout(c);
    a.mask = c->mask_ptr[block];
    for (int k = 0; k < 3; ++k) a.F[k] = c->p.force[k];
    for (int i = 0; i < 27; ++i) a.base[i] = c->base[i];
    a.cd = c->cd;
    a.cf = c->cf;
    a.stream = c->stream;
    return a;
}

lbm_status prepare(lbm_ctx *c)
{
    lbm_status s = ensure_arena(c);
    if (s != LBM_OK) return s;
    return ensure_lists(c);
}

// Next free event of the tracing pool (created on demand).
lbm_status next_event(lbm_ctx *c, int *idx)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e), "cudaEventCreate");
        c->ev_pool.push_back(e);
    }
    *idx = (int)c->ev_used++;
    return LBM_OK;
}

lbm_status mark(lbm_ctx *c, int *idx)
{
    lbm_status s = next_event(c, idx);
    if (s != LBM_OK) return s;
    CK(cudaEventRecord(c->ev_pool[*idx], c->stream), "cudaEventRecord");
    return LBM_OK;
}

lbm_status check_block(lbm_ctx *c, int32_t block)
{
    if (block < 0 || block >= (int32_t)c->blocks.size()) return fail(c, LBM_ERR_ARG, "block index %d out of range", block);
    return LBM_OK;
}

// A block whose PDFs this context holds (every block, or in a partitioned run those of its rank).
lbm_status check_owned(lbm_ctx *c, int32_t block)
{
    lbm_status s = check_block(c, block);
    if (s != LBM_OK) return s;
    if (!c->owner.empty() && c->owner[block] != c->rank)
        return fail(c, LBM_ERR_ARG, "block %d belongs to rank %d, not to this context (rank %d)", block,
                    c->owner[block], c->rank);
    return LBM_OK;
}

// The context exchanges a halo with some peer (then it advances one step per lbm_step call).
bool has_halo(const lbm_ctx *c)
{
    for (const PeerHalo &h : c->plan.halo)
        if (h.n_send_pull + h.n_recv_pull + h.n_send_aa + h.n_recv_aa > 0) return true;
    return false;
}

// The lists of the exchange that must precede the next step with `peer`: two-grid, the pull
// selection forward (owned interior -> the peer's ghosts); AA before the neighbour sweep (layout
// E) the AA selection forward, before the local sweep (layout O) backward (the ghost slots the
// neighbour sweep wrote -> the peer's interior).  ipack/iunpack index the context's device
// lists (4 per peer).
void halo_lists(const lbm_ctx *c, int peer, int *ipack, int *iunpack, int64_t *nsend, int64_t *nrecv)
{
    const PeerHalo &h = c->plan.halo[peer];
    if (c->pattern == LBM_TWO_GRID) {
        *ipack = 0, *iunpack = 1, *nsend = h.n_send_pull, *nrecv = h.n_recv_pull;
    } else if (c->aa_layout == LAYOUT_AA_E) {
        *ipack = 2, *iunpack = 3, *nsend = h.n_send_aa, *nrecv = h.n_recv_aa;
    } else {
        *ipack = 3, *iunpack = 2, *nsend = h.n_recv_aa, *nrecv = h.n_send_aa;
    }
}

const std::vector<HaloRun> &halo_runs(const lbm_ctx *c, int peer, int k)
{
    const PeerHalo &h = c->plan.halo[peer];
    return k == 0 ? h.send_pull : (k == 1 ? h.recv_pull : (k == 2 ? h.send_aa : h.recv_aa));
}

// Records of the per-CTA diagnostics the last sweep wrote (tiles, or CTAs of the list sweep).
int64_t diag_records(const lbm_ctx *c)
{
    return c->sparse ? (c->plan.sparse.nfluid + 255) / 256 : (int64_t)c->plan.tiles.size();
}

lbm_status sparse_args(lbm_ctx *c, int op, SparseArgs &a)
{
    a = SparseArgs{};
    a.op = op;
    a.nbr = c->d_snbr;
    a.links = c->d_slinks;
    a.nlinks = (int64_t)c->plan.sparse.links.size();
    a.params = c->d_params;
    a.blocks = c->d_blocks;
    a.block_of = c->d_sblock;
    a.cell_of = c->d_scell;
    a.nfluid = c->plan.sparse.nfluid;
    a.stride = c->s_stride;
    a.force = c->force ? 1 : 0;
    a.cd = c->cd;
    a.cf = c->cf;
    a.stream = c->stream;
    return LBM_OK;
}

cudaError_t do_sparse(int q, int st, const SparseArgs &s) { LBM_SWITCH(q, st, launch_sparse_, s); }

// The list layout holds the state (copy it from the dense array if it does not).
lbm_status ensure_list(lbm_ctx *c)
{
    if (!c->sparse || c->list_valid) return LBM_OK;
    SparseArgs a;
    sparse_args(c, SPARSE_TO_LIST, a);
    a.dense = c->arr[c->cur];
    a.list = c->sarr[c->cur];
    CK(do_sparse(c->q, c->storage, a), "dense to list copy");
    c->launches++;
    c->list_valid = true;
    return LBM_OK;
}

// The dense arrays hold the state (copy it back from the list layout if they do not).
lbm_status ensure_dense(lbm_ctx *c)
{
    if (!c->sparse || c->dense_valid) return LBM_OK;
    SparseArgs a;
    sparse_args(c, SPARSE_TO_DENSE, a);
    a.dense = c->arr[c->cur];
    a.list = c->sarr[c->cur];
    CK(do_sparse(c->q, c->storage, a), "list to dense copy");
    c->launches++;
    c->dense_valid = true;
    return LBM_OK;
}

// A setter is about to rebuild the lists: a state held only by the list layout goes back to
// the dense arrays first (the rebuilt lists may number the fluid cells differently).
lbm_status before_replan(lbm_ctx *c)
{
    if (c->sparse && c->dev_ready && c->plan_uploaded) return ensure_dense(c);
    return LBM_OK;
}

lbm_status check_peer(lbm_ctx *c, int32_t peer)
{
    if (c->owner.empty()) return fail(c, LBM_ERR_STATE, "not a partitioned context");
    if (peer < 0 || peer >= c->nranks || peer == c->rank) return fail(c, LBM_ERR_ARG, "bad peer rank %d", peer);
    return LBM_OK;
}

// Status of the bounded device-side waits.  wait_status_enqueue queues the copies of the flags
// into the pinned landing zone; after the stream has been synchronised wait_status_take reports
// LBM_ERR_TIMEOUT once after a wait gave up (the flag is then cleared), else LBM_OK.
lbm_status wait_status_enqueue(lbm_ctx *c)
{
    c->h_io->wait_err[0] = c->h_io->wait_err[1] = 0;
    if (c->d_sweep_err)
        CK(cudaMemcpyAsync(&c->h_io->wait_err[0], c->d_sweep_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "read wait status");
    if (c->d_tc_err && c->closure == CLOSURE_MLP)
        CK(cudaMemcpyAsync(&c->h_io->wait_err[1], c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "read network status");
    return LBM_OK;
}

lbm_status wait_status_take(lbm_ctx *c)
{
    const int e0 = c->h_io->wait_err[0], e1 = c->h_io->wait_err[1];
    if (e0) {
        CK(cudaMemsetAsync(c->d_sweep_err, 0, sizeof(int), c->stream), "clear wait status");
        CK(cudaStreamSynchronize(c->stream), "clear wait status");
        if (e0 == 2) return fail(c, LBM_ERR_TIMEOUT, "the wait self-check gave up as designed; the state is untouched");
        return fail(c, LBM_ERR_TIMEOUT, "a bounded wait of the staged sweep gave up; the state is invalid");
    }
    if (e1) {
        CK(cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream), "clear network status");
        CK(cudaStreamSynchronize(c->stream), "clear network status");
        return fail(c, LBM_ERR_TIMEOUT, "a bounded wait of the tensor-core network gave up; the state is invalid");
    }
    return LBM_OK;
}

// Both steps around a synchronisation of their own (calls that read other results first).
lbm_status wait_status(lbm_ctx *c)
{
    lbm_status s = wait_status_enqueue(c);
    if (s != LBM_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "read wait status");
    return wait_status_take(c);
}

}  // namespace

extern "C" {

namespace {
lbm_status create_ctx(const lbm_params *params, const lbm_block_desc *blocks, int32_t nblocks, const int32_t *owner,
                      int32_t nranks, int32_t rank, void *cuda_stream, lbm_ctx **out);
}  // namespace

lbm_status lbm_create_blocks(const lbm_params *params, const lbm_block_desc *blocks, int32_t nblocks,
                             void *cuda_stream, lbm_ctx **out)
{
    return create_ctx(params, blocks, nblocks, nullptr, 1, 0, cuda_stream, out);
}

lbm_status lbm_create_partition(const lbm_params *params, const lbm_block_desc *blocks, int32_t nblocks,
                                const int32_t *owner, int32_t nranks, int32_t rank, void *cuda_stream, lbm_ctx **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!owner || nranks < 1 || rank < 0 || rank >= nranks) return LBM_ERR_ARG;
    bool mine = false;
    for (int32_t b = 0; b < nblocks; ++b) {
        if (owner[b] < 0 || owner[b] >= nranks) return LBM_ERR_ARG;
        mine = mine || owner[b] == rank;
    }
    if (!mine) return LBM_ERR_ARG;
    return create_ctx(params, blocks, nblocks, owner, nranks, rank, cuda_stream, out);
}

lbm_status lbm_partition_morton(const lbm_block_desc *blocks, int32_t nblocks, int32_t nranks, const double *weights,
                                int32_t *owner)
{
    if (!blocks || !owner || nblocks <= 0 || nranks < 1) return LBM_ERR_ARG;
    std::vector<BlockLayout> bl(nblocks);
    std::vector<double> w;
    for (int b = 0; b < nblocks; ++b) {
        for (int a = 0; a < 3; ++a) {
            bl[b].origin[a] = blocks[b].origin[a];
            bl[b].n[a] = blocks[b].size[a];
            if (blocks[b].size[a] < 1) return LBM_ERR_ARG;
        }
        if (weights) {
            if (!(weights[b] >= 0.0) || !std::isfinite(weights[b])) return LBM_ERR_ARG;
            w.push_back(weights[b]);
        }
    }
    std::vector<int32_t> own;
    partition_morton(bl, nranks, weights ? &w : nullptr, own);
    for (int b = 0; b < nblocks; ++b) owner[b] = own[b];
    return LBM_OK;
}

lbm_status lbm_halo_sizes(lbm_ctx *c, int32_t peer, int64_t *send_elems, int64_t *recv_elems)
{
    if (!c || !send_elems || !recv_elems) return LBM_ERR_ARG;
    lbm_status s = check_peer(c, peer);
    if (s != LBM_OK) return s;
    if ((s = build_lists(c)) != LBM_OK) return s;
    int ip, iu;
    halo_lists(c, peer, &ip, &iu, send_elems, recv_elems);
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_ctx *c, int32_t peer, void *dev_buf)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_peer(c, peer);
    if (s != LBM_OK) return s;
    if ((s = prepare(c)) != LBM_OK) return s;
    int ip, iu;
    int64_t ns, nr;
    halo_lists(c, peer, &ip, &iu, &ns, &nr);
    if (ns == 0) return LBM_OK;
    if (!dev_buf) return fail(c, LBM_ERR_ARG, "null halo buffer");
    HaloArgs h{};
    h.arena = c->pattern == LBM_TWO_GRID ? c->arr[c->cur] : c->arr[0];
    h.buf = dev_buf;
    h.runs = c->d_halo[4 * peer + ip];
    h.nruns = (int64_t)halo_runs(c, peer, ip).size();
    h.to_buf = 1;
    h.elem_bytes = c->bpp;
    h.stream = c->stream;
    CK(launch_halo(h), "halo pack launch");
    c->launches++;
    return LBM_OK;
}

lbm_status lbm_halo_unpack(lbm_ctx *c, int32_t peer, const void *dev_buf)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_peer(c, peer);
    if (s != LBM_OK) return s;
    if ((s = prepare(c)) != LBM_OK) return s;
    int ip, iu;
    int64_t ns, nr;
    halo_lists(c, peer, &ip, &iu, &ns, &nr);
    if (nr == 0) return LBM_OK;
    if (!dev_buf) return fail(c, LBM_ERR_ARG, "null halo buffer");
    HaloArgs h{};
    h.arena = c->pattern == LBM_TWO_GRID ? c->arr[c->cur] : c->arr[0];
    h.buf = const_cast<void *>(dev_buf);
    h.runs = c->d_halo[4 * peer + iu];
    h.nruns = (int64_t)halo_runs(c, peer, iu).size();
    h.to_buf = 0;
    h.elem_bytes = c->bpp;
    h.stream = c->stream;
    CK(launch_halo(h), "halo unpack launch");
    c->launches++;
    return LBM_OK;
}

lbm_status lbm_plan_halo(lbm_ctx *c, int32_t peer, int32_t list, int64_t *out, int64_t cap, int64_t *n)
{
    if (!c || !n) return LBM_ERR_ARG;
    lbm_status s = check_peer(c, peer);
    if (s != LBM_OK) return s;
    if (list < 0 || list > 3) return fail(c, LBM_ERR_ARG, "bad halo list %d", list);
    if ((s = build_lists(c)) != LBM_OK) return s;
    const std::vector<HaloRun> &R = halo_runs(c, peer, list);
    *n = (int64_t)R.size();
    if (!out) return LBM_OK;
    if (cap < 4 * *n) return fail(c, LBM_ERR_ARG, "buffer too small");
    for (size_t r = 0; r < R.size(); ++r) {
        out[4 * r] = R[r].arena;
        out[4 * r + 1] = R[r].buf;
        out[4 * r + 2] = R[r].len;
        out[4 * r + 3] = R[r].astride;
    }
    return LBM_OK;
}

}  // extern "C"

namespace {
lbm_status create_ctx(const lbm_params *params, const lbm_block_desc *blocks, int32_t nblocks, const int32_t *owner,
                      int32_t nranks, int32_t rank, void *cuda_stream, lbm_ctx **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!params || !blocks || nblocks <= 0) return LBM_ERR_ARG;
    const lbm_params &p = *params;
    if (p.stencil != LBM_D3Q19 && p.stencil != LBM_D3Q27) return LBM_ERR_ARG;
    if (p.collision != LBM_SRT && p.collision != LBM_TRT && p.collision != LBM_MRT && p.collision != LBM_CUMULANT)
        return LBM_ERR_ARG;
    if (p.storage < LBM_FP64 || p.storage > LBM_FP16_DEV) return LBM_ERR_ARG;
    if (p.pattern != LBM_TWO_GRID && p.pattern != LBM_AA) return LBM_ERR_ARG;
    if (!(p.omega >= 0.0 && p.omega < 2.0)) return LBM_ERR_ARG;
    if ((p.collision == LBM_TRT || p.collision == LBM_MRT) && !(p.magic_lambda > 0.0) && p.omega > 0.0)
        return LBM_ERR_ARG;
    if (p.collision == LBM_CUMULANT) {
        for (int g = 0; g < 9; ++g)
            if (!(p.cumulant_rates[g] >= 0.0 && p.cumulant_rates[g] < 2.0)) return LBM_ERR_ARG;
        if (p.stencil != LBM_D3Q27 || (p.storage != LBM_FP64 && p.storage != LBM_FP32)) return LBM_ERR_UNSUPPORTED;
    }
    if (p.collision == LBM_MRT) {
        for (int g = 0; g < 4; ++g)
            if (!(p.mrt_rates[g] >= 0.0 && p.mrt_rates[g] < 2.0)) return LBM_ERR_ARG;
        if (p.storage != LBM_FP64 && p.storage != LBM_FP32) return LBM_ERR_UNSUPPORTED;
    }
    if (!(p.rho0 > 0.0) || p.diag_interval < 0) return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p.force[a])) return LBM_ERR_ARG;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    c->p = p;
    c->q = p.stencil;
    c->storage = p.storage;
    c->pattern = p.pattern;
    c->bpp = bytes_of(p.storage);
    if (p.pattern == LBM_TWO_GRID && p.storage >= LBM_BF16_DEV) c->tile[2] = 8;  // staged tiles: longer z runs
    c->force = p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0;
    c->stream = (cudaStream_t)cuda_stream;
    c->blocks.resize(nblocks);
    for (int b = 0; b < nblocks; ++b) {
        for (int a = 0; a < 3; ++a) {
            c->blocks[b].origin[a] = blocks[b].origin[a];
            c->blocks[b].n[a] = blocks[b].size[a];
        }
    }
    if (owner) {
        c->owner.assign(owner, owner + nblocks);
        c->nranks = nranks;
        c->rank = rank;
    }
    int64_t elems = 0;
    layout_blocks(c->blocks, c->bpp, c->q, 128, &elems, owner ? &c->owner : nullptr, rank);
    std::string e = check_blocks(c->blocks);
    if (!e.empty()) {
        delete c;
        return LBM_ERR_ARG;
    }
    c->arena_elems = elems;
    c->flags.assign(nblocks, {});
    c->block_param.assign(nblocks, WallParam{{0, 0, 0}, 1.0});
    for (int f = 0; f < 6; ++f) {
        c->face_kind[f] = LBM_NOSLIP;
        c->face_param[f] = WallParam{{0, 0, 0}, 1.0};
    }
    // collision constants
    const double wp = p.omega;
    double wm = wp;
    // TRT: Lambda = (1/w+ - 1/2)(1/w- - 1/2); at w+ = 0 (no relaxation of the even part) the
    // IEEE evaluation gives the limit w- = 2.
    if (p.collision == LBM_TRT || p.collision == LBM_MRT) wm = 1.0 / (p.magic_lambda / (1.0 / wp - 0.5) + 0.5);
    const LatticeView L = lattice_view(c->q);
    const bool dev = c->storage >= LBM_BF16_DEV;
    for (int i = 0; i < 27; ++i) c->base[i] = (dev && i < L.q) ? L.w[i] * p.rho0 : 0.0;
    Coll<double> &d = c->cd;
    d = Coll<double>{};
    d.omega_p = wp;
    d.omega_m = wm;
    d.a_p = 1.0 - 0.5 * wp;
    d.a_m = 1.0 - 0.5 * wm;
    double wc[4] = {0, 0, 0, 0};  // weight per class |c|^2
    for (int i = 0; i < L.q; ++i) wc[L.cx[i] * L.cx[i] + L.cy[i] * L.cy[i] + L.cz[i] * L.cz[i]] = L.w[i];
    d.r = rates_of<double>(wp, wm, wc);
    for (int k2 = 0; k2 < 4; ++k2) d.bw[k2] = 3.0 * d.a_p * wc[k2];
    for (int i = 0; i < L.q; ++i) {
        const double cF = L.cx[i] * p.force[0] + L.cy[i] * p.force[1] + L.cz[i] * p.force[2];
        d.fa[i] = 9.0 * d.a_p * L.w[i] * cF;
        d.fc[i] = 3.0 * d.a_m * L.w[i] * cF;
    }
    for (int a = 0; a < 3; ++a) d.F[a] = p.force[a];
    // MRT: bulk, fourth- and sixth-order rates against omega+, fifth-order against omega- (the
    // TRT rates of their parity); zero for SRT and TRT
    if (p.collision == LBM_MRT) {
        d.mrt_d[0] = p.mrt_rates[0] - wp;
        d.mrt_d[1] = p.mrt_rates[1] - wp;
        d.mrt_d[2] = c->q == 27 ? p.mrt_rates[2] - wm : 0.0;
        d.mrt_d[3] = c->q == 27 ? p.mrt_rates[3] - wp : 0.0;
    }
    if (p.collision == LBM_CUMULANT) {
        d.cum[0] = wp;
        for (int g = 0; g < 9; ++g) d.cum[g + 1] = p.cumulant_rates[g];
        d.cumulant = 1;
        // every rate beyond the bulk at 1: the sweep takes the path that resets the cumulants of
        // order 3..6 without computing them
        d.cum_unit = 1;
        for (int g = 1; g < 9; ++g) d.cum_unit = d.cum_unit && p.cumulant_rates[g] == 1.0;
    }
    d.rho0 = dev ? p.rho0 : 0.0;
    for (int i = 0; i < 27; ++i) d.base[i] = c->base[i];
    // FP32 copy of every constant
    Coll<float> &f = c->cf;
    f.omega_p = (float)d.omega_p;
    f.omega_m = (float)d.omega_m;
    f.a_p = (float)d.a_p;
    f.a_m = (float)d.a_m;
    f.r.wp = (float)d.r.wp;
    f.r.wm = (float)d.r.wm;
    f.r.rest = (float)d.r.rest;
    f.r.alpha = (float)d.r.alpha;
    f.r.beta = (float)d.r.beta;
    for (int k2 = 0; k2 < 4; ++k2) {
        f.r.pw[k2] = (float)d.r.pw[k2];
        f.r.mw[k2] = (float)d.r.mw[k2];
        f.r.pq[k2] = (float)d.r.pq[k2];
        f.bw[k2] = (float)d.bw[k2];
    }
    for (int i = 0; i < 27; ++i) {
        f.fa[i] = (float)d.fa[i];
        f.fc[i] = (float)d.fc[i];
        f.base[i] = (float)d.base[i];
    }
    for (int a = 0; a < 3; ++a) f.F[a] = (float)d.F[a];
    for (int g = 0; g < 4; ++g) f.mrt_d[g] = (float)d.mrt_d[g];
    for (int g = 0; g < 10; ++g) f.cum[g] = (float)d.cum[g];
    f.cumulant = d.cumulant;
    f.cum_unit = d.cum_unit;
    f.rho0 = (float)d.rho0;
    *out = c;
    return LBM_OK;
}
}  // namespace

extern "C" {

size_t lbm_required_bytes(const lbm_ctx *c)
{
    if (!c) return 0;
    const int narr = c->pattern == LBM_TWO_GRID ? 2 : 1;
    const size_t bytes1 = ((size_t)c->arena_elems * c->bpp + 255) / 256 * 256;
    return narr * bytes1 + 256;
}

lbm_status lbm_bind_device_memory(lbm_ctx *c, void *dev_ptr, size_t bytes)
{
    if (!c) return LBM_ERR_ARG;
    if (!dev_ptr) return fail(c, LBM_ERR_ARG, "null device pointer");
    if (c->dev_ready || c->arena_raw) return fail(c, LBM_ERR_STATE, "PDF arrays already allocated");
    if (bytes < lbm_required_bytes(c))
        return fail(c, LBM_ERR_OOM, "bound buffer has %zu bytes, need %zu", bytes, lbm_required_bytes(c));
    c->arena_raw = dev_ptr;
    c->arena_owned = false;
    c->arena_bytes = bytes;
    return LBM_OK;
}

lbm_status lbm_set_face(lbm_ctx *c, int32_t axis, int32_t side, int32_t kind, const double u_wall[3], double rho_wall)
{
    if (!c) return LBM_ERR_ARG;
    if (axis < 0 || axis > 2 || side < 0 || side > 1) return fail(c, LBM_ERR_ARG, "bad face");
    if (kind != LBM_NOSLIP && kind != LBM_VELOCITY && kind != LBM_PRESSURE && kind != LBM_PERIODIC &&
        kind != LBM_ZOUHE_VELOCITY && kind != LBM_ZOUHE_PRESSURE && kind != LBM_REFINE)
        return fail(c, LBM_ERR_ARG, "bad face kind %d", kind);
    if (kind == LBM_REFINE && (c->pattern != LBM_TWO_GRID || c->sparse || !c->owner.empty() ||
                               c->closure != CLOSURE_NONE || (c->storage != LBM_FP64 && c->storage != LBM_FP32)))
        return fail(c, LBM_ERR_UNSUPPORTED, "refinement faces are built for the two-grid pattern, FP64 or FP32 "
                                            "storage, the dense layout of one context and no closure");
    if ((kind == LBM_ZOUHE_VELOCITY || kind == LBM_ZOUHE_PRESSURE) &&
        (c->q != 19 || c->pattern != LBM_TWO_GRID || c->sparse || !c->owner.empty() || c->closure != CLOSURE_NONE))
        return fail(c, LBM_ERR_UNSUPPORTED, "wet-node (Zou-He) faces are built for D3Q19, the two-grid pattern, the "
                                            "dense layout of one context and no closure");
    if (kind == LBM_PERIODIC) {
        if (!c->p.periodic[axis]) return fail(c, LBM_ERR_ARG, "axis %d is not periodic in the parameters", axis);
        return LBM_OK;
    }
    if (!std::isfinite(rho_wall) || rho_wall <= 0.0) return fail(c, LBM_ERR_ARG, "bad wall density");
    lbm_status s0 = before_replan(c);
    if (s0 != LBM_OK) return s0;
    const int f = 2 * axis + side;
    c->face_kind[f] = kind;
    for (int a = 0; a < 3; ++a) c->face_param[f].u[a] = u_wall ? u_wall[a] : 0.0;
    c->face_param[f].rho = rho_wall;
    c->plan_built = false;
    return LBM_OK;
}

lbm_status lbm_set_boundary(lbm_ctx *c, int32_t block, const uint8_t *flags, const double u_wall[3], double rho_wall)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_block(c, block);
    if (s != LBM_OK) return s;
    const BlockLayout &L = c->blocks[block];
    const size_t N = (size_t)L.n[0] * L.n[1] * L.n[2];
    if (!std::isfinite(rho_wall) || rho_wall <= 0.0) return fail(c, LBM_ERR_ARG, "bad wall density");
    if ((s = before_replan(c)) != LBM_OK) return s;
    if (!flags) {
        c->flags[block].clear();
    } else {
        for (size_t n = 0; n < N; ++n)
            if (flags[n] > LBM_PRESSURE) return fail(c, LBM_ERR_ARG, "flag value %d at cell %zu", flags[n], n);
        c->flags[block].assign(flags, flags + N);
    }
    for (int a = 0; a < 3; ++a) c->block_param[block].u[a] = u_wall ? u_wall[a] : 0.0;
    c->block_param[block].rho = rho_wall;
    c->plan_built = false;
    return LBM_OK;
}

lbm_status lbm_init_macroscopic(lbm_ctx *c, int32_t block, const double *rho, const double *u)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_owned(c, block);
    if (s != LBM_OK) return s;
    if (!rho || !u) return fail(c, LBM_ERR_ARG, "null rho or u");
    if ((s = prepare(c)) != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const BlockLayout &L = c->blocks[block];
    const int64_t N = (int64_t)L.n[0] * L.n[1] * L.n[2];
    CellArgs a = cell_args(c, block);
    double *vr = device_view(rho), *vu = device_view(u);
    if (vr && vu) {
        // page-locked host buffers: the kernel reads them over the host link itself
        a.rho = vr;
        a.u = vu;
    } else {
        if ((s = ensure_scratch(c, 4 * N)) != LBM_OK) return s;
        CK(cudaMemcpyAsync(c->d_scratch, rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy rho");
        CK(cudaMemcpyAsync(c->d_scratch + N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy u");
        a.rho = c->d_scratch;
        a.u = c->d_scratch + N;
    }
    CK(do_cells(c->q, c->storage, CELL_INIT, c->force ? 1 : 0, a), "init kernel");
    c->list_valid = false;  // the dense arrays hold the new state
    c->step_diag_valid = false;
    CK(cudaStreamSynchronize(c->stream), "init");
    return LBM_OK;
}

namespace {

// Launch arguments of a step that do not change from step to step.
void step_args(lbm_ctx *c, SweepArgs &sw, FillArgs &fa)
{
    const Plan &P = c->plan;
    sw = SweepArgs{};
    sw.blocks = c->d_blocks;
    sw.tiles = c->d_tiles;
    sw.ntiles = (int64_t)P.tiles.size();
    sw.tx = c->tile[0];
    sw.ty = c->tile[1];
    sw.tz = c->tile[2];
    sw.force = c->force ? 1 : 0;
    // neighbour mode of the launch: 0 none in place, 1 every in-place neighbour is the block
    // itself (wrap arithmetic), 2 general neighbour table
    sw.through = 0;
    for (size_t b = 0; b < c->blocks.size(); ++b) {
        if (!P.through[b]) continue;
        sw.through = std::max(sw.through, 1);
        for (int r = 0; r < 27; ++r)
            if (P.nbr[b][r] >= 0 && P.nbr[b][r] != (int)b) sw.through = 2;
    }
    // The wrap path (1) wraps each periodic axis of a source on its own, while the fill's
    // boundary links, the wet-node pass and the refinement transfers find a boundary cell the
    // way the neighbour table does: a source outside a non-periodic face is the block's own
    // ghost cell, unwrapped along the other axes.  With such boundaries the launch takes the
    // table path, so that the sweep reads the ghost slots where they were written.
    bool refine = false;
    for (int f = 0; f < 6; ++f) refine = refine || c->face_kind[f] == LBM_REFINE;
    if (sw.through == 1 && (!P.links.empty() || !P.zouhe.empty() || refine)) sw.through = 2;
    sw.stage_bytes = c->stage_bytes;
    sw.err = c->d_sweep_err;
    sw.idx32 = !c->wide_index && c->arena_elems <= ((int64_t)1 << 32) ? 1 : 0;
    sw.cd = c->cd;
    sw.cf = c->cf;
    sw.stream = c->stream;
    fa = FillArgs{};
    fa.blocks = c->d_blocks;
    fa.links = c->d_links;
    fa.nlinks = (int64_t)P.links.size();
    fa.params = c->d_params;
    fa.zouhe = c->d_zouhe;
    fa.nzouhe = (int64_t)P.zouhe.size();
    fa.zouhe_pressure = 0;
    for (int f = 0; f < 6; ++f)
        if (c->face_kind[f] == LBM_ZOUHE_PRESSURE) fa.zouhe_pressure |= 1 << f;
    for (int a = 0; a < 3; ++a) fa.F[a] = c->p.force[a];
    for (int i = 0; i < 27; ++i) fa.base[i] = c->base[i];
    fa.stream = c->stream;
}

// Issue one step (fill if needed, then the sweep) on the context's stream and advance the
// layout parity.  diag: the sweep writes the step diagnostics.
lbm_status issue_step(lbm_ctx *c, SweepArgs &sw, FillArgs &fa, bool diag, bool trace)
{
    const Plan &P = c->plan;
    lbm_status s = LBM_OK;
    if (c->pattern == LBM_TWO_GRID) {
        fa.a = c->arr[c->cur];
        fa.mode = FILL_PULL;
        fa.runs = c->d_runs_pull;
        fa.nruns = (int64_t)P.runs_pull.size();
        sw.a = c->arr[c->cur];
        sw.b = c->arr[1 - c->cur];
        sw.kind = SWEEP_PULL;
    } else {
        const bool even = c->aa_layout == LAYOUT_AA_E;
        fa.a = c->arr[0];
        fa.mode = even ? FILL_AA_E : FILL_AA_O;
        fa.runs = c->d_runs_aa;
        fa.nruns = (int64_t)P.runs_aa.size();
        sw.a = c->arr[0];
        sw.b = nullptr;
        sw.kind = even ? SWEEP_AA_NBR : SWEEP_AA_LOCAL;
    }
    int e0 = -1, e1 = -1, e2 = -1;
    if (c->sparse) {
        // the fluid-cell list layout: link slots, then the list sweep (two-grid)
        if ((s = ensure_list(c)) != LBM_OK) return s;
        SparseArgs fl, sp;
        sparse_args(c, SPARSE_FILL, fl);
        fl.dst = c->sarr[c->cur];
        sparse_args(c, SPARSE_SWEEP, sp);
        sp.src = c->sarr[c->cur];
        sp.dst = c->sarr[1 - c->cur];
        sp.partials = diag ? c->d_step_partials : nullptr;
        if (trace && (s = mark(c, &e0)) != LBM_OK) return s;
        if (fl.nlinks > 0) {
            CK(do_sparse(c->q, c->storage, fl), "list boundary fill launch");
            c->launches++;
        }
        if (trace && (s = mark(c, &e1)) != LBM_OK) return s;
        if (sp.nfluid > 0) {
            CK(do_sparse(c->q, c->storage, sp), "list sweep launch");
            c->launches++;
        }
        if (trace) {
            if ((s = mark(c, &e2)) != LBM_OK) return s;
            if (fl.nlinks > 0) c->ev_marks[0].push_back({e0, e1});
            if (sp.nfluid > 0) c->ev_marks[1].push_back({e1, e2});
        }
        c->cur = 1 - c->cur;
        c->dense_valid = false;
        return LBM_OK;
    }
    if (trace && (s = mark(c, &e0)) != LBM_OK) return s;
    if (fa.nlinks + fa.nruns > 0) {
        CK(do_fill(c->q, c->storage, fa), "boundary/ghost fill launch");
        c->launches++;
    }
    if (fa.nzouhe > 0 && c->pattern == LBM_TWO_GRID) {
        // after the fill: a node may read ghost slots the fill wrote
        CK(do_zouhe(c->q, c->storage, fa), "wet-node boundary launch");
        c->launches++;
    }
    if (trace && (s = mark(c, &e1)) != LBM_OK) return s;
    sw.partials = diag ? c->d_step_partials : nullptr;
    if (sw.ntiles > 0 && c->per_block) {
        // one launch per block over its own tile range (comparison mode)
        SweepArgs one = sw;
        for (size_t b = 0; b + 1 < c->tile_start.size(); ++b) {
            one.tiles = sw.tiles + c->tile_start[b];
            one.ntiles = c->tile_start[b + 1] - c->tile_start[b];
            one.partials = diag ? c->d_step_partials + 8 * c->tile_start[b] : nullptr;
            if (one.ntiles == 0) continue;
            CK(sweep_of(c, one), "sweep launch");
            c->launches++;
        }
    } else if (sw.ntiles > 0) {
        CK(sweep_of(c, sw), "sweep launch");
        c->launches++;
    }
    if (trace) {
        if ((s = mark(c, &e2)) != LBM_OK) return s;
        if (fa.nlinks + fa.nruns + fa.nzouhe > 0) c->ev_marks[0].push_back({e0, e1});
        if (sw.ntiles > 0) c->ev_marks[1].push_back({e1, e2});
    }
    if (c->pattern == LBM_TWO_GRID)
        c->cur = 1 - c->cur;
    else
        c->aa_layout = c->aa_layout == LAYOUT_AA_E ? LAYOUT_AA_O : LAYOUT_AA_E;
    return LBM_OK;
}

int parity(const lbm_ctx *c) { return c->pattern == LBM_TWO_GRID ? c->cur : (c->aa_layout == LAYOUT_AA_E ? 0 : 1); }

void drop_graphs(lbm_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_epoch[k] = -1;
    }
}

// Two steps (no diagnostics) as one CUDA-graph launch; the pair ends in the parity it started
// from, so one graph per starting parity serves every later pair.
lbm_status graph_pair(lbm_ctx *c, SweepArgs &sw, FillArgs &fa)
{
    const int k = parity(c);
    if (!c->graph[k] || c->graph_epoch[k] != c->list_epoch) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        const int64_t launches = c->launches;
        const int cur = c->cur, lay = c->aa_layout;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin graph capture");
        lbm_status s1 = issue_step(c, sw, fa, false, false);
        lbm_status s2 = s1 == LBM_OK ? issue_step(c, sw, fa, false, false) : s1;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->launches = launches;  // captured, not yet run
        c->cur = cur;
        c->aa_layout = lay;
        if (s2 != LBM_OK) {
            if (g) cudaGraphDestroy(g);
            return s2;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "end graph capture");
        e = cudaGraphInstantiate(&c->graph[k], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "instantiate step graph");
        c->graph_epoch[k] = c->list_epoch;
    }
    CK(cudaGraphLaunch(c->graph[k], c->stream), "graph launch");
    // account for the two steps the graph ran
    const Plan &P = c->plan;
    const int64_t sweeps = c->per_block ? (int64_t)c->blocks.size() : 1;
    const int64_t per_step = (sw.ntiles > 0 ? sweeps : 0) +
                             ((P.links.size() + (c->pattern == LBM_TWO_GRID ? P.runs_pull.size() : P.runs_aa.size())) > 0 ? 1 : 0);
    c->launches += 2 * per_step;
    return LBM_OK;
}

lbm_status check_diag(lbm_ctx *c)
{
    lbm_diagnostics d;
    lbm_status r = lbm_step_diagnostics(c, &d);
    if (r != LBM_OK) return r;
    if (d.nonfinite > 0 || !std::isfinite(d.mass))
        return fail(c, LBM_ERR_DIVERGED, "non-finite state after step %lld (%lld cells)", (long long)c->steps_done,
                    (long long)d.nonfinite);
    return LBM_OK;
}

}  // namespace

lbm_status lbm_step(lbm_ctx *c, int64_t n)
{
    if (!c) return LBM_ERR_ARG;
    if (n < 0) return fail(c, LBM_ERR_ARG, "negative step count");
    lbm_status s = prepare(c);
    if (s != LBM_OK) return s;
    if (n > 1 && has_halo(c))
        return fail(c, LBM_ERR_STATE, "partitioned context: one step per call (the halo exchange comes between steps)");
    if ((s = ensure_list(c)) != LBM_OK) return s;  // outside any graph capture
    if (c->sparse && n > 0) c->dense_valid = false;  // replayed graphs do not pass through issue_step
    SweepArgs sw;
    FillArgs fa;
    step_args(c, sw, fa);
    const int64_t di = c->p.diag_interval;
    const bool graphs = c->graph_mode && c->stream != nullptr && !c->timing;
    for (int64_t t = 0; t < n;) {
        // diagnostics on the call's last step and on every diag_interval-th step
        auto diag_at = [&](int64_t k) { return k == n - 1 || (di > 0 && (c->steps_done + (k - t) + 1) % di == 0); };
        if (graphs && t + 2 <= n - 1 && !diag_at(t) && !diag_at(t + 1)) {
            if ((s = graph_pair(c, sw, fa)) != LBM_OK) return s;
            c->steps_done += 2;
            c->step_diag_valid = false;
            t += 2;
            continue;
        }
        const bool diag = diag_at(t);
        if ((s = issue_step(c, sw, fa, diag, c->timing)) != LBM_OK) return s;
        c->step_diag_valid = diag;
        c->steps_done++;
        ++t;
        if (di > 0 && c->steps_done % di == 0 && (s = check_diag(c)) != LBM_OK) return s;
    }
    return LBM_OK;
}

lbm_status lbm_set_closure(lbm_ctx *c, int32_t kind, double cs, const float *mlp_params)
{
    if (!c) return LBM_ERR_ARG;
    if (kind != LBM_CLOSURE_NONE && kind != LBM_CLOSURE_SMAGORINSKY && kind != LBM_CLOSURE_MLP)
        return fail(c, LBM_ERR_ARG, "unknown closure kind %d", kind);
    if (kind == LBM_CLOSURE_NONE) {
        c->closure = CLOSURE_NONE;
        drop_graphs(c);
        return LBM_OK;
    }
    if (kind == LBM_CLOSURE_SMAGORINSKY && !(std::isfinite(cs) && cs >= 0.0))
        return fail(c, LBM_ERR_ARG, "bad Smagorinsky constant");
    if (kind == LBM_CLOSURE_MLP && !mlp_params) return fail(c, LBM_ERR_ARG, "null network parameters");
    if (c->q != 19 || c->storage != LBM_FP32 || c->force || c->p.collision == LBM_MRT)
        return fail(c, LBM_ERR_UNSUPPORTED, "closures need D3Q19, FP32 storage, SRT or TRT and no body force");
    for (int f = 0; f < 6; ++f)
        if (c->face_kind[f] == LBM_ZOUHE_VELOCITY || c->face_kind[f] == LBM_ZOUHE_PRESSURE)
            return fail(c, LBM_ERR_UNSUPPORTED, "closures are not combined with wet-node faces");
    if (kind == LBM_CLOSURE_MLP) {
        const MlpDev d = mlp_device_form(mlp_params);
        if (!c->d_mlp) CK(cudaMalloc((void **)&c->d_mlp, sizeof(MlpDev)), "cudaMalloc(network)");
        if (!c->d_tc_err) {
            CK(cudaMalloc((void **)&c->d_tc_err, sizeof(int)), "cudaMalloc(network status)");
            CK(cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream), "clear network status");
        }
        CK(cudaMemcpyAsync(c->d_mlp, &d, sizeof d, cudaMemcpyHostToDevice, c->stream), "copy network");
        CK(cudaStreamSynchronize(c->stream), "copy network");
    }
    c->closure = kind;
    c->closure_cs = cs;
    drop_graphs(c);  // captured sweeps carry the old closure
    return LBM_OK;
}

lbm_status lbm_set_in_place(lbm_ctx *c, int32_t enable)
{
    if (!c) return LBM_ERR_ARG;
    if ((enable != 0) != (c->in_place != 0)) {
        // an AA state after an odd number of steps may hold values in ghost slots (ghost mode)
        // or in neighbour cells (in-place mode): the two forms only agree in the even layout
        if (c->pattern == LBM_AA && c->aa_layout != LAYOUT_AA_E)
            return fail(c, LBM_ERR_STATE, "switch the neighbour mode of an AA context after an even number of steps");
        lbm_status s = before_replan(c);
        if (s != LBM_OK) return s;
        c->in_place = enable != 0;
        c->plan_built = false;  // rebuilt (and re-uploaded) before the next step
        drop_graphs(c);
    }
    return LBM_OK;
}

lbm_status lbm_set_batching(lbm_ctx *c, int32_t batched)
{
    if (!c) return LBM_ERR_ARG;
    c->per_block = batched == 0;
    drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_graph(lbm_ctx *c, int32_t enable)
{
    if (!c) return LBM_ERR_ARG;
    if (enable && c->stream == nullptr)
        return fail(c, LBM_ERR_UNSUPPORTED, "graph mode needs a non-default stream (capture is not allowed on stream 0)");
    if (enable && !c->owner.empty())
        return fail(c, LBM_ERR_UNSUPPORTED, "graph mode replays step pairs; a partitioned context exchanges its halo "
                                            "between steps");
    c->graph_mode = enable != 0;
    if (!enable) drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_index_bits(lbm_ctx *c, int32_t bits)
{
    if (!c) return LBM_ERR_ARG;
    if (bits != 32 && bits != 64) return fail(c, LBM_ERR_ARG, "index bits must be 32 or 64, not %d", bits);
    c->wide_index = bits == 64;
    drop_graphs(c);  // captured launches carry the previous choice
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx *c, int32_t trial_steps, int32_t best[3], int32_t *best_in_place, double *best_ms)
{
    if (!c || !best) return LBM_ERR_ARG;
    if (trial_steps < 1) return fail(c, LBM_ERR_ARG, "trial_steps must be >= 1");
    if (!c->owner.empty()) return fail(c, LBM_ERR_UNSUPPORTED, "autotune runs steps without a halo exchange");
    if (c->sparse) return fail(c, LBM_ERR_UNSUPPORTED, "autotune picks dense tiles; the list layout has none");
    lbm_status s = prepare(c);
    if (s != LBM_OK) return s;
    // keep the simulation state: snapshot the PDF arrays, start every trial from it, restore
    const int narr = c->pattern == LBM_TWO_GRID ? 2 : 1;
    const size_t bytes1 = (size_t)c->arena_elems * c->bpp;
    void *snap = nullptr;
    CK(cudaMalloc(&snap, narr * bytes1), "cudaMalloc(autotune snapshot)");
    for (int k = 0; k < narr; ++k)
        CK(cudaMemcpyAsync((char *)snap + k * bytes1, c->arr[k], bytes1, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
    const int cur = c->cur, lay = c->aa_layout;
    const int64_t steps_done = c->steps_done, launches = c->launches, di = c->p.diag_interval;
    const bool diag_valid = c->step_diag_valid, timing = c->timing;
    const int old[3] = {c->tile[0], c->tile[1], c->tile[2]}, old_in_place = c->in_place;
    // the neighbour mode may change only where both forms of the state agree (see lbm_set_in_place)
    const bool try_modes = c->pattern == LBM_TWO_GRID || lay == LAYOUT_AA_E;
    // the last three give small blocks (a 32^3 box: 32 tiles of 256 x 1 x 4) enough CTAs
    static const int cand[][3] = {{256, 1, 4}, {256, 1, 2}, {256, 1, 8}, {256, 1, 16}, {128, 2, 4}, {128, 2, 8},
                                  {64, 4, 4},  {64, 4, 8},  {32, 8, 4},  {128, 1, 8},  {64, 2, 8}, {64, 1, 16},
                                  {256, 1, 1}, {64, 2, 2},  {32, 4, 1}};
    const int ncand = (int)(sizeof cand / sizeof cand[0]);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    float best_t = 1e30f;
    int bi = -1, bmode = old_in_place;
    c->timing = false;
    c->p.diag_interval = 0;  // trial steps are timed only
    for (int mode = 0; mode < 2 && s == LBM_OK; ++mode) {
        const int in_place = mode == 0 ? old_in_place : !old_in_place;
        if (mode == 1 && !try_modes) break;
        for (int k = 0; k < ncand; ++k) {
            for (int a = 0; a < 3; ++a) c->tile[a] = cand[k][a];
            c->in_place = in_place;
            c->plan_built = false;
            if ((s = prepare(c)) != LBM_OK) break;
            for (int j = 0; j < narr; ++j)
                CK(cudaMemcpyAsync(c->arr[j], (char *)snap + j * bytes1, bytes1, cudaMemcpyDeviceToDevice, c->stream),
                   "trial start");
            c->cur = cur;
            c->aa_layout = lay;
            if ((s = lbm_step(c, 2)) != LBM_OK) break;
            CK(cudaEventRecord(e0, c->stream), "event");
            if ((s = lbm_step(c, trial_steps)) != LBM_OK) break;
            CK(cudaEventRecord(e1, c->stream), "event");
            CK(cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1), "event");
            if (ms < best_t) {
                best_t = ms;
                bi = k;
                bmode = in_place;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int *pick = bi >= 0 ? cand[bi] : old;
    for (int a = 0; a < 3; ++a) c->tile[a] = best[a] = pick[a];
    c->in_place = bi >= 0 ? bmode : old_in_place;
    if (best_in_place) *best_in_place = c->in_place;
    c->plan_built = false;
    drop_graphs(c);
    lbm_status s2 = prepare(c);
    for (int k = 0; k < narr; ++k)
        CK(cudaMemcpyAsync(c->arr[k], (char *)snap + k * bytes1, bytes1, cudaMemcpyDeviceToDevice, c->stream), "restore");
    CK(cudaStreamSynchronize(c->stream), "autotune restore");
    cudaFree(snap);
    c->cur = cur;
    c->aa_layout = lay;
    c->steps_done = steps_done;
    c->launches = launches;
    c->step_diag_valid = diag_valid;
    c->timing = timing;
    c->p.diag_interval = di;
    if (best_ms) *best_ms = bi >= 0 ? best_t / trial_steps : 0.0;
    return s != LBM_OK ? s : s2;
}

lbm_status lbm_get_macroscopic(lbm_ctx *c, int32_t block, double *rho, double *u)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_owned(c, block);
    if (s != LBM_OK) return s;
    if (!rho || !u) return fail(c, LBM_ERR_ARG, "null output");
    if ((s = prepare(c)) != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const BlockLayout &L = c->blocks[block];
    const int64_t N = (int64_t)L.n[0] * L.n[1] * L.n[2];
    CellArgs a = cell_args(c, block);
    double *vr = device_view(rho), *vu = device_view(u);
    if (vr && vu) {
        // page-locked host buffers: the kernel writes them over the host link itself
        a.rho = vr;
        a.u = vu;
        CK(do_cells(c->q, c->storage, CELL_MACRO, 0, a), "macroscopic kernel");
    } else {
        if ((s = ensure_scratch(c, 4 * N)) != LBM_OK) return s;
        a.rho = c->d_scratch;
        a.u = c->d_scratch + N;
        CK(do_cells(c->q, c->storage, CELL_MACRO, 0, a), "macroscopic kernel");
        CK(cudaMemcpyAsync(rho, c->d_scratch, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy rho");
        CK(cudaMemcpyAsync(u, c->d_scratch + N, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy u");
    }
    CK(cudaStreamSynchronize(c->stream), "get_macroscopic");
    return wait_status(c);
}

lbm_status lbm_coarse_moments(lbm_ctx *c, int32_t block, int32_t ratio, double *out)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_owned(c, block);
    if (s != LBM_OK) return s;
    if (!out) return fail(c, LBM_ERR_ARG, "null output");
    const BlockLayout &L = c->blocks[block];
    if (ratio < 1 || L.n[0] % ratio || L.n[1] % ratio || L.n[2] % ratio)
        return fail(c, LBM_ERR_ARG, "block %d (%d x %d x %d) is not divisible by ratio %d", block, L.n[0], L.n[1], L.n[2],
                    ratio);
    if ((s = prepare(c)) != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const int64_t Nc = (int64_t)(L.n[0] / ratio) * (L.n[1] / ratio) * (L.n[2] / ratio);
    if ((s = ensure_scratch(c, 10 * Nc)) != LBM_OK) return s;
    CellArgs a = cell_args(c, block);
    a.f64 = c->d_scratch;
    a.ratio = ratio;
    CK(do_cells(c->q, c->storage, CELL_COARSE, 0, a), "coarse moments kernel");
    CK(cudaMemcpyAsync(out, c->d_scratch, 10 * Nc * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "copy coarse moments");
    CK(cudaStreamSynchronize(c->stream), "coarse_moments");
    return wait_status(c);
}

lbm_status lbm_get_pdfs(lbm_ctx *c, int32_t block, double *f)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_owned(c, block);
    if (s != LBM_OK) return s;
    if (!f) return fail(c, LBM_ERR_ARG, "null output");
    if ((s = prepare(c)) != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const BlockLayout &L = c->blocks[block];
    const int64_t N = (int64_t)L.n[0] * L.n[1] * L.n[2];
    if ((s = ensure_scratch(c, (int64_t)c->q * N)) != LBM_OK) return s;
    CellArgs a = cell_args(c, block);
    a.f64 = c->d_scratch;
    CK(do_cells(c->q, c->storage, CELL_GET, 0, a), "get_pdfs kernel");
    CK(cudaMemcpyAsync(f, c->d_scratch, (size_t)c->q * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "copy pdfs");
    CK(cudaStreamSynchronize(c->stream), "get_pdfs");
    return wait_status(c);
}

lbm_status lbm_get_pdfs_region(lbm_ctx *c, int32_t block, const int32_t origin[3], const int32_t size[3], double *f)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_owned(c, block);
    if (s != LBM_OK) return s;
    if (!f || !origin || !size) return fail(c, LBM_ERR_ARG, "null argument");
    const BlockLayout &L = c->blocks[block];
    for (int a = 0; a < 3; ++a)
        if (size[a] < 1 || origin[a] < 0 || (int64_t)origin[a] + size[a] > L.n[a])
            return fail(c, LBM_ERR_ARG, "region outside block %d along axis %d", block, a);
    if ((s = prepare(c)) != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const int64_t N = (int64_t)size[0] * size[1] * size[2];
    if ((s = ensure_scratch(c, (int64_t)c->q * N)) != LBM_OK) return s;
    CellArgs a = cell_args(c, block);
    a.f64 = c->d_scratch;
    for (int k = 0; k < 3; ++k) {
        a.r0[k] = origin[k];
        a.rn[k] = size[k];
    }
    CK(do_cells(c->q, c->storage, CELL_GET, 0, a), "get_pdfs_region kernel");
    CK(cudaMemcpyAsync(f, c->d_scratch, (size_t)c->q * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "copy pdfs");
    CK(cudaStreamSynchronize(c->stream), "get_pdfs_region");
    return wait_status(c);
}

lbm_status lbm_set_pdfs(lbm_ctx *c, int32_t block, const double *f)
{
    if (!c) return LBM_ERR_ARG;
    lbm_status s = check_owned(c, block);
    if (s != LBM_OK) return s;
    if (!f) return fail(c, LBM_ERR_ARG, "null input");
    if ((s = prepare(c)) != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const BlockLayout &L = c->blocks[block];
    const int64_t N = (int64_t)L.n[0] * L.n[1] * L.n[2];
    if ((s = ensure_scratch(c, (int64_t)c->q * N)) != LBM_OK) return s;
    CK(cudaMemcpyAsync(c->d_scratch, f, (size_t)c->q * N * sizeof(double), cudaMemcpyHostToDevice, c->stream),
       "copy pdfs");
    CellArgs a = cell_args(c, block);
    a.f64 = c->d_scratch;
    CK(do_cells(c->q, c->storage, CELL_SET, 0, a), "set_pdfs kernel");
    c->list_valid = false;  // the dense arrays hold the new state
    c->step_diag_valid = false;
    CK(cudaStreamSynchronize(c->stream), "set_pdfs");
    return LBM_OK;
}

lbm_status lbm_reduce_blocks(lbm_ctx *c, double *out)
{
    if (!c || !out) return LBM_ERR_ARG;
    lbm_status s = prepare(c);
    if (s != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    const int64_t nb = (int64_t)c->blocks.size();
    std::fill(out, out + 8 * nb, 0.0);
    if (c->plan.tiles.empty()) return LBM_OK;
    if ((s = ensure_scratch(c, 8 * nb + nb + 1)) != LBM_OK) return s;  // records + int64 ranges
    // tile ranges of the blocks (tiles are stored block by block) after the output records
    int64_t *d_start = reinterpret_cast<int64_t *>(c->d_scratch + 8 * nb);
    CK(cudaMemcpyAsync(d_start, c->tile_start.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream),
       "copy tile ranges");
    ReduceArgs r{};
    r.a = c->pattern == LBM_TWO_GRID ? c->arr[c->cur] : c->arr[0];
    r.blocks = c->d_blocks;
    r.tiles = c->d_tiles;
    r.ntiles = (int64_t)c->plan.tiles.size();
    r.tx = c->tile[0];
    r.ty = c->tile[1];
    r.tz = c->tile[2];
    r.layout = state_layout(c);
    for (int a = 0; a < 3; ++a) r.F[a] = c->p.force[a];
    for (int i = 0; i < 27; ++i) r.base[i] = c->base[i];
    r.partials = c->d_partials;
    r.out = c->d_out;
    r.stream = c->stream;
    CK(do_reduce(c->q, c->storage, r), "reduction kernels");
    CK(launch_block_final(c->d_partials, d_start, nb, c->d_scratch, c->stream), "per-block reduction");
    CK(cudaMemcpyAsync(out, c->d_scratch, 8 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "copy per-block diagnostics");
    CK(cudaStreamSynchronize(c->stream), "reduce_blocks");
    return wait_status(c);
}

lbm_status lbm_reduce(lbm_ctx *c, lbm_diagnostics *out)
{
    if (!c || !out) return LBM_ERR_ARG;
    lbm_status s = prepare(c);
    if (s != LBM_OK) return s;
    if ((s = ensure_dense(c)) != LBM_OK) return s;
    double h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (!c->plan.tiles.empty()) {
        ReduceArgs r{};
        r.a = c->pattern == LBM_TWO_GRID ? c->arr[c->cur] : c->arr[0];
        r.blocks = c->d_blocks;
        r.tiles = c->d_tiles;
        r.ntiles = (int64_t)c->plan.tiles.size();
        r.tx = c->tile[0];
        r.ty = c->tile[1];
        r.tz = c->tile[2];
        r.layout = state_layout(c);
        for (int a = 0; a < 3; ++a) r.F[a] = c->p.force[a];
        for (int i = 0; i < 27; ++i) r.base[i] = c->base[i];
        r.partials = c->d_partials;
        r.out = c->d_out;
        r.stream = c->stream;
        CK(do_reduce(c->q, c->storage, r), "reduction kernels");
        CK(cudaMemcpyAsync(h, c->d_out, sizeof h, cudaMemcpyDeviceToHost, c->stream), "copy diagnostics");
        CK(cudaStreamSynchronize(c->stream), "reduce");
    }
    out->mass = h[0];
    out->momentum[0] = h[1];
    out->momentum[1] = h[2];
    out->momentum[2] = h[3];
    out->kinetic_energy = h[4];
    out->max_speed = h[5];
    out->nonfinite = (int64_t)h[6];
    out->fluid_cells = (int64_t)h[7];
    return wait_status(c);
}

lbm_status lbm_selfcheck_wait(lbm_ctx *c, int32_t polls)
{
    if (!c) return LBM_ERR_ARG;
    if (polls < 1 || polls > (1 << 20)) return fail(c, LBM_ERR_ARG, "polls %d outside [1, 2^20]", polls);
    lbm_status s = prepare(c);
    if (s != LBM_OK) return s;
    CK(launch_wait_selfcheck(c->d_sweep_err, (uint32_t)polls, c->stream), "wait self-check");
    CK(cudaStreamSynchronize(c->stream), "wait self-check");
    return LBM_OK;
}

lbm_status lbm_step_diagnostics(lbm_ctx *c, lbm_diagnostics *out)
{
    if (!c || !out) return LBM_ERR_ARG;
    if (!c->step_diag_valid || !c->h_io) return fail(c, LBM_ERR_STATE, "no step has run since the state was last set");
    double *h = c->h_io->diag;
    std::fill(h, h + 8, 0.0);
    if (diag_records(c) > 0) {
        CK(launch_reduce_final(c->d_step_partials, diag_records(c), c->d_out, c->stream), "diagnostics kernel");
        CK(cudaMemcpyAsync(h, c->d_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy diagnostics");
    }
    lbm_status ws = wait_status_enqueue(c);
    if (ws != LBM_OK) return ws;
    CK(cudaStreamSynchronize(c->stream), "step diagnostics");  // one synchronisation for both reads
    if ((ws = wait_status_take(c)) != LBM_OK) return ws;
    out->mass = h[0];
    out->momentum[0] = h[1];
    out->momentum[1] = h[2];
    out->momentum[2] = h[3];
    out->kinetic_energy = h[4];
    out->max_speed = h[5];
    out->nonfinite = (int64_t)h[6];
    out->fluid_cells = (int64_t)h[7];
    return LBM_OK;
}

lbm_status lbm_step_diagnostics_post(lbm_ctx *c, int64_t *ticket)
{
    if (!c || !ticket) return LBM_ERR_ARG;
    if (!c->step_diag_valid || !c->h_io) return fail(c, LBM_ERR_STATE, "no step has run since the state was last set");
    int k = -1;
    for (int j = 0; j < LBM_DIAG_SLOTS && k < 0; ++j) {
        const int s = (int)((c->next_ticket + j) % LBM_DIAG_SLOTS);
        if (c->slot_ticket[s] < 0) k = s;
    }
    if (k < 0) return fail(c, LBM_ERR_STATE, "all %d diagnostics slots hold records not yet taken", LBM_DIAG_SLOTS);
    if (!c->slot_done[k]) CK(cudaEventCreateWithFlags(&c->slot_done[k], cudaEventDisableTiming), "cudaEventCreate");
    lbm_ctx::HostIO::Slot &h = c->h_io->slot[k];
    std::fill(h.diag, h.diag + 8, 0.0);
    h.wait_err[0] = h.wait_err[1] = 0;
    const int *tc_err = (c->d_tc_err && c->closure == CLOSURE_MLP) ? c->d_tc_err : nullptr;
    if (diag_records(c) > 0) {
        // the final sum writes the record and the wait-status flags into the slot itself
        lbm_ctx::HostIO::Slot *hd = &c->h_io_dev->slot[k];
        CK(launch_reduce_final_slot(c->d_step_partials, diag_records(c), c->d_out, hd->diag, hd->wait_err,
                                    c->d_sweep_err, tc_err, c->stream),
           "diagnostics kernel");
    } else {
        if (c->d_sweep_err)
            CK(cudaMemcpyAsync(&h.wait_err[0], c->d_sweep_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
               "read wait status");
        if (tc_err)
            CK(cudaMemcpyAsync(&h.wait_err[1], tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
               "read network status");
    }
    CK(cudaEventRecord(c->slot_done[k], c->stream), "cudaEventRecord");
    // the ticket names its slot: ticket % LBM_DIAG_SLOTS == k
    int64_t t = c->next_ticket;
    while (t % LBM_DIAG_SLOTS != k) ++t;
    c->slot_ticket[k] = t;
    c->next_ticket = t + 1;
    *ticket = t;
    return LBM_OK;
}

lbm_status lbm_step_diagnostics_take(lbm_ctx *c, int64_t ticket, lbm_diagnostics *out)
{
    if (!c || !out || ticket < 0) return LBM_ERR_ARG;
    const int k = (int)(ticket % LBM_DIAG_SLOTS);
    if (c->slot_ticket[k] != ticket) return fail(c, LBM_ERR_STATE, "diagnostics ticket %lld is not pending", (long long)ticket);
    c->slot_ticket[k] = -1;
    CK(cudaEventSynchronize(c->slot_done[k]), "step diagnostics");
    const lbm_ctx::HostIO::Slot &h = c->h_io->slot[k];
    if (h.wait_err[0] || h.wait_err[1]) {
        // the flags are cleared and reported as lbm_step_diagnostics reports them
        c->h_io->wait_err[0] = h.wait_err[0];
        c->h_io->wait_err[1] = h.wait_err[1];
        return wait_status_take(c);
    }
    out->mass = h.diag[0];
    out->momentum[0] = h.diag[1];
    out->momentum[1] = h.diag[2];
    out->momentum[2] = h.diag[3];
    out->kinetic_energy = h.diag[4];
    out->max_speed = h.diag[5];
    out->nonfinite = (int64_t)h.diag[6];
    out->fluid_cells = (int64_t)h.diag[7];
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_ctx *c, lbm_info *out)
{
    if (!c || !out) return LBM_ERR_ARG;
    lbm_status s = build_lists(c);
    if (s != LBM_OK) return s;
    const Plan &P = c->plan;
    out->cells = P.cells;
    out->fluid_cells = P.fluid_cells;
    for (int k = 0; k < 4; ++k) out->links[k] = P.link_count[k];
    const bool tg = c->pattern == LBM_TWO_GRID;
    out->ghost_slots = tg ? P.ghost_slots_pull : P.ghost_slots_aa;
    out->ghost_runs = (int64_t)(tg ? P.runs_pull.size() : P.runs_aa.size());
    out->tiles = (int64_t)P.tiles.size();
    out->bytes_per_pdf = c->bpp;
    out->device_bytes = (int64_t)(c->arena_owned ? c->arena_bytes : 0) + (int64_t)c->list_bytes +
                        c->partials_cap * 8 + c->scratch_cap * 8;
    stage_tiles(c, P, nullptr, &out->staged_tiles);
    out->list_entries = c->sparse ? P.sparse.nslots : 0;
    if (c->sparse) out->links[LBM_VELOCITY] = out->links[LBM_PRESSURE] = 0;
    for (const uint64_t w : P.sparse.links) out->links[(w >> 5) & 3u]++;
    return LBM_OK;
}

lbm_status lbm_plan_sparse(lbm_ctx *c, int32_t what, int64_t *out, int64_t cap, int64_t *n)
{
    if (!c || !n) return LBM_ERR_ARG;
    if (!c->sparse) return fail(c, LBM_ERR_STATE, "the context does not use the fluid-cell list layout");
    if (what < 0 || what > 3) return fail(c, LBM_ERR_ARG, "bad list part %d", what);
    lbm_status s = build_lists(c);
    if (s != LBM_OK) return s;
    const SparsePlan &S = c->plan.sparse;
    const int64_t len = what == 0 ? (int64_t)S.nbr.size()
                                  : (what == 1 ? S.nfluid : (what == 2 ? S.nfluid : (int64_t)S.links.size()));
    *n = len;
    if (!out) return LBM_OK;
    if (cap < len) return fail(c, LBM_ERR_ARG, "buffer too small");
    for (int64_t k = 0; k < len; ++k)
        out[k] = what == 0 ? (int64_t)S.nbr[k]
                           : (what == 1 ? S.block_of[k] : (what == 2 ? S.cell_of[k] : (int64_t)S.links[k]));
    return LBM_OK;
}

lbm_status lbm_set_sparse(lbm_ctx *c, int32_t enable)
{
    if (!c) return LBM_ERR_ARG;
    if (enable && c->pattern != LBM_TWO_GRID)
        return fail(c, LBM_ERR_UNSUPPORTED, "the fluid-cell list layout is built for the two-grid pattern");
    bool zouhe = false;
    for (int f = 0; f < 6; ++f) zouhe = zouhe || c->face_kind[f] == LBM_ZOUHE_VELOCITY || c->face_kind[f] == LBM_ZOUHE_PRESSURE;
    if (enable && zouhe) return fail(c, LBM_ERR_UNSUPPORTED, "the fluid-cell list layout has no wet-node faces");
    if (enable && (!c->owner.empty() || c->closure != CLOSURE_NONE || c->p.collision >= LBM_MRT))
        return fail(c, LBM_ERR_UNSUPPORTED, "the fluid-cell list layout is for SRT/TRT contexts holding every block, "
                                            "without a closure");
    if ((enable != 0) == c->sparse) return LBM_OK;
    lbm_status s = LBM_OK;
    if (c->dev_ready && (s = ensure_dense(c)) != LBM_OK) return s;  // the state moves back to the dense arrays
    c->sparse = enable != 0;
    c->plan_built = false;
    c->dense_valid = true;
    c->list_valid = false;
    drop_graphs(c);
    return LBM_OK;
}

lbm_status lbm_set_tile(lbm_ctx *c, int32_t tx, int32_t ty, int32_t tz)
{
    if (!c) return LBM_ERR_ARG;
    if (tx <= 0 || ty <= 0 || tz <= 0 || tx % 32 != 0 || tx * ty > 256 || tx > 32000 || ty > 32000 || tz > 32000)
        return fail(c, LBM_ERR_ARG, "bad tile %d x %d x %d (tx multiple of 32, tx*ty <= 256)", tx, ty, tz);
    lbm_status s = before_replan(c);
    if (s != LBM_OK) return s;
    c->tile[0] = tx;
    c->tile[1] = ty;
    c->tile[2] = tz;
    c->plan_built = false;
    return LBM_OK;
}

lbm_status lbm_enable_timing(lbm_ctx *c, int32_t enable)
{
    if (!c) return LBM_ERR_ARG;
    c->timing = enable != 0;
    return LBM_OK;
}

lbm_status lbm_read_timing(lbm_ctx *c, double ms[2], int64_t count[2], int32_t reset)
{
    if (!c || !ms || !count) return LBM_ERR_ARG;
    for (int k = 0; k < 2; ++k) {
        ms[k] = 0.0;
        count[k] = (int64_t)c->ev_marks[k].size();
    }
    if (!c->ev_marks[0].empty() || !c->ev_marks[1].empty()) {
        CK(cudaStreamSynchronize(c->stream), "synchronise for timing");
        for (int k = 0; k < 2; ++k)
            for (const auto &m : c->ev_marks[k]) {
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, c->ev_pool[m.first], c->ev_pool[m.second]), "cudaEventElapsedTime");
                ms[k] += t;
            }
    }
    if (reset) {
        c->ev_marks[0].clear();
        c->ev_marks[1].clear();
        c->ev_used = 0;
    }
    return LBM_OK;
}

int64_t lbm_kernel_launches(const lbm_ctx *c) { return c ? c->launches : 0; }

lbm_status lbm_stencil_table(int32_t q, int32_t *cv, double *w, int32_t *opp)
{
    if (q != 19 && q != 27) return LBM_ERR_ARG;
    const LatticeView L = lattice_view(q);
    for (int i = 0; i < q; ++i) {
        if (cv) {
            cv[3 * i] = L.cx[i];
            cv[3 * i + 1] = L.cy[i];
            cv[3 * i + 2] = L.cz[i];
        }
        if (w) w[i] = L.w[i];
        if (opp) opp[i] = L.opp[i];
    }
    return LBM_OK;
}

lbm_status lbm_plan_links(lbm_ctx *c, uint64_t *out, int64_t cap, int64_t *n)
{
    if (!c || !n) return LBM_ERR_ARG;
    lbm_status s = build_lists(c);
    if (s != LBM_OK) return s;
    *n = (int64_t)c->plan.links.size();
    if (!out) return LBM_OK;
    if (cap < *n) return fail(c, LBM_ERR_ARG, "buffer too small");
    memcpy(out, c->plan.links.data(), (size_t)*n * sizeof(uint64_t));
    return LBM_OK;
}

lbm_status lbm_plan_runs(lbm_ctx *c, int32_t pattern, int64_t *out, int64_t cap, int64_t *n)
{
    if (!c || !n) return LBM_ERR_ARG;
    lbm_status s = build_lists(c);
    if (s != LBM_OK) return s;
    const std::vector<GhostRun> &R = pattern == LBM_TWO_GRID ? c->plan.runs_pull : c->plan.runs_aa;
    *n = (int64_t)R.size();
    if (!out) return LBM_OK;
    if (cap < 5 * *n) return fail(c, LBM_ERR_ARG, "buffer too small");
    for (size_t r = 0; r < R.size(); ++r) {
        out[5 * r] = R[r].src;
        out[5 * r + 1] = R[r].dst;
        out[5 * r + 2] = R[r].len;
        out[5 * r + 3] = R[r].sstride;
        out[5 * r + 4] = R[r].dstride;
    }
    return LBM_OK;
}

lbm_status lbm_plan_layout(lbm_ctx *c, int32_t block, int64_t out[10])
{
    if (!c || !out) return LBM_ERR_ARG;
    lbm_status s = check_block(c, block);
    if (s != LBM_OK) return s;
    if ((s = build_lists(c)) != LBM_OK) return s;
    const BlockLayout &L = c->blocks[block];
    out[0] = L.xo;
    out[1] = L.pitch;
    out[2] = L.plane;
    out[3] = L.slab;
    out[4] = L.offset;
    out[5] = L.n[0];
    out[6] = L.n[1];
    out[7] = L.n[2];
    out[8] = c->arena_elems;
    out[9] = c->plan.through[block];
    return LBM_OK;
}

lbm_status lbm_plan_neighbors(lbm_ctx *c, int32_t block, int32_t out[27])
{
    if (!c || !out) return LBM_ERR_ARG;
    lbm_status s = check_block(c, block);
    if (s != LBM_OK) return s;
    if ((s = build_lists(c)) != LBM_OK) return s;
    for (int r = 0; r < 27; ++r) out[r] = c->plan.nbr[block][r];
    return LBM_OK;
}

lbm_status lbm_plan_mask(lbm_ctx *c, int32_t block, uint32_t *out, int64_t cap, int64_t *n)
{
    if (!c || !n) return LBM_ERR_ARG;
    lbm_status s = check_block(c, block);
    if (s != LBM_OK) return s;
    if ((s = build_lists(c)) != LBM_OK) return s;
    const std::vector<uint32_t> &m = c->plan.masks[block];
    *n = (int64_t)m.size();
    if (!out) return LBM_OK;
    if (cap < *n) return fail(c, LBM_ERR_ARG, "buffer too small");
    if (*n) memcpy(out, m.data(), (size_t)*n * sizeof(uint32_t));
    return LBM_OK;
}

lbm_status lbm_plan_params(lbm_ctx *c, double *out, int64_t cap, int64_t *n)
{
    if (!c || !n) return LBM_ERR_ARG;
    lbm_status s = build_lists(c);
    if (s != LBM_OK) return s;
    *n = (int64_t)c->plan.params.size();
    if (!out) return LBM_OK;
    if (cap < 4 * *n) return fail(c, LBM_ERR_ARG, "buffer too small");
    for (size_t k = 0; k < c->plan.params.size(); ++k) {
        for (int a = 0; a < 3; ++a) out[4 * k + a] = c->plan.params[k].u[a];
        out[4 * k + 3] = c->plan.params[k].rho;
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------
// Static 2:1 refinement (Sec. 5.1.1, Rohde et al.): a coarse and a fine context side by side
// along x in a domain periodic in all three axes; the transfer lists (refine.cu) are built here
// once from the two blocks' layouts.  See include/lbm.h for the scheme.
// ---------------------------------------------------------------------------------------
struct lbm_refine {
    lbm_ctx *coarse = nullptr, *fine = nullptr;
    int64_t *d_explode = nullptr, *d_coalesce = nullptr;
    int64_t nexplode = 0, ncoalesce = 0;
    // CUDA-graph replay of one coarse step, one graph per (coarse, fine) array parity; valid
    // while both contexts' device lists and arrays are those it captured
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t graph_epoch[4][2] = {};
    void *graph_arr[4][4] = {};
    int64_t graph_launches[4] = {0, 0, 0, 0};
};

namespace {

bool refine_faces(const lbm_ctx *c) { return c->face_kind[0] == LBM_REFINE && c->face_kind[1] == LBM_REFINE; }

// The transfer entries (element offsets relative to an array's base).
void refine_entries(const lbm_ctx *cc, const lbm_ctx *cf, std::vector<int64_t> &ex, std::vector<int64_t> &co)
{
    const BlockLayout &C = cc->blocks[0], &F = cf->blocks[0];
    const LatticeView L = lattice_view(cc->q);
    const int nxc = C.n[0], nxf = F.n[0], nyf = F.n[1], nzf = F.n[2], nyc = C.n[1], nzc = C.n[2];
    auto wrap = [](int v, int n) { return ((v % n) + n) % n; };
    // explosion: fine cells of the first / last column, directions entering through the face;
    // the value comes from the coarse column holding the fine ghost cells (the coarse block's
    // last column beside the fine x- face, its first column beside the fine x+ face)
    for (int side = 0; side < 2; ++side) {
        const int xf = side == 0 ? 0 : nxf - 1, sx = side == 0 ? 1 : -1, xc = side == 0 ? nxc - 1 : 0;
        for (int z = 0; z < nzf; ++z)
            for (int y = 0; y < nyf; ++y)
                for (int i = 0; i < L.q; ++i) {
                    if (L.cx[i] != sx) continue;
                    const int cy = L.cy[i], cz = L.cz[i];
                    ex.push_back(F.offset + (int64_t)i * F.slab + F.cell(xf - sx, y - cy, z - cz));
                    // first fine step: the ghost one cell out; second: the one two cells out
                    ex.push_back(C.offset + (int64_t)i * C.slab + C.cell(xc, wrap(y - cy, nyf) / 2, wrap(z - cz, nzf) / 2));
                    ex.push_back(C.offset + (int64_t)i * C.slab +
                                 C.cell(xc, wrap(y - 2 * cy, nyf) / 2, wrap(z - 2 * cz, nzf) / 2));
                }
    }
    // coalescence: coarse cells beside the fine block, directions coming out of it; the fine
    // cells whose populations streamed into the coarse cell's 8 fine ghost cells: into the one
    // cell out during the second fine step (emitted at t + 1/2), into the two cells out over
    // both steps (emitted at t)
    for (int side = 0; side < 2; ++side) {
        const int xc = side == 0 ? nxc - 1 : 0, sx = side == 0 ? -1 : 1, xf = side == 0 ? 0 : nxf - 1;
        for (int Z = 0; Z < nzc; ++Z)
            for (int Y = 0; Y < nyc; ++Y)
                for (int i = 0; i < L.q; ++i) {
                    if (L.cx[i] != sx) continue;
                    const int cy = L.cy[i], cz = L.cz[i];
                    co.push_back(C.offset + (int64_t)i * C.slab + C.cell(xc - sx, Y - cy, Z - cz));
                    for (int half = 0; half < 2; ++half)
                        for (int dz = 0; dz < 2; ++dz)
                            for (int dy = 0; dy < 2; ++dy) {
                                const int k = half + 1;
                                co.push_back(F.offset + (int64_t)i * F.slab +
                                             F.cell(xf, wrap(2 * Y + dy - k * cy, nyf), wrap(2 * Z + dz - k * cz, nzf)));
                            }
                }
    }
}

lbm_status refine_launch(lbm_ctx *c, bool explode, RefineArgs &a)
{
    CK(explode ? launch_refine_explode(a) : launch_refine_coalesce(a), explode ? "explosion launch" : "coalescence launch");
    c->launches++;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_refine_create(lbm_ctx *cc, lbm_ctx *cf, lbm_refine **out)
{
    if (!cc || !cf || !out || cc == cf) return LBM_ERR_ARG;
    *out = nullptr;
    const char *why = nullptr;
    if (cc->q != cf->q || cc->storage != cf->storage) why = "the two contexts differ in stencil or storage";
    for (const lbm_ctx *c : {cc, cf}) {
        if (why) break;
        if (c->storage != LBM_FP64 && c->storage != LBM_FP32) why = "FP64 or FP32 storage";
        else if (c->pattern != LBM_TWO_GRID) why = "the two-grid pattern";
        else if (c->p.collision != LBM_SRT && c->p.collision != LBM_TRT) why = "SRT or TRT";
        else if (c->blocks.size() != 1 || !c->owner.empty() || c->sparse || c->closure != CLOSURE_NONE)
            why = "one block per context, the dense layout, no closure";
        else if (c->p.periodic[0] || !c->p.periodic[1] || !c->p.periodic[2] || !refine_faces(c))
            why = "x faces of kind LBM_REFINE, y and z periodic";
        else if (!c->flags[0].empty()) why = "no obstacle cells";
        else if (c->graph_mode) why = "no graph mode";
    }
    if (!why && (cc->p.collision != cf->p.collision ||
                 (cc->p.collision == LBM_TRT && cc->p.magic_lambda != cf->p.magic_lambda)))
        why = "the same collision (and Lambda) on both grids";
    if (!why && cc->stream != cf->stream) why = "one stream for both contexts";
    if (!why) {
        const BlockLayout &C = cc->blocks[0], &F = cf->blocks[0];
        if (F.n[0] % 2 != 0 || F.n[1] != 2 * C.n[1] || F.n[2] != 2 * C.n[2])
            why = "the fine block must be 2W x 2ny x 2nz for a coarse block of ny x nz";
    }
    if (!why) {
        // acoustic scaling: the same physical viscosity and body force on both grids
        const double wf = cc->p.omega > 0.0 ? 1.0 / (0.5 + 2.0 * (1.0 / cc->p.omega - 0.5)) : -1.0;
        if (!(std::fabs(cf->p.omega - wf) <= 1e-12 * wf)) why = "fine omega = 1 / (1/2 + 2 (1/omega_c - 1/2))";
        for (int a = 0; a < 3 && !why; ++a)
            if (cf->p.force[a] != 0.5 * cc->p.force[a]) why = "fine force = coarse force / 2";
    }
    if (why) return fail(cc, LBM_ERR_UNSUPPORTED, "refinement: %s", why);
    lbm_status s;
    if ((s = prepare(cc)) != LBM_OK) return s;
    if ((s = prepare(cf)) != LBM_OK) return s;
    std::vector<int64_t> ex, co;
    refine_entries(cc, cf, ex, co);
    lbm_refine *r = new (std::nothrow) lbm_refine();
    if (!r) return LBM_ERR_OOM;
    r->coarse = cc;
    r->fine = cf;
    r->nexplode = (int64_t)ex.size() / 3;
    r->ncoalesce = (int64_t)co.size() / 9;
    lbm_ctx *c = cc;
    cudaError_t e = cudaMalloc(&r->d_explode, ex.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&r->d_coalesce, co.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpy(r->d_explode, ex.data(), ex.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_coalesce, co.data(), co.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(r->d_explode);
        cudaFree(r->d_coalesce);
        delete r;
        return cuda_fail(c, e, "refinement lists");
    }
    *out = r;
    return LBM_OK;
}

namespace {

// One coarse step of the refined pair, enqueued on the contexts' stream.
lbm_status refine_one(lbm_refine *r, SweepArgs &swc, FillArgs &fac, SweepArgs &swf, FillArgs &faf)
{
    lbm_ctx *cc = r->coarse, *cf = r->fine;
    lbm_status s;
    RefineArgs a{};
    a.elem_bytes = cc->bpp;
    a.stream = cc->stream;
    // two fine steps, each after the explosion into the ghost slots it reads
    for (int sub = 1; sub <= 2; ++sub) {
        a.dst = cf->arr[cf->cur];
        a.src = cc->arr[cc->cur];
        a.src2 = nullptr;
        a.ent = r->d_explode;
        a.n = r->nexplode;
        a.sub = sub;
        if ((s = refine_launch(cf, true, a)) != LBM_OK) return s;
        if ((s = issue_step(cf, swf, faf, false, cf->timing)) != LBM_OK) return s;
        if (sub == 1) {
            // coalescence into the coarse ghost slots while both fine states it needs exist:
            // the populations the fine cells emit at the start of each fine step, f*(t)
            // (still in the first step's source array) and f*(t + 1/2) (its result)
            a.dst = cc->arr[cc->cur];
            a.src = cf->arr[cf->cur];
            a.src2 = cf->arr[1 - cf->cur];
            a.ent = r->d_coalesce;
            a.n = r->ncoalesce;
            if ((s = refine_launch(cc, false, a)) != LBM_OK) return s;
        }
    }
    // the coarse step
    return issue_step(cc, swc, fac, false, cc->timing);
}

}  // namespace

lbm_status lbm_refine_step(lbm_refine *r, int64_t n)
{
    if (!r) return LBM_ERR_ARG;
    lbm_ctx *cc = r->coarse, *cf = r->fine;
    if (n < 0) return fail(cc, LBM_ERR_ARG, "negative step count");
    if (!refine_faces(cc) || !refine_faces(cf) || cc->graph_mode || cf->graph_mode)
        return fail(cc, LBM_ERR_STATE, "refinement: a context changed its x faces or took graph mode");
    lbm_status s;
    if ((s = prepare(cc)) != LBM_OK) return s;
    if ((s = prepare(cf)) != LBM_OK) return s;
    SweepArgs swc, swf;
    FillArgs fac, faf;
    step_args(cc, swc, fac);
    step_args(cf, swf, faf);
    // graph replay needs a stream that can be captured; traced steps run one launch at a time
    const bool graphs = cc->stream != nullptr && !cc->timing && !cf->timing;
    for (int64_t t = 0; t < n; ++t) {
        if (!graphs) {
            if ((s = refine_one(r, swc, fac, swf, faf)) != LBM_OK) return s;
        } else {
            const int k = 2 * cc->cur + cf->cur;
            void *arrs[4] = {cc->arr[0], cc->arr[1], cf->arr[0], cf->arr[1]};
            bool stale = !r->graph[k] || r->graph_epoch[k][0] != cc->list_epoch || r->graph_epoch[k][1] != cf->list_epoch;
            for (int j = 0; j < 4 && !stale; ++j) stale = r->graph_arr[k][j] != arrs[j];
            if (stale) {
                if (r->graph[k]) cudaGraphExecDestroy(r->graph[k]);
                r->graph[k] = nullptr;
                const int64_t lc = cc->launches, lf = cf->launches;
                const int curc = cc->cur, curf = cf->cur;
                lbm_ctx *c = cc;
                CK(cudaStreamBeginCapture(cc->stream, cudaStreamCaptureModeThreadLocal), "begin refinement capture");
                lbm_status s1 = refine_one(r, swc, fac, swf, faf);
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamEndCapture(cc->stream, &g);
                r->graph_launches[k] = (cc->launches - lc) + (cf->launches - lf);
                cc->launches = lc;  // captured, not yet run
                cf->launches = lf;
                cc->cur = curc;
                cf->cur = curf;
                if (s1 != LBM_OK) {
                    if (g) cudaGraphDestroy(g);
                    return s1;
                }
                if (e != cudaSuccess) return cuda_fail(c, e, "end refinement capture");
                e = cudaGraphInstantiate(&r->graph[k], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(c, e, "instantiate refinement graph");
                r->graph_epoch[k][0] = cc->list_epoch;
                r->graph_epoch[k][1] = cf->list_epoch;
                for (int j = 0; j < 4; ++j) r->graph_arr[k][j] = arrs[j];
            }
            {
                lbm_ctx *c = cc;
                CK(cudaGraphLaunch(r->graph[k], cc->stream), "refinement graph launch");
            }
            // what the graph did: two fine steps (its arrays back where they were), one coarse
            cc->cur = 1 - cc->cur;
            cc->launches += r->graph_launches[k];
        }
        cf->steps_done += 2;
        cc->steps_done++;
    }
    cc->step_diag_valid = cf->step_diag_valid = false;
    return LBM_OK;
}

void lbm_refine_destroy(lbm_refine *r)
{
    if (!r) return;
    if (r->coarse) cudaStreamSynchronize(r->coarse->stream);
    for (cudaGraphExec_t &g : r->graph)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(r->d_explode);
    cudaFree(r->d_coalesce);
    delete r;
}

const char *lbm_last_error(const lbm_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    if (c->dev_ready || c->arena_owned) cudaStreamSynchronize(c->stream);
    if (c->arena_owned) cudaFree(c->arena_raw);
    dfree(c->d_blocks);
    dfree(c->d_links);
    dfree(c->d_zouhe);
    dfree(c->d_runs_pull);
    dfree(c->d_runs_aa);
    for (HaloDevRun *&h : c->d_halo) dfree(h);
    dfree(c->d_snbr);
    dfree(c->d_sblock);
    dfree(c->d_scell);
    dfree(c->d_slinks);
    if (c->sarr_raw) cudaFree(c->sarr_raw);
    dfree(c->d_tiles);
    dfree(c->d_params);
    dfree(c->d_masks);
    dfree(c->d_partials);
    dfree(c->d_step_partials);
    dfree(c->d_out);
    dfree(c->d_scratch);
    dfree(c->d_mlp);
    dfree(c->d_tc_err);
    dfree(c->d_sweep_err);
    if (c->h_io) cudaFreeHost(c->h_io);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->slot_done)
        if (e) cudaEventDestroy(e);
    drop_graphs(c);
    delete c;
}

}  // extern "C"
