/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann library (liblbm.so).
 *
 * The library runs the hot path of the block-structured lattice Boltzmann method described
 * in the waLBerla paper (arXiv:1909.13772) on one GPU:
 *   - the fused stream-collide sweep (Sec. 5.1.1, Eq. 1-2; Sec. 5.1.2: streaming and
 *     collision fused in one kernel), D3Q19 or D3Q27, SRT or TRT collision (Eq. 3 with
 *     special S), Guo body force (Sec. 5.1.1, body-force paragraph);
 *   - structure-of-arrays PDF fields with one ghost layer per block (Sec. 4.1 structured
 *     grids; Sec. 4.2 fields: SoA layout, padded aligned rows);
 *   - boundary sweeps driven by per-kind boundary link lists built from flag fields
 *     (Sec. 4.4: one index list per boundary condition, each with its own kernel; no-slip,
 *     velocity and pressure kinds from Sec. 5.1.1), plus periodic domain faces;
 *   - the ghost-layer copy between blocks held on the same GPU (Sec. 3.3: PackInfo copies
 *     directly between blocks of one process, without buffers; Sec. 4.2: ghost layers are
 *     exchanged between sweeps);
 *   - device compute with host mirrors only for set-up and output (Sec. 4.3).
 * The paper states its kernels are callable through a C ABI (Sec. 6.1 on code generation);
 * this header is that interface for this library.
 *
 * Conventions
 *   - Every function returns lbm_status and never aborts.  On error, lbm_last_error(ctx)
 *     gives a message.  CUDA errors are caught after each launch sequence (LBM_ERR_CUDA).
 *   - Host buffers are owned by the caller and only touched during the call.
 *   - Device memory is owned by the context (cudaMalloc) or, for the PDF arrays, by the
 *     caller through lbm_bind_device_memory (e.g. a PyTorch tensor).
 *   - A context is not thread-safe; it issues all work on one CUDA stream (given at
 *     creation).  lbm_step returns without synchronising the host; lbm_get_* and
 *     lbm_set_* synchronise the stream.
 *   - Cell arrays on the host are per block, interior cells only, x fastest:
 *     index = x + nx (y + ny z).  Vector fields are SoA: u[a*N + index], a = x, y, z.
 *     PDF arrays are f[i*N + index] in the canonical direction order below.
 *   - Canonical direction order (D3Q19): 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the 12
 *     vectors with |c|^2 = 2 in lexicographic order of (cx,cy,cz).  D3Q27 appends the 8
 *     corner vectors in lexicographic order as 19..26.  Weights: D3Q19 1/3, 1/18, 1/36;
 *     D3Q27 8/27, 2/27, 1/54, 1/216; c_s^2 = 1/3.
 *   - The stored state is the post-collision field f*(x, t) (the right-hand side of Eq. 2);
 *     lbm_get_macroscopic returns rho = sum f*, u = (sum c f* - F/2) / rho.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument */
    LBM_ERR_STATE = 2,       /* call not valid in the context's current state */
    LBM_ERR_CUDA = 3,        /* a CUDA call or kernel launch failed */
    LBM_ERR_OOM = 4,         /* device or host allocation failed / bound buffer too small */
    LBM_ERR_DIVERGED = 5,    /* diagnostics found non-finite values */
    LBM_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    LBM_ERR_UNSUPPORTED = 7  /* valid request the library does not support */
} lbm_status;

enum { LBM_D3Q19 = 19, LBM_D3Q27 = 27 };
/* Collision (Sec. 5.1.1, Eq. 3): SRT and TRT are the special relaxation matrices the paper
 * names; MRT relaxes groups of moments with their own rates: the shear moments with omega,
 * momentum and the third-order moments with omega- (from magic_lambda, as TRT), the bulk,
 * fourth-, fifth- and sixth-order groups with mrt_rates.  The moment space: polynomials of c
 * grouped by degree, each group orthogonal to all lower groups under sum_i w_i a(c_i) b(c_i).
 * MRT is available with FP64 and FP32 storage.
 * Cumulant (Sec. 5.1.1: cumulants instead of moments relaxed towards their equilibria; Geier et
 * al. 2015), D3Q27 with FP64 or FP32 storage: the density-scaled cumulants of the central
 * moments about the half-force-shifted velocity, relaxed in ten groups -- shear (omega) and
 * cumulant_rates[0..8] for the bulk, third-order sums, third-order differences, C_111,
 * fourth-order differences, fourth-order sum, mixed fourth order, fifth and sixth order; all
 * equilibria zero beyond the second order (rho/3 on its diagonal); the body force through the
 * first central moments (-F/2 before, +F/2 after). */
enum { LBM_SRT = 0, LBM_TRT = 1, LBM_MRT = 2, LBM_CUMULANT = 3 };
/* PDF storage: FP64 and FP32 store f_i; the *_DEV forms store f_i - w_i rho0 in 16 bits and
 * collide in FP32. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_BF16_DEV = 2, LBM_FP16_DEV = 3 };
/* Two-grid: source and destination arrays swapped every step.  AA: one array updated in
 * place with alternating even/odd access patterns. */
enum { LBM_TWO_GRID = 0, LBM_AA = 1 };
/* Cell kinds of a flag field, and kinds of a domain face. */
enum { LBM_FLUID = 0, LBM_NOSLIP = 1, LBM_VELOCITY = 2, LBM_PRESSURE = 3, LBM_PERIODIC = 4 };
/* Face kinds only: wet-node velocity and pressure faces (Zou & He; the node is the fluid cell of
 * the first layer, the unknown populations entering it are rebuilt from mass and momentum before
 * each sweep).  D3Q19, two-grid pattern, dense layout; the face's two tangential axes periodic. */
enum { LBM_ZOUHE_VELOCITY = 5, LBM_ZOUHE_PRESSURE = 6 };
/* Face kind only: a refinement interface (lbm_refine_create); the ghost slots the sweep reads
 * through it are written by lbm_refine_step.  Two-grid pattern, FP64/FP32, dense layout. */
enum { LBM_REFINE = 7 };

typedef struct {
    int32_t stencil;       /* LBM_D3Q19 or LBM_D3Q27 */
    int32_t collision;     /* LBM_SRT, LBM_TRT, LBM_MRT or LBM_CUMULANT */
    int32_t storage;       /* LBM_FP64 ... */
    int32_t pattern;       /* LBM_TWO_GRID or LBM_AA */
    double omega;          /* SRT: omega = 1/tau; TRT: omega+ (sets the viscosity); MRT, cumulant:
                              shear rate */
    double magic_lambda;   /* TRT, MRT: Lambda = (1/omega+ - 1/2)(1/omega- - 1/2); 3/16 typical */
    double force[3];       /* constant body force per cell (lattice units), Guo scheme */
    double rho0;           /* reference density (1.0); base of the *_DEV storages */
    int32_t periodic[3];   /* non-zero: the domain is periodic along that axis */
    int32_t diag_interval; /* >0: lbm_step checks the diagnostics every that many steps */
    double mrt_rates[4];   /* MRT: rates of the bulk, fourth-, fifth- and sixth-order groups, each
                              in [0, 2) (fifth and sixth: D3Q27 only); ignored otherwise.  TRT is
                              omega, omega, omega-, omega */
    double cumulant_rates[9]; /* cumulant: rates of the groups after shear (see LBM_CUMULANT),
                                 each in [0, 2); ignored otherwise */
} lbm_params;

/* One block: global cell coordinates of its first interior cell and its interior size.
 * Blocks must not overlap.  The domain is the bounding box of all blocks; cells of the
 * bounding box not covered by any block are treated as no-slip solid. */
typedef struct {
    int64_t origin[3];
    int32_t size[3];
} lbm_block_desc;

/* Domain totals over fluid cells (FP64, deterministic order). */
typedef struct {
    double mass;           /* sum rho */
    double momentum[3];    /* sum rho u (physical velocity, half-force corrected) */
    double kinetic_energy; /* sum rho |u|^2 / 2 */
    double max_speed;      /* max |u| */
    int64_t nonfinite;     /* number of fluid cells with a non-finite PDF */
    int64_t fluid_cells;   /* number of fluid cells */
} lbm_diagnostics;

/* Sizes of the work one lbm_step performs, from the built boundary and ghost lists.  No-slip
 * links (links[LBM_NOSLIP]) are applied inside the sweep from cell masks; velocity and
 * pressure links go through the fill kernel's link list. */
typedef struct {
    int64_t cells;          /* interior cells of all blocks */
    int64_t fluid_cells;    /* interior fluid cells */
    int64_t links[4];       /* boundary links by kind (index LBM_NOSLIP..LBM_PRESSURE) */
    int64_t ghost_slots;    /* PDF values copied by the ghost exchange per step */
    int64_t ghost_runs;     /* copy runs in the ghost exchange list */
    int64_t tiles;          /* sweep tiles (CTAs) per step */
    int64_t bytes_per_pdf;  /* bytes of one stored PDF value */
    int64_t device_bytes;   /* device memory held by the context */
    int64_t staged_tiles;   /* tiles whose source rows the two-grid sweep stages in shared
                               memory by bulk copies (16-bit storage, unmasked full-width tiles) */
    int64_t list_entries;   /* fluid-cell list layout (lbm_set_sparse): entries per direction
                               (fluid cells + boundary link slots); 0 for the dense layout */
} lbm_info;

/* Create a context for `nblocks` blocks.  `cuda_stream` is a cudaStream_t (or NULL for the
 * default stream) on which all work of the context is issued.  Uses the current CUDA
 * device.  No device memory is allocated yet (see lbm_bind_device_memory).
 * Errors: LBM_ERR_ARG for invalid parameters or overlapping blocks.
 * Paper: Sec. 4.1 (the domain as a set of blocks of cells), Sec. 4.2 (per-block fields, SoA, one
 * ghost layer, padded rows). */
lbm_status lbm_create_blocks(const lbm_params *params, const lbm_block_desc *blocks, int32_t nblocks,
                             void *cuda_stream, lbm_ctx **out);

/* ---- partitioned runs (one context per rank / GPU) ---------------------------------------
 * The blocks of one domain are distributed over ranks; each rank holds the PDFs of its own
 * blocks, and the ghost layers of blocks next to another rank's blocks are filled by a halo
 * exchange between steps (Sec. 3.1: blocks distributed over processes along a space-filling
 * curve; Sec. 3.3: ghost-layer exchange of only the PDFs that cross into a neighbour, packed
 * into one message per neighbour process).  The library packs and unpacks; the caller moves
 * the buffers between ranks (NCCL send/recv, or any transport) -- the C ABI carries no
 * communicator.  One step of a partitioned run:
 *     for every peer: lbm_halo_pack(ctx, peer, send_buf[peer])
 *     exchange: send_buf[peer] -> peer, receive recv_buf[peer] from peer (sizes from lbm_halo_sizes)
 *     for every peer: lbm_halo_unpack(ctx, peer, recv_buf[peer])
 *     lbm_step(ctx, 1)
 * and once before the first step after lbm_init_macroscopic / lbm_set_pdfs.  Pack and unpack
 * are enqueued on the context's stream; the buffers must stay valid until that work is done. */

/* Owner rank of every block along the Morton (Z-order) curve of the block centres: blocks in
 * curve order are cut into nranks contiguous pieces of nearly equal weight (weights[b], or the
 * block's cell count when weights is NULL).  Host only (no GPU needed).
 * Errors: LBM_ERR_ARG for empty input, sizes < 1, negative or non-finite weights.
 * Paper: Sec. 3.1 (blocks assigned to processes along a space-filling curve). */
lbm_status lbm_partition_morton(const lbm_block_desc *blocks, int32_t nblocks, int32_t nranks, const double *weights,
                                int32_t *owner);

/* A context for rank `rank` of `nranks` that holds the blocks with owner[b] == rank (owner:
 * nblocks entries in [0, nranks)); the other blocks describe the domain (neighbours, ghost
 * shells) but get no device memory.  Every rank must be created with the same parameters,
 * blocks, owner array, faces and flags: lbm_set_boundary is accepted for every block (the
 * ghost shells of owned blocks take kinds from their neighbours' flags) and must be given for
 * all of them.  Per-block calls that touch PDFs (init, get, set, macroscopic) accept owned
 * blocks only (LBM_ERR_ARG otherwise); lbm_reduce covers the owned blocks (sum the ranks'
 * results).  With a halo to exchange, lbm_step advances one step per call (LBM_ERR_STATE for
 * n > 1), and graph replay and lbm_autotune are refused (LBM_ERR_UNSUPPORTED).
 * Errors: as lbm_create_blocks; LBM_ERR_ARG for a bad owner array or a rank that owns no block.
 * Paper: Sec. 3.1 (distributed blocks), Sec. 4.2 (per-block fields with one ghost layer). */
lbm_status lbm_create_partition(const lbm_params *params, const lbm_block_desc *blocks, int32_t nblocks,
                                const int32_t *owner, int32_t nranks, int32_t rank, void *cuda_stream,
                                lbm_ctx **out);

/* Elements (of the storage type: 8, 4 or 2 bytes) this rank sends to and receives from `peer`
 * in the exchange that must precede the next step.  Two-grid: the crossing PDFs of the
 * owned cells next to the peer's blocks go to the peer's ghost layers.  AA: before the
 * neighbour sweep the same forward exchange of the AA slots; before the local sweep the
 * reverse one (the values the neighbour sweep wrote into ghost slots go back to the peer
 * that owns those cells), so send and receive sizes swap from step to step.  0 and 0 when
 * the two ranks share no face.  Host only.
 * Errors: LBM_ERR_STATE for a context that is not partitioned, LBM_ERR_ARG for a bad peer.
 * Paper: Sec. 3.3 (ghost-layer exchange, only the directions that cross). */
lbm_status lbm_halo_sizes(lbm_ctx *ctx, int32_t peer, int64_t *send_elems, int64_t *recv_elems);

/* Enqueue the pack of this step's halo for `peer` into the device buffer dev_buf (at least
 * send_elems elements of lbm_halo_sizes; caller-owned) on the context's stream.  Nothing is
 * launched when send_elems is 0.
 * Errors: as lbm_halo_sizes; LBM_ERR_ARG for a null buffer; LBM_ERR_CUDA.
 * Paper: Sec. 3.3 (PackInfo: the data of a block face packed into a message buffer). */
lbm_status lbm_halo_pack(lbm_ctx *ctx, int32_t peer, void *dev_buf);

/* Enqueue the unpack of the halo received from `peer` (device buffer of at least recv_elems
 * elements) into this rank's PDF array on the context's stream.
 * Errors: as lbm_halo_pack.
 * Paper: Sec. 3.3 (PackInfo: unpacking the message into the ghost layer). */
lbm_status lbm_halo_unpack(lbm_ctx *ctx, int32_t peer, const void *dev_buf);

/* ---- static 2:1 grid refinement (Sec. 5.1.1: non-uniform grids, the mass-conserving method of
 * Rohde et al. 2006) --------------------------------------------------------------------------
 * A coarse context and a fine context that together fill a domain periodic in x, y and z: the
 * coarse block covers coarse columns [0, A) and the fine block the coarse columns [A, A + W) with
 * 2W x 2ny x 2nz fine cells (the coarse block being A x ny x nz); both have y and z periodic and
 * both x faces of kind LBM_REFINE.  Volumetric scheme, one coarse step:
 *   1. explosion: each fine ghost cell (two layers beyond each fine x face, inside the coarse
 *      column beside it) holds the post-collision populations of its coarse cell;
 *   2. two fine steps (the ghost values streaming one fine cell per step);
 *   3. coalescence: a coarse cell beside the fine block takes, for each direction coming out of
 *      it, the mean over its 8 fine cells of the fine populations that streamed into them
 *      during the two fine steps; then the coarse step.
 * No interpolation and no rescaling of non-equilibrium parts; every population that crosses
 * the interface is counted once on each side, so sum_coarse f + (1/8) sum_fine f is conserved.
 * Requirements (else LBM_ERR_UNSUPPORTED): same stencil, FP64 or FP32 storage, two-grid, SRT or
 * TRT with the same Lambda, one block per context without obstacle cells, no closure, no graph
 * mode, one stream; fine omega = 1 / (1/2 + 2 (1/omega_c - 1/2)) (the same physical viscosity
 * under acoustic scaling) and fine force = coarse force / 2.
 * The object keeps pointers to both contexts: destroy it before them.  Errors: LBM_ERR_ARG for
 * null or identical contexts, LBM_ERR_OOM, LBM_ERR_CUDA. */
typedef struct lbm_refine lbm_refine;
lbm_status lbm_refine_create(lbm_ctx *coarse, lbm_ctx *fine, lbm_refine **out);

/* Enqueue n coarse steps (each: explosion, fine step, coalescence, explosion, fine step,
 * coarse step; the coalescence runs while the fine states at t and t + 1/2, whose emitted
 * populations it averages, both exist) on the contexts' stream.  On a stream other than the
 * legacy default stream, and with tracing off, each coarse step is replayed as a CUDA graph
 * captured once per array parity (its six launches with no host work in between).  The step diagnostics of both contexts are not
 * written (lbm_reduce gives each grid's totals).  Errors: LBM_ERR_STATE if a context's x faces
 * changed or it took graph mode since lbm_refine_create; as lbm_step. */
lbm_status lbm_refine_step(lbm_refine *r, int64_t n);

void lbm_refine_destroy(lbm_refine *r);

/* Bytes of device memory the PDF arrays need (two arrays for two-grid, one for AA),
 * including 256-byte alignment slack.
 * Paper: Sec. 4.2 (field memory layout); the caller-owned buffer has no counterpart there. */
size_t lbm_required_bytes(const lbm_ctx *ctx);

/* Optional: place the PDF arrays in caller-owned device memory `dev_ptr` of `bytes` bytes
 * (at least lbm_required_bytes).  Must be called before any call that touches PDFs.  The
 * caller keeps the buffer alive until lbm_destroy.  Without it the library cudaMallocs.
 * Boundary lists, masks and reduction scratch are always allocated by the library.
 * Errors: LBM_ERR_OOM if too small, LBM_ERR_STATE if the arrays already exist.
 * Paper: Sec. 4.2 (field memory layout); the caller-owned buffer has no counterpart there. */
lbm_status lbm_bind_device_memory(lbm_ctx *ctx, void *dev_ptr, size_t bytes);

/* Kind of the region outside a domain face (axis 0..2, side 0 = low, 1 = high):
 * LBM_NOSLIP, LBM_VELOCITY (wall velocity u_wall, density rho_wall) or LBM_PRESSURE
 * (density rho_wall).  Faces of periodic axes are ignored.  Default: LBM_NOSLIP.
 * Paper: Sec. 5.1.1 (no-slip, velocity and pressure boundary kinds), Sec. 4.1 (periodic domain). */
lbm_status lbm_set_face(lbm_ctx *ctx, int32_t axis, int32_t side, int32_t kind, const double u_wall[3],
                        double rho_wall);

/* Flag field of one block: uint8 per interior cell (LBM_FLUID, LBM_NOSLIP, LBM_VELOCITY,
 * LBM_PRESSURE).  Velocity and pressure cells of this block use (u_wall, rho_wall).  NULL
 * flags = all fluid.  Boundary link lists and ghost-copy lists are (re)built on the host
 * before the next step.  Set flags before lbm_init_macroscopic: a cell that becomes fluid
 * later has no valid PDFs.
 * Paper: Sec. 4.4 (cell flags turned into one index list per boundary kind). */
lbm_status lbm_set_boundary(lbm_ctx *ctx, int32_t block, const uint8_t *flags, const double u_wall[3],
                            double rho_wall);

/* Initial state of one block from density rho[N] and velocity u[3N] (host, FP64): the
 * populations are the equilibrium at (rho, u - F/(2 rho)), so the half-force-corrected
 * velocity equals u; the stored state is their post-collision image, written in the
 * context's current storage layout (two-grid source array or the current AA parity).
 * Non-fluid cells are left untouched.  Page-locked host buffers (cudaHostAlloc, cudaHostRegister,
 * torch pin_memory) are read by the initialising kernel itself over the host link; other host
 * memory goes through a device staging copy.  Synchronises the stream.
 * Paper: Eq. 1 (moments of the equilibrium populations), Sec. 4.3 (set-up on the host, copied to
 * the GPU field). */
lbm_status lbm_init_macroscopic(lbm_ctx *ctx, int32_t block, const double *rho, const double *u);

/* Advance all blocks by n time steps (asynchronous on the context's stream).  Each step:
 * ghost-layer copy and boundary links, then the fused stream-collide sweep.  With
 * diag_interval > 0 the host reads the step diagnostics (lbm_step_diagnostics) every
 * diag_interval steps and returns LBM_ERR_DIVERGED when a value is non-finite.
 * Paper: Eq. 2 (stream and collide), Sec. 5.1.2 (one fused kernel), Sec. 4.4 (boundary sweeps),
 * Sec. 3.3 and 4.2 (ghost layers exchanged between sweeps). */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Density rho[N] and velocity u[3N] of one block's stored state (host FP64 buffers).
 * Non-fluid cells give 0.  Page-locked host buffers are written by the moment kernel itself over
 * the host link; other host memory through a device staging copy.  Synchronises the stream.
 * Paper: Eq. 1 (density and velocity moments), Sec. 4.3 (output through the host mirror). */
lbm_status lbm_get_macroscopic(lbm_ctx *ctx, int32_t block, double *rho, double *u);

/* Canonical post-collision PDFs f[Q*N] of one block (host FP64), whatever the pattern and
 * AA parity.  Non-fluid cells give 0.  Synchronises the stream.
 * Paper: Sec. 4.3 (the GPU field mirrored on the host). */
lbm_status lbm_get_pdfs(lbm_ctx *ctx, int32_t block, double *f);

/* PDFs of a box of a block's interior cells: origin[3] and size[3] in the block's interior
 * coordinates (inside the block), f[i * N + n] with n = x + sx (y + sy z) relative to the box,
 * N = sx sy sz, canonical direction order, FP64 (non-fluid cells read 0).  Synchronises the
 * stream.  Errors: LBM_ERR_ARG (null pointer, box outside the block).
 * Paper: Sec. 4.3 (the GPU field mirrored on the host, here a box of it). */
lbm_status lbm_get_pdfs_region(lbm_ctx *ctx, int32_t block, const int32_t origin[3], const int32_t size[3],
                               double *f);

/* Overwrite one block's state with canonical post-collision PDFs f[Q*N] (host FP64),
 * converted to the storage format.  Checkpoint restart: get_pdfs of every block, then
 * set_pdfs of every block continues the run exactly.  Synchronises the stream.
 * Paper: Sec. 4.3 (host mirror copied to the GPU field). */
lbm_status lbm_set_pdfs(lbm_ctx *ctx, int32_t block, const double *f);

/* Domain totals of the stored state over all fluid cells (FP64, deterministic: fixed
 * per-CTA partial sums reduced in a fixed order).  Synchronises the stream.
 * Paper: Eq. 1 (moments), summed over the domain; the reduction itself has no counterpart in the
 * paper. */
lbm_status lbm_reduce(lbm_ctx *ctx, lbm_diagnostics *out);

/* Diagnostics of the state produced by the most recent lbm_step, computed inside that
 * step's last sweep from the values it was writing (no extra pass over the state): per-cell,
 * per-thread and per-CTA sums in the sweep's arithmetic type (FP64 for FP64 storage; FP32 for
 * FP32 and 16-bit storage, with the mass an exact float-float sum of the stored values per cell
 * and float-float across cells, momentum and energy compensated per thread), FP64 across CTAs,
 * fixed order.  FP32 bounds against the FP64 pass (u = 2^-24): mass (Q + n + 3)^2 u^2 relative,
 * n the cells one thread sweeps (the tile's z extent, twice that in the paired 16-bit tiles),
 * for states whose rest population is at least every other population (each cell's sum is a
 * Fast2Sum chain started there; the deviation storages start it at rho0); momentum
 * 20 u mass + 9 u sum |rho u|.  Cheap enough to read after every step; lbm_reduce is
 * the full-FP64 pass over the stored values.  Synchronises the stream.
 * Errors: LBM_ERR_STATE when the state was set (init, set_pdfs) after the last step.
 * Paper: Eq. 1 (moments), summed over the domain inside the Sec. 5.1.2 sweep; no counterpart in
 * the paper. */
lbm_status lbm_step_diagnostics(lbm_ctx *ctx, lbm_diagnostics *out);

/* The same record read without synchronising the stream, so that a caller who reads every
 * step's diagnostics keeps the GPU busy (step k, post k, take k-1: step k+1 runs while the host
 * waits for record k).  lbm_step_diagnostics_post queues on the context's stream the final sum
 * of the most recent step's per-tile records and its copy, with the wait-status flags, into one
 * of LBM_DIAG_SLOTS pinned host slots, and returns in *ticket a number naming that slot's record;
 * later steps may be issued at once (the stream runs the sum before the next sweep rewrites the
 * tile records).  lbm_step_diagnostics_take waits for that record's copy (an event of its own,
 * not the whole stream), fills *out exactly as lbm_step_diagnostics would have for that step and
 * frees the slot.  Tickets may be taken in any order, each once.
 * Errors: post -- LBM_ERR_ARG (null pointer), LBM_ERR_STATE (no step has run since the state
 * was last set, or all LBM_DIAG_SLOTS slots hold records not yet taken); take -- LBM_ERR_ARG,
 * LBM_ERR_STATE (ticket never posted or already taken), LBM_ERR_TIMEOUT (a bounded wait of a
 * launch before the post gave up, see below; the slot is freed), LBM_ERR_CUDA.
 * Paper: Eq. 1 (moments), summed over the domain inside the Sec. 5.1.2 sweep; the pipelined read
 * has no counterpart in the paper. */
#define LBM_DIAG_SLOTS 4
lbm_status lbm_step_diagnostics_post(lbm_ctx *ctx, int64_t *ticket);
lbm_status lbm_step_diagnostics_take(lbm_ctx *ctx, int64_t ticket, lbm_diagnostics *out);

/* Bounded device-side waits.  The kernels that wait on an mbarrier give up, set a device
 * status flag and return: the staged sweep after 1 s of the GPU's global timer per wait for its
 * bulk copies (the give-up is taken by the whole CTA, which then issues no more copies, waits
 * once more for the copies in flight and returns; later CTAs skip their tiles), the
 * tensor-core network after a fixed number of polls for its MMAs.  Every call that synchronises the
 * stream and reads results (lbm_step_diagnostics, lbm_reduce, lbm_reduce_blocks,
 * lbm_get_macroscopic, lbm_get_pdfs, lbm_get_pdfs_region, lbm_coarse_moments) then returns
 * LBM_ERR_TIMEOUT once and clears the flag; the context stays usable.
 * lbm_selfcheck_wait exercises that path: one device thread waits at most `polls` polls
 * (1 <= polls <= 2^20) on an mbarrier nothing arrives on, gives up and sets the flag; the
 * state is not touched.  Synchronises the stream.  Errors: LBM_ERR_ARG (polls out of range).
 * Paper: none (failure path of this library's bounded device waits). */
lbm_status lbm_selfcheck_wait(lbm_ctx *ctx, int32_t polls);

/* Work sizes of one step (builds the boundary lists if needed).
 * Paper: Sec. 4.4 (sizes of the boundary lists); the other sizes have no counterpart. */
lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *out);

/* Sweep tile shape (cells per CTA along x, y, z; threads = tx * ty).  tx must be a
 * multiple of 32, tx*ty <= 256.  A block narrower than tx gets tiles of its width rounded
 * up to 32 and proportionally more rows.  Takes effect at the next list build.
 * Default 256 x 1 x 4 (256 x 1 x 8 for the two-grid pattern with 16-bit storage).
 * Paper: none (execution shape of the Sec. 5.1.2 sweep on the GPU). */
lbm_status lbm_set_tile(lbm_ctx *ctx, int32_t tx, int32_t ty, int32_t tz);

/* Per-kernel device timing of lbm_step (tracing): when enabled, lbm_step records CUDA events
 * around its fill and sweep launches on the context's stream.  lbm_read_timing synchronises
 * the stream and returns, since the last reset, the summed device milliseconds and launch
 * counts of the two kernels: ms[0]/count[0] = boundary-and-ghost fill, ms[1]/count[1] =
 * stream-collide sweep.  enable = 0 stops recording; lbm_read_timing(ctx, ..., 1) resets.
 * Paper: none (tracing of the Sec. 5.1.2 sweep and the boundary/ghost kernel). */
lbm_status lbm_enable_timing(lbm_ctx *ctx, int32_t enable);
lbm_status lbm_read_timing(lbm_ctx *ctx, double ms[2], int64_t count[2], int32_t reset);

/* batched = 1 (default): one sweep launch per step covers the tiles of every block.
 * batched = 0: one sweep launch per block, as a per-block sweep would be issued; results are
 * bitwise the same (kept to measure what batching gains).
 * Paper: none (launch structure of the Sec. 5.1.2 sweep over all blocks). */
lbm_status lbm_set_batching(lbm_ctx *ctx, int32_t batched);

/* Graph mode: lbm_step replays pairs of steps as one captured CUDA graph (one graph per
 * starting parity, re-captured after the lists change); the last step of each call and the
 * diag_interval steps run as ordinary launches.  Needs a context created with a non-default
 * stream.  Per-kernel tracing (lbm_enable_timing) bypasses the graphs.  Errors:
 * LBM_ERR_UNSUPPORTED on the default stream.
 * Paper: none (launch structure of the Sec. 5.1.2 sweep). */
lbm_status lbm_set_graph(lbm_ctx *ctx, int32_t enable);

/* Index arithmetic of the neighbour addresses in the sweeps that spend their issue slots on
 * them (the AA neighbour sweep, the MRT and cumulant pull gathers, the closure's AA neighbour
 * sweep): bits = 32 (default) uses 32-bit element indices when every PDF array of the context
 * holds at most 2^32 elements and 64-bit ones otherwise; bits = 64 always uses 64-bit ones.
 * Both give the same results bit for bit.  Errors: LBM_ERR_ARG (bits not 32 or 64).
 * Paper: none (address arithmetic of the Sec. 5.1.2 sweep). */
lbm_status lbm_set_index_bits(lbm_ctx *ctx, int32_t bits);

/* Autotuner: times trial_steps steps for each candidate sweep tile shape (a fixed list from
 * 256x1x16 to 32x4x1, including shapes with few cells per CTA for small blocks) and each
 * neighbour mode (lbm_set_in_place; the other mode is tried only
 * where it may be switched: two-grid, or AA after an even number of steps), every trial from
 * the same state; keeps the fastest (best[3], *best_in_place and the time per step in
 * *best_ms, each pointer may be NULL but best) and restores the simulation state exactly (the
 * PDF arrays are snapshot to a temporary device buffer, which is cudaMalloc'd).  The step
 * count and parity are unchanged; diag_interval checks are off during the trials.
 * Paper: none (execution shape of the Sec. 5.1.2 sweep and the Sec. 3.3 neighbour mode). */
lbm_status lbm_autotune(lbm_ctx *ctx, int32_t trial_steps, int32_t best[3], int32_t *best_in_place,
                        double *best_ms);

/* Number of kernels lbm_step launched since the context was created.
 * Paper: none (launch count of the Sec. 5.1.2 step). */
int64_t lbm_kernel_launches(const lbm_ctx *ctx);

/* Canonical velocity set of a stencil (host only, no GPU needed): c[3*q] (cx, cy, cz per
 * direction), w[q], opp[q].  Returns LBM_ERR_ARG for an unknown q.
 * Paper: Sec. 5.1.1 (D3Q19 and D3Q27 stencils; order and weights as stated above). */
lbm_status lbm_stencil_table(int32_t q, int32_t *c, double *w, int32_t *opp);

/* Host-side view of the built lists, for inspection and tests (no GPU needed; builds the
 * lists if needed).  Links: uint64 words, bits 0-4 direction q (pointing from the fluid
 * cell into the boundary), 5-6 kind, 7-9 reserved, 10-17 wall-parameter index, 18-31 block,
 * 32-63 cell index in the block's padded layout.  Runs of `pattern` (LBM_TWO_GRID or LBM_AA): five
 * int64 per run (src, dst, len, src stride, dst stride), offsets in elements from the base
 * of a PDF array.  With out == NULL only the count is returned in *n.
 * Paper: Sec. 4.4 (per-kind boundary index lists). */
lbm_status lbm_plan_links(lbm_ctx *ctx, uint64_t *out, int64_t cap, int64_t *n);
lbm_status lbm_plan_runs(lbm_ctx *ctx, int32_t pattern, int64_t *out, int64_t cap, int64_t *n);
/* Padded layout of a block: out[0..7] = xo, pitch, plane, slab, offset (elements), and the
 * interior size nx, ny, nz.  Cell (x, y, z), each in [-1, n], has index
 * (z+1) plane + (y+1) pitch + xo + x; direction i of it lives at offset + i slab + index.
 * out[8] = arena size in elements; out[9] = 1 when the block reads and writes its neighbour
 * cells in place (every region of its ghost shell is covered by exactly one block with a
 * matching face, or lies outside the domain), 0 when it keeps ghost copies.
 * Paper: Sec. 4.2 (field layout with ghost layers and padded rows). */
lbm_status lbm_plan_layout(lbm_ctx *ctx, int32_t block, int64_t out[10]);
/* Neighbour table of a block: out[r], r = (rx+1) + 3 (ry+1) + 9 (rz+1) for the ghost-shell
 * region on side r_a in {-1, 0, 1} of each axis, is the block covering that region exactly
 * (the block itself across a periodic axis it spans alone), or -1 (outside the domain,
 * uncovered, or no exact match).  The cell of a neighbour read in place is the first (+) or
 * last (-) layer of that block along the crossed axes, the same coordinate along the others.
 * Paper: Sec. 3.3 (blocks of one process exchanging ghost layers directly). */
lbm_status lbm_plan_neighbors(lbm_ctx *ctx, int32_t block, int32_t out[27]);
/* Cell masks of a block in its padded layout (uint32 per cell; *n = 0 when the block needs
 * none): bit 31 = the cell is not fluid; bit i = the pull source x - c_i of direction i is a
 * no-slip cell, so the sweep applies halfway bounce-back for it (Sec. 4.4 boundary handling;
 * no-slip needs no link list). */
lbm_status lbm_plan_mask(lbm_ctx *ctx, int32_t block, uint32_t *out, int64_t cap, int64_t *n);

/* Wall-parameter table of the built lists: (ux, uy, uz, rho) per index.
 * Paper: Sec. 5.1.1 (boundary parameters of the velocity and pressure kinds). */
lbm_status lbm_plan_params(lbm_ctx *ctx, double *out, int64_t cap, int64_t *n);

/* Host-only inspection of a partitioned context's halo lists with `peer`: list 0 send (pull
 * selection), 1 receive (pull), 2 send (AA), 3 receive (AA).  Each run is 4 int64: arena
 * element offset, buffer element offset, length, arena stride; element k of a run moves
 * between arena[offset + k * stride] (in this rank's PDF array) and buffer[buffer offset + k].
 * Send runs read owned interior slots, receive runs address own ghost slots; the peer's
 * matching list covers the same buffer elements in the same order.  out = NULL: *n only.
 * Paper: Sec. 3.3 (ghost-layer exchange lists). */
lbm_status lbm_plan_halo(lbm_ctx *ctx, int32_t peer, int32_t list, int64_t *out, int64_t cap, int64_t *n);

/* Allocation-free diagnostics of a caller-owned PDF field.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code that takes all
 * device memory from its own pool or fixed arena, or that runs where an allocation is not
 * allowed because cudaMalloc/cudaFree can synchronise the device or fail mid-run.
 *   f_dev   : device pointer to a dense canonical field f[i*ncells + n] (i in canonical
 *             direction order, n any cell order), LBM_FP64 (double) or LBM_FP32 (float);
 *             every cell counts as fluid.  Owned by the caller, only read.
 *   force   : body force used for the half-force momentum shift (NULL = zero).
 *   out_dev : device pointer to 8 doubles, written asynchronously on cuda_stream: mass,
 *             momentum x, y, z, kinetic energy, max speed, non-finite cells, cells (the
 *             fields of lbm_diagnostics as lbm_reduce computes them).
 * No memory is allocated: the per-CTA partial sums use a fixed device array of
 * LBM_REDUCE_NOALLOC_MAX_CELLS / 4096 records (2 MiB), which every GPU that loads the
 * library holds until the process exits.  Fields with more than LBM_REDUCE_NOALLOC_MAX_CELLS
 * cells are rejected with LBM_ERR_UNSUPPORTED; BF16/FP16 storages too.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys and re-creates the device's
 * primary context) it is stale, so do not call this function again in such a process.  All
 * calls share the array: each call
 * writes every record it reads, so nothing needs clearing, but calls whose kernels overlap
 * on the GPU (different streams, no ordering between them) race on it.
 * Errors: LBM_ERR_ARG (null pointer, bad stencil, ncells <= 0), LBM_ERR_UNSUPPORTED (storage
 * or size), LBM_ERR_CUDA (launch or address lookup failed). */
#define LBM_REDUCE_NOALLOC_MAX_CELLS 134217728LL
lbm_status lbm_reduce_noalloc(const void *f_dev, int32_t stencil, int32_t storage, int64_t ncells,
                              const double force[3], double *out_dev, void *cuda_stream);

/* ---- Locally varying relaxation --------------------------------------------------------
 * Sec. 5.1.1: the relaxation rate may vary per cell from a local fluid property (turbulence
 * models, cited there after Yu et al. 2005).  With a closure set, every sweep computes omega+
 * of each cell from its pre-collision populations; omega- follows from the context's Lambda
 * (TRT) or equals omega+ (SRT).  tau0 = 1/params.omega.  Non-equilibrium stress:
 *   Pi_ab = sum_i c_ia c_ib f_i - rho (delta_ab / 3 + u_a u_b)
 *   LBM_CLOSURE_SMAGORINSKY: tau = (tau0 + sqrt(tau0^2 + 18 cs^2 sqrt(2 Pi:Pi) / rho)) / 2
 *   LBM_CLOSURE_MLP: tau = tau0 + s_tau softplus(y), y the output of a 7-32-32-1 network
 *     with SiLU hidden units on the features ((rho - 1) s_rho, s_pi Pi_xx, Pi_yy, Pi_zz, Pi_xy,
 *     Pi_xz, Pi_yz), evaluated on the tensor cores: features, weights and hidden activations
 *     rounded to BF16 (nearest even), sums in FP32.
 * Packed network parameters (LBM_MLP_NPARAM floats, row-major): W1[32][7], b1[32],
 * W2[32][32], b2[32], w3[32], b3, s_rho, s_pi, s_tau. */
enum { LBM_CLOSURE_NONE = 0, LBM_CLOSURE_SMAGORINSKY = 1, LBM_CLOSURE_MLP = 2 };
#define LBM_MLP_NPARAM 1348

/* Set the closure of a context.  cs: Smagorinsky constant (kind 1); mlp_params: host array of
 * LBM_MLP_NPARAM floats (kind 2), copied.  Supported for D3Q19, LBM_FP32 storage and zero
 * body force (any block set and boundary kinds); other contexts get LBM_ERR_UNSUPPORTED.
 * kind LBM_CLOSURE_NONE restores the constant rate.  Errors: LBM_ERR_ARG (unknown kind, null
 * params, cs < 0), LBM_ERR_UNSUPPORTED.
 * Paper: Sec. 5.1.1 (per-cell relaxation rates for turbulence models). */
lbm_status lbm_set_closure(lbm_ctx *ctx, int32_t kind, double cs, const float *mlp_params);

/* The network alone: inference on the tensor cores and training in FP32 (loss
 * mean_s (softplus(y_s) - t_s)^2 over a batch, its gradient, Adam steps).  Device arrays:
 * features X[n][7] (FP32, already scaled), targets T[n], outputs y[n]. */
typedef struct lbm_mlp lbm_mlp; /* opaque; owned by the library */

/* Create a network from LBM_MLP_NPARAM packed parameters (host, copied) for batches of up
 * to max_batch samples, issuing work on cuda_stream.  Errors: LBM_ERR_ARG, LBM_ERR_OOM.
 * Paper: Sec. 5.1.1 (per-cell relaxation rates for turbulence models); the network itself is not
 * in the paper. */
lbm_status lbm_mlp_create(const float *params, int64_t max_batch, void *cuda_stream, lbm_mlp **out);
/* Replace / read the parameters (host arrays of LBM_MLP_NPARAM floats); set resets Adam; get
 * synchronises the stream and returns LBM_ERR_TIMEOUT once if an earlier inference gave up.
 * Paper: Sec. 5.1.1 (per-cell relaxation rates for turbulence models); the network itself is not
 * in the paper. */
lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *params);
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *params);
/* y[s] for n samples (asynchronous on the stream), with the BF16 rounding points of the sweep,
 * on the fifth-generation tensor cores (tcgen05, 128-sample tiles, accumulators in tensor
 * memory).  A bounded wait inside that gives up is reported by the next lbm_mlp_get_params as
 * LBM_ERR_TIMEOUT.
 * Paper: Sec. 5.1.1 (per-cell relaxation rates for turbulence models); the network itself is not
 * in the paper. */
lbm_status lbm_mlp_infer(lbm_mlp *m, const float *X_dev, int64_t n, float *y_dev);
/* Loss and gradient (FP32 arithmetic, deterministic summation order) of n <= max_batch
 * samples; loss_host (1 double) and grad_host (LBM_MLP_NPARAM floats, zero for the three
 * scales) may each be NULL.  Synchronises the stream when either is given.
 * Paper: none (training of the closure network). */
lbm_status lbm_mlp_loss_grad(lbm_mlp *m, const float *X_dev, const float *T_dev, int64_t n, double *loss_host,
                             float *grad_host);
/* `iters` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr; scales held fixed) on
 * consecutive batches of `batch` samples cycling through the n samples; loss_history
 * (iters doubles, host, may be NULL) receives each step's batch loss.  Synchronises.
 * Paper: none (training of the closure network). */
lbm_status lbm_mlp_train(lbm_mlp *m, const float *X_dev, const float *T_dev, int64_t n, int64_t batch,
                         int64_t iters, float lr, double *loss_history);
void lbm_mlp_destroy(lbm_mlp *m);

/* Neighbour access across block faces (Sec. 3.3: blocks on one process exchange ghost layers
 * by direct copies): enable != 0 (default) lets a block whose every ghost-shell region is
 * covered exactly by one block read and write those cells in place during the sweep (no
 * ghost copy; a block spanning a periodic axis alone wraps onto itself); enable = 0 gives
 * every block ghost layers filled by the copy runs of the fill kernel before each sweep.  The
 * lists are rebuilt before the next step; the stored state is kept.  Results are identical.
 * Errors: LBM_ERR_STATE when an AA context is after an odd number of steps (its two forms of
 * the odd layout differ: switch after an even number). */
lbm_status lbm_set_in_place(lbm_ctx *ctx, int32_t enable);

/* Fluid-cell list layout of the two-grid sweep (enable != 0) or the dense block layout (0,
 * default).  The list layout keeps only fluid cells -- numbered block by block in (z, y, x)
 * order, one array per direction plus one slot per velocity/pressure link -- and a table with
 * the pull source of each direction of each cell (a fluid cell of the same or a neighbour
 * block, a link slot, or halfway bounce-back): on porous geometries a dense block spends DRAM
 * sectors and warp lanes on solid cells, the list does not (4 (Q - 1) bytes of table per cell
 * and step instead).  Every cell does the dense sweep's arithmetic: results are the same bit
 * for bit.  The dense arrays stay allocated: the state moves to the list before the next
 * step and back when a call reads or writes PDFs (get/set/init/macroscopic/reduce).  Graph
 * replay works; lbm_autotune is refused.
 * Errors: LBM_ERR_UNSUPPORTED for the AA pattern, a partitioned context, MRT or a closure.
 * Paper: Sec. 4.4 (boundary handling by index lists), Sec. 5.1.3 (porous beds of randomly
 * arranged spheres); the list layout itself has no counterpart there. */
lbm_status lbm_set_sparse(lbm_ctx *ctx, int32_t enable);

/* Host-only inspection of the fluid-cell list layout: what = 0 the pull table ((Q - 1) x
 * fluid cells, direction-major: entry index, or INT32_MIN for halfway bounce-back), 1 the
 * block of each fluid cell, 2 its padded-layout cell index in that block, 3 the link words
 * (bits 0-4 direction q, 5-6 kind, 10-17 wall parameter, 32-63 fluid cell; link k fills entry
 * fluid cells + k of direction opp(q)), each as int64.  out = NULL: *n only.
 * Errors: LBM_ERR_STATE unless lbm_set_sparse is on.
 * Paper: Sec. 4.4 (index lists); the list layout itself has no counterpart there. */
lbm_status lbm_plan_sparse(lbm_ctx *ctx, int32_t what, int64_t *out, int64_t cap, int64_t *n);

/* Per-block diagnostics of the stored state (the per-block reductions of the paper's
 * per-block data layout, Sec. 4.1-4.2): out[8 b + k] for block b, k = mass, momentum x, y, z,
 * kinetic energy, max speed, non-finite cells, fluid cells (the lbm_diagnostics fields, as
 * doubles), FP64 sums in a fixed order over the block's tiles.  out: host array of
 * 8 * nblocks doubles.  Synchronises the stream.  Summing the blocks' records gives
 * lbm_reduce up to the order of the sums. */
lbm_status lbm_reduce_blocks(lbm_ctx *ctx, double *out);

/* Box sums of a block for coarse-graining (the filtered fine-grid fields that train and score
 * the learned closure): for each coarse cell of ratio^3 interior cells (every block edge
 * divisible by ratio), the sums over its fluid cells of rho, rho u_x, rho u_y, rho u_z and
 * rho u_a u_b (xx, yy, zz, xy, xz, yz), with rho and u as lbm_get_macroscopic gives them.
 * out: host array of 10 * Nc doubles, out[m * Nc + c], c = X + NX (Y + NY Z), NX = nx / ratio.
 * Synchronises the stream.  Errors: LBM_ERR_ARG (bad block, null out, ratio not dividing).
 * Paper: none (box filter of the learned-closure study). */
lbm_status lbm_coarse_moments(lbm_ctx *ctx, int32_t block, int32_t ratio, double *out);

/* Last error message of the context (never NULL).
 * Paper: none. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Free the context and all device memory it owns (not memory bound by the caller).
 * Paper: Sec. 4.2 (the block fields are released with the context). */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
