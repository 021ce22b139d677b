// plan.hpp -- host-side block layout and the per-step work lists of the LBM sweep.
//
// Everything here is plain C++ on the host (no CUDA calls): it turns the block layout and the
// flag fields into
//   * the padded SoA layout of each block's PDF array (one ghost layer, aligned rows;
//     Sec. 4.2: SoA layout, each line padded so the next one starts aligned),
//   * the boundary link lists, one entry per (fluid cell, direction) whose neighbour is a
//     boundary cell, tagged with the boundary kind (Sec. 4.4: one index list per boundary
//     condition, each treated by its own kernel),
//   * the ghost-copy run lists between blocks on the same GPU and across periodic faces
//     (Sec. 3.3 PackInfo local transfer; only the PDFs that cross into the block are copied),
//   * the sweep tile list (which CTA sweeps which cells of which block),
//   * for a context that owns only some of the blocks (one rank of a partitioned run, blocks
//     given to ranks along a space-filling curve, Sec. 3.1), the halo lists: per peer rank the
//     PDFs this rank sends to the peer's ghost layers and the ones it receives into its own
//     (Sec. 3.3: ghost-layer exchange of the crossing directions only, packed into buffers).
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace lbm {

enum CellKind : uint8_t {
    K_FLUID = 0, K_NOSLIP = 1, K_VELOCITY = 2, K_PRESSURE = 3, K_PERIODIC = 4, K_MIRROR = 5,
    K_ZOUHE = 6  // beyond a wet-node (Zou-He) face: its slots are written before each sweep
};
// face kinds of PlanInput.face_kind beyond the cell kinds (the C ABI's values)
constexpr int kFaceZouHeVelocity = 5, kFaceZouHePressure = 6;

// Wet-node entry: bits 0-2 face (2 axis + side), 3-16 block, 32-63 cell index of the node (a
// fluid cell of the first layer at the face) in its block's padded layout.
inline uint64_t pack_zouhe(int face, int block, int64_t cell)
{
    return (uint64_t)face | ((uint64_t)block << 3) | ((uint64_t)cell << 32);
}

struct WallParam {
    double u[3];
    double rho;
};

struct BlockLayout {
    int64_t origin[3];
    int32_t n[3];    // interior cells
    int32_t xo;      // row index of interior x = 0 (ghost x = -1 sits at xo - 1)
    int32_t pitch;   // elements per row
    int64_t plane;   // pitch * (n[1] + 2)
    int64_t slab;    // plane * (n[2] + 2): elements of one direction
    int64_t offset;  // element offset of this block's array in the PDF arena
    // cell index of interior/ghost coordinate (x, y, z), each in [-1, n]
    int64_t cell(int x, int y, int z) const { return (int64_t)(z + 1) * plane + (int64_t)(y + 1) * pitch + xo + x; }
};

// One ghost-copy run: len elements, element k copied from arena[src + k*sstride] to
// arena[dst + k*dstride] (offsets are relative to the base of the current PDF array).
struct GhostRun {
    int64_t src;
    int64_t dst;
    int32_t len;
    int32_t sstride;
    int32_t dstride;
    int32_t pad;
};

// One halo run of a partitioned context: len elements, element k between the arena slot
// arena + k*astride and buffer element buf + k (the peer's matching run has the same buffer
// range).  Send runs read owned interior slots; receive runs address own ghost slots.
struct HaloRun {
    int64_t arena;
    int64_t buf;
    int32_t len;
    int32_t astride;
};

// The halo lists exchanged with one peer rank, for the two-grid (pull) and the AA selection of
// ghost slots, and their lengths in elements.
struct PeerHalo {
    std::vector<HaloRun> send_pull, recv_pull, send_aa, recv_aa;
    int64_t n_send_pull = 0, n_recv_pull = 0, n_send_aa = 0, n_recv_aa = 0;
};

// Sweep tile: x0, y0, z0 of a box of one block, `width` cells wide, (threads / width) rows
// high and TZ planes deep; flags bit 0: some cell of the tile has a non-zero mask (the kernel
// reads the mask).  The width adapts to the block: a block narrower than the CTA gets tiles
// exactly as wide as the block, whose rows follow each other inside a warp, so narrow blocks
// keep almost every lane busy; wider blocks get tiles TX wide.
struct Tile {
    int32_t block;
    int16_t x0, y0, z0;
    uint8_t flags;
    uint8_t width_m1;  // width - 1 (1..256)
};

// Link word: bits 0-4 direction q (the link points from fluid cell x along c_q into a
// boundary cell), 5-6 kind, 7-9 reserved (0), 10-17 wall-parameter index, 18-31 block,
// 32-63 cell index of x in the block's padded layout.  The boundary cell's slot is found at
// run time like the sweep finds it (own ghost layer, or a neighbour block's cell).
inline uint64_t pack_link(int q, int kind, int param, int block, int64_t cell)
{
    return (uint64_t)q | ((uint64_t)kind << 5) | ((uint64_t)param << 10) | ((uint64_t)block << 18) |
           ((uint64_t)cell << 32);
}
constexpr uint32_t kCellNotFluid = 1u << 31;  // mask bit 31 (the device side calls it kMaskSolid)
constexpr int kMaxParams = 256;
constexpr int kMaxBlocks = 16384;

struct PlanInput {
    int q;
    int bytes_per_pdf;
    int periodic[3];
    int face_kind[6];
    WallParam face_param[6];
    int tile[3];
    int in_place = 1;  // 1: blocks whose faces match their neighbours read them in place; 0: ghost copies only
    std::vector<BlockLayout> const *blocks;
    std::vector<std::vector<uint8_t>> const *flags;  // per block, interior, may be empty (all fluid)
    std::vector<WallParam> const *block_param;       // per block
    // partitioned context: owner rank of every block (nullptr: this context owns all blocks);
    // only blocks with owner == rank get tiles, links, masks and device storage, and the flags
    // of every block must be known (the ghost shells of owned blocks take kinds from them)
    std::vector<int32_t> const *owner = nullptr;
    int rank = 0;
    int sparse = 0;  // also build the fluid-cell list layout (SparsePlan)
};

// Fluid-cell list layout of the two-grid sweep (for porous geometries, where a dense block
// spends sectors and lanes on solid cells): the fluid cells of all blocks numbered block by
// block in (z, y, x) order, n = 0 .. nfluid - 1; each direction's array holds nfluid entries
// plus one slot per velocity/pressure boundary link (filled before each sweep, like the ghost
// slot a dense block's link writes).  nbr[(i - 1) * nfluid + n] is the pull source of
// direction i of cell n: the entry index (a fluid cell, here or in a neighbour block across a
// face or a periodic image, or a link slot), or kSparseBounce: halfway bounce-back, read slot
// opp(i) of n itself.
constexpr int32_t kSparseBounce = (int32_t)0x80000000u;
struct SparsePlan {
    int64_t nfluid = 0, nslots = 0;
    std::vector<int32_t> nbr;             // (Q - 1) x nfluid
    std::vector<uint64_t> links;          // link k: pack_link(q, kind, param, 0, n); writes slot nfluid + k of opp(q)
    std::vector<int32_t> block_of;        // block of each fluid cell
    std::vector<int64_t> cell_of;         // its padded-layout cell index in that block
    std::vector<int64_t> block_start;     // first fluid index of each block (+ nfluid at the end)
};

struct Plan {
    std::vector<uint64_t> links;           // velocity and pressure links, sorted by (kind, block, q, cell)
    std::vector<uint64_t> zouhe;           // wet-node boundary nodes (pack_zouhe), by block
    int64_t link_count[4] = {0, 0, 0, 0};  // by kind; no-slip ones are the mask bits the sweep applies
    std::vector<WallParam> params;         // wall parameter table (faces first)
    std::vector<GhostRun> runs_pull;       // two-grid: slots j of ghost g with g + c_j fluid interior
    std::vector<GhostRun> runs_aa;         // AA: slots j of ghost g with g - c_j fluid interior
    int64_t ghost_slots_pull = 0, ghost_slots_aa = 0;
    std::vector<Tile> tiles;
    // per block: padded-layout cell masks or empty (block with no solid cell and no no-slip
    // neighbour).  Bit 31: the cell is not fluid.  Bit i (1 <= i < Q): the pull source of
    // direction i, x - c_i, is a no-slip cell, so the sweep applies halfway bounce-back
    // itself (f_i(x, t+1) = f*_opp(i)(x, t)) instead of going through a link list.
    std::vector<std::vector<uint32_t>> masks;
    // Per block: the block that exactly covers each of the 26 neighbour regions of its
    // ghost shell (region index (rx+1) + 3 (ry+1) + 9 (rz+1), r = -1/0/+1 per axis; itself
    // across a periodic axis it spans alone), -1 where the region is outside the domain or
    // uncovered.  through[b] = 1 when every region is of one of those two kinds: the kernels
    // then read and write neighbour cells in place (no ghost copies for that block).
    // Otherwise (faces that do not match one block exactly) the block keeps ghost copies.
    std::vector<std::array<int32_t, 27>> nbr;
    std::vector<uint8_t> through;
    int64_t cells = 0, fluid_cells = 0;
    // partitioned context: halo lists per peer rank (index = rank; empty for this rank).  A block
    // with a neighbour on another rank keeps ghost copies (through = 0).
    std::vector<PeerHalo> halo;
    SparsePlan sparse;  // built when PlanInput.sparse is set
};

// Compute the padded layout of each block (alignment in bytes for rows).  With owner (one rank
// of a partitioned run) only the blocks of `rank` are placed in the arena; the others get
// offset -1.
void layout_blocks(std::vector<BlockLayout> &blocks, int bytes_per_pdf, int q, int align_bytes, int64_t *total_elems,
                   const std::vector<int32_t> *owner = nullptr, int rank = 0);

// Partition blocks over nranks along the Morton (Z-order) curve of their centres: blocks in
// curve order are cut into nranks contiguous pieces of nearly equal cell counts (weights, when
// given, replace the cell counts).  owner[b] receives the rank of block b.
void partition_morton(const std::vector<BlockLayout> &blocks, int nranks, const std::vector<double> *weights,
                      std::vector<int32_t> &owner);

// Validate the layout (non-overlapping blocks); returns an empty string or an error.
std::string check_blocks(const std::vector<BlockLayout> &blocks);

// Build all lists.  Returns an empty string or an error.
std::string build_plan(const PlanInput &in, Plan &out);

}  // namespace lbm
