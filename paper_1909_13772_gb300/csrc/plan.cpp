// plan.cpp -- host-side list builder (see plan.hpp).
#include "plan.hpp"

#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>

#include "lattice.cuh"

namespace lbm {

void layout_blocks(std::vector<BlockLayout> &blocks, int bytes_per_pdf, int q, int align_bytes, int64_t *total_elems,
                   const std::vector<int32_t> *owner, int rank)
{
    int a = std::max(1, align_bytes / bytes_per_pdf);
    int64_t off = 0;
    for (size_t i = 0; i < blocks.size(); ++i) {
        auto &b = blocks[i];
        b.xo = a;
        int need = a + b.n[0] + 1;
        b.pitch = (need + a - 1) / a * a;
        b.plane = (int64_t)b.pitch * (b.n[1] + 2);
        b.slab = b.plane * (b.n[2] + 2);
        if (owner && (*owner)[i] != rank) {
            b.offset = -1;
            continue;
        }
        b.offset = off;
        off += (int64_t)q * b.slab;
    }
    *total_elems = off;
}

namespace {
// interleave the low 21 bits of v with two zero bits between them
uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffULL;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}
}  // namespace

void partition_morton(const std::vector<BlockLayout> &blocks, int nranks, const std::vector<double> *weights,
                      std::vector<int32_t> &owner)
{
    const int nb = (int)blocks.size();
    owner.assign(nb, 0);
    if (nb == 0 || nranks <= 1) return;
    int64_t lo[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = blocks[0].origin[a];
        for (const auto &b : blocks) lo[a] = std::min(lo[a], b.origin[a]);
    }
    // key of a block: Morton code of its centre (twice the centre, to stay in integers)
    std::vector<std::pair<uint64_t, int>> key(nb);
    for (int b = 0; b < nb; ++b) {
        uint64_t k = 0;
        for (int a = 0; a < 3; ++a) {
            const uint64_t c = (uint64_t)(2 * (blocks[b].origin[a] - lo[a]) + blocks[b].n[a]);
            k |= spread3(c) << a;
        }
        key[b] = {k, b};
    }
    std::sort(key.begin(), key.end());
    double total = 0.0;
    std::vector<double> w(nb);
    for (int b = 0; b < nb; ++b) {
        w[b] = weights ? (*weights)[b] : (double)blocks[b].n[0] * blocks[b].n[1] * blocks[b].n[2];
        total += w[b];
    }
    // block k of the curve goes to the rank whose share [r, r + 1) total / nranks holds the
    // middle of its weight interval
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) {
        const int b = key[k].second;
        const double mid = acc + 0.5 * w[b];
        int r = (int)(mid / total * nranks);
        owner[b] = std::min(std::max(r, 0), nranks - 1);
        acc += w[b];
    }
}

std::string check_blocks(const std::vector<BlockLayout> &blocks)
{
    if (blocks.empty()) return "no blocks";
    if ((int64_t)blocks.size() > kMaxBlocks) return "too many blocks (max 16384)";
    for (size_t i = 0; i < blocks.size(); ++i) {
        const auto &b = blocks[i];
        for (int a = 0; a < 3; ++a)
            if (b.n[a] < 1 || b.n[a] > 32000) return "block size out of range [1, 32000]";
        if (b.slab >= ((int64_t)1 << 32)) return "block too large (padded cells >= 2^32)";
    }
    // pairwise overlap test, sorted by x origin so the inner loop stops early
    std::vector<int> order(blocks.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int p, int r) { return blocks[p].origin[0] < blocks[r].origin[0]; });
    for (size_t ii = 0; ii < order.size(); ++ii) {
        const auto &A = blocks[order[ii]];
        for (size_t jj = ii + 1; jj < order.size(); ++jj) {
            const auto &B = blocks[order[jj]];
            if (B.origin[0] >= A.origin[0] + A.n[0]) break;
            bool ov = true;
            for (int a = 0; a < 3; ++a)
                ov = ov && A.origin[a] < B.origin[a] + B.n[a] && B.origin[a] < A.origin[a] + A.n[a];
            if (ov) return "blocks overlap";
        }
    }
    return "";
}

namespace {

struct Candidate {
    int block;
    int64_t shift[3];  // global offset added to the candidate's coordinates
};

struct Elem {
    int64_t src, dst;
};

// Append one element copy to a run list, extending the last run when the element continues
// it: along x (strides 1, 1) or along y (strides = the two blocks' row pitches).
// Append one halo element (arena slot, next buffer element) to a halo run list, extending the
// last run along a constant arena stride.
void append_halo(std::vector<HaloRun> &runs, int64_t arena, int64_t buf)
{
    if (!runs.empty()) {
        HaloRun &r = runs.back();
        if (buf == r.buf + r.len && r.len < (1 << 30)) {
            if (r.len == 1 && arena - r.arena != 0 && std::llabs(arena - r.arena) < ((int64_t)1 << 31)) {
                r.astride = (int32_t)(arena - r.arena);
                r.len = 2;
                return;
            }
            if (r.len > 1 && arena == r.arena + (int64_t)r.len * r.astride) {
                r.len += 1;
                return;
            }
        }
    }
    runs.push_back(HaloRun{arena, buf, 1, 1});
}

// One halo element of a block's ghost shell: peer rank, arena slot on this rank, selection
// (bit 0: two-grid pull, bit 1: AA).
struct HaloElem {
    int32_t peer;
    int32_t sel;
    int64_t arena;
};

void append_run(std::vector<GhostRun> &runs, int64_t src, int64_t dst, int32_t spitch, int32_t dpitch)
{
    if (!runs.empty()) {
        GhostRun &r = runs.back();
        if (r.len == 1) {
            int64_t ds = src - r.src, dd = dst - r.dst;
            if ((ds == 1 && dd == 1) || (ds == spitch && dd == dpitch)) {
                r.sstride = (int32_t)ds;
                r.dstride = (int32_t)dd;
                r.len = 2;
                return;
            }
        } else if (src == r.src + (int64_t)r.len * r.sstride && dst == r.dst + (int64_t)r.len * r.dstride &&
                   r.len < (1 << 30)) {
            r.len += 1;
            return;
        }
    }
    runs.push_back(GhostRun{src, dst, 1, 1, 1, 0});
}

struct BlockOut {
    std::vector<uint64_t> zouhe;      // wet-node entries of this block
    std::vector<int32_t> snbr;        // sparse layout: (Q - 1) x (fluid cells of the block), local link marks
    std::vector<uint64_t> slinks;     // sparse layout: the block's link slots, local order
    std::vector<HaloElem> send, recv;  // partitioned context: halo elements of this block's shell
    std::vector<uint64_t> links[4];
    std::vector<GhostRun> runs_pull, runs_aa;
    int64_t slots_pull = 0, slots_aa = 0;
    std::vector<Tile> tiles;
    std::vector<uint32_t> mask;
    int64_t cells = 0, fluid = 0, bounce = 0;
};

}  // namespace

std::string build_plan(const PlanInput &in, Plan &out)
{
    const auto &blocks = *in.blocks;
    const auto &flags = *in.flags;
    const int nb = (int)blocks.size();
    const LatticeView L = lattice_view(in.q);
    // wet-node faces: D3Q19, and the face's tangential axes periodic (no edges between two
    // non-periodic faces, which the reconstruction does not treat)
    for (int f = 0; f < 6; ++f) {
        const int fk = in.face_kind[f], a = f / 2;
        if (in.periodic[a] || (fk != kFaceZouHeVelocity && fk != kFaceZouHePressure)) continue;
        if (in.q != 19) return "wet-node (Zou-He) faces are built for D3Q19";
        if (!in.periodic[(a + 1) % 3] || !in.periodic[(a + 2) % 3])
            return "a wet-node (Zou-He) face needs its two tangential axes periodic";
        if (in.sparse || in.owner) return "wet-node (Zou-He) faces need the dense layout of one context";
    }

    // domain bounding box
    int64_t lo[3], hi[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = blocks[0].origin[a];
        hi[a] = blocks[0].origin[a] + blocks[0].n[a];
        for (const auto &b : blocks) {
            lo[a] = std::min(lo[a], b.origin[a]);
            hi[a] = std::max(hi[a], b.origin[a] + (int64_t)b.n[a]);
        }
        ext[a] = hi[a] - lo[a];
    }

    // wall parameter table: faces first, then the distinct block parameter sets
    out.params.assign(in.face_param, in.face_param + 6);
    std::vector<int> bparam(nb, 0);
    {
        std::map<std::tuple<double, double, double, double>, int> seen;
        for (int b = 0; b < nb; ++b) {
            const WallParam &p = (*in.block_param)[b];
            auto key = std::make_tuple(p.u[0], p.u[1], p.u[2], p.rho);
            auto it = seen.find(key);
            if (it == seen.end()) {
                if ((int)out.params.size() >= kMaxParams) return "too many distinct wall parameter sets (max 250)";
                it = seen.emplace(key, (int)out.params.size()).first;
                out.params.push_back(p);
            }
            bparam[b] = it->second;
        }
    }

    // neighbour candidates: blocks (possibly periodic images) overlapping the dilated box
    std::vector<std::vector<Candidate>> cand(nb);
    std::vector<int> order(nb);
    for (int i = 0; i < nb; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int p, int r) { return blocks[p].origin[0] < blocks[r].origin[0]; });
    std::vector<int64_t> ox(nb);
    for (int i = 0; i < nb; ++i) ox[i] = blocks[order[i]].origin[0];
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; ++b) {
        const auto &B = blocks[b];
        int64_t dlo[3], dhi[3];
        for (int a = 0; a < 3; ++a) {
            dlo[a] = B.origin[a] - 1;
            dhi[a] = B.origin[a] + B.n[a] + 1;
        }
        int srange[3][2];
        for (int a = 0; a < 3; ++a) {
            srange[a][0] = (in.periodic[a] && dlo[a] < lo[a]) ? -1 : 0;
            srange[a][1] = (in.periodic[a] && dhi[a] > hi[a]) ? 1 : 0;
        }
        for (int sz = srange[2][0]; sz <= srange[2][1]; ++sz)
            for (int sy = srange[1][0]; sy <= srange[1][1]; ++sy)
                for (int sx = srange[0][0]; sx <= srange[0][1]; ++sx) {
                    int64_t sh[3] = {sx * ext[0], sy * ext[1], sz * ext[2]};
                    // candidates need origin_x + sh_x < dhi_x and origin_x + n_x + sh_x > dlo_x
                    for (int k = 0; k < nb; ++k) {
                        if (ox[k] + sh[0] >= dhi[0]) break;
                        int c = order[k];
                        const auto &C = blocks[c];
                        if (c == b && sx == 0 && sy == 0 && sz == 0) continue;
                        bool ov = true;
                        for (int a = 0; a < 3; ++a)
                            ov = ov && C.origin[a] + sh[a] < dhi[a] && C.origin[a] + C.n[a] + sh[a] > dlo[a];
                        if (ov) cand[b].push_back(Candidate{c, {sh[0], sh[1], sh[2]}});
                    }
                }
    }

    // neighbour tables: for each region of the ghost shell, the candidate that covers it
    // exactly (same extent along the axes the region does not cross, adjacent along the
    // crossed ones), or -1 when no block covers any of it
    std::vector<std::array<int32_t, 27>> nbrt(nb);
    std::vector<uint8_t> through(nb, 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; ++b) {
        const auto &B = blocks[b];
        for (int r = 0; r < 27; ++r) {
            nbrt[b][r] = -1;
            const int rr[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
            if (r == 13) continue;
            int64_t glo[3], ghi[3];  // region box
            for (int a = 0; a < 3; ++a) {
                glo[a] = rr[a] < 0 ? B.origin[a] - 1 : (rr[a] > 0 ? B.origin[a] + B.n[a] : B.origin[a]);
                ghi[a] = rr[a] < 0 ? B.origin[a] : (rr[a] > 0 ? B.origin[a] + B.n[a] + 1 : B.origin[a] + B.n[a]);
            }
            bool exact = false, touched = false;
            for (const Candidate &cd : cand[b]) {
                const auto &C = blocks[cd.block];
                bool ov = true, ex = true;
                for (int a = 0; a < 3; ++a) {
                    const int64_t clo = C.origin[a] + cd.shift[a], chi = clo + C.n[a];
                    ov = ov && clo < ghi[a] && chi > glo[a];
                    if (rr[a] == 0) ex = ex && clo == B.origin[a] && C.n[a] == B.n[a];
                    if (rr[a] > 0) ex = ex && clo == B.origin[a] + B.n[a];
                    if (rr[a] < 0) ex = ex && chi == B.origin[a];
                }
                if (!ov) continue;
                touched = true;
                if (ex) {
                    nbrt[b][r] = cd.block;
                    exact = true;
                    break;
                }
            }
            if (touched && !exact) through[b] = 0;
        }
    }
    if (!in.in_place) std::fill(through.begin(), through.end(), uint8_t(0));
    // partitioned context: blocks of other ranks are not swept here, and a block with a
    // neighbour on another rank receives that neighbour's PDFs into its ghost layer
    const auto owned = [&](int b) { return !in.owner || (*in.owner)[b] == in.rank; };
    if (in.owner) {
        for (int b = 0; b < nb; ++b) {
            if (!owned(b)) {
                through[b] = 0;
                continue;
            }
            for (const Candidate &cd : cand[b])
                if (!owned(cd.block)) through[b] = 0;
        }
    }

    std::vector<BlockOut> bo(nb);
    std::string err;
    // sparse layout, first pass: number the fluid cells of every block (z, y, x order)
    std::vector<std::vector<int32_t>> fidx(in.sparse ? nb : 0);
    std::vector<int64_t> fstart(nb + 1, 0);
    if (in.sparse) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int b = 0; b < nb; ++b) {
            const auto &B = blocks[b];
            const size_t N = (size_t)B.n[0] * B.n[1] * B.n[2];
            fidx[b].assign(N, -1);
            int32_t k = 0;
            for (size_t c = 0; c < N; ++c)
                if (flags[b].empty() || flags[b][c] == K_FLUID) fidx[b][c] = k++;
            fstart[b + 1] = k;
        }
        for (int b = 0; b < nb; ++b) fstart[b + 1] += fstart[b];
        if (fstart[nb] >= ((int64_t)1 << 30)) return "sparse layout: too many fluid cells (max 2^30)";
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nb; ++b) {
        const auto &B = blocks[b];
        const bool own = owned(b);
        if (!own) {
            // a block of another rank matters here only when it mirrors cells of this rank's
            // blocks in its ghost shell: those are sent to it
            bool feeds = false;
            for (const Candidate &cd : cand[b]) feeds = feeds || owned(cd.block);
            if (!feeds) continue;
        }
        const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
        const int px = nx + 2, py = ny + 2, pz = nz + 2;
        const int64_t np = (int64_t)px * py * pz;
        // local padded index p(x,y,z) = (x+1) + px ((y+1) + py (z+1))
        auto pidx = [&](int x, int y, int z) { return (int64_t)(x + 1) + px * ((int64_t)(y + 1) + (int64_t)py * (z + 1)); };
        auto inside = [&](int x, int y, int z) { return x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz; };
        std::vector<uint8_t> kind(np, 255);
        std::vector<uint16_t> param(np, 0);
        std::vector<int32_t> sblock(np, -1);
        std::vector<int64_t> scell(np, 0);
        std::vector<int64_t> slin(in.sparse ? np : 0, 0);  // sparse: source cell's linear interior index
        const std::vector<uint8_t> &fl = flags[b];
        BlockOut &o = bo[b];
        bool has_solid = false;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    uint8_t k = fl.empty() ? (uint8_t)K_FLUID : fl[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)];
                    int64_t p = pidx(x, y, z);
                    kind[p] = k;
                    param[p] = (uint16_t)bparam[b];
                    if (k != K_FLUID) has_solid = true;
                }
        // shell cells covered by a (periodic image of a) block
        for (const Candidate &cd : cand[b]) {
            const auto &C = blocks[cd.block];
            int64_t ilo[3], ihi[3];
            bool empty = false;
            for (int a = 0; a < 3; ++a) {
                ilo[a] = std::max(B.origin[a] - 1, C.origin[a] + cd.shift[a]);
                ihi[a] = std::min(B.origin[a] + B.n[a] + 1, C.origin[a] + C.n[a] + cd.shift[a]);
                if (ilo[a] >= ihi[a]) empty = true;
            }
            if (empty) continue;
            const std::vector<uint8_t> &cf = flags[cd.block];
            for (int64_t gz = ilo[2]; gz < ihi[2]; ++gz)
                for (int64_t gy = ilo[1]; gy < ihi[1]; ++gy)
                    for (int64_t gx = ilo[0]; gx < ihi[0]; ++gx) {
                        int lx = (int)(gx - B.origin[0]), ly = (int)(gy - B.origin[1]), lz = (int)(gz - B.origin[2]);
                        if (lx >= 0 && lx < nx && ly >= 0 && ly < ny && lz >= 0 && lz < nz) continue;  // interior
                        int cx = (int)(gx - cd.shift[0] - C.origin[0]);
                        int cy = (int)(gy - cd.shift[1] - C.origin[1]);
                        int cz = (int)(gz - cd.shift[2] - C.origin[2]);
                        uint8_t k = cf.empty() ? (uint8_t)K_FLUID
                                               : cf[(size_t)cx + (size_t)C.n[0] * ((size_t)cy + (size_t)C.n[1] * cz)];
                        int64_t p = pidx(lx, ly, lz);
                        if (k == K_FLUID) {
                            kind[p] = K_MIRROR;
                            sblock[p] = cd.block;
                            scell[p] = C.cell(cx, cy, cz);
                            if (in.sparse) slin[p] = cx + (int64_t)C.n[0] * (cy + (int64_t)C.n[1] * cz);
                        } else {
                            kind[p] = k;
                            param[p] = (uint16_t)bparam[cd.block];
                        }
                    }
        }
        // remaining shell cells: outside the domain (face kind) or uncovered (no-slip)
        for (int z = -1; z <= nz; ++z)
            for (int y = -1; y <= ny; ++y)
                for (int x = -1; x <= nx; ++x) {
                    int64_t p = pidx(x, y, z);
                    if (kind[p] != 255) continue;
                    int64_t g[3] = {B.origin[0] + x, B.origin[1] + y, B.origin[2] + z};
                    int face = -1;
                    for (int a = 0; a < 3 && face < 0; ++a) {
                        if (g[a] >= lo[a] && g[a] < hi[a]) continue;
                        if (in.periodic[a]) continue;
                        face = 2 * a + (g[a] < lo[a] ? 0 : 1);
                    }
                    if (face >= 0) {
                        const int fk = in.face_kind[face];
                        kind[p] = (fk == kFaceZouHeVelocity || fk == kFaceZouHePressure) ? (uint8_t)K_ZOUHE : (uint8_t)fk;
                        param[p] = (uint16_t)face;
                    } else {
                        kind[p] = K_NOSLIP;
                        param[p] = 0;
                    }
                }
        if (!own) {
            // halo send elements: for each direction, shell cells of this remote block that
            // mirror a fluid cell of an owned block, in the order the owner of the remote block
            // lists them as receive elements (direction, then z, y, x)
            for (int j = 0; j < L.q; ++j)
                for (int z = -1; z <= nz; ++z)
                    for (int y = -1; y <= ny; ++y)
                        for (int x = -1; x <= nx; ++x) {
                            if (!(x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz)) continue;
                            const int64_t p = pidx(x, y, z);
                            if (kind[p] != K_MIRROR || !owned(sblock[p])) continue;
                            const auto &S = blocks[sblock[p]];
                            int sel = 0;
                            int ax = x + L.cx[j], ay = y + L.cy[j], az = z + L.cz[j];
                            if (inside(ax, ay, az) && kind[pidx(ax, ay, az)] == K_FLUID) sel |= 1;
                            int bx = x - L.cx[j], by = y - L.cy[j], bz = z - L.cz[j];
                            if (inside(bx, by, bz) && kind[pidx(bx, by, bz)] == K_FLUID) sel |= 2;
                            if (sel)
                                o.send.push_back(HaloElem{(*in.owner)[b], sel,
                                                          S.offset + (int64_t)j * S.slab + scell[p]});
                        }
            continue;
        }
        // sparse layout: the pull source of every direction of every fluid cell
        if (in.sparse) {
            const int64_t nf = fstart[b + 1] - fstart[b];
            o.snbr.assign((size_t)(L.q - 1) * nf, 0);
            int64_t n = 0;
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        if (kind[pidx(x, y, z)] != K_FLUID) continue;
                        for (int i = 1; i < L.q; ++i) {
                            const int sx = x - L.cx[i], sy = y - L.cy[i], sz = z - L.cz[i];
                            const int64_t p = pidx(sx, sy, sz);
                            const uint8_t k = kind[p];
                            int32_t v;
                            if (k == K_FLUID) {
                                v = (int32_t)(fstart[b] + fidx[b][sx + (size_t)nx * (sy + (size_t)ny * sz)]);
                            } else if (k == K_MIRROR) {
                                v = (int32_t)(fstart[sblock[p]] + fidx[sblock[p]][slin[p]]);
                            } else if (k == K_VELOCITY || k == K_PRESSURE) {
                                // link slot (local number, made global below): the link of fluid
                                // cell x along opp(i), whose value the sweep reads as direction i
                                v = (int32_t)(0x40000000u | (uint32_t)o.slinks.size());
                                o.slinks.push_back(pack_link(L.opp[i], k, param[p], 0, fstart[b] + n));
                            } else {
                                v = kSparseBounce;
                            }
                            o.snbr[(size_t)(i - 1) * nf + n] = v;
                        }
                        ++n;
                    }
        }
        // wet-node (Zou-He) faces: the fluid cells of the block's first layer at such a face
        for (int fce = 0; fce < 6; ++fce) {
            const int fk = in.face_kind[fce], a = fce / 2, side = fce % 2;
            if (in.periodic[a] || (fk != kFaceZouHeVelocity && fk != kFaceZouHePressure)) continue;
            if (side == 0 ? B.origin[a] != lo[a] : B.origin[a] + B.n[a] != hi[a]) continue;
            const int layer = side == 0 ? 0 : B.n[a] - 1;
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        const int xyz[3] = {x, y, z};
                        if (xyz[a] != layer || kind[pidx(x, y, z)] != K_FLUID) continue;
                        o.zouhe.push_back(pack_zouhe(fce, b, B.cell(x, y, z)));
                    }
        }
        // links: fluid interior cell x, direction q with a boundary neighbour
        for (int qd = 1; qd < L.q; ++qd) {
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        if (kind[pidx(x, y, z)] != K_FLUID) continue;
                        int64_t pn = pidx(x + L.cx[qd], y + L.cy[qd], z + L.cz[qd]);
                        uint8_t k = kind[pn];
                        // no-slip is applied by the sweep from the cell mask (bounce bits)
                        if (k == K_VELOCITY || k == K_PRESSURE)
                            o.links[k].push_back(pack_link(qd, k, param[pn], b, B.cell(x, y, z)));
                    }
        }
        // ghost runs (only for blocks that cannot read their neighbours in place): for each
        // direction, shell cells mirroring a fluid cell, in (z, y, x) order
        const int64_t base = B.offset;
        for (int j = 0; j < L.q && !through[b]; ++j) {
            for (int z = -1; z <= nz; ++z)
                for (int y = -1; y <= ny; ++y)
                    for (int x = -1; x <= nx; ++x) {
                        bool shell = x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz;
                        if (!shell) continue;
                        int64_t p = pidx(x, y, z);
                        if (kind[p] != K_MIRROR) continue;
                        const auto &S = blocks[sblock[p]];
                        int64_t dst = base + (int64_t)j * B.slab + B.cell(x, y, z);
                        // two-grid pull: interior fluid cell g + c_j reads slot j of g
                        int ax = x + L.cx[j], ay = y + L.cy[j], az = z + L.cz[j];
                        const bool pull = inside(ax, ay, az) && kind[pidx(ax, ay, az)] == K_FLUID;
                        // AA: interior fluid cell g - c_j reads and writes slot j of g
                        int bx = x - L.cx[j], by = y - L.cy[j], bz = z - L.cz[j];
                        const bool aa = inside(bx, by, bz) && kind[pidx(bx, by, bz)] == K_FLUID;
                        if (!owned(sblock[p])) {
                            // the source lives on another rank: received into this ghost slot
                            if (pull || aa)
                                o.recv.push_back(HaloElem{(*in.owner)[sblock[p]], (pull ? 1 : 0) | (aa ? 2 : 0), dst});
                            continue;
                        }
                        int64_t src = S.offset + (int64_t)j * S.slab + scell[p];
                        if (pull) {
                            append_run(o.runs_pull, src, dst, S.pitch, B.pitch);
                            o.slots_pull++;
                        }
                        if (aa) {
                            append_run(o.runs_aa, src, dst, S.pitch, B.pitch);
                            o.slots_aa++;
                        }
                    }
        }
        // cell masks: non-fluid bit and bounce-back bits (source x - c_i is no-slip)
        std::vector<uint32_t> cm((size_t)nx * ny * nz, 0u);
        bool any_mask = has_solid;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    uint32_t m = 0;
                    if (kind[pidx(x, y, z)] != K_FLUID) {
                        m = kCellNotFluid;
                    } else {
                        for (int i = 1; i < L.q; ++i) {
                            // the shell's kinds are those of the cells the ghosts stand for
                            if (kind[pidx(x - L.cx[i], y - L.cy[i], z - L.cz[i])] == K_NOSLIP) {
                                m |= 1u << i;
                                o.bounce++;
                            }
                        }
                    }
                    any_mask = any_mask || m != 0;
                    cm[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)] = m;
                }
        if (any_mask) {
            o.mask.assign((size_t)B.slab, kCellNotFluid);
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x)
                        o.mask[(size_t)B.cell(x, y, z)] = cm[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)];
        }
        const int threads = in.tile[0] * in.tile[1], tz = in.tile[2];
        const int tx = nx < threads ? std::min(nx, threads) : in.tile[0], ty = threads / tx;
        for (int z0 = 0; z0 < nz; z0 += tz)
            for (int y0 = 0; y0 < ny; y0 += ty)
                for (int x0 = 0; x0 < nx; x0 += tx) {
                    int64_t nfl = 0;
                    bool masked = false;
                    for (int z = z0; z < std::min(nz, z0 + tz); ++z)
                        for (int y = y0; y < std::min(ny, y0 + ty); ++y)
                            for (int x = x0; x < std::min(nx, x0 + tx); ++x) {
                                nfl += kind[pidx(x, y, z)] == K_FLUID;
                                masked = masked || cm[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)] != 0;
                            }
                    if (nfl == 0) continue;
                    o.tiles.push_back(Tile{b, (int16_t)x0, (int16_t)y0, (int16_t)z0, (uint8_t)(masked ? 1 : 0),
                                           (uint8_t)(tx - 1)});
                }
        o.cells = (int64_t)nx * ny * nz;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) o.fluid += kind[pidx(x, y, z)] == K_FLUID;
    }
    if (!err.empty()) return err;

    out.links.clear();
    out.runs_pull.clear();
    out.runs_aa.clear();
    out.tiles.clear();
    out.masks.assign(nb, {});
    out.nbr = nbrt;
    out.through = through;
    out.cells = out.fluid_cells = 0;
    out.ghost_slots_pull = out.ghost_slots_aa = 0;
    for (int k = 0; k < 4; ++k) out.link_count[k] = 0;
    for (int k = 1; k < 4; ++k)
        for (int b = 0; b < nb; ++b) {
            out.links.insert(out.links.end(), bo[b].links[k].begin(), bo[b].links[k].end());
            out.link_count[k] += (int64_t)bo[b].links[k].size();
        }
    for (int b = 0; b < nb; ++b) out.link_count[K_NOSLIP] += bo[b].bounce;
    out.zouhe.clear();
    for (int b = 0; b < nb; ++b) out.zouhe.insert(out.zouhe.end(), bo[b].zouhe.begin(), bo[b].zouhe.end());
    // sparse layout: global link slots, the index table direction-major, the cell maps
    out.sparse = SparsePlan{};
    if (in.sparse) {
        SparsePlan &S = out.sparse;
        S.nfluid = fstart[nb];
        S.block_start = fstart;
        std::vector<int64_t> lbase(nb + 1, 0);
        for (int b = 0; b < nb; ++b) lbase[b + 1] = lbase[b] + (int64_t)bo[b].slinks.size();
        S.nslots = S.nfluid + lbase[nb];
        if (S.nslots >= ((int64_t)1 << 30)) return "sparse layout: too many entries (max 2^30)";
        for (int b = 0; b < nb; ++b) S.links.insert(S.links.end(), bo[b].slinks.begin(), bo[b].slinks.end());
        S.nbr.assign((size_t)(L.q - 1) * S.nfluid, 0);
        S.block_of.assign(S.nfluid, 0);
        S.cell_of.assign(S.nfluid, 0);
#pragma omp parallel for schedule(dynamic, 4)
        for (int b = 0; b < nb; ++b) {
            const auto &B = blocks[b];
            const int64_t nf = fstart[b + 1] - fstart[b];
            for (int i = 1; i < L.q; ++i)
                for (int64_t n = 0; n < nf; ++n) {
                    int32_t v = bo[b].snbr[(size_t)(i - 1) * nf + n];
                    if (v != kSparseBounce && (v & 0x40000000))
                        v = (int32_t)(S.nfluid + lbase[b] + (v & 0x3fffffff));
                    S.nbr[(size_t)(i - 1) * S.nfluid + fstart[b] + n] = v;
                }
            int64_t n = fstart[b];
            for (int z = 0; z < B.n[2]; ++z)
                for (int y = 0; y < B.n[1]; ++y)
                    for (int x = 0; x < B.n[0]; ++x)
                        if (fidx[b][x + (size_t)B.n[0] * (y + (size_t)B.n[1] * z)] >= 0) {
                            S.block_of[n] = b;
                            S.cell_of[n] = B.cell(x, y, z);
                            ++n;
                        }
            std::vector<int32_t>().swap(bo[b].snbr);
        }
    }
    // halo lists per peer, elements in block order (the same order on both sides)
    out.halo.clear();
    if (in.owner) {
        int nranks = in.rank + 1;
        for (int32_t r : *in.owner) nranks = std::max(nranks, (int)r + 1);
        out.halo.assign(nranks, PeerHalo{});
        for (int b = 0; b < nb; ++b) {
            for (const HaloElem &e : bo[b].send) {
                PeerHalo &h = out.halo[e.peer];
                if (e.sel & 1) append_halo(h.send_pull, e.arena, h.n_send_pull++);
                if (e.sel & 2) append_halo(h.send_aa, e.arena, h.n_send_aa++);
            }
            for (const HaloElem &e : bo[b].recv) {
                PeerHalo &h = out.halo[e.peer];
                if (e.sel & 1) append_halo(h.recv_pull, e.arena, h.n_recv_pull++);
                if (e.sel & 2) append_halo(h.recv_aa, e.arena, h.n_recv_aa++);
            }
        }
    }
    for (int b = 0; b < nb; ++b) {
        out.runs_pull.insert(out.runs_pull.end(), bo[b].runs_pull.begin(), bo[b].runs_pull.end());
        out.runs_aa.insert(out.runs_aa.end(), bo[b].runs_aa.begin(), bo[b].runs_aa.end());
        out.ghost_slots_pull += bo[b].slots_pull;
        out.ghost_slots_aa += bo[b].slots_aa;
        out.tiles.insert(out.tiles.end(), bo[b].tiles.begin(), bo[b].tiles.end());
        out.masks[b].swap(bo[b].mask);
        out.cells += bo[b].cells;
        out.fluid_cells += bo[b].fluid;
    }
    return "";
}

}  // namespace lbm
