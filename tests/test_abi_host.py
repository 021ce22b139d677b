"""C-ABI library checks that need no GPU.

* liblbm.so builds (nvcc cross-compiles here), loads, and exports every function that
  include/lbm.h declares.
* The library's stencil table equals the hand-typed canonical tables in tests/golden/.
* The host-side list builder (boundary links, ghost-copy runs, padded layout) is checked
  by replaying one step of pure streaming (omega = 0: the collision is the identity) on the
  CPU with NumPy from the exported lists, and comparing with the oracle's flag-based push
  step -- for two-grid and for both AA phases, on single and uneven multi-block layouts.
"""
import os
import re

import numpy as np
import pytest

import oracle
from golden_tables import lattice_table
from paper_1909_13772_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = lbm.load_library()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lbm.exported_symbols()) == names


@pytest.mark.parametrize("q", [19, 27])
def test_stencil_table_matches_golden(q):
    c, w, opp = lbm.lbm_stencil_table(q)
    gc, gw = lattice_table(q)
    np.testing.assert_array_equal(c, gc)
    np.testing.assert_array_equal(w, np.array([float(x) for x in gw]))
    for i in range(q):
        np.testing.assert_array_equal(c[opp[i]], -c[i])


def test_create_rejects_bad_arguments():
    p = lbm.make_params(omega=2.5)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create_blocks(p, [((0, 0, 0), (4, 4, 4))])
    p = lbm.make_params()
    with pytest.raises(lbm.LbmError):  # overlapping blocks
        lbm.lbm_create_blocks(p, [((0, 0, 0), (4, 4, 4)), ((2, 0, 0), (4, 4, 4))])
    ctx = lbm.lbm_create_blocks(p, [((0, 0, 0), (4, 4, 4))])
    try:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_tile(ctx, 48, 4, 4)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_boundary(ctx, 3, None)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_boundary(ctx, 0, np.full((4, 4, 4), 7, np.uint8))
    finally:
        lbm.lbm_destroy(ctx)


# ---------------------------------------------------------------------------------------
# CPU replay of the exported lists
# ---------------------------------------------------------------------------------------

class Replay:
    """Arena + lists of a context, replayed with NumPy (identity collision)."""

    def __init__(self, sim, q, shape):
        self.sim, self.q, self.shape = sim, q, shape
        self.c, self.w, self.opp = lbm.lbm_stencil_table(q)
        self.lay = [lbm.lbm_plan_layout(sim.ctx, b) for b in range(len(sim.blocks))]
        self.A = np.full(self.lay[0]["arena_elems"], np.nan)
        self.links = lbm.lbm_plan_links(sim.ctx)
        self.params = lbm.lbm_plan_params(sim.ctx)

    def cell(self, b, x, y, z):
        L = self.lay[b]
        return (z + 1) * L["plane"] + (y + 1) * L["pitch"] + L["xo"] + x

    def doff(self, b, i):
        L = self.lay[b]
        return self.c[i, 0] + self.c[i, 1] * L["pitch"] + self.c[i, 2] * L["plane"]

    def wrap(self, b, x, y, z, d):
        """Index shift for neighbour x + d of interior cells (arrays) along self-periodic axes."""
        L = self.lay[b]
        W = L["wrap"]
        s = np.zeros_like(x, dtype=np.int64)
        for a, (pos, n, stride) in enumerate(((x, L["nx"], 1), (y, L["ny"], L["pitch"]), (z, L["nz"], L["plane"]))):
            if not (W >> a) & 1:
                continue
            if d[a] > 0:
                s = s - np.where(pos == n - 1, n * stride, 0)
            elif d[a] < 0:
                s = s + np.where(pos == 0, n * stride, 0)
        return s

    def interior(self, b):
        (ox, oy, oz), (nx, ny, nz) = self.sim.blocks[b]
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return x.ravel(), y.ravel(), z.ravel(), ox, oy, oz

    def slot(self, layout, b, i, cells, xyz):
        L = self.lay[b]
        if layout == "pull":
            return L["offset"] + i * L["slab"] + cells
        if layout == "E":
            return L["offset"] + self.opp[i] * L["slab"] + cells
        return L["offset"] + i * L["slab"] + cells + self.doff(b, i) + self.wrap(b, *xyz, self.c[i])

    def put(self, f, fluid, layout):
        for b in range(len(self.sim.blocks)):
            x, y, z, ox, oy, oz = self.interior(b)
            keep = fluid[z + oz, y + oy, x + ox]
            cells = self.cell(b, x, y, z)[keep]
            xyz = (x[keep], y[keep], z[keep])
            for i in range(self.q):
                self.A[self.slot(layout, b, i, cells, xyz)] = f[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]]

    def get(self, fluid, layout):
        out = np.zeros((self.q,) + fluid.shape)
        for b in range(len(self.sim.blocks)):
            x, y, z, ox, oy, oz = self.interior(b)
            keep = fluid[z + oz, y + oy, x + ox]
            cells = self.cell(b, x, y, z)[keep]
            xyz = (x[keep], y[keep], z[keep])
            for i in range(self.q):
                out[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]] = self.A[self.slot(layout, b, i, cells, xyz)]
        return out

    def runs(self, pattern, reverse=False):
        for src, dst, n, ss, ds in lbm.lbm_plan_runs(self.sim.ctx, pattern):
            s = src + ss * np.arange(n)
            d = dst + ds * np.arange(n)
            if reverse:
                self.A[s] = self.A[d]
            else:
                self.A[d] = self.A[s]

    def fill_links(self, mode, F=(0.0, 0.0, 0.0)):
        w = self.links
        q = (w & 31).astype(int)
        kind = ((w >> 5) & 3).astype(int)
        bits = ((w >> 7) & 7).astype(int)
        par = ((w >> 10) & 255).astype(int)
        blk = ((w >> 18) & 0x3FFF).astype(int)
        cell = (w >> 32).astype(np.int64)
        base = np.array([self.lay[b]["offset"] for b in blk], dtype=np.int64)
        slab = np.array([self.lay[b]["slab"] for b in blk], dtype=np.int64)
        off = np.array([self.doff(b, qq) for b, qq in zip(blk, q)], dtype=np.int64)
        for k in range(len(w)):  # wrap the boundary cell back along self-periodic axes
            L = self.lay[blk[k]]
            for a, (n, stride) in enumerate(((L["nx"], 1), (L["ny"], L["pitch"]), (L["nz"], L["plane"]))):
                if (bits[k] >> a) & 1:
                    off[k] -= self.c[q[k], a] * n * stride
        o = self.opp[q]
        if mode == "pull":
            src, dst = base + q * slab + cell, base + o * slab + cell + off
        elif mode == "E":
            src, dst = base + o * slab + cell, base + q * slab + cell + off
        else:
            src, dst = base + q * slab + cell + off, base + o * slab + cell
        v = self.A[src]
        p = self.params[par]
        cu_w = (self.c[q] * p[:, :3]).sum(axis=1)
        out = np.where(kind == 1, v, v - 6 * self.w[q] * p[:, 3] * cu_w)
        assert not (kind == 3).any(), "pressure links are replayed on the GPU tests only"
        self.A[dst] = out

    def pull_sweep(self, fluid):
        out = np.zeros((self.q,) + fluid.shape)
        for b in range(len(self.sim.blocks)):
            x, y, z, ox, oy, oz = self.interior(b)
            keep = fluid[z + oz, y + oy, x + ox]
            cells = self.cell(b, x, y, z)[keep]
            L = self.lay[b]
            xyz = (x[keep], y[keep], z[keep])
            for i in range(self.q):
                out[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]] = \
                    self.A[L["offset"] + i * L["slab"] + cells - self.doff(b, i) + self.wrap(b, *xyz, -self.c[i])]
        return out


def _replay_aa_step(R, fluid, phase):
    """One AA step with identity collision on the replay arena; returns canonical f*."""
    if phase == "E":
        R.fill_links("E")
        R.runs(lbm.AA)
        # neighbour sweep: f_i(x) = A[x - c_i][opp i]; write A[x + c_i][i]
        f = np.zeros((R.q,) + fluid.shape)
        for b in range(len(R.sim.blocks)):
            x, y, z, ox, oy, oz = R.interior(b)
            keep = fluid[z + oz, y + oy, x + ox]
            cells = R.cell(b, x, y, z)[keep]
            L = R.lay[b]
            xyz = (x[keep], y[keep], z[keep])
            for i in range(R.q):
                f[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]] = \
                    R.A[L["offset"] + R.opp[i] * L["slab"] + cells - R.doff(b, i) + R.wrap(b, *xyz, -R.c[i])]
        R.put(f, fluid, "O")
        return f
    R.fill_links("O")
    R.runs(lbm.AA, reverse=True)
    f = np.zeros((R.q,) + fluid.shape)
    for b in range(len(R.sim.blocks)):
        x, y, z, ox, oy, oz = R.interior(b)
        keep = fluid[z + oz, y + oy, x + ox]
        cells = R.cell(b, x, y, z)[keep]
        L = R.lay[b]
        for i in range(R.q):
            f[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]] = R.A[L["offset"] + i * L["slab"] + cells]
    R.put(f, fluid, "E")
    return f


def _setup(q, blocks, shape, periodic, faces, flags_global, pattern, uw=(0.0, 0.0, 0.0)):
    p = lbm.make_params(stencil=q, collision=lbm.SRT, storage=lbm.FP64, pattern=pattern, omega=0.0,
                        periodic=periodic)
    sim = lbm.Simulation(p, blocks)
    for f, kind in enumerate(faces):
        if not periodic[f // 2]:
            sim.set_face(f // 2, f % 2, kind, u_wall=uw if kind == lbm.VELOCITY else (0, 0, 0))
    for b, (o, s) in enumerate(sim.blocks):
        sub = flags_global[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]]
        sim.set_boundary(b, sub if sub.any() else None)
    return sim


def _oracle_params(q, shape, periodic, faces, uw=(0.0, 0.0, 0.0)):
    fu = [tuple(uw) if k == lbm.VELOCITY else (0.0, 0.0, 0.0) for k in faces]
    return oracle.OracleParams(shape=shape, q=q, collision=oracle.SRT, omega=0.0, periodic=periodic,
                               face_kind=faces, face_u=tuple(fu))


LAYOUTS = {
    "single": ([((0, 0, 0), (7, 5, 4))], (7, 5, 4)),
    "uneven": ([((0, 0, 0), (3, 2, 4)), ((3, 0, 0), (4, 2, 4)), ((0, 2, 0), (3, 3, 4)), ((3, 2, 0), (4, 3, 4))],
               (7, 5, 4)),
    "tiny": ([((0, 0, 0), (1, 5, 1))], (1, 5, 1)),
}


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("layout", ["single", "uneven", "tiny"])
@pytest.mark.parametrize("walls", [False, True])
def test_replayed_lists_stream_like_oracle(q, layout, walls):
    blocks, shape = LAYOUTS[layout]
    nx, ny, nz = shape
    rng = np.random.default_rng(17)
    periodic = (1, 0, 1) if walls else (1, 1, 1)
    faces = (1, 1, lbm.NOSLIP, lbm.VELOCITY, 1, 1) if walls else (1,) * 6
    uw = (0.03, 0.0, -0.01)
    flags = np.zeros((nz, ny, nx), np.uint8)
    if layout != "tiny":
        flags[1, 2, 2] = lbm.NOSLIP
        flags[2, 1:3, 3] = lbm.NOSLIP
    fluid = flags == 0
    f0 = rng.random((q, nz, ny, nx))
    f0[:, ~fluid] = 0.0
    op = _oracle_params(q, shape, periodic, faces, uw)
    want1 = oracle.run(op, f0, 1, flags=flags)
    want2 = oracle.run(op, want1, 1, flags=flags)
    # two-grid
    sim = _setup(q, blocks, shape, periodic, faces, flags, lbm.TWO_GRID, uw)
    R = Replay(sim, q, shape)
    R.put(f0, fluid, "pull")
    R.fill_links("pull")
    R.runs(lbm.TWO_GRID)
    got = R.pull_sweep(fluid)
    np.testing.assert_array_equal(got[:, fluid], want1[:, fluid])
    sim.close()
    # AA: one neighbour step (E -> O), then one local step (O -> E)
    sim = _setup(q, blocks, shape, periodic, faces, flags, lbm.AA, uw)
    R = Replay(sim, q, shape)
    R.put(f0, fluid, "E")
    got1 = _replay_aa_step(R, fluid, "E")
    np.testing.assert_array_equal(got1[:, fluid], want1[:, fluid])
    np.testing.assert_array_equal(R.get(fluid, "O")[:, fluid], want1[:, fluid])
    got2 = _replay_aa_step(R, fluid, "O")
    np.testing.assert_array_equal(got2[:, fluid], want2[:, fluid])
    sim.close()


def test_channel_link_and_ghost_counts():
    """Channel (walls in y, periodic x/z), D3Q19: 5 wall links per wall cell and wall.  One
    block spanning x and z wraps onto itself: no ghost copies.  Split into two blocks along x,
    each still spans z alone (wraps in z) and copies, per x-face ghost cell, the directions
    that enter the neighbour (wrapping z)."""
    nx, ny, nz = 16, 12, 8
    p = lbm.make_params(stencil=19, periodic=(1, 0, 1))
    sim = lbm.Simulation(p, [((0, 0, 0), (nx, ny, nz))])
    info = sim.info()
    assert info["links"][lbm.NOSLIP] == 2 * 5 * nx * nz
    assert info["cells"] == info["fluid_cells"] == nx * ny * nz
    assert info["ghost_slots"] == 0 and info["ghost_runs"] == 0
    assert lbm.lbm_plan_layout(sim.ctx, 0)["wrap"] == 0b101
    sim.close()
    half = nx // 2
    sim = lbm.Simulation(p, [((0, 0, 0), (half, ny, nz)), ((half, 0, 0), (half, ny, nz))])
    info = sim.info()
    assert info["links"][lbm.NOSLIP] == 2 * 5 * nx * nz
    c, _, _ = lbm.lbm_stencil_table(19)
    slots = 0
    for gx in (-1, half):
        for y in range(ny):
            for z in range(nz):
                for i in range(19):
                    ax, ay, az = gx + c[i, 0], y + c[i, 1], (z + c[i, 2]) % nz
                    slots += (0 <= ax < half) and (0 <= ay < ny)
    assert info["ghost_slots"] == 2 * slots
    sim.close()
