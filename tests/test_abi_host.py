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
        for polls in (0, -3, (1 << 20) + 1):  # checked before any device work
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_selfcheck_wait(ctx, polls)
            assert e.value.status == 1
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_tile(ctx, 48, 4, 4)
        for bits in (16, 0, 128):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_set_index_bits(ctx, bits)
            assert e.value.status == 1
        lbm.lbm_set_index_bits(ctx, 64)
        lbm.lbm_set_index_bits(ctx, 32)
        # pipelined diagnostics: nothing to post before a step, no ticket to take
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step_diagnostics_post(ctx)
        assert e.value.status == 2
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step_diagnostics_take(ctx, 5)
        assert e.value.status == 2
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step_diagnostics_take(ctx, -1)
        assert e.value.status == 1
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
        self.masks = [lbm.lbm_plan_mask(sim.ctx, b) for b in range(len(sim.blocks))]
        self.nbr = [lbm.lbm_plan_neighbors(sim.ctx, b) for b in range(len(sim.blocks))]

    def bits(self, b, cells):
        """Cell masks (bounce-back bits; bit 31 non-fluid) of interior cells, 0 if none."""
        m = self.masks[b]
        return m[cells].astype(np.int64) if m.size else np.zeros_like(cells, dtype=np.int64)

    def bounce(self, b, cells, i):
        return ((self.bits(b, cells) >> i) & 1).astype(bool) if i > 0 else np.zeros(cells.shape, bool)

    def cell(self, b, x, y, z):
        L = self.lay[b]
        return (z + 1) * L["plane"] + (y + 1) * L["pitch"] + L["xo"] + x

    def doff(self, b, i):
        L = self.lay[b]
        return self.c[i, 0] + self.c[i, 1] * L["pitch"] + self.c[i, 2] * L["plane"]

    def resolve(self, b, x, y, z, d):
        """(base, slab, cell) of cells (x, y, z) + d of block b: own (ghost) cell, or the
        neighbour block's cell read in place (first/last layer along crossed axes)."""
        L = self.lay[b]
        sx, sy, sz = x + d[0], y + d[1], z + d[2]
        rx = np.where(sx < 0, -1, np.where(sx >= L["nx"], 1, 0))
        ry = np.where(sy < 0, -1, np.where(sy >= L["ny"], 1, 0))
        rz = np.where(sz < 0, -1, np.where(sz >= L["nz"], 1, 0))
        r = (rx + 1) + 3 * (ry + 1) + 9 * (rz + 1)
        nb = np.where((r != 13) & bool(L["through"]), self.nbr[b][r], -1)
        base = np.full(np.shape(sx), L["offset"], dtype=np.int64)
        slab = np.full(np.shape(sx), L["slab"], dtype=np.int64)
        cell = self.cell(b, sx, sy, sz)
        for k in np.unique(nb[nb >= 0]):
            sel = nb == k
            N = self.lay[k]
            xx = np.where(rx[sel] > 0, 0, np.where(rx[sel] < 0, N["nx"] - 1, sx[sel]))
            yy = np.where(ry[sel] > 0, 0, np.where(ry[sel] < 0, N["ny"] - 1, sy[sel]))
            zz = np.where(rz[sel] > 0, 0, np.where(rz[sel] < 0, N["nz"] - 1, sz[sel]))
            base[sel] = N["offset"]
            slab[sel] = N["slab"]
            cell[sel] = self.cell(k, xx, yy, zz)
        return base, slab, cell

    def coords(self, b, cells):
        L = self.lay[b]
        z = cells // L["plane"] - 1
        r = cells - (z + 1) * L["plane"]
        y = r // L["pitch"] - 1
        x = r - (y + 1) * L["pitch"] - L["xo"]
        return x, y, z

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
        o = self.opp[i]
        moved = L["offset"] + o * L["slab"] + cells  # target x + c_i is no-slip: own slot opp(i)
        base, slab, cell = self.resolve(b, *xyz, self.c[i])
        return np.where(self.bounce(b, cells, o), moved, base + i * slab + cell)

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
        par = ((w >> 10) & 255).astype(int)
        blk = ((w >> 18) & 0x3FFF).astype(int)
        cell = (w >> 32).astype(np.int64)
        base = np.array([self.lay[b]["offset"] for b in blk], dtype=np.int64)
        slab = np.array([self.lay[b]["slab"] for b in blk], dtype=np.int64)
        # the boundary cell x + c_q, resolved like the kernels do
        lb_base = np.zeros(len(w), np.int64)
        lb_slab = np.zeros(len(w), np.int64)
        lb_cell = np.zeros(len(w), np.int64)
        for k in range(len(w)):
            xyz = self.coords(blk[k], np.array([cell[k]]))
            bb, ss, cc = self.resolve(blk[k], *xyz, self.c[q[k]])
            lb_base[k], lb_slab[k], lb_cell[k] = bb[0], ss[0], cc[0]
        o = self.opp[q]
        if mode == "pull":
            src, dst = base + q * slab + cell, lb_base + o * lb_slab + lb_cell
        elif mode == "E":
            src, dst = base + o * slab + cell, lb_base + q * lb_slab + lb_cell
        else:
            src, dst = lb_base + q * lb_slab + lb_cell, base + o * slab + cell
        v = self.A[src]
        p = self.params[par]
        cu_w = (self.c[q] * p[:, :3]).sum(axis=1)
        assert (kind == 2).all(), "no-slip is applied in the sweep; pressure links are replayed on the GPU only"
        self.A[dst] = v - 6 * self.w[q] * p[:, 3] * cu_w

    def pull_sweep(self, fluid):
        out = np.zeros((self.q,) + fluid.shape)
        for b in range(len(self.sim.blocks)):
            x, y, z, ox, oy, oz = self.interior(b)
            keep = fluid[z + oz, y + oy, x + ox]
            cells = self.cell(b, x, y, z)[keep]
            L = self.lay[b]
            xyz = (x[keep], y[keep], z[keep])
            for i in range(self.q):
                bb, ss, cc = self.resolve(b, *xyz, -self.c[i])
                normal = bb + i * ss + cc
                bounced = L["offset"] + self.opp[i] * L["slab"] + cells
                out[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]] = \
                    self.A[np.where(self.bounce(b, cells, i), bounced, normal)]
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
                bb, ss, cc = R.resolve(b, *xyz, -R.c[i])
                normal = bb + R.opp[i] * ss + cc
                bounced = L["offset"] + i * L["slab"] + cells  # E layout keeps f*_opp(i)(x) there
                f[i, (z + oz)[keep], (y + oy)[keep], (x + ox)[keep]] = R.A[np.where(R.bounce(b, cells, i), bounced, normal)]
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


@pytest.mark.parametrize("q", [19, 27])
def test_replayed_lists_mixed_in_place_and_ghost_blocks(q):
    """Block 0 matches its neighbours exactly and reads them in place; blocks 1-3 meet
    faces that match no single block and keep ghost copies.  x has a no-slip and a moving
    wall, y and z are periodic."""
    blocks = [((0, 0, 0), (3, 4, 4)), ((3, 0, 0), (3, 4, 4)), ((6, 0, 0), (4, 4, 2)), ((6, 0, 2), (4, 4, 2))]
    shape = (10, 4, 4)
    periodic = (0, 1, 1)
    faces = (lbm.NOSLIP, lbm.VELOCITY, 1, 1, 1, 1)
    uw = (0.0, 0.02, -0.01)
    nx, ny, nz = shape
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[1, 2, 4] = lbm.NOSLIP
    fluid = flags == 0
    f0 = np.random.default_rng(5).random((q, nz, ny, nx))
    f0[:, ~fluid] = 0.0
    op = _oracle_params(q, shape, periodic, faces, uw)
    want1 = oracle.run(op, f0, 1, flags=flags)
    want2 = oracle.run(op, want1, 1, flags=flags)
    for pattern in (lbm.TWO_GRID, lbm.AA):
        sim = _setup(q, blocks, shape, periodic, faces, flags, pattern, uw)
        assert [lbm.lbm_plan_layout(sim.ctx, b)["through"] for b in range(4)] == [1, 0, 0, 0]
        R = Replay(sim, q, shape)
        if pattern == lbm.TWO_GRID:
            R.put(f0, fluid, "pull")
            R.fill_links("pull")
            R.runs(lbm.TWO_GRID)
            np.testing.assert_array_equal(R.pull_sweep(fluid)[:, fluid], want1[:, fluid])
        else:
            R.put(f0, fluid, "E")
            np.testing.assert_array_equal(_replay_aa_step(R, fluid, "E")[:, fluid], want1[:, fluid])
            np.testing.assert_array_equal(_replay_aa_step(R, fluid, "O")[:, fluid], want2[:, fluid])
        sim.close()


def test_channel_link_and_ghost_counts():
    """Channel (walls in y, periodic x/z), D3Q19: 5 wall links per wall cell and wall (applied
    in the sweep).  One block spanning x and z is its own neighbour: no ghost copies; split
    into two halves along x, each reads the other in place."""
    nx, ny, nz = 16, 12, 8
    p = lbm.make_params(stencil=19, periodic=(1, 0, 1))
    sim = lbm.Simulation(p, [((0, 0, 0), (nx, ny, nz))])
    info = sim.info()
    assert info["links"][lbm.NOSLIP] == 2 * 5 * nx * nz
    assert info["cells"] == info["fluid_cells"] == nx * ny * nz
    assert info["ghost_slots"] == 0 and info["ghost_runs"] == 0
    assert lbm.lbm_plan_layout(sim.ctx, 0)["through"] == 1
    nbr = lbm.lbm_plan_neighbors(sim.ctx, 0)
    for r in range(27):
        rx, ry, rz = r % 3 - 1, (r // 3) % 3 - 1, r // 9 - 1
        assert nbr[r] == (-1 if (ry != 0 or r == 13) else 0)
    assert lbm.lbm_plan_links(sim.ctx).size == 0  # no-slip is applied in the sweep
    m = lbm.lbm_plan_mask(sim.ctx, 0)
    L = lbm.lbm_plan_layout(sim.ctx, 0)
    c, _, _ = lbm.lbm_stencil_table(19)
    bottom = m[(0 + 1) * L["plane"] + (0 + 1) * L["pitch"] + L["xo"] + 3]
    want = sum(1 << i for i in range(1, 19) if c[i, 1] == 1)  # sources at y = -1
    assert bottom == want
    sim.close()
    half = nx // 2
    sim = lbm.Simulation(p, [((0, 0, 0), (half, ny, nz)), ((half, 0, 0), (half, ny, nz))])
    info = sim.info()
    assert info["links"][lbm.NOSLIP] == 2 * 5 * nx * nz
    # the halves meet exactly (and wrap around x onto each other): both read in place
    assert info["ghost_slots"] == 0
    for b in (0, 1):
        assert lbm.lbm_plan_layout(sim.ctx, b)["through"] == 1
        nbr = lbm.lbm_plan_neighbors(sim.ctx, b)
        region = lambda rx, ry, rz: (rx + 1) + 3 * (ry + 1) + 9 * (rz + 1)  # noqa: E731
        assert nbr[region(-1, 0, 0)] == 1 - b and nbr[region(1, 0, 0)] == 1 - b
        assert nbr[region(0, 0, -1)] == b and nbr[region(0, 0, 1)] == b  # itself (periodic)
        assert nbr[region(0, 1, 0)] == -1 and nbr[region(1, -1, 0)] == -1  # walls
    sim.close()


def test_closure_rejects_unsupported_contexts_and_bad_arguments():
    """Host-side checks of lbm_set_closure (no device work on these paths)."""
    def ctx(**kw):
        return lbm.lbm_create_blocks(lbm.make_params(**kw), [((0, 0, 0), (8, 8, 8))])

    for kw in (dict(stencil=27), dict(storage=lbm.FP64), dict(storage=lbm.BF16_DEV), dict(force=(1e-5, 0, 0))):
        c = ctx(**kw)
        try:
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_set_closure(c, lbm.CLOSURE_SMAGORINSKY, cs=0.17)
            assert e.value.status == 7, kw
        finally:
            lbm.lbm_destroy(c)
    c = ctx()
    try:
        for kind, cs in ((3, 0.1), (-1, 0.1), (lbm.CLOSURE_SMAGORINSKY, -0.1), (lbm.CLOSURE_SMAGORINSKY, float("nan"))):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_set_closure(c, kind, cs=cs)
            assert e.value.status == 1
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_closure(c, lbm.CLOSURE_MLP)  # no parameters
        assert e.value.status == 1
        with pytest.raises(ValueError):
            lbm.lbm_set_closure(c, lbm.CLOSURE_MLP, mlp_params=np.zeros(10, np.float32))
        lbm.lbm_set_closure(c, lbm.CLOSURE_SMAGORINSKY, cs=0.17)
        lbm.lbm_set_closure(c, lbm.CLOSURE_NONE)
    finally:
        lbm.lbm_destroy(c)


def test_staged_tile_selection_on_the_host():
    """Which sweep tiles stage their source rows in shared memory (lbm_info.staged_tiles, decided
    on the host when the lists are built): 16-bit storage, two-grid, tiles spanning the block's
    full width in at most two rows, no masks, in-place neighbours only the block itself; the
    16-bit two-grid default tile depth is 8."""
    def info(storage, pattern, blocks, periodic, in_place=True, tile=None):
        p = lbm.make_params(stencil=19, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1.2,
                            periodic=periodic)
        c = lbm.lbm_create_blocks(p, blocks)
        try:
            if not in_place:
                lbm.lbm_set_in_place(c, False)
            if tile:
                lbm.lbm_set_tile(c, *tile)
            return lbm.lbm_get_info(c)
        finally:
            lbm.lbm_destroy(c)

    one = [((0, 0, 0), (256, 12, 9))]
    for st in (lbm.BF16_DEV, lbm.FP16_DEV):
        i = info(st, lbm.TWO_GRID, one, (1, 1, 1))
        assert i["tiles"] == 12 * 2 and i["staged_tiles"] == i["tiles"]  # 12 rows x 2 z-tiles of depth 8
        assert info(st, lbm.AA, one, (1, 1, 1))["staged_tiles"] == 0
    for st in (lbm.FP64, lbm.FP32):
        i = info(st, lbm.TWO_GRID, one, (1, 1, 1))
        assert i["tiles"] == 12 * 3 and i["staged_tiles"] == 0  # depth 4
    # walls in y: the rows next to them carry masks (2 rows x 2 z-tiles)
    assert info(lbm.FP16_DEV, lbm.TWO_GRID, one, (1, 0, 1))["staged_tiles"] == 24 - 4
    # a block narrower than half the CTA (several rows per tile) and tiles narrower than the block
    assert info(lbm.FP16_DEV, lbm.TWO_GRID, [((0, 0, 0), (64, 12, 9))], (1, 1, 1))["staged_tiles"] == 0
    assert info(lbm.FP16_DEV, lbm.TWO_GRID, one, (1, 1, 1), tile=(128, 2, 4))["staged_tiles"] == 0
    # two blocks side by side: in place each reads the other (not staged); with ghost copies the
    # unmasked row pairs are (5 row pairs x 2 z-tiles per block, 2 of them next to a wall)
    two = [((0, 0, 0), (128, 10, 9)), ((128, 0, 0), (128, 10, 9))]
    assert info(lbm.FP16_DEV, lbm.TWO_GRID, two, (1, 0, 1))["staged_tiles"] == 0
    assert info(lbm.FP16_DEV, lbm.TWO_GRID, two, (1, 0, 1), in_place=False)["staged_tiles"] == 2 * (10 - 4)
