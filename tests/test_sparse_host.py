"""Host checks of the fluid-cell list layout (no GPU): every table entry of the list sweep is
in range and names the right value -- for fluid cell n at global position x and direction i,
the pull source x - c_i: that fluid cell (in this or a neighbour block, periodic images
wrapped), halfway bounce-back at a solid cell or a no-slip face, or the slot of the velocity
or pressure link of x along opp(i) -- checked against the flag field and the face kinds alone."""
import numpy as np
import pytest

from paper_1909_13772_gb300 import inputs, lbm

BOUNCE = -(2 ** 31)


def _sim(q=19, porosity=0.6, nb=(3, 2, 2)):
    blocks, shape, _ = inputs.rectilinear_blocks(nb=nb, lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=porosity, seed=7, buffer=4.0)
    p = lbm.make_params(stencil=q, storage=lbm.FP32, periodic=(0, 1, 1))
    sim = lbm.Simulation(p, blocks)
    sim.set_face(0, 0, lbm.VELOCITY, (0.02, 0.0, 0.0), 1.0)
    sim.set_face(0, 1, lbm.PRESSURE, (0.0, 0.0, 0.0), 1.0)
    for b, (o, s) in enumerate(sim.blocks):
        sub = flags[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]]
        sim.set_boundary(b, sub if sub.any() else None)
    lbm.lbm_set_sparse(sim.ctx, True)
    return sim, flags, shape


@pytest.mark.parametrize("q", [19, 27])
def test_list_table_names_the_pull_source_of_every_direction(q):
    sim, flags, shape = _sim(q=q)
    try:
        nbr = lbm.lbm_plan_sparse(sim.ctx, 0)
        blk = lbm.lbm_plan_sparse(sim.ctx, 1)
        cell = lbm.lbm_plan_sparse(sim.ctx, 2)
        links = lbm.lbm_plan_sparse(sim.ctx, 3).astype(np.uint64)
        info = sim.info()
        nf = info["fluid_cells"]
        assert blk.size == nf and nbr.size == (q - 1) * nf
        assert info["list_entries"] == nf + links.size
        c, _, opp = lbm.lbm_stencil_table(q)
        # global position of every fluid cell from (block, padded cell index)
        lay = [lbm.lbm_plan_layout(sim.ctx, b) for b in range(len(sim.blocks))]
        pos = np.zeros((nf, 3), dtype=np.int64)
        for b, (o, s) in enumerate(sim.blocks):
            k = np.flatnonzero(blk == b)
            z, r = np.divmod(cell[k], lay[b]["plane"])
            y, x = np.divmod(r, lay[b]["pitch"])
            pos[k] = np.stack([o[0] + x - lay[b]["xo"], o[1] + y - 1, o[2] + z - 1], axis=1)
        assert np.all(flags[pos[:, 2], pos[:, 1], pos[:, 0]] == 0)
        # fluid cells are numbered block by block in (z, y, x) order: positions are unique
        assert len({tuple(p) for p in pos}) == nf
        index = -np.ones(flags.shape, dtype=np.int64)
        index[pos[:, 2], pos[:, 1], pos[:, 0]] = np.arange(nf)
        # links: (q, kind, fluid cell) -> slot
        lk = {}
        for k, w in enumerate(links):
            lk[(int(w & np.uint64(31)), int((w >> np.uint64(32))))] = (nf + k, int((w >> np.uint64(5)) & np.uint64(3)))
        nx, ny, nz = shape
        for i in range(1, q):
            e = nbr[(i - 1) * nf:i * nf]
            src = pos - c[i]
            src[:, 1] %= ny
            src[:, 2] %= nz
            outside = (src[:, 0] < 0) | (src[:, 0] >= nx)
            inside = ~outside
            kind = np.full(nf, -1)
            kind[inside] = flags[src[inside, 2], src[inside, 1], src[inside, 0]]
            fluid = inside & (kind == 0)
            assert np.array_equal(e[fluid], index[src[fluid, 2], src[fluid, 1], src[fluid, 0]])
            solid = inside & (kind == 1)
            assert np.all(e[solid] == BOUNCE)
            # x- face velocity inlet, x+ face pressure outlet: link slots of x along opp(i)
            for n in np.flatnonzero(outside):
                slot, kd = lk[(int(opp[i]), int(n))]
                assert e[n] == slot
                assert kd == (lbm.VELOCITY if src[n, 0] < 0 else lbm.PRESSURE)
        assert np.all((nbr == BOUNCE) | ((nbr >= 0) & (nbr < info["list_entries"])))
    finally:
        sim.close()


def test_list_layout_is_refused_where_it_does_not_apply():
    p = lbm.make_params(stencil=19, storage=lbm.FP32, pattern=lbm.AA)
    sim = lbm.Simulation(p, [((0, 0, 0), (32, 8, 8))])
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_sparse(sim.ctx, True)
        assert e.value.status == 7
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_plan_sparse(sim.ctx, 0)
        assert e.value.status == 2
    finally:
        sim.close()
