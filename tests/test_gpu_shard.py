"""Partitioned runs on the GPU: every rank's context of a Morton-partitioned block layout in one
process (shard.LocalPartition: the packed halo buffers handed from rank to rank by device
copies on one stream), against one context holding every block.

Each cell does the same arithmetic in both runs -- only where a neighbour's values come from
differs (its in-place cells, a local ghost copy, or the halo) -- so the states must agree bit for
bit: under pure streaming (omega = 0: a permutation of the stored values) and under the full
collision with walls, spheres, inlet, outlet and a body force."""
import numpy as np
import pytest

from gpu_helpers import Case, gather_pdfs, init_sim, oracle_run, normwise
from paper_1909_13772_gb300 import inputs, lbm, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _case(storage, pattern, q=19, collision=lbm.TRT, omega=1 / 0.8, force=(0.0, 0.0, 0.0)):
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 3, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    return Case(shape=shape, blocks=blocks, q=q, collision=collision, storage=storage, pattern=pattern, omega=omega,
                force=force, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags)


def _setup(sim, case):
    for f in range(6):
        if not case.periodic[f // 2]:
            sim.set_face(f // 2, f % 2, case.faces[f], case.face_u[f], case.face_rho[f])
    fl = case.global_flags()
    for b, (o, s) in enumerate(sim.blocks):
        sub = fl[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]]
        sim.set_boundary(b, sub if sub.any() else None)


def _partitioned(case, nranks, start, steps, set_pdfs=False):
    """Run the case on `nranks` contexts; returns the gathered PDFs [q, z, y, x]."""
    p = lbm.make_params(stencil=case.q, collision=case.collision, storage=case.storage, pattern=case.pattern,
                        omega=case.omega, magic_lambda=case.magic_lambda, force=case.force, periodic=case.periodic)
    run = shard.LocalPartition(p, case.block_list(), nranks)
    try:
        for s in run.sims:
            _setup(s, case)
        for b, (o, sz) in enumerate(case.block_list()):
            s = run.sims[run.owner[b]]
            sub = start[..., o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]]
            if set_pdfs:
                s.set_pdfs(b, sub)
            else:
                s.init(b, sub[0], sub[1:])
        run.step(steps)
        nx, ny, nz = case.shape
        out = np.zeros((case.q, nz, ny, nx))
        for b, (o, sz) in enumerate(case.block_list()):
            out[:, o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]] = run.sims[run.owner[b]].pdfs(b)
        peers = [shard.halo_peers(s) for s in run.sims]
    finally:
        run.close()
    assert any(peers)  # the layout really exchanges a halo
    return out


def _whole(case, start, steps, set_pdfs=False):
    sim = case.make_sim()
    try:
        if set_pdfs:
            for b, (o, sz) in enumerate(sim.blocks):
                sim.set_pdfs(b, start[:, o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]])
        else:
            init_sim(sim, start[0], start[1:])
        sim.step(steps)
        return gather_pdfs(sim, case)
    finally:
        sim.close()


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_pure_streaming_partitioned_equals_one_context_bitwise(storage, pattern):
    case = _case(storage, pattern, collision=lbm.SRT, omega=0.0)
    case.faces = (lbm.NOSLIP, lbm.NOSLIP, 1, 1, 1, 1)
    nx, ny, nz = case.shape
    fl = case.global_flags() == 0
    rng = np.random.default_rng(3)
    f0 = rng.random((case.q, nz, ny, nx))
    if storage == lbm.FP32:
        f0 = f0.astype(np.float32).astype(np.float64)
    f0[:, ~fl] = 0.0
    want = _whole(case, f0, 5, set_pdfs=True)
    for nranks in (2, 3):
        got = _partitioned(case, nranks, f0, 5, set_pdfs=True)
        np.testing.assert_array_equal(got[:, fl], want[:, fl])


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_collision_run_partitioned_equals_one_context(storage, pattern):
    case = _case(storage, pattern, force=(1e-6, 0.0, 0.0))
    rho, u = inputs.random_state(case.shape, seed=23, rho_amp=0.01, u_amp=0.02)
    start = np.concatenate([rho[None], u])
    want = _whole(case, start, 12)
    fl = case.global_flags() == 0
    for nranks in (2, 4):
        got = _partitioned(case, nranks, start, 12)
        np.testing.assert_array_equal(got[:, fl], want[:, fl])
    if storage == lbm.FP64:
        # and the oracle of the whole domain agrees to the FP64 gate
        _, ref = oracle_run(case, rho, u, 12)
        assert normwise(got, ref, fl) <= 1e-12


def test_d3q27_partitioned_equals_one_context():
    case = _case(lbm.FP64, lbm.AA, q=27, force=(0.0, 1e-6, 0.0))
    rho, u = inputs.random_state(case.shape, seed=24, rho_amp=0.01, u_amp=0.02)
    start = np.concatenate([rho[None], u])
    want = _whole(case, start, 7)
    fl = case.global_flags() == 0
    got = _partitioned(case, 3, start, 7)
    np.testing.assert_array_equal(got[:, fl], want[:, fl])


def test_partitioned_step_refuses_several_steps_per_call():
    case = _case(lbm.FP32, lbm.TWO_GRID)
    p = lbm.make_params(stencil=19, storage=lbm.FP32, periodic=case.periodic, omega=case.omega)
    run = shard.LocalPartition(p, case.block_list(), 2)
    try:
        for s in run.sims:
            _setup(s, case)
        s = run.sims[0]
        for b in range(len(case.block_list())):
            if run.owner[b] == 0:
                rho, u = inputs.rest(case.block_list()[b][1])
                s.init(b, rho, u)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(s.ctx, 2)
        assert e.value.status == 2  # LBM_ERR_STATE
    finally:
        run.close()


def test_partitioned_diagnostics_equal_the_one_context_totals():
    """The ranks' FP64 totals combined in rank order against lbm_reduce of one context holding
    every block: the same cells, summed in another order (mass and momentum to FP64 rounding,
    the counts and the maximum speed exactly)."""
    case = _case(lbm.FP64, lbm.AA, force=(1e-6, 0.0, 0.0))
    rho, u = inputs.random_state(case.shape, seed=25, rho_amp=0.01, u_amp=0.02)
    sim = case.make_sim()
    try:
        init_sim(sim, rho, u)
        sim.step(6)
        want = sim.reduce()
    finally:
        sim.close()
    p = lbm.make_params(stencil=case.q, collision=case.collision, storage=case.storage, pattern=case.pattern,
                        omega=case.omega, magic_lambda=case.magic_lambda, force=case.force, periodic=case.periodic)
    run = shard.LocalPartition(p, case.block_list(), 3)
    try:
        for s in run.sims:
            _setup(s, case)
        for b, (o, sz) in enumerate(case.block_list()):
            run.sims[run.owner[b]].init(b, rho[o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]],
                                        u[:, o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]])
        run.step(6)
        got = run.reduce()
    finally:
        run.close()
    assert got["fluid_cells"] == want["fluid_cells"] and got["nonfinite"] == 0
    assert got["max_speed"] == want["max_speed"]
    assert abs(got["mass"] - want["mass"]) <= 1e-13 * want["mass"]
    for a in range(3):
        assert abs(got["momentum"][a] - want["momentum"][a]) <= 1e-13 * want["mass"]
    assert abs(got["kinetic_energy"] - want["kinetic_energy"]) <= 1e-12 * want["kinetic_energy"]
