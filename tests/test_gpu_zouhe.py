"""GPU parity of the wet-node (Zou-He) velocity and pressure faces against the oracle's, which
is pinned on the CPU (imposed boundary moments, exact Couette and Poiseuille); and of single
blocks that wrap onto themselves along periodic axes while other faces carry velocity or
pressure boundaries (the launch then reads boundary ghost slots through the neighbour table,
where the fill writes them).  Gates as everywhere: 1e-12 (FP64) and 1e-5 (FP32) normwise."""
import numpy as np
import pytest

from gpu_helpers import TOL, Case, flow_gates, gather_pdfs, init_sim, normwise, oracle_run
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

ZV, ZP = lbm.ZOUHE_VELOCITY, lbm.ZOUHE_PRESSURE


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _compare(case, rho, u, steps):
    sim = case.make_sim()
    try:
        init_sim(sim, rho, u)
        sim.step(steps)
        got = gather_pdfs(sim, case)
    finally:
        sim.close()
    _, want = oracle_run(case, rho, u, steps)
    fl = case.global_flags() == 0
    err = normwise(got, want, fl)
    assert err <= TOL[case.storage], err
    flow_gates(got, want, case.storage, steps, case.q, fl)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("collision", [lbm.SRT, lbm.TRT])
def test_channel_between_wet_node_walls(storage, collision):
    """Walls at the y faces (one at rest, one moving), periodic x and z, a body force."""
    shape = (40, 23, 9)
    case = Case(shape=shape, q=19, collision=collision, storage=storage, omega=1.3, force=(1e-5, 0.0, 2e-6),
                periodic=(1, 0, 1), faces=(1, 1, ZV, ZV, 1, 1),
                face_u=((0.0, 0.0, 0.0),) * 3 + ((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 2)
    rho, u = inputs.random_state(shape, seed=51, rho_amp=0.02, u_amp=0.03)
    _compare(case, rho, u, 30)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
def test_inlet_outlet_with_obstacles_single_block(storage):
    """Velocity inlet at x-, pressure outlet at x+, periodic y and z (one block wrapping onto
    itself), spheres inside."""
    shape = (48, 20, 18)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.7, seed=3, buffer=6.0)
    case = Case(shape=shape, q=19, collision=lbm.TRT, storage=storage, omega=1 / 0.8, periodic=(0, 1, 1),
                faces=(ZV, ZP, 1, 1, 1, 1), face_u=((0.02, 0.005, 0.0),) + ((0.0, 0.0, 0.0),) * 5,
                face_rho=(1.0, 0.995, 1.0, 1.0, 1.0, 1.0), flags=flags)
    rho, u = inputs.random_state(shape, seed=52, rho_amp=0.01, u_amp=0.02)
    _compare(case, rho, u, 40)


def test_inlet_outlet_uneven_blocks():
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    case = Case(shape=shape, blocks=blocks, q=19, collision=lbm.TRT, storage=lbm.FP64, omega=1 / 0.8,
                force=(1e-6, 0.0, 0.0), periodic=(0, 1, 1), faces=(ZV, ZP, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, flags=flags)
    rho, u = inputs.rest(shape)
    _compare(case, rho, u, 40)


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
def test_link_faces_on_a_self_wrapping_block(pattern, storage):
    """Halfway velocity inlet / pressure outlet on x of a single block that is its own
    neighbour along periodic y and z: the diagonal sources at the edges of those faces."""
    shape = (36, 17, 11)
    case = Case(shape=shape, q=19, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1 / 0.8,
                force=(1e-6, 0.0, 0.0), periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.01, -0.005),) + ((0.0, 0.0, 0.0),) * 5)
    rho, u = inputs.random_state(shape, seed=53, rho_amp=0.01, u_amp=0.02)
    _compare(case, rho, u, 31)


def test_wet_node_faces_refuse_what_they_do_not_cover():
    for kw in (dict(pattern=lbm.AA), dict(stencil=lbm.D3Q27)):
        p = lbm.make_params(storage=lbm.FP32, periodic=(0, 1, 1), **kw)
        sim = lbm.Simulation(p, [((0, 0, 0), (16, 8, 8))])
        try:
            with pytest.raises(lbm.LbmError) as e:
                sim.set_face(0, 0, ZV, (0.01, 0.0, 0.0), 1.0)
            assert e.value.status == 7
        finally:
            sim.close()
    p = lbm.make_params(storage=lbm.FP32, periodic=(0, 0, 1))  # a tangential axis not periodic
    sim = lbm.Simulation(p, [((0, 0, 0), (16, 8, 8))])
    try:
        sim.set_face(0, 0, ZV, (0.01, 0.0, 0.0), 1.0)
        with pytest.raises(lbm.LbmError) as e:
            sim.info()
        assert e.value.status == 7
    finally:
        sim.close()
