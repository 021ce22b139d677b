"""GPU parity of the MRT collision (Eq. 3 with one rate per group of moments) against the
oracle's MRT, which is Eq. 3 written out in moment space (moment matrix, diagonal S, inverse)
and pinned on the CPU.  The kernels compute MRT as TRT plus group corrections, so agreement
here checks that route against the definition.  Gates as everywhere: 1e-12 (FP64 storage)
and 1e-5 (FP32) normwise on PDFs, plus the derived flow gates."""
import numpy as np
import pytest

from gpu_helpers import TOL, Case, gather_pdfs, init_sim, normwise, flow_gates, oracle_run
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

# bulk, fourth, fifth, sixth (fifth and sixth act on D3Q27 only)
RATES = (1.45, 0.85, 1.2, 0.7)
ERR_ARG, ERR_UNSUPPORTED = 1, 7  # lbm_status codes


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
    return got


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("q", [19, 27])
def test_periodic_random_state_with_force(storage, pattern, q):
    shape = (45, 19, 13)
    case = Case(shape=shape, q=q, collision=lbm.MRT, storage=storage, pattern=pattern, omega=1.6, magic_lambda=0.3,
                force=(2e-6, -1e-6, 3e-6), mrt_rates=RATES)
    rho, u = inputs.random_state(shape, seed=31, rho_amp=0.02, u_amp=0.04)
    _compare(case, rho, u, 30)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("q", [19, 27])
def test_channel_walls_and_force(storage, q):
    shape = (70, 37, 11)
    case = Case(shape=shape, q=q, collision=lbm.MRT, storage=storage, pattern=lbm.AA, omega=1.0,
                force=(1e-5, 0.0, 0.0), periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1),
                mrt_rates=(1.9, 0.6, 1.5, 1.1))
    rho, u = inputs.random_state(shape, seed=32, rho_amp=0.02, u_amp=0.03)
    _compare(case, rho, u, 40)


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_porous_multiblock(pattern):
    """Uneven blocks read in place, spheres (no-slip masks), velocity inlet, pressure outlet."""
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    case = Case(shape=shape, blocks=blocks, q=19, collision=lbm.MRT, storage=lbm.FP64, pattern=pattern,
                omega=1 / 0.8, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags,
                mrt_rates=RATES)
    rho, u = inputs.rest(case.shape)
    _compare(case, rho, u, 40)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
def test_trt_rates_reproduce_the_trt_sweep(storage):
    """MRT with every group at the TRT rate of its parity adds zero corrections."""
    shape = (40, 17, 9)
    rho, u = inputs.random_state(shape, seed=33, rho_amp=0.02, u_amp=0.04)
    out = []
    for coll in (lbm.TRT, lbm.MRT):
        case = Case(shape=shape, q=27, collision=coll, storage=storage, omega=1.3, force=(1e-6, 0.0, 2e-6))
        sim = case.make_sim()
        try:
            init_sim(sim, rho, u)
            sim.step(12)
            out.append(gather_pdfs(sim, case))
        finally:
            sim.close()
    unit = np.finfo(np.float64 if storage == lbm.FP64 else np.float32).eps
    assert normwise(out[1], out[0]) <= 4 * unit


def test_unsupported_combinations_are_refused():
    p = lbm.make_params(stencil=lbm.D3Q19, collision=lbm.MRT, storage=lbm.FP16_DEV)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p, [((0, 0, 0), (32, 8, 8))])
    assert e.value.status == ERR_UNSUPPORTED
    p = lbm.make_params(stencil=lbm.D3Q19, collision=lbm.MRT, storage=lbm.FP32, mrt_rates=(2.5, 1.0, 1.0, 1.0))
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p, [((0, 0, 0), (32, 8, 8))])
    assert e.value.status == ERR_ARG
    sim = lbm.Simulation(lbm.make_params(stencil=lbm.D3Q19, collision=lbm.MRT, storage=lbm.FP32),
                         [((0, 0, 0), (32, 8, 8))])
    try:
        with pytest.raises(lbm.LbmError) as e:
            sim.set_closure(lbm.CLOSURE_SMAGORINSKY, cs=0.17)
        assert e.value.status == ERR_UNSUPPORTED
    finally:
        sim.close()
