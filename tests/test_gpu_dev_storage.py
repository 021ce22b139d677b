"""16-bit deviation storage (BF16 / FP16 of f_i - w_i rho0, FP32 collision) against the FP64
oracle.  The storage rounds each stored deviation to the format's unit roundoff u (2^-8 for
BF16, 2^-11 for FP16) every step, so after n steps the normwise PDF error is bounded by
n * u * max|f - w rho0| / max|f| (a worst case: errors of opposite sign mostly cancel).  The
tests assert that bound and report the measured error."""
import numpy as np
import pytest

from gpu_helpers import Case, gather_pdfs, init_sim, normwise, oracle_run
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {lbm.BF16_DEV: 2.0 ** -8, lbm.FP16_DEV: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _bound(storage, steps, want, q):
    from oracle import lattice
    _, w, _ = lattice(q)
    dev = np.abs(want - w[:, None, None, None]).max()
    return steps * UNIT_ROUNDOFF[storage] * dev / np.abs(want).max()


@pytest.mark.parametrize("storage", [lbm.BF16_DEV, lbm.FP16_DEV])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("q", [19, 27])
def test_dev_storage_channel_error_within_rounding_bound(storage, pattern, q):
    shape, steps = (70, 37, 11), 40
    case = Case(shape=shape, q=q, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1.0,
                force=(1e-5, 0.0, 0.0), periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho, u = inputs.random_state(shape, seed=21, rho_amp=0.02, u_amp=0.03)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(steps)
    got = gather_pdfs(sim, case)
    sim.close()
    _, want = oracle_run(case, rho, u, steps)
    err = normwise(got, want)
    assert err <= _bound(storage, steps, want, q), err
    # and clearly better than the bound's worst case: rounding errors do not all add up
    assert err <= 0.5 * _bound(storage, steps, want, q), err


@pytest.mark.parametrize("storage", [lbm.BF16_DEV, lbm.FP16_DEV])
def test_dev_storage_porous_multiblock(storage):
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    case = Case(shape=shape, blocks=blocks, q=19, collision=lbm.TRT, storage=storage, pattern=lbm.AA,
                omega=1 / 0.8, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, flags=flags)
    rho, u = inputs.rest(shape)
    steps = 60
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(steps)
    got = gather_pdfs(sim, case)
    sim.close()
    _, want = oracle_run(case, rho, u, steps)
    fl = case.global_flags() == 0
    err = normwise(got, want, fl)
    assert err <= _bound(storage, steps, np.where(fl[None], want, 0.0) + np.where(fl[None], 0.0, 1e-300), 19)


@pytest.mark.parametrize("storage", [lbm.BF16_DEV, lbm.FP16_DEV])
def test_dev_storage_rest_state_stays_at_weights(storage):
    """At rest with rho = rho0 every deviation is zero up to the FP32 rounding of the
    collision, so the 16-bit run keeps the weights to FP32 accuracy (the deviation form is
    what makes this work; storing f_i itself in 16 bits would round w_i by ~1e-3)."""
    case = Case(shape=(40, 9, 6), q=19, storage=storage, omega=1.3)
    rho, u = inputs.rest(case.shape)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(10)
    got = gather_pdfs(sim, case)
    sim.close()
    from oracle import lattice
    _, w, _ = lattice(19)
    assert np.abs(got - w[:, None, None, None]).max() <= 1e-6
