"""GPU parity of the cumulant collision (Sec. 5.1.1: cumulants relaxed towards their equilibria)
against the oracle's, D3Q27.  The two share nothing but the definition: the oracle computes the
central moments by direct sums, the cumulants by the set-partition formula over normalised
moments, and returns through a per-axis closed-form inverse; the kernel runs the per-axis
raw/central transforms on deviations from the rest weights and writes the cumulants in excess
form (zero at equilibrium).  Gates as everywhere: 1e-12 (FP64 storage) and 1e-5 (FP32)
normwise on PDFs, plus the derived flow gates on f - w rho0 and u."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, Case, gather_pdfs, init_sim, normwise, flow_gates, oracle_run
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

# bulk, third sum, third difference, xyz, fourth differences, fourth sum, mixed fourth, fifth, sixth
RATES = (1.3, 1.1, 0.9, 1.4, 1.25, 0.8, 1.15, 1.6, 0.7)
ERR_ARG, ERR_UNSUPPORTED = 1, 7


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _run(case, rho, u, steps):
    sim = case.make_sim()
    try:
        init_sim(sim, rho, u)
        sim.step(steps)
        return gather_pdfs(sim, case)
    finally:
        sim.close()


def _compare(case, rho, u, steps):
    got = _run(case, rho, u, steps)
    _, want = oracle_run(case, rho, u, steps)
    fl = case.global_flags() == 0
    err = normwise(got, want, fl)
    assert err <= TOL[case.storage], err
    flow_gates(got, want, case.storage, steps, case.q, fl)
    return got


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_periodic_random_state_with_force(storage, pattern):
    shape = (45, 19, 13)
    case = Case(shape=shape, q=27, collision=lbm.CUMULANT, storage=storage, pattern=pattern, omega=1.6,
                force=(2e-6, -1e-6, 3e-6), cumulant_rates=RATES)
    rho, u = inputs.random_state(shape, seed=41, rho_amp=0.02, u_amp=0.04)
    _compare(case, rho, u, 30)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_unit_higher_rates_with_force(storage, pattern):
    """Every rate beyond the bulk at 1: the kernel resets the cumulants of order 3..6 without
    computing them (the second-order excess from the raw moments alone); same oracle."""
    shape = (45, 19, 13)
    case = Case(shape=shape, q=27, collision=lbm.CUMULANT, storage=storage, pattern=pattern, omega=1.7,
                force=(3e-6, 1e-6, -2e-6), cumulant_rates=(1.35,) + (1.0,) * 8)
    rho, u = inputs.random_state(shape, seed=44, rho_amp=0.02, u_amp=0.04)
    _compare(case, rho, u, 30)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_channel_walls_and_force(storage, pattern):
    shape = (70, 37, 11)
    case = Case(shape=shape, q=27, collision=lbm.CUMULANT, storage=storage, pattern=pattern, omega=1.0,
                force=(1e-5, 0.0, 0.0), periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1),
                cumulant_rates=(1.9, 0.6, 1.5, 1.1, 1.0, 1.2, 0.9, 1.3, 1.7))
    rho, u = inputs.random_state(shape, seed=42, rho_amp=0.02, u_amp=0.03)
    _compare(case, rho, u, 40)


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_porous_multiblock(pattern):
    """Uneven blocks read in place, spheres (no-slip masks), velocity inlet, pressure outlet."""
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    case = Case(shape=shape, blocks=blocks, q=27, collision=lbm.CUMULANT, storage=lbm.FP64, pattern=pattern,
                omega=1 / 0.8, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags,
                cumulant_rates=RATES)
    rho, u = inputs.rest(case.shape)
    _compare(case, rho, u, 40)


def test_decaying_turbulence_32_long_run():
    """The 32^3 member of the decaying-turbulence family (D3Q27, tau 0.52, max|u| 0.05),
    300 steps, FP64 two-grid and FP32 AA, against the oracle."""
    n = 32
    rho, u = inputs.turbulence(n, seed=1909, kmax=16, umax=0.05)
    for storage, pattern in ((lbm.FP64, lbm.TWO_GRID), (lbm.FP32, lbm.AA)):
        case = Case(shape=(n, n, n), q=27, collision=lbm.CUMULANT, storage=storage, pattern=pattern, omega=1 / 0.52)
        _compare(case, rho, u, 300)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
def test_unit_rates_give_the_product_equilibrium(storage):
    """Every rate 1 and no force: after one step of a uniform flow every cell holds
    rho prod_a p(c_a; u_a) with p(0) = 2/3 - u^2, p(+-1) = (1/3 + u^2 +- u)/2 (closed form)."""
    shape = (32, 4, 4)
    case = Case(shape=shape, q=27, collision=lbm.CUMULANT, storage=storage, omega=1.0, cumulant_rates=(1.0,) * 9)
    u0 = np.array([0.04, -0.03, 0.02])
    rho = np.full(shape[::-1], 1.01)
    u = np.broadcast_to(u0[:, None, None, None], (3,) + shape[::-1]).copy()
    got = _run(case, rho, u, 1)
    cc, _, _ = oracle.lattice(27)

    def p1(ca, ua):
        return 2.0 / 3.0 - ua * ua if ca == 0 else 0.5 * (1.0 / 3.0 + ua * ua + ca * ua)

    want = np.array([1.01 * p1(cc[i, 0], u0[0]) * p1(cc[i, 1], u0[1]) * p1(cc[i, 2], u0[2]) for i in range(27)])
    err = np.abs(got - want[:, None, None, None]).max()
    assert err <= (1e-15 if storage == lbm.FP64 else 4e-8), err


def test_aa_equals_two_grid_bitwise():
    shape = (40, 17, 9)
    rho, u = inputs.random_state(shape, seed=43, rho_amp=0.02, u_amp=0.04)
    out = []
    for pattern in (lbm.TWO_GRID, lbm.AA):
        case = Case(shape=shape, q=27, collision=lbm.CUMULANT, storage=lbm.FP32, pattern=pattern, omega=1.3,
                    force=(1e-6, 0.0, 2e-6), cumulant_rates=RATES)
        out.append(_run(case, rho, u, 12))
    np.testing.assert_array_equal(out[0], out[1])


def test_unsupported_combinations_are_refused():
    for stencil, storage in ((lbm.D3Q19, lbm.FP32), (lbm.D3Q27, lbm.FP16_DEV), (lbm.D3Q27, lbm.BF16_DEV)):
        p = lbm.make_params(stencil=stencil, collision=lbm.CUMULANT, storage=storage)
        with pytest.raises(lbm.LbmError) as e:
            lbm.Simulation(p, [((0, 0, 0), (32, 8, 8))])
        assert e.value.status == ERR_UNSUPPORTED
    p = lbm.make_params(stencil=lbm.D3Q27, collision=lbm.CUMULANT, storage=lbm.FP32,
                        cumulant_rates=(1.0,) * 8 + (2.5,))
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p, [((0, 0, 0), (32, 8, 8))])
    assert e.value.status == ERR_ARG
    sim = lbm.Simulation(lbm.make_params(stencil=lbm.D3Q27, collision=lbm.CUMULANT, storage=lbm.FP32),
                         [((0, 0, 0), (32, 8, 8))])
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_sparse(sim.ctx, True)
        assert e.value.status == ERR_UNSUPPORTED
    finally:
        sim.close()
