"""The sweeps' 32-bit neighbour-index arithmetic (the default where every PDF array holds at most
2^32 elements) against the 64-bit form on the same runs: the same bits in every sweep that has
both -- the AA neighbour sweep of each storage, the MRT and cumulant pull gathers, the closure's
AA neighbour sweep -- through the in-place wrap, the neighbour-block table, bounce-back masks and
the velocity/pressure links, with the fused step diagnostics."""
import numpy as np
import pytest

from gpu_helpers import Case, gather_pdfs, init_sim
from oracle import mlp
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _porous(storage, pattern, q=19, collision=lbm.TRT, **kw):
    """Uneven blocks reading each other in place, spheres, velocity inlet and pressure outlet."""
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    return Case(shape=shape, blocks=blocks, q=q, collision=collision, storage=storage, pattern=pattern,
                omega=1 / 0.8, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags, **kw)


def _box(storage, pattern, q=19, collision=lbm.TRT, **kw):
    """One periodic block: its own neighbour on every face (the wrap path)."""
    return Case(shape=(64, 12, 10), q=q, collision=collision, storage=storage, pattern=pattern, omega=1.3,
                force=(2e-6, -1e-6, 1e-6), **kw)


def _run(case, rho, u, steps, bits, closure=None):
    sim = case.make_sim()
    try:
        lbm.lbm_set_index_bits(sim.ctx, bits)
        if closure is not None:
            sim.set_closure(lbm.CLOSURE_MLP, mlp_params=closure)
        init_sim(sim, rho, u)
        sim.step(steps)
        return gather_pdfs(sim, case), sim.step_diagnostics()
    finally:
        sim.close()


CASES = {
    "fp32-aa-porous": lambda: _porous(lbm.FP32, lbm.AA),
    "fp16-aa-porous": lambda: _porous(lbm.FP16_DEV, lbm.AA),
    "fp64-aa-box": lambda: _box(lbm.FP64, lbm.AA),
    "fp32-aa-box-q27": lambda: _box(lbm.FP32, lbm.AA, q=27),
    "bf16-aa-box": lambda: _box(lbm.BF16_DEV, lbm.AA),
    "fp32-mrt-twogrid-porous": lambda: _porous(lbm.FP32, lbm.TWO_GRID, collision=lbm.MRT,
                                               mrt_rates=(1.3, 1.1, 1.0, 1.0)),
    "fp64-mrt-aa-box": lambda: _box(lbm.FP64, lbm.AA, collision=lbm.MRT, mrt_rates=(1.3, 1.1, 1.0, 1.0)),
    "fp32-cumulant-twogrid-box": lambda: _box(lbm.FP32, lbm.TWO_GRID, q=27, collision=lbm.CUMULANT,
                                              cumulant_rates=(1.3, 1.1, 0.9, 1.4, 1.25, 0.8, 1.15, 1.6, 0.7)),
    "fp32-cumulant-aa-porous": lambda: _porous(lbm.FP32, lbm.AA, q=27, collision=lbm.CUMULANT),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_32_bit_indices_equal_64_bit(name):
    case = CASES[name]()
    rho, u = inputs.random_state(case.shape, seed=31, rho_amp=0.02, u_amp=0.03)
    f32, d32 = _run(case, rho, u, 7, 32)
    f64, d64 = _run(case, rho, u, 7, 64)
    np.testing.assert_array_equal(f32, f64)
    assert d32 == d64


def test_closure_aa_32_bit_indices_equal_64_bit():
    case = Case(shape=(64, 16, 8), storage=lbm.FP32, pattern=lbm.AA, omega=1 / 0.505)
    n = 64
    rho, u = inputs.turbulence(n, seed=5, kmax=n // 4, umax=0.08)
    rho, u = np.ascontiguousarray(rho[:8, :16, :64]), np.ascontiguousarray(u[:, :8, :16, :64])
    net = mlp.init_params(seed=12, s_rho=20.0, s_pi=200.0, s_tau=0.02)
    f32, d32 = _run(case, rho, u, 5, 32, closure=net)
    f64, d64 = _run(case, rho, u, 5, 64, closure=net)
    np.testing.assert_array_equal(f32, f64)
    assert d32 == d64
