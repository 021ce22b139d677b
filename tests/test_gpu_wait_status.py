"""Failure path of the bounded device-side waits, exercised without any GPU fault: one device
thread waits on an mbarrier that nothing arrives on, gives up after a bounded number of polls
and sets the status flag (lbm_selfcheck_wait); the host reads it at the next synchronising call
(LBM_ERR_TIMEOUT, once), and the context keeps working with its state untouched."""
import numpy as np
import pytest

from gpu_helpers import Case, gather_pdfs, init_sim
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

TIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


@pytest.mark.parametrize("storage", [lbm.FP32, lbm.FP16_DEV])
def test_wait_timeout_reported_once_and_context_stays_usable(storage):
    shape = (256, 12, 9)  # FP16: full-width unmasked tiles take the staged (bulk-copy) path
    case = Case(shape=shape, storage=storage, pattern=lbm.TWO_GRID, omega=1.3, force=(1e-5, 0.0, 0.0),
                periodic=(1, 0, 1))
    rho, u = inputs.random_state(shape, seed=41, rho_amp=0.02, u_amp=0.03)
    ref = case.make_sim()
    init_sim(ref, rho, u)
    ref.step(6)
    want = gather_pdfs(ref, case)
    ref.close()

    s = case.make_sim()
    init_sim(s, rho, u)
    s.step(3)
    s.step_diagnostics()
    lbm.lbm_selfcheck_wait(s.ctx, 256)
    with pytest.raises(lbm.LbmError) as e:
        s.step_diagnostics()
    assert e.value.status == TIMEOUT
    s.step_diagnostics()  # reported once, then cleared
    lbm.lbm_selfcheck_wait(s.ctx, 256)
    t = lbm.lbm_step_diagnostics_post(s.ctx)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_diagnostics_take(s.ctx, t)  # the pipelined read reports it too
    assert e.value.status == TIMEOUT
    lbm.lbm_step_diagnostics_take(s.ctx, lbm.lbm_step_diagnostics_post(s.ctx))
    lbm.lbm_selfcheck_wait(s.ctx, 1)
    with pytest.raises(lbm.LbmError) as e:
        s.pdfs(0)
    assert e.value.status == TIMEOUT
    s.step(3)
    d = s.step_diagnostics()
    got = gather_pdfs(s, case)
    s.close()
    assert d["nonfinite"] == 0
    np.testing.assert_array_equal(got, want)  # the self-check left the state alone
