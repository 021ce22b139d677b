"""lbm_reduce_noalloc: the allocation-free reduction, for callers that cannot call cudaMalloc
(all their device memory comes from their own pool, or they run where an allocation would
synchronise the device).  It must give the same diagnostics as the context's lbm_reduce for
the same state, on consecutive calls that reuse its fixed scratch array.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process (its first call performs the
per-device set-up)."""
import numpy as np
import pytest

from gpu_helpers import Case, init_sim
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


def _close(got, want):
    assert abs(got[0] / want["mass"] - 1) < 1e-13
    np.testing.assert_allclose(got[1:4], want["momentum"], rtol=1e-10, atol=1e-14)
    assert abs(got[4] / want["kinetic_energy"] - 1) < 1e-10
    assert abs(got[5] / want["max_speed"] - 1) < 1e-10
    assert got[6] == want["nonfinite"] == 0
    assert got[7] == want["fluid_cells"]


@pytest.mark.parametrize("storage,q", [(lbm.FP64, 19), (lbm.FP32, 19), (lbm.FP32, 27)])
def test_noalloc_reduction_matches_lbm_reduce_on_consecutive_calls(storage, q):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    shape = (70, 37, 11)
    force = (1e-5, 2e-6, 0.0)
    case = Case(shape=shape, q=q, collision=lbm.TRT, storage=storage, omega=1.1, force=force, periodic=(1, 0, 1),
                faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho, u = inputs.random_state(shape, seed=31, rho_amp=0.02, u_amp=0.03)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    dtype = torch.float64 if storage == lbm.FP64 else torch.float32
    stream = torch.cuda.current_stream()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (3, 4):  # two calls in a row, on two different states
        sim.step(steps)
        want = sim.reduce()
        f = torch.from_numpy(sim.pdfs(0).reshape(q, -1)).to(dtype).cuda().contiguous()
        out.fill_(float("nan"))
        lbm.lbm_reduce_noalloc(f.data_ptr(), q, storage, f.shape[1], force, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        _close(out.cpu().numpy(), want)
    sim.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = torch.zeros(19, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_reduce_noalloc(f.data_ptr(), 19, lbm.FP32, lbm.REDUCE_NOALLOC_MAX_CELLS + 1, None, out.data_ptr())
    assert e.value.status == 7
    with pytest.raises(lbm.LbmError):
        lbm.lbm_reduce_noalloc(f.data_ptr(), 19, lbm.BF16_DEV, 1, None, out.data_ptr())
