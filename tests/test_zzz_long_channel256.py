"""The channel workload at its configured length: 256^3 D3Q19 TRT (Lambda = 3/16, tau = 1),
no-slip walls in y (solid ghost layers), periodic x and z, body force 1e-6, from rest, 10,000
steps, in FP64 and FP32, two-grid and AA -- the launch configuration the benchmark times.

The flow is invariant in x and z, so every column of the field must equal the oracle's run of
one 1 x 256 x 1 periodic column for the same 10,000 steps.  Compared: eight seeded columns, one
full x-y plane and one full y-z plane (every column of those).  Every column does the same
arithmetic, so all of them are equal bit for bit.  FP64: PDFs within 1e-12 of max|f| and the
flow signal itself -- the deviations f_i - w_i and the velocity -- within the derived rounding
gates of flow_gates; after 10,000 steps from rest the centre-line velocity is ~1e-2, so a
wrong force or boundary term is far outside them.  FP32: plain FP32 populations (f ~ w, ulp
~ 4e-9) cannot carry 10,000 increments of ~1e-7 without drift -- the roundings of a slowly
varying cell repeat their sign and the mass drifts linearly (7e-5 after 10,000 steps, the
same in a float32 emulation of the column) -- so the FP32 gates are the linear-growth ones
(flow_gates growth="linear", and 2 n u max|f| on the PDFs); the 1e-5 gate of FP32 holds at
the short runs of the other tests.

Run time: the FP64 steps take about a minute per pattern on one GB300 (FP64-pipe bound)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, UNIT_ROUNDOFF, Case, flow_gates, oracle_run
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

N, STEPS, FORCE = 256, 10000, (1e-6, 0.0, 0.0)


@pytest.fixture(scope="module")
def column():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()
    col = Case(shape=(1, N, 1), q=19, collision=lbm.TRT, storage=lbm.FP64, omega=1.0, force=FORCE,
               periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho, u = inputs.rest(col.shape)
    _, want = oracle_run(col, rho, u, STEPS)
    return want[:, 0, :, 0]  # [q, y]


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_channel256_10k_steps_equals_column_oracle(column, storage, pattern):
    case = Case(shape=(N, N, N), q=19, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1.0, force=FORCE,
                periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    sim = case.make_sim()
    try:
        rho, u = inputs.rest(case.shape)
        sim.init(0, rho, u)
        sim.step(STEPS)
        rng = np.random.default_rng(256)
        cols = [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(8)]
        got = [sim.pdfs_region(0, (x, 0, z), (1, N, 1))[:, 0, :, 0] for x, z in cols]
        zplane = int(rng.integers(0, N))
        xplane = int(rng.integers(0, N))
        xy = sim.pdfs_region(0, (0, 0, zplane), (N, N, 1))[:, 0]           # [q, y, x]
        yz = sim.pdfs_region(0, (xplane, 0, 0), (1, N, N))[:, :, :, 0]     # [q, z, y]
    finally:
        sim.close()
    want = column
    fmax = np.abs(want).max()
    # the flow is well developed: centre-line velocity ~1e-2 (uniform acceleration F t away from
    # the walls), so the deviations carry the signal the gates below look at
    c, _, _ = oracle.lattice(19)
    assert (c[:, 0] @ want[:, N // 2]) / want[:, N // 2].sum() > 5e-3
    growth = "sqrt" if storage == lbm.FP64 else "linear"
    tol = TOL[storage] if storage == lbm.FP64 else 2.0 * STEPS * UNIT_ROUNDOFF[storage]
    ref = got[0]
    for g in got:
        assert np.array_equal(g, ref)
    for a in range(N):
        assert np.array_equal(xy[:, :, a], ref), ("x", a)
        assert np.array_equal(yz[:, a, :], ref), ("z", a)
    assert np.abs(ref - want).max() <= tol * fmax
    flow_gates(ref, want, storage, STEPS, 19, growth=growth)
