"""(Long runs sort last among the GPU tests.) The porous-bed configuration's reduced oracle case
over a long run: the porous-bed generator at 4^3 blocks (64 uneven blocks reading each other in
place, spheres, velocity inlet and pressure outlet), D3Q19 TRT tau = 0.8, FP64, 1,000 steps from
rest, both patterns (and the fluid-cell list layout of the two-grid sweep), against the oracle's values stored by tests/golden/make_porous_minibed.py
(5 min of oracle time): 1,024 sampled fluid PDFs (gate 1e-12 of max |f|) and the FP64 mass and
momentum of the fluid cells. Written when no GPU time was left: its first run is the next GPU
test run."""
import importlib.util
import os

import numpy as np
import pytest

from gpu_helpers import Case, init_sim
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "porous_minibed_fp64.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _generator():
    spec = importlib.util.spec_from_file_location("make_porous_minibed",
                                                  os.path.join(HERE, "golden", "make_porous_minibed.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    return gen


def _record():
    rec, rows = {}, []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("maxabs", "mass"):
                rec[parts[0]] = float(parts[1])
            elif parts[0] == "momentum":
                rec["momentum"] = np.array([float(v) for v in parts[1:4]])
            else:
                rows.append((int(parts[0]), int(parts[1]), int(parts[2]), int(parts[3]), float(parts[4])))
    return rec, rows


@pytest.mark.parametrize("pattern,sparse", [(lbm.TWO_GRID, False), (lbm.AA, False), (lbm.TWO_GRID, True)])
def test_porous_minibed_fp64_1000_steps_matches_oracle_record(pattern, sparse):
    """sparse: the fluid-cell list layout (lbm_set_sparse) instead of the dense blocks."""
    gen = _generator()
    rec, rows = _record()
    blocks, shape, flags = gen.geometry()
    idx = np.array([r[:4] for r in rows])
    np.testing.assert_array_equal(idx, gen.sample_positions(flags))
    want = np.array([r[4] for r in rows])
    case = Case(shape=shape, blocks=blocks, q=19, collision=lbm.TRT, storage=lbm.FP64, pattern=pattern,
                omega=1 / gen.TAU, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags)
    rho, u = inputs.rest(shape)
    sim = case.make_sim()
    try:
        if sparse:
            lbm.lbm_set_sparse(sim.ctx, True)
        init_sim(sim, rho, u)
        sim.step(gen.STEPS)
        got = np.full(len(rows), np.nan)
        maxabs = 0.0
        for b, (o, s) in enumerate(sim.blocks):
            f = sim.pdfs(b)  # [q][z][y][x] of the block, non-fluid cells 0
            maxabs = max(maxabs, float(np.abs(f).max()))
            inside = np.all([(idx[:, 3 - a] >= o[a]) & (idx[:, 3 - a] < o[a] + s[a]) for a in range(3)], axis=0)
            k = np.nonzero(inside)[0]
            got[k] = f[idx[k, 0], idx[k, 1] - o[2], idx[k, 2] - o[1], idx[k, 3] - o[0]]
        d = sim.reduce()
    finally:
        sim.close()
    assert not np.isnan(got).any()
    assert np.abs(got - want).max() <= 1e-12 * rec["maxabs"], np.abs(got - want).max() / rec["maxabs"]
    assert abs(maxabs / rec["maxabs"] - 1) <= 1e-12
    assert abs(d["mass"] / rec["mass"] - 1) <= 1e-12
    assert np.abs(np.array(d["momentum"]) - rec["momentum"]).max() <= 1e-12 * rec["mass"]
