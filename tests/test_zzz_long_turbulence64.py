"""(Long runs sort last among the GPU tests.) The FP64 reference run of the decaying-turbulence
family -- the run the FP32 and 16-bit storage errors of the turbulence workload are measured
against -- parity-checked against the oracle over a long run: the 64^3 member (D3Q27 TRT, Lambda
= 3/16, tau = 0.52, random-phase k^-5/3 start of inputs.turbulence with seed 1909, shells 1..32,
max|u| = 0.05; fully periodic) after 2,000 steps, AA pattern as the bench launches it. The
oracle's values come from tests/golden/make_turbulence64.py (2 min of oracle time, so they are
stored): 1,024 sampled PDFs, max |f| and the FP64 mass and momentum. A relative 1e-14
perturbation of the start stays at ~1e-14 over the first 400 oracle steps (no chaotic growth at
this Reynolds number), so the gate 1e-12 of max |f| tests the kernels, not the flow."""
import os

import numpy as np
import pytest

from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "turbulence64_d3q27_fp64.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _record():
    rec, rows = {}, []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("maxabs", "mass", "kinetic_energy"):
                rec[parts[0]] = float(parts[1])
            elif parts[0] == "momentum":
                rec["momentum"] = [float(v) for v in parts[1:4]]
            else:
                rows.append((int(parts[0]), int(parts[1]), int(parts[2]), int(parts[3]), float(parts[4])))
    return rec, rows


def test_turbulence64_fp64_2000_steps_matches_oracle_record():
    rec, rows = _record()
    assert len(rows) == 1024
    n = 64
    rho, u = inputs.turbulence(n, seed=1909, kmax=32, umax=0.05)
    p = lbm.make_params(stencil=27, collision=lbm.TRT, storage=lbm.FP64, pattern=lbm.AA, omega=1 / 0.52,
                        periodic=(1, 1, 1))
    sim = lbm.Simulation(p, [((0, 0, 0), (n, n, n))])
    try:
        sim.init(0, rho, u)
        sim.step(2000)
        f = sim.pdfs(0)
        d = sim.reduce()
    finally:
        sim.close()
    idx = np.array([r[:4] for r in rows])
    want = np.array([r[4] for r in rows])
    got = f[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]
    assert np.abs(got - want).max() <= 1e-12 * rec["maxabs"], np.abs(got - want).max() / rec["maxabs"]
    assert abs(np.abs(f).max() / rec["maxabs"] - 1) <= 1e-12
    assert abs(d["mass"] / rec["mass"] - 1) <= 1e-12
    assert np.abs(np.array(d["momentum"]) - np.array(rec["momentum"])).max() <= 1e-9
