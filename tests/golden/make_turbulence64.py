"""Writes turbulence64_d3q27_fp64.txt: the oracle's state after 2,000 steps of the 64^3 member of
the decaying-turbulence family (D3Q27 TRT, Lambda = 3/16, tau = 0.52, random-phase k^-5/3 start
of inputs.turbulence with seed 1909, shells 1..32, max|u| = 0.05; fully periodic), sampled at
1,024 seeded (direction, z, y, x) positions, with the field's max |f| and its FP64 diagnostics.
Calls only the oracle and the seeded input generator.  Run from the repository root:
    python tests/golden/make_turbulence64.py"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1909_13772_gb300 import inputs  # noqa: E402

N, STEPS, TAU, SAMPLES = 64, 2000, 0.52, 1024


def sample_positions(q=27, n=N, count=SAMPLES, seed=2000):
    """The sampled (i, z, y, x) positions (the GPU test draws the same ones)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, q, count), rng.integers(0, n, count), rng.integers(0, n, count),
                     rng.integers(0, n, count)], axis=1)


def main():
    rho, u = inputs.turbulence(N, seed=1909, kmax=32, umax=0.05)
    p = oracle.OracleParams(shape=(N, N, N), q=27, collision=oracle.TRT, omega=1 / TAU, magic_lambda=3 / 16,
                            periodic=(1, 1, 1))
    f = oracle.run(p, oracle.init(p, rho, u), STEPS)
    d = oracle.diagnostics(p, f)
    pos = sample_positions()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "turbulence64_d3q27_fp64.txt")
    with open(out, "w") as fh:
        fh.write("# oracle state after %d steps, 64^3 D3Q27 TRT tau=0.52, inputs.turbulence(64, seed=1909, "
                 "kmax=32, umax=0.05); written by tests/golden/make_turbulence64.py\n" % STEPS)
        fh.write("maxabs %r\n" % float(np.abs(f).max()))
        fh.write("mass %r\n" % d["mass"])
        fh.write("momentum %r %r %r\n" % tuple(d["momentum"]))
        fh.write("kinetic_energy %r\n" % d["kinetic_energy"])
        for i, z, y, x in pos:
            fh.write("%d %d %d %d %r\n" % (i, z, y, x, float(f[i, z, y, x])))


if __name__ == "__main__":
    main()
