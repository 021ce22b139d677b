"""Writes porous_minibed_fp64.txt: the oracle's state after 1,000 steps of the porous-bed mini
configuration -- the porous-bed generator at 4^3 blocks (rectilinear_blocks(nb=(4, 4, 4),
lo=16, hi=64, seed=4096); sphere_packing(radius=8, porosity=0.40, seed=7)), D3Q19 TRT
(Lambda = 3/16, tau = 0.8), velocity inlet u = (0.02, 0, 0) at x-, pressure outlet rho = 1 at
x+, periodic y and z, from rest -- sampled at 1,024 seeded fluid (direction, z, y, x) positions,
with the field's max |f| over fluid cells and the FP64 mass and momentum of the fluid cells.
Calls only the oracle and the seeded input generators.  Run from the repository root:
    python tests/golden/make_porous_minibed.py"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1909_13772_gb300 import inputs  # noqa: E402

NB, STEPS, TAU, SAMPLES = 4, 1000, 0.8, 1024


def geometry():
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(NB, NB, NB), lo=16, hi=64, seed=4096)
    flags = inputs.sphere_packing(shape, radius=8.0, porosity=0.40, seed=7)
    return blocks, shape, flags


def params(shape):
    return oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1 / TAU, magic_lambda=3 / 16,
                               periodic=(0, 1, 1), face_kind=(oracle.VELOCITY, oracle.PRESSURE, 1, 1, 1, 1),
                               face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6)


def sample_positions(flags, q=19, count=SAMPLES, seed=1000):
    """Seeded (i, z, y, x) positions on fluid cells (the GPU test draws the same ones)."""
    fz, fy, fx = np.nonzero(flags == 0)
    rng = np.random.default_rng(seed)
    k = rng.integers(0, fz.size, count)
    return np.stack([rng.integers(0, q, count), fz[k], fy[k], fx[k]], axis=1)


def main():
    _, shape, flags = geometry()
    p = params(shape)
    rho, u = inputs.rest(shape)
    f = oracle.run(p, oracle.init(p, rho, u, flags=flags), STEPS, flags=flags)
    d = oracle.diagnostics(p, f, flags=flags)  # fluid cells only
    ff = f[:, flags == 0]
    pos = sample_positions(flags)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "porous_minibed_fp64.txt")
    with open(out, "w") as fh:
        fh.write("# oracle state after %d steps of the 4^3-block porous mini-bed (D3Q19 TRT tau=0.8, inlet 0.02, "
                 "outlet rho=1); written by tests/golden/make_porous_minibed.py\n" % STEPS)
        fh.write("maxabs %r\n" % float(np.abs(ff).max()))
        fh.write("mass %r\n" % d["mass"])
        fh.write("momentum %r %r %r\n" % tuple(d["momentum"]))
        for i, z, y, x in pos:
            fh.write("%d %d %d %d %r\n" % (i, z, y, x, float(f[i, z, y, x])))


if __name__ == "__main__":
    main()
