"""Writes channel_column_2000.txt: the oracle's state of the 256^3 channel workload (D3Q19,
Lambda = 3/16, tau = 1, no-slip walls in y, periodic x and z, body force (1e-6, 0, 0), from
rest) after 2,000 steps, as one 1 x 256 x 1 column -- the flow is x- and z-invariant, so this
column is every column of the full field -- for TRT and for MRT with the bulk and fourth-order
rates the benchmark's MRT variants use.  bench.py states each sweep variant's error against
it.  Calls only the oracle and the seeded input generator.  Run from the repository root:
    python tests/golden/make_channel_column.py"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1909_13772_gb300 import inputs  # noqa: E402

H, STEPS, FORCE, OMEGA, LAMBDA = 256, 2000, (1e-6, 0.0, 0.0), 1.0, 3.0 / 16.0
MRT_BULK, MRT_FOURTH = 1.4, 1.2
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "channel_column_2000.txt")


def column(collision):
    mrt = oracle.mrt_rates(19, OMEGA, LAMBDA, bulk=MRT_BULK, fourth=MRT_FOURTH)
    p = oracle.OracleParams(shape=(1, H, 1), q=19, collision=collision, omega=OMEGA, magic_lambda=LAMBDA,
                            force=FORCE, periodic=(1, 0, 1), face_kind=(1, 1, oracle.NOSLIP, oracle.NOSLIP, 1, 1),
                            mrt_s=mrt)
    rho, u = inputs.rest((1, H, 1))
    return oracle.run(p, oracle.init(p, rho, u), STEPS)[:, 0, :, 0]  # [q, y]


def main():
    with open(PATH, "w") as fh:
        fh.write("# oracle column of the 256^3 channel after %d steps (D3Q19, tau=1, Lambda=3/16, F=1e-6, walls "
                 "in y); rows: collision y f_0 .. f_18; MRT rates bulk=%r fourth=%r; written by "
                 "tests/golden/make_channel_column.py\n" % (STEPS, MRT_BULK, MRT_FOURTH))
        for name, coll in (("trt", oracle.TRT), ("mrt", oracle.MRT)):
            f = column(coll)
            for y in range(H):
                fh.write("%s %d %s\n" % (name, y, " ".join(repr(float(v)) for v in f[:, y])))


def read(path=PATH):
    """{collision name: f[q, y]} from the record."""
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            parts = line.split()
            out.setdefault(parts[0], {})[int(parts[1])] = [float(v) for v in parts[2:]]
    return {k: np.array([v[y] for y in range(len(v))]).T for k, v in out.items()}


if __name__ == "__main__":
    main()
