"""Static 2:1 grid refinement (Sec. 5.1.1: non-uniform grids by the mass-conserving method of
Rohde et al.): a coarse and a fine context side by side along x in a domain periodic in x, y
and z, coupled by the library's explosion and coalescence transfers (lbm_refine_*).

The coarse block covers the coarse columns [0, A) of an nx x ny x nz box and the fine block the
columns [A, nx) with 2 (nx - A) x 2 ny x 2 nz cells.  The fine grid's rate and force follow from
acoustic scaling (tau_f - 1/2 = 2 (tau_c - 1/2), F_f = F_c / 2).  Marshalling only: every step,
transfer and reduction runs in the library's kernels.
"""
from __future__ import annotations


from . import lbm


def fine_omega(omega_c: float) -> float:
    """The fine grid's rate for the same physical viscosity (two fine steps per coarse step)."""
    return 1.0 / (0.5 + 2.0 * (1.0 / omega_c - 0.5))


class RefinedRun:
    """A refined run: ``coarse`` and ``fine`` are lbm.Simulation objects (one block each);
    ``step(n)`` advances n coarse steps."""

    def __init__(self, params, shape, a, stream=None):
        nx, ny, nz = (int(v) for v in shape)
        a = int(a)
        if not 0 < a < nx:
            raise ValueError("the refined columns [a, nx) must leave coarse columns on the left")
        self.shape, self.a = (nx, ny, nz), a
        pc = lbm.make_params(stencil=params.stencil, collision=params.collision, storage=params.storage,
                             pattern=params.pattern, omega=params.omega, magic_lambda=params.magic_lambda,
                             force=tuple(params.force), periodic=(0, 1, 1))
        pf = lbm.make_params(stencil=params.stencil, collision=params.collision, storage=params.storage,
                             pattern=params.pattern, omega=fine_omega(params.omega),
                             magic_lambda=params.magic_lambda, force=tuple(0.5 * f for f in params.force),
                             periodic=(0, 1, 1))
        self.coarse = lbm.Simulation(pc, [((0, 0, 0), (a, ny, nz))], stream=stream)
        self.fine = lbm.Simulation(pf, [((0, 0, 0), (2 * (nx - a), 2 * ny, 2 * nz))], stream=stream)
        self._r = None
        try:
            for s in (self.coarse, self.fine):
                for side in (0, 1):
                    s.set_face(0, side, lbm.REFINE)
        except Exception:
            self.close()
            raise

    def _coupling(self):
        if self._r is None:
            self._r = lbm.lbm_refine_create(self.coarse.ctx, self.fine.ctx)
        return self._r

    def init(self, rho_c, u_c, rho_f, u_f):
        """Initial fields of both grids: coarse [z, y, x] over the coarse block, fine over the
        fine block (the caller samples its field at each grid's cell centres)."""
        self.coarse.init(0, rho_c, u_c)
        self.fine.init(0, rho_f, u_f)

    def step(self, n=1):
        lbm.lbm_refine_step(self._coupling(), n, self.coarse.ctx)

    def reduce(self):
        """Volume-weighted totals: coarse cells count 1, fine cells 1/8 (FP64)."""
        dc, df = self.coarse.reduce(), self.fine.reduce()
        return {"mass": dc["mass"] + df["mass"] / 8.0,
                "momentum": tuple(a + b / 8.0 for a, b in zip(dc["momentum"], df["momentum"])),
                "kinetic_energy": dc["kinetic_energy"] + df["kinetic_energy"] / 8.0,
                "max_speed": max(dc["max_speed"], df["max_speed"]),
                "nonfinite": dc["nonfinite"] + df["nonfinite"]}

    def close(self):
        if self._r is not None:
            lbm.lbm_refine_destroy(self._r)
            self._r = None
        for s in (getattr(self, "fine", None), getattr(self, "coarse", None)):
            if s is not None:
                s.close()
