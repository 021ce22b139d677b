"""Shared set-up for the GPU parity tests: one description drives both the CUDA path (through
the C ABI) and the oracle (on the global domain), from the same seeded inputs."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle
from paper_1909_13772_gb300 import lbm

TOL = {lbm.FP64: 1e-12, lbm.FP32: 1e-5}
UNIT_ROUNDOFF = {lbm.FP64: 2.0 ** -53, lbm.FP32: 2.0 ** -24}


@dataclass
class Case:
    shape: tuple
    blocks: list | None = None  # default: one block covering the domain
    q: int = 19
    collision: int = lbm.TRT
    storage: int = lbm.FP64
    pattern: int = lbm.TWO_GRID
    omega: float = 1.2
    magic_lambda: float = 3.0 / 16.0
    force: tuple = (0.0, 0.0, 0.0)
    periodic: tuple = (1, 1, 1)
    faces: tuple = (1, 1, 1, 1, 1, 1)
    face_u: tuple = field(default_factory=lambda: ((0.0, 0.0, 0.0),) * 6)
    face_rho: tuple = (1.0,) * 6
    flags: np.ndarray | None = None
    tile: tuple | None = None
    mrt_rates: tuple | None = None  # MRT: bulk, fourth-, fifth-, sixth-order rates (None: TRT's)
    cumulant_rates: tuple | None = None  # cumulant: the nine rates after shear (None: all 1)

    def block_list(self):
        return self.blocks or [((0, 0, 0), self.shape)]

    def oracle_params(self):
        mrt_s = (1.0,) * 7
        if self.collision == lbm.MRT:
            b, f4, f5, f6 = self.mrt_rates or (None,) * 4
            mrt_s = oracle.mrt_rates(self.q, self.omega, self.magic_lambda, bulk=b, fourth=f4, fifth=f5, sixth=f6)
        return oracle.OracleParams(shape=self.shape, q=self.q, collision=self.collision, omega=self.omega,
                                   magic_lambda=self.magic_lambda, force=self.force, periodic=self.periodic,
                                   face_kind=self.faces, face_u=self.face_u, face_rho=self.face_rho, mrt_s=mrt_s,
                                   cum_s=tuple(self.cumulant_rates or (1.0,) * 9))

    def global_flags(self):
        nx, ny, nz = self.shape
        return self.flags if self.flags is not None else np.zeros((nz, ny, nx), np.uint8)

    def make_sim(self, stream=None, device_buffer=None):
        p = lbm.make_params(stencil=self.q, collision=self.collision, storage=self.storage, pattern=self.pattern,
                            omega=self.omega, magic_lambda=self.magic_lambda, force=self.force,
                            periodic=self.periodic, mrt_rates=self.mrt_rates, cumulant_rates=self.cumulant_rates)
        sim = lbm.Simulation(p, self.block_list(), stream=stream, device_buffer=device_buffer)
        if self.tile:
            sim.set_tile(*self.tile)
        for f in range(6):
            if not self.periodic[f // 2]:
                sim.set_face(f // 2, f % 2, self.faces[f], self.face_u[f], self.face_rho[f])
        fl = self.global_flags()
        for b, (o, s) in enumerate(sim.blocks):
            sub = fl[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]]
            sim.set_boundary(b, sub if sub.any() else None)
        return sim


def split(sim, field_global):
    """Per-block views of a global [..., z, y, x] array."""
    out = []
    for (o, s) in sim.blocks:
        out.append(field_global[..., o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]])
    return out


def init_sim(sim, rho, u):
    for b, (r, v) in enumerate(zip(split(sim, rho), split(sim, u))):
        sim.init(b, r, v)


def gather_pdfs(sim, case):
    nx, ny, nz = case.shape
    f = np.zeros((case.q, nz, ny, nx))
    for b, (o, s) in enumerate(sim.blocks):
        f[:, o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]] = sim.pdfs(b)
    return f


def gather_macro(sim, case):
    nx, ny, nz = case.shape
    rho = np.zeros((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    for b, (o, s) in enumerate(sim.blocks):
        r, v = sim.macroscopic(b)
        rho[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]] = r
        u[:, o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]] = v
    return rho, u


def normwise(a, b, mask=None):
    """max |a - b| / max |b| over the (masked) entries: the error measure of the parity gate."""
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    return float(np.abs(a - b).max() / np.abs(b).max())


def oracle_run(case, rho, u, steps):
    p = case.oracle_params()
    fl = case.global_flags()
    kinds = set(np.unique(fl).tolist())
    cu = cr = None
    if kinds & {oracle.VELOCITY, oracle.PRESSURE}:
        raise NotImplementedError("interior velocity/pressure cells are not used in these cases")
    f0 = oracle.init(p, rho, u, flags=fl)
    return f0, oracle.run(p, f0, steps, flags=fl, cell_u=cu, cell_rho=cr)


def flow_gates(got, want, storage, steps, q, fluid=None, rho0=1.0, growth="sqrt"):
    """Gates on the flow signal, not only on raw PDFs: the normwise errors of the deviations
    f_i - w_i rho0 and of the velocity sum(c f) / sum(f), against derived tolerances.

    Every step stores each value rounded (unit roundoff u of the storage).  The collision damps
    those errors in the non-conserved moments; in the conserved ones (mass, momentum) they are
    not damped.  growth="sqrt": over a short run of a state that changes from step to step they
    add up like a random walk, sqrt(n) u max|f| per value after n steps, and the gate allows 10
    times that.  growth="linear": in a long run of a slowly varying state (the channel from
    rest) consecutive roundings of the same cell repeat their sign, so they can add up
    linearly, n u max|f| per value, and the gate allows 2 times that (a float32 emulation of
    the 10,000-step channel column drifts by 1.1 n u in mass).  The deviation gate is that per-
    value error relative to max|f - w rho0|; the velocity gate the error of a momentum sum over
    the directions with c_a != 0 relative to max|u|.  Returns (dev_err, dev_tol, u_err, u_tol)."""
    c, w, _ = oracle.lattice(q)
    g = got.reshape(q, -1)
    o = want.reshape(q, -1)
    if fluid is not None:
        m = np.asarray(fluid).reshape(-1)
        g, o = g[:, m], o[:, m]
    n = max(int(steps), 1)
    unit = UNIT_ROUNDOFF[storage]
    per_value = (10.0 * np.sqrt(n) if growth == "sqrt" else 2.0 * n) * unit * np.abs(o).max()
    dev_o = o - w[:, None] * rho0
    dev_err = float(np.abs(g - o).max() / np.abs(dev_o).max())
    dev_tol = per_value / float(np.abs(dev_o).max())
    ug = (c.T.astype(np.float64) @ g) / g.sum(0)
    uo = (c.T.astype(np.float64) @ o) / o.sum(0)
    umax = float(np.abs(uo).max())
    u_err = float(np.abs(ug - uo).max() / umax)
    moving = int((np.abs(c[:, 0]) > 0).sum())
    u_tol = moving * per_value / float(o.sum(0).min()) / umax
    assert dev_err <= dev_tol, ("deviation", dev_err, dev_tol)
    assert u_err <= u_tol, ("velocity", u_err, u_tol)
    return dev_err, dev_tol, u_err, u_tol
