"""ctypes wrapper around ``lbm_oracle.c`` (test infrastructure only; see the C file's header).

Arrays follow the oracle's global layout: PDFs ``f[i, z, y, x]``, scalars ``[z, y, x]``,
vectors ``[a, z, y, x]``.  Everything is float64 / uint8 and C-contiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

FLUID, NOSLIP, VELOCITY, PRESSURE, PERIODIC = 0, 1, 2, 3, 4
ZOUHE_VELOCITY, ZOUHE_PRESSURE = 5, 6  # face kinds only: wet-node (Zou-He) boundaries, D3Q19
SRT, TRT, MRT, CUMULANT = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction) into ``oracle/_build``."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _CParams(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3), ("face_kind", ctypes.c_int32 * 6),
        ("omega", ctypes.c_double), ("magic_lambda", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("face_u", (ctypes.c_double * 3) * 6),
        ("face_rho", ctypes.c_double * 6), ("mrt_s", ctypes.c_double * 7), ("cum_s", ctypes.c_double * 9),
    ]


@dataclass
class OracleParams:
    """Global-domain description for the oracle.

    ``face_kind[2*axis+side]`` gives the kind outside each non-periodic face (NOSLIP, VELOCITY
    or PRESSURE); ``face_u`` / ``face_rho`` its wall velocity / density.
    """
    shape: tuple  # (nx, ny, nz)
    q: int = 19
    collision: int = SRT
    omega: float = 1.0
    magic_lambda: float = 3.0 / 16.0
    force: tuple = (0.0, 0.0, 0.0)
    periodic: tuple = (1, 1, 1)
    face_kind: tuple = (NOSLIP,) * 6
    face_u: tuple = field(default_factory=lambda: ((0.0, 0.0, 0.0),) * 6)
    face_rho: tuple = (1.0,) * 6
    # MRT: rates of the moment groups momentum, shear, bulk, third, fourth, fifth, sixth order
    mrt_s: tuple = (1.0,) * 7
    # cumulant (D3Q27): rates of the groups bulk; third order sums, differences, xyz; fourth
    # order diagonal-pair differences, their sum, the mixed ones; fifth; sixth (shear = omega)
    cum_s: tuple = (1.0,) * 9

    def cstruct(self) -> _CParams:
        c = _CParams()
        c.q, c.collision = int(self.q), int(self.collision)
        c.nx, c.ny, c.nz = (int(v) for v in self.shape)
        for a in range(3):
            c.periodic[a] = int(bool(self.periodic[a]))
            c.force[a] = float(self.force[a])
        for k in range(6):
            c.face_kind[k] = int(self.face_kind[k])
            c.face_rho[k] = float(self.face_rho[k])
            for a in range(3):
                c.face_u[k][a] = float(self.face_u[k][a])
        c.omega, c.magic_lambda = float(self.omega), float(self.magic_lambda)
        for g in range(7):
            c.mrt_s[g] = float(self.mrt_s[g])
        for g in range(9):
            c.cum_s[g] = float(self.cum_s[g])
        return c


class _CClosure(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("cs", ctypes.c_double),
                ("mlp", ctypes.POINTER(ctypes.c_float))]


NO_CLOSURE, SMAGORINSKY, MLP = 0, 1, 2


def _closure(kind=NO_CLOSURE, cs=0.0, mlp=None):
    c = _CClosure()
    c.kind, c.cs = int(kind), float(cs)
    keep = None
    if mlp is not None:
        keep = np.ascontiguousarray(mlp, dtype=np.float32)
        c.mlp = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return c, keep


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.POINTER
        dp, ip, u8p = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint8)
        pp = P(_CParams)
        lib.orc_lattice.argtypes = [ctypes.c_int, ip, dp, ip]
        lib.orc_lattice.restype = ctypes.c_int
        lib.orc_omega_minus.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_omega_minus.restype = ctypes.c_double
        lib.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        lib.orc_equilibrium.restype = None
        lib.orc_collide.argtypes = [pp, dp, dp]
        lib.orc_collide.restype = None
        lib.orc_init.argtypes = [pp, u8p, dp, dp, dp]
        lib.orc_init.restype = ctypes.c_int
        lib.orc_run.argtypes = [pp, u8p, dp, dp, dp, dp, ctypes.c_int64]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_macroscopic.argtypes = [pp, u8p, dp, dp, dp]
        lib.orc_macroscopic.restype = ctypes.c_int
        lib.orc_collide_closure.argtypes = [pp, P(_CClosure), dp, dp]
        lib.orc_collide_closure.restype = ctypes.c_double
        lib.orc_run_closure.argtypes = [pp, P(_CClosure), u8p, dp, dp, dp, dp, ctypes.c_int64]
        lib.orc_run_closure.restype = ctypes.c_int
        lib.orc_stream.argtypes = [pp, u8p, dp, dp, dp, dp]
        lib.orc_stream.restype = ctypes.c_int
        lib.orc_mrt_matrix.argtypes = [ctypes.c_int, dp, dp, ip]
        lib.orc_mrt_matrix.restype = ctypes.c_int
        lib.orc_refine_fine_params.argtypes = [pp, ctypes.c_int32, ctypes.c_int32, pp]
        lib.orc_refine_fine_params.restype = ctypes.c_int
        lib.orc_refine_run.argtypes = [pp, ctypes.c_int32, ctypes.c_int32, dp, dp, ctypes.c_int64]
        lib.orc_refine_run.restype = ctypes.c_int
        lib.orc_cumulants.argtypes = [pp, dp, dp, dp]
        lib.orc_cumulants.restype = ctypes.c_int
        lib.orc_cumulants_to_f.argtypes = [ctypes.c_double, dp, dp, dp]
        lib.orc_cumulants_to_f.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        lib.orc_get_threads.argtypes = []
        lib.orc_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def set_threads(n: int) -> None:
    _L().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_L().orc_get_threads())


def lattice(q: int):
    """(c[q,3] int, w[q] float64, opp[q] int) from the oracle's own enumeration."""
    c = np.zeros(3 * q, dtype=np.intc)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.intc)
    rc = _L().orc_lattice(q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                          opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise ValueError("orc_lattice(%d) failed: %d" % (q, rc))
    return c.reshape(q, 3).astype(np.int64), w, opp.astype(np.int64)


def mrt_matrix(q: int):
    """(M[q,q], M^-1[q,q], group[q]) of the oracle's MRT moment space."""
    M = np.zeros((q, q), dtype=np.float64)
    Mi = np.zeros((q, q), dtype=np.float64)
    g = np.zeros(q, dtype=np.intc)
    rc = _L().orc_mrt_matrix(q, _dp(M), _dp(Mi), g.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise ValueError("orc_mrt_matrix(%d) failed: %d" % (q, rc))
    return M, Mi, g.astype(np.int64)


def mrt_rates(q: int, omega: float, magic_lambda: float, bulk=None, fourth=None, fifth=None, sixth=None):
    """MRT group rates (momentum, shear, bulk, third, ..., sixth) for a shear rate omega and a
    third-order rate from Lambda; groups left at None take the TRT rate of their parity."""
    om = omega_minus(omega, magic_lambda)
    pick = lambda v, d: d if v is None else float(v)  # noqa: E731
    return (om, omega, pick(bulk, omega), om, pick(fourth, omega), pick(fifth, om), pick(sixth, omega))


def cumulants(p: OracleParams, f):
    """(C[3,3,3] indexed [c, b, a] for the cumulant of x^a y^b z^c, rho, u) of one D3Q27 cell:
    density-scaled cumulants of order >= 2 about the force-shifted velocity u; C[0,0,0] = rho,
    the first-order entries are the central first moments (-F/2)."""
    fin = np.ascontiguousarray(f, dtype=np.float64)
    C = np.zeros(27, dtype=np.float64)
    ru = np.zeros(4, dtype=np.float64)
    cp = p.cstruct()
    if _L().orc_cumulants(ctypes.byref(cp), _dp(fin), _dp(C), _dp(ru)) != 0:
        raise ValueError("orc_cumulants needs q = 27")
    return C.reshape(3, 3, 3), float(ru[0]), ru[1:].copy()


def cumulants_to_f(rho: float, u, C) -> np.ndarray:
    """Populations of one D3Q27 cell from rho, u and C[3,3,3] (as returned by cumulants)."""
    uu = np.ascontiguousarray(u, dtype=np.float64)
    Cc = np.ascontiguousarray(C, dtype=np.float64).reshape(27)
    f = np.zeros(27, dtype=np.float64)
    if _L().orc_cumulants_to_f(float(rho), _dp(uu), _dp(Cc), _dp(f)) != 0:
        raise ValueError("orc_cumulants_to_f failed")
    return f


def omega_minus(omega_plus: float, magic_lambda: float) -> float:
    return float(_L().orc_omega_minus(omega_plus, magic_lambda))


def equilibrium(q: int, rho: float, u) -> np.ndarray:
    uu = np.ascontiguousarray(u, dtype=np.float64)
    feq = np.zeros(q, dtype=np.float64)
    _L().orc_equilibrium(q, float(rho), _dp(uu), _dp(feq))
    return feq


def collide_cell(p: OracleParams, f) -> np.ndarray:
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(p.q, dtype=np.float64)
    cp = p.cstruct()
    _L().orc_collide(ctypes.byref(cp), _dp(fin), _dp(out))
    return out


def _check_flags(p: OracleParams, flags):
    nx, ny, nz = p.shape
    if flags is None:
        flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    if flags.shape != (nz, ny, nx):
        raise ValueError("flags must have shape (nz, ny, nx)")
    return flags


def init(p: OracleParams, rho, u, flags=None) -> np.ndarray:
    """Post-collision initial state f*(x, 0) from density ``rho[z,y,x]`` and velocity ``u[3,z,y,x]``."""
    nx, ny, nz = p.shape
    flags = _check_flags(p, flags)
    rho = np.ascontiguousarray(np.broadcast_to(rho, (nz, ny, nx)), dtype=np.float64)
    u = np.ascontiguousarray(np.broadcast_to(u, (3, nz, ny, nx)), dtype=np.float64)
    f = np.zeros((p.q, nz, ny, nx), dtype=np.float64)
    cp = p.cstruct()
    rc = _L().orc_init(ctypes.byref(cp), _u8(flags), _dp(rho), _dp(u), _dp(f))
    if rc != 0:
        raise RuntimeError("orc_init failed: %d" % rc)
    return f


def collide_closure(p: OracleParams, f, kind=NO_CLOSURE, cs=0.0, mlp=None):
    """(omega+, post-collision populations) of one cell under a closure."""
    fin = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(p.q, dtype=np.float64)
    cp = p.cstruct()
    cl, keep = _closure(kind, cs, mlp)
    om = _L().orc_collide_closure(ctypes.byref(cp), ctypes.byref(cl), _dp(fin), _dp(out))
    del keep
    return float(om), out


def run(p: OracleParams, f, nsteps: int, flags=None, cell_u=None, cell_rho=None, closure=None) -> np.ndarray:
    """Advance the post-collision state ``f`` by ``nsteps`` steps (returns a new array).
    ``closure``: optional dict(kind=SMAGORINSKY, cs=...) or dict(kind=MLP, mlp=params)."""
    flags = _check_flags(p, flags)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    work = np.zeros_like(f)
    if cell_u is not None:
        cell_u = np.ascontiguousarray(cell_u, dtype=np.float64)
    if cell_rho is not None:
        cell_rho = np.ascontiguousarray(cell_rho, dtype=np.float64)
    kinds = set(np.unique(flags).tolist())
    if (VELOCITY in kinds and (cell_u is None or cell_rho is None)) or (PRESSURE in kinds and cell_rho is None):
        raise ValueError("interior velocity/pressure cells need cell_u / cell_rho")
    cp = p.cstruct()
    cl, keep = _closure(**(closure or {}))
    rc = _L().orc_run_closure(ctypes.byref(cp), ctypes.byref(cl), _u8(flags), _dp(cell_u), _dp(cell_rho), _dp(f),
                              _dp(work), int(nsteps))
    del keep
    if rc != 0:
        raise RuntimeError("orc_run failed: %d" % rc)
    return f


def stream(p: OracleParams, f, flags=None, cell_u=None, cell_rho=None) -> np.ndarray:
    """Pre-collision field f(t + 1) of the post-collision state ``f`` = f*(t): the streaming
    half of one step with its boundaries (zeros at non-fluid cells)."""
    flags = _check_flags(p, flags)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    if cell_u is not None:
        cell_u = np.ascontiguousarray(cell_u, dtype=np.float64)
    if cell_rho is not None:
        cell_rho = np.ascontiguousarray(cell_rho, dtype=np.float64)
    cp = p.cstruct()
    rc = _L().orc_stream(ctypes.byref(cp), _u8(flags), _dp(cell_u), _dp(cell_rho), _dp(f), _dp(out))
    if rc != 0:
        raise RuntimeError("orc_stream failed: %d" % rc)
    return out


def macroscopic(p: OracleParams, f, flags=None):
    """(rho[z,y,x], u[3,z,y,x]) of the stored post-collision state."""
    nx, ny, nz = p.shape
    flags = _check_flags(p, flags)
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros((nz, ny, nx), dtype=np.float64)
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    cp = p.cstruct()
    rc = _L().orc_macroscopic(ctypes.byref(cp), _u8(flags), _dp(f), _dp(rho), _dp(u))
    if rc != 0:
        raise RuntimeError("orc_macroscopic failed: %d" % rc)
    return rho, u


def diagnostics(p: OracleParams, f, flags=None) -> dict:
    """Domain totals over fluid cells: mass, momentum, kinetic energy, max speed."""
    flags = _check_flags(p, flags)
    rho, u = macroscopic(p, f, flags)
    fl = flags == FLUID
    mom = [(rho * u[a])[fl].sum() for a in range(3)]
    speed2 = (u * u).sum(axis=0)
    return {
        "mass": float(rho[fl].sum()),
        "momentum": tuple(float(m) for m in mom),
        "kinetic_energy": float((0.5 * rho * speed2)[fl].sum()),
        "max_speed": float(np.sqrt(speed2[fl].max())) if fl.any() else 0.0,
    }


# ---- static 2:1 refinement (see the refinement section of lbm_oracle.c) ----------------------

def refine_fine_params(p: OracleParams, a: int, b: int) -> OracleParams:
    """Parameters of the fine grid over the coarse columns [a, b): 2x the cells per axis,
    tau_f - 1/2 = 2 (tau_c - 1/2), force / 2."""
    cp = p.cstruct()
    out = _CParams()
    rc = _L().orc_refine_fine_params(ctypes.byref(cp), int(a), int(b), ctypes.byref(out))
    if rc != 0:
        raise ValueError("refinement not supported for these parameters: %d" % rc)
    from dataclasses import replace
    return replace(p, shape=(out.nx, out.ny, out.nz), omega=out.omega, force=tuple(out.force))


def refine_slab_flags(p: OracleParams, a: int, b: int) -> np.ndarray:
    """Coarse flag field with the refined columns [a, b) marked non-fluid."""
    nx, ny, nz = p.shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    x = np.arange(nx)
    fl[..., ((x - a) % nx) < (b - a)] = NOSLIP
    return fl


def refine_init(p: OracleParams, a: int, b: int, rho_c, u_c, rho_f, u_f):
    """(fc, ff): the post-collision initial states of both grids from their own fields."""
    pf = refine_fine_params(p, a, b)
    fc = init(p, rho_c, u_c, flags=refine_slab_flags(p, a, b))
    ff = init(pf, rho_f, u_f)
    return fc, ff


def refine_run(p: OracleParams, a: int, b: int, fc, ff, nsteps: int):
    """Advance both grids by nsteps coarse steps (returns new arrays)."""
    fc = np.array(fc, dtype=np.float64, order="C", copy=True)
    ff = np.array(ff, dtype=np.float64, order="C", copy=True)
    cp = p.cstruct()
    rc = _L().orc_refine_run(ctypes.byref(cp), int(a), int(b), _dp(fc), _dp(ff), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_refine_run failed: %d" % rc)
    return fc, ff
