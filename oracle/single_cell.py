"""Independent NumPy restatement of one cell's collision (test infrastructure only).

Written separately from ``lbm_oracle.c`` (vectorised NumPy, lattice built with itertools,
moment sums as matrix products) so that a slip in either one (a dropped term, a wrong sign,
a transposed operand) shows up when the two are compared on random cells.

Formulas (waLBerla paper, Sec. 5.1, Eq. 1-3; constants as read in the oracle):
  rho = sum f,  u = (sum c f + F/2) / rho
  feq = w rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2)
  S   = w (3 (c - u) + 9 (c.u) c) . F
  SRT: f* = f - omega (f - feq) + (1 - omega/2) S
  TRT: even/odd split over opposite pairs, rates omega+ and omega- from Lambda.
"""
from __future__ import annotations

import itertools

import numpy as np


def velocity_set(q: int):
    """(c[q,3], w[q]) for D3Q19 / D3Q27 in the library-wide canonical order."""
    if q not in (19, 27):
        raise ValueError(q)
    weights = {19: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}, 27: {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}}[q]
    axis_order = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    vecs = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(x * x for x in v) in weights]

    def key(v):
        n2 = sum(x * x for x in v)
        if n2 == 1:
            return (1, axis_order.index(v))
        return (n2, v)

    vecs.sort(key=key)
    c = np.array(vecs, dtype=np.float64)
    w = np.array([weights[int(round((v * v).sum()))] for v in c])
    return c, w


def opposite(c):
    return np.array([int(np.flatnonzero((c == -ci).all(axis=1))[0]) for ci in c])


def collide(f, q, collision, omega, magic_lambda=3 / 16, force=(0.0, 0.0, 0.0)):
    """Post-collision populations of one cell; ``collision`` is "srt" or "trt"."""
    c, w = velocity_set(q)
    f = np.asarray(f, dtype=np.float64)
    F = np.asarray(force, dtype=np.float64)
    rho = f.sum()
    u = (c.T @ f + F / 2) / rho
    cu = c @ u
    feq = w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))
    S = w * ((3 * (c - u) + 9 * cu[:, None] * c) @ F)
    if collision == "srt":
        return f - omega * (f - feq) + (1 - omega / 2) * S
    om = 1.0 / (magic_lambda / (1.0 / omega - 0.5) + 0.5)
    o = opposite(c)
    even = lambda g: (g + g[o]) / 2  # noqa: E731
    odd = lambda g: (g - g[o]) / 2  # noqa: E731
    return (f - omega * (even(f) - even(feq)) - om * (odd(f) - odd(feq))
            + (1 - omega / 2) * even(S) + (1 - om / 2) * odd(S))


# ---------------------------------------------------------------------------------------
# MRT (Eq. 3) through orthogonal projectors.  The moment groups are the degree classes of
# polynomials in c (momentum; shear; bulk; third, fourth, fifth, sixth order), each taken
# with everything of lower classes removed under the weighted product sum_i w_i a_i b_i.
# Here that is done with a QR factorisation of the sqrt(w)-scaled polynomial values (NumPy's
# Householder QR: the leading columns of Q span the leading columns of the input), instead
# of the C oracle's Gram-Schmidt rows and Gauss-Jordan inverse.  With P_g the projector onto
# group g, acting on populations as P_g = W^(1/2) Q_g Q_g^T W^(-1/2):
#   f* = f - sum_g s_g P_g (f - feq) + sum_g (1 - s_g/2) P_g S.
# ---------------------------------------------------------------------------------------
def _mrt_polys(q):
    """Polynomial columns (values at the velocities) and group labels, in degree order."""
    c, w = velocity_set(q)
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    cols, groups = [], []

    def add(g, *vals):
        for v in vals:
            cols.append(np.asarray(v, dtype=np.float64) * np.ones(len(c)))
            groups.append(g)

    add(0, 1.0)
    add(1, x, y, z)
    add(2, x * y, x * z, y * z, 2 * x * x - y * y - z * z, y * y - z * z)
    add(3, x * x + y * y + z * z)
    add(4, x * (y * y + z * z), x * (y * y - z * z), y * (x * x + z * z), y * (x * x - z * z),
        z * (x * x + y * y), z * (x * x - y * y))
    if q == 27:
        add(4, x * y * z)
    add(5, x * x * y * y, x * x * z * z, y * y * z * z)
    if q == 27:
        add(5, x * x * y * z, y * y * x * z, z * z * x * y)
        add(6, x * x * y * y * z, x * x * z * z * y, y * y * z * z * x)
        add(7, x * x * y * y * z * z)
    return np.stack(cols, axis=1), np.array(groups), c, w


def mrt_projectors(q):
    """{group: P_g[q, q]} acting on populations."""
    A, groups, c, w = _mrt_polys(q)
    sw = np.sqrt(w)
    Qm, R = np.linalg.qr(sw[:, None] * A)
    if np.min(np.abs(np.diag(R))) < 1e-10:
        raise ValueError("moment polynomials are not independent on D3Q%d" % q)
    out = {}
    for g in np.unique(groups):
        Qg = Qm[:, groups == g]
        out[int(g)] = (sw[:, None] * (Qg @ Qg.T)) / sw[None, :]
    return out


def collide_mrt(f, q, rates, force=(0.0, 0.0, 0.0)):
    """Post-collision populations under MRT; ``rates`` = (momentum, shear, bulk, third,
    fourth, fifth, sixth) group rates (mass is conserved)."""
    c, w = velocity_set(q)
    f = np.asarray(f, dtype=np.float64)
    F = np.asarray(force, dtype=np.float64)
    rho = f.sum()
    u = (c.T @ f + F / 2) / rho
    cu = c @ u
    feq = w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))
    S = w * ((3 * (c - u) + 9 * cu[:, None] * c) @ F)
    out = f.copy()
    for g, P in mrt_projectors(q).items():
        s = 0.0 if g == 0 else rates[g - 1]
        out += -s * (P @ (f - feq)) + (1 - s / 2) * (P @ S)
    return out
