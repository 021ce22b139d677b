"""Seeded synthetic inputs (initial fields, geometries, block layouts).

This module holds no lattice Boltzmann arithmetic: it only produces the initial density and
velocity fields, flag fields and block layouts that both the CUDA path and the oracle take
as input.  Every generator is deterministic in its arguments (NumPy ``default_rng(seed)``).

Workloads (the paper's own geometries -- artery tree, vocal fold, crystal filter and the
porous beds of Sec. 5.1.3 -- are not available; these stand in for them):
  * ``taylor_green``   2-D Taylor-Green vortex extruded in z (decays as exp(-2 nu k^2 t)).
  * ``rest``           uniform density, zero velocity (body-force-driven channel start).
  * ``turbulence``     random-phase solenoidal field with E(k) ~ k^(-5/3).
  * ``random_state``   random density/velocity fields for parity tests.
  * ``sphere_packing`` Boolean model of overlapping spheres ("randomly arranged spheres").
  * ``log_uniform_slabs`` / ``rectilinear_blocks``  uneven rectilinear block layouts.
"""
from __future__ import annotations

import math
import os

import numpy as np

FLUID, NOSLIP, VELOCITY, PRESSURE = 0, 1, 2, 3


def taylor_green(n: int, u0: float = 0.01, rho0: float = 1.0, nz: int | None = None, wavelength: int | None = None):
    """2-D Taylor-Green vortex on an n x n x nz periodic box, extruded in z.

    u_x = u0 cos(kx) sin(ky),  u_y = -u0 sin(kx) cos(ky),  u_z = 0,  k = 2 pi / wavelength,
    rho = rho0 (1 - 3/4 u0^2 (cos 2kx + cos 2ky))  (the vortex's pressure field, c_s^2 = 1/3).
    x, y are cell indices.  Returns rho[z,y,x], u[3,z,y,x] (float64).
    """
    nz = n if nz is None else nz
    lam = n if wavelength is None else wavelength
    k = 2.0 * math.pi / lam
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y, x]
    ux = u0 * np.cos(k * X) * np.sin(k * Y)
    uy = -u0 * np.sin(k * X) * np.cos(k * Y)
    rho2 = rho0 * (1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * X) + np.cos(2 * k * Y)))
    rho = np.broadcast_to(rho2, (nz, n, n)).copy()
    u = np.zeros((3, nz, n, n))
    u[0] = ux
    u[1] = uy
    return rho, u


def rest(shape, rho0: float = 1.0):
    """Uniform rho0, zero velocity; shape = (nx, ny, nz)."""
    nx, ny, nz = shape
    return np.full((nz, ny, nx), rho0), np.zeros((3, nz, ny, nx))


def random_state(shape, seed: int, rho_amp: float = 0.05, u_amp: float = 0.05, rho0: float = 1.0):
    """Smooth-free random fields for parity tests: rho in rho0*(1 +- rho_amp), |u_a| <= u_amp."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rho = rho0 * (1.0 + rho_amp * (2.0 * rng.random((nz, ny, nx)) - 1.0))
    u = u_amp * (2.0 * rng.random((3, nz, ny, nx)) - 1.0)
    return rho, u


def turbulence(n: int, seed: int = 1909, kmax: int = 32, umax: float = 0.05, dtype=np.float64):
    """Random-phase solenoidal velocity on an n^3 periodic box with E(k) ~ k^(-5/3).

    Fourier modes on integer shells 1 <= |k| <= kmax get amplitude k^(-11/6) (so that the
    shell energy 4 pi k^2 A^2 goes as k^(-5/3)), a random direction (Gaussian 3-vector) and a
    random phase uniform on [0, 2 pi) from ``default_rng(seed)``; the Leray projection
    removes the compressive part; the real field is rescaled to max |u| = umax.  rho = 1.
    Returns rho[z,y,x], u[3,z,y,x].
    """
    rng = np.random.default_rng(seed)
    try:  # multithreaded transforms when SciPy is present (same transforms, same results)
        import scipy.fft as _fft
        kw = {"workers": os.cpu_count() or 1}
    except ImportError:  # pragma: no cover
        _fft, kw = np.fft, {}
    kf = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    KZ, KY, KX = kf[:, None, None], kf[None, :, None], kr[None, None, :]  # half spectrum along x
    k2 = KX * KX + KY * KY + KZ * KZ
    kmag = np.sqrt(k2)
    shell = np.rint(kmag)
    amp = np.where((shell >= 1) & (shell <= kmax), np.maximum(kmag, 1e-30) ** (-11.0 / 6.0), 0.0)
    del shell, kmag
    uh = np.exp(1j * rng.uniform(0.0, 2.0 * math.pi, size=k2.shape))
    uh *= amp
    del amp
    uh = rng.standard_normal((3,) + k2.shape) * uh[None]
    with np.errstate(invalid="ignore", divide="ignore"):
        inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    del k2

    def project(uh):
        # Leray projection: remove the component along k
        kdotu = (KX * uh[0] + KY * uh[1] + KZ * uh[2]) * inv_k2
        uh[0] -= KX * kdotu
        uh[1] -= KY * kdotu
        uh[2] -= KZ * kdotu
        return uh

    def to_real(uh):
        return np.stack([_fft.irfftn(uh[a], s=(n, n, n), axes=(0, 1, 2), **kw) for a in range(3)])

    u = to_real(project(uh))
    # the real part of a half spectrum is not exactly Hermitian on the kx = 0 and Nyquist
    # planes: project the real field once more so it is solenoidal to rounding
    uh = np.stack([_fft.rfftn(u[a], axes=(0, 1, 2), **kw) for a in range(3)])
    u = to_real(project(uh))
    del uh
    speed = np.sqrt((u * u).sum(axis=0)).max()
    u *= umax / speed
    return np.ones((n, n, n), dtype=dtype), u.astype(dtype, copy=False)


def log_uniform_slabs(nslabs: int, lo: int, hi: int, rng) -> np.ndarray:
    """Slab widths drawn log-uniform on [lo, hi] (rounded to integers)."""
    w = np.exp(rng.uniform(math.log(lo), math.log(hi), size=nslabs))
    return np.clip(np.rint(w), lo, hi).astype(np.int64)


def rectilinear_blocks(nb=(16, 16, 16), lo: int = 16, hi: int = 64, seed: int = 4096):
    """Uneven rectilinear layout: per-axis slab widths log-uniform on [lo, hi].

    Faces of neighbouring blocks match exactly.  Returns (list of (origin, size)), domain
    shape (nx, ny, nz), and the per-axis slab widths.
    """
    rng = np.random.default_rng(seed)
    widths = [log_uniform_slabs(nb[a], lo, hi, rng) for a in range(3)]
    starts = [np.concatenate([[0], np.cumsum(w)[:-1]]) for w in widths]
    blocks = []
    for k in range(nb[2]):
        for j in range(nb[1]):
            for i in range(nb[0]):
                blocks.append(((int(starts[0][i]), int(starts[1][j]), int(starts[2][k])),
                               (int(widths[0][i]), int(widths[1][j]), int(widths[2][k]))))
    shape = tuple(int(w.sum()) for w in widths)
    return blocks, shape, widths


def sphere_packing(shape, radius: float = 8.0, porosity: float = 0.40, seed: int = 7, buffer: float | None = None,
                   periodic=(False, True, True)):
    """Boolean model of overlapping spheres, returned as a flag field uint8[z,y,x] (1 = solid).

    Centres are uniform in the packed region (x in [buffer, nx - buffer), all of y and z);
    spheres wrap across periodic axes; a cell is solid when its centre (index + 1/2) lies
    within ``radius`` of a sphere centre.  Spheres are added in batches (shrinking near the
    target) until the porosity of the packed region is <= ``porosity``.
    """
    nx, ny, nz = shape
    buf = 2.0 * radius if buffer is None else buffer
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    x0, x1 = int(math.floor(buf)), int(math.ceil(nx - buf))
    region = solid[:, :, x0:x1]
    vol_region = region.size
    vsph = 4.0 / 3.0 * math.pi * radius ** 3
    r = int(math.ceil(radius))
    off = np.arange(-r, r + 1)

    def add(c):
        cx, cy, cz = c
        ix = np.floor(cx).astype(int) + off
        iy = np.floor(cy).astype(int) + off
        iz = np.floor(cz).astype(int) + off
        dx = (ix + 0.5 - cx) ** 2
        dy = (iy + 0.5 - cy) ** 2
        dz = (iz + 0.5 - cz) ** 2
        m = (dz[:, None, None] + dy[None, :, None] + dx[None, None, :]) <= radius * radius
        if periodic[0]:
            ix = ix % nx
        if periodic[1]:
            iy = iy % ny
        if periodic[2]:
            iz = iz % nz
        okx = (ix >= 0) & (ix < nx)
        oky = (iy >= 0) & (iy < ny)
        okz = (iz >= 0) & (iz < nz)
        m = m & okz[:, None, None] & oky[None, :, None] & okx[None, None, :]
        zz, yy, xx = np.nonzero(m)
        solid[iz[zz], iy[yy], ix[xx]] = True

    while True:
        phi = 1.0 - region.sum() / vol_region
        if phi <= porosity:
            break
        # expected spheres still needed under the Boolean model, at least one
        need = max(1, int(0.5 * vol_region * (math.log(phi) - math.log(porosity)) / vsph))
        for _ in range(need):
            c = (rng.uniform(buf, nx - buf), rng.uniform(0, ny), rng.uniform(0, nz))
            add(c)
    return solid.astype(np.uint8)
