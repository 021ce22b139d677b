"""Pins for the oracle's streaming, boundaries and time stepping (CPU only).

Each test checks the oracle against something the mathematics or fluid mechanics fixes,
not against a second copy of its own formulas:
  * omega = 0 and F = 0 make the collision the identity, so a periodic step is the exact
    shift of each population by c_i (Eq. 2) -- bitwise.
  * uniform acceleration by a body force: u(t) = u0 + t F / rho exactly.
  * Taylor-Green vortex decay rate exp(-2 nu k^2 t), nu = (1/omega - 1/2)/3.
  * Poiseuille flow with TRT, Lambda = 3/16 and halfway bounce-back: the parabola is exact.
  * Couette flow (velocity bounce-back on one wall): the linear profile is exact.
  * Pressure anti-bounce-back: rest state at the wall density is a fixed point; a pressure
    drop drives a channel flow with the Poiseuille flow rate (within compressibility error).
  * Conservation: mass exactly, momentum gains N F per step.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1909_13772_gb300 import inputs


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("q", [19, 27])
def test_pure_streaming_is_exact_shift(q):
    shape = (5, 4, 3)
    p = oracle.OracleParams(shape=shape, q=q, collision=oracle.SRT, omega=0.0)
    c, _, _ = oracle.lattice(q)
    rng = np.random.default_rng(8)
    f = rng.random((q,) + shape[::-1])
    g = oracle.run(p, f, 1)
    for i in range(q):
        want = np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(g[i], want)


@pytest.mark.parametrize("q", [19, 27])
def test_pure_streaming_with_walls_permutes_values(q):
    """omega = 0 with no-slip walls: each step is a permutation of the stored values."""
    shape = (4, 5, 3)
    p = oracle.OracleParams(shape=shape, q=q, collision=oracle.SRT, omega=0.0, periodic=(1, 0, 0),
                            face_kind=(1, 1, 1, 1, 1, 1))
    flags = np.zeros(shape[::-1], dtype=np.uint8)
    flags[1, 2, 1] = oracle.NOSLIP  # an interior obstacle too
    rng = np.random.default_rng(9)
    f = rng.random((q,) + shape[::-1])
    f[:, flags == oracle.NOSLIP] = 0.0
    g = oracle.run(p, f, 3, flags=flags)
    fl = flags == oracle.FLUID
    np.testing.assert_array_equal(np.sort(g[:, fl].ravel()), np.sort(f[:, fl].ravel()))


@pytest.mark.parametrize("q,coll", [(19, oracle.SRT), (19, oracle.TRT), (27, oracle.TRT)])
def test_uniform_acceleration(q, coll):
    shape = (3, 4, 2)
    F = (2e-5, -1e-5, 3e-6)
    u0 = np.array([0.01, -0.02, 0.005])
    p = oracle.OracleParams(shape=shape, q=q, collision=coll, omega=1.3, force=F)
    rho = np.ones(shape[::-1])
    u = np.broadcast_to(u0[:, None, None, None], (3,) + shape[::-1])
    f = oracle.init(p, rho, u)
    r0, v0 = oracle.macroscopic(p, f)
    np.testing.assert_allclose(v0, u, rtol=0, atol=1e-16)
    n = 40
    g = oracle.run(p, f, n)
    r, v = oracle.macroscopic(p, g)
    np.testing.assert_allclose(r, 1.0, rtol=0, atol=1e-14)
    want = u0 + n * np.array(F)
    for a in range(3):
        np.testing.assert_allclose(v[a], want[a], rtol=0, atol=1e-15)


def _tgv_amplitude(u, k):
    nz, ny, nx = u.shape[1:]
    x = np.arange(nx)
    y = np.arange(ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    mode = np.cos(k * X) * np.sin(k * Y)
    return (u[0] * mode[None]).sum() / (mode * mode).sum() / nz


@pytest.mark.parametrize("q", [19, 27])
def test_taylor_green_decay_rate(q):
    """32^3, SRT, tau = 0.6, u0 = 0.01, 100 steps: A(t) vs exp(-2 nu k^2 t), nu = (tau - 1/2)/3.

    The equilibrium start carries no viscous stress, so the first ~10 steps are a transient
    (rate ~24 % high); over steps 20..100 the decay rate is that of the Navier-Stokes vortex
    up to the O(k^2) lattice error (measured ~1e-4; tolerance 5e-3)."""
    n, tau, t0, steps = 32, 0.6, 20, 100
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / n
    p = oracle.OracleParams(shape=(n, n, n), q=q, collision=oracle.SRT, omega=1 / tau)
    rho, u = inputs.taylor_green(n, u0=0.01)
    f = oracle.run(p, oracle.init(p, rho, u), t0)
    a0 = _tgv_amplitude(oracle.macroscopic(p, f)[1], k)
    g = oracle.run(p, f, steps - t0)
    a1 = _tgv_amplitude(oracle.macroscopic(p, g)[1], k)
    rate = -math.log(a1 / a0) / (steps - t0)
    want = 2 * nu * k * k
    assert abs(rate / want - 1) < 5e-3, (rate, want)


def _channel(H, q, coll, omega, F=(0.0, 0.0, 0.0), lam=3 / 16, top=oracle.NOSLIP, uw=(0.0, 0.0, 0.0)):
    fu = [(0.0, 0.0, 0.0)] * 6
    fu[3] = uw
    return oracle.OracleParams(shape=(1, H, 1), q=q, collision=coll, omega=omega, magic_lambda=lam, force=F,
                               periodic=(1, 0, 1), face_kind=(1, 1, oracle.NOSLIP, top, 1, 1),
                               face_u=tuple(fu), face_rho=(1.0,) * 6)


def _run_to_steady(p, f, width):
    """Run until the slowest diffusive mode exp(-nu (pi/width)^2 t) has decayed by e^-40."""
    nu = (1.0 / p.omega - 0.5) / 3.0
    return oracle.run(p, f, int(40.0 / (nu * (math.pi / width) ** 2)) + 1)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("omega", [1.0, 1.6, 0.7])
def test_poiseuille_exact_trt_magic(q, omega):
    """TRT, Lambda = 3/16, halfway bounce-back: u(y) = F/(2 nu) (y + 1/2)(H - 1/2 - y) exactly,
    for any omega+ and any amplitude (the nonlinear equilibrium terms cancel in a
    unidirectional flow); density stays 1 up to accumulated rounding."""
    H = 12
    nu = (1 / omega - 0.5) / 3
    y = np.arange(H)
    for F in (5e-5, 2e-4):
        p = _channel(H, q, oracle.TRT, omega, F=(F, 0.0, 0.0))
        rho, u = inputs.rest((1, H, 1))
        f = _run_to_steady(p, oracle.init(p, rho, u), H)
        r, v = oracle.macroscopic(p, f)
        # uniform density; its mean drifts only by accumulated rounding (~1e-16 per step),
        # and the steady profile is F / (2 rho nu) (...) for that density
        assert r.max() - r.min() < 1e-13
        assert abs(r.mean() - 1.0) < 1e-11
        want = F / (2 * nu * r.mean()) * (y + 0.5) * (H - 0.5 - y)
        assert _rel(v[0, 0, :, 0], want) < 1e-12
        assert np.abs(v[1:]).max() < 1e-12 * want.max()


def _startup_series(H, F, nu, t, nmax=2001):
    """Plane Poiseuille flow driven from rest by a constant body force F (rho = 1) between
    walls at eta = 0 and eta = H, eta = y + 1/2: the steady parabola minus the decaying odd sine
    modes of its Fourier series (the solution of u_t = nu u_yy + F, u = 0 at the walls)."""
    eta = np.arange(H) + 0.5
    u = F / (2 * nu) * eta * (H - eta)
    for n in range(1, nmax, 2):
        u -= 4 * F * H * H / (nu * math.pi ** 3 * n ** 3) * np.sin(n * math.pi * eta / H) * math.exp(
            -nu * (n * math.pi / H) ** 2 * t)
    return u


@pytest.mark.parametrize("H,steps,tau,tol", [(256, 10000, 1.0, 2e-5), (64, 1000, 0.8, 2e-4)])
def test_channel_startup_follows_the_series(H, steps, tau, tol):
    """The C2 channel from rest (TRT Lambda = 3/16, halfway no-slip walls at y = -1/2 and H - 1/2,
    x/z-invariant, so one 1 x H x 1 column), after `steps` steps, against the start-up series of
    plane Poiseuille flow.  At the full C2 size (H = 256, tau = 1, 10,000 steps: far from
    steady) the oracle is within 6e-6 of max u; the series taken half a step earlier or later,
    or a velocity without the half-force correction, is off by 5e-5."""
    F = 1e-6
    nu = (tau - 0.5) / 3.0
    p = oracle.OracleParams(shape=(1, H, 1), q=19, collision=oracle.TRT, omega=1 / tau, magic_lambda=3 / 16,
                            force=(F, 0.0, 0.0), periodic=(1, 0, 1),
                            face_kind=(1, 1, oracle.NOSLIP, oracle.NOSLIP, 1, 1))
    rho, u = inputs.rest((1, H, 1))
    f = oracle.run(p, oracle.init(p, rho, u), steps)
    v = oracle.macroscopic(p, f)[1][0, 0, :, 0]
    want = _startup_series(H, F, nu, steps)
    assert np.abs(v - want).max() <= tol * np.abs(want).max()


def test_poiseuille_srt_is_not_exact():
    """Negative control: SRT at tau = 1.9 has Lambda = 1.96 and a viscosity-dependent wall
    slip, so the same comparison must fail (shows the exact test has teeth)."""
    H, F, omega = 12, 1e-4, 1 / 1.9
    nu = (1 / omega - 0.5) / 3
    p = _channel(H, 19, oracle.SRT, omega, F=(F, 0.0, 0.0))
    rho, u = inputs.rest((1, H, 1))
    f = _run_to_steady(p, oracle.init(p, rho, u), H)
    v = oracle.macroscopic(p, f)[1]
    y = np.arange(H)
    want = F / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    assert _rel(v[0, 0, :, 0], want) > 1e-3


@pytest.mark.parametrize("q,coll", [(19, oracle.SRT), (19, oracle.TRT), (27, oracle.TRT)])
def test_couette_exact(q, coll):
    """Bottom wall at rest, top wall moving with u_w (velocity bounce-back), no force:
    u_x(y) = u_w (y + 1/2) / H exactly."""
    H, uw = 10, 0.01
    p = _channel(H, q, coll, 1.25, top=oracle.VELOCITY, uw=(uw, 0.0, 0.0))
    rho, u = inputs.rest((1, H, 1))
    f = _run_to_steady(p, oracle.init(p, rho, u), 2 * H)
    v = oracle.macroscopic(p, f)[1]
    y = np.arange(H)
    assert _rel(v[0, 0, :, 0], uw * (y + 0.5) / H) < 1e-12


def test_pressure_rest_state_is_fixed_point():
    shape = (6, 5, 1)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1.1, periodic=(0, 0, 1),
                            face_kind=(oracle.PRESSURE, oracle.PRESSURE, 1, 1, 1, 1), face_rho=(1.02,) * 6)
    rho, u = inputs.rest(shape, rho0=1.02)
    f = oracle.init(p, rho, u)
    g = oracle.run(p, f, 20)
    np.testing.assert_allclose(g, f, rtol=0, atol=1e-16)


def test_pressure_uniform_flow_is_fixed_point():
    """A uniform flow at the wall density through two pressure faces is an exact fixed point:
    anti-bounce-back returns feq_opp(rho_w, u_b) when f* = feq(rho_w, u_b).  Pins the sign,
    the factor 2 and both quadratic coefficients of the pressure rule."""
    shape = (5, 3, 2)
    for q in (19, 27):
        p = oracle.OracleParams(shape=shape, q=q, collision=oracle.TRT, omega=0.9, periodic=(0, 1, 1),
                                face_kind=(oracle.PRESSURE, oracle.PRESSURE, 1, 1, 1, 1), face_rho=(1.0,) * 6)
        rho = np.ones(shape[::-1])
        u = np.zeros((3,) + shape[::-1])
        u[0], u[1], u[2] = 0.05, 0.02, -0.01
        f = oracle.init(p, rho, u)
        g = oracle.run(p, f, 15)
        np.testing.assert_allclose(g, f, rtol=0, atol=1e-15)


def test_pressure_driven_channel_flow():
    """Pressure anti-bounce-back at x-/x+ (rho_in > rho_out), no-slip walls in y.  Without
    extrapolation of u_b the rule leaves an O(shear) density jump at the faces, so the
    interior gradient is ~4-8 % above (rho_in - rho_out)/L; the density is linear inside and
    the centreline velocity matches Poiseuille for the measured interior gradient (2 %)."""
    L, H = 48, 9
    r_in, r_out, omega = 1.003, 0.997, 1.2
    nu = (1 / omega - 0.5) / 3
    p = oracle.OracleParams(shape=(L, H, 1), q=19, collision=oracle.TRT, omega=omega, periodic=(0, 0, 1),
                            face_kind=(oracle.PRESSURE, oracle.PRESSURE, 1, 1, 1, 1),
                            face_rho=(r_in, r_out, 1, 1, 1, 1))
    rho, u = inputs.rest((L, H, 1))
    f = _run_to_steady(p, oracle.init(p, rho, u), H)
    r, v = oracle.macroscopic(p, f)
    prof = r[0, H // 2, :]
    x = np.arange(L)
    fit = np.polyfit(x[2:-2], prof[2:-2], 1)
    assert np.abs(np.polyval(fit, x[2:-2]) - prof[2:-2]).max() < 0.01 * (r_in - r_out)
    nominal = (r_in - r_out) / L
    assert 1.0 < -fit[0] / nominal < 1.1
    umax = -fit[0] / 3.0 / (2 * nu) * (H / 2) ** 2
    mid = v[0, 0, H // 2, L // 2]
    assert abs(mid / umax - 1) < 0.02, (mid, umax)


@pytest.mark.parametrize("q,coll", [(19, oracle.TRT), (27, oracle.SRT)])
def test_conservation_periodic_with_force(q, coll):
    shape = (6, 5, 4)
    F = np.array([3e-5, 0.0, -1e-5])
    p = oracle.OracleParams(shape=shape, q=q, collision=coll, omega=1.4, force=tuple(F))
    rho, u = inputs.random_state(shape, seed=5)
    f = oracle.init(p, rho, u)
    d0 = oracle.diagnostics(p, f)
    n = 50
    g = oracle.run(p, f, n)
    d1 = oracle.diagnostics(p, g)
    N = np.prod(shape)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    np.testing.assert_allclose(np.array(d1["momentum"]) - np.array(d0["momentum"]), n * N * F, rtol=1e-11, atol=1e-13)


def test_noslip_conserves_mass_with_obstacle():
    shape = (7, 6, 5)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1.5, periodic=(1, 0, 0),
                            face_kind=(1, 1, 1, 1, 1, 1), force=(1e-4, 0, 0))
    flags = np.zeros(shape[::-1], dtype=np.uint8)
    flags[2, 2:4, 3:5] = oracle.NOSLIP
    rho, u = inputs.random_state(shape, seed=6)
    f = oracle.init(p, rho, u, flags=flags)
    m0 = oracle.diagnostics(p, f, flags)["mass"]
    g = oracle.run(p, f, 60, flags=flags)
    assert abs(oracle.diagnostics(p, g, flags)["mass"] - m0) <= 1e-13 * m0
