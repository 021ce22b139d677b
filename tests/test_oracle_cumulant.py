"""Pins for the oracle's cumulant collision (Sec. 5.1.1 of the paper: cumulants instead of
moments relaxed towards their equilibria, after Geier et al. 2015), D3Q27, CPU only.

What fixes the result, independently of the oracle's own set-partition table and its per-axis
back-transform:
  * the definition of a cumulant: the Taylor coefficients of the logarithm of the discrete
    Laplace transform sum_i f_i exp(xi . c_i), computed here by truncated power-series
    arithmetic (no moment-cumulant formula), both for the oracle's forward map and, through
    the post-collision populations, for its inverse;
  * the tensor-product structure of D3Q27: with every cumulant of order >= 3 at zero and the
    second-order ones at rho/3, the populations are the product of three one-dimensional
    distributions on {-1, 0, 1} with mean u_a and variance 1/3, a closed form; it is the
    collision's output when every rate is 1 and a fixed point for any rates;
  * rates 0 give the identity;
  * conservation of mass and the momentum gain of exactly F, for any rates;
  * with a body force and equal shear and bulk rates, the second moments after the collision
    are those of the Guo scheme, Pi* = Pi - w (Pi - rho (I/3 + u u)) + (1 - w/2)(u F + F u);
  * physics: a shear wave decays at nu k^2 with nu = (1/w - 1/2)/3, and a uniform flow keeps
    its density and velocity and relaxes to the product equilibrium.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

GROUPS = {
    # group -> list of combinations, each a dict {(a, b, c): coefficient} of cumulants C_abc
    1: [{(1, 1, 0): 1}, {(1, 0, 1): 1}, {(0, 1, 1): 1}, {(2, 0, 0): 1, (0, 2, 0): -1}, {(2, 0, 0): 1, (0, 0, 2): -1}],
    2: [{(2, 0, 0): 1, (0, 2, 0): 1, (0, 0, 2): 1}],
    3: [{(1, 2, 0): 1, (1, 0, 2): 1}, {(2, 1, 0): 1, (0, 1, 2): 1}, {(2, 0, 1): 1, (0, 2, 1): 1}],
    4: [{(1, 2, 0): 1, (1, 0, 2): -1}, {(2, 1, 0): 1, (0, 1, 2): -1}, {(2, 0, 1): 1, (0, 2, 1): -1}],
    5: [{(1, 1, 1): 1}],
    6: [{(2, 2, 0): 1, (2, 0, 2): -2, (0, 2, 2): 1}, {(2, 2, 0): 1, (2, 0, 2): 1, (0, 2, 2): -2}],
    7: [{(2, 2, 0): 1, (2, 0, 2): 1, (0, 2, 2): 1}],
    8: [{(2, 1, 1): 1}, {(1, 2, 1): 1}, {(1, 1, 2): 1}],
    9: [{(2, 2, 1): 1}, {(2, 1, 2): 1}, {(1, 2, 2): 1}],
    10: [{(2, 2, 2): 1}],
}


def _lattice():
    c, w, _ = oracle.lattice(27)
    return c, w


def _cells(n, seed, amp=0.1, drift=0.05):
    rng = np.random.default_rng(seed)
    c, w = _lattice()
    out = []
    for _ in range(n):
        u = drift * rng.uniform(-1, 1, 3)
        f = w * (1.0 + 3 * c @ u) * (1.0 + amp * rng.standard_normal(27))
        out.append(f)
    return out


def _params(omega, cum_s, F=(0.0, 0.0, 0.0)):
    return oracle.OracleParams(shape=(1, 1, 1), q=27, collision=oracle.CUMULANT, omega=omega, cum_s=tuple(cum_s),
                               force=F)


# ---- the definition: cumulants as Taylor coefficients of log sum_i f_i exp(xi . c_i) ----

def _series_mul(A, B):
    """Product of two power series in (x, y, z) truncated at degree 2 in each variable
    (arrays [a, b, c] of coefficients of x^a y^b z^c).  A coefficient of degree (a, b, c) of a
    product only involves factors of degree <= (a, b, c), so the truncation is exact."""
    out = np.zeros((3, 3, 3))
    for a1, b1, c1 in itertools.product(range(3), repeat=3):
        if A[a1, b1, c1] == 0.0:
            continue
        for a2, b2, c2 in itertools.product(range(3 - a1), range(3 - b1), range(3 - c1)):
            out[a1 + a2, b1 + b2, c1 + c2] += A[a1, b1, c1] * B[a2, b2, c2]
    return out


def series_cumulants(f):
    """Density-scaled cumulants rho * k_abc of the populations f (a, b, c <= 2): the
    coefficients of log M(xi) times a! b! c!, with M(xi) = sum_i f_i exp(xi . c_i)."""
    c, _ = _lattice()
    M = np.zeros((3, 3, 3))
    for i in range(27):
        e = [np.array([1.0, c[i, a], c[i, a] ** 2 / 2.0]) for a in range(3)]
        M += f[i] * np.einsum("a,b,c->abc", *e)
    rho = M[0, 0, 0]
    X = M / rho
    X[0, 0, 0] = 0.0
    # log(1 + X) = sum_k (-1)^(k+1) X^k / k; X^k vanishes beyond total degree 6
    logM = np.zeros((3, 3, 3))
    P = X.copy()
    for k in range(1, 7):
        logM += (-1) ** (k + 1) * P / k
        P = _series_mul(P, X)
    fact = np.array([1.0, 1.0, 2.0])
    k_abc = logM * fact[:, None, None] * fact[None, :, None] * fact[None, None, :]
    return rho * k_abc, rho


def _oracle_C(f, F=(0.0, 0.0, 0.0)):
    """The oracle's cumulants as [a, b, c]."""
    C, rho, u = oracle.cumulants(_params(1.0, (1.0,) * 9, F), f)
    return np.transpose(C, (2, 1, 0)), rho, u


def _combo(C, combo):
    return sum(v * C[k] for k, v in combo.items())


def test_forward_cumulants_match_the_log_series():
    for f in _cells(12, seed=1):
        want, rho = series_cumulants(f)
        got, rho_o, _ = _oracle_C(f)
        for a, b, c in itertools.product(range(3), repeat=3):
            if a + b + c >= 2:
                assert abs(got[a, b, c] - want[a, b, c]) <= 1e-14 * rho, (a, b, c)


def test_back_transform_round_trip():
    for f in _cells(8, seed=2):
        C, rho, u = oracle.cumulants(_params(1.0, (1.0,) * 9, (1e-3, -2e-3, 5e-4)), f)
        back = oracle.cumulants_to_f(rho, u, C)
        assert np.abs(back - f).max() <= 1e-15


def test_each_group_relaxes_alone():
    """One group at rate 1, every other rate 0: that group's combinations reach their
    equilibrium (rho for the bulk trace, 0 otherwise) and every other combination, and every
    moment of order <= 1, is unchanged -- measured by the log-series cumulants of f*."""
    for g in range(1, 11):
        rates = [0.0] * 10
        rates[g - 1] = 1.0
        p = _params(rates[0], rates[1:])
        for f in _cells(3, seed=10 + g):
            before, rho = series_cumulants(f)
            after, rho2 = series_cumulants(oracle.collide_cell(p, f))
            assert abs(rho2 - rho) <= 1e-15
            for h, combos in GROUPS.items():
                for cb in combos:
                    x0, x1 = _combo(before, cb), _combo(after, cb)
                    if h == g:
                        eq = rho if h == 2 else 0.0
                        assert abs(x1 - eq) <= 3e-15, (g, cb)
                    else:
                        assert abs(x1 - x0) <= 3e-15, (g, h, cb)


def test_generic_rates_scale_each_combination():
    rng = np.random.default_rng(5)
    for trial in range(4):
        rates = rng.uniform(0.3, 1.9, 10)
        p = _params(rates[0], rates[1:])
        for f in _cells(3, seed=20 + trial):
            before, rho = series_cumulants(f)
            after, _ = series_cumulants(oracle.collide_cell(p, f))
            for h, combos in GROUPS.items():
                eq = rho if h == 2 else 0.0
                for cb in combos:
                    want = (1.0 - rates[h - 1]) * (_combo(before, cb) - eq) + eq
                    assert abs(_combo(after, cb) - want) <= 5e-15, (h, cb)


def product_equilibrium(rho, u):
    """rho prod_a p(c_a; u_a) with p(0) = 2/3 - u^2, p(+-1) = (1/3 + u^2 +- u)/2."""
    c, _ = _lattice()
    def p1(ca, ua):
        return 2.0 / 3.0 - ua * ua if ca == 0 else 0.5 * (1.0 / 3.0 + ua * ua + ca * ua)
    return np.array([rho * p1(c[i, 0], u[0]) * p1(c[i, 1], u[1]) * p1(c[i, 2], u[2]) for i in range(27)])


def test_all_rates_one_give_the_product_equilibrium():
    c, _ = _lattice()
    for f in _cells(8, seed=3):
        rho = f.sum()
        u = c.T @ f / rho
        got = oracle.collide_cell(_params(1.0, (1.0,) * 9), f)
        assert np.abs(got - product_equilibrium(rho, u)).max() <= 2e-16 * 4


def test_product_equilibrium_is_a_fixed_point_for_any_rates():
    rng = np.random.default_rng(7)
    for _ in range(6):
        rho = 1.0 + 0.05 * rng.standard_normal()
        u = 0.08 * rng.uniform(-1, 1, 3)
        feq = product_equilibrium(rho, u)
        rates = rng.uniform(0.2, 1.95, 10)
        got = oracle.collide_cell(_params(rates[0], rates[1:]), feq)
        assert np.abs(got - feq).max() <= 1e-15


def test_rates_zero_are_the_identity():
    for f in _cells(6, seed=4):
        got = oracle.collide_cell(_params(0.0, (0.0,) * 9), f)
        assert np.abs(got - f).max() <= 1e-15


def test_mass_and_momentum_with_force():
    c, _ = _lattice()
    rng = np.random.default_rng(8)
    F = (2e-4, -1e-4, 3e-4)
    for f in _cells(6, seed=6):
        rates = rng.uniform(0.2, 1.95, 10)
        got = oracle.collide_cell(_params(rates[0], rates[1:], F), f)
        assert abs(got.sum() - f.sum()) <= 2e-15
        assert np.abs(c.T @ got - (c.T @ f + np.array(F))).max() <= 2e-15


def test_second_moments_follow_the_guo_scheme():
    """Equal shear and bulk rates w: Pi* = Pi - w (Pi - rho (I/3 + u u)) + (1 - w/2)(u F + F u)
    with u = (j + F/2)/rho, whatever the higher-order rates."""
    c, _ = _lattice()
    rng = np.random.default_rng(9)
    F = np.array([3e-4, -2e-4, 1e-4])
    for f in _cells(6, seed=30, amp=0.05):
        w = rng.uniform(0.4, 1.9)
        others = rng.uniform(0.2, 1.95, 8)
        got = oracle.collide_cell(_params(w, (w,) + tuple(others), tuple(F)), f)
        rho = f.sum()
        u = (c.T @ f + 0.5 * F) / rho
        Pi = np.einsum("i,ia,ib->ab", f, c, c)
        want = Pi - w * (Pi - rho * (np.eye(3) / 3.0 + np.outer(u, u))) + (1 - w / 2) * (np.outer(u, F) + np.outer(F, u))
        Pis = np.einsum("i,ia,ib->ab", got, c, c)
        assert np.abs(Pis - want).max() <= 1e-15


def test_uniform_flow_keeps_its_moments_and_relaxes_to_the_product_equilibrium():
    """A uniform state streams onto itself, so the step is the collision alone: density and
    velocity stay, and the populations approach the product equilibrium (the polynomial
    equilibrium of the initial state is not a fixed point of the cumulant collision)."""
    shape = (4, 4, 4)
    rng = np.random.default_rng(11)
    rates = rng.uniform(0.5, 1.5, 10)
    p = oracle.OracleParams(shape=shape, q=27, collision=oracle.CUMULANT, omega=rates[0], cum_s=tuple(rates[1:]),
                            periodic=(1, 1, 1))
    u0 = np.array([0.03, -0.02, 0.01])
    rho = np.full(shape[::-1], 1.02)
    u = np.broadcast_to(u0[:, None, None, None], (3,) + shape[::-1])
    f0 = oracle.init(p, rho, u)
    f1 = oracle.run(p, f0, 120)
    r1, u1 = oracle.macroscopic(p, f1)
    assert np.abs(r1 - 1.02).max() <= 1e-14
    assert np.abs(u1 - u).max() <= 1e-14
    assert np.abs(f1 - f1[:, :1, :1, :1]).max() == 0.0
    assert np.abs(f1[:, 0, 0, 0] - product_equilibrium(1.02, u0)).max() <= 1e-14


@pytest.mark.parametrize("tau", [0.6, 0.9])
def test_shear_wave_decays_at_the_viscous_rate(tau):
    """u_x = A sin(2 pi y / N) on a periodic 4 x N x 4 box: the amplitude decays as
    exp(-nu k^2 t), nu = (tau - 1/2)/3 from the shear rate alone."""
    N = 48
    shape = (4, N, 4)
    omega = 1.0 / tau
    p = oracle.OracleParams(shape=shape, q=27, collision=oracle.CUMULANT, omega=omega,
                            cum_s=(1.0, 1.3, 1.1, 1.2, 1.0, 1.0, 1.4, 1.0, 1.0), periodic=(1, 1, 1))
    y = np.arange(N)
    k = 2 * math.pi / N
    A = 1e-3
    rho = np.ones(shape[::-1])
    u = np.zeros((3,) + shape[::-1])
    u[0] = A * np.sin(k * y)[None, :, None]
    f = oracle.init(p, rho, u)
    s = np.sin(k * y)
    steps = 300
    amp = []
    for t in (100, steps):
        g = oracle.run(p, f, t)
        _, uu = oracle.macroscopic(p, g)
        amp.append((uu[0].mean(axis=(0, 2)) * s).sum() / (s * s).sum())
    rate = math.log(amp[0] / amp[1]) / (steps - 100)
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1.0) < 2e-3
