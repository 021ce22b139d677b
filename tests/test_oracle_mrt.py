"""Pins for the oracle's MRT collision (Eq. 3 of the paper: Omega = -M^-1 S (M f - m_eq) with a
stated moment matrix M and one relaxation rate per group of moments), CPU only.

What fixes the result, independently of the oracle's own Gram-Schmidt and Gauss-Jordan code:
  * linear algebra: M M^-1 = I, the rows are orthogonal under the weighted product, the group
    sizes are the dimensions of the degree classes on each lattice;
  * the equilibrium and the Guo source are polynomials of degree <= 2 in c times w, so every
    moment of degree >= 3 (orthogonal to all quadratics) vanishes for them;
  * the paper's statement that SRT and TRT are special choices of S: all rates equal gives the
    (separately pinned) SRT oracle, even groups at omega+ and odd groups at omega- the TRT one;
  * the momentum rate is irrelevant under Guo forcing (the half-force shift and the source's
    (1 - s/2) factor cancel for any s): changing it changes nothing;
  * conservation of mass and the momentum gain of exactly F for any rates; the equilibrium is
    a fixed point for any rates;
  * the physics of the rates: the deviatoric non-equilibrium stress relaxes by (1 - s_shear),
    its trace by (1 - s_bulk);
  * a NumPy restatement through Householder QR projectors (oracle/single_cell.py), a different
    route to the same group subspaces;
  * plane Poiseuille flow with halfway bounce-back at Lambda = 3/16 between the shear and the
    third-order rates is exact for any fourth-, fifth- and sixth-order rate, and (negative
    control) not exact once the bulk rate differs from the shear rate.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import single_cell
from paper_1909_13772_gb300 import inputs

GROUP_SIZES = {19: [1, 3, 5, 1, 6, 3], 27: [1, 3, 5, 1, 7, 6, 3, 1]}


def _cells(q, n, seed, amp=0.1):
    rng = np.random.default_rng(seed)
    _, w, _ = oracle.lattice(q)
    return [w * (1.0 + amp * rng.standard_normal(q)) for _ in range(n)]


def _rates(q, rng):
    return tuple(rng.uniform(0.2, 1.95, 7))


def _collide(q, rates, f, F=(0.0, 0.0, 0.0)):
    p = oracle.OracleParams(shape=(1, 1, 1), q=q, collision=oracle.MRT, mrt_s=rates, force=F)
    return oracle.collide_cell(p, f)


@pytest.mark.parametrize("q", [19, 27])
def test_moment_matrix_structure(q):
    M, Mi, g = oracle.mrt_matrix(q)
    _, w, _ = oracle.lattice(q)
    assert np.abs(M @ Mi - np.eye(q)).max() < 1e-13
    assert np.abs(Mi @ M - np.eye(q)).max() < 1e-13
    G = (M * w) @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-15
    assert np.bincount(g).tolist() == GROUP_SIZES[q]
    # rows of degree >= 3 are orthogonal to every polynomial of degree <= 2 in c
    c, _, _ = oracle.lattice(q)
    quad = [np.ones(q)] + [c[:, a].astype(float) for a in range(3)]
    quad += [(c[:, a] * c[:, b]).astype(float) for a, b in itertools.combinations_with_replacement(range(3), 2)]
    for k in np.flatnonzero(g >= 4):
        for pq in quad:
            assert abs((w * M[k] * pq).sum()) < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_higher_moments_of_equilibrium_and_source_vanish(q):
    M, _, g = oracle.mrt_matrix(q)
    c, w, _ = oracle.lattice(q)
    rng = np.random.default_rng(4)
    for _ in range(20):
        rho, u, F = 1 + 0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(3), 1e-3 * rng.standard_normal(3)
        feq = oracle.equilibrium(q, rho, u)
        cu = c @ u
        S = w * ((3 * (c - u) + 9 * cu[:, None] * c) @ F)
        assert np.abs((M @ feq)[g >= 4]).max() < 1e-15
        assert np.abs((M @ S)[g >= 4]).max() < 1e-17


@pytest.mark.parametrize("q", [19, 27])
def test_all_rates_equal_is_srt(q):
    rng = np.random.default_rng(5)
    for f in _cells(q, 50, 6):
        om, F = rng.uniform(0.3, 1.9), tuple(1e-3 * rng.standard_normal(3))
        a = _collide(q, (om,) * 7, f, F)
        b = oracle.collide_cell(oracle.OracleParams(shape=(1, 1, 1), q=q, collision=oracle.SRT, omega=om,
                                                    force=F), f)
        assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max()


@pytest.mark.parametrize("q", [19, 27])
def test_parity_rates_are_trt(q):
    rng = np.random.default_rng(7)
    for f in _cells(q, 50, 8):
        om, lam, F = rng.uniform(0.3, 1.9), rng.uniform(0.05, 1.0), tuple(1e-3 * rng.standard_normal(3))
        a = _collide(q, oracle.mrt_rates(q, om, lam), f, F)
        b = oracle.collide_cell(oracle.OracleParams(shape=(1, 1, 1), q=q, collision=oracle.TRT, omega=om,
                                                    magic_lambda=lam, force=F), f)
        assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max()


@pytest.mark.parametrize("q", [19, 27])
def test_momentum_rate_is_irrelevant_under_guo_forcing(q):
    rng = np.random.default_rng(9)
    for f in _cells(q, 30, 10):
        r = list(_rates(q, rng))
        F = tuple(1e-3 * rng.standard_normal(3))
        a = _collide(q, tuple(r), f, F)
        r[0] = rng.uniform(0.2, 1.95)
        b = _collide(q, tuple(r), f, F)
        assert np.abs(a - b).max() <= 2e-16 * np.abs(a).max()


@pytest.mark.parametrize("q", [19, 27])
def test_conservation_and_fixed_point_for_any_rates(q):
    c, w, _ = oracle.lattice(q)
    rng = np.random.default_rng(11)
    for f in _cells(q, 30, 12):
        r, F = _rates(q, rng), 1e-3 * rng.standard_normal(3)
        g = _collide(q, r, f, tuple(F))
        assert abs(g.sum() - f.sum()) < 1e-15
        assert np.abs(c.T @ g - (c.T @ f + F)).max() < 1e-16
        rho, u = 1 + 0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(3)
        feq = oracle.equilibrium(q, rho, u)
        assert np.abs(_collide(q, r, feq) - feq).max() <= 4 * np.finfo(float).eps * np.abs(feq).max()


def _stress_neq(c, f):
    rho = f.sum()
    u = c.T @ f / rho
    return np.einsum("ia,ib,i->ab", c, c, f) - rho * (np.eye(3) / 3 + np.outer(u, u))


@pytest.mark.parametrize("q", [19, 27])
def test_shear_and_bulk_stress_relax_with_their_rates(q):
    """F = 0: the collision keeps rho and u, and maps the non-equilibrium stress Pi to
    (1 - s_shear) dev(Pi) + (1 - s_bulk) tr(Pi) I / 3, whatever the other rates are."""
    c, _, _ = oracle.lattice(q)
    c = c.astype(np.float64)
    rng = np.random.default_rng(13)
    for f in _cells(q, 30, 14):
        r = _rates(q, rng)
        g = _collide(q, r, f)
        P0, P1 = _stress_neq(c, f), _stress_neq(c, g)
        tr0, tr1 = np.trace(P0), np.trace(P1)
        dev0, dev1 = P0 - tr0 * np.eye(3) / 3, P1 - tr1 * np.eye(3) / 3
        assert np.abs(dev1 - (1 - r[1]) * dev0).max() < 1e-15
        assert abs(tr1 - (1 - r[2]) * tr0) < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_qr_restatement_agrees(q):
    rng = np.random.default_rng(15)
    for f in _cells(q, 50, 16):
        r, F = _rates(q, rng), tuple(1e-3 * rng.standard_normal(3))
        a = _collide(q, r, f, F)
        b = single_cell.collide_mrt(f, q, r, F)
        assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def _channel(H, q, rates, F):
    return oracle.OracleParams(shape=(1, H, 1), q=q, collision=oracle.MRT, force=F, periodic=(1, 0, 1),
                               face_kind=(1, 1, oracle.NOSLIP, oracle.NOSLIP, 1, 1), mrt_s=rates)


def _poiseuille_error(q, omega, F=2e-4, H=12, **extra):
    nu = (1 / omega - 0.5) / 3
    p = _channel(H, q, oracle.mrt_rates(q, omega, 3 / 16, **extra), (F, 0.0, 0.0))
    rho, u = inputs.rest((1, H, 1))
    f = oracle.run(p, oracle.init(p, rho, u), int(40.0 / (nu * (math.pi / H) ** 2)) + 1)
    r, v = oracle.macroscopic(p, f)
    y = np.arange(H)
    want = F / (2 * nu * r.mean()) * (y + 0.5) * (H - 0.5 - y)
    return np.abs(v[0, 0, :, 0] - want).max() / want.max(), r.max() - r.min()


@pytest.mark.parametrize("q,omega,extra", [
    (19, 1.6, dict(fourth=0.9)),
    (19, 0.7, dict(fourth=1.7)),
    (27, 1.0, dict(fourth=0.9, fifth=1.1, sixth=0.8)),
    (27, 1.6, dict(fourth=1.3, fifth=0.6, sixth=1.9)),
])
def test_poiseuille_exact_at_the_magic_combination(q, omega, extra):
    err, drho = _poiseuille_error(q, omega, **extra)
    assert err < 1e-12 and drho < 1e-13


@pytest.mark.parametrize("q", [19, 27])
def test_poiseuille_not_exact_with_a_different_bulk_rate(q):
    """Negative control: the bulk rate couples to the normal stresses at the walls, so the
    same comparison fails once it differs from the shear rate."""
    err, drho = _poiseuille_error(q, 1.6, bulk=1.2)
    assert err > 1e-6 and drho > 1e-6


@pytest.mark.parametrize("q", [19, 27])
def test_periodic_run_conserves_mass_and_gains_momentum(q):
    shape = (5, 4, 3)
    rng = np.random.default_rng(17)
    F = (2e-5, -1e-5, 5e-6)
    p = oracle.OracleParams(shape=shape, q=q, collision=oracle.MRT, force=F, mrt_s=_rates(q, rng))
    rho, u = inputs.random_state(shape, seed=3, rho_amp=0.02, u_amp=0.03)
    f0 = oracle.init(p, rho, u)
    d0 = oracle.diagnostics(p, f0)
    steps = 20
    d1 = oracle.diagnostics(p, oracle.run(p, f0, steps))
    n = np.prod(shape)
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-14
    for a in range(3):
        assert abs(d1["momentum"][a] - d0["momentum"][a] - steps * n * F[a]) < 1e-13
