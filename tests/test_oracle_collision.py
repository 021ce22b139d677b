"""Pins for the oracle's single-cell collision (CPU only).

What the method fixes (Sec. 5.1, Eq. 1-3, SRT/TRT as special cases of Eq. 3, Guo forcing):
  * the equilibrium is a fixed point of the collision without force;
  * the collision conserves mass exactly and adds exactly F to the momentum;
  * TRT with omega- = omega+ is SRT;
  * an independent NumPy restatement agrees on random cells.
"""
import numpy as np
import pytest

import oracle
from oracle import single_cell

VARIANTS = [(q, coll) for q in (19, 27) for coll in (oracle.SRT, oracle.TRT)]


def _params(q, coll, omega, force=(0.0, 0.0, 0.0), lam=3 / 16):
    return oracle.OracleParams(shape=(1, 1, 1), q=q, collision=coll, omega=omega, magic_lambda=lam, force=force)


def _random_cell(rng, q, rho_amp=0.1, u_amp=0.08, noneq=0.02):
    rho = 1.0 + rho_amp * (2 * rng.random() - 1)
    u = u_amp * (2 * rng.random(3) - 1)
    feq = oracle.equilibrium(q, rho, u)
    return feq * (1.0 + noneq * (2 * rng.random(q) - 1))


@pytest.mark.parametrize("q,coll", VARIANTS)
def test_equilibrium_is_fixed_point(q, coll):
    rng = np.random.default_rng(1)
    for omega in (0.3, 1.0, 1.6, 1.95):
        p = _params(q, coll, omega)
        for _ in range(20):
            rho = 0.9 + 0.2 * rng.random()
            u = 0.1 * (2 * rng.random(3) - 1)
            feq = oracle.equilibrium(q, rho, u)
            np.testing.assert_allclose(oracle.collide_cell(p, feq), feq, rtol=0, atol=1e-15)


@pytest.mark.parametrize("q,coll", VARIANTS)
def test_mass_exact_and_momentum_gains_force(q, coll):
    c, _, _ = oracle.lattice(q)
    rng = np.random.default_rng(2)
    for omega in (0.5, 1.0, 1.7):
        F = 1e-3 * (2 * rng.random(3) - 1)
        p = _params(q, coll, omega, force=F)
        for _ in range(30):
            f = _random_cell(rng, q)
            fs = oracle.collide_cell(p, f)
            assert abs(fs.sum() - f.sum()) <= 1e-15
            np.testing.assert_allclose(c.T @ fs - c.T @ f, F, rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", [19, 27])
def test_trt_with_equal_rates_is_srt(q):
    rng = np.random.default_rng(3)
    for omega in (0.6, 1.0, 1.8):
        lam = (1 / omega - 0.5) ** 2  # makes omega- equal omega+
        assert abs(oracle.omega_minus(omega, lam) - omega) < 1e-15
        F = 1e-4 * (2 * rng.random(3) - 1)
        ps = _params(q, oracle.SRT, omega, force=F)
        pt = _params(q, oracle.TRT, omega, force=F, lam=lam)
        for _ in range(20):
            f = _random_cell(rng, q)
            np.testing.assert_allclose(oracle.collide_cell(pt, f), oracle.collide_cell(ps, f), rtol=0, atol=1e-15)


@pytest.mark.parametrize("q,coll", VARIANTS)
def test_matches_numpy_restatement(q, coll):
    rng = np.random.default_rng(4)
    name = "srt" if coll == oracle.SRT else "trt"
    for k in range(100):
        omega = 0.2 + 1.75 * rng.random()
        lam = 0.05 + 0.5 * rng.random()
        F = 1e-3 * (2 * rng.random(3) - 1)
        p = _params(q, coll, omega, force=F, lam=lam)
        f = _random_cell(rng, q)
        want = single_cell.collide(f, q, name, omega, lam, F)
        np.testing.assert_allclose(oracle.collide_cell(p, f), want, rtol=0, atol=2e-15)


def test_omega_minus_definition():
    # Lambda = (1/w+ - 1/2)(1/w- - 1/2): w+ = 1 (tau = 1), Lambda = 3/16 -> 1/w- = 3/8 + 1/2
    assert abs(oracle.omega_minus(1.0, 3 / 16) - 1 / 0.875) < 1e-15
    for wp in (0.4, 1.2, 1.9):
        for lam in (1 / 12, 3 / 16, 1 / 4):
            wm = oracle.omega_minus(wp, lam)
            assert abs((1 / wp - 0.5) * (1 / wm - 0.5) - lam) < 1e-15


@pytest.mark.parametrize("q,coll", VARIANTS)
def test_relaxation_of_shear_stress(q, coll):
    """The traceless second moment of f - feq (the shear stress) relaxes by (1 - omega+)
    per collision without force: the even part carries the stress and relaxes with omega+."""
    c, _, _ = oracle.lattice(q)
    rng = np.random.default_rng(5)
    for omega in (0.7, 1.3):
        p = _params(q, coll, omega, lam=0.1)
        for _ in range(10):
            f = _random_cell(rng, q)
            rho = f.sum()
            u = c.T @ f / rho
            feq = oracle.equilibrium(q, rho, u)
            fs = oracle.collide_cell(p, f)
            pi_in = np.einsum("ia,ib,i->ab", c, c, f - feq)
            pi_out = np.einsum("ia,ib,i->ab", c, c, fs - feq)
            np.testing.assert_allclose(pi_out, (1 - omega) * pi_in, rtol=0, atol=1e-15)
