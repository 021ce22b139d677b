"""Pins for the oracle's lattice and equilibrium (CPU only).

The lattice must satisfy the exact isotropy identities that make the method recover the
Navier-Stokes equations with c_s^2 = 1/3 (Sec. 5.1 names the stencils; the identities are
the mathematics), and must equal the hand-typed canonical tables in tests/golden/.
"""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

import oracle
from oracle import single_cell
from golden_tables import lattice_table


@pytest.mark.parametrize("q", [19, 27])
def test_lattice_matches_golden_table(q):
    c, w, opp = oracle.lattice(q)
    gc, gw = lattice_table(q)
    np.testing.assert_array_equal(c, gc)
    np.testing.assert_array_equal(w, np.array([float(x) for x in gw]))
    for i in range(q):
        np.testing.assert_array_equal(c[opp[i]], -c[i])


@pytest.mark.parametrize("q", [19, 27])
def test_lattice_exact_isotropy(q):
    """Exact rational check: sum w = 1, odd moments vanish, sum w c_a c_b = delta/3,
    sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9."""
    gc, gw = lattice_table(q)
    d = lambda a, b: 1 if a == b else 0  # noqa: E731
    assert sum(gw) == 1
    for a in range(3):
        assert sum(w * int(c[a]) for c, w in zip(gc, gw)) == 0
    for a, b in product(range(3), repeat=2):
        assert sum(w * int(c[a] * c[b]) for c, w in zip(gc, gw)) == Fraction(d(a, b), 3)
    for a, b, e in product(range(3), repeat=3):
        assert sum(w * int(c[a] * c[b] * c[e]) for c, w in zip(gc, gw)) == 0
    for a, b, e, g in product(range(3), repeat=4):
        want = Fraction(d(a, b) * d(e, g) + d(a, e) * d(b, g) + d(a, g) * d(b, e), 9)
        assert sum(w * int(c[a] * c[b] * c[e] * c[g]) for c, w in zip(gc, gw)) == want


@pytest.mark.parametrize("q", [19, 27])
def test_numpy_restatement_uses_same_lattice(q):
    c, w, _ = oracle.lattice(q)
    nc, nw = single_cell.velocity_set(q)
    np.testing.assert_array_equal(c, nc.astype(np.int64))
    np.testing.assert_allclose(w, nw, rtol=0, atol=1e-17)


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_moments(q):
    """sum feq = rho, sum c feq = rho u, sum c c feq = rho/3 I + rho u u (2nd-order equilibrium)."""
    c, _, _ = oracle.lattice(q)
    rng = np.random.default_rng(11)
    for _ in range(50):
        rho = 0.8 + 0.4 * rng.random()
        u = 0.1 * (2 * rng.random(3) - 1)
        feq = oracle.equilibrium(q, rho, u)
        assert abs(feq.sum() - rho) <= 4e-16 * rho
        np.testing.assert_allclose(c.T @ feq, rho * u, rtol=0, atol=4e-16)
        second = np.einsum("ia,ib,i->ab", c, c, feq)
        np.testing.assert_allclose(second, rho / 3 * np.eye(3) + rho * np.outer(u, u), rtol=0, atol=6e-16)


def test_equilibrium_at_rest_is_weights():
    for q in (19, 27):
        _, w, _ = oracle.lattice(q)
        np.testing.assert_array_equal(oracle.equilibrium(q, 1.0, np.zeros(3)), w)
