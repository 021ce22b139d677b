"""Pins for the locally varying relaxation of the oracle (CPU only): Smagorinsky and the
learned-closure network (Sec. 5.1.1: relaxation rates varied per cell from a local fluid
property; turbulence models after Yu et al. 2005, cited there)."""
import numpy as np
import pytest

import oracle
from oracle import mlp, single_cell


def _params(q=19, omega=1 / 0.51):
    return oracle.OracleParams(shape=(1, 1, 1), q=q, collision=oracle.TRT, omega=omega, magic_lambda=3 / 16)


def _cells(q, n, seed, noneq=0.02):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        rho = 1.0 + 0.05 * (2 * rng.random() - 1)
        u = 0.06 * (2 * rng.random(3) - 1)
        out.append(oracle.equilibrium(q, rho, u) * (1 + noneq * (2 * rng.random(q) - 1)))
    return out


def _pi_neq(q, f):
    """Non-equilibrium stress from the NumPy lattice (independent of the C oracle)."""
    c, _ = single_cell.velocity_set(q)
    rho = f.sum()
    u = c.T @ f / rho
    m = np.einsum("ia,ib,i->ab", c, c, f)
    return rho, m - rho * (np.eye(3) / 3 + np.outer(u, u))


@pytest.mark.parametrize("q", [19, 27])
def test_smagorinsky_solves_its_self_consistency(q):
    """(tau - tau0)/3 = cs^2 |S| with |S| = 3 sqrt(2 Pi:Pi) / (2 rho tau): the relaxation time
    the oracle returns must satisfy the eddy-viscosity equation it comes from."""
    p = _params(q)
    tau0 = 1 / p.omega
    for cs in (0.1, 0.17, 0.3):
        for f in _cells(q, 20, 1):
            om, _ = oracle.collide_closure(p, f, oracle.SMAGORINSKY, cs=cs)
            tau = 1 / om
            rho, pi = _pi_neq(q, f)
            smag = 3 * np.sqrt(2 * (pi * pi).sum()) / (2 * rho * tau)
            assert abs((tau - tau0) / 3 - cs * cs * smag) < 1e-13
            assert tau > tau0


@pytest.mark.parametrize("q", [19, 27])
def test_closures_reduce_to_trt(q):
    p = _params(q)
    off = mlp.init_params(seed=3, s_tau=0.0)  # s_tau = 0: the network cannot change tau
    for f in _cells(q, 10, 2):
        want = oracle.collide_cell(p, f)
        om, got = oracle.collide_closure(p, f, oracle.SMAGORINSKY, cs=0.0)
        assert om == p.omega
        np.testing.assert_array_equal(got, want)
        om, got = oracle.collide_closure(p, f, oracle.MLP, mlp=off)
        assert om == p.omega
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("kind", [oracle.SMAGORINSKY, oracle.MLP])
def test_closure_collision_conserves_mass_and_momentum(kind):
    p = _params(19)
    net = mlp.init_params(seed=4, s_rho=10.0, s_pi=200.0, s_tau=0.05)
    c, _, _ = oracle.lattice(19)
    for f in _cells(19, 20, 3):
        om, fs = oracle.collide_closure(p, f, kind, cs=0.17, mlp=net)
        assert abs(fs.sum() - f.sum()) < 1e-15
        np.testing.assert_allclose(c.T @ fs, c.T @ f, rtol=0, atol=1e-16)


def test_mlp_closure_tau_matches_numpy_network():
    """The C oracle's network (loops, BF16 rounding emulated by bit operations) against the
    NumPy restatement (matrix products, BF16 via a separate rounding routine)."""
    p = _params(19)
    net = mlp.init_params(seed=5, s_rho=10.0, s_pi=300.0, s_tau=0.05)
    sc = mlp.unpack(net)["scales"]
    for f in _cells(19, 30, 4, noneq=0.05):
        om, _ = oracle.collide_closure(p, f, oracle.MLP, mlp=net)
        rho, pi = _pi_neq(19, f)
        x = np.array([(rho - 1) * sc[0], pi[0, 0] * sc[1], pi[1, 1] * sc[1], pi[2, 2] * sc[1],
                      pi[0, 1] * sc[1], pi[0, 2] * sc[1], pi[1, 2] * sc[1]])
        tau = mlp.tau_of(net, x[None], 1 / p.omega)[0]
        assert abs(1 / om - tau) < 1e-9 * tau


def test_network_gradient_matches_finite_differences():
    """Pins the backward formulas of the NumPy network: central differences in FP64."""
    rng = np.random.default_rng(6)
    net = mlp.init_params(seed=7).astype(np.float64)
    X = rng.normal(size=(64, 7))
    T = rng.uniform(0, 2, size=64)
    loss, g = mlp.loss_and_grad(net, X, T)
    h = 1e-6
    for k in rng.choice(mlp.NPARAM - 3, size=60, replace=False):
        e = np.zeros_like(net)
        e[k] = h
        fd = (mlp.loss_and_grad(net + e, X, T)[0] - mlp.loss_and_grad(net - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])
    assert np.all(g[-3:] == 0)


def test_smagorinsky_run_reduces_to_trt_when_cs_is_zero():
    from paper_1909_13772_gb300 import inputs
    shape = (12, 10, 8)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1 / 0.52)
    rho, u = inputs.random_state(shape, seed=8, rho_amp=0.01, u_amp=0.03)
    f0 = oracle.init(p, rho, u)
    a = oracle.run(p, f0, 5)
    b = oracle.run(p, f0, 5, closure=dict(kind=oracle.SMAGORINSKY, cs=0.0))
    np.testing.assert_array_equal(a, b)
    c = oracle.run(p, f0, 5, closure=dict(kind=oracle.SMAGORINSKY, cs=0.17))
    assert np.abs(c - a).max() > 1e-8  # the model does act on a non-equilibrium state
