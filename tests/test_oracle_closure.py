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
    """The C oracle's network (loops, BF16 weights rounded by bit operations) against the NumPy
    model (matrix products, BF16 weights from a separate rounding routine): both exact FP64."""
    p = _params(19)
    net = mlp.init_params(seed=5, s_rho=10.0, s_pi=300.0, s_tau=0.05)
    sc = mlp.unpack(net)["scales"]
    for f in _cells(19, 30, 4, noneq=0.05):
        om, _ = oracle.collide_closure(p, f, oracle.MLP, mlp=net)
        rho, pi = _pi_neq(19, f)
        x = np.array([(rho - 1) * sc[0], pi[0, 0] * sc[1], pi[1, 1] * sc[1], pi[2, 2] * sc[1],
                      pi[0, 1] * sc[1], pi[0, 2] * sc[1], pi[1, 2] * sc[1]])
        tau = mlp.tau_model(net, x[None], 1 / p.omega)[0]
        assert abs(1 / om - tau) < 1e-12 * tau


def _dense_net(seed, b_shift=0.0, positive_w2=False):
    d = mlp.unpack(mlp.init_params(seed=seed))
    rng = np.random.default_rng(seed + 1)
    d["b1"] = rng.uniform(-0.5, 0.5, 32) + b_shift
    d["b2"] = rng.uniform(-0.5, 0.5, 32) + b_shift
    if positive_w2:
        d["W2"] = np.abs(d["W2"])
    d["b3"] = np.array([0.3])
    return mlp.pack(d)


def test_model_network_slope_at_zero():
    """SiLU(0) = 0 and SiLU'(0) = 1/2: with zero biases the network's gradient at x = 0 is
    (1/4) w3^T W2 W1 (BF16 weights).  A transposed weight, a dropped layer or a wrong SiLU
    slope changes it."""
    d = mlp.unpack(_dense_net(11))
    d["b1"][:] = 0.0
    d["b2"][:] = 0.0
    net = mlp.pack(d)
    W = mlp.model_weights(net)
    want = 0.25 * (W["w3"] @ W["W2"] @ W["W1"])
    eps = 1e-5
    for k in range(7):
        e = np.zeros((2, 7))
        e[0, k], e[1, k] = eps, -eps
        y = mlp.forward_model(net, e)
        assert abs((y[0] - y[1]) / (2 * eps) - want[k]) <= 1e-8 * max(1.0, abs(want[k]))
    assert mlp.forward_model(net, np.zeros((1, 7)))[0] == np.float64(np.float32(0.3))


def test_model_network_saturated_regime_is_affine():
    """SiLU(z) -> z for z >> 1: with biases +60 and non-negative W2 every unit saturates and
    the network equals the affine map b3 + w3 . (W2 (W1 x + b1) + b2); a dropped bias or a
    misplaced layer breaks it."""
    net = _dense_net(12, b_shift=60.0, positive_w2=True)
    W = mlp.model_weights(net)
    X = np.random.default_rng(3).standard_normal((50, 7))
    affine = (X @ W["W1"].T + W["b1"]) @ W["W2"].T + W["b2"]
    assert affine.min() > 30.0
    want = affine @ W["w3"] + W["b3"][0]
    np.testing.assert_allclose(mlp.forward_model(net, X), want, rtol=1e-12, atol=1e-11)


def test_model_network_hidden_unit_permutation_invariance():
    """Relabelling the hidden units of either layer (rows of W and b, columns of the next
    weight matrix) leaves y unchanged; a transposed W2 does not have that symmetry."""
    net = _dense_net(13)
    d = mlp.unpack(net)
    rng = np.random.default_rng(4)
    p1, p2 = rng.permutation(32), rng.permutation(32)
    e = dict(d)
    e["W1"], e["b1"] = d["W1"][p1], d["b1"][p1]
    e["W2"] = d["W2"][p2][:, p1]
    e["b2"], e["w3"] = d["b2"][p2], d["w3"][p2]
    X = rng.standard_normal((40, 7))
    np.testing.assert_allclose(mlp.forward_model(mlp.pack(e), X), mlp.forward_model(net, X), rtol=1e-13, atol=1e-13)
    t = dict(e)
    t["W2"] = e["W2"].T.copy()
    assert np.abs(mlp.forward_model(mlp.pack(t), X) - mlp.forward_model(net, X)).max() > 1e-3


def test_model_network_matches_torch_float64():
    """Against the textbook layers of another library: torch.nn.functional.linear and silu in
    float64, same BF16 weights."""
    torch = pytest.importorskip("torch")
    net = _dense_net(14)
    W = mlp.model_weights(net)
    X = np.random.default_rng(5).standard_normal((64, 7))
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))  # noqa: E731
    F = torch.nn.functional
    h = F.silu(F.linear(T(X), T(W["W1"]), T(W["b1"])))
    h = F.silu(F.linear(h, T(W["W2"]), T(W["b2"])))
    y = F.linear(h, T(W["w3"][None]), T(W["b3"])).numpy()[:, 0]
    np.testing.assert_allclose(mlp.forward_model(net, X), y, rtol=1e-13, atol=1e-13)


def _features(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 7)) * np.array([0.5, 1, 1, 1, 0.7, 0.7, 0.7])
    return X.astype(np.float32).astype(np.float64)


def _round_bits(v, bits):
    m, e = np.frexp(v)
    return np.ldexp(np.round(m * 2.0 ** bits) / 2.0 ** bits, e)


def _rounded_inference(net, X, rnd):
    """The network with its features and hidden activations rounded by ``rnd`` (exact SiLU, FP64
    sums): the arithmetic the BF16 inference bound is derived for, with rnd = BF16."""
    W = mlp.model_weights(net)
    h1 = rnd(mlp._silu(rnd(X) @ W["W1"].T + W["b1"]))
    h2 = rnd(mlp._silu(h1 @ W["W2"].T + W["b2"]))
    return h2 @ W["w3"] + W["b3"][0]


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_inference_bound_covers_bf16_rounding_and_rejects_coarser(seed):
    """The per-sample bound of the BF16 inference holds for features and activations rounded to
    BF16 (every sample, with room: the median sample uses a small part of it), and fails when
    the rounding points keep 5 significant bits instead of 8 -- the bound is tight enough to
    tell the two apart."""
    net = _dense_net(seed)
    X = _features(20000, seed)
    y, bound = mlp.inference_error_bound(net, X, silu_approx=False)
    np.testing.assert_allclose(y, mlp.forward_model(net, X), rtol=0, atol=0)
    r = np.abs(_rounded_inference(net, X, mlp.bf16) - y) / bound
    assert r.max() <= 1.0 and np.median(r) < 0.2, (r.max(), np.median(r))
    coarse = np.abs(_rounded_inference(net, X, lambda v: _round_bits(v, 5)) - y) / bound
    assert (coarse > 1.0).mean() > 0.02, (coarse > 1.0).mean()
    # the bound is small against the output itself (a wrong layer would be off by O(1))
    assert np.median(bound) < 0.05 * np.median(np.abs(y))


def test_stream_then_collide_equals_one_step():
    """orc_stream is the first half of orc_run: colliding its output cell by cell gives the
    next state bit for bit (walls in y, body force); in a periodic box it is np.roll."""
    from paper_1909_13772_gb300 import inputs
    shape = (9, 7, 5)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1.3, force=(1e-5, 0, 0),
                            periodic=(1, 0, 1), face_kind=(1, 1, oracle.NOSLIP, oracle.NOSLIP, 1, 1))
    rho, u = inputs.random_state(shape, seed=3, rho_amp=0.01, u_amp=0.02)
    f0 = oracle.init(p, rho, u)
    pre = oracle.stream(p, f0)
    nxt = oracle.run(p, f0, 1)
    for z in range(shape[2]):
        for y in range(shape[1]):
            for x in range(shape[0]):
                np.testing.assert_array_equal(oracle.collide_cell(p, pre[:, z, y, x]), nxt[:, z, y, x])
    pp = oracle.OracleParams(shape=shape, q=27)
    f = np.random.default_rng(1).random((27,) + shape[::-1])
    c, _, _ = oracle.lattice(27)
    pre = oracle.stream(pp, f)
    for i in range(27):
        np.testing.assert_array_equal(pre[i], np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)))


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
