"""GPU parity of the locally varying relaxation (Sec. 5.1.1: per-cell relaxation rates from a
local fluid property): the closure sweep with Smagorinsky and with the learned-closure network
(tensor-core inference fused into the collision), and the network's inference and training
kernels, against the CPU oracle (oracle/lbm_oracle.c, oracle/mlp.py)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle.closure_bound import network_step_bound
from gpu_helpers import TOL, Case, gather_pdfs, init_sim, normwise, oracle_run, split
from oracle import mlp
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _features(n, seed):
    """Seeded features in the range the closure sees: (rho - 1) s_rho and s_pi Pi_neq of order 1."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 7)) * np.array([0.5, 1, 1, 1, 0.7, 0.7, 0.7])
    return X.astype(np.float32)


def _net(seed, s_rho=20.0, s_pi=200.0, s_tau=0.02):
    """A network whose weights are far from the initial ones (so that every unit matters)."""
    p = mlp.unpack(mlp.init_params(seed=seed, s_rho=s_rho, s_pi=s_pi, s_tau=s_tau))
    rng = np.random.default_rng(seed + 100)
    p["b1"] = rng.uniform(-0.5, 0.5, 32)
    p["b2"] = rng.uniform(-0.5, 0.5, 32)
    p["w3"] = p["w3"] * 3.0
    p["b3"] = np.array([0.3])
    return mlp.pack(p)


def test_network_inference_matches_model_within_bound(torch):
    """Tensor-core inference (BF16 features, weights and activations, FP32 sums, SiLU from
    tanh.approx) against the deployed network in exact FP64 (oracle/mlp.py forward_model):
    every sample within the bound derived from that arithmetic (inference_error_bound), the
    typical sample well inside it.  Ragged n (not a multiple of the 128-sample tile)."""
    P = _net(5)
    n = 4099
    X = _features(n, 1)
    want, bound = mlp.inference_error_bound(P, X.astype(np.float64))
    m = lbm.lbm_mlp_create(P, 16, None)
    try:
        Xd = torch.from_numpy(X).cuda()
        yd = torch.full((n + 32,), 7.0, device="cuda")  # sentinel tail must stay untouched
        lbm.lbm_mlp_infer(m, Xd.data_ptr(), n, yd.data_ptr())
        torch.cuda.synchronize()
        got = yd.cpu().numpy().astype(np.float64)
    finally:
        lbm.lbm_mlp_destroy(m)
    assert np.all(got[n:] == 7.0)
    ratio = np.abs(got[:n] - want) / bound
    assert np.all(ratio <= 1.0), (ratio.max(), np.abs(got[:n] - want).max())
    assert np.median(ratio) < 0.25, np.median(ratio)
    # the bound itself is small against the output (a wrong layer would be off by O(1))
    assert np.median(bound) < 0.05 * np.median(np.abs(want))


def test_network_inference_zero_and_one_sample(torch):
    P = _net(6)
    m = lbm.lbm_mlp_create(P, 1, None)
    try:
        X = _features(1, 2)
        Xd = torch.from_numpy(X).cuda()
        yd = torch.zeros(1, device="cuda")
        lbm.lbm_mlp_infer(m, Xd.data_ptr(), 0, yd.data_ptr())  # n = 0: nothing launched
        lbm.lbm_mlp_infer(m, Xd.data_ptr(), 1, yd.data_ptr())
        torch.cuda.synchronize()
        want, bound = mlp.inference_error_bound(P, X.astype(np.float64))
        assert abs(float(yd[0]) - want[0]) <= bound[0]
    finally:
        lbm.lbm_mlp_destroy(m)


@pytest.mark.parametrize("n", [1, 130, 3000])
def test_network_gradient_matches_oracle(torch, n):
    """FP32 training gradient (deterministic per-CTA partials) against the FP64 explicit
    backward of oracle/mlp.py; n spans one partial chunk, several chunks and several CTAs
    with a ragged tail."""
    P = _net(7)
    X = _features(n, 3)
    rng = np.random.default_rng(4)
    T = rng.uniform(0.0, 2.0, n).astype(np.float32)
    want_loss, want_g = mlp.loss_and_grad(P, X.astype(np.float64), T.astype(np.float64))
    m = lbm.lbm_mlp_create(P, 4096, None)
    try:
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        loss, g = lbm.lbm_mlp_loss_grad(m, Xd.data_ptr(), Td.data_ptr(), n)
        loss2, g2 = lbm.lbm_mlp_loss_grad(m, Xd.data_ptr(), Td.data_ptr(), n)
    finally:
        lbm.lbm_mlp_destroy(m)
    assert np.array_equal(g, g2) and loss == loss2  # fixed summation order
    assert abs(loss - want_loss) <= 1e-5 * want_loss
    # FP32 forward/backward of a 32-wide network: normwise error of the gradient ~1e-6
    assert normwise(g.astype(np.float64), want_g) < 5e-5
    assert np.all(g[-3:] == 0)  # the scales are not trained


def test_training_fits_a_teacher_and_is_deterministic(torch):
    """Adam on the GPU reduces the loss of a network fitting another network's outputs;
    two runs from the same start give bit-identical parameters."""
    teacher = _net(11)
    X = _features(8192, 5)
    T = mlp._softplus(mlp.forward(teacher, X.astype(np.float64))).astype(np.float32)
    start = mlp.init_params(seed=12, s_rho=20.0, s_pi=200.0, s_tau=0.02)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    out = []
    for _ in range(2):
        m = lbm.lbm_mlp_create(start, 1024, None)
        try:
            hist = lbm.lbm_mlp_train(m, Xd.data_ptr(), Td.data_ptr(), X.shape[0], 1024, 400, 3e-3)
            out.append((hist, lbm.lbm_mlp_get_params(m)))
        finally:
            lbm.lbm_mlp_destroy(m)
    (h1, p1), (h2, p2) = out
    assert np.array_equal(p1, p2) and np.array_equal(h1, h2)
    full0 = mlp.loss_and_grad(start, X.astype(np.float64), T.astype(np.float64))[0]
    full1 = mlp.loss_and_grad(p1, X.astype(np.float64), T.astype(np.float64))[0]
    assert full1 < 0.1 * full0, (full0, full1)
    assert np.all(p1[-3:] == start[-3:])


def _turb_case(shape, pattern, closure, blocks=None, periodic=(1, 1, 1), faces=(1,) * 6, collision=lbm.TRT):
    return Case(shape=shape, blocks=blocks, storage=lbm.FP32, pattern=pattern, omega=1 / 0.505,
                collision=collision, periodic=periodic, faces=faces)


def _turb_state(shape, seed):
    n = max(shape)
    rho, u = inputs.turbulence(n, seed=seed, kmax=n // 4, umax=0.08)
    nx, ny, nz = shape
    return np.ascontiguousarray(rho[:nz, :ny, :nx]), np.ascontiguousarray(u[:, :nz, :ny, :nx])


def _closure_run(case, closure, steps, seed=21):
    rho, u = _turb_state(case.shape, seed)
    sim = case.make_sim()
    try:
        if closure["kind"] == oracle.SMAGORINSKY:
            sim.set_closure(lbm.CLOSURE_SMAGORINSKY, cs=closure["cs"])
        else:
            sim.set_closure(lbm.CLOSURE_MLP, mlp_params=closure["mlp"])
        init_sim(sim, rho, u)
        sim.step(steps)
        got = gather_pdfs(sim, case)
    finally:
        sim.close()
    p = case.oracle_params()
    fl = case.global_flags()
    f0 = oracle.init(p, rho, u, flags=fl)
    want = oracle.run(p, f0, steps, flags=fl, closure=closure)
    plain = oracle.run(p, f0, steps, flags=fl)
    return got, want, plain


SMAG = dict(kind=oracle.SMAGORINSKY, cs=0.17)


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_smagorinsky_sweep_matches_oracle(torch, pattern):
    """Periodic box (the block is its own neighbour: wrap path), ragged sizes."""
    case = _turb_case((40, 21, 9), pattern, SMAG)
    got, want, plain = _closure_run(case, SMAG, 6)
    assert normwise(got, want) < TOL[lbm.FP32]
    assert normwise(plain, want) > 100 * TOL[lbm.FP32]  # the closure changed the flow


def _mlp_steps_within_bound(case, net, rho, u, steps, check_effect=True, sample=None):
    """Each of `steps` closure steps from the oracle's state: the GPU sets the oracle state
    f*(t) (FP64 -> FP32), sweeps once and is compared with the oracle's f*(t+1) cell by cell
    and direction by direction, within the derived bound (oracle/closure_bound.py) plus the
    FP32 gate.  AA contexts alternate their two sweeps from step to step.  `sample`: compare a
    seeded random fraction of the fluid cells only (large boxes).  Returns the largest ratio of
    error to bound."""
    p = case.oracle_params()
    fl = case.global_flags()
    fluid = fl == 0
    if sample is not None:
        keep = np.random.default_rng(17).random(fl.shape) < sample
        fluid = fluid & keep
    cl = dict(kind=oracle.MLP, mlp=net)
    f = oracle.init(p, rho, u, flags=fl)
    sim = case.make_sim()
    worst = 0.0
    try:
        sim.set_closure(lbm.CLOSURE_MLP, mlp_params=net)
        init_sim(sim, rho, u)
        for t in range(steps):
            for b, fb in enumerate(split(sim, f)):
                sim.set_pdfs(b, np.ascontiguousarray(fb))
            sim.step(1)
            got = gather_pdfs(sim, case)
            want = oracle.run(p, f, 1, flags=fl, closure=cl)
            pre = oracle.stream(p, f, flags=fl)[:, fluid]
            net_b, dwp = network_step_bound(p, net, pre, np.ones(pre.shape[1], bool))
            gate = TOL[lbm.FP32] * np.abs(want[:, fl == 0]).max()
            err = np.abs(got - want)[:, fluid]
            ratio = err / (net_b + gate)
            assert ratio.max() <= 1.0, (t, ratio.max(), err.max(), gate)
            worst = max(worst, float(ratio.max()))
            if check_effect:
                # the closure's effect on the step is far above the network's share of the bound
                plain = oracle.run(p, f, 1, flags=fl)
                effect = np.abs(want - plain)[:, fluid].max(axis=0)
                assert np.median(effect / (net_b.max(axis=0) + 1e-300)) > 20
            f = want
    finally:
        sim.close()
    return worst


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_mlp_sweep_matches_oracle(torch, pattern):
    """Periodic box (the block is its own neighbour: wrap path), ragged sizes, 4 steps (both AA
    sweeps twice)."""
    net = _net(31)
    case = _turb_case((40, 21, 9), pattern, None)
    rho, u = _turb_state(case.shape, 21)
    _mlp_steps_within_bound(case, net, rho, u, 4)


@pytest.mark.parametrize("kind", ["smag", "mlp"])
def test_closure_sweep_multiblock_walls(torch, kind):
    """Four blocks reading each other in place (general neighbour table), no-slip walls on z,
    an obstacle (masks, bounce-back bits), two-grid and AA."""
    shape = (48, 20, 12)
    blocks = [((0, 0, 0), (24, 20, 12)), ((24, 0, 0), (24, 10, 12)), ((24, 10, 0), (24, 10, 12))]
    fl = np.zeros((12, 20, 48), np.uint8)
    fl[4:8, 6:12, 20:30] = oracle.NOSLIP
    for pattern in (lbm.TWO_GRID, lbm.AA):
        case = _turb_case(shape, pattern, None, blocks=blocks, periodic=(1, 1, 0))
        case.flags = fl
        if kind == "smag":
            got, want, _ = _closure_run(case, SMAG, 5)
            assert normwise(got, want, mask=fl == 0) < TOL[lbm.FP32], pattern
        else:
            rho, u = _turb_state(case.shape, 21)
            _mlp_steps_within_bound(case, _net(41), rho, u, 3, check_effect=False)


def test_closure_with_graph_replay_and_diagnostics(torch):
    """Graph-captured step pairs and the fused step diagnostics run the closure sweep too."""
    cl = dict(kind=oracle.MLP, mlp=_net(51))
    case = _turb_case((64, 16, 8), lbm.AA, cl)
    rho, u = _turb_state(case.shape, 3)
    res = []
    for graph in (False, True):
        s = torch.cuda.Stream()
        sim = case.make_sim(stream=s.cuda_stream)
        try:
            sim.set_closure(lbm.CLOSURE_MLP, mlp_params=cl["mlp"])
            if graph:
                lbm.lbm_set_graph(sim.ctx, 1)
            init_sim(sim, rho, u)
            sim.step(11)
            d = sim.step_diagnostics()
            res.append((gather_pdfs(sim, case), d))
        finally:
            sim.close()
    assert np.array_equal(res[0][0], res[1][0])
    full = oracle.diagnostics(case.oracle_params(), res[0][0].astype(np.float64))
    # the fused mass sums each cell's stored FP32 values exactly (float-float, <= Q^2 2^-48
    # relative per cell); a thread's n = 4 cells and the CTA's pairs add FP32 low parts, within
    # (Q + n + 3)^2 2^-48 in all; FP64 from the CTA records on
    assert abs(res[0][1]["mass"] - full["mass"]) < ((19 + 4 + 3) ** 2 * 2.0 ** -48 + 1e-13) * full["mass"]


def test_clearing_the_closure_restores_the_plain_sweep(torch):
    case = _turb_case((32, 8, 8), lbm.TWO_GRID, SMAG)
    rho, u = _turb_state(case.shape, 4)
    out = []
    for clear in (False, True):
        sim = case.make_sim()
        try:
            if clear:
                sim.set_closure(lbm.CLOSURE_SMAGORINSKY, cs=0.2)
                sim.set_closure(lbm.CLOSURE_NONE)
            init_sim(sim, rho, u)
            sim.step(4)
            out.append(gather_pdfs(sim, case))
        finally:
            sim.close()
    assert np.array_equal(out[0], out[1])


def test_mlp_sweep_at_the_coarse_study_size(torch):
    """The learned-closure coarse configuration itself: 128^3 periodic box, D3Q19 TRT
    tau0 = 0.502, FP32 AA, random-phase start with max|u| = 0.1, a trained-like network; three
    steps (neighbour, local, neighbour sweep), each against the oracle within the derived
    bound on a seeded eighth of the cells (262,144 cells, every direction)."""
    n = 128
    rho, u = inputs.turbulence(n, seed=9, kmax=n // 4, umax=0.1)
    net = _net(61, s_rho=100.0, s_pi=300.0, s_tau=1e-3)
    case = Case(shape=(n, n, n), storage=lbm.FP32, pattern=lbm.AA, omega=1 / 0.502)
    _mlp_steps_within_bound(case, net, rho, u, 3, check_effect=False, sample=0.125)


def test_inference_after_training_uses_the_trained_parameters(torch):
    """lbm_mlp_train converts the trained parameters to the inference form on the device; the
    result must equal, bit for bit, a network created from the read-back parameters (host
    conversion)."""
    X = _features(5000, 8)
    T = np.abs(np.random.default_rng(9).standard_normal(5000)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = lbm.lbm_mlp_create(_net(71), 1024, None)
    m2 = None
    try:
        lbm.lbm_mlp_train(m, Xd.data_ptr(), Td.data_ptr(), 5000, 1024, 25, 3e-3)
        y1 = torch.empty(5000, device="cuda")
        lbm.lbm_mlp_infer(m, Xd.data_ptr(), 5000, y1.data_ptr())
        trained = lbm.lbm_mlp_get_params(m)
        m2 = lbm.lbm_mlp_create(trained, 16, None)
        y2 = torch.empty(5000, device="cuda")
        lbm.lbm_mlp_infer(m2, Xd.data_ptr(), 5000, y2.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
        assert not np.array_equal(trained, _net(71))
    finally:
        lbm.lbm_mlp_destroy(m)
        if m2 is not None:
            lbm.lbm_mlp_destroy(m2)
