"""GPU side of the learned-closure study: the box-filter kernel against the oracle, and a small
end-to-end study (fine FP64 runs -> targets -> GPU training -> coarse runs) in which the
trained network must beat plain coarse TRT on the energy-spectrum error against the filtered
fine run."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_helpers import Case, init_sim
from paper_1909_13772_gb300 import closure_study as cs
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _box_sums(rho, u, r):
    nz, ny, nx = rho.shape
    def box(f):
        return f.reshape(nz // r, r, ny // r, r, nx // r, r).sum(axis=(1, 3, 5))
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    return np.stack([box(rho)] + [box(rho * u[a]) for a in range(3)] + [box(rho * u[a] * u[b]) for a, b in pairs])


@pytest.mark.parametrize("storage,pattern,r", [(lbm.FP64, lbm.AA, 4), (lbm.FP64, lbm.TWO_GRID, 2),
                                               (lbm.FP32, lbm.AA, 3)])
def test_coarse_moments_match_oracle(torch, storage, pattern, r):
    shape = (24, 12, 6) if r != 4 else (32, 16, 8)
    case = Case(shape=shape, storage=storage, pattern=pattern, omega=1 / 0.52, force=(1e-5, 0, 0))
    rho, u = inputs.random_state(shape, seed=5, rho_amp=0.02, u_amp=0.04)
    sim = case.make_sim()
    try:
        init_sim(sim, rho, u)
        sim.step(5)  # odd: the AA state sits in its odd layout
        got = sim.coarse_moments(0, r)
    finally:
        sim.close()
    p = case.oracle_params()
    f = oracle.run(p, oracle.init(p, rho, u), 5)
    orho, ou = oracle.macroscopic(p, f)
    want = _box_sums(orho, ou, r)
    tol = 1e-12 if storage == lbm.FP64 else 1e-5
    for m in range(10):
        assert np.abs(got[m] - want[m]).max() <= tol * np.abs(want[m]).max() + 1e-300, m


def test_coarse_moments_rejects_non_dividing_ratio(torch):
    case = Case(shape=(12, 12, 12), storage=lbm.FP32)
    sim = case.make_sim()
    try:
        with pytest.raises(lbm.LbmError):
            sim.coarse_moments(0, 5)
    finally:
        sim.close()


def test_trained_closure_beats_plain_trt(torch):
    """Small study in the under-resolved regime: 128^3 fine FP64 runs (3 training seeds), 32^3
    coarse runs at tau = 0.502, max |u| = 0.1, about three large-eddy turnovers.  Plain TRT
    piles up energy at the grid scale (or diverges); the trained network must do better on
    both spectrum scores, and its run must stay finite."""
    res = cs.study(n_f=128, r=4, tau_c=0.502, coarse_steps=512, snap_every=64, train_seeds=range(1, 4),
                   test_seed=9, umax=0.1, sample=16384, iters=1500, batch=8192, lr=2e-3, log=lambda *a: None)
    runs = res["runs"]
    assert runs["mlp"]["finite"] and runs["smagorinsky"]["finite"]
    assert res["loss"][1] < 0.5 * res["loss"][0]

    def score(name, key):
        v = runs[name][key]
        return v if runs[name]["finite"] and np.isfinite(v) else np.inf

    for key in ("spectrum_error_final", "log_spectrum_error_final"):
        assert score("mlp", key) < score("trt", key), (key, runs["mlp"][key], runs["trt"][key])
