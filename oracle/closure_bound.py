"""Tolerance of one closure-sweep step with the learned network against the FP64 oracle (test
infrastructure only, like the rest of this package).

The oracle's network is the model in exact FP64 (BF16 weights, oracle/mlp.py); the GPU's
collision evaluates it with BF16 features and activations, FP32 sums and a fast SiLU, from
features it computes in FP32.  Per fluid cell and direction the post-collision populations of
one step therefore differ by at most

    |d omega+| |n+_i| + |d omega-| |n-_i|  +  the FP32 collision's own rounding

where n+-_i = (f_i +- f_opp) / 2 - (feq_i +- feq_opp) / 2 are the non-equilibrium parts the
rates multiply (pre-collision state of the oracle), d omega+ follows from the network's bound
on y through tau = tau0 + s_tau softplus(y) and omega+ = 1 / tau, and d omega- from omega- =
1 / (Lambda / (tau - 1/2) + 1/2) at the ends of the tau interval (both rates are monotone in
tau).  The FP32 rounding term is the FP32 parity gate, 1e-5 max|f|.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import mlp

U32 = 2.0 ** -24
SOFTPLUS_ERR = 2.0 ** -17  # fast exp/log softplus: absolute error per unit of (1 + softplus)


def pre_collision_features(q, f_pre, scales):
    """(rho, u, x, x_err) per cell of a pre-collision field f_pre[i, ...] (FP64): the network's
    features x = ((rho - 1) s_rho, s_pi Pi_neq) and a bound on their error when computed in FP32
    from the FP32-rounded populations (sums of at most 19 terms, a few products)."""
    c, w, _ = oracle.lattice(q)
    f = f_pre.reshape(q, -1)
    rho = f.sum(0)
    safe = np.where(rho > 0, rho, 1.0)
    u = (c.T.astype(np.float64) @ f) / safe
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    x = np.zeros((f.shape[1], 7))
    err = np.zeros_like(x)
    af = np.abs(f).sum(0)
    x[:, 0] = (rho - 1.0) * scales[0]
    err[:, 0] = scales[0] * 40 * U32 * af + U32 * np.abs(x[:, 0])
    for k, (a, b) in enumerate(pairs):
        cc = (c[:, a] * c[:, b]).astype(np.float64)
        s = cc @ f
        pi = s - rho * ((1.0 / 3.0 if a == b else 0.0) + u[a] * u[b])
        x[:, 1 + k] = pi * scales[1]
        err[:, 1 + k] = scales[1] * 40 * U32 * ((1.0 + np.abs(cc)) @ np.abs(f)) + U32 * np.abs(x[:, 1 + k])
    return rho, u, x, err


def omega_minus(tau, lam):
    return 1.0 / (lam / (tau - 0.5) + 0.5)


def network_step_bound(p: oracle.OracleParams, net, f_pre, fluid):
    """Per (direction, cell) bound on |gpu - oracle| after one closure step from the same state,
    without the FP32 rounding term; and the network's own bound on |d omega+| per cell."""
    q = p.q
    sc = mlp.unpack(net)["scales"]
    tau0 = 1.0 / p.omega
    rho, u, x, xerr = pre_collision_features(q, f_pre, sc)
    y, dy = mlp.inference_error_bound(net, x, feat_err=xerr, silu_approx=True)
    sp = mlp._softplus(y)
    tau = tau0 + sc[2] * sp
    dtau = sc[2] * (mlp._sigmoid(y + dy) * dy + SOFTPLUS_ERR * (1.0 + mlp._softplus(y + dy))) + 4 * U32 * tau
    lo, hi = tau - dtau, tau + dtau
    dwp = 1.0 / lo - 1.0 / tau
    if p.collision == oracle.TRT:
        wm = omega_minus(tau, p.magic_lambda)
        dwm = np.maximum(np.abs(omega_minus(hi, p.magic_lambda) - wm), np.abs(wm - omega_minus(lo, p.magic_lambda)))
    else:
        dwm = dwp
    c, w, opp = oracle.lattice(q)
    f = f_pre.reshape(q, -1)
    cu = c.astype(np.float64) @ u
    usq = (u * u).sum(0)
    feq = w[:, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)
    n_p = 0.5 * (f + f[opp]) - 0.5 * (feq + feq[opp])
    n_m = 0.5 * (f - f[opp]) - 0.5 * (feq - feq[opp])
    b = 1.01 * (dwp * np.abs(n_p) + dwm * np.abs(n_m))
    b[:, ~fluid.reshape(-1)] = 0.0
    return b.reshape(f_pre.shape), dwp.reshape(f_pre.shape[1:])
