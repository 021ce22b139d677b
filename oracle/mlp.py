"""NumPy oracle of the learned closure's network (test infrastructure only).

The network of the learned-closure collision (Sec. 5.1.1: relaxation rates varied per cell
from a local property, read from a field): 7 features -> 32 SiLU -> 32 SiLU -> 1 output y,
tau = tau0 + s_tau * softplus(y).  Packed float parameters:
    W1[32][7], b1[32], W2[32][32], b2[32], w3[32], b3, s_rho, s_pi, s_tau
Training objective (one sample: features x, target t = (tau_target - tau0) / s_tau):
    L = mean over samples of (softplus(y(x)) - t)^2
This file restates the network in FP64 with explicit backward formulas (no autograd), for
checking the GPU training kernels; ``forward_bf16`` rounds at the inference kernel's points.
"""
from __future__ import annotations

import numpy as np

H, IN = 32, 7
SIZES = {"W1": (H, IN), "b1": (H,), "W2": (H, H), "b2": (H,), "w3": (H,), "b3": (1,), "scales": (3,)}
NPARAM = sum(int(np.prod(v)) for v in SIZES.values())  # 1348


def unpack(p):
    out, k = {}, 0
    for name, shape in SIZES.items():
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name in SIZES]).astype(np.float32)


def init_params(seed=0, s_rho=1.0, s_pi=1.0, s_tau=1.0):
    """Seeded initial weights (uniform +-1/sqrt(fan_in)) and the feature/output scales."""
    rng = np.random.default_rng(seed)
    d = {
        "W1": rng.uniform(-1, 1, (H, IN)) / np.sqrt(IN), "b1": np.zeros(H),
        "W2": rng.uniform(-1, 1, (H, H)) / np.sqrt(H), "b2": np.zeros(H),
        "w3": rng.uniform(-1, 1, H) / np.sqrt(H), "b3": np.array([-2.0]),
        "scales": np.array([s_rho, s_pi, s_tau]),
    }
    return pack(d)


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _softplus(y):
    return np.where(y > 30.0, y, np.log1p(np.exp(np.minimum(y, 30.0))))


def forward(p, X):
    """y for features X[n, 7] (FP64 throughout)."""
    d = unpack(p)
    Z1 = X @ d["W1"].T + d["b1"]
    H1 = _silu(Z1)
    Z2 = H1 @ d["W2"].T + d["b2"]
    H2 = _silu(Z2)
    return H2 @ d["w3"] + d["b3"][0]


def loss_and_grad(p, X, T):
    """(loss, gradient over the packed parameters; scales get zero gradient)."""
    d = unpack(p)
    n = X.shape[0]
    Z1 = X @ d["W1"].T + d["b1"]
    H1 = _silu(Z1)
    Z2 = H1 @ d["W2"].T + d["b2"]
    H2 = _silu(Z2)
    y = H2 @ d["w3"] + d["b3"][0]
    sp = _softplus(y)
    r = sp - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / (1.0 + np.exp(-y)) / n          # d loss / d y
    g = {"w3": H2.T @ dy, "b3": np.array([dy.sum()])}
    dZ2 = np.outer(dy, d["w3"]) * _dsilu(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ d["W2"]) * _dsilu(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    g["scales"] = np.zeros(3)
    return loss, np.concatenate([np.ravel(g[k]) for k in SIZES])


def _bf16(v):
    f = np.asarray(v, dtype=np.float32).copy()
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, X):
    """y with features, hidden activations and weights rounded to BF16 (inference points)."""
    d = unpack(p)
    x = _bf16(X)
    H1 = _bf16(_silu(x @ _bf16(d["W1"]).T + d["b1"]))
    H2 = _bf16(_silu(H1 @ _bf16(d["W2"]).T + d["b2"]))
    return H2 @ _bf16(d["w3"]) + d["b3"][0]


def tau_of(p, X, tau0):
    s_tau = unpack(p)["scales"][2]
    return tau0 + s_tau * _softplus(forward_bf16(p, X))
