"""NumPy oracle of the learned closure's network (test infrastructure only).

The network of the learned-closure collision (Sec. 5.1.1: relaxation rates varied per cell
from a local property): 7 features -> 32 SiLU -> 32 SiLU -> 1 output y,
tau = tau0 + s_tau * softplus(y).  Packed float parameters:
    W1[32][7], b1[32], W2[32][32], b2[32], w3[32], b3, s_rho, s_pi, s_tau
Two forms of the same network:
  * ``forward``: the network being trained (the packed FP32 weights as they are), FP64
    arithmetic, with explicit backward formulas (no autograd) in ``loss_and_grad``; it checks
    the GPU training kernels.  Training objective (features x, target
    t = (tau_target - tau0) / s_tau): L = mean over samples of (softplus(y(x)) - t)^2.
  * ``forward_model``: the network as deployed in the collision.  Its weight matrices are
    BF16 numbers (the packed weights rounded to nearest even), its biases the packed FP32
    values; features, sums, SiLU and activations are exact FP64.  This is the definition the
    GPU inference and the closure sweep are compared with.
``inference_error_bound`` is the tolerance of that comparison: a per-sample bound on
|y_gpu - y_model| derived from the GPU's documented arithmetic (features and hidden
activations rounded to BF16, FP32 sums, SiLU through tanh.approx.f32).
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


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = _sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def _softplus(y):
    return np.where(y > 30.0, y, np.log1p(np.exp(np.minimum(y, 30.0))))


def forward(p, X):
    """y for features X[n, 7]: the trained network (FP32 weights), FP64 throughout."""
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


def bf16(v):
    """Round to the nearest BF16 number (ties to even), returned as float64."""
    f = np.asarray(v, dtype=np.float32).copy()
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def model_weights(p):
    """The deployed network's parameters: W1, W2, w3 rounded to BF16, biases as packed."""
    d = unpack(p)
    for k in ("W1", "W2", "w3"):
        d[k] = bf16(d[k])
    return d


def forward_model(p, X):
    """y of the deployed network for features X[n, 7] (BF16 weights, exact FP64 otherwise)."""
    d = model_weights(p)
    H1 = _silu(X @ d["W1"].T + d["b1"])
    H2 = _silu(H1 @ d["W2"].T + d["b2"])
    return H2 @ d["w3"] + d["b3"][0]


def tau_model(p, X, tau0):
    s_tau = unpack(p)["scales"][2]
    return tau0 + s_tau * _softplus(forward_model(p, X))


# ---- tolerance of the BF16 inference contract ---------------------------------------------
U_BF16 = 2.0 ** -8        # unit roundoff of BF16 (8 significant bits, round to nearest even)
TANH_REL = 2.0 ** -10.9   # maximum relative error of tanh.approx.f32 (PTX ISA)
ACC_REL = 2.0 ** -22      # per term of an FP32 sum (twice the unit roundoff: covers truncation)
SILU_LIP = 1.1            # max |SiLU'(z)| = 1.0998 (at z = 2.40)


def _silu_eval_err(a):
    """|SiLU evaluation error| at |z| <= a of SiLU(z) = h (1 + tanh h), h = z / 2, from
    tanh.approx.f32: |h| TANH_REL |tanh h|, plus the FP32 rounding of the final FMA."""
    return 0.5 * a * TANH_REL * np.tanh(0.5 * a) + 2.0 ** -23 * a


def inference_error_bound(p, X, feat_err=None, silu_approx=True):
    """(y_model, bound) per sample: |y - y_model| <= bound for y computed with the BF16
    inference arithmetic.  That arithmetic: features rounded to BF16, each hidden layer
    z = b + W h summed in FP32 from BF16 weights and BF16 inputs, SiLU evaluated
    (tanh.approx.f32 when ``silu_approx``, else exactly) and rounded to BF16, the output layer
    summed in FP32.  ``feat_err`` (shape of X, or None): an absolute error of the features
    themselves before their rounding (e.g. from computing them in FP32).

    Derivation.  Every rounding or evaluation error is a source e_s at one value v_s (a
    feature, a hidden activation, a pre-activation sum) with |e_s| <= r_s:
        feature x_i : r = 2^-8 |x_i| + feat_err_i
        activation h: r = 2^-8 |h| + SiLU evaluation error (|z|/2 2^-10.9 tanh(|z|/2) + 2^-23 |z|)
        sum z       : r = n 2^-22 (|b| + sum |W||h|)
    To first order y - y_model = sum_s (dy/dv_s) e_s, with the exact sensitivities dy/dv of the
    FP64 model (backpropagation), so |y - y_model| <= sum_s |dy/dv_s| r_s.  The remainder of
    the linearisation comes from the curvature of SiLU (|SiLU''| <= 1/2, so a perturbation dz
    of a pre-activation changes SiLU by SiLU'(z) dz + at most dz^2 / 4) and from rounding the
    perturbed instead of the exact activation (2^-8 times the activation's own error); it is
    bounded layer by layer with |W| and added."""
    X = np.asarray(X, dtype=np.float64)
    if X.shape[0] > 65536:  # in chunks: the per-sample sensitivities take 224 doubles each
        parts = [inference_error_bound(p, X[k:k + 65536], None if feat_err is None else feat_err[k:k + 65536],
                                       silu_approx) for k in range(0, X.shape[0], 65536)]
        return np.concatenate([a for a, _ in parts]), np.concatenate([b for _, b in parts])
    d = model_weights(p)
    W1, b1, W2, b2, w3, b3 = d["W1"], d["b1"], d["W2"], d["b2"], d["w3"], d["b3"][0]
    es = _silu_eval_err if silu_approx else (lambda a: 0.0 * a)
    u = U_BF16
    # model and sensitivities
    z1 = X @ W1.T + b1
    h1 = _silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = _silu(z2)
    y = h2 @ w3 + b3
    g_h2 = np.broadcast_to(w3, h2.shape)     # dy/dh2
    g_z2 = g_h2 * _dsilu(z2)                 # dy/dz2
    g_h1 = g_z2 @ W2                         # dy/dh1
    g_z1 = g_h1 * _dsilu(z1)                 # dy/dz1
    g_x = g_z1 @ W1                          # dy/dx
    # source radii
    r_x = u * np.abs(X) + (0.0 if feat_err is None else (1.0 + u) * np.abs(feat_err))
    r_z1 = ACC_REL * (IN + 1) * (np.abs(b1) + (np.abs(X) + r_x) @ np.abs(W1).T)
    r_h1 = u * np.abs(h1) + es(np.abs(z1))
    r_z2 = ACC_REL * (H + 1) * (np.abs(b2) + (np.abs(h1) + r_h1) @ np.abs(W2).T)
    r_h2 = u * np.abs(h2) + es(np.abs(z2))
    r_y = ACC_REL * (H + 1) * (abs(b3) + np.abs(h2) @ np.abs(w3))
    first = ((np.abs(g_x) * r_x).sum(1) + (np.abs(g_z1) * r_z1).sum(1) + (np.abs(g_h1) * r_h1).sum(1)
             + (np.abs(g_z2) * r_z2).sum(1) + (np.abs(g_h2) * r_h2).sum(1) + r_y)
    # first-order bounds of the pre-activation errors (for the remainder)
    dz1 = r_x @ np.abs(W1).T + r_z1
    M = np.tensordot(_dsilu(z1)[:, :, None] * W1[None], W2, axes=([1], [1]))  # dz2/dx: [n, i, k]
    dz2 = (np.abs(M) * r_x[:, :, None]).sum(1) + (r_h1 + np.abs(_dsilu(z1)) * r_z1) @ np.abs(W2).T + r_z2
    # second-order remainder, layer by layer
    e_h1 = SILU_LIP * dz1 + r_h1                                # first-order activation error
    rem_h1 = 0.25 * dz1 * dz1 + u * e_h1
    rem_z2 = rem_h1 @ np.abs(W2).T
    dz2t = dz2 + rem_z2
    e_h2 = SILU_LIP * dz2t + r_h2
    rem_h2 = SILU_LIP * rem_z2 + 0.25 * (dz2t * dz2t) + u * e_h2
    rem = rem_h2 @ np.abs(w3)
    return y, first + rem
