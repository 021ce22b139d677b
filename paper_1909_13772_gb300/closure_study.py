"""Learned-closure study on decaying turbulence: training data from box-filtered fine-grid runs,
training of the closure network on the GPU, and the a-posteriori comparison of coarse runs
(plain TRT, Smagorinsky, the trained network) against the filtered fine run.

The paper lets the relaxation rate vary per cell from a local fluid property, read from a
field, and names turbulence models among its uses (Sec. 5.1.1).  This module builds the data
for such a closure from the method itself and scores it; every lattice Boltzmann step, the
filtering sums, the network's training and its inference run in the library's kernels.  The
host computes only what turns the filtered sums into training pairs and scores (finite
differences of a 3-D array, local averages, FFT energy spectra).

Readings (the paper fixes none of this):
  * fine run: D3Q19 TRT (Lambda 3/16), FP64 storage, AA pattern, periodic n_f^3 box, random-
    phase k^(-5/3) velocity field (``inputs.turbulence``), rho = 1.  Acoustic scaling between
    the grids: dx and dt both r times smaller on the fine grid, so the same physical viscosity
    has nu_f = r nu_c, i.e. tau_f = 1/2 + r (tau_c - 1/2), and r fine steps make one coarse step.
  * filter: box average over r^3 fine cells, density-weighted for velocity:
        rho_bar = <rho>,  u_bar = <rho u> / rho_bar,
        sub-grid stress  T_ab = <rho u_a u_b> - rho_bar u_bar_a u_bar_b.
  * coarse strain S_ab = (d_a u_b + d_b u_a) / 2 by second-order central differences on the
    periodic coarse grid (spacing 1).
  * target: the eddy viscosity that best explains the deviatoric sub-grid stress as
    T^d = -2 rho_bar nu_t S^d, by least squares over the 3^3 neighbourhood of each cell
    (numerator and denominator averaged before the division, as in Lilly's least-squares form
    of the Germano identity), clipped at 0:
        nu_t = max(0, -<T^d : S^d> / (2 <rho_bar S^d : S^d>)),  tau_t = tau_c + 3 nu_t.
  * features: the network sees the cell's pre-collision density and non-equilibrium stress.
    For a coarse run relaxing with tau_t, the Chapman-Enskog expansion gives
    Pi_neq = -(2/3) rho_bar tau_t S (lattice units), so the training features are
    ((rho_bar - 1) s_rho, s_pi Pi_neq) with that Pi_neq.
  * score: shell-summed kinetic energy spectrum E(k), k = 1 .. N_c/2 on the coarse grid; the
    error of a coarse run is sum_k |E(k) - E_ref(k)| / sum_k E_ref(k), E_ref from the filtered
    fine run at the same physical time.  Coarse runs start from the filtered fine initial state.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, lbm

MLP_NPARAM = lbm.MLP_NPARAM
H, IN = 32, 7


# ---- host-side analysis ------------------------------------------------------------------

def filtered_fields(m, r):
    """(rho_bar, u_bar[3], T_sgs[6]) from the box sums of lbm_coarse_moments (r^3 cells each)."""
    n = float(r ** 3)
    rho = m[0] / n
    u = m[1:4] / n / rho
    T = np.empty((6,) + rho.shape)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for k, (a, b) in enumerate(pairs):
        T[k] = m[4 + k] / n - rho * u[a] * u[b]
    return rho, u, T


def strain(u):
    """S (xx, yy, zz, xy, xz, yz) of u[3, z, y, x] by central differences, periodic, spacing 1."""
    def d(f, axis):  # axis: 0 = x, 1 = y, 2 = z of the [z, y, x] array
        ax = 2 - axis
        return 0.5 * (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax))
    g = [[d(u[b], a) for b in range(3)] for a in range(3)]  # g[a][b] = d_a u_b
    return np.stack([g[0][0], g[1][1], g[2][2], 0.5 * (g[0][1] + g[1][0]), 0.5 * (g[0][2] + g[2][0]),
                     0.5 * (g[1][2] + g[2][1])])


def _dev(t):
    tr = (t[0] + t[1] + t[2]) / 3.0
    out = t.copy()
    out[0] -= tr
    out[1] -= tr
    out[2] -= tr
    return out


def _ddot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + 2.0 * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5])


def _box3(f):
    out = np.zeros_like(f)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out += np.roll(f, (dz, dy, dx), axis=(0, 1, 2))
    return out / 27.0


def targets(rho, u, T, tau_c):
    """(tau_t, S, nu_t) per coarse cell (see the module header)."""
    S = strain(u)
    Sd, Td = _dev(S), _dev(T)
    num = _box3(_ddot(Td, Sd))
    den = _box3(2.0 * rho * _ddot(Sd, Sd))
    nu = np.where(den > 0, -num / np.where(den > 0, den, 1.0), 0.0)
    nu = np.maximum(nu, 0.0)
    return tau_c + 3.0 * nu, S, nu


def features(rho, S, tau, s_rho, s_pi):
    """Network inputs [n, 7] for cells with density rho, strain S and relaxation time tau."""
    pi = -(2.0 / 3.0) * rho * tau * S
    X = np.concatenate([((rho - 1.0) * s_rho)[None], pi * s_pi]).reshape(7, -1).T
    return np.ascontiguousarray(X, dtype=np.float32)


def spectrum(u):
    """Shell-summed kinetic energy E(k), k = 0 .. N/2, of u[3, N, N, N] (periodic, unit density)."""
    N = u.shape[-1]
    kf = np.fft.fftfreq(N, d=1.0 / N)
    kr = np.fft.rfftfreq(N, d=1.0 / N)
    kmag = np.sqrt(kf[:, None, None] ** 2 + kf[None, :, None] ** 2 + kr[None, None, :] ** 2)
    shell = np.rint(kmag).astype(np.int64)
    wgt = np.full(kr.shape, 2.0)  # half spectrum: interior x modes stand for their conjugates
    wgt[0] = 1.0
    if N % 2 == 0:
        wgt[-1] = 1.0
    e = np.zeros(shell.shape)
    for a in range(3):
        uh = np.fft.rfftn(u[a]) / float(N ** 3)
        e += 0.5 * (uh.real ** 2 + uh.imag ** 2)
    e *= wgt[None, None, :]
    E = np.bincount(shell.ravel(), weights=e.ravel(), minlength=N // 2 + 2)
    return E[:N // 2 + 1]


def spectrum_error(E, E_ref):
    """Relative L1 error of the spectrum over shells 1 .. N/2 (dominated by the energetic shells)."""
    k = slice(1, len(E_ref))
    return float(np.abs(E[k] - E_ref[k]).sum() / E_ref[k].sum())


def log_spectrum_error(E, E_ref):
    """Mean |ln(E / E_ref)| over shells 1 .. N/2 (every shell counts alike: shows pile-up or
    over-damping near the grid cut-off)."""
    k = slice(1, len(E_ref))
    return float(np.mean(np.abs(np.log(np.maximum(E[k], 1e-300) / E_ref[k]))))


# ---- runs through the library ------------------------------------------------------------

def _stream():
    import torch
    return torch.cuda.Stream()


def fine_run(n_f, r, seed, tau_c, coarse_steps, snap_every, kmax, umax, stream=None):
    """Fine FP64 run; returns [(coarse step, m)] with m the box sums at each snapshot."""
    tau_f = 0.5 + r * (tau_c - 0.5)
    p = lbm.make_params(stencil=19, collision=lbm.TRT, storage=lbm.FP64, pattern=lbm.AA, omega=1.0 / tau_f,
                        periodic=(1, 1, 1))
    rho, u = inputs.turbulence(n_f, seed=seed, kmax=kmax, umax=umax)
    sim = lbm.Simulation(p, [((0, 0, 0), (n_f, n_f, n_f))], stream=stream)
    out = []
    try:
        sim.init(0, rho, u)
        del rho, u
        out.append((0, sim.coarse_moments(0, r)))
        for t in range(snap_every, coarse_steps + 1, snap_every):
            sim.step(r * snap_every)
            out.append((t, sim.coarse_moments(0, r)))
    finally:
        sim.close()
    return out


def coarse_run(rho0, u0, tau_c, steps, closure, snap_every, stream=None):
    """Coarse FP32 run from (rho0, u0); closure = None | ("smag", cs) | ("mlp", params).
    Returns ([(step, u)], ms per step)."""
    import torch
    N = rho0.shape[0]
    p = lbm.make_params(stencil=19, collision=lbm.TRT, storage=lbm.FP32, pattern=lbm.AA, omega=1.0 / tau_c,
                        periodic=(1, 1, 1))
    sim = lbm.Simulation(p, [((0, 0, 0), (N, N, N))], stream=stream)
    out = []
    try:
        if closure is not None and closure[0] == "smag":
            sim.set_closure(lbm.CLOSURE_SMAGORINSKY, cs=closure[1])
        elif closure is not None:
            sim.set_closure(lbm.CLOSURE_MLP, mlp_params=closure[1])
        sim.init(0, rho0, u0)
        out.append((0, sim.macroscopic(0)[1]))
        t_ms, n_t = 0.0, 0
        for t in range(snap_every, steps + 1, snap_every):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s = stream if stream is not None else torch.cuda.current_stream()
            e0.record(s)
            sim.step(snap_every)
            e1.record(s)
            e1.synchronize()
            t_ms += e0.elapsed_time(e1)
            n_t += snap_every
            out.append((t, sim.macroscopic(0)[1]))
    finally:
        sim.close()
    return out, t_ms / max(n_t, 1)


def init_params(seed, s_rho, s_pi, s_tau):
    """Initial network: uniform +-1/sqrt(fan_in) weights, zero hidden biases, output bias -2."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (H, IN)) / math.sqrt(IN)
    W2 = rng.uniform(-1, 1, (H, H)) / math.sqrt(H)
    w3 = rng.uniform(-1, 1, H) / math.sqrt(H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [-2.0],
                           [s_rho, s_pi, s_tau]]).astype(np.float32)


def training_set(snaps, r, tau_c, sample, rng):
    """Training pairs (rho, S, tau_t) from the snapshots of one fine run, `sample` cells per
    snapshot drawn without replacement."""
    rows = []
    for _, m in snaps:
        rho, u, T = filtered_fields(m, r)
        tau_t, S, _ = targets(rho, u, T, tau_c)
        n = rho.size
        idx = rng.choice(n, size=min(sample, n), replace=False)
        rows.append((rho.ravel()[idx], S.reshape(6, -1)[:, idx], tau_t.ravel()[idx]))
    rho = np.concatenate([a for a, _, _ in rows])
    S = np.concatenate([b for _, b, _ in rows], axis=1)
    tau = np.concatenate([c for _, _, c in rows])
    return rho, S, tau


def train(rho, S, tau, tau_c, iters, batch, lr, seed=0):
    """Train the closure network on the GPU; returns (params, loss history, scales)."""
    import torch
    pi = -(2.0 / 3.0) * rho * tau * S
    s_rho = 1.0 / max(float(np.std(rho)), 1e-12)
    s_pi = 1.0 / max(float(np.sqrt(np.mean(pi * pi))), 1e-12)
    s_tau = max(float(np.mean(tau - tau_c)), 1e-6)
    X = features(rho, S, tau, s_rho, s_pi)
    T = ((tau - tau_c) / s_tau).astype(np.float32)
    P0 = init_params(seed, s_rho, s_pi, s_tau)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    m = lbm.lbm_mlp_create(P0, batch, None)
    try:
        hist = lbm.lbm_mlp_train(m, Xd.data_ptr(), Td.data_ptr(), X.shape[0], batch, iters, lr)
        P = lbm.lbm_mlp_get_params(m)
    finally:
        lbm.lbm_mlp_destroy(m)
    return P, hist, dict(s_rho=s_rho, s_pi=s_pi, s_tau=s_tau)


def study(n_f=512, r=4, tau_c=0.502, coarse_steps=256, snap_every=32, train_seeds=range(1, 9), test_seed=9,
          kmax=None, umax=0.05, sample=65536, iters=3000, batch=16384, lr=2e-3, cs=0.17, log=print):
    """The whole study; returns a JSON-able dict of results."""
    import torch
    torch.cuda.set_device(0)
    kmax = kmax or n_f // 4
    N = n_f // r
    t0 = time.time()
    rng = np.random.default_rng(0)
    parts = []
    for seed in train_seeds:
        snaps = fine_run(n_f, r, seed, tau_c, coarse_steps, snap_every, kmax, umax)
        parts.append(training_set(snaps[1:], r, tau_c, sample, rng))
        log("fine run seed %d: %d snapshots (%.0f s)" % (seed, len(snaps), time.time() - t0))
    rho = np.concatenate([a for a, _, _ in parts])
    S = np.concatenate([b for _, b, _ in parts], axis=1)
    tau = np.concatenate([c for _, _, c in parts])
    P, hist, scales = train(rho, S, tau, tau_c, iters, batch, lr)
    log("trained on %d samples: loss %.4g -> %.4g; target nu_t mean %.3g, zero for %.1f %% of cells" % (
        tau.size, hist[0], hist[-1], (tau.mean() - tau_c) / 3, 100 * np.mean(tau == tau_c)))
    # test seed: fine reference and the three coarse runs from its filtered initial state
    snaps = fine_run(n_f, r, test_seed, tau_c, coarse_steps, snap_every, kmax, umax)
    ref = {t: filtered_fields(m, r) for t, m in snaps}
    rho0, u0, _ = ref[0]
    E_ref = {t: spectrum(v[1]) for t, v in ref.items()}
    res = {"config": dict(n_fine=n_f, ratio=r, n_coarse=N, tau_c=tau_c, tau_f=0.5 + r * (tau_c - 0.5),
                          coarse_steps=coarse_steps, snap_every=snap_every, train_seeds=list(train_seeds),
                          test_seed=test_seed, kmax=kmax, umax=umax, samples=int(tau.size), iters=iters,
                          batch=batch, lr=lr, cs=cs, scales=scales),
           "loss": [float(hist[0]), float(hist[-1])],
           "target_tau_mean": float(tau.mean()), "target_zero_fraction": float(np.mean(tau == tau_c)),
           "runs": {}}
    for name, cl in (("trt", None), ("smagorinsky", ("smag", cs)), ("mlp", ("mlp", P))):
        out, ms = coarse_run(rho0, u0, tau_c, coarse_steps, cl, snap_every)
        spec = {t: spectrum(u) for t, u in out if t > 0}
        errs = {t: spectrum_error(E, E_ref[t]) for t, E in spec.items()}
        lerrs = {t: log_spectrum_error(E, E_ref[t]) for t, E in spec.items()}
        final = out[-1][1]
        res["runs"][name] = {"ms_per_step": ms, "mlups": N ** 3 / ms / 1e3,
                             "spectrum_error": {str(t): e for t, e in errs.items()},
                             "spectrum_error_final": errs[coarse_steps],
                             "spectrum_error_mean": float(np.mean(list(errs.values()))),
                             "log_spectrum_error": {str(t): e for t, e in lerrs.items()},
                             "log_spectrum_error_final": lerrs[coarse_steps],
                             "log_spectrum_error_mean": float(np.mean(list(lerrs.values()))),
                             "energy": {str(t): float(0.5 * (u * u).sum()) for t, u in out},
                             "E_final": spec[coarse_steps].tolist(),
                             "finite": bool(np.isfinite(final).all())}
        log("%-12s %.3f ms/step  spectrum error final %.4f mean %.4f | log final %.4f mean %.4f" % (
            name, ms, errs[coarse_steps], res["runs"][name]["spectrum_error_mean"], lerrs[coarse_steps],
            res["runs"][name]["log_spectrum_error_mean"]))
    res["energy_ref"] = {str(t): float(0.5 * (v[1] ** 2).sum()) for t, v in ref.items()}
    res["E_ref_final"] = E_ref[coarse_steps].tolist()
    res["seconds"] = time.time() - t0
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--fine", type=int, default=512)
    ap.add_argument("--ratio", type=int, default=4)
    ap.add_argument("--tau", type=float, default=0.502)
    ap.add_argument("--steps", type=int, default=256, help="coarse steps")
    ap.add_argument("--snap", type=int, default=32, help="coarse steps between snapshots")
    ap.add_argument("--train-seeds", default="1-8")
    ap.add_argument("--test-seed", type=int, default=9)
    ap.add_argument("--sample", type=int, default=65536, help="training cells per snapshot")
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--umax", type=float, default=0.05)
    ap.add_argument("--kmax", type=int, default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    lo, _, hi = a.train_seeds.partition("-")
    seeds = range(int(lo), int(hi or lo) + 1)
    res = study(a.fine, a.ratio, a.tau, a.steps, a.snap, seeds, a.test_seed, kmax=a.kmax, umax=a.umax,
                sample=a.sample, iters=a.iters, batch=a.batch, lr=a.lr)
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")
    short = {k: v for k, v in res.items() if k != "E_ref_final"}
    short["runs"] = {k: {kk: vv for kk, vv in v.items() if kk != "E_final"} for k, v in res["runs"].items()}
    print(json.dumps(short, indent=1))


if __name__ == "__main__":
    main()
