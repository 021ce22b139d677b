"""Host check of the error bounds stated for the step diagnostics of FP32 sweeps (include/lbm.h,
lbm_step_diagnostics): the arithmetic scheme of a CTA's record, restated with NumPy float32 on
random stored values, against exact sums (math.fsum).  Mass: per cell a Fast2Sum chain over the
stored values, per thread TwoSum across its n cells (low parts added in FP32), per CTA a
butterfly over each warp and the warps in order, high parts by TwoSum and low parts in FP32:
within (Q + n + 3)^2 u^2 of the mass, for states whose rest population is at least every other
one (the chains' Fast2Sum precondition).  Momentum-like sums: per thread Kahan's compensated
sum, the pair's difference, then the same 12 pairwise FP32 additions: within 9 u sum |x|."""
import math

import numpy as np

F = np.float32
U = 2.0 ** -24


def two_sum(s, x):
    t = (s + x).astype(F)
    b = (t - s).astype(F)
    e = ((s - (t - b)) + (x - b)).astype(F)
    return t, e


def cta_mass(vals, rho0=0.0):
    """vals[cell, thread, q] (float32) -> the record's mass (float64) by the stated scheme."""
    ncell, nthr, q = vals.shape
    hi = np.zeros(nthr, F)
    lo = np.zeros(nthr, F)
    for c in range(ncell):
        m = np.full(nthr, rho0, F)
        e = np.zeros(nthr, F)
        for i in range(q):
            x = vals[c, :, i]
            t = (m + x).astype(F)
            e = (e + (x - (t - m))).astype(F)  # Fast2Sum error, accumulated in FP32
            m = t
        hi, eh = two_sum(hi, m)
        lo = (lo + (eh + e)).astype(F)
    # butterfly over each warp of 32 threads (every lane ends with the same pair)
    hi = hi.reshape(-1, 32)
    lo = lo.reshape(-1, 32)
    o = 16
    while o:
        idx = np.arange(32) ^ o
        bh, bl = hi[:, idx], lo[:, idx]
        hi, e = two_sum(hi, bh)
        lo = ((lo + bl) + e).astype(F)
        o >>= 1
    th, tl = hi[0, 0], lo[0, 0]
    for w in range(1, hi.shape[0]):
        th, e = two_sum(np.array([th], F), np.array([hi[w, 0]], F))
        tl = ((np.array([tl], F) + F(lo[w, 0])) + e).astype(F)
        th, tl = th[0], tl[0]
    return float(th) + float(tl)


def cta_sum(x):
    """x[cell, thread] (float32) -> Kahan per thread, the pair's difference, pairwise per CTA."""
    s = np.zeros(x.shape[1], F)
    c = np.zeros(x.shape[1], F)
    for k in range(x.shape[0]):
        y = (x[k] - c).astype(F)
        t = (s + y).astype(F)
        c = ((t - s) - y).astype(F)
        s = t
    v = (s - c).astype(F).reshape(-1, 32)
    o = 16
    while o:
        v = (v + v[:, np.arange(32) ^ o]).astype(F)
        o >>= 1
    t = v[0, 0]
    for w in range(1, v.shape[0]):
        t = F(t + v[w, 0])
    return float(t)


def _populations(rng, ncell, noise):
    """Stored D3Q19 populations near equilibrium: w_i rho (1 + noise g), with the rest
    population kept at least every other population (the stated precondition)."""
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    rho = 1.0 + 0.05 * rng.standard_normal((ncell, 256, 1))
    f = w * rho * (1.0 + noise * rng.standard_normal((ncell, 256, 19)))
    f[..., 0] = np.maximum(f[..., 0], f[..., 1:].max(axis=-1))
    return f.astype(F)


def test_mass_record_within_stated_bound():
    rng = np.random.default_rng(5)
    q = 19
    for n in (4, 8, 16, 32):
        for noise in (0.02, 0.3):
            vals = _populations(rng, n, noise)
            got = cta_mass(vals)
            exact = math.fsum(vals.astype(np.float64).ravel())
            rel = abs(got - exact) / exact
            assert rel <= (q + n + 3) ** 2 * U * U, (n, noise, rel / (U * U))


def test_mass_record_of_deviations_within_stated_bound():
    # 16-bit storages: the chain starts at rho0 and adds the stored deviations f_i - w_i rho0
    rng = np.random.default_rng(6)
    q = 19
    vals = (1e-3 * rng.standard_normal((4, 256, q))).astype(F)
    got = cta_mass(vals, rho0=1.0)
    exact = math.fsum(vals.astype(np.float64).ravel()) + 4 * 256 * 1.0
    assert abs(got - exact) / exact <= (q + 4 + 3) ** 2 * U * U


def test_momentum_record_within_stated_bound():
    rng = np.random.default_rng(7)
    for ncell in (4, 16, 64):
        x = (0.05 * rng.standard_normal((ncell, 256)) * (1.0 + rng.random((ncell, 256)))).astype(F)
        got = cta_sum(x)
        exact = math.fsum(x.astype(np.float64).ravel())
        assert abs(got - exact) <= 9 * U * float(np.abs(x.astype(np.float64)).sum())


def test_bound_would_catch_a_plain_float32_sum():
    # negative control: summing the stored values in plain FP32 breaks the mass bound
    rng = np.random.default_rng(8)
    vals = _populations(rng, 32, 0.05)
    plain = F(0)
    for v in vals.ravel():
        plain = F(plain + v)
    exact = math.fsum(vals.astype(np.float64).ravel())
    assert abs(float(plain) - exact) / exact > (19 + 32 + 3) ** 2 * U * U
