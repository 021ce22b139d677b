"""Host-side analysis of the learned-closure study (CPU only): filtered fields, strain, the
least-squares eddy-viscosity target, features and the energy spectrum, each against a case
whose answer is known in closed form."""
import math

import numpy as np

from paper_1909_13772_gb300 import closure_study as cs


def _grid(n):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return x, y, z


def test_spectrum_of_single_modes_and_parseval():
    n = 16
    x, y, z = _grid(n)
    u = np.zeros((3, n, n, n))
    u[0] = 0.3 * np.sin(2 * math.pi * 3 * y / n)          # shell 3, energy 0.5 * 0.09 / 2
    u[1] = 0.2 * np.cos(2 * math.pi * (4 * x + 3 * z) / n)  # |k| = 5, energy 0.5 * 0.04 / 2
    E = cs.spectrum(u)
    assert abs(E[3] - 0.0225) < 1e-14 and abs(E[5] - 0.01) < 1e-14
    assert abs(E.sum() - 0.5 * (u * u).sum(axis=0).mean()) < 1e-14
    assert np.all(np.delete(E, [3, 5]) < 1e-28)
    # Nyquist mode along x (weight 1 in the half spectrum)
    v = np.zeros((3, n, n, n))
    v[2] = 0.1 * np.cos(math.pi * x)
    assert abs(cs.spectrum(v)[n // 2] - 0.5 * 0.01) < 1e-14


def test_strain_of_a_sine_shear_is_exact_central_difference():
    n = 12
    x, y, z = _grid(n)
    k = 2 * math.pi / n
    u = np.zeros((3, n, n, n))
    u[0] = np.sin(k * y)
    S = cs.strain(u)
    # central difference of sin: cos(k y) sin(k) (exact for the discrete operator)
    want = 0.5 * np.cos(k * y) * math.sin(k)
    assert np.allclose(S[3], want, atol=1e-15, rtol=0)
    assert np.all(np.delete(S, 3, axis=0) == 0)


def test_target_recovers_an_exact_eddy_viscosity():
    """T^d = -2 rho nu S^d everywhere gives nu back; the opposite sign (backscatter) clips to 0."""
    n, nu = 10, 3e-4
    rng = np.random.default_rng(2)
    u = 0.01 * rng.standard_normal((3, n, n, n))
    rho = 1.0 + 0.01 * rng.standard_normal((n, n, n))
    S = cs.strain(u)
    T = -2.0 * rho * nu * cs._dev(S)
    T[:3] += 0.1  # an isotropic part does not matter
    tau_t, S2, nu_t = cs.targets(rho, u, T, 0.502)
    # the local least-squares average of rho-weighted terms recovers nu where rho is constant
    # in the neighbourhood; here rho varies by 1 %, so within 5 %
    assert np.allclose(nu_t, nu, rtol=0.05)
    assert np.allclose(tau_t, 0.502 + 3 * nu_t)
    rho1 = np.ones((n, n, n))
    _, _, nu1 = cs.targets(rho1, u, -2.0 * nu * cs._dev(S), 0.502)
    assert np.allclose(nu1, nu, rtol=1e-12)
    _, _, nu2 = cs.targets(rho1, u, 2.0 * nu * cs._dev(S), 0.502)
    assert np.all(nu2 == 0)


def test_filtered_fields_from_box_sums():
    """Box sums of a field whose cells share one velocity give that velocity and zero stress;
    two velocities in one box give the Favre-filtered stress rho_a rho_b (du)^2 / (rho_a + rho_b)^2."""
    m = np.zeros((10, 1, 1, 1))
    r = 2
    rho_c = np.array([1.0] * 4 + [1.2] * 4)
    u_c = np.array([0.01] * 4 + [0.03] * 4)
    m[0] = rho_c.sum()
    m[1] = (rho_c * u_c).sum()
    m[4] = (rho_c * u_c * u_c).sum()
    rho, u, T = cs.filtered_fields(m, r)
    rb = rho_c.mean()
    ub = (rho_c * u_c).mean() / rb
    assert abs(rho[0, 0, 0] - rb) < 1e-15 and abs(u[0, 0, 0, 0] - ub) < 1e-15
    want = (rho_c * (u_c - ub) ** 2).mean()
    assert abs(T[0, 0, 0, 0] - want) < 1e-17
    assert np.all(T[1:] == 0)


def test_features_follow_chapman_enskog_stress():
    rho = np.array([[[1.01]]])
    S = np.arange(6, dtype=float).reshape(6, 1, 1, 1) * 1e-3
    X = cs.features(rho, S, np.array([[[0.51]]]), 10.0, 100.0)
    assert X.shape == (1, 7) and X.dtype == np.float32
    assert abs(X[0, 0] - 0.1) < 1e-6
    assert np.allclose(X[0, 1:], -(2 / 3) * 1.01 * 0.51 * S.ravel() * 100.0, rtol=1e-6)


def test_initial_network_layout():
    P = cs.init_params(3, 1.0, 2.0, 3.0)
    assert P.shape == (cs.MLP_NPARAM,) and P.dtype == np.float32
    assert list(P[-3:]) == [1.0, 2.0, 3.0] and P[-4] == -2.0
