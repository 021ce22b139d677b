"""Pins for the oracle's static 2:1 grid refinement (Sec. 5.1.1: the mass-conserving method of
Rohde et al. for non-uniform grids), CPU only.

What fixes the result, independently of the oracle's explosion / coalescence code:
  * conservation: the volume-weighted mass sum_coarse f + (1/8) sum_fine f stays constant to
    rounding over many steps from a random state, and so does the momentum without a force; with
    a body force the momentum grows by exactly F per coarse cell volume and coarse step;
  * a uniform flow (equilibrium on both grids) is a fixed point;
  * physics: a shear wave whose variation runs across the refined columns decays at nu k^2 with
    the coarse grid's nu = (tau_c - 1/2)/3, as on a uniform grid -- which needs the fine grid's
    rate (tau_f - 1/2 = 2 (tau_c - 1/2)), two fine steps per coarse step and a transfer at the
    interface that neither loses nor double-counts populations;
  * the velocity field is continuous across the interfaces (the coarse cells next to the refined
    columns and the fine cells next to them follow the same sine).
"""
import math

import numpy as np
import pytest

import oracle


def _setup(q=19, coll=oracle.TRT, tau=0.8, shape=(24, 4, 4), a=8, b=16, force=(0.0, 0.0, 0.0)):
    p = oracle.OracleParams(shape=shape, q=q, collision=coll, omega=1 / tau, periodic=(1, 1, 1), force=force)
    return p, oracle.refine_fine_params(p, a, b), a, b


def _mass_mom(fc, ff, q):
    c, _, _ = oracle.lattice(q)
    sc, sf = fc.reshape(q, -1).sum(1), ff.reshape(q, -1).sum(1)
    return sc.sum() + sf.sum() / 8.0, c.T @ sc + c.T @ sf / 8.0


def _random(p, pf, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = p.shape
    nf, nyf, nzf = pf.shape
    return (1 + 0.01 * rng.standard_normal((nz, ny, nx)), 0.02 * rng.standard_normal((3, nz, ny, nx)),
            1 + 0.01 * rng.standard_normal((nzf, nyf, nf)), 0.02 * rng.standard_normal((3, nzf, nyf, nf)))


def test_fine_parameters_follow_acoustic_scaling():
    p, pf, a, b = _setup(tau=0.8, force=(1e-5, 0.0, -2e-5))
    assert pf.shape == (16, 8, 8)
    assert abs(1 / pf.omega - (0.5 + 2 * 0.3)) < 1e-15
    assert pf.force == (5e-6, 0.0, -1e-5)
    with pytest.raises(ValueError):
        oracle.refine_fine_params(oracle.OracleParams(shape=(24, 4, 4), collision=oracle.MRT), 8, 16)
    with pytest.raises(ValueError):
        oracle.refine_fine_params(oracle.OracleParams(shape=(24, 4, 4), periodic=(1, 0, 1)), 8, 16)


@pytest.mark.parametrize("q,coll", [(19, oracle.TRT), (27, oracle.SRT)])
def test_mass_and_momentum_are_conserved(q, coll):
    p, pf, a, b = _setup(q=q, coll=coll, tau=0.7)
    fc, ff = oracle.refine_init(p, a, b, *_random(p, pf, 1))
    m0, j0 = _mass_mom(fc, ff, q)
    fc, ff = oracle.refine_run(p, a, b, fc, ff, 60)
    m1, j1 = _mass_mom(fc, ff, q)
    assert abs(m1 - m0) <= 1e-14 * 60 * m0
    assert np.abs(j1 - j0).max() <= 1e-14 * 60 * m0


def test_body_force_adds_F_per_coarse_volume_and_step():
    F = (2e-5, -1e-5, 3e-5)
    p, pf, a, b = _setup(force=F)
    fc, ff = oracle.refine_init(p, a, b, *_random(p, pf, 2))
    _, j0 = _mass_mom(fc, ff, 19)
    steps = 40
    fc, ff = oracle.refine_run(p, a, b, fc, ff, steps)
    m1, j1 = _mass_mom(fc, ff, 19)
    vol = np.prod(p.shape)
    assert np.abs(j1 - j0 - steps * vol * np.array(F)).max() <= 1e-13 * m1


def test_uniform_flow_is_a_fixed_point():
    p, pf, a, b = _setup(q=27, coll=oracle.TRT)
    nx, ny, nz = p.shape
    nf, nyf, nzf = pf.shape
    u0 = np.array([0.03, -0.01, 0.02])
    fc, ff = oracle.refine_init(p, a, b, np.full((nz, ny, nx), 1.01), np.broadcast_to(u0[:, None, None, None], (3, nz, ny, nx)),
                                np.full((nzf, nyf, nf), 1.01), np.broadcast_to(u0[:, None, None, None], (3, nzf, nyf, nf)))
    fc2, ff2 = oracle.refine_run(p, a, b, fc, ff, 10)
    assert np.abs(fc2 - fc).max() <= 1e-15 and np.abs(ff2 - ff).max() <= 1e-15


@pytest.mark.parametrize("coll,tau", [(oracle.TRT, 0.8), (oracle.SRT, 0.6), (oracle.TRT, 0.55)])
def test_shear_wave_across_the_refined_columns_decays_at_the_viscous_rate(coll, tau):
    nx, a, b = 48, 16, 32
    p, pf, a, b = _setup(coll=coll, tau=tau, shape=(nx, 2, 2), a=a, b=b)
    nf, nyf, nzf = pf.shape
    A, k = 1e-3, 2 * math.pi / nx
    xc = np.arange(nx) + 0.5                 # coarse cell centres
    xf = a + (np.arange(nf) + 0.5) / 2.0     # fine cell centres, coarse units
    uc = np.zeros((3, 2, 2, nx))
    uc[1] = A * np.sin(k * xc)
    uf = np.zeros((3, nzf, nyf, nf))
    uf[1] = A * np.sin(k * xf)
    fc, ff = oracle.refine_init(p, a, b, np.ones((2, 2, nx)), uc, np.ones((nzf, nyf, nf)), uf)
    coarse = ((np.arange(nx) - a) % nx) >= (b - a)
    flags = oracle.refine_slab_flags(p, a, b)

    def profiles(fc, ff):
        _, u1 = oracle.macroscopic(p, fc, flags=flags)
        _, u2 = oracle.macroscopic(pf, ff)
        return u1[1].mean(axis=(0, 1)), u2[1].mean(axis=(0, 1))

    def amp(fc, ff):
        vc, vf = profiles(fc, ff)
        num = (vc * np.sin(k * xc))[coarse].sum() + 0.5 * (vf * np.sin(k * xf)).sum()
        den = (np.sin(k * xc) ** 2)[coarse].sum() + 0.5 * (np.sin(k * xf) ** 2).sum()
        return num / den

    s1 = oracle.refine_run(p, a, b, fc, ff, 200)
    s2 = oracle.refine_run(p, a, b, s1[0], s1[1], 400)
    rate = math.log(amp(*s1) / amp(*s2)) / 400
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1.0) < 3e-3
    # continuity: both grids follow the decayed sine, the interface cells included
    vc, vf = profiles(*s2)
    a2 = amp(*s2)
    assert np.abs(vc[coarse] - a2 * np.sin(k * xc[coarse])).max() <= 0.01 * a2
    assert np.abs(vf - a2 * np.sin(k * xf)).max() <= 0.01 * a2
