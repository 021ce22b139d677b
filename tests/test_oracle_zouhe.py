"""Pins for the oracle's wet-node (Zou-He) velocity and pressure faces, CPU only.

  * The reconstruction's defining constraints, checked on the pre-collision field of random
    states (orc_stream): at every boundary node the populations carry exactly the imposed
    momentum j = rho u_w - F/2 (velocity face) or the imposed density with zero tangential
    velocity (pressure face), while every other cell is untouched by the pass.
  * Flows whose exact solutions the wet-node walls reproduce: plane Couette flow between a wall
    node at rest and a moving one, u_x(y) = u_w y / (H - 1), and plane Poiseuille flow between two
    walls at rest driven by a body force, u_x(y) = F / (2 nu) y (H - 1 - y), with the walls at the
    nodes (y = 0 and H - 1), for SRT and TRT at several rates; halfway bounce-back walls, one cell
    further out, miss that parabola (negative control).
  * A uniform flow between a velocity inlet and a pressure outlet is a fixed point.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1909_13772_gb300 import inputs

ZV, ZP = oracle.ZOUHE_VELOCITY, oracle.ZOUHE_PRESSURE


def _channel(H, coll, omega, F=(0.0, 0.0, 0.0), top_u=0.0, kinds=(ZV, ZV)):
    fu = [(0.0, 0.0, 0.0)] * 6
    fu[3] = (top_u, 0.0, 0.0)
    return oracle.OracleParams(shape=(1, H, 1), q=19, collision=coll, omega=omega, force=F, periodic=(1, 0, 1),
                               face_kind=(1, 1, kinds[0], kinds[1], 1, 1), face_u=tuple(fu))


def _steady(p, H):
    nu = (1 / p.omega - 0.5) / 3
    rho, u = inputs.rest((1, H, 1))
    return oracle.run(p, oracle.init(p, rho, u), int(60 / (nu * (math.pi / H) ** 2)))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reconstruction_imposes_the_boundary_moments(axis):
    shape = [6, 7, 5]
    shape[axis] = 9
    shape = tuple(shape)
    c, _, _ = oracle.lattice(19)
    uw = np.array([0.02, -0.01, 0.015])
    F = np.array([2e-5, -1e-5, 3e-5])
    periodic = [1, 1, 1]
    periodic[axis] = 0
    kinds = [1] * 6
    kinds[2 * axis], kinds[2 * axis + 1] = ZV, ZP
    fu = [(0.0, 0.0, 0.0)] * 6
    fu[2 * axis] = tuple(uw)
    frho = [1.0] * 6
    frho[2 * axis + 1] = 1.01
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1.3, force=tuple(F),
                            periodic=tuple(periodic), face_kind=tuple(kinds), face_u=tuple(fu), face_rho=tuple(frho))
    rho, u = inputs.random_state(shape, seed=17, rho_amp=0.02, u_amp=0.03)
    f = oracle.init(p, rho, u)
    pre = oracle.stream(p, f)
    plain = oracle.stream(oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1.3, force=tuple(F),
                                              periodic=tuple(periodic), face_kind=(1,) * 6), f)
    sl = [slice(None)] * 3
    for side, layer in ((0, 0), (1, shape[axis] - 1)):
        sl[2 - axis] = layer
        g = pre[(slice(None),) + tuple(sl)].reshape(19, -1)
        r = g.sum(0)
        j = np.einsum("ia,in->an", c.astype(float), g)
        if side == 0:  # velocity face: j = rho u_w - F/2
            want = r[None] * uw[:, None] - F[:, None] / 2
            assert np.abs(j - want).max() < 1e-15
        else:  # pressure face: rho = rho_w, tangential velocity zero
            assert np.abs(r - 1.01).max() < 1e-15
            t = [b for b in range(3) if b != axis]
            assert np.abs(j[t] + F[t, None] / 2).max() < 1e-15
    # the pass touches only the incoming populations of the boundary nodes
    inner = [slice(None)] * 3
    inner[2 - axis] = slice(1, shape[axis] - 1)
    np.testing.assert_array_equal(pre[(slice(None),) + tuple(inner)], plain[(slice(None),) + tuple(inner)])


@pytest.mark.parametrize("coll,omega", [(oracle.SRT, 1.0), (oracle.SRT, 1.6), (oracle.TRT, 1.6), (oracle.TRT, 0.7)])
def test_couette_between_wet_node_walls_is_exact(coll, omega):
    H, uw = 12, 0.01
    f = _steady(_channel(H, coll, omega, top_u=uw), H)
    _, v = oracle.macroscopic(_channel(H, coll, omega, top_u=uw), f)
    y = np.arange(H)
    assert np.abs(v[0, 0, :, 0] - uw * y / (H - 1)).max() < 2e-12 * uw


@pytest.mark.parametrize("coll,omega", [(oracle.SRT, 1.0), (oracle.SRT, 1.6), (oracle.TRT, 1.6), (oracle.TRT, 0.7)])
def test_poiseuille_between_wet_node_walls_is_exact(coll, omega):
    H, F = 12, 1e-4
    nu = (1 / omega - 0.5) / 3
    p = _channel(H, coll, omega, F=(F, 0.0, 0.0))
    r, v = oracle.macroscopic(p, _steady(p, H))
    y = np.arange(H)
    want = F / (2 * nu) * y * (H - 1 - y)
    assert np.abs(v[0, 0, :, 0] - want).max() < 2e-12 * want.max()
    assert r.max() - r.min() < 1e-13


def test_halfway_walls_miss_the_wet_node_parabola():
    H, F, omega = 12, 1e-4, 1.0
    nu = (1 / omega - 0.5) / 3
    p = _channel(H, oracle.TRT, omega, F=(F, 0.0, 0.0), kinds=(oracle.NOSLIP, oracle.NOSLIP))
    _, v = oracle.macroscopic(p, _steady(p, H))
    y = np.arange(H)
    want = F / (2 * nu) * y * (H - 1 - y)
    assert np.abs(v[0, 0, :, 0] - want).max() > 0.05 * want.max()


def test_uniform_flow_between_inlet_and_outlet_is_a_fixed_point():
    shape, u0 = (10, 4, 3), 0.03
    fu = [(0.0, 0.0, 0.0)] * 6
    fu[0] = (u0, 0.0, 0.0)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1.2, periodic=(0, 1, 1),
                            face_kind=(ZV, ZP, 1, 1, 1, 1), face_u=tuple(fu), face_rho=(1.0,) * 6)
    rho = np.ones(shape[::-1])
    u = np.zeros((3,) + shape[::-1])
    u[0] = u0
    f0 = oracle.init(p, rho, u)
    f = oracle.run(p, f0, 200)
    assert np.abs(f - f0).max() < 1e-14


def test_zou_he_faces_need_d3q19():
    p = oracle.OracleParams(shape=(6, 4, 3), q=27, collision=oracle.TRT, omega=1.2, periodic=(0, 1, 1),
                            face_kind=(ZV, ZP, 1, 1, 1, 1))
    rho, u = inputs.rest((6, 4, 3))
    with pytest.raises(RuntimeError):
        oracle.run(p, oracle.init(p, rho, u), 1)
