"""The porous-bed workload at its full size: 16^3 = 4096 uneven blocks (edges log-uniform in
[16, 64], default_rng(4096)), the Boolean sphere packing (R = 8, porosity 0.40,
default_rng(7)), velocity inlet u = (0.02, 0, 0) at x-, pressure outlet rho = 1 at x+, periodic
y and z, D3Q19 TRT tau = 0.8, FP32 -- 604 x 644 x 580 cells.  Three steps from a smooth seeded
state (two of them replayed as a CUDA graph for the two-grid pattern), then five 8^3 regions
against the oracle run on each region's neighbourhood: at the inlet, at the outlet, at an
interior block corner (the neighbourhood spans eight blocks), at the periodic corner where y and
z wrap, and around a sphere surface.

After s steps a value depends only on cells within s of it, so the oracle runs on the region
widened by 3 cells (clipped at the inlet and outlet faces, wrapped in y and z); the faces of
that box that cut through the domain take no-slip, whose wrong values travel one cell per step
and stay in the widening.  Gates: PDFs 1e-5 of max|f| and the derived flow gates."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, flow_gates
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

STEPS, H = 3, 3


def _state(x, y, z):
    """Smooth seeded initial density and velocity at global cell coordinates (periodic in y, z
    with the domain's periods, so the wrapped neighbourhoods see the same field)."""
    ny, nz = 644, 580
    ky, kz = 2 * math.pi * 7 / ny, 2 * math.pi * 5 / nz
    rho = 1.0 + 0.01 * np.sin(0.11 * x + 0.3) * np.cos(ky * y) + 0.005 * np.cos(kz * z + 0.7)
    u = np.stack([0.02 + 0.01 * np.sin(ky * y + 0.2) * np.cos(0.07 * x),
                  0.008 * np.cos(kz * z) * np.sin(0.05 * x + 1.0),
                  0.008 * np.sin(ky * y + kz * z)])
    return rho, u


@pytest.fixture(scope="module")
def geometry():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(16, 16, 16), lo=16, hi=64, seed=4096)
    flags = inputs.sphere_packing(shape, radius=8.0, porosity=0.40, seed=7)
    assert shape == (604, 644, 580)
    return blocks, shape, flags


def _regions(blocks, shape, flags):
    """(block, origin in the block, global origin) of the five 8^3 regions."""
    nx, ny, nz = shape

    def block_at(gx, gy, gz):
        for b, (o, s) in enumerate(blocks):
            if all(o[a] <= g < o[a] + s[a] for a, g in enumerate((gx, gy, gz))):
                return b
        raise AssertionError

    out = []
    # inlet: x = 0; outlet: the last 8 cells in x
    for gx in (0, nx - 8):
        g = (gx, 301, 277)
        out.append((block_at(*g), g))
    # interior block corner: the high corner of a middle block
    b = block_at(nx // 2, ny // 2, nz // 2)
    o, s = blocks[b]
    out.append((b, tuple(o[a] + s[a] - 8 for a in range(3))))
    # the periodic corner y = z = 0 (its neighbourhood wraps in y and z)
    g = (317, 0, 0)
    out.append((block_at(*g), g))
    # a region cut by a sphere surface: first candidate with between 20 % and 80 % fluid
    for gz in range(40, nz - 48, 24):
        g = (nx // 3, 200, gz)
        bb = block_at(*g)
        o, s = blocks[bb]
        g = tuple(min(max(g[a], o[a]), o[a] + s[a] - 8) for a in range(3))
        frac = (flags[g[2]:g[2] + 8, g[1]:g[1] + 8, g[0]:g[0] + 8] == 0).mean()
        if 0.2 < frac < 0.8:
            out.append((bb, g))
            break
    assert len(out) == 5
    return [(b, tuple(g[a] - blocks[b][0][a] for a in range(3)), g) for b, g in out]


def _oracle_region(shape, flags, g, pattern_omega):
    nx, ny, nz = shape
    x0, x1 = max(g[0] - H, 0), min(g[0] + 8 + H, nx)
    ix = np.arange(x0, x1)
    iy = np.arange(g[1] - H, g[1] + 8 + H) % ny
    iz = np.arange(g[2] - H, g[2] + 8 + H) % nz
    sub = np.ascontiguousarray(flags[np.ix_(iz, iy, ix)])
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    rho, u = _state(X.astype(np.float64), Y.astype(np.float64), Z.astype(np.float64))
    faces = (lbm.VELOCITY if x0 == 0 else lbm.NOSLIP, lbm.PRESSURE if x1 == nx else lbm.NOSLIP,
             lbm.NOSLIP, lbm.NOSLIP, lbm.NOSLIP, lbm.NOSLIP)
    p = oracle.OracleParams(shape=(len(ix), len(iy), len(iz)), q=19, collision=oracle.TRT, omega=pattern_omega,
                            magic_lambda=3 / 16, periodic=(0, 0, 0), face_kind=faces,
                            face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5)
    f = oracle.run(p, oracle.init(p, rho, u, flags=sub), STEPS, flags=sub)
    lx = g[0] - x0
    return f[:, H:H + 8, H:H + 8, lx:lx + 8], sub[H:H + 8, H:H + 8, lx:lx + 8] == 0


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_full_size_porous_bed_regions_match_oracle(geometry, pattern):
    import torch
    blocks, shape, flags = geometry
    omega = 1 / 0.8
    p = lbm.make_params(stencil=19, collision=lbm.TRT, storage=lbm.FP32, pattern=pattern, omega=omega,
                        magic_lambda=3 / 16, periodic=(0, 1, 1))
    stream = torch.cuda.Stream()
    sim = lbm.Simulation(p, blocks, stream=stream.cuda_stream)
    regions = _regions(blocks, shape, flags)
    try:
        sim.set_face(0, 0, lbm.VELOCITY, (0.02, 0.0, 0.0), 1.0)
        sim.set_face(0, 1, lbm.PRESSURE, (0.0, 0.0, 0.0), 1.0)
        for b, (o, sz) in enumerate(sim.blocks):
            sub = flags[o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]]
            sim.set_boundary(b, sub if sub.any() else None)
        for b, (o, sz) in enumerate(sim.blocks):
            Z, Y, X = np.meshgrid(np.arange(o[2], o[2] + sz[2]), np.arange(o[1], o[1] + sz[1]),
                                  np.arange(o[0], o[0] + sz[0]), indexing="ij")
            rho, u = _state(X.astype(np.float64), Y.astype(np.float64), Z.astype(np.float64))
            sim.init(b, rho, u)
        if pattern == lbm.TWO_GRID:
            lbm.lbm_set_graph(sim.ctx, True)
        sim.step(STEPS)
        got = [sim.pdfs_region(b, lo, (8, 8, 8)) for b, lo, _ in regions]
    finally:
        sim.close()
    for (b, lo, g), gr in zip(regions, got):
        want, fluid = _oracle_region(shape, flags, g, omega)
        assert fluid.any()
        err = np.abs(gr - want)[:, fluid].max() / np.abs(want[:, fluid]).max()
        assert err <= TOL[lbm.FP32], (g, err)
        assert np.all(gr[:, ~fluid] == 0)
        flow_gates(gr, want, lbm.FP32, STEPS, 19, fluid)
