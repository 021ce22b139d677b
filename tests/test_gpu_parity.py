"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Gate: normwise max relative PDF error <= 1e-12 (FP64 storage) and <= 1e-5 (FP32
storage), max_x,i |gpu - oracle| / max_x,i |oracle| over fluid cells.  Sizes span several
sweep tiles plus a ragged tail in every axis."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, Case, flow_gates, gather_macro, gather_pdfs, init_sim, normwise, oracle_run, split
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _compare(case, rho, u, steps, tol=None):
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(steps)
    got = gather_pdfs(sim, case)
    _, want = oracle_run(case, rho, u, steps)
    fl = case.global_flags() == 0
    err = normwise(got, want, fl)
    sim.close()
    assert err <= (tol or TOL[case.storage]), err
    if tol is None:
        flow_gates(got, want, case.storage, steps, case.q, fl)
    return got, want, err


# ---- C1: Taylor-Green vortex, D3Q19 SRT, 32^3, FP64, 100 steps ---------------------------
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_taylor_green_fp64_matches_oracle_and_decay(pattern):
    n, tau, steps = 32, 0.6, 100
    case = Case(shape=(n, n, n), q=19, collision=lbm.SRT, storage=lbm.FP64, pattern=pattern, omega=1 / tau)
    rho, u = inputs.taylor_green(n, u0=0.01)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(20)
    v20 = gather_macro(sim, case)[1]
    sim.step(steps - 20)
    got = gather_pdfs(sim, case)
    v100 = gather_macro(sim, case)[1]
    sim.close()
    _, want = oracle_run(case, rho, u, steps)
    assert normwise(got, want) <= 1e-12
    k = 2 * math.pi / n
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    mode = np.cos(k * X) * np.sin(k * Y)
    amp = lambda v: (v[0] * mode[None]).sum() / (mode * mode).sum() / n  # noqa: E731
    rate = -math.log(amp(v100) / amp(v20)) / (steps - 20)
    nu = (tau - 0.5) / 3
    assert abs(rate / (2 * nu * k * k) - 1) < 5e-3


# ---- channel with walls and body force (C2 family), several tiles + ragged tails -----------
@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("q", [19, 27])
def test_channel_trt_force(storage, pattern, q):
    shape = (70, 37, 11)
    case = Case(shape=shape, q=q, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1.0,
                force=(1e-5, 0.0, 0.0), periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho, u = inputs.random_state(shape, seed=21, rho_amp=0.02, u_amp=0.03)
    _compare(case, rho, u, 40)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("collision", [lbm.SRT, lbm.TRT])
def test_periodic_random_state(storage, collision):
    shape = (45, 19, 13)
    case = Case(shape=shape, q=27, collision=collision, storage=storage, omega=1.7, magic_lambda=0.25,
                force=(2e-6, -1e-6, 3e-6))
    rho, u = inputs.random_state(shape, seed=5)
    _compare(case, rho, u, 30)


def _porous_case(storage, pattern, q=19):
    """Uneven multi-block layout, spheres, velocity inlet at x-, pressure outlet at x+."""
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    return Case(shape=shape, blocks=blocks, q=q, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1 / 0.8,
                periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags)


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_porous_multiblock(storage, pattern):
    case = _porous_case(storage, pattern)
    rho, u = inputs.rest(case.shape)
    _compare(case, rho, u, 60)


def test_porous_multiblock_d3q27():
    case = _porous_case(lbm.FP64, lbm.AA, q=27)
    rho, u = inputs.rest(case.shape)
    _compare(case, rho, u, 25)


# ---- pure streaming: omega = 0 and F = 0 make lbm_step a permutation -- bitwise ----------
@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("q", [19, 27])
def test_pure_streaming_bitwise(storage, pattern, q):
    case = _porous_case(storage, pattern, q=q)
    case.collision = lbm.SRT
    case.omega = 0.0
    case.faces = (lbm.NOSLIP, lbm.NOSLIP, 1, 1, 1, 1)
    nx, ny, nz = case.shape
    fl = case.global_flags() == 0
    rng = np.random.default_rng(3)
    f0 = rng.random((q, nz, ny, nx))
    if storage == lbm.FP32:
        f0 = f0.astype(np.float32).astype(np.float64)
    f0[:, ~fl] = 0.0
    sim = case.make_sim()
    for b, (o, s) in enumerate(sim.blocks):
        sim.set_pdfs(b, f0[:, o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]])
    sim.step(3)
    got = gather_pdfs(sim, case)
    sim.close()
    want = oracle.run(case.oracle_params(), f0, 3, flags=case.global_flags())
    np.testing.assert_array_equal(got[:, fl], want[:, fl])


# ---- checkpoint / restart and determinism ------------------------------------------------
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("split_at", [4, 5])
def test_checkpoint_restart_bitwise(pattern, split_at):
    case = _porous_case(lbm.FP32, pattern)
    rho, u = inputs.random_state(case.shape, seed=9, rho_amp=0.01, u_amp=0.01)
    a = case.make_sim()
    init_sim(a, rho, u)
    a.step(10)
    want = gather_pdfs(a, case)
    a.close()
    b = case.make_sim()
    init_sim(b, rho, u)
    b.step(split_at)
    saved = [b.pdfs(k) for k in range(len(b.blocks))]
    b.close()
    c = case.make_sim()
    for k, f in enumerate(saved):
        c.set_pdfs(k, f)
    c.step(10 - split_at)
    got = gather_pdfs(c, case)
    c.close()
    np.testing.assert_array_equal(got, want)


def test_aa_equals_two_grid():
    base = _porous_case(lbm.FP64, lbm.TWO_GRID)
    rho, u = inputs.rest(base.shape)
    out = []
    for pattern in (lbm.TWO_GRID, lbm.AA):
        base.pattern = pattern
        s = base.make_sim()
        init_sim(s, rho, u)
        s.step(7)
        out.append(gather_pdfs(s, base))
        s.close()
    assert normwise(out[1], out[0], base.global_flags() == 0) <= 1e-14


def test_tile_shape_does_not_change_results():
    case = Case(shape=(70, 21, 9), q=19, storage=lbm.FP32, force=(1e-5, 0, 0), periodic=(1, 0, 1),
                faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho, u = inputs.random_state(case.shape, seed=2, rho_amp=0.01, u_amp=0.02)
    res = []
    for tile in ((32, 1, 1), (64, 4, 4), (128, 2, 3), (256, 1, 8)):
        case.tile = tile
        s = case.make_sim()
        init_sim(s, rho, u)
        s.step(12)
        res.append(gather_pdfs(s, case))
        s.close()
    for r in res[1:]:
        np.testing.assert_array_equal(r, res[0])


# ---- reductions and failure detection ----------------------------------------------------
def test_reduction_matches_oracle_and_is_deterministic():
    case = _porous_case(lbm.FP64, lbm.TWO_GRID)
    rho, u = inputs.random_state(case.shape, seed=12, rho_amp=0.02, u_amp=0.02)
    s = case.make_sim()
    init_sim(s, rho, u)
    s.step(5)
    d1, d2 = s.reduce(), s.reduce()
    s.close()
    assert d1 == d2
    _, f = oracle_run(case, rho, u, 5)
    want = oracle.diagnostics(case.oracle_params(), f, case.global_flags())
    assert abs(d1["mass"] / want["mass"] - 1) < 1e-13
    np.testing.assert_allclose(d1["momentum"], want["momentum"], rtol=1e-10, atol=1e-14)
    assert abs(d1["kinetic_energy"] / want["kinetic_energy"] - 1) < 1e-10
    assert abs(d1["max_speed"] / want["max_speed"] - 1) < 1e-10
    assert d1["nonfinite"] == 0
    assert d1["fluid_cells"] == int((case.global_flags() == 0).sum())


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_per_block_reduction_matches_oracle(pattern):
    """lbm_reduce_blocks: each block's record against the oracle's moments over that block's
    region; the records add up to lbm_reduce."""
    case = _porous_case(lbm.FP64, pattern)
    rho, u = inputs.random_state(case.shape, seed=13, rho_amp=0.02, u_amp=0.02)
    s = case.make_sim()
    init_sim(s, rho, u)
    s.step(5)
    per = s.reduce_blocks()
    tot = s.reduce()
    blocks = s.blocks
    s.close()
    _, f = oracle_run(case, rho, u, 5)
    orho, ou = oracle.macroscopic(case.oracle_params(), f, case.global_flags())
    fluid = case.global_flags() == 0
    assert per.shape == (len(blocks), 8)
    for b, (o, sz) in enumerate(blocks):
        sl = (slice(o[2], o[2] + sz[2]), slice(o[1], o[1] + sz[1]), slice(o[0], o[0] + sz[0]))
        fl, r, v = fluid[sl], orho[sl], ou[(slice(None),) + sl]
        assert per[b, 7] == fl.sum()
        if not fl.any():
            assert np.all(per[b, :7] == 0)
            continue
        assert abs(per[b, 0] - r[fl].sum()) <= 1e-13 * r[fl].sum()
        for a in range(3):
            assert abs(per[b, 1 + a] - (r * v[a])[fl].sum()) <= 1e-10 * r[fl].sum() * 0.02
        e = (0.5 * r * (v * v).sum(axis=0))[fl].sum()
        assert abs(per[b, 4] - e) <= 1e-10 * e
        assert abs(per[b, 5] - np.sqrt((v * v).sum(axis=0))[fl].max()) <= 1e-12
        assert per[b, 6] == 0
    assert abs(per[:, 0].sum() - tot["mass"]) <= 1e-13 * tot["mass"]
    assert per[:, 7].sum() == tot["fluid_cells"]


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32])
@pytest.mark.parametrize("pattern,steps", [(lbm.TWO_GRID, 5), (lbm.AA, 5), (lbm.AA, 6)])
def test_macroscopic_output_matches_oracle_elementwise(storage, pattern, steps):
    """lbm_get_macroscopic (the a8 output kernel) cell by cell: (1) against the oracle's moments
    of the very state the GPU holds (rho = sum f*, u = (sum c f* - F/2) / rho), to FP64
    rounding; (2) against the oracle's own run, within the PDF gate carried to the moments.
    Uneven blocks, spheres, velocity inlet, pressure outlet, a body force, walls in z; odd and
    even AA parities (the two layouts the kernel reads)."""
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    case = Case(shape=shape, blocks=blocks, q=19, collision=lbm.TRT, storage=storage, pattern=pattern,
                omega=1 / 0.8, force=(2e-5, -1e-5, 5e-6), periodic=(0, 1, 0),
                faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, lbm.NOSLIP, lbm.NOSLIP),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, flags=flags)
    rho, u = inputs.random_state(shape, seed=41, rho_amp=0.02, u_amp=0.02)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(steps)
    grho, gu = gather_macro(sim, case)
    gf = gather_pdfs(sim, case)
    sim.close()
    p = case.oracle_params()
    fl = case.global_flags()
    fluid = fl == 0
    # (1) the output kernel alone: moments of the GPU's own stored state
    orho, ou = oracle.macroscopic(p, gf, fl)
    assert np.abs(grho - orho)[fluid].max() <= 1e-14
    assert np.abs(gu - ou)[:, fluid].max() <= 1e-14
    assert np.all(grho[~fluid] == 0) and np.all(gu[:, ~fluid] == 0)
    # (2) against the oracle's run: |d rho| <= Q e, |d u| <= (10 e + |u| |d rho|) / rho with
    # e = the PDF gate times max|f|
    _, want = oracle_run(case, rho, u, steps)
    wrho, wu = oracle.macroscopic(p, want, fl)
    e = TOL[storage] * np.abs(want[:, fluid]).max()
    drho = np.abs(grho - wrho)[fluid]
    assert drho.max() <= 19 * e
    du = np.abs(gu - wu)[:, fluid]
    assert np.all(du <= (10 * e + np.abs(wu[:, fluid]) * 19 * e) / wrho[fluid] + 1e-300)


@pytest.mark.parametrize("storage,pattern", [(lbm.FP32, lbm.TWO_GRID), (lbm.FP64, lbm.AA), (lbm.FP16_DEV, lbm.TWO_GRID)])
def test_page_locked_host_buffers_equal_pageable(storage, pattern):
    """Page-locked host buffers are read (init) and written (macroscopic output) by the kernels
    directly; pageable ones go through the device staging copy: the same bits either way."""
    torch = pytest.importorskip("torch")
    case = _porous_case(storage, pattern)
    rho, u = inputs.random_state(case.shape, seed=17, rho_amp=0.02, u_amp=0.02)
    out = []
    for pinned in (False, True):
        s = case.make_sim()
        try:
            keep = []
            for b, (o, sz) in enumerate(s.blocks):
                r = np.ascontiguousarray(rho[o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]])
                v = np.ascontiguousarray(u[:, o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]])
                if pinned:
                    tr, tv = torch.from_numpy(r).pin_memory(), torch.from_numpy(v).pin_memory()
                    keep += [tr, tv]
                    r, v = tr.numpy(), tv.numpy()
                lbm.lbm_init_macroscopic(s.ctx, b, r, v)
            s.step(4)
            got = []
            for b, (o, sz) in enumerate(s.blocks):
                n = sz[0] * sz[1] * sz[2]
                if pinned:
                    tr = torch.empty(n, dtype=torch.float64).pin_memory()
                    tv = torch.empty(3 * n, dtype=torch.float64).pin_memory()
                    keep += [tr, tv]
                    r, v = tr.numpy(), tv.numpy()
                else:
                    r, v = np.empty(n), np.empty(3 * n)
                lbm.lbm_get_macroscopic(s.ctx, b, r, v)
                got.append((r.copy(), v.copy()))
            out.append((gather_pdfs(s, case), got))
        finally:
            s.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for (r0, v0), (r1, v1) in zip(out[0][1], out[1][1]):
        np.testing.assert_array_equal(r0, r1)
        np.testing.assert_array_equal(v0, v1)


def test_macroscopic_output_removes_half_the_force():
    """At rest under a body force the stored post-collision state carries sum c f* = F/2 per
    cell; the output velocity (sum c f* - F/2) / rho is zero there (and F/(2 rho) if the shift
    were missing).  Both hold up to rounding: each stored value is within a few roundings of
    its own magnitude in the storage precision (the equilibrium, the relaxation of a near-zero
    non-equilibrium part and the final sum: at most 8 eps |f_i|), and the FP64 sums here and in
    the output kernel add at most Q eps64 sum |c_a f_i| each, so per cell and axis
    |sum c_a f - F_a/2| <= (8 eps + Q eps64) S_a and |u_a| <= (8 eps + 2 Q eps64) S_a / rho with
    S_a = sum_i |c_ia f_i| = 1/3 (FP32: 3.2e-7 against F/2 >= 5e-6)."""
    shape = (40, 9, 7)
    F = (3e-5, -2e-5, 1e-5)
    e64 = np.finfo(np.float64).eps
    for storage in (lbm.FP64, lbm.FP32):
        eps = np.finfo(np.float64 if storage == lbm.FP64 else np.float32).eps
        case = Case(shape=shape, storage=storage, force=F, omega=1.3)
        sim = case.make_sim()
        rho, u = inputs.rest(shape)
        sim.init(0, rho, u)
        grho, gu = sim.macroscopic(0)
        f = sim.pdfs(0)
        sim.close()
        c, _, _ = oracle.lattice(19)
        c = c.astype(np.float64)
        j = np.einsum("ia,i...->a...", c, f)
        S = np.einsum("ia,i...->a...", np.abs(c), np.abs(f))
        for a in range(3):
            assert np.all(np.abs(j[a] - F[a] / 2) <= (8 * eps + 19 * e64) * S[a])
            assert np.all(np.abs(gu[a]) <= (8 * eps + 38 * e64) * S[a] / grho)
            assert (8 * eps + 38 * e64) * S[a].max() < 0.07 * abs(F[a])  # the shift is visible


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_ghost_copies_equal_in_place_neighbours(pattern):
    """lbm_set_in_place(0) (ghost layers filled by copy runs) gives the same state bit for bit
    as in-place neighbour access, including a switch between the two after an even number of
    steps; an AA switch after an odd number is refused."""
    case = _porous_case(lbm.FP32, pattern)
    rho, u = inputs.random_state(case.shape, seed=21, rho_amp=0.02, u_amp=0.02)
    out = []
    for mode in ("in_place", "ghost", "switch"):
        s = case.make_sim()
        if mode == "ghost":
            lbm.lbm_set_in_place(s.ctx, False)
        init_sim(s, rho, u)
        s.step(4)
        if mode == "switch":
            lbm.lbm_set_in_place(s.ctx, False)
        s.step(5)
        if mode == "switch" and pattern == lbm.AA:
            with pytest.raises(lbm.LbmError):
                lbm.lbm_set_in_place(s.ctx, True)
        s.step(1)
        out.append(gather_pdfs(s, case))
        if mode == "ghost":
            info = s.info()
            assert info["ghost_runs"] > 0
        s.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_divergence_is_reported():
    case = Case(shape=(40, 9, 6), storage=lbm.FP32)
    p = lbm.make_params(stencil=19, storage=lbm.FP32, omega=1.2, diag_interval=2)
    sim = lbm.Simulation(p, case.block_list())
    rho, u = inputs.rest(case.shape)
    sim.init(0, rho, u)
    sim.step(2)
    f = sim.pdfs(0)
    f[3, 2, 4, 7] = np.nan
    sim.set_pdfs(0, f)
    with pytest.raises(lbm.LbmError) as e:
        sim.step(4)
    assert e.value.status == 5
    assert sim.reduce()["nonfinite"] >= 1
    sim.close()


def test_bound_torch_buffer_and_stream():
    import torch
    case = Case(shape=(33, 10, 7), storage=lbm.FP32, pattern=lbm.AA, periodic=(1, 0, 1),
                faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    p = lbm.make_params(stencil=19, storage=lbm.FP32, pattern=lbm.AA, omega=1.3, periodic=(1, 0, 1))
    stream = torch.cuda.Stream()
    probe = lbm.Simulation(p, case.block_list())
    need = lbm.lbm_required_bytes(probe.ctx)
    probe.close()
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    sim = lbm.Simulation(p, case.block_list(), stream=stream.cuda_stream, device_buffer=buf)
    rho, u = inputs.random_state(case.shape, seed=4, rho_amp=0.01, u_amp=0.01)
    sim.init(0, rho, u)
    sim.step(6)
    got = sim.pdfs(0)
    assert sim.launches() == 6  # one sweep per step: no-slip walls need no fill launch
    sim.close()
    case.omega = 1.3
    _, want = oracle_run(case, rho, u, 6)
    assert normwise(got, want) <= 1e-5


# Bounds of the fused step diagnostics against the FP64 pass over the stored state (lbm_reduce).
# Mass: with FP32 arithmetic each cell's stored values are summed exactly as a float-float pair
# (error terms in FP32: at most Q^2 u^2 rho per cell, u = 2^-24); a thread's n cells add up to
# (2 Q n + n^2) u^2 in its FP32 low part; the CTA adds the threads' pairs with the low parts in
# FP32, 12 additions deep (3 (Q + n) u^2): within (Q + n + 3)^2 u^2 in all, n = 4 cells per
# thread in the default 256 x 1 x 4 tiles; both sides' FP64 sums add < 1e-13.  Momentum: the
# collision's FP32 moment rho u of a cell (a sum of 19 values, then the half-force term) against
# the FP64 moment of the stored values (rounded once more): at most 20 u sum_i f_i = 20 u rho per
# cell; per thread Kahan's compensation (2u of the magnitudes sum |rho u| <= mass max|u|), the
# pair's difference (u) and the CTA's 12 FP32 additions (6u): 20 u mass + 9 u mass max|u| <=
# 29 u mass.  Kinetic energy: the velocities differ by at most 24 u per cell, so
# |d sum rho u^2 / 2| <= 24 u sum rho |u| <= 24 u sqrt(2 mass KE) (Cauchy-Schwarz), plus 24 u KE
# for rho and 9 u KE for the sums; max |u|: 24 u.
DIAG_MASS_TOL = {lbm.FP64: 1e-13, lbm.FP32: (19 + 4 + 3) ** 2 * 2.0 ** -48 + 1e-13}
U32 = 2.0 ** -24


@pytest.mark.parametrize("storage,pattern", [(lbm.FP64, lbm.TWO_GRID), (lbm.FP64, lbm.AA), (lbm.FP32, lbm.TWO_GRID),
                                             (lbm.FP32, lbm.AA)])
def test_step_diagnostics_match_full_reduction(storage, pattern):
    """The diagnostics fused into the last sweep of lbm_step agree with the full FP64 pass
    over the stored state, within the bounds derived above."""
    case = _porous_case(storage, pattern)
    rho, u = inputs.random_state(case.shape, seed=14, rho_amp=0.02, u_amp=0.02)
    s = case.make_sim()
    init_sim(s, rho, u)
    with pytest.raises(lbm.LbmError):
        s.step_diagnostics()  # state was set, no step yet
    s.step(3)
    fused, full = s.step_diagnostics(), s.reduce()
    s.close()
    assert abs(fused["mass"] / full["mass"] - 1) < DIAG_MASS_TOL[storage]
    if storage == lbm.FP64:
        assert max(abs(a - b) for a, b in zip(fused["momentum"], full["momentum"])) <= 1e-10 * max(
            abs(v) for v in full["momentum"])
        assert abs(fused["kinetic_energy"] / full["kinetic_energy"] - 1) < 1e-10
        assert abs(fused["max_speed"] / full["max_speed"] - 1) < 1e-10
    else:
        m, ke = full["mass"], full["kinetic_energy"]
        assert max(abs(a - b) for a, b in zip(fused["momentum"], full["momentum"])) <= 29 * U32 * m
        assert abs(fused["kinetic_energy"] - ke) <= U32 * (24 * np.sqrt(2 * m * ke) + 33 * ke)
        assert abs(fused["max_speed"] - full["max_speed"]) <= 24 * U32
    assert fused["nonfinite"] == 0 and fused["fluid_cells"] == full["fluid_cells"]


@pytest.mark.parametrize("storage", [lbm.FP16_DEV, lbm.BF16_DEV])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_step_diagnostics_mass_16bit_storage(storage, pattern):
    """16-bit deviation storage: the fused mass is the exact sum of rho0 + the stored (rounded)
    deviations, so it matches the FP64 pass over the stored field within the bound stated for
    FP32 arithmetic, (Q + n + 3)^2 u^2 with n the cells a thread sweeps; the 256-wide periodic
    box takes the staged (bulk-copy) two-grid path."""
    case = Case(shape=(256, 12, 10), storage=storage, pattern=pattern, omega=1.3, force=(1e-5, 2e-6, 0.0))
    rho, u = inputs.random_state(case.shape, seed=15, rho_amp=0.02, u_amp=0.03)
    s = case.make_sim()
    init_sim(s, rho, u)
    s.step(5)
    fused, full = s.step_diagnostics(), s.reduce()
    s.close()
    # staged 16-bit tiles: 8 z steps of two cells per thread, n = 16 (AA: n = 4)
    assert abs(fused["mass"] / full["mass"] - 1) < (19 + 16 + 3) ** 2 * 2.0 ** -48 + 1e-13
    assert fused["fluid_cells"] == full["fluid_cells"] and fused["nonfinite"] == 0


@pytest.mark.parametrize("storage,pattern", [(lbm.FP32, lbm.TWO_GRID), (lbm.FP32, lbm.AA), (lbm.FP16_DEV, lbm.AA)])
def test_pipelined_step_diagnostics_equal_synchronised_reads(storage, pattern):
    """Records posted after each step and taken after the next step was issued are the records
    lbm_step_diagnostics reads for the same steps, bit for bit; full slots and unknown or
    retaken tickets are errors that leave the context usable."""
    case = _porous_case(storage, pattern)
    rho, u = inputs.random_state(case.shape, seed=16, rho_amp=0.02, u_amp=0.02)
    a, b = case.make_sim(), case.make_sim()
    init_sim(a, rho, u)
    init_sim(b, rho, u)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_diagnostics_post(a.ctx)  # state was set, no step yet
    got, want, pending = [], [], None
    for _ in range(7):
        a.step(1)
        t = lbm.lbm_step_diagnostics_post(a.ctx)
        if pending is not None:
            got.append(lbm.lbm_step_diagnostics_take(a.ctx, pending))
        pending = t
        b.step(1)
        want.append(b.step_diagnostics())
    got.append(lbm.lbm_step_diagnostics_take(a.ctx, pending))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_diagnostics_take(a.ctx, pending)  # taken already
    a.step(1)
    b.step(1)
    want.append(b.step_diagnostics())
    tickets = [lbm.lbm_step_diagnostics_post(a.ctx) for _ in range(lbm.DIAG_SLOTS)]
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_diagnostics_post(a.ctx)  # every slot holds an untaken record
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step_diagnostics_take(a.ctx, max(tickets) + 1)  # never posted
    last = [lbm.lbm_step_diagnostics_take(a.ctx, t) for t in reversed(tickets)]
    got.append(a.step_diagnostics())
    a.close()
    b.close()
    assert len(got) == len(want) == 8
    assert got == want
    assert all(d == want[-1] for d in last)


def test_full_size_channel_equals_column_oracle():
    """256^3 channel (the benchmark workload and launch configuration, FP32 and FP64): the
    flow is x- and z-invariant, so every column must equal the oracle's 1 x 256 x 1 run."""
    n, steps = 256, 20
    force = (1e-6, 0.0, 0.0)
    col = Case(shape=(1, n, 1), q=19, collision=lbm.TRT, storage=lbm.FP64, omega=1.0, force=force,
               periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho1, u1 = inputs.rest(col.shape)
    _, want = oracle_run(col, rho1, u1, steps)
    for storage in (lbm.FP32, lbm.FP64):
        case = Case(shape=(n, n, n), q=19, collision=lbm.TRT, storage=storage, omega=1.0, force=force,
                    periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
        s = case.make_sim()
        rho, u = inputs.rest(case.shape)
        s.init(0, rho, u)
        s.step(steps)
        f = s.pdfs(0)
        s.close()
        rng = np.random.default_rng(0)
        for _ in range(8):
            x, z = rng.integers(0, n, 2)
            assert normwise(f[:, z, :, x], want[:, 0, :, 0]) <= TOL[storage]
        # x/z invariance of the whole field
        assert np.abs(f - f[:, :1, :, :1]).max() <= TOL[storage] * np.abs(f).max()


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_graph_mode_equals_plain_launches(pattern):
    """Step pairs replayed as CUDA graphs give bitwise the same state as plain launches,
    including an odd step count and a call that spans both graph parities."""
    import torch
    case = _porous_case(lbm.FP32, pattern)
    rho, u = inputs.random_state(case.shape, seed=17, rho_amp=0.01, u_amp=0.02)
    out = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        s = case.make_sim(stream=stream.cuda_stream)
        if graphs:
            lbm.lbm_set_graph(s.ctx, True)
        init_sim(s, rho, u)
        s.step(9)
        s.step(4)
        out.append(gather_pdfs(s, case))
        launches = s.launches()
        s.close()
    np.testing.assert_array_equal(out[1], out[0])


def test_graph_mode_needs_a_stream():
    case = Case(shape=(40, 9, 6), storage=lbm.FP32)
    s = case.make_sim()
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_graph(s.ctx, True)
    s.close()


@pytest.mark.parametrize("pattern,at", [(lbm.AA, 3), (lbm.AA, 4), (lbm.TWO_GRID, 3)])
def test_autotune_keeps_state_and_results(pattern, at):
    """The autotuner (tile shapes and, where allowed, the neighbour mode) leaves the state, step
    count and parity as they were, and later steps equal those of an untuned run bit for bit."""
    case = _porous_case(lbm.FP32, pattern)
    rho, u = inputs.random_state(case.shape, seed=19, rho_amp=0.01, u_amp=0.02)
    a = case.make_sim()
    init_sim(a, rho, u)
    a.step(at)
    before = gather_pdfs(a, case)
    best, ms, in_place = lbm.lbm_autotune(a.ctx, 4)
    assert ms > 0 and best[0] * best[1] <= 256
    np.testing.assert_array_equal(gather_pdfs(a, case), before)
    a.step(8 - at)
    tuned = gather_pdfs(a, case)
    a.close()
    b = case.make_sim()
    init_sim(b, rho, u)
    b.step(8)
    np.testing.assert_array_equal(gather_pdfs(b, case), tuned)
    b.close()


def test_per_block_launches_equal_batched():
    case = _porous_case(lbm.FP32, lbm.TWO_GRID)
    rho, u = inputs.random_state(case.shape, seed=23, rho_amp=0.01, u_amp=0.02)
    out = []
    for batched in (True, False):
        s = case.make_sim()
        lbm.lbm_set_batching(s.ctx, batched)
        init_sim(s, rho, u)
        s.step(5)
        out.append((gather_pdfs(s, case), s.step_diagnostics(), s.launches()))
        s.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    assert out[1][1] == out[0][1]
    assert out[1][2] == 5 * len(case.blocks) + (out[0][2] - 5)  # one sweep per block per step


@pytest.mark.parametrize("storage", [lbm.FP16_DEV, lbm.BF16_DEV])
@pytest.mark.parametrize("in_place", [False, True])
def test_two_grid_staged_rows_two_blocks_match_oracle(storage, in_place):
    """Two 128-wide blocks side by side in x, periodic in x and z, walls in y.  Ghost copies: the
    blocks' rows are staged with one 16-byte ghost copy on the side each direction reads from.
    In place: a block reads the other one, so its tiles take the direct path."""
    shape = (256, 10, 9)
    blocks = [((0, 0, 0), (128, 10, 9)), ((128, 0, 0), (128, 10, 9))]
    case = Case(shape=shape, blocks=blocks, storage=storage, pattern=lbm.TWO_GRID, omega=1.4,
                force=(2e-5, 0.0, 1e-6), periodic=(1, 0, 1))
    rho, u = inputs.random_state(shape, seed=37, rho_amp=0.02, u_amp=0.03)
    s = case.make_sim()
    lbm.lbm_set_in_place(s.ctx, in_place)
    info = s.info()
    if in_place:
        assert info["staged_tiles"] == 0
    else:
        assert 0 < info["staged_tiles"] < info["tiles"]
    init_sim(s, rho, u)
    steps = 6
    s.step(steps)
    got = gather_pdfs(s, case)
    s.close()
    _, want = oracle_run(case, rho, u, steps)
    from oracle import lattice
    _, w, _ = lattice(19)
    ur = 2.0 ** -8 if storage == lbm.BF16_DEV else 2.0 ** -11
    bound = (steps + 1) * ur * np.abs(want - w[:, None, None, None]).max() / np.abs(want).max()
    assert normwise(got, want) <= bound


@pytest.mark.parametrize("storage", [lbm.FP32, lbm.FP16_DEV, lbm.BF16_DEV])
@pytest.mark.parametrize("shape,periodic,in_place,tz", [((256, 12, 10), (1, 1, 1), True, None),
                                                        ((128, 9, 7), (1, 0, 1), True, None),
                                                        ((128, 9, 7), (1, 0, 1), False, None),
                                                        ((256, 6, 5), (0, 1, 1), True, None),
                                                        ((256, 12, 10), (1, 1, 1), True, 3),
                                                        ((128, 9, 7), (1, 0, 1), False, 1)])
def test_two_grid_staged_rows_match_oracle(storage, shape, periodic, in_place, tz):
    """Blocks 128 or 256 cells wide: with 16-bit storage the two-grid sweep stages the source
    rows of their unmasked tiles in shared memory by bulk copies (wrapped rows for self-periodic
    blocks, ghost rows otherwise); walls in y or x give masked tiles that take the direct path,
    and FP32 storage takes the direct path everywhere.  Tile depths 8 (the 16-bit default), 4, 3
    and 1 leave ragged z runs and runs shorter than the two stages.  The last step writes the
    diagnostics (the staged path of that variant too)."""
    case = Case(shape=shape, storage=storage, pattern=lbm.TWO_GRID, omega=1.3, force=(1e-5, 2e-6, 0.0),
                periodic=periodic)
    rho, u = inputs.random_state(shape, seed=31, rho_amp=0.02, u_amp=0.03)
    s = case.make_sim()
    if not in_place:
        lbm.lbm_set_in_place(s.ctx, False)
    if tz is not None:
        s.set_tile(256, 1, tz)
    info = s.info()
    if storage == lbm.FP32:
        assert info["staged_tiles"] == 0
    elif all(periodic):
        assert info["staged_tiles"] == info["tiles"]
    elif periodic[0] == 1:
        # walls in y: the tiles of the rows next to them carry masks, the others are staged
        assert 0 < info["staged_tiles"] < info["tiles"]
    init_sim(s, rho, u)
    steps = 7
    s.step(steps)
    d = s.step_diagnostics()
    got = gather_pdfs(s, case)
    s.close()
    _, want = oracle_run(case, rho, u, steps)
    err = normwise(got, want)
    if storage == lbm.FP32:
        assert err < TOL[lbm.FP32], err
    else:
        from oracle import lattice
        _, w, _ = lattice(19)
        ur = 2.0 ** -8 if storage == lbm.BF16_DEV else 2.0 ** -11
        bound = (steps + 1) * ur * np.abs(want - w[:, None, None, None]).max() / np.abs(want).max()
        assert err <= bound, (err, bound)
    full = oracle.diagnostics(case.oracle_params(), want)
    assert abs(d["mass"] / full["mass"] - 1) < 1e-5
