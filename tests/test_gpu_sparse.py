"""The fluid-cell list layout of the two-grid sweep (lbm_set_sparse) against the dense block
layout: every cell does the same arithmetic in both, so after any number of steps the states
are equal bit for bit -- on uneven blocks read in place across faces and periodic images,
spheres (halfway bounce-back), velocity inlet and pressure outlet links, with and without a
body force, in every storage format and both stencils; the move of the state between the two
layouts (switching mid-run, PDF reads and writes between steps) keeps every bit; the step
diagnostics agree to FP64 summation order."""
import numpy as np
import pytest

from gpu_helpers import Case, gather_pdfs, init_sim, split
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _porous(storage, q=19, force=(0.0, 0.0, 0.0), nb=(3, 2, 2), porosity=0.6):
    blocks, shape, _ = inputs.rectilinear_blocks(nb=nb, lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=porosity, seed=7, buffer=4.0)
    return Case(shape=shape, blocks=blocks, q=q, collision=lbm.TRT, storage=storage, pattern=lbm.TWO_GRID,
                omega=1 / 0.8, force=force, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6, flags=flags)


def _run(case, rho, u, steps, sparse, switch_at=None):
    sim = case.make_sim()
    try:
        if sparse:
            lbm.lbm_set_sparse(sim.ctx, True)
        init_sim(sim, rho, u)
        if switch_at is None:
            sim.step(steps)
        else:
            sim.step(switch_at)
            lbm.lbm_set_sparse(sim.ctx, not sparse)
            sim.step(steps - switch_at)
        info = sim.info()
        return gather_pdfs(sim, case), sim.step_diagnostics(), info
    finally:
        sim.close()


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32, lbm.FP16_DEV, lbm.BF16_DEV])
@pytest.mark.parametrize("q", [19, 27])
def test_list_layout_equals_dense_bitwise(storage, q):
    case = _porous(storage, q=q, force=(2e-6, 0.0, 1e-6))
    rho, u = inputs.random_state(case.shape, seed=41, rho_amp=0.01, u_amp=0.02)
    dense, dd, _ = _run(case, rho, u, 9, False)
    lst, dl, info = _run(case, rho, u, 9, True)
    fl = case.global_flags() == 0
    np.testing.assert_array_equal(lst[:, fl], dense[:, fl])
    assert info["list_entries"] >= info["fluid_cells"] > 0
    assert info["links"][lbm.VELOCITY] > 0 and info["links"][lbm.PRESSURE] > 0
    assert dl["fluid_cells"] == dd["fluid_cells"] == info["fluid_cells"]
    # the same stored values: the exact (float-float) mass sums agree to FP64 order; momentum is a
    # compensated sum in the arithmetic type per thread (a dense thread walks several cells, a
    # list thread one), then (FP32) the pair's difference and 12 pairwise FP32 additions per CTA:
    # within 9 u sum |rho u| <= 9 u mass max|u| of the exact sum on each side, u its roundoff
    assert abs(dl["mass"] / dd["mass"] - 1) < 1e-12
    u = 2.0 ** (-53 if storage == lbm.FP64 else -24)
    assert np.abs(np.array(dl["momentum"]) - np.array(dd["momentum"])).max() <= (
        18 * u * dd["mass"] * dd["max_speed"] + 1e-12 * dd["mass"])


@pytest.mark.parametrize("switch_at", [3, 4])
def test_switching_layouts_mid_run_keeps_every_bit(switch_at):
    case = _porous(lbm.FP32)
    rho, u = inputs.random_state(case.shape, seed=42, rho_amp=0.01, u_amp=0.02)
    want, _, _ = _run(case, rho, u, 10, False)
    fl = case.global_flags() == 0
    for start_sparse in (True, False):
        got, _, _ = _run(case, rho, u, 10, start_sparse, switch_at=switch_at)
        np.testing.assert_array_equal(got[:, fl], want[:, fl])


def test_reads_and_writes_between_list_steps():
    """PDF reads, a PDF write of one block and graph replay between steps of the list layout:
    the same as the dense layout doing the same."""
    case = _porous(lbm.FP64)
    rho, u = inputs.random_state(case.shape, seed=43, rho_amp=0.01, u_amp=0.02)
    out = []
    for sparse in (False, True):
        import torch
        st = torch.cuda.Stream()
        sim = case.make_sim(stream=st.cuda_stream)
        try:
            if sparse:
                lbm.lbm_set_sparse(sim.ctx, True)
            lbm.lbm_set_graph(sim.ctx, True)
            init_sim(sim, rho, u)
            sim.step(6)
            f1 = sim.pdfs(1)
            sim.set_pdfs(1, f1 * 1.0001)  # a write into the dense arrays mid-run
            sim.step(7)
            r, v = sim.macroscopic(0)
            out.append((gather_pdfs(sim, case), r, v, sim.reduce()))
        finally:
            sim.close()
    fl = case.global_flags() == 0
    np.testing.assert_array_equal(out[1][0][:, fl], out[0][0][:, fl])
    np.testing.assert_array_equal(out[1][1], out[0][1])
    np.testing.assert_array_equal(out[1][2], out[0][2])
    assert out[1][3]["mass"] == out[0][3]["mass"]


def test_list_layout_refuses_what_it_does_not_cover():
    case = _porous(lbm.FP32)
    case.pattern = lbm.AA
    sim = case.make_sim()
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_sparse(sim.ctx, True)
        assert e.value.status == 7
    finally:
        sim.close()
    case.pattern = lbm.TWO_GRID
    sim = case.make_sim()
    try:
        lbm.lbm_set_sparse(sim.ctx, True)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_autotune(sim.ctx, 2)
        assert e.value.status == 7
    finally:
        sim.close()
