"""16-bit deviation storage (BF16 / FP16 of f_i - w_i rho0, FP32 collision) against the FP64
oracle.  The storage rounds each stored deviation to the format's unit roundoff u (2^-8 for
BF16, 2^-11 for FP16) every step, so after n steps the normwise PDF error is bounded by
n * u * max|f - w rho0| / max|f| (a worst case: errors of opposite sign mostly cancel).  The
tests assert that bound and report the measured error."""
import numpy as np
import pytest

from gpu_helpers import Case, gather_pdfs, init_sim, normwise, oracle_run
from paper_1909_13772_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {lbm.BF16_DEV: 2.0 ** -8, lbm.FP16_DEV: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load_library()


def _bound(storage, steps, want, q):
    from oracle import lattice
    _, w, _ = lattice(q)
    dev = np.abs(want - w[:, None, None, None]).max()
    return steps * UNIT_ROUNDOFF[storage] * dev / np.abs(want).max()


@pytest.mark.parametrize("storage", [lbm.BF16_DEV, lbm.FP16_DEV])
@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
@pytest.mark.parametrize("q", [19, 27])
def test_dev_storage_channel_error_within_rounding_bound(storage, pattern, q):
    shape, steps = (70, 37, 11), 40
    case = Case(shape=shape, q=q, collision=lbm.TRT, storage=storage, pattern=pattern, omega=1.0,
                force=(1e-5, 0.0, 0.0), periodic=(1, 0, 1), faces=(1, 1, lbm.NOSLIP, lbm.NOSLIP, 1, 1))
    rho, u = inputs.random_state(shape, seed=21, rho_amp=0.02, u_amp=0.03)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(steps)
    got = gather_pdfs(sim, case)
    sim.close()
    _, want = oracle_run(case, rho, u, steps)
    err = normwise(got, want)
    assert err <= _bound(storage, steps, want, q), err
    # and clearly better than the bound's worst case: rounding errors do not all add up
    assert err <= 0.5 * _bound(storage, steps, want, q), err


@pytest.mark.parametrize("storage", [lbm.BF16_DEV, lbm.FP16_DEV])
def test_dev_storage_porous_multiblock(storage):
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(3, 2, 2), lo=9, hi=21, seed=4)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    case = Case(shape=shape, blocks=blocks, q=19, collision=lbm.TRT, storage=storage, pattern=lbm.AA,
                omega=1 / 0.8, periodic=(0, 1, 1), faces=(lbm.VELOCITY, lbm.PRESSURE, 1, 1, 1, 1),
                face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, flags=flags)
    rho, u = inputs.rest(shape)
    steps = 60
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(steps)
    got = gather_pdfs(sim, case)
    sim.close()
    _, want = oracle_run(case, rho, u, steps)
    fl = case.global_flags() == 0
    err = normwise(got, want, fl)
    assert err <= _bound(storage, steps, np.where(fl[None], want, 0.0) + np.where(fl[None], 0.0, 1e-300), 19)


@pytest.mark.parametrize("storage", [lbm.BF16_DEV, lbm.FP16_DEV])
def test_dev_storage_rest_state_stays_at_weights(storage):
    """At rest with rho = rho0 every deviation is zero up to the FP32 rounding of the
    collision, so the 16-bit run keeps the weights to FP32 accuracy (the deviation form is
    what makes this work; storing f_i itself in 16 bits would round w_i by ~1e-3)."""
    case = Case(shape=(40, 9, 6), q=19, storage=storage, omega=1.3)
    rho, u = inputs.rest(case.shape)
    sim = case.make_sim()
    init_sim(sim, rho, u)
    sim.step(10)
    got = gather_pdfs(sim, case)
    sim.close()
    from oracle import lattice
    _, w, _ = lattice(19)
    assert np.abs(got - w[:, None, None, None]).max() <= 1e-6


def _oracle_region(q, omega, rho, u, origin, size, steps):
    """Oracle PDFs of the box origin/size of a periodic field after `steps` steps, from the
    (2 steps + box) neighbourhood only: init of the neighbourhood, then per step streaming
    f_i(x) = f*_i(x - c_i) and the single-cell collision of the oracle."""
    import oracle
    n = rho.shape[0]
    h = steps
    idx = [(np.arange(o - h, o + s + h) % n) for o, s in zip(origin, size)]  # x, y, z
    sub_rho = rho[np.ix_(idx[2], idx[1], idx[0])]
    sub_u = u[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    ext = tuple(s + 2 * h for s in size)
    p = oracle.OracleParams(shape=ext, q=q, collision=oracle.TRT, omega=omega, magic_lambda=3 / 16,
                            periodic=(1, 1, 1))
    f = oracle.init(p, sub_rho, sub_u)
    c, _, _ = oracle.lattice(q)
    for k in range(1, steps + 1):
        nz, ny, nx = f.shape[1] - 2, f.shape[2] - 2, f.shape[3] - 2
        g = np.empty((q, nz, ny, nx))
        for i in range(q):
            cx, cy, cz = c[i]
            g[i] = f[i, 1 - cz:1 - cz + nz, 1 - cy:1 - cy + ny, 1 - cx:1 - cx + nx]
        out = np.empty_like(g)
        for zz in range(nz):
            for yy in range(ny):
                for xx in range(nx):
                    out[:, zz, yy, xx] = oracle.collide_cell(p, g[:, zz, yy, xx])
        f = out
    return f


@pytest.mark.parametrize("storage", [lbm.FP32, lbm.FP16_DEV])
def test_full_size_d3q27_turbulence_regions_match_oracle(storage):
    """The decaying-turbulence configuration at its full size: 512^3 periodic box, D3Q27 TRT
    tau = 0.52, AA pattern (the bench's launch), random-phase start; after two steps (one
    neighbour and one local sweep) two 8^3 regions -- one inside, one at the corner where every
    neighbour wraps -- against the oracle computed from their neighbourhoods."""
    n, steps = 512, 2
    rho, u = inputs.turbulence(n, seed=1909, kmax=32, umax=0.05)
    p = lbm.make_params(stencil=27, collision=lbm.TRT, storage=storage, pattern=lbm.AA, omega=1 / 0.52,
                        periodic=(1, 1, 1))
    sim = lbm.Simulation(p, [((0, 0, 0), (n, n, n))])
    try:
        sim.init(0, rho, u)
        sim.step(steps)
        regions = [((301, 77, 190), (8, 8, 8)), ((0, 0, 0), (8, 8, 8))]
        got = [sim.pdfs_region(0, o, s) for o, s in regions]
    finally:
        sim.close()
    for (o, s), g in zip(regions, got):
        want = _oracle_region(27, 1 / 0.52, rho, u, o, s, steps)
        err = normwise(g, want)
        if storage == lbm.FP32:
            assert err < 1e-5, err
        else:
            assert err <= _bound(storage, steps + 1, want, 27), err
