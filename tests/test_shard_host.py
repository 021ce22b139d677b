"""Host logic of partitioned runs (no GPU): the Morton partition, the halo lists of every rank
against the ghost-copy lists of one unpartitioned context, and the exchange itself emulated on
host arrays -- in one process, and between two gloo ranks through the same exchange helper the
GPU runs use.

The emulation fills every owned interior slot with a number that names it (direction, global
cell), moves the values along the ranks' halo runs exactly as the pack and unpack kernels do
(element k of a run: arena[offset + k * stride] <-> buffer[buffer offset + k]) and checks that
every received ghost slot holds the value of the cell it mirrors (periodic images included),
so a wrong cell, slot, order or peer anywhere in the lists fails."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1909_13772_gb300 import inputs, lbm  # noqa: E402


def _morton(x, y, z):
    """Z-order key, bits of x, y, z interleaved (x lowest), written bit by bit."""
    k = 0
    for bit in range(21):
        k |= ((x >> bit) & 1) << (3 * bit) | ((y >> bit) & 1) << (3 * bit + 1) | ((z >> bit) & 1) << (3 * bit + 2)
    return k


def _case(nb=(3, 2, 2), seed=4, q=19, pattern=lbm.TWO_GRID, periodic=(0, 1, 1)):
    blocks, shape, _ = inputs.rectilinear_blocks(nb=nb, lo=9, hi=21, seed=seed)
    flags = inputs.sphere_packing(shape, radius=3.0, porosity=0.6, seed=7, buffer=4.0)
    p = lbm.make_params(stencil=q, storage=lbm.FP32, pattern=pattern, periodic=periodic)
    return blocks, shape, flags, p


def _make(p, blocks, flags, owner=None, nranks=1, rank=0):
    sim = lbm.Simulation(p, blocks, owner=owner, nranks=nranks, rank=rank)
    sim.set_face(0, 0, lbm.VELOCITY, (0.02, 0.0, 0.0), 1.0)
    sim.set_face(0, 1, lbm.PRESSURE, (0.0, 0.0, 0.0), 1.0)
    for b, (o, s) in enumerate(sim.blocks):
        sub = flags[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]]
        sim.set_boundary(b, sub if sub.any() else None)
    return sim


def test_morton_partition_is_contiguous_balanced_and_deterministic():
    blocks, _, _ = inputs.rectilinear_blocks(nb=(6, 5, 4), lo=8, hi=40, seed=11)
    lo = np.min([o for o, _ in blocks], axis=0)
    keys = [_morton(*(2 * (np.array(o) - lo) + np.array(s)).tolist()) for o, s in blocks]
    order = np.argsort(keys, kind="stable")
    cells = np.array([np.prod(s) for _, s in blocks], dtype=float)
    for n in (1, 2, 3, 7, 16):
        own = lbm.lbm_partition_morton(blocks, n)
        assert np.array_equal(own, lbm.lbm_partition_morton(blocks, n))
        assert np.all(np.diff(own[order]) >= 0)  # contiguous pieces of the curve, ranks in order
        w = np.bincount(own, weights=cells, minlength=n)
        assert len(np.unique(own)) == n
        assert np.all(np.abs(w - cells.sum() / n) <= cells.max())
    # explicit weights (e.g. fluid cells) steer the cut
    wts = np.linspace(1.0, 5.0, len(blocks))
    own = lbm.lbm_partition_morton(blocks, 4, wts)
    w = np.bincount(own, weights=wts, minlength=4)
    assert np.all(np.abs(w - wts.sum() / 4) <= wts.max())


def _layouts(sim):
    return [lbm.lbm_plan_layout(sim.ctx, b) for b in range(len(sim.blocks))]


def _slot_id(q, j, g, shape):
    """The number naming slot j of global cell g (1-based, so 0 never names a slot)."""
    nx, ny, nz = shape
    return 1 + j + q * (g[0] + nx * (g[1] + ny * g[2]))


def _arena(sim, lay, shape, q, fill=True):
    """A host stand-in for the rank's PDF array: every owned interior slot holds its name."""
    owned = [b for b in range(len(sim.blocks)) if sim.owner is None or sim.owner[b] == sim.rank]
    size = max(lay[b]["offset"] + q * lay[b]["slab"] for b in owned)
    A = np.zeros(size, dtype=np.int64)
    if not fill:
        return A
    for b in owned:
        (o, s), L = sim.blocks[b], lay[b]
        z, y, x = np.meshgrid(np.arange(s[2]), np.arange(s[1]), np.arange(s[0]), indexing="ij")
        cell = (z + 1) * L["plane"] + (y + 1) * L["pitch"] + L["xo"] + x
        for j in range(q):
            A[L["offset"] + j * L["slab"] + cell] = _slot_id(q, j, (o[0] + x, o[1] + y, o[2] + z), shape)
    return A


def _decode(sim, lay, off, q):
    """(block, slot, local x, y, z) of an arena offset of this rank."""
    for b, L in enumerate(lay):
        if L["offset"] < 0 or not (L["offset"] <= off < L["offset"] + q * L["slab"]):
            continue
        j, cell = divmod(off - L["offset"], L["slab"])
        z, r = divmod(cell, L["plane"])
        y, x = divmod(r, L["pitch"])
        return b, j, x - L["xo"], y - 1, z - 1
    raise AssertionError("offset %d outside every owned block" % off)


def _expected(sim, lay, off, q, shape, periodic):
    b, j, x, y, z = _decode(sim, lay, off, q)
    o = sim.blocks[b][0]
    g = [o[0] + x, o[1] + y, o[2] + z]
    for a in range(3):
        if periodic[a]:
            g[a] %= shape[a]
    return _slot_id(q, j, g, shape)


def _pack(A, runs, buf):
    for arena, boff, n, stride in runs:
        buf[boff:boff + n] = A[arena + stride * np.arange(n)]


def _unpack(A, runs, buf):
    for arena, boff, n, stride in runs:
        A[arena + stride * np.arange(n)] = buf[boff:boff + n]


def _size(runs):
    return int((runs[:, 1] + runs[:, 2]).max()) if runs.size else 0


@pytest.mark.parametrize("q,nranks,pattern", [(19, 2, lbm.TWO_GRID), (19, 3, lbm.AA), (27, 4, lbm.TWO_GRID)])
def test_halo_lists_deliver_every_mirrored_slot(q, nranks, pattern):
    blocks, shape, flags, p = _case(q=q, pattern=pattern)
    periodic = (0, 1, 1)
    owner = lbm.lbm_partition_morton(blocks, nranks)
    sims = [_make(p, blocks, flags, owner, nranks, r) for r in range(nranks)]
    try:
        lays = [_layouts(s) for s in sims]
        A = [_arena(s, lays[r], shape, q) for r, s in enumerate(sims)]
        sel = (0, 1) if pattern == lbm.TWO_GRID else (2, 3)
        # forward: every rank packs for every peer, then every rank unpacks
        bufs = {}
        for r in range(nranks):
            for peer in range(nranks):
                if peer == r:
                    continue
                send = lbm.lbm_plan_halo(sims[r].ctx, peer, sel[0])
                recv = lbm.lbm_plan_halo(sims[peer].ctx, r, sel[1])
                assert _size(send) == _size(recv)
                assert lbm.lbm_halo_sizes(sims[r].ctx, peer)[0] == _size(send)
                bufs[(r, peer)] = np.zeros(_size(send), dtype=np.int64)
                _pack(A[r], send, bufs[(r, peer)])
        received = 0
        for (r, peer), buf in bufs.items():
            recv = lbm.lbm_plan_halo(sims[peer].ctx, r, sel[1])
            _unpack(A[peer], recv, buf)
            for arena, boff, n, stride in recv:
                for k in range(n):
                    off = arena + stride * k
                    assert A[peer][off] == _expected(sims[peer], lays[peer], off, q, shape, periodic)
                    # the value came from the peer the list names
                    assert owner[_decode_src(A[peer][off], q, shape, blocks)] == r
                received += n
        assert received > 0
        if pattern == lbm.AA:
            # reverse exchange: what the neighbour sweep leaves in a ghost slot goes back to the
            # interior slot it mirrors (here: the negated name, so the round trip is visible)
            for r in range(nranks):
                for peer in range(nranks):
                    if peer != r:
                        for arena, boff, n, stride in lbm.lbm_plan_halo(sims[r].ctx, peer, 3):
                            idx = arena + stride * np.arange(n)
                            A[r][idx] = -A[r][idx]
            back = {}
            for r in range(nranks):
                for peer in range(nranks):
                    if peer != r:
                        rv = lbm.lbm_plan_halo(sims[r].ctx, peer, 3)
                        back[(r, peer)] = np.zeros(_size(rv), dtype=np.int64)
                        _pack(A[r], rv, back[(r, peer)])
            for (r, peer), buf in back.items():
                snd = lbm.lbm_plan_halo(sims[peer].ctx, r, 2)
                _unpack(A[peer], snd, buf)
                for arena, boff, n, stride in snd:
                    for k in range(n):
                        off = arena + stride * k
                        assert A[peer][off] == -_expected(sims[peer], lays[peer], off, q, shape, periodic)
    finally:
        for s in sims:
            s.close()


def _decode_src(value, q, shape, blocks):
    """Block holding the global cell a slot name refers to."""
    nx, ny, _ = shape
    cell = (value - 1) // q
    g = (cell % nx, (cell // nx) % ny, cell // (nx * ny))
    for b, (o, s) in enumerate(blocks):
        if all(o[a] <= g[a] < o[a] + s[a] for a in range(3)):
            return b
    raise AssertionError("no block holds %s" % (g,))


@pytest.mark.parametrize("pattern", [lbm.TWO_GRID, lbm.AA])
def test_partitioned_lists_cover_the_unpartitioned_ghost_copies(pattern):
    """Ghost copies of one context that holds every block (in-place access off) = the union
    over ranks of the local ghost copies and the halo receive lists, slot by slot."""
    q, nranks = 19, 3
    blocks, shape, flags, p = _case(pattern=pattern)
    whole = _make(p, blocks, flags)
    lbm.lbm_set_in_place(whole.ctx, False)
    owner = lbm.lbm_partition_morton(blocks, nranks)
    sims = [_make(p, blocks, flags, owner, nranks, r) for r in range(nranks)]
    try:
        def global_dst(sim, lay, runs_dst):
            out = set()
            for off in runs_dst:
                b, j, x, y, z = _decode(sim, lay, off, q)
                out.add((b, j, x, y, z))
            return out

        lay_w = _layouts(whole)
        want = set()
        for src, dst, n, ss, ds in lbm.lbm_plan_runs(whole.ctx, pattern):
            want |= global_dst(whole, lay_w, [dst + ds * k for k in range(n)])
        got = set()
        for r, s in enumerate(sims):
            lay = _layouts(s)
            for src, dst, n, ss, ds in lbm.lbm_plan_runs(s.ctx, pattern):
                got |= global_dst(s, lay, [dst + ds * k for k in range(n)])
            for peer in range(nranks):
                if peer != r:
                    for arena, boff, n, stride in lbm.lbm_plan_halo(s.ctx, peer, 1 if pattern == lbm.TWO_GRID else 3):
                        got |= global_dst(s, lay, [arena + stride * k for k in range(n)])
        assert got == want and len(want) > 0
    finally:
        whole.close()
        for s in sims:
            s.close()


def test_remote_blocks_are_refused_for_pdf_calls():
    blocks, shape, flags, p = _case()
    owner = lbm.lbm_partition_morton(blocks, 2)
    sim = _make(p, blocks, flags, owner, 2, 0)
    try:
        b = int(np.flatnonzero(owner == 1)[0])
        rho, u = inputs.rest(sim.blocks[b][1])
        with pytest.raises(lbm.LbmError) as e:
            sim.init(b, rho, u)
        assert e.value.status == 1 and "belongs to rank 1" in str(e.value)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_halo_sizes(sim.ctx, 0)  # itself is no peer
        assert e.value.status == 1
    finally:
        sim.close()
    with pytest.raises(lbm.LbmError):  # a rank that owns no block
        lbm.Simulation(p, blocks, owner=np.zeros(len(blocks), np.int32), nranks=2, rank=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, q_out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1909_13772_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q = 19
        blocks, shape, flags, p = _case()
        owner = lbm.lbm_partition_morton(blocks, world)
        sim = _make(p, blocks, flags, owner, world, rank)
        lay = _layouts(sim)
        A = _arena(sim, lay, shape, q)
        peer = 1 - rank
        send_runs, recv_runs = lbm.lbm_plan_halo(sim.ctx, peer, 0), lbm.lbm_plan_halo(sim.ctx, peer, 1)
        ns, nr = lbm.lbm_halo_sizes(sim.ctx, peer)
        buf = np.zeros(ns, dtype=np.int64)
        _pack(A, send_runs, buf)
        recv = {peer: torch.zeros(nr, dtype=torch.int64)}
        shard.exchange_buffers({peer: torch.from_numpy(buf)}, recv)
        _unpack(A, recv_runs, recv[peer].numpy())
        bad = 0
        for arena, boff, n, stride in recv_runs:
            for k in range(n):
                off = arena + stride * k
                bad += int(A[off] != _expected(sim, lay, off, q, shape, (0, 1, 1)))
        sim.close()
        q_out.put((rank, ns, nr, bad))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_the_halo():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, s0, v0, bad0), (r1, s1, v1, bad1) = out
    assert (r0, r1) == (0, 1)
    assert s0 == v1 > 0 and s1 == v0 > 0
    assert bad0 == 0 and bad1 == 0


def test_combine_diagnostics_sums_in_rank_order_and_takes_the_max_speed():
    from paper_1909_13772_gb300 import shard
    a = {"mass": 1.0, "momentum": (1e-3, 0.0, -2e-3), "kinetic_energy": 0.5, "max_speed": 0.02, "nonfinite": 0,
         "fluid_cells": 10}
    b = {"mass": 1e-16, "momentum": (0.0, 1.0, 0.0), "kinetic_energy": 0.25, "max_speed": 0.05, "nonfinite": 2,
         "fluid_cells": 7}
    c = {"mass": -1.0, "momentum": (0.0, 0.0, 0.0), "kinetic_energy": 0.0, "max_speed": 0.01, "nonfinite": 0,
         "fluid_cells": 3}
    d = shard.combine_diagnostics([a, b, c])
    assert d["mass"] == (1.0 + 1e-16) + -1.0  # the rank order, not a reassociated sum
    assert d["momentum"] == (1e-3, 1.0, -2e-3)
    assert d["kinetic_energy"] == 0.75 and d["max_speed"] == 0.05
    assert d["nonfinite"] == 2 and d["fluid_cells"] == 20


def _gloo_reduce_rank(rank, world, port, q_out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1909_13772_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = {"mass": 0.1 * (rank + 1), "momentum": (1e-17 * rank, -rank, 3.0), "kinetic_energy": 2.0 ** -rank,
                 "max_speed": 0.01 * (3 - rank), "nonfinite": rank, "fluid_cells": 1000 + rank}
        q_out.put((rank, shard.allreduce_diagnostics(local)))
    finally:
        dist.destroy_process_group()


def test_three_gloo_ranks_allreduce_the_diagnostics_identically():
    pytest.importorskip("torch")
    from paper_1909_13772_gb300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_reduce_rank, args=(r, 3, port, q)) for r in range(3)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    want = shard.combine_diagnostics([
        {"mass": 0.1 * (r + 1), "momentum": (1e-17 * r, -r, 3.0), "kinetic_energy": 2.0 ** -r,
         "max_speed": 0.01 * (3 - r), "nonfinite": r, "fluid_cells": 1000 + r} for r in range(3)])
    for _, got in out:
        assert got == want  # every rank the same bits, in rank order
