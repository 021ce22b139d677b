"""Partitioned runs: the blocks of one domain spread over ranks (one per GPU), each rank sweeping
its own blocks and exchanging the ghost-layer halo with its neighbour ranks between steps.

Paper: Sec. 3.1 (blocks distributed over processes along a space-filling curve, here the Morton
curve of the block centres, lbm_partition_morton) and Sec. 3.3 (ghost-layer exchange: only the
PDFs that cross into a neighbour's ghost layer, packed into one message per neighbour).  The
library packs and unpacks (lbm_halo_pack / lbm_halo_unpack); this module moves the buffers:

* ``PartitionedRun`` -- one rank of a torch.distributed job: point-to-point send/recv of the
  packed buffers (NCCL between GPUs; any backend whose tensors live where the buffers do);
* ``LocalPartition`` -- every rank's context in one process on one GPU, the buffers handed over
  by device copies on one stream (no waits between kernels of different contexts).

Domain totals (mass, momentum, kinetic energy, ...) are each rank's FP64 totals over its own
blocks (lbm_reduce), gathered to every rank and combined there in rank order
(``combine_diagnostics``), so every rank holds the same bits from run to run.

Marshalling only: every PDF moves through the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import lbm

_TORCH_DTYPE = {lbm.FP64: "float64", lbm.FP32: "float32", lbm.BF16_DEV: "bfloat16", lbm.FP16_DEV: "float16"}


def _dtype(storage):
    import torch
    return getattr(torch, _TORCH_DTYPE[storage])


def halo_peers(sim) -> list:
    """Ranks this context exchanges a halo with (for either pattern and parity)."""
    out = []
    for p in range(sim.nranks):
        if p == sim.rank:
            continue
        if any(lbm.lbm_plan_halo(sim.ctx, p, k).size for k in range(4)):
            out.append(p)
    return out


def _capacity(sim, peer):
    """Largest send and receive sizes with a peer over both AA parities (two-grid: one size)."""
    rows = [lbm.lbm_plan_halo(sim.ctx, peer, k) for k in range(4)]
    n = [int((r[:, 1] + r[:, 2]).max()) if r.size else 0 for r in rows]
    return max(n)


_DIAG_SUMS = ("mass", "momentum", "kinetic_energy", "nonfinite", "fluid_cells")


def _diag_vector(d) -> list:
    """One rank's totals as 8 doubles: mass, momentum x/y/z, kinetic energy, max speed,
    non-finite cells, fluid cells (counts are exact in FP64 up to 2^53)."""
    return [float(d["mass"])] + [float(v) for v in d["momentum"]] + [
        float(d["kinetic_energy"]), float(d["max_speed"]), float(d["nonfinite"]), float(d["fluid_cells"])]


def combine_diagnostics(per_rank: list) -> dict:
    """Domain totals from the ranks' own totals, in rank order: sums for mass, momentum, kinetic
    energy and the counts, maximum for the speed (FP64, a fixed order, no reassociation)."""
    rows = [_diag_vector(d) if isinstance(d, dict) else [float(v) for v in d] for d in per_rank]
    acc = list(rows[0])
    for r in rows[1:]:
        for k in range(8):
            acc[k] = max(acc[k], r[k]) if k == 5 else acc[k] + r[k]
    return {"mass": acc[0], "momentum": (acc[1], acc[2], acc[3]), "kinetic_energy": acc[4], "max_speed": acc[5],
            "nonfinite": int(acc[6]), "fluid_cells": int(acc[7])}


def allreduce_diagnostics(local: dict, group=None) -> dict:
    """Every rank's totals gathered to every rank (one all-gather of 8 doubles per rank) and
    combined in rank order: the same result, bit for bit, on every rank."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    v = torch.tensor(_diag_vector(local), dtype=torch.float64, device=dev)
    parts = [torch.empty_like(v) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, v, group=group)
    return combine_diagnostics([p.cpu().tolist() for p in parts])


def exchange_buffers(send: dict, recv: dict, group=None):
    """Post every send and receive of one halo exchange at once and wait for all of them:
    send[peer] / recv[peer] are tensors (empty ones are skipped)."""
    import torch.distributed as dist
    ops = []
    for p, t in sorted(send.items()):
        if t.numel():
            ops.append(dist.P2POp(dist.isend, t, p, group))
    for p, t in sorted(recv.items()):
        if t.numel():
            ops.append(dist.P2POp(dist.irecv, t, p, group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()


class PartitionedRun:
    """Rank `rank` of a `world`-rank run of one domain (every rank passes the same params,
    blocks, faces and flags).  The context works on the current torch stream, so the library's
    pack kernels, the communication and the unpack kernels are ordered on it."""

    def __init__(self, params, blocks, rank, world, owner=None, group=None):
        import torch
        self.owner = lbm.lbm_partition_morton(blocks, world) if owner is None else np.asarray(owner, np.int32)
        self.stream = torch.cuda.current_stream()
        self.sim = lbm.Simulation(params, blocks, stream=self.stream.cuda_stream, owner=self.owner, nranks=world,
                                  rank=rank)
        self.rank, self.world, self.group = rank, world, group
        self._peers = None
        self._send, self._recv = {}, {}

    def owned(self):
        return [b for b in range(len(self.sim.blocks)) if self.owner[b] == self.rank]

    def _buffers(self):
        import torch
        if self._peers is None:
            self._peers = halo_peers(self.sim)
            dt = _dtype(self.sim.params.storage)
            for p in self._peers:
                n = _capacity(self.sim, p)
                self._send[p] = torch.empty(n, dtype=dt, device="cuda")
                self._recv[p] = torch.empty(n, dtype=dt, device="cuda")

    def exchange(self):
        """The halo exchange that must precede the next step."""
        self._buffers()
        send, recv = {}, {}
        for p in self._peers:
            ns, nr = lbm.lbm_halo_sizes(self.sim.ctx, p)
            if ns:
                lbm.lbm_halo_pack(self.sim.ctx, p, self._send[p].data_ptr())
            send[p], recv[p] = self._send[p][:ns], self._recv[p][:nr]
        exchange_buffers(send, recv, self.group)
        for p in self._peers:
            if recv[p].numel():
                lbm.lbm_halo_unpack(self.sim.ctx, p, recv[p].data_ptr())

    def step(self, n=1):
        for _ in range(int(n)):
            self.exchange()
            lbm.lbm_step(self.sim.ctx, 1)

    def reduce(self):
        """Domain totals of the current state (FP64, the same bits on every rank)."""
        return allreduce_diagnostics(self.sim.reduce(), self.group)

    def close(self):
        self.sim.close()


class LocalPartition:
    """Every rank's context of a partitioned run in one process on one GPU: the packed
    buffers go from rank to rank by device copies, all on one stream."""

    def __init__(self, params, blocks, nranks, owner=None, stream=None):
        import torch
        self.owner = lbm.lbm_partition_morton(blocks, nranks) if owner is None else np.asarray(owner, np.int32)
        self.stream = stream or torch.cuda.current_stream()
        self.sims = [lbm.Simulation(params, blocks, stream=self.stream.cuda_stream, owner=self.owner, nranks=nranks,
                                    rank=r) for r in range(nranks)]
        self.nranks = nranks
        self._bufs = None

    def _buffers(self):
        import torch
        if self._bufs is None:
            self._bufs = {}
            dt = _dtype(self.sims[0].params.storage)
            for r, s in enumerate(self.sims):
                for p in halo_peers(s):
                    self._bufs[(r, p)] = torch.empty(_capacity(s, p), dtype=dt, device="cuda")

    def exchange(self):
        self._buffers()
        import torch
        with torch.cuda.stream(self.stream):
            sizes = {}
            for (r, p), buf in self._bufs.items():
                ns, _ = lbm.lbm_halo_sizes(self.sims[r].ctx, p)
                sizes[(r, p)] = ns
                if ns:
                    lbm.lbm_halo_pack(self.sims[r].ctx, p, buf.data_ptr())
            for (r, p), buf in self._bufs.items():
                # rank p receives what r packed for it (the same element order on both sides)
                _, nr = lbm.lbm_halo_sizes(self.sims[p].ctx, r)
                if nr != sizes[(r, p)]:
                    raise RuntimeError("halo sizes of ranks %d and %d disagree" % (r, p))
                if nr:
                    lbm.lbm_halo_unpack(self.sims[p].ctx, r, buf.data_ptr())

    def step(self, n=1):
        for _ in range(int(n)):
            self.exchange()
            for s in self.sims:
                lbm.lbm_step(s.ctx, 1)

    def reduce(self):
        """Domain totals of the current state: every rank's own totals combined in rank order."""
        return combine_diagnostics([s.reduce() for s in self.sims])

    def close(self):
        for s in self.sims:
            s.close()
