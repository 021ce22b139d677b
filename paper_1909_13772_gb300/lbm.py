"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every function of the C ABI is exposed under the same name; each raises ``LbmError`` on a
non-zero status.  ``Simulation`` bundles a context with NumPy-friendly calls.  All compute
runs in the library's CUDA kernels; there is no CPU fallback -- if the library cannot be
built or loaded, importing the functions fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

D3Q19, D3Q27 = 19, 27
SRT, TRT, MRT, CUMULANT = 0, 1, 2, 3
FP64, FP32, BF16_DEV, FP16_DEV = 0, 1, 2, 3
TWO_GRID, AA = 0, 1
FLUID, NOSLIP, VELOCITY, PRESSURE, PERIODIC = 0, 1, 2, 3, 4
ZOUHE_VELOCITY, ZOUHE_PRESSURE = 5, 6  # face kinds only: wet-node (Zou-He) faces
REFINE = 7  # face kind only: a refinement interface (lbm_refine_create)

STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_STATE", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_OOM",
          5: "LBM_ERR_DIVERGED", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_UNSUPPORTED"}


class LbmError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__("%s: %s" % (STATUS.get(status, status), message))


class lbm_params(ctypes.Structure):
    _fields_ = [("stencil", ctypes.c_int32), ("collision", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("pattern", ctypes.c_int32), ("omega", ctypes.c_double), ("magic_lambda", ctypes.c_double),
                ("force", ctypes.c_double * 3), ("rho0", ctypes.c_double), ("periodic", ctypes.c_int32 * 3),
                ("diag_interval", ctypes.c_int32), ("mrt_rates", ctypes.c_double * 4),
                ("cumulant_rates", ctypes.c_double * 9)]


class lbm_block_desc(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_int64 * 3), ("size", ctypes.c_int32 * 3)]


class lbm_diagnostics(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("kinetic_energy", ctypes.c_double),
                ("max_speed", ctypes.c_double), ("nonfinite", ctypes.c_int64), ("fluid_cells", ctypes.c_int64)]


class lbm_info(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("fluid_cells", ctypes.c_int64), ("links", ctypes.c_int64 * 4),
                ("ghost_slots", ctypes.c_int64), ("ghost_runs", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("bytes_per_pdf", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("staged_tiles", ctypes.c_int64),
                ("list_entries", ctypes.c_int64)]


_lib = None
_P = ctypes.POINTER
_vp, _dp, _u8p, _i32p, _i64p, _u64p = (ctypes.c_void_p, _P(ctypes.c_double), _P(ctypes.c_uint8),
                                       _P(ctypes.c_int32), _P(ctypes.c_int64), _P(ctypes.c_uint64))
_SIGS = {
    "lbm_create_blocks": ([_P(lbm_params), _P(lbm_block_desc), ctypes.c_int32, _vp, _P(_vp)], ctypes.c_int),
    "lbm_create_partition": ([_P(lbm_params), _P(lbm_block_desc), ctypes.c_int32, _i32p, ctypes.c_int32,
                              ctypes.c_int32, _vp, _P(_vp)], ctypes.c_int),
    "lbm_partition_morton": ([_P(lbm_block_desc), ctypes.c_int32, ctypes.c_int32, _dp, _i32p], ctypes.c_int),
    "lbm_halo_sizes": ([_vp, ctypes.c_int32, _i64p, _i64p], ctypes.c_int),
    "lbm_halo_pack": ([_vp, ctypes.c_int32, _vp], ctypes.c_int),
    "lbm_halo_unpack": ([_vp, ctypes.c_int32, _vp], ctypes.c_int),
    "lbm_plan_halo": ([_vp, ctypes.c_int32, ctypes.c_int32, _i64p, ctypes.c_int64, _i64p], ctypes.c_int),
    "lbm_set_sparse": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_plan_sparse": ([_vp, ctypes.c_int32, _i64p, ctypes.c_int64, _i64p], ctypes.c_int),
    "lbm_required_bytes": ([_vp], ctypes.c_size_t),
    "lbm_bind_device_memory": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "lbm_set_face": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _dp, ctypes.c_double], ctypes.c_int),
    "lbm_set_boundary": ([_vp, ctypes.c_int32, _u8p, _dp, ctypes.c_double], ctypes.c_int),
    "lbm_init_macroscopic": ([_vp, ctypes.c_int32, _dp, _dp], ctypes.c_int),
    "lbm_step": ([_vp, ctypes.c_int64], ctypes.c_int),
    "lbm_get_macroscopic": ([_vp, ctypes.c_int32, _dp, _dp], ctypes.c_int),
    "lbm_get_pdfs": ([_vp, ctypes.c_int32, _dp], ctypes.c_int),
    "lbm_set_pdfs": ([_vp, ctypes.c_int32, _dp], ctypes.c_int),
    "lbm_get_pdfs_region": ([_vp, ctypes.c_int32, _i32p, _i32p, _dp], ctypes.c_int),
    "lbm_reduce": ([_vp, _P(lbm_diagnostics)], ctypes.c_int),
    "lbm_step_diagnostics": ([_vp, _P(lbm_diagnostics)], ctypes.c_int),
    "lbm_step_diagnostics_post": ([_vp, _i64p], ctypes.c_int),
    "lbm_step_diagnostics_take": ([_vp, ctypes.c_int64, _P(lbm_diagnostics)], ctypes.c_int),
    "lbm_selfcheck_wait": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_get_info": ([_vp, _P(lbm_info)], ctypes.c_int),
    "lbm_set_tile": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "lbm_kernel_launches": ([_vp], ctypes.c_int64),
    "lbm_set_graph": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_set_index_bits": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_set_batching": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_set_in_place": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_autotune": ([_vp, ctypes.c_int32, _i32p, _i32p, _dp], ctypes.c_int),
    "lbm_enable_timing": ([_vp, ctypes.c_int32], ctypes.c_int),
    "lbm_read_timing": ([_vp, _dp, _i64p, ctypes.c_int32], ctypes.c_int),
    "lbm_stencil_table": ([ctypes.c_int32, _i32p, _dp, _i32p], ctypes.c_int),
    "lbm_plan_links": ([_vp, _u64p, ctypes.c_int64, _i64p], ctypes.c_int),
    "lbm_plan_runs": ([_vp, ctypes.c_int32, _i64p, ctypes.c_int64, _i64p], ctypes.c_int),
    "lbm_plan_layout": ([_vp, ctypes.c_int32, _i64p], ctypes.c_int),
    "lbm_plan_neighbors": ([_vp, ctypes.c_int32, _i32p], ctypes.c_int),
    "lbm_plan_params": ([_vp, _dp, ctypes.c_int64, _i64p], ctypes.c_int),
    "lbm_plan_mask": ([_vp, ctypes.c_int32, _P(ctypes.c_uint32), ctypes.c_int64, _i64p], ctypes.c_int),
    "lbm_reduce_noalloc": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _dp, _vp, _vp], ctypes.c_int),
    "lbm_reduce_blocks": ([_vp, _dp], ctypes.c_int),
    "lbm_coarse_moments": ([_vp, ctypes.c_int32, ctypes.c_int32, _dp], ctypes.c_int),
    "lbm_set_closure": ([_vp, ctypes.c_int32, ctypes.c_double, _P(ctypes.c_float)], ctypes.c_int),
    "lbm_mlp_create": ([_P(ctypes.c_float), ctypes.c_int64, _vp, _P(_vp)], ctypes.c_int),
    "lbm_mlp_set_params": ([_vp, _P(ctypes.c_float)], ctypes.c_int),
    "lbm_mlp_get_params": ([_vp, _P(ctypes.c_float)], ctypes.c_int),
    "lbm_mlp_infer": ([_vp, _vp, ctypes.c_int64, _vp], ctypes.c_int),
    "lbm_mlp_loss_grad": ([_vp, _vp, _vp, ctypes.c_int64, _dp, _P(ctypes.c_float)], ctypes.c_int),
    "lbm_mlp_train": ([_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float, _dp],
                      ctypes.c_int),
    "lbm_mlp_destroy": ([_vp], None),
    "lbm_last_error": ([_vp], ctypes.c_char_p),
    "lbm_destroy": ([_vp], None),
    "lbm_refine_create": ([_vp, _vp, _P(_vp)], ctypes.c_int),
    "lbm_refine_step": ([_vp, ctypes.c_int64], ctypes.c_int),
    "lbm_refine_destroy": ([_vp], None),
}


def library_path() -> str:
    from . import build as _build
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load liblbm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    override = os.environ.get("LBM_LIBRARY")
    if override:
        path = override
    else:
        path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError("liblbm.so not found at %s; run paper_1909_13772_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a, ctype):
    return a.ctypes.data_as(_P(ctype)) if a is not None else None


def _check(ctx, status):
    if status != 0:
        msg = load_library().lbm_last_error(ctx).decode() if ctx else ""
        raise LbmError(status, msg)


# ---- the C ABI under its own names ------------------------------------------------------

def _block_array(blocks):
    arr = (lbm_block_desc * len(blocks))()
    for k, (o, s) in enumerate(blocks):
        for a in range(3):
            arr[k].origin[a] = int(o[a])
            arr[k].size[a] = int(s[a])
    return arr


def lbm_create_blocks(params: lbm_params, blocks, stream=None):
    """blocks: sequence of (origin(3), size(3)).  Returns an opaque context handle."""
    L = load_library()
    arr = _block_array(blocks)
    out = ctypes.c_void_p()
    st = L.lbm_create_blocks(ctypes.byref(params), arr, len(blocks), ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if st != 0:
        raise LbmError(st, "lbm_create_blocks rejected the parameters or block layout")
    return out


def lbm_create_partition(params: lbm_params, blocks, owner, nranks, rank, stream=None):
    """A context of rank `rank` holding the blocks with owner[b] == rank."""
    L = load_library()
    arr = _block_array(blocks)
    own = np.ascontiguousarray(owner, dtype=np.int32)
    if own.shape != (len(blocks),):
        raise ValueError("owner needs one entry per block")
    out = ctypes.c_void_p()
    st = L.lbm_create_partition(ctypes.byref(params), arr, len(blocks), _ptr(own, ctypes.c_int32), int(nranks),
                                int(rank), ctypes.c_void_p(stream or 0), ctypes.byref(out))
    if st != 0:
        raise LbmError(st, "lbm_create_partition rejected the parameters, blocks or owner array")
    return out


def lbm_partition_morton(blocks, nranks, weights=None) -> np.ndarray:
    """Owner rank of every block along the Morton curve of the block centres (host only)."""
    L = load_library()
    arr = _block_array(blocks)
    own = np.zeros(len(blocks), dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    st = L.lbm_partition_morton(arr, len(blocks), int(nranks), _ptr(w, ctypes.c_double), _ptr(own, ctypes.c_int32))
    if st != 0:
        raise LbmError(st, "lbm_partition_morton rejected its arguments")
    return own


def lbm_halo_sizes(ctx, peer):
    """(send, receive) elements of the exchange with `peer` that must precede the next step."""
    ns, nr = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load_library().lbm_halo_sizes(ctx, int(peer), ctypes.byref(ns), ctypes.byref(nr)))
    return ns.value, nr.value


def lbm_halo_pack(ctx, peer, dev_ptr: int):
    _check(ctx, load_library().lbm_halo_pack(ctx, int(peer), ctypes.c_void_p(dev_ptr)))


def lbm_halo_unpack(ctx, peer, dev_ptr: int):
    _check(ctx, load_library().lbm_halo_unpack(ctx, int(peer), ctypes.c_void_p(dev_ptr)))


def lbm_refine_create(coarse_ctx, fine_ctx):
    """Coupling of a coarse and a fine context (static 2:1 refinement); errors reported on the
    coarse context."""
    r = _vp()
    _check(coarse_ctx, load_library().lbm_refine_create(coarse_ctx, fine_ctx, ctypes.byref(r)))
    return r


def lbm_refine_step(r, n, coarse_ctx=None):
    _check(coarse_ctx, load_library().lbm_refine_step(r, int(n)))


def lbm_refine_destroy(r):
    load_library().lbm_refine_destroy(r)


def lbm_plan_halo(ctx, peer, which) -> np.ndarray:
    """Halo runs with `peer` (which: 0 send pull, 1 receive pull, 2 send AA, 3 receive AA) as
    rows (arena offset, buffer offset, length, arena stride)."""
    L = load_library()
    n = ctypes.c_int64()
    _check(ctx, L.lbm_plan_halo(ctx, int(peer), int(which), None, 0, ctypes.byref(n)))
    out = np.zeros(4 * n.value, dtype=np.int64)
    _check(ctx, L.lbm_plan_halo(ctx, int(peer), int(which), _ptr(out, ctypes.c_int64), 4 * n.value, ctypes.byref(n)))
    return out.reshape(n.value, 4)


def lbm_required_bytes(ctx) -> int:
    return int(load_library().lbm_required_bytes(ctx))


def lbm_bind_device_memory(ctx, dev_ptr: int, nbytes: int):
    _check(ctx, load_library().lbm_bind_device_memory(ctx, ctypes.c_void_p(dev_ptr), nbytes))


def lbm_set_face(ctx, axis, side, kind, u_wall=(0.0, 0.0, 0.0), rho_wall=1.0):
    u = _arr(u_wall, np.float64)
    _check(ctx, load_library().lbm_set_face(ctx, axis, side, kind, _ptr(u, ctypes.c_double), float(rho_wall)))


def lbm_set_boundary(ctx, block, flags, u_wall=(0.0, 0.0, 0.0), rho_wall=1.0):
    f = None if flags is None else _arr(flags, np.uint8)
    u = _arr(u_wall, np.float64)
    _check(ctx, load_library().lbm_set_boundary(ctx, block, _ptr(f, ctypes.c_uint8), _ptr(u, ctypes.c_double),
                                                float(rho_wall)))


def lbm_init_macroscopic(ctx, block, rho, u):
    r = _arr(rho, np.float64)
    v = _arr(u, np.float64)
    _check(ctx, load_library().lbm_init_macroscopic(ctx, block, _ptr(r, ctypes.c_double), _ptr(v, ctypes.c_double)))


def lbm_step(ctx, n: int = 1):
    _check(ctx, load_library().lbm_step(ctx, int(n)))


def lbm_get_macroscopic(ctx, block, rho_out, u_out):
    _check(ctx, load_library().lbm_get_macroscopic(ctx, block, _ptr(rho_out, ctypes.c_double),
                                                   _ptr(u_out, ctypes.c_double)))


def lbm_get_pdfs(ctx, block, f_out):
    _check(ctx, load_library().lbm_get_pdfs(ctx, block, _ptr(f_out, ctypes.c_double)))


def lbm_get_pdfs_region(ctx, block, origin, size, q):
    """PDFs [q, sz, sy, sx] of the box origin (x, y, z) / size (sx, sy, sz) of a block."""
    o = _arr(origin, np.int32)
    n = _arr(size, np.int32)
    f = np.empty((q, int(n[2]), int(n[1]), int(n[0])), np.float64)
    _check(ctx, load_library().lbm_get_pdfs_region(ctx, block, _ptr(o, ctypes.c_int32), _ptr(n, ctypes.c_int32),
                                                   _ptr(f, ctypes.c_double)))
    return f


def lbm_set_pdfs(ctx, block, f):
    a = _arr(f, np.float64)
    _check(ctx, load_library().lbm_set_pdfs(ctx, block, _ptr(a, ctypes.c_double)))


def lbm_reduce(ctx) -> dict:
    d = lbm_diagnostics()
    _check(ctx, load_library().lbm_reduce(ctx, ctypes.byref(d)))
    return {"mass": d.mass, "momentum": tuple(d.momentum), "kinetic_energy": d.kinetic_energy,
            "max_speed": d.max_speed, "nonfinite": d.nonfinite, "fluid_cells": d.fluid_cells}


def lbm_step_diagnostics(ctx) -> dict:
    d = lbm_diagnostics()
    _check(ctx, load_library().lbm_step_diagnostics(ctx, ctypes.byref(d)))
    return {"mass": d.mass, "momentum": tuple(d.momentum), "kinetic_energy": d.kinetic_energy,
            "max_speed": d.max_speed, "nonfinite": d.nonfinite, "fluid_cells": d.fluid_cells}


def lbm_step_diagnostics_post(ctx) -> int:
    t = ctypes.c_int64()
    _check(ctx, load_library().lbm_step_diagnostics_post(ctx, ctypes.byref(t)))
    return t.value


def lbm_step_diagnostics_take(ctx, ticket) -> dict:
    d = lbm_diagnostics()
    _check(ctx, load_library().lbm_step_diagnostics_take(ctx, ticket, ctypes.byref(d)))
    return {"mass": d.mass, "momentum": tuple(d.momentum), "kinetic_energy": d.kinetic_energy,
            "max_speed": d.max_speed, "nonfinite": d.nonfinite, "fluid_cells": d.fluid_cells}


def lbm_selfcheck_wait(ctx, polls=1024):
    _check(ctx, load_library().lbm_selfcheck_wait(ctx, polls))


def lbm_get_info(ctx) -> dict:
    i = lbm_info()
    _check(ctx, load_library().lbm_get_info(ctx, ctypes.byref(i)))
    return {"cells": i.cells, "fluid_cells": i.fluid_cells, "links": tuple(i.links), "ghost_slots": i.ghost_slots,
            "ghost_runs": i.ghost_runs, "tiles": i.tiles, "bytes_per_pdf": i.bytes_per_pdf,
            "device_bytes": i.device_bytes, "staged_tiles": i.staged_tiles, "list_entries": i.list_entries}


def lbm_set_tile(ctx, tx, ty, tz):
    _check(ctx, load_library().lbm_set_tile(ctx, tx, ty, tz))


def lbm_set_batching(ctx, batched=True):
    _check(ctx, load_library().lbm_set_batching(ctx, 1 if batched else 0))


def lbm_set_sparse(ctx, enable=True):
    """Fluid-cell list layout of the two-grid sweep (True) or the dense block layout (False)."""
    _check(ctx, load_library().lbm_set_sparse(ctx, 1 if enable else 0))


def lbm_plan_sparse(ctx, what) -> np.ndarray:
    """Host copy of a part of the fluid-cell list layout (0 table, 1 block, 2 cell, 3 links)."""
    L = load_library()
    n = ctypes.c_int64()
    _check(ctx, L.lbm_plan_sparse(ctx, int(what), None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.int64)
    if n.value:
        _check(ctx, L.lbm_plan_sparse(ctx, int(what), _ptr(out, ctypes.c_int64), n.value, ctypes.byref(n)))
    return out


def lbm_set_in_place(ctx, enable=True):
    """Read matching neighbour blocks in place (True, default) or fill ghost layers by copies."""
    _check(ctx, load_library().lbm_set_in_place(ctx, 1 if enable else 0))


def lbm_set_graph(ctx, enable=True):
    _check(ctx, load_library().lbm_set_graph(ctx, 1 if enable else 0))


def lbm_set_index_bits(ctx, bits):
    _check(ctx, load_library().lbm_set_index_bits(ctx, int(bits)))


def lbm_autotune(ctx, trial_steps=20):
    """(best tile (tx, ty, tz), ms per step of the best candidate, in-place neighbour mode of
    it); the state is unchanged."""
    best = np.zeros(3, dtype=np.int32)
    mode = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(ctx, load_library().lbm_autotune(ctx, int(trial_steps), _ptr(best, ctypes.c_int32), ctypes.byref(mode),
                                            ctypes.byref(ms)))
    return tuple(int(v) for v in best), ms.value, bool(mode.value)


def lbm_kernel_launches(ctx) -> int:
    return int(load_library().lbm_kernel_launches(ctx))


def lbm_enable_timing(ctx, enable=True):
    _check(ctx, load_library().lbm_enable_timing(ctx, 1 if enable else 0))


def lbm_read_timing(ctx, reset=True) -> dict:
    """{'fill': (ms, launches), 'sweep': (ms, launches)} summed since the last reset."""
    ms = np.zeros(2, dtype=np.float64)
    cnt = np.zeros(2, dtype=np.int64)
    _check(ctx, load_library().lbm_read_timing(ctx, _ptr(ms, ctypes.c_double), _ptr(cnt, ctypes.c_int64),
                                               1 if reset else 0))
    return {"fill": (float(ms[0]), int(cnt[0])), "sweep": (float(ms[1]), int(cnt[1]))}


def lbm_stencil_table(q: int):
    c = np.zeros(3 * q, dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    st = load_library().lbm_stencil_table(q, _ptr(c, ctypes.c_int32), _ptr(w, ctypes.c_double),
                                          _ptr(opp, ctypes.c_int32))
    if st != 0:
        raise LbmError(st, "unknown stencil %d" % q)
    return c.reshape(q, 3), w, opp


def lbm_plan_links(ctx) -> np.ndarray:
    L = load_library()
    n = ctypes.c_int64()
    _check(ctx, L.lbm_plan_links(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.uint64)
    _check(ctx, L.lbm_plan_links(ctx, _ptr(out, ctypes.c_uint64), n.value, ctypes.byref(n)))
    return out


def lbm_plan_runs(ctx, pattern) -> np.ndarray:
    L = load_library()
    n = ctypes.c_int64()
    _check(ctx, L.lbm_plan_runs(ctx, pattern, None, 0, ctypes.byref(n)))
    out = np.zeros(5 * n.value, dtype=np.int64)
    _check(ctx, L.lbm_plan_runs(ctx, pattern, _ptr(out, ctypes.c_int64), 5 * n.value, ctypes.byref(n)))
    return out.reshape(n.value, 5)


def lbm_plan_layout(ctx, block) -> dict:
    out = np.zeros(10, dtype=np.int64)
    _check(ctx, load_library().lbm_plan_layout(ctx, block, _ptr(out, ctypes.c_int64)))
    keys = ("xo", "pitch", "plane", "slab", "offset", "nx", "ny", "nz", "arena_elems", "through")
    return {k: int(v) for k, v in zip(keys, out)}


def lbm_plan_mask(ctx, block) -> np.ndarray:
    L = load_library()
    n = ctypes.c_int64()
    _check(ctx, L.lbm_plan_mask(ctx, block, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.uint32)
    if n.value:
        _check(ctx, L.lbm_plan_mask(ctx, block, _ptr(out, ctypes.c_uint32), n.value, ctypes.byref(n)))
    return out


def lbm_plan_neighbors(ctx, block) -> np.ndarray:
    out = np.zeros(27, dtype=np.int32)
    _check(ctx, load_library().lbm_plan_neighbors(ctx, block, _ptr(out, ctypes.c_int32)))
    return out


def lbm_plan_params(ctx) -> np.ndarray:
    L = load_library()
    n = ctypes.c_int64()
    _check(ctx, L.lbm_plan_params(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros(4 * n.value, dtype=np.float64)
    _check(ctx, L.lbm_plan_params(ctx, _ptr(out, ctypes.c_double), 4 * n.value, ctypes.byref(n)))
    return out.reshape(n.value, 4)


REDUCE_NOALLOC_MAX_CELLS = 134217728
DIAG_SLOTS = 4  # pinned slots of the pipelined step-diagnostics read


def lbm_reduce_noalloc(f_dev_ptr: int, stencil: int, storage: int, ncells: int, force, out_dev_ptr: int, stream=None):
    """Allocation-free diagnostics of a caller-owned dense device field (see include/lbm.h);
    writes 8 doubles to out_dev_ptr asynchronously on ``stream``."""
    F = _arr(force if force is not None else (0.0, 0.0, 0.0), np.float64)
    st = load_library().lbm_reduce_noalloc(ctypes.c_void_p(f_dev_ptr), stencil, storage, int(ncells),
                                           _ptr(F, ctypes.c_double), ctypes.c_void_p(out_dev_ptr),
                                           ctypes.c_void_p(stream or 0))
    if st != 0:
        why = {1: "null pointer, unknown stencil or ncells <= 0",
               7: "storage must be FP64 or FP32 and ncells <= %d" % REDUCE_NOALLOC_MAX_CELLS,
               3: "CUDA launch or scratch address lookup failed"}.get(st, "")
        raise LbmError(st, "lbm_reduce_noalloc: " + why)


def lbm_reduce_blocks(ctx, nblocks) -> np.ndarray:
    """Per-block diagnostics: array [nblocks, 8] (mass, momentum x/y/z, kinetic energy, max
    speed, non-finite cells, fluid cells)."""
    out = np.empty((nblocks, 8), np.float64)
    _check(ctx, load_library().lbm_reduce_blocks(ctx, _ptr(out, ctypes.c_double)))
    return out


def lbm_coarse_moments(ctx, block, ratio, shape) -> np.ndarray:
    """Box sums over ratio^3 cells: array [10, NZ, NY, NX] (rho, rho u (3), rho u_a u_b (6));
    ``shape`` = the block's interior size (nx, ny, nz)."""
    nx, ny, nz = shape
    out = np.empty((10, nz // ratio, ny // ratio, nx // ratio), np.float64)
    _check(ctx, load_library().lbm_coarse_moments(ctx, block, ratio, _ptr(out, ctypes.c_double)))
    return out


CLOSURE_NONE, CLOSURE_SMAGORINSKY, CLOSURE_MLP = 0, 1, 2
MLP_NPARAM = 1348


def lbm_set_closure(ctx, kind, cs=0.0, mlp_params=None):
    """Per-cell relaxation from a closure (Smagorinsky constant cs, or packed network
    parameters, MLP_NPARAM floats)."""
    P = _arr(mlp_params, np.float32) if mlp_params is not None else None
    if P is not None and P.size != MLP_NPARAM:
        raise ValueError("network parameters must have %d entries" % MLP_NPARAM)
    _check(ctx, load_library().lbm_set_closure(ctx, int(kind), float(cs), _ptr(P, ctypes.c_float)))


def _mlp_check(status, what):
    if status != 0:
        raise LbmError(status, what)


def lbm_mlp_create(params, max_batch, stream=None):
    P = _arr(params, np.float32)
    if P.size != MLP_NPARAM:
        raise ValueError("network parameters must have %d entries" % MLP_NPARAM)
    h = _vp()
    _mlp_check(load_library().lbm_mlp_create(_ptr(P, ctypes.c_float), int(max_batch), _vp(stream or 0),
                                             ctypes.byref(h)), "lbm_mlp_create")
    return h


def lbm_mlp_set_params(m, params):
    P = _arr(params, np.float32)
    if P.size != MLP_NPARAM:
        raise ValueError("network parameters must have %d entries" % MLP_NPARAM)
    _mlp_check(load_library().lbm_mlp_set_params(m, _ptr(P, ctypes.c_float)), "lbm_mlp_set_params")


def lbm_mlp_get_params(m) -> np.ndarray:
    P = np.empty(MLP_NPARAM, np.float32)
    _mlp_check(load_library().lbm_mlp_get_params(m, _ptr(P, ctypes.c_float)), "lbm_mlp_get_params")
    return P


def lbm_mlp_infer(m, X_dev_ptr: int, n: int, y_dev_ptr: int):
    """y[s] = network output for features X[n][7] (device pointers, FP32)."""
    _mlp_check(load_library().lbm_mlp_infer(m, _vp(X_dev_ptr), int(n), _vp(y_dev_ptr)), "lbm_mlp_infer")


def lbm_mlp_loss_grad(m, X_dev_ptr: int, T_dev_ptr: int, n: int):
    """(loss, gradient[MLP_NPARAM]) of mean (softplus(y) - t)^2 over n samples."""
    loss = np.zeros(1, np.float64)
    g = np.empty(MLP_NPARAM, np.float32)
    _mlp_check(load_library().lbm_mlp_loss_grad(m, _vp(X_dev_ptr), _vp(T_dev_ptr), int(n), _ptr(loss, ctypes.c_double),
                                                _ptr(g, ctypes.c_float)), "lbm_mlp_loss_grad")
    return float(loss[0]), g


def lbm_mlp_train(m, X_dev_ptr: int, T_dev_ptr: int, n: int, batch: int, iters: int, lr: float) -> np.ndarray:
    """Adam steps on consecutive batches; returns the per-step batch losses."""
    hist = np.zeros(max(int(iters), 1), np.float64)
    _mlp_check(load_library().lbm_mlp_train(m, _vp(X_dev_ptr), _vp(T_dev_ptr), int(n), int(batch), int(iters),
                                            float(lr), _ptr(hist, ctypes.c_double)), "lbm_mlp_train")
    return hist[:int(iters)]


def lbm_mlp_destroy(m):
    load_library().lbm_mlp_destroy(m)


def lbm_last_error(ctx) -> str:
    return load_library().lbm_last_error(ctx).decode()


def lbm_destroy(ctx):
    load_library().lbm_destroy(ctx)


# ---- convenience wrapper ----------------------------------------------------------------

def make_params(stencil=D3Q19, collision=TRT, storage=FP32, pattern=TWO_GRID, omega=1.0, magic_lambda=3.0 / 16.0,
                force=(0.0, 0.0, 0.0), rho0=1.0, periodic=(1, 1, 1), diag_interval=0, mrt_rates=None,
                cumulant_rates=None) -> lbm_params:
    """lbm_params; ``mrt_rates`` (MRT only): rates of the bulk, fourth-, fifth- and sixth-order
    groups, default the TRT rates of their parity (omega, omega, omega-, omega);
    ``cumulant_rates`` (cumulant only): the nine rates after shear (bulk, third-order sums,
    differences, xyz, fourth-order differences, sum, mixed, fifth, sixth), default all 1."""
    p = lbm_params()
    p.stencil, p.collision, p.storage, p.pattern = stencil, collision, storage, pattern
    p.omega, p.magic_lambda, p.rho0 = float(omega), float(magic_lambda), float(rho0)
    for a in range(3):
        p.force[a] = float(force[a])
        p.periodic[a] = int(bool(periodic[a]))
    p.diag_interval = int(diag_interval)
    if mrt_rates is None:
        wm = 1.0 / (magic_lambda / (1.0 / omega - 0.5) + 0.5) if omega > 0 else 2.0
        mrt_rates = (omega, omega, wm, omega)
    for g in range(4):
        p.mrt_rates[g] = float(mrt_rates[g])
    for g, v in enumerate((1.0,) * 9 if cumulant_rates is None else cumulant_rates):
        p.cumulant_rates[g] = float(v)
    return p


class Simulation:
    """A context plus NumPy marshalling.  Per-block host arrays are [z, y, x] (scalars),
    [3, z, y, x] (velocity) and [q, z, y, x] (PDFs)."""

    def __init__(self, params: lbm_params, blocks, stream=None, device_buffer=None, owner=None, nranks=1, rank=0):
        """owner (optional): owner rank of every block -- the context of rank `rank` of a
        partitioned run (lbm_create_partition) holds only that rank's blocks."""
        self.params = params
        self.q = params.stencil
        self.blocks = [(tuple(int(v) for v in o), tuple(int(v) for v in s)) for o, s in blocks]
        self.owner = None if owner is None else np.asarray(owner, dtype=np.int32)
        self.rank, self.nranks = int(rank), int(nranks)
        if self.owner is None:
            self.ctx = lbm_create_blocks(params, self.blocks, stream)
        else:
            self.ctx = lbm_create_partition(params, self.blocks, self.owner, nranks, rank, stream)
        self._buffer = device_buffer
        if device_buffer is not None:
            lbm_bind_device_memory(self.ctx, device_buffer.data_ptr(), device_buffer.numel() * device_buffer.element_size())

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, b):
        nx, ny, nz = self.blocks[b][1]
        return nz, ny, nx

    def set_face(self, axis, side, kind, u_wall=(0.0, 0.0, 0.0), rho_wall=1.0):
        lbm_set_face(self.ctx, axis, side, kind, u_wall, rho_wall)

    def set_boundary(self, b, flags, u_wall=(0.0, 0.0, 0.0), rho_wall=1.0):
        if flags is not None and np.asarray(flags).shape != self.shape(b):
            raise ValueError("flags of block %d must have shape %s" % (b, self.shape(b)))
        lbm_set_boundary(self.ctx, b, flags, u_wall, rho_wall)

    def init(self, b, rho, u):
        nz, ny, nx = self.shape(b)
        lbm_init_macroscopic(self.ctx, b, np.broadcast_to(rho, (nz, ny, nx)),
                             np.broadcast_to(u, (3, nz, ny, nx)))

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def macroscopic(self, b):
        nz, ny, nx = self.shape(b)
        rho = np.zeros((nz, ny, nx))
        u = np.zeros((3, nz, ny, nx))
        lbm_get_macroscopic(self.ctx, b, rho, u)
        return rho, u

    def pdfs(self, b):
        nz, ny, nx = self.shape(b)
        f = np.zeros((self.q, nz, ny, nx))
        lbm_get_pdfs(self.ctx, b, f)
        return f

    def set_pdfs(self, b, f):
        lbm_set_pdfs(self.ctx, b, f)

    def reduce(self):
        return lbm_reduce(self.ctx)

    def step_diagnostics(self):
        return lbm_step_diagnostics(self.ctx)

    def info(self):
        return lbm_get_info(self.ctx)

    def set_tile(self, tx, ty, tz):
        lbm_set_tile(self.ctx, tx, ty, tz)

    def launches(self):
        return lbm_kernel_launches(self.ctx)

    def reduce_blocks(self):
        return lbm_reduce_blocks(self.ctx, len(self.blocks))

    def pdfs_region(self, b, origin, size):
        return lbm_get_pdfs_region(self.ctx, b, origin, size, self.q)

    def coarse_moments(self, b, ratio):
        return lbm_coarse_moments(self.ctx, b, ratio, self.blocks[b][1])

    def set_closure(self, kind, cs=0.0, mlp_params=None):
        lbm_set_closure(self.ctx, kind, cs, mlp_params)
