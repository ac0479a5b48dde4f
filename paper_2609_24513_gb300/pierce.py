"""ctypes binding of libpierce.so (include/pierce.h).

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  The functions keep the C names.  Host arrays are numpy arrays;
device arrays may be torch CUDA tensors (their data pointers are passed).
Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_lib = None

PJ_OK = 0
PJ_PENDING = 9
PJ_LEAF_FILTERED, PJ_LEAF_EXACT, PJ_LEAF_STATIC = 0, 1, 2
PJ_LAUNCH_PERSISTENT, PJ_LAUNCH_PER_PAIR = 0, 1
PJ_FRONT_NONE, PJ_FRONT_STREAM = -1, -2   # pj_join_opts.wave_levels
# pj_join_opts.predicate (the paper's join predicates, Sec. 3.2-3.4)
PJ_PRED_INTERSECTS, PJ_PRED_OVERLAP, PJ_PRED_CONTAINS, PJ_PRED_WITHIN, PJ_PRED_ANY_VERTEX = range(5)
PREDICATES = {"intersects": 0, "overlap": 1, "contains": 2, "within": 3, "any_vertex": 4}

_STATUS = {1: "PJ_ERR_INVALID_ARG", 2: "PJ_ERR_NOT_QUANTIZED", 3: "PJ_ERR_NOT_MANIFOLD",
           4: "PJ_ERR_NO_MEMORY", 5: "PJ_ERR_BUSY", 6: "PJ_ERR_TIMEOUT", 7: "PJ_ERR_CUDA",
           8: "PJ_ERR_INTERNAL", 9: "PJ_PENDING"}


class PierceError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS.get(code, str(code)), msg))
        self.code = code


class pj_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("budget_bytes", ctypes.c_int64), ("wait_limit_us", ctypes.c_int64),
                ("serve_streams", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class pj_bvh_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("leaf_size", ctypes.c_int32)]


class pj_join_opts(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("warps_per_pair", ctypes.c_int32), ("leaf_mode", ctypes.c_int32),
                ("launch_mode", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("out_host", ctypes.c_int32), ("keep_flags", ctypes.c_int32),
                ("record_cycles", ctypes.c_int32), ("spill_budget", ctypes.c_int32),
                ("wave_levels", ctypes.c_int32), ("kernel_times", ctypes.c_int32),
                ("wait_polls", ctypes.c_int32), ("predicate", ctypes.c_int32)]


class pj_pairs(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("pairs", ctypes.POINTER(ctypes.c_int32)),
                ("on_device", ctypes.c_int32), ("pairs_malloc", ctypes.c_int32),
                ("n_candidates", ctypes.c_int64), ("flags", ctypes.c_void_p),
                ("device_ms", ctypes.c_float), ("mbb_ms", ctypes.c_float),
                ("refine_ms", ctypes.c_float), ("compact_ms", ctypes.c_float),
                ("parity_ms", ctypes.c_float), ("front_ms", ctypes.c_float),
                ("tasks_ms", ctypes.c_float), ("expand_ms", ctypes.c_float),
                ("leaf_ms", ctypes.c_float), ("reserved3", ctypes.c_float),
                ("cycles", ctypes.c_void_p), ("impl", ctypes.c_void_p)]


class pj_counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "pairs_refined", "node_pairs", "box_tests", "leaf_pairs", "edge_slab_tests",
        "segtri_tests", "exact_fallbacks", "parity_rays", "parity_nodes",
        "parity_tri_tests", "bytes_fetched", "pairs_hit", "kernel_launches",
        "tasks_spilled", "tasks_resumed", "bytes_tasks", "bytes_parity", "bytes_expand",
        "bytes_leaf", "parity_handed_over")]


class pj_dataset_info(ctypes.Structure):
    _fields_ = [("n_meshes", ctypes.c_int64), ("n_verts", ctypes.c_int64),
                ("n_tris", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("bvh_nodes", ctypes.c_int64), ("bvh_width", ctypes.c_int32),
                ("bvh_leaf_size", ctypes.c_int32), ("bvh_max_depth", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class pj_tune_space(ctypes.Structure):
    _fields_ = [("widths", ctypes.c_int32 * 3), ("n_widths", ctypes.c_int32),
                ("leaf_sizes", ctypes.c_int32 * 4), ("n_leaf_sizes", ctypes.c_int32),
                ("warps", ctypes.c_int32 * 3), ("n_warps", ctypes.c_int32),
                ("wave_levels", ctypes.c_int32 * 4), ("n_wave_levels", ctypes.c_int32),
                ("sample_permille", ctypes.c_int32), ("repeats", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class pj_tune_entry(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("warps_per_pair", ctypes.c_int32), ("wave_levels", ctypes.c_int32),
                ("ms", ctypes.c_float), ("reserved", ctypes.c_float)]


class pj_query(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("self_join", ctypes.c_int32),
                ("window_lo", ctypes.c_int32 * 3), ("window_hi", ctypes.c_int32 * 3),
                ("reserved", ctypes.c_int32)]


class pj_query_stats(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("n_a", ctypes.c_int64), ("n_b", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("batch_id", ctypes.c_int32),
                ("batch_queries", ctypes.c_int32)]


class pj_estimate(ctypes.Structure):
    _fields_ = [("e_final", ctypes.c_double), ("slots", ctypes.c_double),
                ("cells_occupied", ctypes.c_int64), ("grid", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class pj_dsjoin_opts(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("predicate", ctypes.c_int32), ("materialize", ctypes.c_int32),
                ("fixed_slots", ctypes.c_int64), ("grid", ctypes.c_int32),
                ("out_host", ctypes.c_int32)]


class pj_dsjoin_stats(ctypes.Structure):
    _fields_ = [("edges", ctypes.c_int64), ("node_visits", ctypes.c_int64),
                ("tri_tests", ctypes.c_int64), ("hits", ctypes.c_int64),
                ("parity_rays", ctypes.c_int64), ("recheck_pairs", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("relaunches", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("estimate", ctypes.c_double),
                ("ms_total", ctypes.c_float), ("ms_estimate", ctypes.c_float),
                ("ms_trace", ctypes.c_float), ("ms_materialize", ctypes.c_float)]


class pj_host_meshes(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("tris", ctypes.c_void_p),
                ("mesh_vert_off", ctypes.c_void_p), ("mesh_tri_off", ctypes.c_void_p),
                ("n_meshes", ctypes.c_int64)]


class pj_tiled_opts(ctypes.Structure):
    _fields_ = [("device_budget", ctypes.c_int64), ("grid", ctypes.c_int32),
                ("width", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("out_host", ctypes.c_int32), ("join", pj_join_opts)]


class pj_tiled_stats(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("cells_joined", ctypes.c_int64), ("mesh_copies", ctypes.c_int64),
                ("max_cell_bytes", ctypes.c_int64), ("pairs_in_cells", ctypes.c_int64),
                ("ms_total", ctypes.c_float), ("ms_gather", ctypes.c_float),
                ("ms_device", ctypes.c_float), ("reserved2", ctypes.c_float)]


# pj_dsjoin_opts.materialize (the paper's strategies, Sec. 3.5)
PJ_MAT_ESTIMATED, PJ_MAT_TWO_PASS, PJ_MAT_FIXED = range(3)
MATERIALIZE = {"estimated": 0, "two_pass": 1, "fixed": 2}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32

# name -> (restype, argtypes)
SIGNATURES = {
    "pj_join_tiled": (_i32, [_vp, ctypes.POINTER(pj_host_meshes), ctypes.POINTER(pj_host_meshes),
                             _i32, ctypes.POINTER(pj_tiled_opts), ctypes.POINTER(pj_pairs),
                             ctypes.POINTER(pj_tiled_stats)]),
    "pj_dataset_join": (_i32, [_vp, _i32, _i32, _i32, ctypes.POINTER(pj_dsjoin_opts),
                               ctypes.POINTER(pj_pairs), ctypes.POINTER(pj_dsjoin_stats)]),
    "pj_estimate_join": (_i32, [_vp, _i32, _i32, _i32, _vp, ctypes.POINTER(pj_estimate)]),
    "pj_create": (_i32, [ctypes.POINTER(pj_config), ctypes.POINTER(_vp)]),
    "pj_destroy": (_i32, [_vp]),
    "pj_last_error": (ctypes.c_char_p, [_vp]),
    "pj_load_meshes": (_i32, [_vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _i32,
                              ctypes.POINTER(_i32)]),
    "pj_free_dataset": (_i32, [_vp, _i32]),
    "pj_build_bvh": (_i32, [_vp, _i32, ctypes.POINTER(pj_bvh_params)]),
    "pj_dataset_info_get": (_i32, [_vp, _i32, ctypes.POINTER(pj_dataset_info)]),
    "pj_join_intersects": (_i32, [_vp, _i32, _i32, _vp, _i64, _i32, _vp,
                                  ctypes.POINTER(pj_pairs)]),
    "pj_join_intersects_ex": (_i32, [_vp, _i32, _i32, _vp, _vp, _i64, _i32, _i32,
                                     ctypes.POINTER(pj_join_opts), _vp,
                                     ctypes.POINTER(pj_pairs)]),
    "pj_free_pairs": (_i32, [_vp, ctypes.POINTER(pj_pairs)]),
    "pj_join_intersects_noalloc": (_i32, [_vp, _i32, _i32, _vp, _i64, _vp, _vp, _vp, _vp]),
    "pj_autotune": (_i32, [_vp, _i32, _i32, _vp, _i64, _i32, ctypes.POINTER(pj_tune_space),
                           ctypes.POINTER(pj_join_opts), ctypes.POINTER(pj_tune_entry), _i32,
                           ctypes.POINTER(_i32)]),
    "pj_submit": (_i32, [_vp, ctypes.POINTER(pj_query), ctypes.POINTER(_i64)]),
    "pj_poll": (_i32, [_vp, _i64, _i32, ctypes.POINTER(pj_pairs),
                       ctypes.POINTER(pj_query_stats)]),
    "pj_get_counters": (_i32, [_vp, ctypes.POINTER(pj_counters)]),
    "pj_reset_counters": (_i32, [_vp]),
    "pj_segtri_batch": (_i32, [_vp, _vp, _vp, _i64, _i32, _vp, ctypes.POINTER(_i64), _vp]),
    "pj_export_bvh": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(_i64)]),
    "pj_export_mesh_data": (_i32, [_vp, _i32, _vp, _vp, _vp]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpierce.so (raise if it is missing; build it first on request)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libpierce.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def _is_device(x) -> bool:
    return x is not None and not isinstance(x, np.ndarray) and getattr(x, "is_cuda", False)


_CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _stream_ptr(stream):
    """cudaStream_t for the C ABI.  None -> NULL (the context's own stream).
    A torch stream whose handle is 0 is the legacy default stream, which the
    ABI would read as NULL, so it is passed as cudaStreamLegacy."""
    if stream is None:
        return None
    h = stream if isinstance(stream, int) else int(stream.cuda_stream)
    return h if h != 0 else _CUDA_STREAM_LEGACY


def _check(ctx, rc):
    if rc != PJ_OK:
        msg = load().pj_last_error(ctx).decode() if ctx else ""
        raise PierceError(rc, msg)


# ---------------------------------------------------------------------------
# Functions with the C names
# ---------------------------------------------------------------------------

def pj_create(device: int = 0, budget_bytes: int = 0, wait_limit_us: int = 0,
              serve_streams: int = 0):
    cfg = pj_config(device, 0, budget_bytes, wait_limit_us, serve_streams, 0)
    h = _vp()
    rc = load().pj_create(ctypes.byref(cfg), ctypes.byref(h))
    if rc != PJ_OK:
        raise PierceError(rc, "pj_create failed")
    return h.value


def pj_destroy(ctx):
    _check(None, load().pj_destroy(ctx))


def pj_last_error(ctx) -> str:
    return load().pj_last_error(ctx).decode()


def pj_load_meshes(ctx, xyz, tris, mesh_vert_off, mesh_tri_off) -> int:
    """xyz (V x 3 float32) and tris (F x 3 int32): numpy arrays (host) or torch
    CUDA tensors (device).  Offsets: numpy int64 (host)."""
    dev = _is_device(xyz)
    if dev != _is_device(tris):
        raise ValueError("xyz and tris must both be host or both be device arrays")
    if not dev:
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        tris = np.ascontiguousarray(tris, dtype=np.int32)
    else:
        xyz, tris = xyz.contiguous(), tris.contiguous()
    voff = np.ascontiguousarray(mesh_vert_off, dtype=np.int64)
    toff = np.ascontiguousarray(mesh_tri_off, dtype=np.int64)
    nv = int(xyz.shape[0]) if xyz.ndim == 2 else int(xyz.numel() // 3 if dev else xyz.size // 3)
    nt = int(tris.shape[0]) if tris.ndim == 2 else int(tris.numel() // 3 if dev else tris.size // 3)
    out = _i32()
    rc = load().pj_load_meshes(ctx, _ptr(xyz), nv, _ptr(tris), nt, _ptr(voff), _ptr(toff),
                               len(voff) - 1, 1 if dev else 0, ctypes.byref(out))
    _check(ctx, rc)
    return out.value


def pj_free_dataset(ctx, ds: int):
    _check(ctx, load().pj_free_dataset(ctx, ds))


def pj_build_bvh(ctx, ds: int, width: int = 4, leaf_size: int = 4):
    p = pj_bvh_params(width, leaf_size)
    _check(ctx, load().pj_build_bvh(ctx, ds, ctypes.byref(p)))


def pj_dataset_info_get(ctx, ds: int) -> dict:
    info = pj_dataset_info()
    _check(ctx, load().pj_dataset_info_get(ctx, ds, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in pj_dataset_info._fields_ if f != "reserved"}


def pj_join_intersects_ex(ctx, a: int, b: int, cand=None, cand_offsets=None, self_join=False,
                          width=0, leaf_size=0, warps_per_pair=0, leaf_mode=PJ_LEAF_FILTERED,
                          launch_mode=PJ_LAUNCH_PERSISTENT, use_graph=False, out_host=True,
                          keep_flags=False, record_cycles=False, spill_budget=0, wave_levels=0,
                          kernel_times=False, wait_polls=0, predicate=PJ_PRED_INTERSECTS,
                          stream=None):
    """Run the join.  Returns the filled pj_pairs (free it with pj_free_pairs).

    cand / cand_offsets: None (device bounding-box filter join), numpy int32
    arrays (host) or torch CUDA int32 tensors (device)."""
    dev = _is_device(cand)
    n = 0
    if cand is not None:
        if not dev:
            cand = np.ascontiguousarray(cand, dtype=np.int32).reshape(-1, 2)
            if cand_offsets is not None:
                cand_offsets = np.ascontiguousarray(cand_offsets, dtype=np.int32).reshape(-1, 3)
        n = int(cand.shape[0])
    opts = pj_join_opts(width, leaf_size, warps_per_pair, leaf_mode, launch_mode,
                        int(use_graph), int(out_host), int(keep_flags), int(record_cycles),
                        int(spill_budget), int(wave_levels), int(kernel_times), int(wait_polls),
                        int(PREDICATES.get(predicate, predicate)))
    res = pj_pairs()
    rc = load().pj_join_intersects_ex(ctx, a, b, _ptr(cand), _ptr(cand_offsets), n,
                                      1 if dev else 0, int(self_join), ctypes.byref(opts),
                                      _stream_ptr(stream), ctypes.byref(res))
    _check(ctx, rc)
    return res


def _host_meshes(ds):
    xyz = np.ascontiguousarray(ds.xyz, dtype=np.float32)
    tris = np.ascontiguousarray(ds.tris, dtype=np.int32)
    voff = np.ascontiguousarray(ds.voff, dtype=np.int64)
    toff = np.ascontiguousarray(ds.toff, dtype=np.int64)
    keep = (xyz, tris, voff, toff)
    return pj_host_meshes(xyz.ctypes.data, tris.ctypes.data, voff.ctypes.data,
                          toff.ctypes.data, len(voff) - 1), keep


def pj_join_tiled(ctx, dsA, dsB=None, self_join=False, device_budget=0, grid=0, width=0,
                  leaf_size=0, **join_kw):
    """Out-of-core join of two host datasets (objects with xyz/tris/voff/toff)
    by grid tiling.  join_kw: pj_join_opts fields for each cell's join
    (predicate, leaf_mode, ...).  Returns (pairs K x 2 int32 sorted, stats)."""
    ha, keep_a = _host_meshes(dsA)
    hb, keep_b = _host_meshes(dsB if dsB is not None else dsA)
    jo = pj_join_opts()
    for k, v in join_kw.items():
        setattr(jo, k, int(PREDICATES.get(v, v)) if k == "predicate" else int(v))
    opts = pj_tiled_opts(int(device_budget), int(grid), int(width), int(leaf_size), 1, jo)
    res, st = pj_pairs(), pj_tiled_stats()
    _check(ctx, load().pj_join_tiled(ctx, ctypes.byref(ha), ctypes.byref(hb), int(bool(self_join)),
                                     ctypes.byref(opts), ctypes.byref(res), ctypes.byref(st)))
    try:
        pairs = pairs_to_numpy(res)
    finally:
        pj_free_pairs(ctx, res)
    del keep_a, keep_b
    return pairs, {k: getattr(st, k) for k, _ in pj_tiled_stats._fields_}


def pj_dataset_join(ctx, a: int, b: int, self_join=False, width=0, leaf_size=0,
                    predicate="intersects", materialize="estimated", fixed_slots=0, grid=0):
    """The dataset-level join (one BVH per dataset, every edge traced, pairs
    deduplicated by the chosen materialisation).  Returns (pairs K x 2 int32
    sorted, stats dict)."""
    opts = pj_dsjoin_opts(int(width), int(leaf_size), int(PREDICATES.get(predicate, predicate)),
                          int(MATERIALIZE.get(materialize, materialize)), int(fixed_slots),
                          int(grid), 1)
    res, st = pj_pairs(), pj_dsjoin_stats()
    _check(ctx, load().pj_dataset_join(ctx, a, b, int(bool(self_join)), ctypes.byref(opts),
                                       ctypes.byref(res), ctypes.byref(st)))
    try:
        pairs = pairs_to_numpy(res)
    finally:
        pj_free_pairs(ctx, res)
    return pairs, {k: getattr(st, k) for k, _ in pj_dsjoin_stats._fields_}


def pj_estimate_join(ctx, a: int, b: int, grid: int = 16, cells: bool = False):
    """The paper's selectivity estimate (Sec. 3.5) of the join of datasets a
    and b on a grid x grid x grid grid.  Returns a dict (e_final, slots,
    cells_occupied, grid, ms), with the per-cell E_i (grid^3 float64, index
    (x G + y) G + z) under "cells" when asked for."""
    out = pj_estimate()
    g = grid if grid > 0 else 16
    buf = np.zeros(g ** 3, np.float64) if cells else None
    _check(ctx, load().pj_estimate_join(ctx, a, b, int(grid), _ptr(buf), ctypes.byref(out)))
    r = {k: getattr(out, k) for k, _ in pj_estimate._fields_}
    if cells:
        r["cells"] = buf
    return r


def pj_join_intersects(ctx, a: int, b: int, cand=None, self_join=False, stream=None):
    """The plain entry point (device-resident result).  Returns pj_pairs."""
    res = pj_pairs()
    n = 0
    if cand is not None:
        cand = np.ascontiguousarray(cand, dtype=np.int32).reshape(-1, 2)
        n = cand.shape[0]
    rc = load().pj_join_intersects(ctx, a, b, _ptr(cand), n, int(self_join),
                                   _stream_ptr(stream), ctypes.byref(res))
    _check(ctx, rc)
    return res


def pj_join_intersects_noalloc(ctx, a: int, b: int, d_cand, d_flags, d_pairs, d_count,
                               stream=None):
    """Allocation-free join on caller-owned torch CUDA tensors: d_cand (n x 2
    int32), d_flags (n uint8), d_pairs (n x 2 int32), d_count (1 int64).
    Enqueues the work and returns; synchronise the stream before reading."""
    n = int(d_cand.shape[0]) if d_cand is not None else 0
    _check(ctx, load().pj_join_intersects_noalloc(ctx, a, b, _ptr(d_cand), n, _ptr(d_flags),
                                                  _ptr(d_pairs), _ptr(d_count),
                                                  _stream_ptr(stream)))


def pj_free_pairs(ctx, res: pj_pairs):
    _check(ctx, load().pj_free_pairs(ctx, ctypes.byref(res)))


def pj_autotune(ctx, a: int, b: int, cand=None, self_join=False, widths=(2, 4, 8),
                leaf_sizes=(1, 2, 4, 8), warps=(1, 2, 4), wave_levels=(0,), sample_permille=0,
                repeats=0, seed=0):
    """Measure every configuration of the space on a calibration sample.
    Returns (best pj_join_opts as a dict, table of measured entries)."""
    sp = pj_tune_space()
    for name, vals, cap in (("widths", widths, 3), ("leaf_sizes", leaf_sizes, 4),
                            ("warps", warps, 3), ("wave_levels", wave_levels, 4)):
        vals = list(vals)[:cap]
        arr = getattr(sp, name)
        for k, v in enumerate(vals):
            arr[k] = int(v)
        setattr(sp, "n_" + name, len(vals))
    sp.sample_permille, sp.repeats, sp.seed = int(sample_permille), int(repeats), int(seed)
    n = 0
    if cand is not None:
        cand = np.ascontiguousarray(cand, dtype=np.int32).reshape(-1, 2)
        n = cand.shape[0]
    best = pj_join_opts()
    cap = 3 * 4 * 3 * 4
    table = (pj_tune_entry * cap)()
    tn = _i32()
    _check(ctx, load().pj_autotune(ctx, a, b, _ptr(cand), n, int(self_join), ctypes.byref(sp),
                                   ctypes.byref(best), table, cap, ctypes.byref(tn)))
    best_d = {f: getattr(best, f) for f, _ in pj_join_opts._fields_ if f != "reserved"}
    rows = [{f: getattr(table[k], f) for f, _ in pj_tune_entry._fields_ if f != "reserved"}
            for k in range(tn.value)]
    return best_d, rows


def pj_submit(ctx, a: int, b: int, window_lo, window_hi, self_join=False) -> int:
    """Queue a window join query; returns its ticket."""
    q = pj_query(a, b, int(self_join), (ctypes.c_int32 * 3)(*[int(v) for v in window_lo]),
                 (ctypes.c_int32 * 3)(*[int(v) for v in window_hi]), 0)
    t = _i64()
    _check(ctx, load().pj_submit(ctx, ctypes.byref(q), ctypes.byref(t)))
    return t.value


def pj_poll(ctx, ticket: int, wait=True):
    """None while the query is pending (wait=False); else (pairs K x 2 numpy,
    stats dict)."""
    res = pj_pairs()
    st = pj_query_stats()
    rc = load().pj_poll(ctx, int(ticket), int(bool(wait)), ctypes.byref(res), ctypes.byref(st))
    if rc == PJ_PENDING:
        return None
    _check(ctx, rc)
    try:
        pairs = pairs_to_numpy(res)
    finally:
        pj_free_pairs(ctx, res)
    return pairs, {f: getattr(st, f) for f, _ in pj_query_stats._fields_}


def pj_get_counters(ctx) -> dict:
    c = pj_counters()
    _check(ctx, load().pj_get_counters(ctx, ctypes.byref(c)))
    return {f: int(getattr(c, f)) for f, _ in pj_counters._fields_ if f != "reserved"}


def pj_reset_counters(ctx):
    _check(ctx, load().pj_reset_counters(ctx))


def pj_segtri_batch(ctx, pq, abc, res, mode=PJ_LEAF_FILTERED, stream=None) -> int:
    """pq (n x 6), abc (n x 9) float32 and res (n uint8): torch CUDA tensors.
    Returns the number of filter fallbacks."""
    nfb = _i64()
    _check(ctx, load().pj_segtri_batch(ctx, _ptr(pq), _ptr(abc), int(res.numel()), mode,
                                       _ptr(res), ctypes.byref(nfb), _stream_ptr(stream)))
    return nfb.value


def pj_export_bvh(ctx, ds: int, width: int, leaf_size: int, n_tris: int, n_meshes: int):
    """(nodes [n, W + 1, 8] int32 words, roots [M], tri_order [F]) as numpy arrays."""
    n = _i64()
    lib = load()
    _check(ctx, lib.pj_export_bvh(ctx, ds, width, leaf_size, None, None, None, ctypes.byref(n)))
    nodes = np.zeros((n.value, width + 1, 8), dtype=np.int32)
    roots = np.zeros(n_meshes, dtype=np.int32)
    order = np.zeros(n_tris, dtype=np.int32)
    _check(ctx, lib.pj_export_bvh(ctx, ds, width, leaf_size, _ptr(nodes), _ptr(roots),
                                  _ptr(order), ctypes.byref(n)))
    return nodes, roots, order


def pj_export_mesh_data(ctx, ds: int, n_meshes: int, n_tris: int):
    aabb = np.zeros((n_meshes, 6), dtype=np.float32)
    lex = np.zeros(n_meshes, dtype=np.int32)
    own = np.zeros(n_tris, dtype=np.uint8)
    _check(ctx, load().pj_export_mesh_data(ctx, ds, _ptr(aabb), _ptr(lex), _ptr(own)))
    return aabb, lex, own


# ---------------------------------------------------------------------------
# Convenience wrappers
# ---------------------------------------------------------------------------

class _DeviceView:
    """A raw device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def device_to_numpy(ptr, n: int, dtype) -> np.ndarray:
    """Copy n elements of a library-owned device buffer to a numpy array."""
    import torch
    dt = np.dtype(dtype)
    if n == 0 or not ptr:
        return np.zeros(0, dtype=dt)
    code = {np.dtype(np.uint8): "|u1", np.dtype(np.int32): "<i4", np.dtype(np.uint32): "<i4",
            np.dtype(np.int64): "<i8"}[dt]
    t = torch.as_tensor(_DeviceView(ptr, n, code), device="cuda")
    return t.cpu().numpy().view(dt)


def pairs_to_numpy(res: pj_pairs) -> np.ndarray:
    """Copy a host-resident result (out_host=True) into a numpy array."""
    if res.on_device:
        raise ValueError("result is on the device; join with out_host=True")
    k = int(res.count)
    if k == 0:
        return np.zeros((0, 2), dtype=np.int32)
    return np.ctypeslib.as_array(res.pairs, shape=(k, 2)).copy()


class Context:
    """Owns a pj_ctx; datasets are loaded from objects with xyz/tris/voff/toff."""

    def __init__(self, device: int = 0, **cfg):
        self.h = pj_create(device, **cfg)

    def close(self):
        if self.h:
            pj_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load(self, ds, device_tensors: bool = False) -> int:
        if device_tensors:
            import torch
            xyz = torch.from_numpy(np.ascontiguousarray(ds.xyz, dtype=np.float32)).cuda()
            tris = torch.from_numpy(np.ascontiguousarray(ds.tris, dtype=np.int32)).cuda()
            return pj_load_meshes(self.h, xyz, tris, ds.voff, ds.toff)
        return pj_load_meshes(self.h, ds.xyz, ds.tris, ds.voff, ds.toff)

    def build(self, ds: int, width: int = 4, leaf_size: int = 4):
        pj_build_bvh(self.h, ds, width, leaf_size)

    def join(self, a: int, b: int, cand=None, **kw):
        """Sorted intersecting pairs as numpy (K x 2), plus the raw result info."""
        kw.setdefault("out_host", True)
        res = pj_join_intersects_ex(self.h, a, b, cand=cand, **kw)
        try:
            pairs = pairs_to_numpy(res)
            info = dict(count=int(res.count), n_candidates=int(res.n_candidates),
                        device_ms=res.device_ms, mbb_ms=res.mbb_ms, refine_ms=res.refine_ms,
                        compact_ms=res.compact_ms)
        finally:
            pj_free_pairs(self.h, res)
        return pairs, info

    def submit(self, a: int, b: int, window_lo, window_hi, self_join=False) -> int:
        return pj_submit(self.h, a, b, window_lo, window_hi, self_join)

    def poll(self, ticket: int, wait=True):
        return pj_poll(self.h, ticket, wait)

    def counters(self) -> dict:
        return pj_get_counters(self.h)

    def reset_counters(self):
        pj_reset_counters(self.h)
