"""Exact CPU oracle for the mesh intersection join -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it; see ``oracle.c`` for the definitions it implements
(paper Sec. 3.1-3.4: strict edge/face crossing in both directions, +z parity
for containment, intersection = crossing OR containment).

A dataset is any object with the attributes ``xyz`` (V x 3 float32, integer
valued in [0, 2^18)), ``tris`` (F x 3 int32, mesh-local vertex ids), ``voff``
and ``toff`` (M + 1 int64 offsets).

``oracle.estimate`` (plain numpy) states the paper's selectivity estimate
(Sec. 3.5); ``join(..., predicate=)`` also evaluates the overlap, containment
and within joins (Sec. 3.2, 3.3).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(hand-built cases, exact rational re-derivations, closed forms, invariants,
winding numbers and a convex separating-axis cross-check).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f32p = ctypes.POINTER(ctypes.c_float)


class _Dataset(ctypes.Structure):
    _fields_ = [("xyz", _f32p), ("tris", _i32p), ("voff", _i64p),
                ("toff", _i64p), ("nmesh", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    D = ctypes.POINTER(_Dataset)
    lib.orc_orient3d.restype = ctypes.c_int64
    lib.orc_orient3d.argtypes = [_i64p] * 4
    lib.orc_orient2d_xy.restype = ctypes.c_int64
    lib.orc_orient2d_xy.argtypes = [_i64p] * 3
    lib.orc_segtri_strict.restype = ctypes.c_int32
    lib.orc_segtri_strict.argtypes = [_i64p] * 5
    lib.orc_point_in_closed_triangle.restype = ctypes.c_int32
    lib.orc_point_in_closed_triangle.argtypes = [_i64p] * 4
    lib.orc_ray_up_hits.restype = ctypes.c_int32
    lib.orc_ray_up_hits.argtypes = [_i64p] * 4
    lib.orc_intersects_pair.restype = ctypes.c_int32
    lib.orc_intersects_pair.argtypes = [D, ctypes.c_int64, D, ctypes.c_int64,
                                        _i32p, ctypes.c_int32, _i64p]
    lib.orc_cross_pair.restype = ctypes.c_int32
    lib.orc_cross_pair.argtypes = [D, ctypes.c_int64, D, ctypes.c_int64, ctypes.c_int32]
    lib.orc_inside_pair.restype = ctypes.c_int32
    lib.orc_inside_pair.argtypes = [D, ctypes.c_int64, D, ctypes.c_int64]
    lib.orc_rep_vertex.restype = ctypes.c_int64
    lib.orc_rep_vertex.argtypes = [D, ctypes.c_int64, D, ctypes.c_int64]
    lib.orc_point_query.restype = ctypes.c_int32
    lib.orc_point_query.argtypes = [_i64p, D, ctypes.c_int64]
    lib.orc_join.restype = ctypes.c_int64
    lib.orc_join.argtypes = [D, D, _i32p, _i32p, ctypes.c_int64, ctypes.c_int32,
                             _u8p, _i64p]
    lib.orc_join_pred.restype = ctypes.c_int64
    lib.orc_join_pred.argtypes = [D, D, _i32p, _i32p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_int32, _u8p, _i64p]
    lib.orc_mbb_candidates.restype = ctypes.c_int64
    lib.orc_mbb_candidates.argtypes = [D, D, ctypes.c_int32, _i32p, ctypes.c_int64]
    lib.orc_is_closed_manifold.restype = ctypes.c_int32
    lib.orc_is_closed_manifold.argtypes = [D, ctypes.c_int64]
    _lib = lib
    return lib


class OracleError(RuntimeError):
    pass


def _pt(x) -> ctypes.Array:
    a = (ctypes.c_int64 * 3)(*[int(v) for v in x])
    return a


def _ptr(arr: np.ndarray, ct):
    return arr.ctypes.data_as(ctypes.POINTER(ct))


class _DS:
    """Keeps the numpy buffers alive for the duration of a call."""

    def __init__(self, ds):
        self.xyz = np.ascontiguousarray(ds.xyz, dtype=np.float32).reshape(-1, 3)
        self.tris = np.ascontiguousarray(ds.tris, dtype=np.int32).reshape(-1, 3)
        self.voff = np.ascontiguousarray(ds.voff, dtype=np.int64)
        self.toff = np.ascontiguousarray(ds.toff, dtype=np.int64)
        self.c = _Dataset(_ptr(self.xyz, ctypes.c_float), _ptr(self.tris, ctypes.c_int32),
                          _ptr(self.voff, ctypes.c_int64), _ptr(self.toff, ctypes.c_int64),
                          len(self.voff) - 1)

    @property
    def ref(self):
        return ctypes.byref(self.c)


def _check(rc):
    if rc <= -10:
        raise OracleError({-11: "coordinate not an integer in [0, 2^18)",
                           -12: "triangle vertex index out of range",
                           -13: "bad argument", -14: "out of memory"}.get(int(rc), str(rc)))
    return rc


# ---- exact primitives ------------------------------------------------------

def orient3d(a, b, c, d) -> int:
    """det[b-a; c-a; d-a] (exact int64)."""
    return int(_load().orc_orient3d(_pt(a), _pt(b), _pt(c), _pt(d)))


def orient2d_xy(a, b, c) -> int:
    return int(_load().orc_orient2d_xy(_pt(a), _pt(b), _pt(c)))


def segtri_strict(p, q, a, b, c) -> bool:
    """Open segment pq crosses open triangle abc transversally."""
    return bool(_load().orc_segtri_strict(_pt(p), _pt(q), _pt(a), _pt(b), _pt(c)))


def point_in_closed_triangle(v, a, b, c) -> bool:
    return bool(_load().orc_point_in_closed_triangle(_pt(v), _pt(a), _pt(b), _pt(c)))


def ray_up_hits(v, a, b, c) -> bool:
    """Perturbed +z ray from v hits triangle abc (counted for parity)."""
    return bool(_load().orc_ray_up_hits(_pt(v), _pt(a), _pt(b), _pt(c)))


# ---- mesh-level ------------------------------------------------------------

def point_query(v, ds, i: int):
    """(parity of the +z ray from v against mesh i, v on mesh i's surface)."""
    d = _DS(ds)
    r = _check(_load().orc_point_query(_pt(v), d.ref, i))
    return bool(r & 1), bool(r & 2)


def rep_vertex(dsB, j: int, dsA, i: int) -> int:
    """Mesh-local index of B_j's representative vertex w.r.t. A_i, or -1 if
    every vertex of B_j lies on A_i's surface."""
    a, b = _DS(dsA), _DS(dsB)
    return int(_check(_load().orc_rep_vertex(b.ref, j, a.ref, i)))


def intersects(dsA, i: int, dsB, j: int, tier: int = 1, off=None) -> bool:
    a, b = _DS(dsA), _DS(dsB)
    o = None
    if off is not None:
        o = np.ascontiguousarray(off, dtype=np.int32)
        o = _ptr(o, ctypes.c_int32)
    return bool(_check(_load().orc_intersects_pair(a.ref, i, b.ref, j, o, tier, None)))


def cross(dsA, i: int, dsB, j: int, tier: int = 1) -> bool:
    a, b = _DS(dsA), _DS(dsB)
    return bool(_check(_load().orc_cross_pair(a.ref, i, b.ref, j, tier)))


def inside(dsB, j: int, dsA, i: int) -> bool:
    """inside(B_j, A_i): B_j's representative vertex lies inside A_i."""
    a, b = _DS(dsA), _DS(dsB)
    return bool(_check(_load().orc_inside_pair(b.ref, j, a.ref, i)))


# The paper's join predicates (Sec. 3.2-3.4): intersects = overlap OR
# containment either way; overlap = a surface crossing; contains = A_i holds
# B_j with no crossing (Alg. 2); within = the role swap (B_j holds A_i).
# "any_vertex" adds to intersects any vertex of either mesh strictly inside
# the other (a completeness mode for crossings through edges and vertices only).
PREDICATES = {"intersects": 0, "overlap": 1, "contains": 2, "within": 3, "any_vertex": 4}


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # not Linux
        return os.cpu_count() or 1


def join(dsA, dsB, cand: np.ndarray, tier: int = 2, offsets=None, stats: bool = False,
         predicate: str = "intersects", threads: int = 1):
    """Refine candidate pairs (n x 2 int32) under `predicate` (a key of
    PREDICATES).  Returns uint8 flags[n] (and the counters [segment/triangle
    tests, parity rays] if stats).

    threads > 1 (None: every host core) splits the list into contiguous
    shards that that many threads refine at once; each shard is one plain
    single-threaded call of the C code on its own slice of the list and of
    the flags, so the result does not depend on the sharding."""
    pred = PREDICATES[predicate]
    a, b = _DS(dsA), _DS(dsB)
    cand = np.ascontiguousarray(cand, dtype=np.int32).reshape(-1, 2)
    n = cand.shape[0]
    flags = np.zeros(max(n, 1), dtype=np.uint8)
    if offsets is not None:
        offsets = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
        if offsets.shape[0] != n:
            raise OracleError("one offset per candidate is required")
    lib = _load()

    def run(lo: int, hi: int) -> np.ndarray:
        st = np.zeros(2, dtype=np.int64)
        if hi <= lo:
            return st
        cp = _ptr(cand[lo:hi], ctypes.c_int32)
        op = None if offsets is None else _ptr(offsets[lo:hi], ctypes.c_int32)
        fp = _ptr(flags[lo:hi], ctypes.c_uint8)
        sp = _ptr(st, ctypes.c_int64)
        if pred == 0:
            _check(lib.orc_join(a.ref, b.ref, cp, op, hi - lo, tier, fp, sp))
        else:
            _check(lib.orc_join_pred(a.ref, b.ref, cp, op, hi - lo, tier, pred, fp, sp))
        return st

    if threads is None:
        threads = host_cores()
    threads = max(1, min(int(threads), n))
    if threads == 1:
        st = run(0, n)
    else:
        # many more shards than threads: pair costs differ by orders of
        # magnitude, so small shards keep every thread busy to the end
        import concurrent.futures as cf
        bounds = np.linspace(0, n, min(n, 32 * threads) + 1).astype(np.int64)
        with cf.ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(run, bounds[:-1].tolist(), bounds[1:].tolist()))
        st = np.sum(parts, axis=0)
    flags = flags[:n]
    return (flags, st) if stats else flags


def mbb_candidates(dsA, dsB, self_join: bool = False) -> np.ndarray:
    """All (i, j) whose closed mesh bounding boxes meet, sorted; i < j if self_join."""
    a, b = _DS(dsA), _DS(dsB)
    lib = _load()
    n = _check(lib.orc_mbb_candidates(a.ref, b.ref, int(self_join), None, 0))
    out = np.zeros((max(n, 1), 2), dtype=np.int32)
    _check(lib.orc_mbb_candidates(a.ref, b.ref, int(self_join), _ptr(out, ctypes.c_int32), n))
    return out[:n]


def join_all(dsA, dsB, self_join: bool = False, tier: int = 2):
    """Sorted (i, j) pairs of the intersection join over all mesh pairs.

    Pairs whose bounding boxes do not meet are skipped: a crossing point lies
    in both boxes and a containing mesh's box contains the contained one."""
    cand = mbb_candidates(dsA, dsB, self_join)
    flags = join(dsA, dsB, cand, tier=tier)
    return cand[flags.astype(bool)]


def is_closed_manifold(ds, k: int) -> bool:
    d = _DS(ds)
    return bool(_check(_load().orc_is_closed_manifold(d.ref, k)))
