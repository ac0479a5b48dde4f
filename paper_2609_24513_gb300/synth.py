"""Seeded synthetic inputs: closed triangle meshes quantized to the 2^18 grid.

This module only generates inputs.  It holds none of the join's arithmetic
(no orientation predicates, no crossing, parity or bounding-box join), so both
the CUDA path and the CPU oracle can be fed from it.

A dataset is a ``MeshSet``: ``xyz`` (V x 3 float32, integer valued in
[0, 2^18)), ``tris`` (F x 3 int32, mesh-local vertex ids, outward
counter-clockwise), ``voff``/``toff`` (M + 1 int64 offsets).

Workload shapes follow the paper's data families (Sec. 4.2: tessellated
spheres, simulated cell nuclei and blood vessels, cubes):

* ``tiny_spheres``  -- 20 + 20 level-2 icospheres (320 triangles), radius
  U[0.05, 0.15] of the box, random rotation, centres in a sub-cube sized so
  that about half of the 400 bounding-box pairs overlap.
* ``pathology``     -- nuclei (level 4/5 icospheres with a smooth 10 % radial
  noise field, log-normal radius with mean 1/200 box) and vessels (16-sided
  capped tubes swept along cubic B-splines, 10k-50k triangles, radius
  U[1/300, 1/100] box).
* hand-built solids (boxes, tetrahedra, octahedra) for exact test cases.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRID = 1 << 18          # coordinates are integers in [0, GRID)
QMAX = GRID - 1


@dataclasses.dataclass
class MeshSet:
    xyz: np.ndarray
    tris: np.ndarray
    voff: np.ndarray
    toff: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nmesh(self) -> int:
        return len(self.voff) - 1

    def mesh(self, k: int):
        """(vertices V_k x 3 float32, triangles F_k x 3 local int32) of mesh k."""
        v = self.xyz[self.voff[k]:self.voff[k + 1]]
        t = self.tris[self.toff[k]:self.toff[k + 1]]
        return v, t


def concat(meshes, meta=None) -> MeshSet:
    """Build a MeshSet from a list of (vertices, triangles) with local ids."""
    vs = [np.asarray(v, dtype=np.float32).reshape(-1, 3) for v, _ in meshes]
    ts = [np.asarray(t, dtype=np.int32).reshape(-1, 3) for _, t in meshes]
    voff = np.zeros(len(meshes) + 1, dtype=np.int64)
    toff = np.zeros(len(meshes) + 1, dtype=np.int64)
    voff[1:] = np.cumsum([len(v) for v in vs])
    toff[1:] = np.cumsum([len(t) for t in ts])
    xyz = np.concatenate(vs) if vs else np.zeros((0, 3), np.float32)
    tris = np.concatenate(ts) if ts else np.zeros((0, 3), np.int32)
    return MeshSet(np.ascontiguousarray(xyz), np.ascontiguousarray(tris), voff, toff,
                   dict(meta or {}))


def subset(ds: MeshSet, ids) -> MeshSet:
    return concat([ds.mesh(int(k)) for k in ids], ds.meta)


def quantize(x01: np.ndarray) -> np.ndarray:
    """Unit-cube coordinates -> grid integers (round half to even, clamped)."""
    q = np.rint(np.asarray(x01, dtype=np.float64) * QMAX)
    return np.clip(q, 0, QMAX).astype(np.float32)


# ---------------------------------------------------------------------------
# Hand-built solids (integer coordinates, outward counter-clockwise faces)
# ---------------------------------------------------------------------------

_BOX_T = np.array([[0, 2, 1], [0, 3, 2],      # z = lo  (normal -z)
                   [4, 5, 6], [4, 6, 7],      # z = hi  (normal +z)
                   [0, 1, 5], [0, 5, 4],      # y = lo
                   [3, 6, 2], [3, 7, 6],      # y = hi
                   [0, 4, 7], [0, 7, 3],      # x = lo
                   [1, 2, 6], [1, 6, 5]],     # x = hi
                  dtype=np.int32)


def box(lo, hi):
    """Axis-aligned box [lo, hi] as 8 vertices / 12 triangles."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float32)
    return v, _BOX_T.copy()


def tetra(p0, p1, p2, p3):
    """Tetrahedron; faces are oriented so that the fourth point is behind each."""
    v = np.array([p0, p1, p2, p3], dtype=np.float64)
    faces = [[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]
    centre = v.mean(axis=0)
    out = []
    for f in faces:
        a, b, c = v[f]
        n = np.cross(b - a, c - a)
        out.append(f if np.dot(n, a - centre) > 0 else [f[0], f[2], f[1]])
    return v.astype(np.float32), np.array(out, dtype=np.int32)


def octahedron(c, r):
    cx, cy, cz = c
    v = np.array([[cx + r, cy, cz], [cx - r, cy, cz], [cx, cy + r, cz],
                  [cx, cy - r, cz], [cx, cy, cz + r], [cx, cy, cz - r]], dtype=np.float32)
    t = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int32)
    return v, t


def translate(mesh, d):
    v, t = mesh
    return (np.asarray(v, dtype=np.float32) + np.asarray(d, dtype=np.float32), t)


# ---------------------------------------------------------------------------
# Icospheres
# ---------------------------------------------------------------------------

_ICO_CACHE: dict = {}


def icosphere(level: int):
    """Unit icosphere after `level` midpoint subdivisions (float64 vertices).

    Counts: V = 10 * 4^L + 2, F = 20 * 4^L.  Faces are outward CCW."""
    if level in _ICO_CACHE:
        return _ICO_CACHE[level]
    p = (1.0 + 5 ** 0.5) / 2
    v = [[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
         [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
         [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]]
    f = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = [tuple(x) for x in f]
    for _ in range(level):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces, dtype=np.int32)
    # orient outward (the template is star-shaped around the origin)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    _ICO_CACHE[level] = (V, F)
    return V, F


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniform random rotation matrices (from unit quaternions)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _smooth_field(rng, n_terms=8):
    """A smooth function on the unit sphere with values in [-1, 1]: a sum of
    low-frequency 3-D sinusoids normalised by the sum of their amplitudes."""
    dirs = rng.normal(size=(n_terms, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    freq = rng.uniform(1.0, 3.0, size=n_terms)
    phase = rng.uniform(0, 2 * np.pi, size=n_terms)
    amp = rng.uniform(0.5, 1.0, size=n_terms)
    w = dirs * freq[:, None]

    def f(u):
        return (np.sin(u @ w.T + phase) * amp).sum(axis=1) / amp.sum()
    return f


def _placed_sphere(level, centre, radius, R, noise=None):
    V, F = icosphere(level)
    if noise is not None:
        V = V * (1.0 + noise(V))[:, None]
    X = (V @ R.T) * radius + centre
    return quantize(X), F


def tiny_spheres(seed: int, n_a: int = 20, n_b: int = 20, level: int = 2,
                 r_range=(0.05, 0.15), target_overlap: float = 0.5):
    """Two datasets of icospheres; about `target_overlap` of the n_a * n_b
    bounding-box pairs overlap.  Returns (A, B)."""
    rng = np.random.default_rng(seed)
    ra = rng.uniform(*r_range, size=n_a)
    rb = rng.uniform(*r_range, size=n_b)
    ua = rng.uniform(-0.5, 0.5, size=(n_a, 3))
    ub = rng.uniform(-0.5, 0.5, size=(n_b, 3))
    Ra = random_rotations(rng, n_a)
    Rb = random_rotations(rng, n_b)

    # sub-cube side s: bisect on the fraction of sphere pairs whose bounding
    # cubes [c - r, c + r] overlap on every axis (placement parameters only)
    def frac(s):
        d = np.abs((ua[:, None, :] - ub[None, :, :]) * s)
        lim = (ra[:, None] + rb[None, :])[..., None]
        return float(np.all(d <= lim, axis=2).mean())
    lo, hi = 0.05, 0.68
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if frac(mid) > target_overlap:
            lo = mid
        else:
            hi = mid
    s = 0.5 * (lo + hi)
    A = concat([_placed_sphere(level, 0.5 + s * ua[k], ra[k], Ra[k]) for k in range(n_a)],
               dict(kind="tiny_spheres", seed=seed, side=s, level=level))
    B = concat([_placed_sphere(level, 0.5 + s * ub[k], rb[k], Rb[k]) for k in range(n_b)],
               dict(kind="tiny_spheres", seed=seed, side=s, level=level))
    return A, B


# ---------------------------------------------------------------------------
# Pathology-shaped data: nuclei and vessels
# ---------------------------------------------------------------------------

def nuclei(seed: int, n: int = 10000, mean_r: float = 1.0 / 200, sigma: float = 0.3,
           levels=(4, 5), noise_amp: float = 0.10, region=(0.0, 1.0)):
    """Noisy icospheres with log-normal radii (mean `mean_r` of the box)."""
    rng = np.random.default_rng(seed)
    mu = math.log(mean_r) - 0.5 * sigma * sigma
    r = np.exp(rng.normal(mu, sigma, size=n))
    r = np.clip(r, 400.0 / QMAX, 4 * mean_r)    # level-5 edges stay >= ~13 units
    lev = rng.choice(np.asarray(levels), size=n)
    lo, hi = region
    margin = r * (1 + noise_amp) + 2.0 / QMAX
    c = lo + margin[:, None] + rng.uniform(size=(n, 3)) * (hi - lo - 2 * margin[:, None])
    R = random_rotations(rng, n)
    # smooth radial field per mesh: 8 low-frequency sinusoids (see _smooth_field)
    nt = 8
    dirs = rng.normal(size=(n, nt, 3))
    dirs /= np.linalg.norm(dirs, axis=2, keepdims=True)
    w = dirs * rng.uniform(1.0, 3.0, size=(n, nt, 1))
    phase = rng.uniform(0, 2 * np.pi, size=(n, nt))
    amp = rng.uniform(0.5, 1.0, size=(n, nt))
    out = [None] * n
    w32, ph32, amp32 = w.astype(np.float32), phase.astype(np.float32), amp.astype(np.float32)
    for L in np.unique(lev):
        U, F = icosphere(int(L))
        U32 = U.astype(np.float32)
        ids = np.nonzero(lev == L)[0]
        for k0 in range(0, len(ids), 64):
            blk = ids[k0:k0 + 64]
            f = np.matmul(U32[None], w32[blk].transpose(0, 2, 1)) + ph32[blk][:, None, :]
            f = np.matmul(np.sin(f), amp32[blk][:, :, None])[..., 0] / amp32[blk].sum(axis=1)[:, None]
            X = U[None, :, :] * (1.0 + noise_amp * f.astype(np.float64))[:, :, None]
            X = np.matmul(X, R[blk].transpose(0, 2, 1)) * r[blk][:, None, None] + c[blk][:, None, :]
            Q = quantize(X)
            for j, k in enumerate(blk):
                out[k] = (Q[j], F)
    return concat(out, dict(kind="nuclei", seed=seed, n=n))


def _bspline(ctrl: np.ndarray, m: int) -> np.ndarray:
    """Clamped uniform cubic B-spline through the end control points, m samples."""
    n = len(ctrl)
    k = 3
    knots = np.concatenate([np.zeros(k), np.linspace(0, 1, n - k + 1), np.ones(k)])
    t = np.linspace(0, 1, m)
    t[-1] = 1 - 1e-12

    def basis(i, d, t):
        if d == 0:
            return ((knots[i] <= t) & (t < knots[i + 1])).astype(float)
        out = np.zeros_like(t)
        den = knots[i + d] - knots[i]
        if den > 0:
            out += (t - knots[i]) / den * basis(i, d - 1, t)
        den = knots[i + d + 1] - knots[i + 1]
        if den > 0:
            out += (knots[i + d + 1] - t) / den * basis(i + 1, d - 1, t)
        return out
    B = np.stack([basis(i, k, t) for i in range(n)], axis=1)
    return B @ ctrl


def _tube(curve: np.ndarray, radius: float, rings: int, sides: int = 16):
    """Capped tube of `rings` rings swept along a dense polyline `curve`.
    Triangles: 2 * sides * (rings - 1) + 2 * sides = 32 * rings for 16 sides."""
    seg = np.linalg.norm(np.diff(curve, axis=0), axis=1)
    s = np.concatenate([[0], np.cumsum(seg)])
    st = np.linspace(0, s[-1], rings)
    C = np.stack([np.interp(st, s, curve[:, d]) for d in range(3)], axis=1)
    T = np.gradient(C, axis=0)
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    # parallel-transport frames (no twist)
    a = np.array([1.0, 0, 0]) if abs(T[0, 0]) < 0.9 else np.array([0, 1.0, 0])
    N = np.empty_like(T)
    N[0] = np.cross(T[0], a)
    N[0] /= np.linalg.norm(N[0])
    for i in range(1, rings):
        n = N[i - 1] - np.dot(N[i - 1], T[i]) * T[i]
        N[i] = n / np.linalg.norm(n)
    Bn = np.cross(T, N)
    th = 2 * np.pi * np.arange(sides) / sides
    ring = (C[:, None, :] + radius * (np.cos(th)[None, :, None] * N[:, None, :] +
                                      np.sin(th)[None, :, None] * Bn[:, None, :]))
    V = np.concatenate([ring.reshape(-1, 3), C[:1], C[-1:]])
    c0, c1 = rings * sides, rings * sides + 1
    faces = []
    i = np.arange(rings - 1)[:, None]
    k = np.arange(sides)[None, :]
    a0 = i * sides + k
    a1 = i * sides + (k + 1) % sides
    b0 = (i + 1) * sides + k
    b1 = (i + 1) * sides + (k + 1) % sides
    faces.append(np.stack([a0, b0, b1], axis=-1).reshape(-1, 3))
    faces.append(np.stack([a0, b1, a1], axis=-1).reshape(-1, 3))
    kk = np.arange(sides)
    faces.append(np.stack([np.full(sides, c0), kk, (kk + 1) % sides], axis=-1))
    last = (rings - 1) * sides
    faces.append(np.stack([np.full(sides, c1), last + (kk + 1) % sides, last + kk], axis=-1))
    F = np.concatenate(faces).astype(np.int32)
    # outward orientation: positive enclosed signed volume
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum()
    if vol < 0:
        F = F[:, [0, 2, 1]]
    return V, F


def _curve_ok(curve, radius):
    """Reject curves that bend tighter than 3 radii or pass within 3 radii of
    themselves away from the neighbourhood of a point."""
    seg = np.linalg.norm(np.diff(curve, axis=0), axis=1)
    s = np.concatenate([[0], np.cumsum(seg)])
    d1 = np.gradient(curve, s, axis=0)
    d2 = np.gradient(d1, s, axis=0)
    kappa = np.linalg.norm(np.cross(d1, d2), axis=1) / np.maximum(
        np.linalg.norm(d1, axis=1) ** 3, 1e-30)
    if np.any(kappa[2:-2] * 3 * radius > 1):
        return False
    # non-local approach: samples spaced well below the 3-radius threshold
    step = max(1, int(len(curve) * radius / max(s[-1], 1e-12)))
    P, sp = curve[::step], s[::step]
    sq = (P * P).sum(axis=1)
    D2 = sq[:, None] + sq[None, :] - 2 * P @ P.T
    far = np.abs(sp[:, None] - sp[None, :]) > 8 * radius
    return not np.any(D2[far] < (3 * radius) ** 2)


def vessels(seed: int, n: int = 500, f_range=(10000, 50000), r_range=(1.0 / 300, 1.0 / 100),
            span=(0.3, 1.0), sides: int = 16):
    """Capped 16-sided tubes swept along random cubic B-splines."""
    rng = np.random.default_rng(seed)
    meshes = []
    while len(meshes) < n:
        radius = rng.uniform(*r_range)
        F = rng.uniform(*f_range)
        rings = max(2, int(round(F / (2 * sides))))
        ext = rng.uniform(*span)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t = np.linspace(-0.5, 0.5, 6)[:, None]
        ctrl = t * d * ext + rng.uniform(-0.15, 0.15, size=(6, 3)) * ext
        m = 2 * radius + 4.0 / QMAX
        lo, hi = ctrl.min(axis=0), ctrl.max(axis=0)
        room = (1 - 2 * m) - (hi - lo)
        if np.any(room <= 0):
            continue
        ctrl = ctrl - lo + m + rng.uniform(size=3) * room
        curve = _bspline(ctrl, 4096)
        if not _curve_ok(curve, radius):
            continue
        V, T = _tube(curve, radius, rings, sides)
        meshes.append((quantize(V), T))
    return concat(meshes, dict(kind="vessels", seed=seed, n=n))


def pathology(seed: int, n_nuclei: int = 10000, n_vessels: int = 500):
    """(A = nuclei, B = vessels) in one unit cube."""
    return nuclei(seed, n_nuclei), vessels(seed + 1, n_vessels)


# ---------------------------------------------------------------------------
# Seeded sampling helpers shared by tests and the benchmark
# ---------------------------------------------------------------------------

def sample_indices(seed: int, n: int, k: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)) if k else np.zeros(0, np.int64)
