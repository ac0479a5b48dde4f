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


def mesh_boxes(ds: MeshSet) -> np.ndarray:
    """M x 6 float32 (lo x, y, z, hi x, y, z) of each mesh's vertices."""
    out = np.zeros((ds.nmesh, 6), dtype=np.float32)
    for k in range(ds.nmesh):
        v = ds.xyz[ds.voff[k]:ds.voff[k + 1]]
        out[k, :3], out[k, 3:] = v.min(0), v.max(0)
    return out


def windows(seed: int, n: int, half_range=(1 << 10, 1 << 16)):
    """n query windows on the grid: centres uniform, half-sizes log-uniform in
    half_range (grid units), clipped to the grid.  Returns (lo, hi), n x 3
    int32 each."""
    rng = np.random.default_rng(seed)
    c = rng.integers(0, GRID, size=(n, 3))
    h = np.exp(rng.uniform(np.log(half_range[0]), np.log(half_range[1]), size=(n, 3)))
    lo = np.clip(c - h, 0, QMAX).astype(np.int32)
    hi = np.clip(c + h, 0, QMAX).astype(np.int32)
    return lo, hi


def serving_windows(seed: int, n: int, frac_range=(1e-3, 1.0)):
    """n cube windows whose volume, as a fraction of the grid cube, is
    log-uniform in frac_range, placed uniformly inside the grid.  Over a
    dataset spread through the cube, a window selects about that fraction
    of its meshes (10 to 10,000 of 10,000 nuclei for the default range).
    Returns (lo, hi), n x 3 int32 each."""
    rng = np.random.default_rng(seed)
    f = np.exp(rng.uniform(np.log(frac_range[0]), np.log(frac_range[1]), size=n))
    side = np.minimum(np.cbrt(f) * QMAX, QMAX)
    lo = rng.uniform(0, 1, size=(n, 3)) * (QMAX - side)[:, None]
    lo = np.floor(lo).astype(np.int64)
    hi = np.minimum(lo + np.ceil(side)[:, None].astype(np.int64), QMAX)
    return lo.astype(np.int32), hi.astype(np.int32)


def poisson_arrivals(seed: int, rate: float, n: int) -> np.ndarray:
    """n arrival times (seconds from 0) of a Poisson stream of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


# ---------------------------------------------------------------------------
# Batching workload: many candidate pairs of very uneven size, built from a
# pool of template meshes placed by per-pair integer translations
# ---------------------------------------------------------------------------

def latlong_sphere(faces: int, radius: float, centre, rng, noise_amp: float = 0.05):
    """Closed latitude/longitude sphere with about `faces` triangles
    (F = 2 s (r - 1) for s segments and r rings), smooth radial noise."""
    s = max(3, int(round(math.sqrt(faces / 2.0))))
    r = max(2, int(round(faces / (2.0 * s))) + 1)
    lat = np.linspace(0, np.pi, r + 1)[1:-1]            # r - 1 interior rings
    lon = np.linspace(0, 2 * np.pi, s, endpoint=False)
    ring = np.stack([np.sin(lat)[:, None] * np.cos(lon)[None, :],
                     np.sin(lat)[:, None] * np.sin(lon)[None, :],
                     np.cos(lat)[:, None] * np.ones_like(lon)[None, :]], axis=-1).reshape(-1, 3)
    U = np.concatenate([[[0, 0, 1.0]], ring, [[0, 0, -1.0]]])
    field = _smooth_field(rng)
    X = U * (1.0 + noise_amp * field(U))[:, None] * radius + np.asarray(centre)
    N, S = 0, len(U) - 1
    idx = lambda i, j: 1 + i * s + (j % s)               # ring i, segment j
    faces_l = []
    for j in range(s):
        faces_l.append((N, idx(0, j), idx(0, j + 1)))
    for i in range(r - 2):
        for j in range(s):
            faces_l.append((idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)))
            faces_l.append((idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)))
    for j in range(s):
        faces_l.append((S, idx(r - 2, j + 1), idx(r - 2, j)))
    F = np.array(faces_l, dtype=np.int32)
    a, b, c = X[F[:, 0]], X[F[:, 1]], X[F[:, 2]]
    if np.einsum("ij,ij->i", a - centre, np.cross(b - a, c - a)).sum() < 0:
        F = F[:, [0, 2, 1]]
    return quantize(X), F


def _short_tube(rng, faces: int, centre, radius: float, length: float):
    rings = max(2, int(round(faces / 32.0)))
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    e = np.cross(d, rng.normal(size=3))
    e /= np.linalg.norm(e)
    t = np.linspace(-0.5, 0.5, 5)[:, None]
    ctrl = np.asarray(centre) + t * d * length + (t ** 2 - 0.1) * e * length * 0.3
    curve = _bspline(ctrl, 1024)
    V, T = _tube(curve, radius, rings)
    return quantize(V), T


def batching(seed: int, n_pairs: int = 100000, n_templates: int = 2000,
             f_range=(200, 50000), classes=(0.30, 0.10, 0.60)):
    """(A templates, B templates, candidates n x 2, offsets n x 3, intended
    class per pair: 0 crossing, 1 containment, 2 disjoint with overlapping
    boxes).  Face counts are log-uniform in f_range; half the templates are
    noisy spheres and half short swept tubes (spheres below 1,000 faces).
    Every template sits at the box centre; pair k tests A_i against B_j
    translated by offsets[k]."""
    rng = np.random.default_rng(seed)
    centre = np.full(3, 0.5)

    def pool(n):
        meshes, radius, kind = [], [], []
        for _ in range(n):
            F = math.exp(rng.uniform(math.log(f_range[0]), math.log(f_range[1])))
            if F < 1000 or rng.random() < 0.5:
                rr = rng.uniform(0.01, 0.04)
                meshes.append(latlong_sphere(int(F), rr, centre, rng))
                kind.append(0)
            else:
                rr = rng.uniform(0.003, 0.008)
                meshes.append(_short_tube(rng, int(F), centre, rr, rng.uniform(0.04, 0.1)))
                kind.append(1)
            v = meshes[-1][0].astype(np.float64)
            radius.append(np.linalg.norm(v - v.mean(axis=0), axis=1).max())
        return meshes, np.array(radius), np.array(kind)

    ma, ra, ka = pool(n_templates)
    mb, rb, kb = pool(n_templates)
    A = concat(ma, dict(kind="batching_templates", seed=seed))
    B = concat(mb, dict(kind="batching_templates", seed=seed + 1))
    lo_a = np.stack([v.min(axis=0) for v, _ in ma]).astype(np.int64)
    hi_a = np.stack([v.max(axis=0) for v, _ in ma]).astype(np.int64)
    lo_b = np.stack([v.min(axis=0) for v, _ in mb]).astype(np.int64)
    hi_b = np.stack([v.max(axis=0) for v, _ in mb]).astype(np.int64)
    ca, cb = (lo_a + hi_a) / 2.0, (lo_b + hi_b) / 2.0
    spheres_a = np.nonzero(ka == 0)[0]
    cls = rng.choice(3, size=n_pairs, p=np.asarray(classes) / np.sum(classes))
    cand = np.zeros((n_pairs, 2), dtype=np.int32)
    off = np.zeros((n_pairs, 3), dtype=np.int64)
    small_b = np.argsort(rb)
    for k in range(n_pairs):
        if cls[k] == 1:
            i = int(rng.choice(spheres_a))
            # a B template well inside A's inscribed ball
            fit = small_b[: max(1, np.searchsorted(rb[small_b], 0.35 * ra[i]))]
            j = int(rng.choice(fit))
            u = rng.normal(size=3)
            d = u / np.linalg.norm(u) * rng.uniform(0, 0.15) * ra[i]
        else:
            i, j = int(rng.integers(n_templates)), int(rng.integers(n_templates))
            if cls[k] == 0:
                u = rng.normal(size=3)
                d = u / np.linalg.norm(u) * ra[i] * rng.uniform(0.85, 1.05)
            else:
                h = (hi_a[i] - lo_a[i] + hi_b[j] - lo_b[j]) / 2.0
                d = rng.choice([-1.0, 1.0], size=3) * h * rng.uniform(0.8, 0.95, size=3)
        o = np.rint(ca[i] + d - cb[j]).astype(np.int64)
        o = np.clip(o, -lo_b[j], QMAX - hi_b[j])
        cand[k] = (i, j)
        off[k] = o
    return A, B, cand, off.astype(np.int32), cls.astype(np.int8)


# ---------------------------------------------------------------------------
# Urban precision stress: extruded star-shaped buildings with pitched roofs
# on a jittered grid, some sharing walls exactly, plus boxes and cylinders
# ---------------------------------------------------------------------------

def building(footprint: np.ndarray, z0: int, height: int, roof: int, bands: int):
    """Closed prism over a star-shaped integer footprint (n x 2, counter-
    clockwise around its first point's kernel centre), walls split into
    `bands` rows, pitched roof to an apex over the footprint centre.
    F = 2 n (bands + 1)."""
    n = len(footprint)
    cx, cy = np.rint(footprint.mean(axis=0))
    levels = np.rint(np.linspace(z0, z0 + height, bands + 1)).astype(np.int64)
    rings = [np.column_stack([footprint, np.full(n, z)]) for z in levels]
    V = np.concatenate([[[cx, cy, z0]]] + rings + [[[cx, cy, z0 + height + roof]]]).astype(np.float64)
    bot, apex = 0, len(V) - 1
    vid = lambda lv, k: 1 + lv * n + (k % n)
    F = []
    for k in range(n):
        F.append((bot, vid(0, k + 1), vid(0, k)))
    for lv in range(bands):
        for k in range(n):
            F.append((vid(lv, k), vid(lv, k + 1), vid(lv + 1, k + 1)))
            F.append((vid(lv, k), vid(lv + 1, k + 1), vid(lv + 1, k)))
    for k in range(n):
        F.append((apex, vid(bands, k), vid(bands, k + 1)))
    return V.astype(np.float32), np.array(F, dtype=np.int32)


def _star(rng, n, R):
    th = np.sort(2 * np.pi * (np.arange(n) + rng.uniform(-0.3, 0.3, size=n)) / n)
    rr = R * rng.uniform(0.6, 1.0, size=n)
    return np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)


def _rect(w, h, per_side):
    """Rectangle boundary, counter-clockwise, per_side points on each side."""
    t = np.arange(per_side) / per_side
    pts = [np.stack([-w / 2 + w * t, np.full(per_side, -h / 2)], 1),
           np.stack([np.full(per_side, w / 2), -h / 2 + h * t], 1),
           np.stack([w / 2 - w * t, np.full(per_side, h / 2)], 1),
           np.stack([np.full(per_side, -w / 2), h / 2 - h * t], 1)]
    return np.concatenate(pts)


def cylinder(centre, radius: float, height: float, sides: int, z_axis=True):
    """Capped cylinder (4 * sides triangles) around a vertical axis."""
    th = 2 * np.pi * np.arange(sides) / sides
    ring = np.stack([radius * np.cos(th), radius * np.sin(th)], 1)
    cx, cy, cz = centre
    V = np.concatenate([[[cx, cy, cz]],
                        np.column_stack([ring + [cx, cy], np.full(sides, cz)]),
                        np.column_stack([ring + [cx, cy], np.full(sides, cz + height)]),
                        [[cx, cy, cz + height]]])
    F = []
    for k in range(sides):
        a, b = 1 + k, 1 + (k + 1) % sides
        F += [(0, b, a), (a, b, b + sides), (a, b + sides, a + sides),
              (len(V) - 1, a + sides, b + sides)]
    return np.rint(V).astype(np.float32), np.array(F, dtype=np.int32)


def urban(seed: int, n_buildings: int = 50000, n_parts: int = 5000,
          f_range=(100, 2000), degenerate_frac: float = 0.05):
    """One dataset for a self join: buildings (F log-uniform in f_range, 6-64
    footprint sides) on a jittered grid; a `degenerate_frac` share of them
    come as exactly adjacent rectangular pairs sharing a wall plane, an edge
    or a corner; plus boxes and cylinders placed among them."""
    rng = np.random.default_rng(seed)
    side = int(math.ceil(math.sqrt(n_buildings)))
    cell = QMAX / (side + 6.0)          # a 3-cell margin keeps every mesh on the grid
    meshes, tags = [], []
    k = 0
    while k < n_buildings:
        gx, gy = k % side, k // side
        base = np.array([(gx + 3.5) * cell, (gy + 3.5) * cell])
        F = math.exp(rng.uniform(math.log(f_range[0]), math.log(f_range[1])))
        z0 = int(rng.integers(1000, 3000))
        height = int(rng.integers(int(0.5 * cell), int(3 * cell)))
        if rng.random() < degenerate_frac and k + 1 < n_buildings:
            # two rectangular buildings touching exactly
            w, h = int(0.45 * cell), int(0.35 * cell)
            per = max(2, int(F / 16))
            bands = max(1, int(F / (2 * 4 * per)) - 1)
            fp = np.rint(_rect(w, h, per) + base).astype(np.int64)
            meshes.append(building(fp.astype(np.float64), z0, height, int(0.3 * h), bands))
            mode = rng.integers(3)
            shift = {0: (w, 0), 1: (w, h), 2: (w, int(h / 2))}[int(mode)]
            fp2 = fp + np.array(shift)
            meshes.append(building(fp2.astype(np.float64), z0 if mode != 1 else z0 + height // 3,
                                   height, int(0.3 * h), bands))
            tags += ["shared_wall", "shared_wall"] if mode != 1 else ["shared_edge", "shared_edge"]
            k += 2
            continue
        n = int(rng.integers(6, max(7, min(64, int(F / 4)) + 1)))
        bands = max(1, int(round(F / (2 * n))) - 1)
        R = cell * rng.uniform(0.35, 0.7)
        fp = np.rint(_star(rng, n, R) + base + rng.uniform(-0.2, 0.2, size=2) * cell)
        meshes.append(building(fp, z0, height, int(rng.uniform(0.2, 0.5) * R), bands))
        tags.append("building")
        k += 1
    for _ in range(n_parts):
        c = np.array([rng.uniform(3 * cell, QMAX - 3 * cell), rng.uniform(3 * cell, QMAX - 3 * cell),
                      rng.uniform(800, 3000)])
        if rng.random() < 0.5:
            h = rng.uniform(0.3, 1.5, size=3) * cell
            meshes.append(box(np.rint(c), np.rint(c + h)))
            tags.append("box")
        else:
            meshes.append(cylinder(c, rng.uniform(0.1, 0.5) * cell, rng.uniform(0.5, 2) * cell,
                                   int(rng.integers(8, 33))))
            tags.append("cylinder")
    meshes = [(np.asarray(v, np.float32), t) for v, t in meshes]
    return concat(meshes, dict(kind="urban", seed=seed, tags=tags))
