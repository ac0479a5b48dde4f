"""The FP32 filter bounds of the leaf tests and the conservative slab test,
checked on the CPU.

The segment/triangle test is exact on the 2^18 grid (the strict reading of
Sec. 3.2 and the robustness discussion of Sec. 3.6): five orientation signs,
each the sign of det[a - p; b - p; c - p] for four grid points.  The kernel
first evaluates each determinant in FP32 and trusts the sign when
|det_f32| > 2^-18 D^3, where D is the largest side of a box holding all four
points; otherwise it decides the sign exactly.  The claim behind that bound:
every difference is at most D per coordinate, each permanent of the triple
products is at most 6 D^3, and the FP32 evaluation (two rounded products and
a rounded difference per cross-product component, three rounded products and
two rounded sums for the dot product, no fused multiply-add) errs by less
than 30 u D^3 < 2^-18 D^3 with u = 2^-24.

numpy float32 arithmetic rounds every product, sum and difference to nearest
exactly like the kernel's explicit round-to-nearest intrinsics, so these
tests reproduce the kernel's FP32 values bit for bit and compare them with the
exact integer determinant: the error stays below the bound on random,
near-coplanar and extreme-magnitude inputs, so a certified sign is always the
exact sign.
"""
import numpy as np
import pytest

QMAX = (1 << 18) - 1


def det_f32(p, a, b, c):
    """FP32 dot3(a - p, cross3(b - p, c - p)), in the kernel's operation order."""
    f = np.float32
    A, B, C = (np.asarray(v, f) - np.asarray(p, f) for v in (a, b, c))
    cx = B[:, 1] * C[:, 2] - B[:, 2] * C[:, 1]
    cy = B[:, 2] * C[:, 0] - B[:, 0] * C[:, 2]
    cz = B[:, 0] * C[:, 1] - B[:, 1] * C[:, 0]
    return (A[:, 0] * cx + A[:, 1] * cy) + A[:, 2] * cz


def det_exact(p, a, b, c):
    """The same determinant in int64 (differences < 2^19, |det| < 2^57)."""
    A, B, C = (np.asarray(v, np.int64) - np.asarray(p, np.int64) for v in (a, b, c))
    cx = B[:, 1] * C[:, 2] - B[:, 2] * C[:, 1]
    cy = B[:, 2] * C[:, 0] - B[:, 0] * C[:, 2]
    cz = B[:, 0] * C[:, 1] - B[:, 1] * C[:, 0]
    return A[:, 0] * cx + A[:, 1] * cy + A[:, 2] * cz


def det_perm_f32(p, a, b, c):
    """The per-test filter of the other front ends: the FP32 determinant and
    its error bound 2^-21 x (the permanent, evaluated in FP32), each value
    rounded to nearest in the kernel's order."""
    f = np.float32
    A, B, C = (np.asarray(v, f) - np.asarray(p, f) for v in (a, b, c))
    p1, p2 = B[:, 1] * C[:, 2], B[:, 2] * C[:, 1]
    p3, p4 = B[:, 2] * C[:, 0], B[:, 0] * C[:, 2]
    p5, p6 = B[:, 0] * C[:, 1], B[:, 1] * C[:, 0]
    m = (p1 - p2, p3 - p4, p5 - p6)
    pm = (np.abs(p1) + np.abs(p2), np.abs(p3) + np.abs(p4), np.abs(p5) + np.abs(p6))
    det = (A[:, 0] * m[0] + A[:, 1] * m[1]) + A[:, 2] * m[2]
    perm = (np.abs(A[:, 0]) * pm[0] + np.abs(A[:, 1]) * pm[1]) + np.abs(A[:, 2]) * pm[2]
    return det, perm * f(2.0 ** -21)


def check_perm(p, a, b, c):
    """Error below the per-test bound; a certified sign equals the exact sign."""
    det, err = det_perm_f32(p, a, b, c)
    e = det_exact(p, a, b, c)
    assert (det == det_f32(p, a, b, c)).all()   # the same determinant as the static filter
    gap = np.abs(det.astype(np.float64) - e.astype(np.float64))
    assert (gap <= err.astype(np.float64)).all()
    cert = np.abs(det) > err
    assert (np.sign(det[cert]) == np.sign(e[cert])).all()
    return cert


def check(p, a, b, c, D):
    """Error below the bound; a certified sign equals the exact sign."""
    f = det_f32(p, a, b, c).astype(np.float64)
    e = det_exact(p, a, b, c)
    bound = (np.asarray(D, np.float64) ** 3) * 2.0 ** -18
    err = np.abs(f - e.astype(np.float64))
    # e as float64 is exact to 2^-52 relative; the margin below covers it
    assert (err <= bound).all(), float((err / bound).max())
    cert = np.abs(f) > bound
    assert (np.sign(f[cert]) == np.sign(e[cert])).all()
    return err / bound, cert


def boxed_points(rng, n, D):
    """n quadruples of grid points inside a box of side D placed on the grid."""
    D = np.asarray(D, np.int64)
    x0 = rng.integers(0, QMAX - D + 1, size=(n, 3)) if D.ndim == 0 else \
        (rng.random((n, 3)) * (QMAX - D + 1)[:, None]).astype(np.int64)
    Dv = D if D.ndim else np.full(n, int(D))
    pts = [x0 + (rng.random((n, 3)) * (Dv[:, None] + 1)).astype(np.int64) for _ in range(4)]
    return pts, Dv


@pytest.mark.parametrize("D", [1, 7, 100, 4096, 1 << 15, QMAX])
def test_static_bound_random(D):
    rng = np.random.default_rng(7000 + D % 997)
    (p, a, b, c), Dv = boxed_points(rng, 400_000, D)
    ratio, _ = check(p, a, b, c, Dv)
    # the analysis leaves a factor of about 2 (30 u against 64 u)
    assert ratio.max() < 0.6


def test_static_bound_mixed_sizes():
    rng = np.random.default_rng(7100)
    n = 1_000_000
    D = np.exp(rng.uniform(0, np.log(QMAX), size=n)).astype(np.int64).clip(1, QMAX)
    (p, a, b, c), Dv = boxed_points(rng, n, D)
    check(p, a, b, c, Dv)


def test_static_bound_near_coplanar():
    """p on the plane of a, b, c (an integer barycentric point) or one grid
    step off it: exact determinants zero or near zero, where a wrong
    certified sign would show."""
    rng = np.random.default_rng(7200)
    n = 600_000
    D = np.exp(rng.uniform(np.log(16), np.log(QMAX), size=n)).astype(np.int64)
    (a, _, _, _), Dv = boxed_points(rng, n, D)
    a = np.minimum(a, QMAX - D[:, None])                # room for the triangle
    q = D[:, None] // 4
    b = a + 4 * (rng.random((n, 3)) * (q + 1)).astype(np.int64)
    c = a + 4 * (rng.random((n, 3)) * (q + 1)).astype(np.int64)
    i = rng.integers(0, 5, size=n)
    j = (rng.random(n) * (5 - i)).astype(np.int64)      # i + j <= 4
    p = (a * (4 - i - j)[:, None] + b * i[:, None] + c * j[:, None]) // 4
    off = rng.random(n) < 0.5
    p[off] += rng.integers(-1, 2, size=(int(off.sum()), 3))
    lo, hi = np.minimum(np.minimum(a, b), c), np.maximum(np.maximum(a, b), c)
    p = np.clip(p, lo, hi)                              # inside the box of a, b, c
    _, cert = check(p, a, b, c, Dv)
    e = det_exact(p, a, b, c)
    assert (e == 0).sum() > n // 4   # exact zeros occur and are never certified
    assert not cert[e == 0].any()
    assert ((e != 0) & (np.abs(e) < 1000)).sum() > 1000


def test_static_bound_extremes():
    """Box corners: the permanents reach their maximum 6 D^3 order."""
    rng = np.random.default_rng(7300)
    n = 200_000
    D = QMAX
    corner = lambda: rng.integers(0, 2, size=(n, 3)) * D
    p, a, b, c = corner(), corner(), corner(), corner()
    check(p, a, b, c, np.full(n, D))
    # near-corners, one unit inside
    jig = lambda v: np.clip(v + rng.integers(-1, 2, size=(n, 3)), 0, QMAX)
    check(jig(p), jig(a), jig(b), jig(c), np.full(n, D))


def test_per_test_bound_random_and_near_coplanar():
    rng = np.random.default_rng(7400)
    n = 600_000
    D = np.exp(rng.uniform(0, np.log(QMAX), size=n)).astype(np.int64).clip(1, QMAX)
    (p, a, b, c), _ = boxed_points(rng, n, D)
    cert = check_perm(p, a, b, c)
    assert cert.mean() > 0.9               # random orientations are nearly all certified
    # near the plane: midpoints and small offsets from it
    q = D[:, None] // 4
    a = np.minimum(a, QMAX - D[:, None])
    b = a + 4 * (rng.random((n, 3)) * (q + 1)).astype(np.int64)
    c = a + 4 * (rng.random((n, 3)) * (q + 1)).astype(np.int64)
    p = (2 * a + b + c) // 4 + rng.integers(-1, 2, size=(n, 3))
    p = np.clip(p, np.minimum(np.minimum(a, b), c), np.maximum(np.maximum(a, b), c))
    cert = check_perm(p, a, b, c)
    e = det_exact(p, a, b, c)
    assert not cert[e == 0].any() and (e == 0).sum() > 1000


# -- the conservative slab test of the breadth-first and per-warp fronts --------

def slab_hit_f32(p, q, lo, hi):
    """The kernels' segment/box slab test in FP32, in their operation order:
    t = (bound - p) * rcp(d) with a correctly rounded reciprocal (numpy's
    float32 1/d), t_enter <= t_exit * (1 + 2^-20)."""
    f = np.float32
    p, q, lo, hi = (np.asarray(v, f) for v in (p, q, lo, hi))
    d = q - p
    tmin = np.zeros(len(p), f)
    tmax = np.ones(len(p), f)
    big = f(1e30)
    for k in range(3):
        z = d[:, k] == 0
        inv = np.where(z, f(0), f(1) / np.where(z, f(1), d[:, k]))
        t0 = np.where(z, np.where(p[:, k] >= lo[:, k], -big, big), (lo[:, k] - p[:, k]) * inv)
        t1 = np.where(z, np.where(p[:, k] <= hi[:, k], big, -big), (hi[:, k] - p[:, k]) * inv)
        tmin = np.maximum(tmin, np.minimum(t0, t1))
        tmax = np.minimum(tmax, np.maximum(t0, t1))
    return tmin <= tmax * f(1.00000095367431640625)


def seg_box_exact(p, q, lo, hi):
    """Whether the closed segment meets the closed box, in exact rationals:
    t ranges (num / den, den > 0) intersected over the axes and [0, 1]."""
    p, q, lo, hi = (np.asarray(v, np.int64) for v in (p, q, lo, hi))
    n = len(p)
    d = q - p
    a_num, a_den = np.zeros(n, np.int64), np.ones(n, np.int64)     # t_enter
    b_num, b_den = np.ones(n, np.int64), np.ones(n, np.int64)      # t_exit
    ok = np.ones(n, bool)
    for k in range(3):
        z = d[:, k] == 0
        ok &= ~z | ((p[:, k] >= lo[:, k]) & (p[:, k] <= hi[:, k]))
        s = np.where(d[:, k] < 0, -1, 1)
        den = np.where(z, 1, np.abs(d[:, k]))
        n0, n1 = s * (lo[:, k] - p[:, k]), s * (hi[:, k] - p[:, k])
        e_num, x_num = np.minimum(n0, n1), np.maximum(n0, n1)
        # t_enter = max(t_enter, e_num / den); t_exit = min(t_exit, x_num / den)
        later = ~z & (e_num * a_den > a_num * den)
        a_num, a_den = np.where(later, e_num, a_num), np.where(later, den, a_den)
        sooner = ~z & (x_num * b_den < b_num * den)
        b_num, b_den = np.where(sooner, x_num, b_num), np.where(sooner, den, b_den)
    return ok & (a_num * b_den <= b_num * a_den)


def test_slab_never_rejects_a_met_box_random():
    rng = np.random.default_rng(7500)
    n = 1_000_000
    S = np.exp(rng.uniform(0, np.log(QMAX), size=n)).astype(np.int64)[:, None]
    base = (rng.random((n, 3)) * (QMAX - S)).astype(np.int64)
    pt = lambda: base + (rng.random((n, 3)) * (S + 1)).astype(np.int64)
    p, q, u, v = pt(), pt(), pt(), pt()
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    met = seg_box_exact(p, q, lo, hi)
    hit = slab_hit_f32(p, q, lo, hi)
    assert not (met & ~hit).any()
    assert 0.05 < met.mean() < 0.95


def test_slab_never_rejects_a_touched_box():
    """Boxes that the segment only touches: a corner, an edge or a face of
    the box lies on a grid point of the segment."""
    rng = np.random.default_rng(7600)
    n = 600_000
    step = rng.integers(-64, 65, size=(n, 3))
    step[np.abs(step).sum(axis=1) == 0, 0] = 1
    m = rng.integers(1, 2000, size=n)
    span = np.abs(step) * m[:, None]
    p = (rng.random((n, 3)) * (QMAX - span)).astype(np.int64) + np.where(step < 0, span, 0)
    q = p + step * m[:, None]
    j = (rng.random(n) * (m + 1)).astype(np.int64)
    x = p + step * j[:, None]                          # a grid point on the segment
    ext = rng.integers(0, 500, size=(n, 3))
    side = rng.integers(0, 3, size=(n, 3))              # box below, above or around x per axis
    lo = np.where(side == 0, x - ext, np.where(side == 1, x, x - ext))
    hi = np.where(side == 0, x, np.where(side == 1, x + ext, x + ext))
    lo, hi = np.clip(lo, 0, QMAX), np.clip(hi, 0, QMAX)
    assert seg_box_exact(p, q, lo, hi).all()           # x is in the closed box
    assert slab_hit_f32(p, q, lo, hi).all()
