"""Pins of the oracle's exact primitives against independent exact arithmetic.

orient3d is checked against sympy's exact determinant; the strict
segment/triangle test against a rational re-derivation (plane parameter t and
the crossing point's barycentric signs, in Fractions); the closed-triangle
point test against barycentric coordinates solved in Fractions.  Lattice
inputs with tiny coordinate ranges make ties (zeros) frequent, so a wrong
strictness or sign rule fails here.
"""
from fractions import Fraction

import numpy as np
import pytest
import sympy

import oracle

QMAX = (1 << 18) - 1


def _det_sympy(a, b, c, d):
    M = sympy.Matrix([[b[i] - a[i] for i in range(3)],
                      [c[i] - a[i] for i in range(3)],
                      [d[i] - a[i] for i in range(3)]])
    return int(M.det())


def test_orient3d_hand_values():
    o = (0, 0, 0)
    assert oracle.orient3d(o, (1, 0, 0), (0, 1, 0), (0, 0, 1)) == 1
    assert oracle.orient3d(o, (0, 1, 0), (1, 0, 0), (0, 0, 1)) == -1
    assert oracle.orient3d(o, (1, 0, 0), (0, 1, 0), (5, 7, 0)) == 0
    # extreme magnitudes: full grid span in every difference
    m = QMAX
    assert oracle.orient3d(o, (m, 0, 0), (0, m, 0), (0, 0, m)) == m ** 3


def test_orient3d_matches_exact_determinant():
    rng = np.random.default_rng(7)
    for _ in range(300):
        P = rng.integers(0, QMAX + 1, size=(4, 3))
        assert oracle.orient3d(*P) == _det_sympy(*P)
    # constructed coplanar points: d = a + i (b - a) + j (c - a), kept in range
    n = 0
    while n < 200:
        a = rng.integers(1000, 200000, size=3)
        b = a + rng.integers(-500, 500, size=3)
        c = a + rng.integers(-500, 500, size=3)
        i, j = rng.integers(-20, 20, size=2)
        d = a + i * (b - a) + j * (c - a)
        if np.any(d < 0) or np.any(d > QMAX):
            continue
        assert oracle.orient3d(a, b, c, d) == 0 == _det_sympy(a, b, c, d)
        d2 = d.copy()
        d2[rng.integers(3)] += 1
        assert oracle.orient3d(a, b, c, d2) == _det_sympy(a, b, c, d2)
        n += 1


def test_orient2d_xy():
    assert oracle.orient2d_xy((0, 0, 9), (1, 0, 3), (0, 1, 5)) == 1
    assert oracle.orient2d_xy((0, 0, 0), (0, 1, 0), (1, 0, 0)) == -1
    assert oracle.orient2d_xy((0, 0, 0), (2, 2, 0), (5, 5, 7)) == 0


# -- strict segment/triangle crossing ----------------------------------------

def _cross(u, v):
    return (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])


def _sub(u, v):
    return tuple(x - y for x, y in zip(u, v))


def _dot(u, v):
    return sum(x * y for x, y in zip(u, v))


def segtri_rational(p, q, a, b, c):
    """Open segment pq meets open triangle abc at one interior point."""
    p, q, a, b, c = (tuple(int(x) for x in t) for t in (p, q, a, b, c))
    n = _cross(_sub(b, a), _sub(c, a))
    if n == (0, 0, 0):
        return False
    sp, sq = _dot(n, _sub(p, a)), _dot(n, _sub(q, a))
    if sp == 0 or sq == 0 or (sp > 0) == (sq > 0):
        return False
    t = Fraction(sp, sp - sq)                     # plane crossing, strictly in (0, 1)
    X = tuple(Fraction(p[i]) + t * (q[i] - p[i]) for i in range(3))
    for s, e in ((a, b), (b, c), (c, a)):
        edge = _sub(e, s)
        w = tuple(X[i] - s[i] for i in range(3))
        if _dot(_cross(edge, w), n) <= 0:        # on an edge line or outside
            return False
    return True


def test_segtri_hand_cases():
    a, b, c = (0, 0, 0), (10, 0, 0), (0, 10, 0)
    assert oracle.segtri_strict((2, 2, -1), (2, 2, 1), a, b, c)
    assert oracle.segtri_strict((2, 2, 1), (2, 2, -1), a, b, c)
    assert not oracle.segtri_strict((2, 2, 0), (2, 2, 1), a, b, c)      # endpoint on the face
    assert not oracle.segtri_strict((5, 0, -1), (5, 0, 1), a, b, c)     # through an edge
    assert not oracle.segtri_strict((0, 0, -1), (0, 0, 1), a, b, c)     # through a vertex
    assert not oracle.segtri_strict((1, 1, 0), (3, 2, 0), a, b, c)      # coplanar
    assert not oracle.segtri_strict((20, 20, -1), (20, 20, 1), a, b, c)  # misses
    assert not oracle.segtri_strict((2, 2, 1), (2, 2, 3), a, b, c)      # same side
    # zero-area triangle never hits
    assert not oracle.segtri_strict((1, 0, -1), (1, 0, 1), (0, 0, 0), (2, 0, 0), (4, 0, 0))


@pytest.mark.parametrize("span,n", [(3, 4000), (6, 3000), (QMAX + 1, 1500)])
def test_segtri_matches_rational(span, n):
    rng = np.random.default_rng(span)
    hits = 0
    for _ in range(n):
        P = rng.integers(0, span, size=(5, 3))
        exp = segtri_rational(*P)
        assert oracle.segtri_strict(*P) == exp, P.tolist()
        hits += exp
    assert hits > 0


def test_segtri_symmetries():
    """Swapping p and q, or cyclically rotating / reversing the triangle,
    never changes the result."""
    rng = np.random.default_rng(11)
    for _ in range(2000):
        p, q, a, b, c = rng.integers(0, 5, size=(5, 3))
        r = oracle.segtri_strict(p, q, a, b, c)
        assert oracle.segtri_strict(q, p, a, b, c) == r
        assert oracle.segtri_strict(p, q, b, c, a) == r
        assert oracle.segtri_strict(p, q, a, c, b) == r


# -- point in closed triangle --------------------------------------------------

def in_triangle_rational(v, a, b, c):
    v, a, b, c = (tuple(int(x) for x in t) for t in (v, a, b, c))
    e1, e2, w = _sub(b, a), _sub(c, a), _sub(v, a)
    n = _cross(e1, e2)
    assert n != (0, 0, 0)
    if _dot(n, w) != 0:
        return False
    # solve w = s e1 + t e2 via the Gram system
    g11, g12, g22 = _dot(e1, e1), _dot(e1, e2), _dot(e2, e2)
    r1, r2 = _dot(w, e1), _dot(w, e2)
    den = g11 * g22 - g12 * g12
    s = Fraction(r1 * g22 - r2 * g12, den)
    t = Fraction(g11 * r2 - g12 * r1, den)
    return s >= 0 and t >= 0 and s + t <= 1


def test_point_in_closed_triangle_matches_rational():
    rng = np.random.default_rng(3)
    n_in = 0
    for _ in range(3000):
        a, b, c = rng.integers(0, 5, size=(3, 3))
        if _cross(_sub(b, a), _sub(c, a)) == (0, 0, 0):
            continue
        # half of the points are drawn on the triangle's plane lattice
        if rng.random() < 0.5:
            s, t = rng.integers(-1, 3, size=2)
            v = a + s * (b - a) + t * (c - a)
        else:
            v = rng.integers(0, 5, size=3)
        exp = in_triangle_rational(v, a, b, c)
        assert oracle.point_in_closed_triangle(v, a, b, c) == exp
        n_in += exp
    assert n_in > 100


def test_point_in_degenerate_triangle():
    # collinear corners: the hull is a segment
    a, b, c = (0, 0, 0), (4, 4, 4), (2, 2, 2)
    assert oracle.point_in_closed_triangle((1, 1, 1), a, b, c)
    assert oracle.point_in_closed_triangle((4, 4, 4), a, b, c)
    assert not oracle.point_in_closed_triangle((5, 5, 5), a, b, c)
    assert not oracle.point_in_closed_triangle((1, 1, 2), a, b, c)
    # coincident corners: a single point
    assert oracle.point_in_closed_triangle((3, 3, 3), (3, 3, 3), (3, 3, 3), (3, 3, 3))
    assert not oracle.point_in_closed_triangle((3, 3, 4), (3, 3, 3), (3, 3, 3), (3, 3, 3))


# -- the perturbed upward ray ------------------------------------------------

def test_ray_up_hand_cases():
    a, b, c = (0, 0, 5), (10, 0, 5), (0, 10, 5)          # ccw from above
    assert oracle.ray_up_hits((2, 2, 0), a, b, c)
    assert oracle.ray_up_hits((2, 2, 0), a, c, b)          # orientation irrelevant
    assert not oracle.ray_up_hits((2, 2, 6), a, b, c)      # above the triangle
    assert not oracle.ray_up_hits((2, 2, 5), a, b, c)      # on it: never counted
    assert not oracle.ray_up_hits((20, 2, 0), a, b, c)
    vert = ((0, 0, 0), (10, 0, 0), (0, 0, 10))             # vertical: zero xy area
    assert not oracle.ray_up_hits((2, 0, -5), *vert)
    # a ray through the shared edge of two triangles hits exactly one of them
    sq = [(0, 0, 5), (10, 0, 5), (10, 10, 5), (0, 10, 5)]
    t1, t2 = (sq[0], sq[1], sq[2]), (sq[0], sq[2], sq[3])
    for v in [(5, 5, 0), (0, 0, 0), (3, 3, 1)]:
        assert oracle.ray_up_hits(v, *t1) + oracle.ray_up_hits(v, *t2) == 1, v
    # the perturbed point (x + e, y + e^2) leaves the square at its far corner
    assert oracle.ray_up_hits((10, 10, 0), *t1) + oracle.ray_up_hits((10, 10, 0), *t2) == 0
    # ... and through the shared vertex of a triangle fan exactly one
    centre = (5, 5, 5)
    ring = [(0, 0, 5), (10, 0, 5), (10, 10, 5), (0, 10, 5)]
    fan = [(centre, ring[k], ring[(k + 1) % 4]) for k in range(4)]
    assert sum(oracle.ray_up_hits((5, 5, 0), *t) for t in fan) == 1
