"""Pins of the oracle's mesh-level predicates: parity, representative vertex,
cross, intersects and the join.

Independent references used here: coordinate tests for boxes and octahedra,
half-space tests for tetrahedra and icospheres (Python integers), the
generalised winding number (solid angles in float64) for non-convex tubes,
closed forms for axis-aligned boxes and spheres, an exact convex
separating-axis test over exhaustive lattice placements, and invariants of the
predicate (swap, translation, axis permutation, reflection, relabelling).
"""
import itertools
import os
import sys

import numpy as np
import pytest

import oracle
from cases import HAND, lattice_case_sets, sat_overlap
from paper_2609_24513_gb300 import synth

QMAX = synth.QMAX


def one(mesh):
    return synth.concat([mesh])


# -- generators --------------------------------------------------------------

def _directed_edges_once(v, t):
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    u = np.unique(e, axis=0)
    rev = {(int(a), int(b)) for a, b in u}
    return len(u) == len(e) and all((b, a) in rev for a, b in rev)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere_counts_and_closure(level):
    V, F = synth.icosphere(level)
    assert len(F) == 20 * 4 ** level and len(V) == 10 * 4 ** level + 2
    assert _directed_edges_once(V, F)


def test_generated_meshes_are_closed_and_consistently_oriented():
    A, B = synth.tiny_spheres(1001)
    Vn = synth.vessels(5, n=3, f_range=(2000, 4000))
    N = synth.nuclei(6, n=3)
    for ds in (A, B, Vn, N):
        for k in range(ds.nmesh):
            v, t = ds.mesh(k)
            assert oracle.is_closed_manifold(ds, k)
            assert _directed_edges_once(v, t)
            # no repeated positions after quantisation
            assert len(np.unique(v, axis=0)) == len(v)
    for k in range(Vn.nmesh):
        v, t = Vn.mesh(k)
        rings = (len(v) - 2) // 16
        assert len(t) == 32 * rings


def test_manifold_check_rejects_open_and_t_junction():
    v, t = synth.box((0, 0, 0), (4, 4, 4))
    assert oracle.is_closed_manifold(one((v, t)), 0)
    assert not oracle.is_closed_manifold(one((v, t[:-1])), 0)            # a hole
    t2 = np.concatenate([t, t[:1]])                                      # an edge used 3+ times
    assert not oracle.is_closed_manifold(one((v, t2)), 0)


# -- parity and surface membership on lattices ----------------------------------

def _check_lattice(mesh, inside_fn, on_fn, span):
    ds = one(mesh)
    n_in = n_on = 0
    for p in itertools.product(range(span), repeat=3):
        par, on = oracle.point_query(p, ds, 0)
        exp_on = on_fn(p)
        assert on == exp_on, p
        if not on:
            assert par == inside_fn(p), p
            n_in += par
        n_on += on
    return n_in, n_on


def test_parity_box_lattice():
    lo, hi = (2, 2, 2), (6, 6, 6)

    def inside(p):
        return all(lo[i] < p[i] < hi[i] for i in range(3))

    def on(p):
        return all(lo[i] <= p[i] <= hi[i] for i in range(3)) and not inside(p)
    assert _check_lattice(synth.box(lo, hi), inside, on, 9) == (27, 125 - 27)


def test_parity_octahedron_lattice():
    c, r = (4, 4, 4), 3

    def l1(p):
        return sum(abs(p[i] - c[i]) for i in range(3))
    n_in, n_on = _check_lattice(synth.octahedron(c, r), lambda p: l1(p) < r, lambda p: l1(p) == r, 9)
    assert n_in == 25 and n_on == 38


def _tet_planes(P):
    v, t = synth.tetra(*P)
    v = v.astype(np.int64)
    planes = []
    for f in t:
        a, b, c = (tuple(int(x) for x in v[i]) for i in f)
        n = np.cross(np.subtract(b, a), np.subtract(c, a)).astype(object)
        planes.append((n, a))
    return (v, t), planes


def test_parity_random_tetrahedra_lattice():
    rng = np.random.default_rng(5)
    done = tot_in = 0
    while done < 12:
        P = rng.integers(0, 7, size=(4, 3))
        M = np.array([P[1] - P[0], P[2] - P[0], P[3] - P[0]])
        if round(abs(np.linalg.det(M))) == 0:
            continue
        mesh, planes = _tet_planes(P)

        def side(p):
            return [int(np.dot(n, np.subtract(p, a))) for n, a in planes]

        def inside(p):
            return all(s < 0 for s in side(p))

        def on(p):
            s = side(p)
            return all(x <= 0 for x in s) and any(x == 0 for x in s)
        n_in, n_on = _check_lattice(mesh, inside, on, 7)
        assert n_on >= 4
        tot_in += n_in
        done += 1
    assert tot_in > 0


def _winding(p, V, F):
    """Generalised winding number (sum of signed solid angles / 4 pi)."""
    a = V[F[:, 0]] - p
    b = V[F[:, 1]] - p
    c = V[F[:, 2]] - p
    la, lb, lc = (np.linalg.norm(x, axis=1) for x in (a, b, c))
    num = np.einsum("ij,ij->i", a, np.cross(b, c))
    den = (la * lb * lc + np.einsum("ij,ij->i", a, b) * lc +
           np.einsum("ij,ij->i", a, c) * lb + np.einsum("ij,ij->i", b, c) * la)
    return 2 * np.arctan2(num, den).sum() / (4 * np.pi)


@pytest.mark.parametrize("kind", ["tube", "nucleus"])
def test_parity_matches_winding_number(kind):
    ds = synth.vessels(21, n=1, f_range=(3000, 3000)) if kind == "tube" else synth.nuclei(22, n=1, levels=(3,))
    v, t = ds.mesh(0)
    V = v.astype(np.float64)
    rng = np.random.default_rng(9)
    lo, hi = V.min(axis=0), V.max(axis=0)
    n_in = n_checked = 0
    # sample around the mesh; half of the points near random vertices
    for k in range(300):
        if k % 2:
            p = rng.integers(lo.astype(int), hi.astype(int) + 1)
        else:
            p = V[rng.integers(len(V))].astype(int) + rng.integers(-60, 61, size=3)
        w = _winding(p.astype(np.float64), V, t)
        if abs(w - round(w)) > 1e-3:
            continue
        par, on = oracle.point_query(p, ds, 0)
        if on:
            continue
        assert par == (int(round(w)) % 2 == 1), (p, w)
        n_in += par
        n_checked += 1
    assert n_checked > 200 and n_in > 10


def test_parity_convex_icosphere_halfspaces():
    A, _ = synth.tiny_spheres(3, n_a=1, n_b=1)
    v, t = A.mesh(0)
    vi = v.astype(np.int64)
    a = vi[t[:, 0]]
    n = np.cross(vi[t[:, 1]] - a, vi[t[:, 2]] - a)
    rng = np.random.default_rng(1)
    lo, hi = vi.min(axis=0), vi.max(axis=0)
    n_in = 0
    for _ in range(300):
        p = rng.integers(lo, hi + 1)
        s = np.einsum("ij,ij->i", n, p - a)
        if np.any(s == 0) and np.all(s <= 0):
            continue                    # on the surface
        par, on = oracle.point_query(p, A, 0)
        assert not on
        assert par == bool(np.all(s < 0))
        n_in += par
    assert n_in > 20


def test_rep_vertex_skips_vertices_on_surface():
    outer = synth.box((100, 100, 100), (120, 120, 120))
    inner = synth.box((100, 105, 105), (110, 115, 115))      # shares the face x = 100
    A, B = one(outer), one(inner)
    r = oracle.rep_vertex(B, 0, A, 0)
    v, _ = B.mesh(0)
    assert tuple(v[r]) == (110, 105, 105)
    same = one(outer)
    assert oracle.rep_vertex(same, 0, A, 0) == -1           # every vertex on the surface


# -- hand-built join cases (P1) -----------------------------------------------

def _case(ma, mb):
    return one(ma), one(mb)


@pytest.mark.parametrize("name", list(HAND))
def test_hand_built_cases(name):
    ma, mb, exp = HAND[name]
    A, B = _case(ma, mb)
    for tier in (1, 2):
        assert oracle.intersects(A, 0, B, 0, tier=tier) == exp
        assert oracle.intersects(B, 0, A, 0, tier=tier) == exp


def test_nested_spheres_contain_without_crossing():
    big = synth._placed_sphere(3, np.array([0.5, 0.5, 0.5]), 0.2, np.eye(3))
    small = synth._placed_sphere(2, np.array([0.52, 0.49, 0.5]), 0.05, np.eye(3))
    A, B = _case(big, small)
    assert not oracle.cross(A, 0, B, 0)
    assert oracle.inside(B, 0, A, 0) and not oracle.inside(A, 0, B, 0)
    assert oracle.intersects(A, 0, B, 0) and oracle.intersects(B, 0, A, 0)


# -- closed forms (P2) ----------------------------------------------------------

def _diag_degenerate(alo, ahi, blo, bhi):
    """Does an edge of box A cross a face of box B exactly on the face's
    triangulation diagonal (from (lo, lo) to (hi, hi) in face coordinates)?"""
    for ax in range(3):                          # A edges parallel to axis ax
        u, w = [d for d in range(3) if d != ax]
        for cu in (alo[u], ahi[u]):
            for cw in (alo[w], ahi[w]):
                if (cu - blo[u]) * (bhi[w] - blo[w]) == (cw - blo[w]) * (bhi[u] - blo[u]):
                    return True
    return False


def test_axis_aligned_boxes_closed_form():
    rng = np.random.default_rng(17)
    n_true = n = 0
    while n < 400:
        c = rng.choice(np.arange(1000, 1060), size=(3, 4), replace=False)
        alo, ahi = np.minimum(c[:, 0], c[:, 1]), np.maximum(c[:, 0], c[:, 1])
        blo, bhi = np.minimum(c[:, 2], c[:, 3]), np.maximum(c[:, 2], c[:, 3])
        if _diag_degenerate(alo, ahi, blo, bhi) or _diag_degenerate(blo, bhi, alo, ahi):
            continue
        exp = bool(np.all((alo < bhi) & (blo < ahi)))
        A, B = _case(synth.box(alo, ahi), synth.box(blo, bhi))
        assert oracle.intersects(A, 0, B, 0, tier=2) == exp, (alo, ahi, blo, bhi)
        n_true += exp
        n += 1
    assert 50 < n_true < 350


def test_spheres_closed_form():
    rng = np.random.default_rng(23)
    n_t = n_f = 0
    for _ in range(60):
        meshes, rho, R, cen = [], [], [], []
        radii = rng.uniform(0.01, 0.05, size=2)
        u = rng.normal(size=3)
        centres = [np.full(3, 0.5), 0.5 + u / np.linalg.norm(u) * rng.uniform(0, radii.sum() * 1.3)]
        for _k in range(2):
            r, c = radii[_k], centres[_k]
            v, t = synth._placed_sphere(2, c, r, synth.random_rotations(rng, 1)[0])
            vd = v.astype(np.float64)
            cc = c * QMAX
            a = vd[t[:, 0]]
            nrm = np.cross(vd[t[:, 1]] - a, vd[t[:, 2]] - a)
            nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
            rho.append(np.abs(np.einsum("ij,ij->i", nrm, a - cc)).min())
            R.append(np.linalg.norm(vd - cc, axis=1).max())
            meshes.append((v, t))
            cen.append(cc)
        d = np.linalg.norm(cen[0] - cen[1])
        A, B = _case(*meshes)
        res = oracle.intersects(A, 0, B, 0, tier=2)
        if d + 2 < rho[0] + rho[1] or d + min(R) + 2 < max(rho):
            assert res
            n_t += 1
        elif d > R[0] + R[1] + 2:
            assert not res
            n_f += 1
    assert n_t > 5 and n_f > 5


# -- invariants (P3) -----------------------------------------------------------

def _transform(ds, fn_v=None, perm=None):
    meshes = []
    for k in range(ds.nmesh):
        v, t = ds.mesh(k)
        v = v.astype(np.int64)
        if fn_v is not None:
            v = fn_v(v)
        if perm is not None:
            v, t = perm(v, t, k)
        meshes.append((v.astype(np.float32), t))
    return synth.concat(meshes)


@pytest.fixture(scope="module")
def tiny():
    A, B = synth.tiny_spheres(1001)
    cand = oracle.mbb_candidates(A, B)
    flags = oracle.join(A, B, cand, tier=2)
    return A, B, cand, flags


def test_tier1_equals_tier2_on_all_pairs(tiny):
    A, B, cand, flags = tiny
    allp = np.array([(i, j) for i in range(A.nmesh) for j in range(B.nmesh)], dtype=np.int32)
    f1 = oracle.join(A, B, allp, tier=1)
    f2 = oracle.join(A, B, allp, tier=2)
    assert (f1 == f2).all()
    got = allp[f1.astype(bool)]
    assert np.array_equal(got, oracle.join_all(A, B))
    assert 0 < flags.sum() < len(cand)


def test_swap_symmetry(tiny):
    A, B, cand, flags = tiny
    f = oracle.join(B, A, cand[:, ::-1], tier=2)
    assert (f == flags).all()


@pytest.mark.parametrize("name", ["translate", "permute axes", "reflect x", "relabel"])
def test_invariants(tiny, name):
    A, B, cand, flags = tiny
    rng = np.random.default_rng(31)
    if name == "translate":
        d = np.array([1234, -777, 4321])
        fn, perm = (lambda v: v + d), None
    elif name == "permute axes":
        fn, perm = (lambda v: v[:, [2, 0, 1]]), None
    elif name == "reflect x":
        fn, perm = (lambda v: np.stack([QMAX - v[:, 0], v[:, 1], v[:, 2]], axis=1)), None
    else:
        def perm(v, t, k):
            p = rng.permutation(len(v))
            inv = np.argsort(p)
            t2 = inv[t]
            t2 = t2[rng.permutation(len(t2))]
            sh = rng.integers(0, 3, size=len(t2))
            t2 = np.stack([np.roll(r, s) for r, s in zip(t2, sh)])
            flip = rng.random(len(t2)) < 0.3
            t2[flip] = t2[flip][:, [0, 2, 1]]
            return v[p], t2.astype(np.int32)
        fn = None
    A2, B2 = _transform(A, fn, perm), _transform(B, fn, perm)
    assert (oracle.join(A2, B2, cand, tier=2) == flags).all()


# -- exhaustive lattice placements vs the convex separating-axis test (P4) -------

def test_exhaustive_lattice_vs_sat():
    A, B, cand, meta = lattice_case_sets()
    f1 = oracle.join(A, B, cand, tier=1)
    f2 = oracle.join(A, B, cand, tier=2)
    assert (f1 == f2).all()
    exceptions = []
    for k, (i, j) in enumerate(cand):
        va, ta = A.mesh(int(i))
        vb, tb = B.mesh(int(j))
        sat = sat_overlap(va.astype(np.int64), ta, vb.astype(np.int64), tb)
        if f1[k]:
            assert sat, meta[k]                              # soundness, always
        elif sat:
            exceptions.append(k)
    # completeness: every miss is a degenerate contact that a generic
    # perturbation (scale by 64, shift B by (1, 2, 3)) turns into a detected hit
    for k in exceptions:
        i, j = cand[k]
        va, ta = A.mesh(int(i))
        vb, tb = B.mesh(int(j))
        Ap = synth.concat([(va * 64 - 1000, ta)])
        Bp = synth.concat([(vb * 64 - 1000 + np.array([1, 2, 3], np.float32), tb)])
        assert sat_overlap(Ap.xyz.astype(np.int64), ta, Bp.xyz.astype(np.int64), tb)
        assert oracle.intersects(Ap, 0, Bp, 0), meta[k]
    # 161 of the 3087 placements overlap; 40 are found and the other 121 are
    # aligned lattice contacts, all of them degenerate by the check above
    n_hit = int(f1.sum())
    assert n_hit == 40 and len(exceptions) == 121


def _golden_contacts():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "lattice_contacts.txt")
    out = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        na, nb, dx, dy, dz, v = line.split()
        out.append((na, nb, int(dx), int(dy), int(dz), int(v)))
    return out


def test_lattice_contacts_golden():
    """The stored set of overlapping lattice placements and the strict
    predicate's verdict on each (written by tests/golden/make_lattice_contacts.py
    from the oracle and the exact separating-axis test) is reproduced."""
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_lattice_contacts
    gold = _golden_contacts()
    assert make_lattice_contacts.rows() == gold
    assert sum(r[5] for r in gold) == 40 and len(gold) == 161
