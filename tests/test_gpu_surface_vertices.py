"""Containment when the first vertices of a mesh lie on the other mesh's
surface (Sec. 3.3: the representative vertex is the lexicographically
smallest one not on the other surface).  A finely tessellated box touches a
larger one along a whole face, from inside or from outside, so that its 121
face vertices -- the first ones in lexicographic order -- all lie on the
larger box's surface and the search must pass several blocks of 32 vertices
before one decides.  CPU: the oracle against the geometry; GPU: every
predicate, both roles, on the streaming and per-warp front ends, against the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import pierce, synth


def fine_box(lo, hi, n):
    """The box [lo, hi] with every face cut into an n x n grid of squares
    (two triangles each), outward-facing; (hi - lo) divisible by n."""
    lo, hi = np.asarray(lo, np.int64), np.asarray(hi, np.int64)
    assert np.all((hi - lo) % n == 0)
    step = (hi - lo) // n
    ids, verts, tris = {}, [], []

    def vid(g):
        g = tuple(g)
        if g not in ids:
            ids[g] = len(verts)
            verts.append(lo + step * np.asarray(g))
        return ids[g]

    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for s in (0, 1):
            for u in range(n):
                for w in range(n):
                    def P(uu, ww):
                        g = [0, 0, 0]
                        g[a], g[b], g[c] = s * n, uu, ww
                        return vid(g)
                    p00, p10, p11, p01 = P(u, w), P(u + 1, w), P(u + 1, w + 1), P(u, w + 1)
                    if s == 1:   # normal +a: (b, c) counter-clockwise seen from +a
                        tris += [[p00, p10, p11], [p00, p11, p01]]
                    else:
                        tris += [[p00, p11, p10], [p00, p01, p11]]
    return np.asarray(verts, np.float32), np.asarray(tris, np.int32)


BIG = fine_box((100, 100, 100), (196, 196, 196), 24)
INSIDE = fine_box((100, 120, 120), (140, 160, 160), 10)     # min-x face on BIG's min-x face
OUTSIDE = fine_box((196, 120, 120), (236, 160, 160), 10)    # min-x face on BIG's max-x face
PREDS = ("intersects", "contains", "within")


def _sets():
    T = synth.concat([BIG])
    Q = synth.concat([INSIDE, OUTSIDE])
    cand = np.array([[0, 0], [0, 1]], np.int32)
    return T, Q, cand


def test_oracle_follows_the_geometry():
    T, Q, cand = _sets()
    # INSIDE lies in BIG (their surfaces only touch): intersecting, contained;
    # OUTSIDE only touches BIG's face: neither
    assert oracle.join(T, Q, cand, predicate="intersects").tolist() == [1, 0]
    assert oracle.join(T, Q, cand, predicate="contains").tolist() == [1, 0]
    assert oracle.join(T, Q, cand, predicate="within").tolist() == [0, 0]
    assert oracle.join(Q, T, cand[:, ::-1].copy(), predicate="within").tolist() == [1, 0]
    # the case it is built for: the first 121 vertices of INSIDE in
    # lexicographic order lie on BIG's surface
    v = INSIDE[0].astype(np.int64)
    first = v[np.lexsort((v[:, 2], v[:, 1], v[:, 0]))][:121]
    assert np.all(first[:, 0] == 100)


MODES = {
    "stream_l2": dict(width=4, leaf_size=2, wave_levels=pierce.PJ_FRONT_STREAM),
    "stream_l4": dict(width=4, leaf_size=4, wave_levels=pierce.PJ_FRONT_STREAM),
    "warps": dict(width=4, leaf_size=4, wave_levels=pierce.PJ_FRONT_NONE, warps_per_pair=2),
    "w8_stream": dict(width=8, leaf_size=2, wave_levels=pierce.PJ_FRONT_STREAM),
}


@pytest.mark.gpu
@pytest.mark.parametrize("mode", sorted(MODES))
def test_every_predicate_both_roles(mode):
    T, Q, cand = _sets()
    kw = dict(MODES[mode])
    W, L = kw.pop("width"), kw.pop("leaf_size")
    ctx = pierce.Context(0)
    try:
        ht, hq = ctx.load(T), ctx.load(Q)
        ctx.build(ht, W, L)
        ctx.build(hq, W, L)
        for (ha, hb, A, B, c) in ((ht, hq, T, Q, cand), (hq, ht, Q, T, cand[:, ::-1].copy())):
            for p in PREDS:
                want = oracle.join(A, B, c, predicate=p)
                res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, cand=c, width=W, leaf_size=L,
                                                   keep_flags=True, out_host=True, predicate=p,
                                                   **kw)
                got = pierce.device_to_numpy(res.flags, int(res.n_candidates), np.uint8)
                pierce.pj_free_pairs(ctx.h, res)
                assert np.array_equal(got, want), (mode, p)
    finally:
        ctx.close()
