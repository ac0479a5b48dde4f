"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Pair sets are compared exactly (integer results: no tolerance).  Inputs are
seeded synthetic meshes: the tiny-spheres workload (full pair set), the
hand-built cases, exhaustive lattice placements, instanced (translated)
candidates, self joins, and error paths.  The full-size pathology workload is
in test_gpu_pathology.py.
"""
import os

import numpy as np
import pytest

import oracle
from cases import HAND, lattice_case_sets
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pierce.Context(0)
    yield c
    c.close()


def _load(ctx, ds, shapes=((4, 4),), device=False):
    h = ctx.load(ds, device_tensors=device)
    for W, L in shapes:
        ctx.build(h, W, L)
    return h


@pytest.fixture(scope="module")
def tiny(ctx):
    out = []
    for seed in (1001, 1002, 1003):
        A, B = synth.tiny_spheres(seed)
        exp = oracle.join_all(A, B, tier=2)
        ha = _load(ctx, A, shapes=[(w, l) for w in (2, 4, 8) for l in (1, 2, 4, 8)])
        hb = _load(ctx, B, shapes=[(w, l) for w in (2, 4, 8) for l in (1, 2, 4, 8)], device=True)
        out.append((A, B, ha, hb, exp))
    return out


@pytest.mark.parametrize("W", [2, 4, 8])
@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_tiny_spheres_all_bvh_shapes(ctx, tiny, W, L):
    for A, B, ha, hb, exp in tiny:
        got, info = ctx.join(ha, hb, width=W, leaf_size=L)
        assert info["n_candidates"] == len(oracle.mbb_candidates(A, B))
        assert np.array_equal(got, exp)
        got, _ = ctx.join(ha, hb, width=W, leaf_size=L, wave_levels=pierce.PJ_FRONT_STREAM)
        assert np.array_equal(got, exp), "stream"


@pytest.mark.parametrize("mode", ["exact", "warps2", "warps4", "per_pair", "explicit", "graph",
                                  "spill1", "spill3", "nospill", "nowave", "wave1", "wave9",
                                  "stream", "stream_exact", "stream_graph"])
def test_tiny_spheres_modes(ctx, tiny, mode):
    for A, B, ha, hb, exp in tiny:
        kw = {}
        cand = None
        if mode == "exact":
            kw["leaf_mode"] = pierce.PJ_LEAF_EXACT
        elif mode == "warps2":
            kw["warps_per_pair"] = 2
        elif mode == "warps4":
            kw["warps_per_pair"] = 4
        elif mode == "per_pair":
            kw["launch_mode"] = pierce.PJ_LAUNCH_PER_PAIR
        elif mode == "explicit":
            # every pair, not only bounding-box candidates, in reverse order
            cand = np.array([(i, j) for i in range(A.nmesh) for j in range(B.nmesh)][::-1],
                            dtype=np.int32)
        elif mode == "graph":
            kw["use_graph"] = True
        elif mode == "spill1":
            kw["spill_budget"] = 1      # every pair continues in the later passes
            kw["use_graph"] = True
        elif mode == "spill3":
            kw["spill_budget"] = 3
        elif mode == "nospill":
            kw["spill_budget"] = -1
        elif mode == "nowave":
            kw["wave_levels"] = -1
        elif mode == "wave1":
            kw["wave_levels"] = 1
            kw["spill_budget"] = 1
        elif mode == "wave9":
            kw["wave_levels"] = 9
            kw["use_graph"] = True
        elif mode == "stream":
            kw["wave_levels"] = pierce.PJ_FRONT_STREAM
        elif mode == "stream_exact":
            kw["wave_levels"] = pierce.PJ_FRONT_STREAM
            kw["leaf_mode"] = pierce.PJ_LEAF_EXACT
        elif mode == "stream_graph":
            kw["wave_levels"] = pierce.PJ_FRONT_STREAM
            kw["use_graph"] = True
        got, _ = ctx.join(ha, hb, cand=cand, width=4, leaf_size=4, **kw)
        if mode == "explicit":
            got = got[np.lexsort((got[:, 1], got[:, 0]))]
        assert np.array_equal(got, exp), mode


def test_repeated_joins_identical(ctx, tiny):
    A, B, ha, hb, exp = tiny[0]
    for _ in range(5):
        got, _ = ctx.join(ha, hb, width=8, leaf_size=2, use_graph=True)
        assert np.array_equal(got, exp)


@pytest.mark.parametrize("name", list(HAND))
def test_hand_built_cases(ctx, name):
    ma, mb, exp = HAND[name]
    A, B = synth.concat([ma]), synth.concat([mb])
    ha, hb = _load(ctx, A, ((4, 4), (2, 1))), _load(ctx, B, ((4, 4), (2, 1)))
    cand = np.array([[0, 0]], dtype=np.int32)
    for W, L in ((4, 4), (2, 1)):
        for mode in (pierce.PJ_LEAF_FILTERED, pierce.PJ_LEAF_EXACT):
            got, _ = ctx.join(ha, hb, cand=cand, width=W, leaf_size=L, leaf_mode=mode)
            assert (len(got) == 1) == exp
            got, _ = ctx.join(hb, ha, cand=cand, width=W, leaf_size=L, leaf_mode=mode)
            assert (len(got) == 1) == exp


def test_nested_spheres(ctx):
    big = synth._placed_sphere(3, np.array([0.5, 0.5, 0.5]), 0.2, np.eye(3))
    small = synth._placed_sphere(2, np.array([0.52, 0.49, 0.5]), 0.05, np.eye(3))
    A, B = synth.concat([big]), synth.concat([small])
    ha, hb = _load(ctx, A), _load(ctx, B)
    got, _ = ctx.join(ha, hb)
    assert got.tolist() == [[0, 0]]
    got, _ = ctx.join(hb, ha)
    assert got.tolist() == [[0, 0]]


def test_exhaustive_lattice(ctx):
    A, B, cand, meta = lattice_case_sets()
    exp = oracle.join(A, B, cand, tier=1)
    # the stored verdicts on the overlapping placements agree with the oracle
    gold = {}
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                  "lattice_contacts.txt")):
        if not line.startswith("#") and line.strip():
            na, nb, dx, dy, dz, v = line.split()
            gold[(na, nb, (int(dx), int(dy), int(dz)))] = int(v)
    keyed = {(na, nb, tuple(int(x) for x in o)): int(exp[k]) for k, (na, nb, o) in enumerate(meta)}
    assert all(keyed[key] == v for key, v in gold.items()) and len(gold) == 161
    ha, hb = _load(ctx, A, ((4, 4), (2, 1), (8, 8))), _load(ctx, B, ((4, 4), (2, 1), (8, 8)))
    for W, L in ((4, 4), (2, 1), (8, 8)):
        for mode, wave in ((pierce.PJ_LEAF_FILTERED, 0), (pierce.PJ_LEAF_EXACT, -1)):
            res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, cand=cand, width=W, leaf_size=L,
                                               leaf_mode=mode, wave_levels=wave, out_host=True)
            got = pierce.pairs_to_numpy(res)
            pierce.pj_free_pairs(ctx.h, res)
            assert np.array_equal(got, cand[exp.astype(bool)]), (W, L, mode)


def test_instanced_candidates(ctx):
    """Per-candidate translations of B: many placements share one mesh."""
    A, B = synth.tiny_spheres(77, n_a=4, n_b=4)
    rng = np.random.default_rng(5)
    cand, offs = [], []
    for _ in range(300):
        i, j = rng.integers(0, 4, size=2)
        va, _ = A.mesh(int(i))
        vb, _ = B.mesh(int(j))
        # shift B_j so that its centre lands near A_i's centre (kept on the grid)
        d = np.rint(va.mean(axis=0) - vb.mean(axis=0) + rng.normal(0, 30000, size=3))
        d = np.clip(d, -vb.min(axis=0), synth.QMAX - vb.max(axis=0))
        cand.append((i, j))
        offs.append(d)
    cand = np.array(cand, dtype=np.int32)
    offs = np.array(offs, dtype=np.int32)
    exp = oracle.join(A, B, cand, tier=2, offsets=offs)
    assert 20 < exp.sum() < 280
    ha, hb = _load(ctx, A), _load(ctx, B)
    res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, cand=cand, cand_offsets=offs, out_host=True)
    got = pierce.pairs_to_numpy(res)
    pierce.pj_free_pairs(ctx.h, res)
    assert np.array_equal(got, cand[exp.astype(bool)])


def test_self_join(ctx):
    A, _ = synth.tiny_spheres(2024, n_a=40, n_b=1)
    exp = oracle.join_all(A, A, self_join=True)
    h = _load(ctx, A)
    got, info = ctx.join(h, h, self_join=True)
    assert np.array_equal(got, exp)
    assert np.all(got[:, 0] < got[:, 1])


def test_empty_and_no_overlap(ctx):
    A = synth.concat([synth.box((10, 10, 10), (20, 20, 20))])
    B = synth.concat([synth.box((100, 100, 100), (120, 120, 120))])
    ha, hb = _load(ctx, A), _load(ctx, B)
    got, info = ctx.join(ha, hb)
    assert info["n_candidates"] == 0 and len(got) == 0
    got, info = ctx.join(ha, hb, cand=np.zeros((0, 2), np.int32))
    assert len(got) == 0
    got, info = ctx.join(ha, hb, cand=np.array([[0, 0]], np.int32))
    assert len(got) == 0


def test_load_rejects_bad_input(ctx):
    v, t = synth.box((10, 10, 10), (20, 20, 20))
    bad = v.copy()
    bad[3, 1] += 0.5
    with pytest.raises(pierce.PierceError) as e:
        ctx.load(synth.concat([(bad, t)]))
    assert e.value.code == 2
    with pytest.raises(pierce.PierceError) as e:
        ctx.load(synth.concat([(v, t[:-1])]))          # open mesh
    assert e.value.code == 3
    neg = v.copy()
    neg[0, 0] = -1
    with pytest.raises(pierce.PierceError):
        ctx.load(synth.concat([(neg, t)]))
    # the context is still usable
    h = _load(ctx, synth.concat([(v, t)]))
    with pytest.raises(pierce.PierceError) as e:
        ctx.join(h, h, cand=np.array([[0, 5]], np.int32))
    assert e.value.code == 1
    got, _ = ctx.join(h, h, cand=np.array([[0, 0]], np.int32))
    assert len(got) == 0                            # identical meshes: false


def test_mesh_data_and_bvh_structure(ctx):
    A, _ = synth.tiny_spheres(31, n_a=6, n_b=1)
    extra = synth.nuclei(32, n=2, levels=(3,))
    ds = synth.concat([A.mesh(k) for k in range(A.nmesh)] + [extra.mesh(k) for k in range(2)])
    h = _load(ctx, ds, ((2, 1), (4, 4), (8, 8), (4, 1)))
    aabb, lex, own = pierce.pj_export_mesh_data(ctx.h, h, ds.nmesh, len(ds.tris))
    for k in range(ds.nmesh):
        v, t = ds.mesh(k)
        assert np.array_equal(aabb[k], np.concatenate([v.min(axis=0), v.max(axis=0)]))
        order = np.lexsort((v[:, 2], v[:, 1], v[:, 0]))
        assert lex[k] == order[0]
        o = own[ds.toff[k]:ds.toff[k + 1]]
        edges = []
        for f, bits in zip(t, o):
            for e in range(3):
                if bits >> e & 1:
                    a, b = f[e], f[(e + 1) % 3]
                    edges.append((min(a, b), max(a, b)))
        assert len(edges) == len(set(edges)) == len(t) * 3 // 2
    info = pierce.pj_dataset_info_get(ctx.h, h)
    assert info["n_edges"] == len(ds.tris) * 3 // 2
    for W, L in ((2, 1), (4, 4), (8, 8), (4, 1)):
        nodes, roots, order = pierce.pj_export_bvh(ctx.h, h, W, L, len(ds.tris), ds.nmesh)
        f = nodes.view(np.float32)
        own_lo, own_hi = f[:, 0, 0:3], f[:, 0, 3:6]
        lo = f[:, 1:, 0:3].transpose(0, 2, 1)          # [node, axis, child]
        hi = f[:, 1:, 3:6].transpose(0, 2, 1)
        child = nodes[:, 1:, 6].view(np.uint32)
        live = child != 0xFFFFFFFF
        # a node's own box is the union of its live children's boxes
        for n in range(len(nodes)):
            m = live[n]
            assert np.array_equal(own_lo[n], lo[n][:, m].min(axis=1))
            assert np.array_equal(own_hi[n], hi[n][:, m].max(axis=1))
        for k in range(ds.nmesh):
            v, t = ds.mesh(k)
            ordk = order[ds.toff[k]:ds.toff[k + 1]]
            assert sorted(ordk.tolist()) == list(range(len(t)))
            seen = np.zeros(len(t), dtype=int)
            stack = [(int(roots[k]), 1)]
            while stack:
                n, depth = stack.pop()
                for s in range(W):
                    c = int(child[n, s])
                    if c == 0xFFFFFFFF:
                        assert np.all(lo[n, :, s] > hi[n, :, s])
                        continue
                    blo, bhi = lo[n, :, s], hi[n, :, s]
                    if c & 0x80000000:
                        first, cnt = (c >> 3) & 0x0FFFFFFF, (c & 7) + 1
                        assert cnt <= L
                        for p in range(first, first + cnt):
                            tri = ordk[p]
                            seen[tri] += 1
                            pts = v[t[tri]]
                            assert np.all(pts.min(axis=0) >= blo) and np.all(pts.max(axis=0) <= bhi)
                    else:
                        clo, chi = lo[c], hi[c]
                        live = child[c] != 0xFFFFFFFF
                        assert np.all(clo[:, live] >= blo[:, None]) and np.all(chi[:, live] <= bhi[:, None])
                        stack.append((c, depth + 1))
            assert np.all(seen == 1)


def test_segtri_batch_matches_oracle(ctx):
    import torch
    rng = np.random.default_rng(8)
    groups = []
    groups.append(rng.integers(0, 4, size=(4000, 5, 3)))                 # many ties
    groups.append(rng.integers(0, synth.QMAX + 1, size=(2000, 5, 3)))    # full range
    # near-degenerate: segment through the triangle's plane close to an edge
    near = []
    for _ in range(2000):
        a = rng.integers(1000, 250000, size=3)
        b = a + rng.integers(-3000, 3000, size=3)
        c = a + rng.integers(-3000, 3000, size=3)
        m = (a + b) // 2 + rng.integers(-2, 3, size=3)
        n = np.cross(b - a, c - a)
        n = n / max(np.abs(n).max(), 1)
        p = np.rint(m - 50 * n + rng.integers(-1, 2, size=3))
        q = np.rint(m + 50 * n + rng.integers(-1, 2, size=3))
        near.append(np.clip(np.stack([p, q, a, b, c]), 0, synth.QMAX))
    groups.append(np.array(near, dtype=np.int64))
    # exact zeros at full-range coordinates, which the filter cannot certify
    # by magnitude: all five points (or p or q with the triangle) in one
    # axis-aligned plane, and edges starting at a triangle vertex
    zeros = []
    for i in range(3000):
        X = rng.integers(0, synth.QMAX + 1, size=(5, 3))
        k = int(rng.integers(0, 3))
        kind = i % 3
        if kind == 0:
            X[:, k] = X[0, k]                       # everything in the plane x_k = const
        elif kind == 1:
            X[[0, 2, 3, 4], k] = X[2, k]            # p and the triangle in the plane
            X[1] = X[0] + rng.integers(-5000, 5000, size=3)
        else:
            X[0] = X[2 + int(rng.integers(0, 3))]   # p is a triangle vertex
        zeros.append(np.clip(X, 0, synth.QMAX))
    groups.append(np.array(zeros, dtype=np.int64))
    P = np.concatenate(groups).astype(np.int64)
    exp = np.array([oracle.segtri_strict(*x) for x in P], dtype=np.uint8)
    pq = torch.from_numpy(P[:, :2].reshape(-1, 6).astype(np.float32)).cuda()
    abc = torch.from_numpy(P[:, 2:].reshape(-1, 9).astype(np.float32)).cuda()
    for mode in (pierce.PJ_LEAF_FILTERED, pierce.PJ_LEAF_STATIC, pierce.PJ_LEAF_EXACT):
        res = torch.zeros(len(P), dtype=torch.uint8, device="cuda")
        nfb = pierce.pj_segtri_batch(ctx.h, pq, abc, res, mode=mode)
        assert np.array_equal(res.cpu().numpy(), exp), mode
        if mode != pierce.PJ_LEAF_EXACT:
            assert 0 < nfb < len(P)
    assert exp.sum() > 100


def test_counters_move(ctx, tiny):
    A, B, ha, hb, exp = tiny[0]
    ctx.reset_counters()
    ctx.join(ha, hb, width=4, leaf_size=4)
    c = ctx.counters()
    assert c["pairs_refined"] == len(oracle.mbb_candidates(A, B))
    assert c["pairs_hit"] == len(exp)
    assert c["segtri_tests"] > 0 and c["node_pairs"] > 0 and c["bytes_fetched"] > 0


def test_parity_rays_along_every_axis(ctx):
    """Containment is decided by a parity ray along the axis and direction
    that leaves the target's box soonest; the result must equal the oracle's
    +z parity for every choice.  Small tetrahedra sit inside and outside a
    noisy sphere and a straight vertical tube, near each face of their boxes."""
    rng = np.random.default_rng(12)
    sphere = synth._placed_sphere(3, np.array([0.5, 0.5, 0.5]), 0.1, np.eye(3),
                                  noise=lambda u: 0.05 * np.sin(3 * u[:, 0]))
    z = np.linspace(0.2, 0.8, 64)
    curve = np.stack([np.full_like(z, 0.3), np.full_like(z, 0.7), z], axis=1)
    V, T = synth._tube(curve, 0.03, 40)
    tube = (synth.quantize(V), T)
    A = synth.concat([sphere, tube])
    smalls, cand = [], []
    for target, (v, _) in enumerate([sphere, tube]):
        lo, hi = v.min(axis=0), v.max(axis=0)
        for _ in range(150):
            p = lo + rng.uniform(0.02, 0.98, size=3) * (hi - lo)
            k = rng.integers(3)
            p[k] = (lo[k] + rng.uniform(0.0, 0.08) * (hi[k] - lo[k])) if rng.random() < 0.5 else \
                (hi[k] - rng.uniform(0.0, 0.08) * (hi[k] - lo[k]))
            d = rng.integers(40, 400, size=(3, 3))
            t = synth.tetra(p, p + [d[0, 0], 0, 0], p + [0, d[1, 1], 0], p + [0, 0, d[2, 2]])
            smalls.append((np.rint(t[0]).astype(np.float32), t[1]))
            cand.append((target, len(smalls) - 1))
    B = synth.concat(smalls)
    cand = np.array(cand, dtype=np.int32)
    exp = oracle.join(A, B, cand, tier=2)
    assert 30 < exp.sum() < len(cand) - 30
    ha, hb = _load(ctx, A, ((4, 4), (8, 2))), _load(ctx, B, ((4, 4), (8, 2)))
    for W, L in ((4, 4), (8, 2)):
        for wave in (0, -1):
            got, _ = ctx.join(ha, hb, cand=cand, width=W, leaf_size=L, wave_levels=wave)
            assert np.array_equal(got, cand[exp.astype(bool)]), (W, L, wave)


def test_autotune_picks_a_measured_configuration(ctx):
    A, B = synth.tiny_spheres(1003)
    exp = oracle.join_all(A, B, tier=2)
    ha, hb = ctx.load(A), ctx.load(B)
    best, table = pierce.pj_autotune(ctx.h, ha, hb, widths=(2, 4), leaf_sizes=(2, 4),
                                     warps=(1, 2), wave_levels=(0, -1), repeats=2, seed=3)
    assert len(table) == 2 * 2 * 2 * 2
    fastest = min(table, key=lambda r: r["ms"])
    assert (best["width"], best["leaf_size"], best["warps_per_pair"], best["wave_levels"]) == \
        (fastest["width"], fastest["leaf_size"], fastest["warps_per_pair"], fastest["wave_levels"])
    # only the winning BVH shape is kept, and it is the dataset default now
    info = pierce.pj_dataset_info_get(ctx.h, ha)
    assert (info["bvh_width"], info["bvh_leaf_size"]) == (best["width"], best["leaf_size"])
    got, _ = ctx.join(ha, hb, **{k: best[k] for k in ("width", "leaf_size", "warps_per_pair",
                                                      "wave_levels")})
    assert np.array_equal(got, exp)
    with pytest.raises(pierce.PierceError):
        pierce.pj_autotune(ctx.h, ha, hb, widths=(3,))


def _bipyramid(n, c, r, h, phase=0.0):
    """Closed double cone over an n-gon: every triangle contains one of the
    two apexes, so the boxes of any two triangles of one half meet."""
    a = 2 * np.pi * (np.arange(n) + phase) / n
    ring = np.stack([c[0] + r * np.cos(a), c[1] + r * np.sin(a), np.full(n, c[2])], 1)
    V = np.vstack([ring, [c[0], c[1], c[2] + h], [c[0], c[1], c[2] - h]])
    F = []
    for i in range(n):
        j = (i + 1) % n
        F += [(n, i, j), (n + 1, j, i)]
    return synth.quantize(V), np.array(F, dtype=np.int32)


@pytest.mark.parametrize("W,L", [(8, 1), (4, 1), (2, 1), (4, 4)])
def test_dense_overlap_stack_spills(ctx, W, L):
    """Node pairs that all overlap: a bipyramid's triangles all touch an
    apex, so against itself (or a twisted or shifted copy) nearly every
    child pair of a (node, node) step survives.  A streaming warp's task
    stack then overflows and hands its older half to the later passes.  The
    identical copy does not intersect (no strict crossing, every vertex on
    the other surface); the twisted and shifted ones do.  Oracle-checked."""
    m = _bipyramid(1000, (0.5, 0.5, 0.5), 0.2, 0.2)
    tw = _bipyramid(1000, (0.5, 0.5, 0.5), 0.2, 0.2, phase=0.5)
    sh = synth.translate(m, (1.0, 0.0, 0.0))
    A, B = synth.concat([m, m, m]), synth.concat([m, tw, sh])
    cand = np.array([[0, 0], [1, 1], [2, 2]], dtype=np.int32)
    exp = oracle.join(A, B, cand, tier=2)
    assert exp.tolist() == [0, 1, 1]
    ha, hb = _load(ctx, A, ((W, L),)), _load(ctx, B, ((W, L),))
    ctx.reset_counters()
    got, _ = ctx.join(ha, hb, cand=cand, width=W, leaf_size=L, wave_levels=pierce.PJ_FRONT_STREAM)
    assert got.tolist() == [[1, 1], [2, 2]]
    assert ctx.counters()["tasks_spilled"] > 0
    for kw in (dict(), dict(spill_budget=-1), dict(spill_budget=1), dict(use_graph=True),
               dict(wave_levels=-1), dict(leaf_mode=pierce.PJ_LEAF_EXACT),
               dict(wave_levels=pierce.PJ_FRONT_STREAM, use_graph=True),
               dict(wave_levels=pierce.PJ_FRONT_STREAM, leaf_mode=pierce.PJ_LEAF_EXACT)):
        got, _ = ctx.join(ha, hb, cand=cand, width=W, leaf_size=L, **kw)
        assert got.tolist() == [[1, 1], [2, 2]], kw


def test_stream_wait_timeout_falls_back(ctx, tiny):
    """Every bounded wait of the streaming kernel limited to one poll: idle
    warps give up at once, the kernel records the error word, and the host
    redoes the join by plain depth-first traversal -- the same pairs, more
    kernel launches.  (The wait runs out on purpose; nothing faults.)"""
    A, B, ha, hb, exp = tiny[0]
    before = ctx.counters()["kernel_launches"]
    got, _ = ctx.join(ha, hb, width=4, leaf_size=4, wave_levels=pierce.PJ_FRONT_STREAM)
    normal = ctx.counters()["kernel_launches"] - before
    before = ctx.counters()["kernel_launches"]
    got2, _ = ctx.join(ha, hb, width=4, leaf_size=4, wave_levels=pierce.PJ_FRONT_STREAM,
                       wait_polls=1)
    redone = ctx.counters()["kernel_launches"] - before
    assert np.array_equal(got, exp) and np.array_equal(got2, exp)
    assert redone > normal
    # the queue is clean again afterwards: the next join is exact and fast-path
    got3, _ = ctx.join(ha, hb, width=4, leaf_size=4, wave_levels=pierce.PJ_FRONT_STREAM)
    assert np.array_equal(got3, exp)
