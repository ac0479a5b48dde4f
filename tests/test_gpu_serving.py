"""Serving through pj_submit / pj_poll.

A window query's answer is the set of intersecting pairs among the meshes
whose closed boxes meet the window.  It must not depend on how the query was
scheduled: alone, batched with many others, split into several batches by a
small admission budget, or submitted from several threads at once.  Every
answer is checked against the oracle: on the full pathology workload the
oracle's verdict on all of its bounding-box candidates, restricted to the
window, is the expected answer.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu


def _restrict(pairs, boxA, boxB, lo, hi):
    """Pairs of `pairs` whose A and B meshes both have boxes meeting [lo, hi]."""
    def meets(box):
        return np.all((box[:, :3] <= hi) & (lo <= box[:, 3:]), axis=1)
    ma, mb = meets(boxA), meets(boxB)
    if len(pairs) == 0:
        return pairs.reshape(0, 2)
    keep = ma[pairs[:, 0]] & mb[pairs[:, 1]]
    return pairs[keep]


def _alone(ctx, ha, hb, lo, hi, self_join=False):
    out = []
    for k in range(len(lo)):
        t = ctx.submit(ha, hb, lo[k], hi[k], self_join)
        out.append(ctx.poll(t, wait=True))
    return out


def _mixed(ctx, ha, hb, lo, hi, self_join=False):
    tickets = [ctx.submit(ha, hb, lo[k], hi[k], self_join) for k in range(len(lo))]
    return [ctx.poll(t, wait=True) for t in tickets]


def test_small_case_matches_oracle_alone_and_mixed():
    A, B = synth.tiny_spheres(4101, n_a=30, n_b=30)
    truth = oracle.join_all(A, B)
    bA, bB = synth.mesh_boxes(A), synth.mesh_boxes(B)
    lo, hi = synth.windows(4102, 24, half_range=(1 << 14, 1 << 17))
    with pierce.Context(0) as ctx:
        ha, hb = ctx.load(A), ctx.load(B)
        ctx.build(ha, 4, 4)
        ctx.build(hb, 4, 4)
        alone = _alone(ctx, ha, hb, lo, hi)
        mixed = _mixed(ctx, ha, hb, lo, hi)
    nonempty = 0
    for k in range(len(lo)):
        want = _restrict(truth, bA, bB, lo[k], hi[k])
        assert np.array_equal(alone[k][0], want), k
        assert np.array_equal(mixed[k][0], want), k
        nonempty += len(want) > 0
        st = mixed[k][1]
        assert st["n_pairs"] == len(want)
        assert st["t_submit"] <= st["t_admit"] <= st["t_launch"] <= st["t_done"]
    assert nonempty >= 4


@pytest.fixture(scope="module")
def pathology_served(pathology_truth):
    """The full pathology datasets resident with cached BVHs, and the
    oracle's pair set over all of their candidates."""
    A, B, cand, flags = pathology_truth
    ctx = pierce.Context(0, serve_streams=4)
    ha, hb = ctx.load(A), ctx.load(B)
    ctx.build(ha, 4, 4)
    ctx.build(hb, 4, 4)
    full = cand[flags.astype(bool)]
    bA, bB = synth.mesh_boxes(A), synth.mesh_boxes(B)
    yield A, B, ctx, ha, hb, full, bA, bB
    ctx.close()


def test_alone_equals_mixed_on_pathology(pathology_served):
    A, B, ctx, ha, hb, full, bA, bB = pathology_served
    lo, hi = synth.serving_windows(4202, 96)
    alone = _alone(ctx, ha, hb, lo, hi)
    mixed = _mixed(ctx, ha, hb, lo, hi)
    batched = 0
    for k in range(len(lo)):
        want = _restrict(full, bA, bB, lo[k], hi[k])
        assert np.array_equal(alone[k][0], want), k
        assert np.array_equal(mixed[k][0], want), k
        assert alone[k][1]["n_candidates"] == mixed[k][1]["n_candidates"]
        batched += mixed[k][1]["batch_queries"] > 1
    assert batched > 0                          # the mix did form batches
    assert sum(len(a[0]) for a in alone) > 50


def test_small_budget_splits_batches_and_keeps_answers(pathology_served):
    A, B, _, _, _, full, bA, bB = pathology_served
    lo, hi = synth.serving_windows(4203, 40, frac_range=(1e-3, 0.05))
    with pierce.Context(0, serve_streams=2) as probe:
        pa, pb = probe.load(A), probe.load(B)
        probe.build(pa, 4, 4)
        probe.build(pb, 4, 4)
        sizes = [probe.poll(probe.submit(pa, pb, lo[k], hi[k]))[1]["device_bytes"]
                 for k in range(len(lo))]
    budget = 2 * max(sizes)
    with pierce.Context(0, serve_streams=3, budget_bytes=budget) as ctx:
        ha, hb = ctx.load(A), ctx.load(B)
        ctx.build(ha, 4, 4)
        ctx.build(hb, 4, 4)
        got = _mixed(ctx, ha, hb, lo, hi)
        # a query larger than the whole budget is refused at submission
        with pytest.raises(pierce.PierceError) as e:
            ctx.submit(ha, hb, (0, 0, 0), (synth.QMAX,) * 3)
        assert e.value.code == 5
    per_batch = {}
    for k in range(len(lo)):
        assert np.array_equal(got[k][0], _restrict(full, bA, bB, lo[k], hi[k])), k
        st = got[k][1]
        per_batch[st["batch_id"]] = per_batch.get(st["batch_id"], 0) + st["device_bytes"]
    assert max(per_batch.values()) <= budget
    assert len(per_batch) > 1


def test_threads_submit_and_poll_concurrently(pathology_served):
    A, B, ctx, ha, hb, full, bA, bB = pathology_served
    lo, hi = synth.serving_windows(4204, 64)
    results = {}
    errors = []

    def client(ids):
        try:
            ts = [(k, ctx.submit(ha, hb, lo[k], hi[k])) for k in ids]
            for k, t in ts:
                results[k] = ctx.poll(t, wait=True)[0]
        except Exception as exc:  # surfaced below
            errors.append(exc)

    threads = [threading.Thread(target=client, args=(list(range(c, 64, 4)),)) for c in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors
    for k in range(64):
        assert np.array_equal(results[k], _restrict(full, bA, bB, lo[k], hi[k])), k


def test_self_join_window_and_nonblocking_poll():
    A, _ = synth.tiny_spheres(4301, n_a=40, n_b=1)
    truth = oracle.join_all(A, A, self_join=True)
    bA = synth.mesh_boxes(A)
    lo, hi = synth.windows(4302, 8, half_range=(1 << 15, 1 << 17))
    with pierce.Context(0) as ctx:
        h = ctx.load(A)
        ctx.build(h, 4, 4)
        tickets = [ctx.submit(h, h, lo[k], hi[k], self_join=True) for k in range(len(lo))]
        got = {}
        for _ in range(200000):
            for k, t in enumerate(tickets):
                if k not in got:
                    r = ctx.poll(t, wait=False)
                    if r is not None:
                        got[k] = r[0]
            if len(got) == len(tickets):
                break
        assert len(got) == len(tickets)
    for k in range(len(lo)):
        assert np.array_equal(got[k], _restrict(truth, bA, bA, lo[k], hi[k])), k


def test_dataset_in_use_cannot_be_freed():
    A, B = synth.tiny_spheres(4401, n_a=10, n_b=10)
    with pierce.Context(0) as ctx:
        ha, hb = ctx.load(A), ctx.load(B)
        ctx.build(ha, 4, 4)
        ctx.build(hb, 4, 4)
        t = ctx.submit(ha, hb, (0, 0, 0), (synth.QMAX,) * 3)
        with pytest.raises(pierce.PierceError) as e:
            pierce.pj_free_dataset(ctx.h, ha)
        assert e.value.code == 5
        ctx.poll(t, wait=True)
        pierce.pj_free_dataset(ctx.h, ha)       # polled: free now succeeds
        with pytest.raises(pierce.PierceError):
            ctx.poll(t, wait=True)              # the ticket was released
