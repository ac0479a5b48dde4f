"""The allocation-free join (pj_join_intersects_noalloc) through the C ABI,
against the oracle and the regular entry point, on two calls in a row.

That entry point is for callers that cannot call cudaMalloc: loops that must
not stall on the allocator's implicit device synchronisation, or programs
whose device memory belongs to another allocator or budget.  They pass every
buffer themselves; the kernels' small scratch is a fixed device array inside
the library, shared by every call.  Results are pair sets, compared exactly.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu


def _noalloc(ctx, ha, hb, cand, torch):
    n = len(cand)
    d_cand = torch.from_numpy(np.ascontiguousarray(cand, dtype=np.int32)).cuda()
    # outputs start as garbage: the call must overwrite everything it reports
    d_flags = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    d_pairs = torch.full((n, 2), -5, dtype=torch.int32, device="cuda")
    d_count = torch.full((1,), -9, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    pierce.pj_join_intersects_noalloc(ctx.h, ha, hb, d_cand, d_flags, d_pairs, d_count,
                                      stream=stream)
    torch.cuda.synchronize()
    k = int(d_count.item())
    return k, d_pairs[:max(k, 0)].cpu().numpy(), d_flags.cpu().numpy()


def test_noalloc_join_matches_oracle_and_regular_join_on_two_calls():
    torch = pytest.importorskip("torch")
    A, B = synth.tiny_spheres(1002)
    every = np.array([(i, j) for i in range(A.nmesh) for j in range(B.nmesh)], np.int32)
    # first call: every pair; second call: a different, shorter list in
    # reverse order, so stale scratch from the first call would show
    lists = (every, every[: len(every) // 2][::-1].copy())
    truth = [oracle.join(A, B, c, tier=2) for c in lists]
    with pierce.Context(0) as ctx:
        ha, hb = ctx.load(A), ctx.load(B)
        ctx.build(ha, 4, 4)
        ctx.build(hb, 4, 4)
        for cand, exp in zip(lists, truth):
            ref, _ = ctx.join(ha, hb, cand=cand)
            k, pairs, flags = _noalloc(ctx, ha, hb, cand, torch)
            assert np.array_equal(flags, exp)                 # the oracle, every candidate
            assert k == len(ref) == int(exp.sum()) > 0
            assert np.array_equal(pairs, ref)
            assert np.array_equal(pairs, cand[exp.astype(bool)])


def test_noalloc_join_reports_a_bad_id_then_recovers():
    torch = pytest.importorskip("torch")
    A, B = synth.tiny_spheres(1003)
    cand = oracle.mbb_candidates(A, B)
    exp = oracle.join(A, B, cand, tier=2)
    bad = cand.copy()
    bad[3] = (A.nmesh, 0)                       # idA out of range
    with pierce.Context(0) as ctx:
        ha, hb = ctx.load(A), ctx.load(B)
        ctx.build(ha, 4, 4)
        ctx.build(hb, 4, 4)
        k, _, flags = _noalloc(ctx, ha, hb, bad, torch)
        assert k == -1
        assert flags[3] == 0                    # the bad candidate is skipped
        keep = np.arange(len(cand)) != 3
        assert np.array_equal(flags[keep], exp[keep])
        # the next call on the same scratch starts clean
        k, pairs, flags = _noalloc(ctx, ha, hb, cand, torch)
        assert k == int(exp.sum())
        assert np.array_equal(pairs, cand[exp.astype(bool)])


def test_noalloc_join_rejects_too_many_candidates_and_mixed_bvh_shapes():
    torch = pytest.importorskip("torch")
    A, B = synth.tiny_spheres(5, n_a=2, n_b=2)
    with pierce.Context(0) as ctx:
        h, hb = ctx.load(A), ctx.load(B)
        ctx.build(h, 4, 4)
        ctx.build(hb, 4, 4)
        small = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
        flags = torch.zeros(2, dtype=torch.uint8, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        lib = pierce.load()
        rc = lib.pj_join_intersects_noalloc(
            ctx.h, h, h, small.data_ptr(), 16777217, flags.data_ptr(), small.data_ptr(),
            count.data_ptr(), None)
        assert rc == 1                                # PJ_ERR_INVALID_ARG, nothing launched
        assert "16777216" in pierce.pj_last_error(ctx.h)
        # B's last build has another shape than A's: refused, nothing queued
        ctx.build(hb, 8, 2)
        rc = lib.pj_join_intersects_noalloc(
            ctx.h, h, hb, small.data_ptr(), 2, flags.data_ptr(), small.data_ptr(),
            count.data_ptr(), None)
        assert rc == 1
        assert "width or leaf size" in pierce.pj_last_error(ctx.h)
        assert ctypes.sizeof(ctypes.c_int64) == 8
