"""The allocation-free join (pj_join_intersects_noalloc) against the regular
entry point, through the C ABI, on two calls in a row.

That entry point is for callers that cannot call cudaMalloc: code running
while a stream is captured into a CUDA graph, loops that must not stall on the
allocator's implicit device synchronisation, or programs whose device memory
belongs to another allocator.  They pass every buffer themselves; the kernels'
small scratch is a fixed device array inside the library.  Results are pair
sets, compared exactly.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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


def test_noalloc_join_matches_regular_join_on_two_calls():
    torch = pytest.importorskip("torch")
    A, B = synth.tiny_spheres(1002)
    with pierce.Context(0) as ctx:
        ha, hb = ctx.load(A), ctx.load(B)
        ctx.build(ha, 4, 4)
        ctx.build(hb, 4, 4)
        every = np.array([(i, j) for i in range(A.nmesh) for j in range(B.nmesh)], np.int32)
        # first call: every pair; second call: a different, shorter list in
        # reverse order, so stale scratch from the first call would show
        for cand in (every, every[: len(every) // 2][::-1].copy()):
            ref, _ = ctx.join(ha, hb, cand=cand)
            k, pairs, flags = _noalloc(ctx, ha, hb, cand, torch)
            assert k == len(ref) > 0
            assert np.array_equal(pairs, ref)
            assert np.array_equal(cand[flags.astype(bool)], ref)
            assert set(np.unique(flags)) <= {0, 1}


def test_noalloc_join_rejects_too_many_candidates():
    torch = pytest.importorskip("torch")
    A, _ = synth.tiny_spheres(5, n_a=2, n_b=1)
    with pierce.Context(0) as ctx:
        h = ctx.load(A)
        ctx.build(h, 4, 4)
        small = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
        flags = torch.zeros(2, dtype=torch.uint8, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = pierce.load().pj_join_intersects_noalloc(
            ctx.h, h, h, small.data_ptr(), 16777217, flags.data_ptr(), small.data_ptr(),
            count.data_ptr(), None)
        assert rc == 1                                # PJ_ERR_INVALID_ARG, nothing launched
        assert "16777216" in pierce.pj_last_error(ctx.h)
        assert ctypes.sizeof(ctypes.c_int64) == 8
