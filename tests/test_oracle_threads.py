"""The oracle's sharded driver (``oracle.join(..., threads=n)``) returns the
same flags and counters as one single-threaded call, with and without
per-candidate translations and for every join predicate."""
import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import synth


@pytest.mark.parametrize("threads", [2, 3, None])
def test_sharded_join_equals_single_call(threads):
    A, B = synth.tiny_spheres(1003)
    cand = oracle.mbb_candidates(A, B)
    f1, s1 = oracle.join(A, B, cand, stats=True)
    fn, sn = oracle.join(A, B, cand, stats=True, threads=threads)
    assert np.array_equal(f1, fn) and np.array_equal(s1, sn)
    for pred in oracle.PREDICATES:
        assert np.array_equal(oracle.join(A, B, cand, predicate=pred),
                              oracle.join(A, B, cand, predicate=pred, threads=threads))


def test_sharded_join_with_translations():
    A, B, cand, off, _ = synth.batching(3001, n_pairs=120, n_templates=20)
    f1 = oracle.join(A, B, cand, offsets=off)
    f4 = oracle.join(A, B, cand, offsets=off, threads=4)
    assert np.array_equal(f1, f4) and 0 < f1.sum() < len(f1)
    assert len(oracle.join(A, B, cand[:0], offsets=off[:0], threads=4)) == 0
    with pytest.raises(oracle.OracleError):
        oracle.join(A, B, cand, offsets=off[:-1], threads=4)
