import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(ROOT)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# one line per oracle reference computed in this session, printed at the end
_NOTES = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libpierce.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # tests that need a GPU are skipped cleanly when none is present
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    for line in _NOTES:
        terminalreporter.write_line(line)


def oracle_flags(name, dsA, dsB, cand, offsets=None):
    """The oracle's verdict on every candidate, refined on every host core;
    the core count and the time go to the session summary."""
    import oracle
    cores = oracle.host_cores()
    t0 = time.time()
    flags = oracle.join(dsA, dsB, cand, tier=2, offsets=offsets, threads=cores)
    _NOTES.append("oracle reference %s: %d candidates, %d intersecting, %.1f s on %d host cores"
                  % (name, len(cand), int(flags.sum()), time.time() - t0, cores))
    return flags


@pytest.fixture(scope="session")
def pathology_truth():
    """The full pathology workload (10,000 nuclei x 500 vessels, seed 2001),
    its bounding-box candidates and the oracle's flag for every candidate.
    Computed once per session: the pathology parity and serving tests share
    it."""
    import oracle
    from paper_2609_24513_gb300 import synth
    A, B = synth.pathology(2001)
    cand = oracle.mbb_candidates(A, B)
    flags = oracle_flags("pathology 10,000 x 500", A, B, cand)
    return A, B, cand, flags
