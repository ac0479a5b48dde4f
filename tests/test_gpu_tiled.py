"""Out-of-core join by grid tiling (pj_join_tiled, paper Sec. 3.6): host
datasets, a coarse grid, every mesh copied to the cells its box touches,
cells joined one by one, each pair kept in its reference point's cell.  The
result must equal the oracle's pair set whatever the grid: tiny spheres at
1 to 5 cells per axis, a predicate other than intersects, an urban self join,
and the full pathology join under a device budget that forces tiling."""
import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pierce.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("grid", [1, 2, 3, 5])
def test_tiny_spheres_any_grid(ctx, grid):
    A, B = synth.tiny_spheres(1003)
    want = oracle.join_all(A, B)
    got, st = pierce.pj_join_tiled(ctx.h, A, B, grid=grid)
    assert np.array_equal(got, want)
    assert st["grid"] == grid and st["cells_joined"] >= 1
    if grid > 1:
        assert st["mesh_copies"] > A.nmesh           # boxes straddling cells are copied
        assert st["pairs_in_cells"] >= len(got)


def test_overlap_predicate_and_self_join(ctx):
    A, B = synth.tiny_spheres(1001)
    cand = oracle.mbb_candidates(A, B)
    want = cand[oracle.join(A, B, cand, predicate="overlap").astype(bool)]
    got, _ = pierce.pj_join_tiled(ctx.h, A, B, grid=3, predicate="overlap")
    assert np.array_equal(got, want)
    U = synth.urban(5001, n_buildings=1500, n_parts=150)
    want_u = oracle.join_all(U, U, self_join=True)
    got_u, st = pierce.pj_join_tiled(ctx.h, U, self_join=True, grid=4)
    assert np.array_equal(got_u, want_u)
    assert np.all(got_u[:, 0] < got_u[:, 1]) and st["cells_joined"] > 1


def test_budget_chooses_the_grid_and_refuses_too_small(ctx):
    A, B = synth.tiny_spheres(1002)
    want = oracle.join_all(A, B)
    got, st = pierce.pj_join_tiled(ctx.h, A, B, device_budget=1_600_000)
    assert np.array_equal(got, want)
    assert st["grid"] > 1 and st["max_cell_bytes"] <= 1_600_000
    with pytest.raises(pierce.PierceError) as e:
        pierce.pj_join_tiled(ctx.h, A, B, device_budget=1000)
    assert e.value.code == 4                          # PJ_ERR_NO_MEMORY


def test_pathology_full_under_a_budget(ctx, pathology_truth):
    A, B, cand, flags = pathology_truth
    got, st = pierce.pj_join_tiled(ctx.h, A, B, device_budget=6 << 30)
    assert np.array_equal(got, cand[flags.astype(bool)])
    assert st["grid"] > 1
    print("tiled pathology join: grid %d, %d cells, %d mesh copies, largest cell %.2f GB, "
          "%.0f ms (device %.0f, gather %.0f overlapped)"
          % (st["grid"], st["cells_joined"], st["mesh_copies"], st["max_cell_bytes"] / 1e9,
             st["ms_total"], st["ms_device"], st["ms_gather"]))
