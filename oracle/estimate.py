"""Selectivity estimate of a join (paper Sec. 3.5) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module; the product library never calls it
and shares no code with it.  It is the plain, slow statement of the estimator
the paper uses to size its result hashmap, in the paper's order and notation:

  1. overlay both datasets with a regular grid of G x G x G cells;
  2. per cell and dataset k: N_k, the number of objects whose axis-aligned
     box touches the cell; S_k, the mean over those objects of the mean box
     side (width, height, depth averaged); VolRatio_k, the mean over them of
     mesh volume / box volume;
  3. interaction volume V_int = (S_1 + S_2 + eps)^3 (the Minkowski sum of
     two cubes of the mean sides, eps = 1e-3), P_base = V_int / V_cell;
  4. shape factor F_shape = (sqrt(VolRatio_1 VolRatio_2))^gamma, gamma = 0.8;
  5. P = min(P_base F_shape, 1); the cell's expected pairs E_i = N_1 N_2 P;
  6. E_final = sum over cells of E_i; hashmap slots = E_final / 0.5.

Readings where the paper is silent (each listed in the design notes):
  - lengths are measured in units of the grid's full extent, coordinates
    divided by 2^18 - 1, so that eps = 1e-3 is small against the objects;
  - the grid covers the bounding box of both datasets together, split into
    G^3 equal cells (G is a parameter; the paper does not give one);
  - "touches" is closed: a box whose face lies on a cell boundary touches the
    cells on both sides;
  - a mesh's volume is |sum over triangles of det[a, b, c]| / 6 (divergence
    theorem, float64), so orientation does not matter.

Parity status: pinned by ``tests/test_oracle_estimate.py`` (brute-force cell
counts, exact box volumes, convex-hull volumes, the Minkowski-sum probability
checked by sampling, the estimate against the true number of box-overlapping
pairs for uniform cubes, symmetry and scaling identities).
"""
from __future__ import annotations

import numpy as np

QMAX = (1 << 18) - 1
EPS = 1e-3
GAMMA = 0.8
LOAD_FACTOR = 0.5


def mesh_volume(v: np.ndarray, t: np.ndarray) -> float:
    """|sum over triangles of det[a, b, c]| / 6 for a closed mesh (float64;
    vertices shifted to the first one so that the terms stay small)."""
    p = np.asarray(v, np.float64)
    p = p - p[0]
    a, b, c = p[t[:, 0]], p[t[:, 1]], p[t[:, 2]]
    return abs(float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum())) / 6.0


def object_stats(ds):
    """Per mesh: box lo, hi (unit coordinates), mean side, volume ratio."""
    n = ds.nmesh
    lo, hi = np.zeros((n, 3)), np.zeros((n, 3))
    side, ratio = np.zeros(n), np.zeros(n)
    for k in range(n):
        v, t = ds.mesh(k)
        vd = np.asarray(v, np.float64)
        lo[k], hi[k] = vd.min(axis=0) / QMAX, vd.max(axis=0) / QMAX
        ext = hi[k] - lo[k]
        side[k] = ext.mean()
        box_vol = float(np.prod(ext))
        ratio[k] = mesh_volume(v, t) / QMAX ** 3 / box_vol if box_vol > 0 else 0.0
    return lo, hi, side, ratio


def cell_stats(stats, g0, cw, G):
    """N, sum of mean sides and sum of volume ratios per cell (G^3 arrays)."""
    lo, hi, side, ratio = stats
    N, S, R = np.zeros((G, G, G)), np.zeros((G, G, G)), np.zeros((G, G, G))
    for k in range(len(side)):
        i0 = np.clip(np.floor((lo[k] - g0) / cw).astype(int), 0, G - 1)
        i1 = np.clip(np.floor((hi[k] - g0) / cw).astype(int), 0, G - 1)
        sl = tuple(slice(i0[d], i1[d] + 1) for d in range(3))
        N[sl] += 1
        S[sl] += side[k]
        R[sl] += ratio[k]
    return N, S, R


def grid_of(stats1, stats2, G):
    lo = np.minimum(stats1[0].min(axis=0), stats2[0].min(axis=0))
    hi = np.maximum(stats1[1].max(axis=0), stats2[1].max(axis=0))
    cw = np.maximum(hi - lo, 1.0 / QMAX) / G
    return lo, cw


def estimate(ds1, ds2, G: int = 16, eps: float = EPS, gamma: float = GAMMA):
    """E_final for the join of ds1 and ds2 over a G^3 grid; also returns the
    per-cell E_i (G^3) and the hashmap slot count E_final / 0.5."""
    s1, s2 = object_stats(ds1), object_stats(ds2)
    g0, cw = grid_of(s1, s2, G)
    N1, S1, R1 = cell_stats(s1, g0, cw, G)
    N2, S2, R2 = cell_stats(s2, g0, cw, G)
    E = np.zeros((G, G, G))
    occ = (N1 > 0) & (N2 > 0)
    v_cell = float(np.prod(cw))
    m1, m2 = S1[occ] / N1[occ], S2[occ] / N2[occ]
    r1, r2 = R1[occ] / N1[occ], R2[occ] / N2[occ]
    p_base = (m1 + m2 + eps) ** 3 / v_cell
    f_shape = np.sqrt(r1 * r2) ** gamma
    P = np.minimum(p_base * f_shape, 1.0)
    E[occ] = N1[occ] * N2[occ] * P
    e_final = float(E.sum())
    return e_final, E, e_final / LOAD_FACTOR
