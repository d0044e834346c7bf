"""Shared helpers for the GPU parity tests: tolerances and oracle-side checks.

Tolerance (float32 matrix profile against the float64 oracle, Def. 3 / Def. 6):
  |P_gpu - P_ref| <= 1e-3 * max(P_ref, d_floor),  d_floor = 1e-2 * sqrt(2m).
The floor covers exact repeats (P_ref = 0), whose float32 distance cannot be
told apart from ~sqrt(2m * 2^-24).  Nearest-neighbour indices must match,
except where the GPU's neighbour is a tie: its oracle distance meets the same
bar against P_ref.  The float64 path uses 1e-9 relative.
"""
import math

import numpy as np

from oracle import tsk_oracle as o

MP_REL_TOL = 1e-3
FP64_REL_TOL = 1e-9


def within_mp_tol(P_gpu, P_ref, m, rel=MP_REL_TOL, floor=None):
    """Elementwise |P_gpu - P_ref| <= rel * max(P_ref, floor) (see the module docstring)."""
    P_gpu = np.asarray(P_gpu, dtype=np.float64)
    P_ref = np.asarray(P_ref, dtype=np.float64)
    fl = d_floor(m) if floor is None else floor
    return np.abs(P_gpu - P_ref) <= rel * np.maximum(P_ref, fl)


def d_floor(m: int) -> float:
    return 1e-2 * math.sqrt(2 * m)


def check_profile(x, m, excl, P_gpu, I_gpu, rows=None, rel=MP_REL_TOL, floor=None):
    """Compare a GPU profile (at `rows`, default all) with the oracle; return the max error ratio."""
    x = np.asarray(x, dtype=np.float64)
    l = len(x) - m + 1
    rows = np.arange(l) if rows is None else np.asarray(rows)
    P_ref, I_ref = o.mp_rows(x, m, excl, rows)
    Pg = np.asarray(P_gpu, dtype=np.float64)[rows]
    Ig = np.asarray(I_gpu)[rows]
    fl = d_floor(m) if floor is None else floor
    inf_ref = np.isinf(P_ref)
    assert np.array_equal(inf_ref, np.isinf(Pg)), "rows without admissible neighbour differ"
    assert np.all(Ig[inf_ref] == -1)
    ok = ~inf_ref
    scale = np.maximum(P_ref[ok], fl)
    err = np.abs(Pg[ok] - P_ref[ok]) / scale
    worst = float(err.max()) if err.size else 0.0
    good = within_mp_tol(Pg[ok], P_ref[ok], m, rel, fl)
    assert good.all(), f"max rel error {worst:.3g} > {rel} at row {rows[ok][int(np.argmin(good))]}"
    # indices: equal, or a tie at the same distance
    diff = np.where(ok & (Ig != I_ref))[0]
    Z, _, _, _ = o.znorm_windows(x, m)
    for r in diff:
        i, j = int(rows[r]), int(Ig[r])
        assert j >= 0 and abs(i - j) >= excl, (i, j)
        dij = float(np.sqrt(((Z[i] - Z[j]) ** 2).sum()))
        assert within_mp_tol(dij, P_ref[r], m, rel, fl) and abs(dij - Pg[r]) <= 1e-4 * max(dij, fl), \
            (i, j, dij, P_ref[r])
    return worst


def check_discords(res_gpu, res_ref, A_ref=None, tie_rel=1e-6):
    """Discord lists (idx, grp, score, nn): indices equal or tied within tie_rel."""
    for (ig, gg, sg, ng), (ir, gr, sr, nr) in zip(res_gpu, res_ref):
        if ig != ir:
            assert A_ref is not None and A_ref[ig] >= (1 - tie_rel) * A_ref[ir], (ig, ir)
