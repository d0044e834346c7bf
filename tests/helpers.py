"""Shared helpers for the GPU parity tests: tolerances and oracle-side checks.

Tolerances (float32 matrix profile against the float64 oracle):
  |P_gpu - P_ref| <= 1e-3 * max(P_ref, d_floor),  d_floor = 1e-2 * sqrt(2m)
The floor covers exact repeats (P_ref = 0), where float32 data still leave a
residual distance.  Nearest-neighbour indices must match, except where the
GPU's neighbour is a tie: its oracle distance equals P_ref within the same
tolerance.  The float64 path uses 1e-9 relative.
"""
import math

import numpy as np

from oracle import tsk_oracle as o

MP_REL_TOL = 1e-3
FP64_REL_TOL = 1e-9


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
    assert worst <= rel, f"max rel error {worst:.3g} > {rel} at row {rows[ok][int(np.argmax(err))]}"
    # indices: equal, or a tie at the same distance
    diff = np.where(ok & (Ig != I_ref))[0]
    Z, _, _, _ = o.znorm_windows(x, m)
    for r in diff:
        i, j = int(rows[r]), int(Ig[r])
        assert j >= 0 and abs(i - j) >= excl, (i, j)
        dij = float(np.sqrt(((Z[i] - Z[j]) ** 2).sum()))
        assert abs(dij - P_ref[r]) <= rel * max(P_ref[r], fl), (i, j, dij, P_ref[r])
    return worst


def check_discords(res_gpu, res_ref, A_ref=None, tie_rel=1e-6):
    """Discord lists (idx, grp, score, nn): indices equal or tied within tie_rel."""
    for (ig, gg, sg, ng), (ir, gr, sr, nr) in zip(res_gpu, res_ref):
        if ig != ir:
            assert A_ref is not None and A_ref[ig] >= (1 - tie_rel) * A_ref[ir], (ig, ir)
