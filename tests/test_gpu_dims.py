"""GPU parity of dimension detection (Alg. 3) and the refinement profile against the oracle.

The discords fed to both sides are the oracle's own (Alg. 2 on the oracle's
sketch) or seeded positions; every per-dimension score, neighbour and chosen
dimension is compared.
"""
import math

import numpy as np
import pytest

from oracle import tsk_oracle as o
from paper_2311_03393_gb300 import synth

from helpers import MP_REL_TOL, d_floor, within_mp_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_03393_gb300 import build
    build.build()
    import paper_2311_03393_gb300 as t
    return t


def _check_dims(series, R, queries, m, excl, got, rel=MP_REL_TOL, train=None):
    """Compare GPU outputs for one series with the oracle's Alg. 3 on the same (i*, g*) queries."""
    T = np.asarray(series, dtype=np.float64)
    Tn = T if train is None else np.asarray(train, dtype=np.float64)
    fl = d_floor(m)
    valid = [(i, g) for (i, g) in queries if i >= 0]
    picks, scores, nns = o.dimension_detection(T, R, valid, m, excl, T_train=train)
    q = 0
    for r, (i, g) in enumerate(queries):
        if i < 0:
            assert got["dim"][r] == -1 and math.isnan(got["score"][r]) and got["nn"][r] == -1
            continue
        ref_s, ref_nn = scores[q], nns[q]
        gs = got["scores"][r]
        member = ~np.isnan(ref_s)
        assert np.array_equal(member, ~np.isnan(gs)), (r, member, gs)
        for j in np.flatnonzero(member):
            if np.isinf(ref_s[j]):
                assert np.isinf(gs[j])
                continue
            assert within_mp_tol(gs[j], ref_s[j], m, rel), (r, j, gs[j], ref_s[j])
        j_ref, s_ref, nn_ref = picks[q]
        j_gpu = int(got["dim"][r])
        if j_ref < 0:
            assert j_gpu == -1
        elif j_gpu != j_ref:  # a tie within the tolerance
            assert j_gpu >= 0 and member[j_gpu]
            assert within_mp_tol(ref_s[j_gpu], s_ref, m, rel), (r, j_gpu, j_ref)
        elif math.isinf(s_ref):
            assert math.isinf(got["score"][r]) and got["nn"][r] == -1
        else:
            assert within_mp_tol(got["score"][r], s_ref, m, rel)
            nn_gpu = int(got["nn"][r])
            if nn_gpu != nn_ref:  # the neighbour must be an equally near window
                Zq, _, _, _ = o.znorm_windows(T[j_ref], m)
                Zt, _, _, _ = o.znorm_windows(Tn[j_ref], m)
                dd = float(np.linalg.norm(Zq[i] - Zt[nn_gpu])) if nn_gpu >= 0 else math.inf
                assert (train is not None or abs(i - nn_gpu) >= excl) and within_mp_tol(dd, s_ref, m, rel)
        q += 1


def _run(tsk, Ts, R, queries, m, excl, dtype=torch.float32, gather=False, train=None):
    """Ts: list of (d, n_s) arrays; queries: per series list of K (i*, g*); train: list like Ts."""
    d = Ts[0].shape[0]
    T = torch.cat([torch.as_tensor(np.ascontiguousarray(t)).reshape(-1) for t in Ts]).to("cuda", dtype)
    lens = [t.shape[1] for t in Ts]
    idx = torch.tensor([[i for i, _ in qs] for qs in queries], dtype=torch.int32, device="cuda")
    grp = torch.tensor([[g for _, g in qs] for qs in queries], dtype=torch.int32, device="cuda")
    Tt, tl = None, None
    if train is not None:
        Tt = torch.cat([torch.as_tensor(np.ascontiguousarray(t)).reshape(-1) for t in train]).to("cuda", dtype)
        tl = [t.shape[1] for t in train]
    res = tsk.dimension_detection(T, torch.as_tensor(R, dtype=torch.float32).cuda(), lens, d, m, idx, grp, excl,
                                  all_scores=True, gather=gather, T_train=Tt, train_len=tl)
    tsk.sync()
    return T, lens, {k: v.cpu().numpy() for k, v in res.items()}


def test_planted_dimension_matches_the_oracle_pipeline(tsk):
    """Alg. 2 on the oracle's sketch gives (i*, g*); both sides then run Alg. 3."""
    d, n, m, k, p = 6, 2600, 40, 3, 1500
    rng = np.random.default_rng(5)
    t = np.arange(n)
    T = np.stack([rng.uniform(0.5, 2.0) * np.sin(2 * np.pi * t / q + rng.uniform(0, 2 * np.pi))
                  for q in [10, 20, 25, 50, 20, 10]])
    T[4, p:p + m] = rng.normal(0.0, 1.0, m)
    excl = synth.default_excl(m)
    R = synth.count_sketch_R(d, k, seed=8)
    res, _, _, _ = o.sketched_discords(T, R, m, excl, 2, m)
    queries = [(i, g) for (i, g, _, _) in res]
    for dtype in (torch.float32, torch.float64):
        _, _, got = _run(tsk, [T], R, [queries], m, excl, dtype)
        _check_dims(T, R, queries, m, excl, {key: v[0] for key, v in got.items()})
        assert got["dim"][0][0] == 4


@pytest.mark.parametrize("kind", ["gaussian", "count"])
def test_ragged_batch_every_score(tsk, kind):
    """Several chunks and ragged tails, queries near both ends, an empty slot, float32 input."""
    rng = np.random.default_rng(21 if kind == "gaussian" else 22)
    d, k, m, excl = 12, 4, 50, 13
    lens = [3000, 1100, 2300, 64]
    Ts = [np.cumsum(rng.normal(size=(d, n)), axis=1).astype(np.float32) for n in lens]
    R = synth.gaussian_R(d, k, 3) if kind == "gaussian" else synth.count_sketch_R(d, k, 4)
    K = 4
    queries = []
    for n in lens:
        l = n - m + 1
        qs = [(0, 0), (l - 1, 1 % k), (int(rng.integers(0, l)), int(rng.integers(0, k))), (-1, 0)]
        queries.append(qs[:K])
    _, _, got = _run(tsk, Ts, R, queries, m, excl)
    for s, T in enumerate(Ts):
        _check_dims(T, R, queries[s], m, excl, {key: v[s] for key, v in got.items()})


@pytest.mark.parametrize("m", [40, 512, 600])
def test_more_discords_than_a_batch_holds(tsk, m):
    """20 discords per series: the scan stages at most 16 per batch (fewer for long windows: 14 at
    m = 512 and 600), so a second batch follows the first on every chunk.  A stream with a large
    offset and a small spread; float32 and float64."""
    rng = np.random.default_rng(24 + m)
    d, k, n = 4, 2, 4200
    excl = synth.default_excl(m)
    T = np.cumsum(rng.normal(size=(d, n)), axis=1)
    T[2] = 1.0e4 + 1e-2 * T[2]
    R = synth.gaussian_R(d, k, 6)
    l = n - m + 1
    queries = [(int(i), int(rng.integers(0, k))) for i in rng.integers(0, l, 20)]
    for dtype in (torch.float32, torch.float64):
        Ts = T.astype(np.float32) if dtype == torch.float32 else T
        _, _, got = _run(tsk, [Ts], R, [queries], m, excl, dtype)
        _check_dims(Ts, R, queries, m, excl, {key: v[0] for key, v in got.items()})


def test_constant_windows_empty_group_and_no_neighbour(tsk):
    n, m, excl = 1500, 32, 8
    rng = np.random.default_rng(7)
    sq = np.where((np.arange(n) // 300) % 2 == 0, 0.0, 1.0)          # long constant runs
    steps = np.repeat(rng.integers(0, 3, n // 100 + 1), 100)[:n] * 1.0
    T = np.stack([sq, np.cumsum(rng.normal(size=n)), steps, sq * 5.0 + 2.0]).astype(np.float32)
    R = np.zeros((4, 3), dtype=np.float32)
    R[[0, 2, 3], 0] = 1.0      # constant-heavy streams
    R[1, 1] = -1.0             # one random walk
    queries = [(10, 0), (320, 0), (700, 1), (5, 2)]                  # group 2 is empty
    _, _, got = _run(tsk, [T], R, [queries], m, excl)
    _check_dims(T, R, queries, m, excl, {key: v[0] for key, v in got.items()})
    # a series too short for any admissible neighbour: every score is +inf
    Ts = np.cumsum(rng.normal(size=(2, 40)), axis=1).astype(np.float32)
    _, _, got = _run(tsk, [Ts], np.ones((2, 1), np.float32), [[(3, 0)]], 32, 8)
    assert got["dim"][0][0] == 0 and np.isinf(got["score"][0][0]) and got["nn"][0][0] == -1


def test_gather_and_refinement_profile(tsk):
    d, m, excl = 5, 30, 8
    rng = np.random.default_rng(31)
    Ts = [np.cumsum(rng.normal(size=(d, n)), axis=1) for n in (1800, 900)]
    R = synth.gaussian_R(d, 2, 5)
    queries = [[(400, 0), (1200, 1)], [(100, 1), (-1, 0)]]
    T, lens, got = _run(tsk, Ts, R, queries, m, excl, dtype=torch.float64, gather=True)
    sel = got["T_sel"]
    off = 0
    for s, Tn in enumerate(Ts):
        n = Tn.shape[1]
        for r in range(2):
            j = got["dim"][s][r]
            want = Tn[j] if j >= 0 else np.zeros(n)
            np.testing.assert_array_equal(sel[off:off + n], want)
            off += n
    ref = tsk.refine_dimensions(torch.as_tensor(sel).cuda(), lens, 2, m, excl, mp_precision="fp64")
    tsk.sync()
    for s, Tn in enumerate(Ts):
        for r in range(2):
            j = got["dim"][s][r]
            if j < 0:
                continue
            i, score, nn = o.refine_dimension(Tn, j, m, excl)
            assert int(ref["idx"][s, r]) == i and int(ref["nn"][s, r]) == nn
            assert abs(float(ref["score"][s, r]) - score) <= 1e-9 * score
            assert score >= got["score"][s][r] * (1 - 1e-9)


def test_full_size_water_dimensions(tsk):
    """d=51, n=50000, m=100: the planted windows and seeded windows, all 8 sketch groups (Gaussian R)."""
    wl = synth.workload(2)
    T = wl.series[0]
    d, n = T.shape
    m, k = wl.m, wl.k
    excl = synth.default_excl(m)
    rng = np.random.default_rng(77)
    queries = [(p, int(rng.integers(0, k))) for (_, _, p) in wl.planted]
    queries += [(int(rng.integers(0, n - m + 1)), int(rng.integers(0, k))) for _ in range(3)]
    _, _, got = _run(tsk, [T], wl.R, [queries], m, excl)
    _check_dims(T, wl.R, queries, m, excl, {key: v[0] for key, v in got.items()})


def test_train_test_form_every_score_and_the_ab_refinement(tsk):
    """Alg. 3 as printed: test windows scored against every window of the training streams."""
    rng = np.random.default_rng(71)
    d, k, m = 8, 3, 40
    test_lens, train_lens = [2500, 900], [1800, 3100]
    test = [np.cumsum(rng.normal(size=(d, n)), axis=1) for n in test_lens]
    train = [np.cumsum(rng.normal(size=(d, n)), axis=1) for n in train_lens]
    R = synth.gaussian_R(d, k, 9)
    queries = [[(int(rng.integers(0, n - m + 1)), int(rng.integers(0, k))) for _ in range(3)] for n in test_lens]
    for dtype in (torch.float32, torch.float64):
        _, _, got = _run(tsk, test, R, queries, m, 0, dtype=dtype, gather=(dtype == torch.float64), train=train)
        for s in range(2):
            _check_dims(test[s], R, queries[s], m, 0, {key: v[s] for key, v in got.items()}, train=train[s])
    # gather + AB refinement (float64 input, float32 AB profile)
    ref = tsk.refine_dimensions(torch.as_tensor(got["T_sel"]).cuda(), test_lens, 3, m,
                                T_sel_train=torch.as_tensor(got["T_sel_train"]).cuda(), train_len=train_lens)
    tsk.sync()
    for s in range(2):
        for r in range(3):
            j = int(got["dim"][s][r])
            i, score, nn = o.refine_dimension(test[s], j, m, 0, T_train=train[s])
            A, _ = o.mp_abjoin(test[s][j], train[s][j], m)
            gi = int(ref["idx"][s, r])
            assert gi == i or A[gi] >= (1 - 1e-3) * A[i]
            assert within_mp_tol(float(ref["score"][s, r]), score, m)
