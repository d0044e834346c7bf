"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-type the oracle's own formula: each compares it with a hand
derivation, a closed form reached another way, a library routine, an
invariant, a special case, or brute force on tiny inputs.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.stats

from oracle import tsk_oracle as o
from paper_2311_03393_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_cases(name):
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "case":
                cur = cases.setdefault(vals[0], {})
            else:
                cur.setdefault(key, []).append([float(v) for v in vals])
    return cases


# --- Def. 3/6: hand-derived profiles ----------------------------------------

@pytest.mark.parametrize("name", ["alternating", "alternating_wide", "spikes_const", "spikes"])
def test_golden_tiny_profiles(name):
    c = _read_cases("tiny_mp.txt")[name]
    x = np.array(c["x"][0])
    m, excl = int(c["m"][0][0]), int(c["excl"][0][0])
    P, I = o.mp_selfjoin(x, m, excl)
    np.testing.assert_allclose(P, np.array(c["P"][0]), rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(I, np.array(c["I"][0], dtype=np.int64))


def test_closed_form_matches_direct_distance():
    """dist^2 = 2 m (1 - rho) with rho from numpy's Pearson correlation (library routine)."""
    rng = np.random.default_rng(1)
    for m in (4, 17, 100):
        for _ in range(50):
            a = np.cumsum(rng.normal(size=m)) * rng.uniform(0.1, 10) + rng.normal() * 100
            b = rng.normal(size=m) + 0.5 * a
            rho = np.corrcoef(a, b)[0, 1]
            assert o.zdist(a, b) == pytest.approx(math.sqrt(max(0.0, 2 * m * (1 - rho))), rel=1e-10, abs=1e-10)


def test_window_stats_match_library():
    rng = np.random.default_rng(2)
    x = np.cumsum(rng.normal(size=500))
    m = 37
    Z, mu, sd, const = o.znorm_windows(x, m)
    for i in (0, 1, 100, 463):
        w = x[i:i + m]
        assert mu[i] == pytest.approx(np.mean(w), rel=1e-13)
        assert sd[i] == pytest.approx(np.std(w), rel=1e-12)
        np.testing.assert_allclose(Z[i], scipy.stats.zscore(w), rtol=1e-10, atol=1e-12)
    assert not const.any()


def test_brute_force_tiny_against_itertools():
    """Profile vs an explicit enumeration of all admissible pairs with library z-scores."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=23)
    m, excl = 5, 2
    l = len(x) - m + 1
    zs = [scipy.stats.zscore(x[i:i + m]) for i in range(l)]
    P, I = o.mp_selfjoin(x, m, excl)
    for i in range(l):
        best, arg = math.inf, -1
        for j in range(l):
            if abs(i - j) >= excl:
                dd = float(np.linalg.norm(zs[i] - zs[j]))
                if dd < best:
                    best, arg = dd, j
        assert P[i] == pytest.approx(best, rel=1e-12)
        assert I[i] == arg


def test_periodic_signal_has_zero_profile():
    """An exactly periodic stream (period p > excl) has an exact repeat for every window."""
    p, m = 25, 40
    t = np.arange(m + 3 * p)
    x = np.sin(2 * np.pi * t / p) + 0.3 * np.cos(4 * np.pi * t / p)
    P, I = o.mp_selfjoin(x, m, o_excl := math.ceil(m / 4))
    assert o_excl < p
    assert np.all(P < 1e-6)
    assert np.all(np.abs(np.abs(I - np.arange(len(I))) % p) == 0)


def test_white_noise_profile_scale():
    """For i.i.d. noise the pairwise correlations concentrate at 0, distances at sqrt(2m)."""
    rng = np.random.default_rng(4)
    m = 64
    x = rng.normal(size=3000)
    W = np.lib.stride_tricks.sliding_window_view(x, m)[::97]
    Z = scipy.stats.zscore(W, axis=1)
    d = [np.linalg.norm(Z[a] - Z[b]) for a in range(len(Z)) for b in range(a + 1, len(Z))]
    assert np.median(d) == pytest.approx(math.sqrt(2 * m), rel=0.05)
    P, _ = o.mp_rows(x, m, 16, [10, 1500, 2900])
    assert np.all(P < math.sqrt(2 * m)) and np.all(P > 0.5 * math.sqrt(2 * m))


def test_profile_invariant_to_scale_sign_shift():
    rng = np.random.default_rng(5)
    x = np.cumsum(rng.normal(size=300))
    m, excl = 20, 5
    P0, I0 = o.mp_selfjoin(x, m, excl)
    for c, b in ((3.5, -7.0), (-0.01, 1e3), (-1.0, 0.0)):
        P1, I1 = o.mp_selfjoin(c * x + b, m, excl)
        np.testing.assert_allclose(P1, P0, rtol=1e-7, atol=1e-7)
        np.testing.assert_array_equal(I1, I0)


def test_constant_window_rules_against_hand_values():
    x = np.concatenate([np.full(10, 3.0), np.arange(10.0), np.full(10, 3.0)])
    m, excl = 5, 2
    P, I = o.mp_selfjoin(x, m, excl)
    l = len(x) - m + 1
    const = [np.ptp(x[i:i + m]) == 0 for i in range(l)]
    for i in range(l):
        if const[i]:
            assert P[i] == 0.0 and const[I[i]]
        else:
            assert P[i] <= math.sqrt(m) + 1e-12


# --- Sec. III-A: z-normalisation and sketch ----------------------------------

def test_global_znorm_matches_scipy_zscore():
    T, _ = synth.random_walks(6, 700, 50, 1, seed=6, dtype=np.float64)
    Tbar, mu, sigma = o.global_znorm(T)
    np.testing.assert_allclose(Tbar, scipy.stats.zscore(T, axis=1, ddof=0), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(sigma, np.std(T, axis=1), rtol=1e-12)


def test_globally_constant_stream_contributes_nothing():
    """A constant stream has no shape: the sketch of the other streams is unchanged by it."""
    T, _ = synth.random_walks(4, 300, 20, 0, seed=19, dtype=np.float64)
    Tc = np.vstack([T, np.full((1, 300), 7.5)])
    R = synth.gaussian_R(5, 2, 20).astype(np.float64)
    Tbar, _, sigma = o.global_znorm(Tc)
    assert sigma[4] == 0 and np.all(Tbar[4] == 0)
    np.testing.assert_allclose(o.sketch(Tbar, R), o.sketch(o.global_znorm(T)[0], R[:4]), rtol=0, atol=1e-12)


def test_fig1_sum_of_streams_is_the_k1_sketch_and_keeps_the_discord():
    """Fig. 1: the MP of the sum of z-normalised streams still shows a discord of one stream."""
    n, m = 1200, 60
    rng = np.random.default_rng(7)
    t = np.arange(n)
    T = np.stack([np.sin(2 * np.pi * t / 50 + ph) + 0.05 * rng.normal(size=n)
                  for ph in rng.uniform(0, 6.28, size=5)])
    p = 600
    T[0, p:p + m] = rng.normal(size=m) * 0.5
    R = np.ones((5, 1))
    Tbar, _, _ = o.global_znorm(T)
    S = o.sketch(Tbar, R)
    np.testing.assert_allclose(S[0], np.sum(scipy.stats.zscore(T, axis=1), axis=0), rtol=1e-10, atol=1e-10)
    res = o.discord_topk(*o.profile_streams(S, m, m // 4), K=1, topk_excl=m)
    assert abs(res[0][0] - p) <= m


def test_count_sketch_permutation_gives_the_exact_profiles():
    """k = d with h a permutation: every sketch stream is +-T_bar_j, so its MP is T_j's MP."""
    d, n, m = 5, 400, 24
    T, _ = synth.random_walks(d, n, m, 1, seed=8, dtype=np.float64)
    h = np.array([2, 4, 1, 0, 3])          # not an involution: catches a transposed R
    s = np.array([1, -1, -1, 1, -1])
    R = np.zeros((d, d))
    R[np.arange(d), h] = s
    Tbar, _, _ = o.global_znorm(T)
    S = o.sketch(Tbar, R)
    np.testing.assert_allclose(S, o.sketch_alg1(Tbar, h, s, d), rtol=0, atol=1e-13)
    for j in range(d):
        Pe, Ie = o.mp_selfjoin(T[j], m, 6)
        Ps, Is = o.mp_selfjoin(S[h[j]], m, 6)
        np.testing.assert_allclose(Ps, Pe, rtol=1e-7, atol=1e-7)


def test_dimension_delete_then_add_equals_rebuild():
    """Sec. III-C linearity: removing then re-adding a dimension restores the sketch."""
    d, n, k = 7, 500, 3
    T, _ = synth.random_walks(d, n, 20, 0, seed=9, dtype=np.float64)
    R = synth.gaussian_R(d, k, 10).astype(np.float64)
    for bf16 in (False, True):
        S = o.sketch(o.global_znorm(T)[0], R, bf16=bf16)
        S_minus = o.update_dims(S, T[[2, 5]], R[[2, 5]], [-1, -1], bf16=bf16)
        keep = [0, 1, 3, 4, 6]
        np.testing.assert_allclose(S_minus, o.sketch(o.global_znorm(T[keep])[0], R[keep], bf16=bf16),
                                   rtol=0, atol=1e-12)
        S_back = o.update_dims(S_minus, T[[2, 5]], R[[2, 5]], [1, 1], bf16=bf16)
        np.testing.assert_allclose(S_back, S, rtol=0, atol=1e-12)


def test_lemma1_count_sketch_unbiased_with_stated_variance():
    """Lemma 1: E[s(j) S^(h(j))_i] = T_bar^(j)_i, Var = (1/k) sum_{j' != j} (T_bar^(j')_i)^2."""
    d, k, n = 12, 4, 6
    rng = np.random.default_rng(11)
    Tbar = rng.normal(size=(d, n))
    draws = 6000
    est = np.empty((draws, d, n))
    for r in range(draws):
        h, s = synth.count_sketch_hashes(d, k, seed=1000 + r)
        S = o.sketch_alg1(Tbar, h, s, k)
        est[r] = s[:, None] * S[h]
    mean = est.mean(axis=0)
    var = est.var(axis=0)
    want_var = (np.sum(Tbar ** 2, axis=0)[None, :] - Tbar ** 2) / k
    se = np.sqrt(want_var / draws)
    assert np.all(np.abs(mean - Tbar) < 5 * se + 1e-12)
    np.testing.assert_allclose(var, want_var, rtol=0.12)


# --- Def. 5 / Alg. 2 ---------------------------------------------------------

def test_aggregate_and_topk_tie_rules():
    rows = {}
    with open(os.path.join(GOLDEN, "topk_ties.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, *vals = line.split()
                rows.setdefault(key, []).append([float(v) for v in vals])
    P = np.array(rows["P"])
    I = np.array(rows["I"], dtype=np.int64)
    K, te = int(rows["K"][0][0]), int(rows["topk_excl"][0][0])
    res = o.discord_topk(P, I, K, te)
    want = [(int(r[0]), int(r[1]), r[2], int(r[3])) for r in rows["R"]]
    assert res == want


def test_all_zero_scores_return_group_zero():
    """Alg. 2 starts from a best-so-far of 0 with a strict '>': all-zero scores give g = 0."""
    P = np.zeros((3, 5))
    I = np.zeros((3, 5), dtype=np.int64)
    res = o.discord_topk(P, I, 1, 2)
    assert res[0][:3] == (0, 0, 0.0)


def test_planted_discord_is_the_discord_of_its_stream():
    """Sanity on the small random-walk workload: the planted stream's own discord is the planted window.

    (Random walks carry natural discords of similar size, so the planted one
    need not be the top across all streams; the paper notes this difficulty.)
    """
    wl = synth.workload(1)
    T = wl.series[0]
    (_, j, p), = wl.planted
    excl = synth.default_excl(wl.m)
    P, I = o.mp_selfjoin(T[j], wl.m, excl)
    assert abs(int(np.argmax(P)) - p) <= wl.m


# --- adjoint -----------------------------------------------------------------

def test_adjoint_matches_central_differences_of_full_forward():
    d, n, m, k, K = 5, 260, 16, 3, 2
    T, _ = synth.random_walks(d, n, m, 2, seed=12, dtype=np.float64)
    R = synth.gaussian_R(d, k, 13).astype(np.float64)
    excl = synth.default_excl(m)
    res, S, P, I = o.sketched_discords(T, R, m, excl, K, m)
    sel = [(i, g, nn) for (i, g, _, nn) in res]
    dT, dR = o.grad_selected(T, R, sel, m)
    rng = np.random.default_rng(14)
    support = [(j, t) for (i, g, nn) in sel for j in range(d) for t in list(range(i, i + m)) + list(range(nn, nn + m))]
    cT = [support[q] for q in rng.choice(len(support), 20, replace=False)] + \
         [tuple(v) for v in zip(rng.integers(0, d, 10), rng.integers(0, n, 10))]
    fdT = o.central_difference(lambda X: o.topk_loss(X, R, m, excl, K, m), T, cT, 1e-5)
    got = np.array([dT[c] for c in cT])
    np.testing.assert_allclose(got, fdT, rtol=1e-5, atol=1e-7)
    cR = [(j, g) for j in range(d) for g in range(k)]
    fdR = o.central_difference(lambda X: o.topk_loss(T, X, m, excl, K, m), R, cR, 1e-5)
    np.testing.assert_allclose([dR[c] for c in cR], fdR, rtol=1e-5, atol=1e-7)


def test_fixed_selection_loss_equals_topk_loss():
    d, n, m, k, K = 4, 220, 12, 2, 2
    T, _ = synth.random_walks(d, n, m, 1, seed=15, dtype=np.float64)
    R = synth.gaussian_R(d, k, 16).astype(np.float64)
    excl = synth.default_excl(m)
    res, _, _, _ = o.sketched_discords(T, R, m, excl, K, m)
    sel = [(i, g, nn) for (i, g, _, nn) in res]
    assert o.selected_loss(T, R, sel, m) == pytest.approx(o.topk_loss(T, R, m, excl, K, m), rel=1e-12)


# --- number format and counting ---------------------------------------------

def test_bf16_round_matches_torch_for_float32_inputs():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    x = np.concatenate([
        rng.normal(size=20000).astype(np.float32),
        (rng.normal(size=2000) * 1e-30).astype(np.float32),
        (rng.normal(size=2000) * 1e30).astype(np.float32),
        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 2 ** -130, 0.0, -0.0], dtype=np.float32),
    ])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(o.bf16_round(x.astype(np.float64)), want)


def test_bf16_round_float64_ties_to_even_exactly():
    """Rounding from float64 (not via float32) checked with exact rationals."""
    rng = np.random.default_rng(18)
    vals = list(rng.normal(size=300) * 10.0 ** rng.integers(-5, 5, size=300))
    vals += [1 + 2 ** -8, 1 + 2 ** -8 + 2 ** -40, 1 + 3 * 2 ** -8, 1 + 2 ** -8 - 2 ** -45]
    for v in vals:
        v = float(v)
        e = math.frexp(abs(v))[1]
        ulp = Fraction(2) ** (e - 8)
        q = Fraction(abs(v)) / ulp
        lo = math.floor(q)
        rem = q - lo
        r = lo + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1) else 0)
        want = math.copysign(float(r * ulp), v)
        assert o.bf16_round(np.array([v]))[0] == want, v


def test_cell_count_by_enumeration():
    for n, m, excl in ((50, 7, 2), (31, 5, 10), (12, 12, 1), (40, 10, 3)):
        l = n - m + 1
        brute = sum(1 for i in range(l) for j in range(i + 1, l) if j - i >= excl)
        assert o.cells(n, m, excl) == brute


# ---------------------------------------------------------------------------
# Alg. 3: dimension detection and its refinement
# ---------------------------------------------------------------------------

def _zscore_windows_scipy(x, m):
    """Every length-m window z-scored by scipy (ddof 0); constant windows -> zeros."""
    W = np.lib.stride_tricks.sliding_window_view(np.asarray(x, dtype=np.float64), m)
    Z = np.zeros_like(W)
    for t in range(W.shape[0]):
        if np.ptp(W[t]) > 0:
            Z[t] = scipy.stats.zscore(W[t])
    return Z


def _brute_row(x, m, excl, i):
    """min over |t - i| >= excl of the direct z-normalised distance, lowest t on ties."""
    Z = _zscore_windows_scipy(x, m)
    best, arg = math.inf, -1
    for t in range(Z.shape[0]):
        if abs(t - i) < excl:
            continue
        dist = float(np.linalg.norm(Z[i] - Z[t]))
        if dist < best:
            best, arg = dist, t
    return best, arg


def test_dim_groups_follow_the_count_sketch_hashes():
    d, k, seed = 40, 6, 11
    h, _ = synth.count_sketch_hashes(d, k, seed)
    groups = o.dim_groups(synth.count_sketch_R(d, k, seed))
    for g in range(k):
        assert list(groups[g]) == [j for j in range(d) if h[j] == g]
    assert sum(len(J) for J in groups) == d
    for J in o.dim_groups(synth.gaussian_R(d, k, seed)):
        assert list(J) == list(range(d))


def test_dimension_detection_recovers_the_planted_dimension():
    """A noise burst planted in stream 4 of periodic streams: Alg. 2 finds its time, Alg. 3 its dimension."""
    d, n, m, k, p = 6, 700, 40, 3, 350
    rng = np.random.default_rng(5)
    t = np.arange(n)
    periods = [10, 20, 25, 50, 20, 10]           # every sum of these repeats with period 100
    T = np.stack([rng.uniform(0.5, 2.0) * np.sin(2 * np.pi * t / q + rng.uniform(0, 2 * np.pi))
                  for q in periods])
    T[4, p:p + m] = rng.normal(0.0, 1.0, m)
    excl = synth.default_excl(m)
    R = synth.count_sketch_R(d, k, seed=8)
    res, _, _, _ = o.sketched_discords(T, R, m, excl, 1, m)
    i_star, g_star = res[0][0], res[0][1]
    assert abs(i_star - p) <= m and R[4, g_star] != 0
    picks, scores, nns = o.dimension_detection(T, R, [(i_star, g_star)], m, excl)
    assert picks[0][0] == 4
    for j in range(d):
        if R[j, g_star] == 0:
            assert math.isnan(scores[0, j]) and nns[0, j] == -1
        else:
            b, a = _brute_row(T[j], m, excl, i_star)
            assert abs(scores[0, j] - b) <= 1e-9 * max(1.0, b)
            # near-zero distances of the periodic streams may tie; the neighbour must still be a minimiser
            Z = _zscore_windows_scipy(T[j], m)
            assert abs(float(np.linalg.norm(Z[i_star] - Z[nns[0, j]])) - b) <= 1e-9 * max(1.0, b)
            assert j != 4 or nns[0, j] == a


def test_dimension_detection_tie_zero_and_empty_rules():
    rng = np.random.default_rng(3)
    n, m, excl = 300, 20, 5
    y = np.cumsum(rng.normal(size=n))
    per = np.tile(np.sin(2 * np.pi * np.arange(25) / 25), n // 25 + 1)[:n]
    T = np.stack([per, y, np.cumsum(rng.normal(size=n)), y.copy(), per * 3.0 + 1.0])
    R = np.zeros((5, 3))
    R[[0, 1, 3], 0] = [1.0, -1.0, 1.0]   # J_0 = {0, 1, 3}: 1 and 3 identical
    R[[0, 4], 1] = [1.0, 1.0]            # J_1 = {0, 4}: both periodic, every score 0
    i = 120
    picks, scores, _ = o.dimension_detection(T, R, [(i, 0), (i, 1), (i, 2)], m, excl)
    assert scores[0, 0] < 1e-6 and scores[0, 1] == scores[0, 3] > 0
    assert picks[0][0] == 1                                  # lowest j among the tied maxima
    assert picks[1][0] == 0 and picks[1][1] < 1e-6           # no score above 0 -> lowest j of J
    assert picks[2][0] == -1 and math.isnan(picks[2][1]) and picks[2][2] == -1  # empty group


def test_dimension_detection_invariant_to_affine_maps_of_streams():
    T, _ = synth.random_walks(4, 400, 30, 1, seed=9, dtype=np.float64)
    R = synth.gaussian_R(4, 2, seed=1)
    picks, scores, nns = o.dimension_detection(T, R, [(150, 0), (40, 1)], 30, 8)
    T2 = T * np.array([[2.5], [-0.5], [1e-3], [7.0]]) + np.array([[3.0], [-100.0], [0.0], [1e4]])
    picks2, scores2, nns2 = o.dimension_detection(T2, R, [(150, 0), (40, 1)], 30, 8)
    assert [p[0] for p in picks] == [p[0] for p in picks2]
    np.testing.assert_allclose(scores, scores2, rtol=1e-7)
    np.testing.assert_array_equal(nns, nns2)


def test_refinement_is_the_brute_force_discord_of_the_stream():
    T, _ = synth.random_walks(3, 240, 20, 1, seed=13, dtype=np.float64, discord_streams=[1])
    excl = 5
    i, score, nn = o.refine_dimension(T, 1, 20, excl)
    rows = [_brute_row(T[1], 20, excl, t) for t in range(240 - 20 + 1)]
    best = max(range(len(rows)), key=lambda t: (rows[t][0], -t))
    assert i == best and abs(score - rows[best][0]) <= 1e-9 * rows[best][0] and nn == rows[best][1]
    # the refined score is at least the Alg. 3 score of any window of that stream
    picks, _, _ = o.dimension_detection(T, np.ones((3, 1)), [(37, 0)], 20, excl)
    assert score >= o.mp_rows(T[1], 20, excl, [37])[0][0]


# ---------------------------------------------------------------------------
# Def. 6 AB join and Alg. 2 / Alg. 3 in their train/test form
# ---------------------------------------------------------------------------

def test_abjoin_against_brute_force_pairs():
    rng = np.random.default_rng(41)
    a = np.cumsum(rng.normal(size=37))
    b = np.cumsum(rng.normal(size=29))
    b[5:11] = 2.0                                    # constant training windows
    m = 6
    Za, Zb = _zscore_windows_scipy(a, m), _zscore_windows_scipy(b, m)
    P, I = o.mp_abjoin(a, b, m)
    for i in range(len(Za)):
        dists = [float(np.linalg.norm(Za[i] - Zb[j])) for j in range(len(Zb))]
        jb = min(range(len(dists)), key=lambda j: (dists[j], j))
        assert abs(P[i] - dists[jb]) <= 1e-9 and I[i] == jb


def test_abjoin_rows_against_brute_force_pairs():
    """abjoin_rows (the sampled-row form the full-size GPU tests use) against scipy z-scores, every row."""
    rng = np.random.default_rng(43)
    a = np.cumsum(rng.normal(size=48))
    b = np.cumsum(rng.normal(size=31))
    a[10:18] = -1.0                                  # constant test windows
    m = 7
    Za, Zb = _zscore_windows_scipy(a, m), _zscore_windows_scipy(b, m)
    rows = list(range(len(Za)))
    P, I = o.abjoin_rows(a, b, m, rows)
    for r, i in enumerate(rows):
        dists = [float(np.linalg.norm(Za[i] - Zb[j])) for j in range(len(Zb))]
        jb = min(range(len(dists)), key=lambda j: (dists[j], j))
        assert abs(P[r] - dists[jb]) <= 1e-9 and I[r] == jb


def test_exact_discords_against_brute_force_profiles():
    """exact_discords (Def. 5 over the raw dimensions, then Alg. 2's ranked list) against
    per-dimension brute-force profiles from scipy z-scores, aggregated and ranked by hand."""
    rng = np.random.default_rng(44)
    d, n, m, K = 3, 70, 8, 3
    T = np.cumsum(rng.normal(size=(d, n)), axis=1)
    excl = 2
    l = n - m + 1
    P = np.array([[_brute_row(T[j], m, excl, i)[0] for i in range(l)] for j in range(d)])
    I = np.array([[_brute_row(T[j], m, excl, i)[1] for i in range(l)] for j in range(d)])
    A = P.max(axis=0)
    G = np.array([min(j for j in range(d) if P[j, i] == A[i]) for i in range(l)])
    want, Am = [], A.copy()
    for _ in range(K):
        i = int(np.argmax(Am))
        want.append((i, int(G[i]), float(A[i]), int(I[G[i], i])))
        Am[max(0, i - m + 1):i + m] = -np.inf
    got = o.exact_discords(T, m, excl, K, m)
    assert [(g[0], g[1], g[3]) for g in got] == [(w[0], w[1], w[3]) for w in want]
    assert np.allclose([g[2] for g in got], [w[2] for w in want], rtol=0, atol=1e-9)


def test_abjoin_of_a_series_with_itself_is_zero_and_the_closest_pair_is_shared():
    rng = np.random.default_rng(42)
    x = np.cumsum(rng.normal(size=300))
    P, I = o.mp_abjoin(x, x, 20)
    assert np.all(P < 1e-6)
    Z = _zscore_windows_scipy(x, 20)
    assert all(np.linalg.norm(Z[i] - Z[I[i]]) < 1e-6 for i in range(0, len(P), 17))
    # min over test rows of P_ab == min over training rows of P_ba (the same closest pair)
    y = np.cumsum(rng.normal(size=250))
    Pab, _ = o.mp_abjoin(x, y, 20)
    Pba, _ = o.mp_abjoin(y, x, 20)
    assert abs(Pab.min() - Pba.min()) <= 1e-9


def test_ab_discord_finds_the_window_that_training_never_saw():
    """Test = train everywhere but one replaced window: the AB discord (exact and sketched) is there."""
    d, n, m, k, p = 5, 600, 30, 2, 333
    rng = np.random.default_rng(43)
    t = np.arange(n)
    train = np.stack([np.sin(2 * np.pi * t / q + rng.uniform(0, 6)) for q in (15, 20, 25, 30, 50)])
    test = train.copy()
    test[3, p:p + m] = rng.normal(size=m)
    res, P, _ = o.ab_discords(test, train, m, 1, m)
    assert abs(res[0][0] - p) < m and res[0][1] == 3
    R = synth.count_sketch_R(d, k, seed=2)
    res_s, _, _ = o.ab_discords(test, train, m, 1, m, R=R)
    assert abs(res_s[0][0] - p) < m and R[3, res_s[0][1]] != 0
    picks, _, _ = o.dimension_detection(test, R, [(res_s[0][0], res_s[0][1])], m, 0, T_train=train)
    assert picks[0][0] == 3


def test_ab_identity_count_sketch_gives_the_exact_ab_profiles():
    rng = np.random.default_rng(44)
    d, m = 3, 16
    train = np.cumsum(rng.normal(size=(d, 200)), axis=1)
    test = np.cumsum(rng.normal(size=(d, 150)), axis=1)
    R = np.diag([1.0, -1.0, 1.0])                     # k = d, h(j) = j
    _, Ps, Is = o.ab_discords(test, train, m, 2, m, R=R)
    _, Pe, Ie = o.ab_discords(test, train, m, 2, m)
    np.testing.assert_allclose(Ps, Pe, rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(Is, Ie)


def test_ab_refinement_is_the_brute_force_ab_discord_of_the_stream():
    rng = np.random.default_rng(45)
    train = np.cumsum(rng.normal(size=(2, 160)), axis=1)
    test = np.cumsum(rng.normal(size=(2, 120)), axis=1)
    m = 12
    i, score, nn = o.refine_dimension(test, 1, m, 0, T_train=train)
    Za, Zb = _zscore_windows_scipy(test[1], m), _zscore_windows_scipy(train[1], m)
    best = [min((float(np.linalg.norm(Za[t] - Zb[u])), u) for u in range(len(Zb))) for t in range(len(Za))]
    ib = max(range(len(best)), key=lambda t: (best[t][0], -t))
    assert i == ib and abs(score - best[ib][0]) <= 1e-9 and nn == best[ib][1]


def test_point_update_equals_sketching_the_updated_series_with_the_build_normalisation():
    rng = np.random.default_rng(46)
    d, n, k = 7, 300, 3
    T = np.cumsum(rng.normal(size=(d, n)), axis=1)
    R = synth.gaussian_R(d, k, 4)
    Tbar, mu, sigma = o.global_znorm(T)
    S = o.sketch(Tbar, R)
    ups = [(2, 10, 0.5), (2, 10, -1.25), (6, 299, 3.0), (0, 0, -2.0)]   # repeated point included
    T2 = T.copy()
    for j, i, dl in ups:
        T2[j, i] += dl
    want = R.T @ ((T2 - mu[:, None]) / sigma[:, None])
    np.testing.assert_allclose(o.point_update(S, R, sigma, ups), want, rtol=0, atol=1e-12)
    # a count sketch moves only stream h(j), by s(j) delta / sigma_j
    h, sg = synth.count_sketch_hashes(d, k, 5)
    Rc = synth.count_sketch_R(d, k, 5)
    D = o.point_update(np.zeros((k, n)), Rc, sigma, [(4, 50, 1.0)])
    assert np.count_nonzero(D) == 1 and D[h[4], 50] == pytest.approx(sg[4] / sigma[4])


def test_znorm_with_build_statistics_matches_scipy():
    rng = np.random.default_rng(47)
    T = np.cumsum(rng.normal(size=(4, 90)), axis=1)
    T[2] = 3.0                                            # sigma = 0 stream
    out = o.znorm_with(T, T.mean(axis=1), T.std(axis=1))
    np.testing.assert_allclose(out[[0, 1, 3]], scipy.stats.zscore(T[[0, 1, 3]], axis=1, ddof=0), rtol=1e-12, atol=1e-12)
    assert np.all(out[2] == 0.0)
