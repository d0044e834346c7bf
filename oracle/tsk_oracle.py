"""FP64 CPU oracle for sketched multidimensional discord mining.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the library never does, and it
shares no code, header, table or constant with the CUDA path.

It restates, plainly and slowly, what Yeh et al., "Sketching Multidimensional
Time Series for Fast Discord Mining" (arXiv 2311.03393) defines:

  * Def. 2/3   subsequences, z-normalised Euclidean distance, 1NN distance
  * Def. 4/6   discord and self-join matrix profile (P, and its argmin index I)
  * Def. 5     multidimensional discord = argmax over (time, dimension)
  * Sec. III-A global z-normalisation of every stream, then the sketch of
               Alg. 1 (count sketch), written as S = R^T T_bar for a (d, k) R
  * Alg. 2     time detection: per sketch stream MP discord, keep the best group
  * Def. 6     the AB-join profile (T_test != T_train): every test window's
               1NN distance among all training windows, with no exclusion
  * Alg. 2/3   in their AB-join form (test against train)
  * Alg. 3     dimension detection: for the discord window i* of group g*,
               the 1NN distance of that window in every raw stream j of the
               group J_g*, keep the largest; then the optional refinement
               (a whole self-join profile of the chosen stream)
  * Sec. III-C dimension addition/deletion by linearity of the sketch, and the
               point update (one sample of one dimension changes by delta)
  * the adjoint of the top-K aggregated discord scores (not in the paper; the
    derivative of the same definitions, checked against central differences)

Everything is float64.  Loops follow the definitions; numpy reductions and one
library matmul serve as steps, with no blocking or reordering beyond that.

Readings where the paper is silent (the same readings the CUDA path takes):
  * exclusion: pairs with |i - j| < excl are trivial matches (excl = ceil(m/4)
    by default); a window with no admissible neighbour gets P = inf, I = -1.
  * sigma is the population standard deviation (ddof = 0), so that
    dist^2 = 2 m (1 - rho).  A globally constant stream z-normalises to zeros.
  * a window is constant when its variance <= 1e-12 * max(1, mean^2); its
    z-normalised form is the zero vector, hence dist(const, const) = 0 and
    dist(const, non-const) = sqrt(m).
  * ties: lowest neighbour index j, lowest discord index i, lowest group g.
  * top-K: repeat argmax, then mask |i - i*| < topk_excl (default m).
  * Alg. 3: J_g = {j : R[j, g] != 0} (the dimensions a count sketch hashes
    to g; every dimension for a dense Gaussian R).  Self-join form: the
    score of stream j is the self-join profile value of window i* in T_j.
    j* = the first j (ascending) with a score above every earlier one,
    starting from 0; when no score exceeds 0, the lowest j of J_g* (score 0);
    an empty J_g* gives j* = -1.  Refinement = the top-1 discord of T_j*'s
    own self-join profile.
  * point update: the stream's global normalisation (mean, sigma) of the
    build is held fixed, so T_j[i] += delta moves sketch stream g at time i
    by R[j, g] * delta / sigma_j (Alg. 1's s(j) delta for a count sketch and
    unit sigma).
  * AB join: train and test are each z-normalised over their own length
    before sketching ("respectively", Sec. III-A), sketched with the same R;
    every training window is a candidate (no exclusion), lowest j on ties.
  * bf16-matched sketch: T_bar and R are rounded to bfloat16 (round to nearest,
    ties to even, from the float64 value) before the float64 sum.
"""
from __future__ import annotations

import math

import numpy as np

CONST_REL_VAR = 1e-12


# ---------------------------------------------------------------------------
# Number format
# ---------------------------------------------------------------------------

def bf16_round(x) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 value, ties to even.

    bfloat16 keeps 8 significant bits (1 implicit + 7 stored) and float32's
    exponent range (normal >= 2^-126, subnormal spacing 2^-133, max finite
    (2 - 2^-7) 2^127).  Written from that format definition with frexp/ldexp.
    """
    x = np.asarray(x, dtype=np.float64)
    frac, ex = np.frexp(x)                      # x = frac * 2^ex, 0.5 <= |frac| < 1
    normal = np.abs(x) >= 2.0 ** -126
    # 8 significant bits: scale frac to [128, 256) and round half to even
    r_norm = np.ldexp(np.rint(np.ldexp(frac, 8)), ex - 8)
    # subnormal range: fixed spacing 2^-133
    r_sub = np.ldexp(np.rint(np.ldexp(x, 133)), -133)
    out = np.where(normal, r_norm, r_sub)
    # halfway between the largest finite value (2 - 2^-7) 2^127 and 2^128:
    # at or above it the nearest-even result is infinity
    halfway = (2.0 - 2.0 ** -8) * 2.0 ** 127
    out = np.where(np.abs(x) >= halfway, np.copysign(np.inf, x), out)
    out = np.where(np.isnan(x), np.nan, out)
    return out


# ---------------------------------------------------------------------------
# Sec. III-A: global z-normalisation and the sketch (Alg. 1)
# ---------------------------------------------------------------------------

def global_znorm(T):
    """Per-stream z-normalisation over the whole length (Sec. III-A, T_bar).

    T: (d, n).  Returns (T_bar, mu, sigma), sigma the population std.  A
    stream that is constant over its whole length (sigma = 0) has no shape to
    contribute and z-normalises to the zero stream.
    """
    T = np.asarray(T, dtype=np.float64)
    mu = T.mean(axis=1)
    sigma = np.sqrt(((T - mu[:, None]) ** 2).mean(axis=1))
    Tbar = np.zeros_like(T)
    live = sigma > 0
    Tbar[live] = (T[live] - mu[live, None]) / sigma[live, None]
    return Tbar, mu, sigma


def sketch(Tbar, R, bf16: bool = False) -> np.ndarray:
    """S = R^T T_bar: sketch stream g is sum_j R[j, g] T_bar[j] (Alg. 1 as a matrix).

    With a count-sketch R (one +-1 per row, at column h(j)) this is exactly
    Alg. 1's S^(h(j)) += s(j) T_bar^(j).  With bf16=True both operands are
    first rounded to bfloat16; products and sums stay float64.
    """
    Tbar = np.asarray(Tbar, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    if bf16:
        Tbar = bf16_round(Tbar)
        R = bf16_round(R)
    return R.T @ Tbar


def sketch_alg1(Tbar, h, s, k) -> np.ndarray:
    """Alg. 1 literally: start from zeros, add s(j) T_bar^(j) into row h(j)."""
    Tbar = np.asarray(Tbar, dtype=np.float64)
    S = np.zeros((k, Tbar.shape[1]))
    for j in range(Tbar.shape[0]):
        S[int(h[j])] += float(s[j]) * Tbar[j]
    return S


def update_dims(S, T_dims, R_rows, op, bf16: bool = False) -> np.ndarray:
    """Sec. III-C: add (op=+1) or delete (op=-1) dimensions by linearity.

    S (k, n); T_dims (nd, n) raw streams; R_rows (nd, k) their projection rows.
    Each dimension is globally z-normalised on its own, then S += op r_j T_bar_j.
    """
    S = np.array(S, dtype=np.float64, copy=True)
    Tb, _, _ = global_znorm(T_dims)
    R_rows = np.asarray(R_rows, dtype=np.float64)
    if bf16:
        Tb = bf16_round(Tb)
        R_rows = bf16_round(R_rows)
    for q in range(Tb.shape[0]):
        S += float(op[q]) * np.outer(R_rows[q], Tb[q])
    return S


# ---------------------------------------------------------------------------
# Def. 2/3/6: subsequences, z-normalised distance, self-join matrix profile
# ---------------------------------------------------------------------------

def windows(x, m: int) -> np.ndarray:
    """All length-m subsequences x[i:i+m] (Def. 2), shape (n - m + 1, m)."""
    x = np.asarray(x, dtype=np.float64)
    return np.lib.stride_tricks.sliding_window_view(x, m)


def znorm_windows(x, m: int):
    """z-normalise every subsequence; constant windows map to the zero vector.

    Returns (Z (l, m), mean (l,), std (l,), const (l,) bool).
    """
    W = windows(x, m)
    mu = W.mean(axis=1)
    var = ((W - mu[:, None]) ** 2).mean(axis=1)
    const = var <= CONST_REL_VAR * np.maximum(1.0, mu * mu)
    sd = np.sqrt(var)
    Z = np.zeros_like(W)
    nc = ~const
    Z[nc] = (W[nc] - mu[nc, None]) / sd[nc, None]
    return Z, mu, sd, const


def zdist(a, b) -> float:
    """z-normalised Euclidean distance between two equal-length subsequences (Def. 3)."""
    Z, _, _, _ = znorm_windows(np.concatenate([np.asarray(a, float), np.asarray(b, float)]), len(a))
    return float(np.sqrt(((Z[0] - Z[len(a)]) ** 2).sum()))


def mp_rows(x, m: int, excl: int, rows) -> tuple:
    """Self-join matrix profile at the given rows (Def. 6 with T_test = T_train).

    For each i in rows: P[i] = min over j with |i - j| >= excl of
    ||z(x[i:i+m]) - z(x[j:j+m])||, I[i] = the lowest such argmin j.
    No admissible j: P = inf, I = -1.
    """
    Z, _, _, _ = znorm_windows(x, m)
    l = Z.shape[0]
    rows = np.asarray(rows, dtype=np.int64)
    P = np.empty(len(rows))
    I = np.empty(len(rows), dtype=np.int64)
    jj = np.arange(l)
    for r, i in enumerate(rows):
        d = np.sqrt(((Z - Z[i]) ** 2).sum(axis=1))
        d[np.abs(jj - i) < excl] = np.inf
        j = int(np.argmin(d))
        if np.isinf(d[j]):
            P[r], I[r] = np.inf, -1
        else:
            P[r], I[r] = d[j], j
    return P, I


def mp_selfjoin(x, m: int, excl: int) -> tuple:
    """The whole self-join matrix profile (P, I) of one stream, row by row."""
    l = len(x) - m + 1
    if l <= 0:
        return np.empty(0), np.empty(0, dtype=np.int64)
    return mp_rows(x, m, excl, np.arange(l))


# ---------------------------------------------------------------------------
# Def. 5 / Alg. 2: aggregation over streams and the ranked discords
# ---------------------------------------------------------------------------

def aggregate(P_streams) -> tuple:
    """Max over streams per time index (Def. 5): A[i] = max_g P_g[i], G[i] the lowest such g."""
    P = np.asarray(P_streams, dtype=np.float64)
    G = np.argmax(P, axis=0)
    A = P[G, np.arange(P.shape[1])]
    return A, G


def discord_topk(P_streams, I_streams, K: int, topk_excl: int) -> list:
    """Ranked discords (Alg. 2 generalised to a list of K).

    Repeatedly take i* = argmax A (lowest i on ties), report
    (i*, G[i*], A[i*], I_G[i*]), then mask |i - i*| < topk_excl.
    Stops early when every index is masked.
    """
    A, G = aggregate(P_streams)
    I = np.asarray(I_streams)
    A = A.copy()
    live = np.ones(len(A), dtype=bool)
    out = []
    for _ in range(K):
        if not live.any():
            break
        cand = np.where(live, A, -np.inf)
        i = int(np.argmax(cand))
        if not live[i]:
            break
        out.append((i, int(G[i]), float(A[i]), int(I[G[i], i])))
        lo, hi = max(0, i - topk_excl + 1), min(len(A), i + topk_excl)
        live[lo:hi] = False
    return out


def profile_streams(X, m: int, excl: int) -> tuple:
    """(P, I) for every row of X (k, n)."""
    Ps, Is = [], []
    for g in range(X.shape[0]):
        P, I = mp_selfjoin(X[g], m, excl)
        Ps.append(P)
        Is.append(I)
    return np.array(Ps), np.array(Is)


def exact_discords(T, m: int, excl: int, K: int, topk_excl: int) -> list:
    """Exact multidimensional discords: one MP per raw dimension, max over d (Def. 5)."""
    P, I = profile_streams(np.asarray(T, dtype=np.float64), m, excl)
    return discord_topk(P, I, K, topk_excl)


def sketched_discords(T, R, m: int, excl: int, K: int, topk_excl: int, bf16: bool = False):
    """Sketch (Sec. III-A, Alg. 1) then time detection on the k sketch streams (Alg. 2)."""
    Tbar, _, _ = global_znorm(T)
    S = sketch(Tbar, R, bf16=bf16)
    P, I = profile_streams(S, m, excl)
    return discord_topk(P, I, K, topk_excl), S, P, I


# ---------------------------------------------------------------------------
# Adjoint of the summed top-K aggregated scores
# ---------------------------------------------------------------------------

def window_distance(x, i: int, j: int, m: int) -> float:
    """dist(x[i:i+m], x[j:j+m]) by Def. 3."""
    return zdist(np.asarray(x)[i:i + m], np.asarray(x)[j:j + m])


def grad_selected(T, R, selected, m: int, dscore=None) -> tuple:
    """Gradient of L = sum_r w_r dist(S_g[i_r:+m], S_g[j_r:+m]) w.r.t. T and R.

    selected: [(i, g, j)] with the discord index i, its group g and its nearest
    neighbour j (held fixed: the min and max selections are piecewise constant).
    For x = S_g[i:i+m], y = S_g[j:j+m], rho their Pearson correlation and
    x_hat, y_hat the z-normalised windows (population sigma):
        d dist / d x = (rho x_hat - y_hat) / (sigma_x dist)
        d dist / d y = (rho y_hat - x_hat) / (sigma_y dist)
    then dT_bar = R dS, dR = T_bar dS^T, and through the global z-normalisation
        dT_j = (dT_bar_j - mean(dT_bar_j) - T_bar_j mean(dT_bar_j * T_bar_j)) / sigma_j.
    Constant windows or zero distance contribute no gradient.
    """
    T = np.asarray(T, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    Tbar, _, sigma = global_znorm(T)
    S = R.T @ Tbar
    dS = np.zeros_like(S)
    if dscore is None:
        dscore = np.ones(len(selected))
    for (i, g, j), w in zip(selected, dscore):
        x = S[g, i:i + m]
        y = S[g, j:j + m]
        sx, sy = x.std(), y.std()
        mx, my = x.mean(), y.mean()
        if sx <= 0 or sy <= 0:
            continue
        xh, yh = (x - mx) / sx, (y - my) / sy
        dist = np.sqrt(((xh - yh) ** 2).sum())
        if dist <= 0:
            continue
        rho = (xh * yh).sum() / m
        dS[g, i:i + m] += w * (rho * xh - yh) / (sx * dist)
        dS[g, j:j + m] += w * (rho * yh - xh) / (sy * dist)
    dTbar = R @ dS
    dR = Tbar @ dS.T
    dT = np.zeros_like(T)
    live = sigma > 0
    dT[live] = (dTbar[live] - dTbar[live].mean(axis=1, keepdims=True)
                - Tbar[live] * (dTbar[live] * Tbar[live]).mean(axis=1, keepdims=True)) / sigma[live, None]
    return dT, dR


def selected_loss(T, R, selected, m: int, dscore=None) -> float:
    """L = sum_r w_r dist(S_g[i_r:+m], S_g[j_r:+m]) with the selections held fixed."""
    Tbar, _, _ = global_znorm(T)
    S = np.asarray(R, dtype=np.float64).T @ Tbar
    if dscore is None:
        dscore = np.ones(len(selected))
    return float(sum(w * window_distance(S[g], i, j, m) for (i, g, j), w in zip(selected, dscore)))


def topk_loss(T, R, m: int, excl: int, K: int, topk_excl: int) -> float:
    """L = sum of the top-K aggregated discord scores of the FP64 sketched path."""
    res, _, _, _ = sketched_discords(T, R, m, excl, K, topk_excl)
    return float(sum(r[2] for r in res))


def central_difference(f, X, coords, h: float) -> np.ndarray:
    """(f(X + h e_c) - f(X - h e_c)) / (2h) at each coordinate tuple c."""
    X = np.array(X, dtype=np.float64, copy=True)
    out = np.empty(len(coords))
    for q, c in enumerate(coords):
        c = tuple(c)
        x0 = X[c]
        X[c] = x0 + h
        fp = f(X)
        X[c] = x0 - h
        fm = f(X)
        X[c] = x0
        out[q] = (fp - fm) / (2.0 * h)
    return out


# ---------------------------------------------------------------------------
# Counting
# ---------------------------------------------------------------------------

def cells(n: int, m: int, excl: int) -> int:
    """Unordered window pairs (i, j), j - i >= excl, of one stream: (l - excl)(l - excl + 1)/2."""
    l = n - m + 1
    e = l - excl
    return max(0, e) * max(0, e + 1) // 2


# ---------------------------------------------------------------------------
# Alg. 3: discord dimension detection (second phase) and its refinement
# ---------------------------------------------------------------------------

def dim_groups(R) -> list:
    """J_g for every sketch stream g: the dimensions j with R[j, g] != 0 (Sec. III-C, Alg. 3 input)."""
    R = np.asarray(R)
    return [np.flatnonzero(R[:, g] != 0) for g in range(R.shape[1])]


def dimension_detection(T, R, discords, m: int, excl: int, T_train=None) -> tuple:
    """Alg. 3 for every discord (i*, g*) of the time-detection phase.

    For j in J_g* (ascending), s^(j) and its neighbour are the self-join
    profile value and index of window i* in raw stream T_j (Def. 6 at one
    row) or, with T_train, the AB-join value of test window i* of T_j against
    the training stream T_train[j].  Keep j* with s_bsf starting at 0 and a
    strict '>'.
    Returns (picks, scores, nns): picks[r] = (j*, s^(j*), nn^(j*)), scores
    and nns of shape (len(discords), d) with NaN / -1 outside J_g*.
    """
    T = np.asarray(T, dtype=np.float64)
    d = T.shape[0]
    groups = dim_groups(R)
    picks = []
    scores = np.full((len(discords), d), np.nan)
    nns = np.full((len(discords), d), -1, dtype=np.int64)
    for r, (i_star, g_star) in enumerate(discords):
        J = groups[g_star]
        s_bsf, j_star = 0.0, -1
        for j in J:
            if T_train is None:
                P, I = mp_rows(T[j], m, excl, [i_star])
            else:
                P, I = abjoin_rows(T[j], np.asarray(T_train, dtype=np.float64)[j], m, [i_star])
            scores[r, j], nns[r, j] = P[0], I[0]
            if P[0] > s_bsf:
                s_bsf, j_star = P[0], int(j)
        if j_star < 0 and len(J):
            j_star = int(J[0])  # every score is 0
        if j_star < 0:
            picks.append((-1, math.nan, -1))
        else:
            picks.append((j_star, float(scores[r, j_star]), int(nns[r, j_star])))
    return picks, scores, nns


def refine_dimension(T, j: int, m: int, excl: int, topk_excl: int | None = None, T_train=None) -> tuple:
    """Refinement after Alg. 3: the top-1 discord (i, score, nn) of stream j's own self-join
    profile or, with T_train, of its AB-join profile against training stream j."""
    if T_train is None:
        P, I = mp_selfjoin(np.asarray(T, dtype=np.float64)[j], m, excl)
    else:
        P, I = mp_abjoin(np.asarray(T, dtype=np.float64)[j], np.asarray(T_train, dtype=np.float64)[j], m)
    (i, _, score, nn), = discord_topk(P[None, :], I[None, :], 1, m if topk_excl is None else topk_excl)
    return i, score, nn


# ---------------------------------------------------------------------------
# Def. 6 AB join (test against train) and Alg. 2 in that form
# ---------------------------------------------------------------------------

def abjoin_rows(a, b, m: int, rows) -> tuple:
    """AB-join profile of test stream a against training stream b at the given test rows (Def. 6).

    For each test window i: P[i] = min over every training window j of
    ||z(a[i:i+m]) - z(b[j:j+m])||, I[i] = the lowest such argmin j.
    """
    Za, _, _, _ = znorm_windows(a, m)
    Zb, _, _, _ = znorm_windows(b, m)
    rows = np.asarray(rows, dtype=np.int64)
    P = np.empty(len(rows))
    I = np.empty(len(rows), dtype=np.int64)
    for r, i in enumerate(rows):
        d = np.sqrt(((Zb - Za[i]) ** 2).sum(axis=1))
        j = int(np.argmin(d))
        P[r], I[r] = d[j], j
    return P, I


def mp_abjoin(a, b, m: int) -> tuple:
    """(P, I) for every test window of a against training stream b."""
    return abjoin_rows(a, b, m, np.arange(len(a) - m + 1))


def ab_discords(T_test, T_train, m: int, K: int, topk_excl: int, R=None, bf16: bool = False):
    """Ranked discords of the test series against the training series (Def. 5 in AB form, Alg. 2).

    With R: both series are z-normalised over their own length and sketched
    with the same R (Sec. III-A, Alg. 1), and the k sketch streams are
    AB-joined.  Without R: the exact d-dimensional form on the raw streams.
    Returns (ranked list, P, I).
    """
    if R is None:
        A = np.asarray(T_test, dtype=np.float64)
        B = np.asarray(T_train, dtype=np.float64)
    else:
        A = sketch(global_znorm(T_test)[0], R, bf16)
        B = sketch(global_znorm(T_train)[0], R, bf16)
    Ps, Is = [], []
    for g in range(A.shape[0]):
        P, I = mp_abjoin(A[g], B[g], m)
        Ps.append(P)
        Is.append(I)
    P, I = np.array(Ps), np.array(Is)
    return discord_topk(P, I, K, topk_excl), P, I


def point_update(S, R, sigma, updates) -> np.ndarray:
    """Sec. III-C point update: for each (j, i, delta), T_j[i] += delta moves every
    sketch stream g at time i by R[j, g] * delta / sigma_j (sigma_j of the build)."""
    S = np.array(S, dtype=np.float64, copy=True)
    R = np.asarray(R, dtype=np.float64)
    for j, i, delta in updates:
        S[:, i] += R[j, :] * (delta / sigma[j])
    return S


def znorm_with(T, mu, sigma) -> np.ndarray:
    """T_bar under given per-stream statistics (the build's, for point updates): (T - mu) / sigma, 0 where sigma = 0."""
    T = np.asarray(T, dtype=np.float64)
    out = np.zeros_like(T)
    live = np.asarray(sigma) > 0
    out[live] = (T[live] - np.asarray(mu)[live, None]) / np.asarray(sigma)[live, None]
    return out
