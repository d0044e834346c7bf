"""GPU parity: every entry point of the C ABI against the FP64 oracle.

Inputs are seeded synthetic workloads; sizes keep the oracle to seconds while
spanning several bands of diagonals, several row blocks and ragged tails.
"""
import math

import numpy as np
import pytest

from oracle import tsk_oracle as o
from paper_2311_03393_gb300 import synth

from helpers import FP64_REL_TOL, MP_REL_TOL, check_discords, check_profile

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


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _streams(tsk, xs, m, excl, precision="fp32", rows=None, dtype=torch.float32):
    X = _cuda(np.concatenate([np.asarray(x).ravel() for x in xs]), dtype)
    lens = [len(x) for x in xs]
    P, I = tsk.mp_selfjoin(X, lens, m, excl, precision=precision)
    tsk.sync()
    P, I = P.cpu().numpy(), I.cpu().numpy()
    out, off = [], 0
    for n in lens:
        out.append((P[off:off + n], I[off:off + n]))
        off += n
    return out


# --- matrix profile -----------------------------------------------------------

@pytest.mark.parametrize("rows_per_unit", [0, 64, 32])
def test_mp_selfjoin_fp32_ragged_streams(tsk, rows_per_unit):
    tsk.set_tile_rows(rows_per_unit)
    try:
        m, excl = 100, 25
        rng = np.random.default_rng(100)
        xs = [np.cumsum(rng.normal(size=n)).astype(np.float32) for n in (3001, 1187, 640)]
        xs.append(synth.traffic(1, 2400, 144, 1, seed=101)[0][0])
        res = _streams(tsk, xs, m, excl)
        for x, (P, I) in zip(xs, res):
            l = len(x) - m + 1
            assert np.all(np.isnan(P[l:])) and np.all(I[l:] == -1)
            check_profile(x.astype(np.float64), m, excl, P[:l], I[:l])
    finally:
        tsk.set_tile_rows(0)


def test_mp_selfjoin_fp32_float64_input_and_odd_exclusion(tsk):
    m, excl = 37, 13
    x, _ = synth.random_walks(1, 2200, m, 1, seed=102, dtype=np.float64)
    (P, I), = _streams(tsk, [x[0]], m, excl, dtype=torch.float64)
    l = len(x[0]) - m + 1
    check_profile(x[0], m, excl, P[:l], I[:l])


def test_mp_selfjoin_fp64_exact(tsk):
    m, excl = 50, 13
    x, _ = synth.random_walks(2, 1500, m, 1, seed=103, dtype=np.float64)
    res = _streams(tsk, [x[0], x[1]], m, excl, precision="fp64", dtype=torch.float64)
    for xi, (P, I) in zip(x, res):
        l = len(xi) - m + 1
        P_ref, I_ref = o.mp_selfjoin(xi, m, excl)
        np.testing.assert_allclose(P[:l], P_ref, rtol=FP64_REL_TOL, atol=1e-9)
        np.testing.assert_array_equal(I[:l], I_ref)


def test_constant_windows_and_exact_repeats(tsk):
    """Square waves: constant windows (zero-vector rule) and exact repeats (distance 0)."""
    m, excl = 40, 10
    t = np.arange(1500)
    sq = (((t + 7) % 300) < 150).astype(np.float32)
    mixed = np.concatenate([np.full(200, 2.0), np.cumsum(np.random.default_rng(104).normal(size=700)),
                            np.full(300, -1.0)]).astype(np.float32)
    res = _streams(tsk, [sq, mixed], m, excl)
    for x, (P, I) in zip([sq, mixed], res):
        l = len(x) - m + 1
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l])
    for prec in ("fp64",):
        res = _streams(tsk, [sq, mixed], m, excl, precision=prec, dtype=torch.float64)
        for x, (P, I) in zip([sq, mixed], res):
            l = len(x) - m + 1
            P_ref, I_ref = o.mp_selfjoin(x.astype(np.float64), m, excl)
            np.testing.assert_allclose(P[:l], P_ref, rtol=FP64_REL_TOL, atol=1e-6)


def test_degenerate_lengths(tsk):
    """n = m (one window), l < 2 excl (windows without admissible neighbour)."""
    m = 16
    rng = np.random.default_rng(105)
    xs = [rng.normal(size=16).astype(np.float32), rng.normal(size=20).astype(np.float32),
          rng.normal(size=40).astype(np.float32)]
    res = _streams(tsk, xs, m, 4)
    for x, (P, I) in zip(xs, res):
        l = len(x) - m + 1
        check_profile(x.astype(np.float64), m, 4, P[:l], I[:l])


@pytest.mark.parametrize("case", ["offset", "long_m", "m2"])
def test_offsets_long_and_shortest_subsequences(tsk, case):
    """A large offset under a small spread (float32 anchors and statistics must not cancel),
    a long subsequence (m = 1000: long anchors, several bands), and the shortest one (m = 2)."""
    rng = np.random.default_rng(107)
    if case == "offset":
        m, excl = 64, 16
        xs = [(2.5e4 + np.cumsum(rng.normal(size=n))).astype(np.float32) for n in (3000, 1700)]
    elif case == "long_m":
        m, excl = 1000, 250
        xs = [np.cumsum(rng.normal(size=n)).astype(np.float32) for n in (6000, 2600)]
    else:
        m, excl = 2, 1
        xs = [rng.normal(size=n).astype(np.float32) for n in (1500, 700)]
    res = _streams(tsk, xs, m, excl)
    for x, (P, I) in zip(xs, res):
        l = len(x) - m + 1
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l], rows=np.arange(0, l, 3))


def test_stream_mask_leaves_masked_outputs_untouched(tsk):
    m = 32
    rng = np.random.default_rng(106)
    xs = [rng.normal(size=500).astype(np.float32) for _ in range(3)]
    X = _cuda(np.concatenate(xs))
    P = torch.full((1500,), 7.0, device="cuda")
    I = torch.full((1500,), 7, dtype=torch.int32, device="cuda")
    tsk.mp_selfjoin(X, [500] * 3, m, 8, mask=[1, 0, 1], P=P, I=I)
    tsk.sync()
    P, I = P.cpu().numpy(), I.cpu().numpy()
    assert np.all(P[500:1000] == 7.0) and np.all(I[500:1000] == 7)
    check_profile(xs[2].astype(np.float64), m, 8, P[1000:1000 + 469], I[1000:1000 + 469])


def test_bad_arguments_raise(tsk):
    X = _cuda(np.zeros(100, dtype=np.float32))
    with pytest.raises(Exception):
        tsk.mp_selfjoin(X, [100], 101)     # m > len
    with pytest.raises(Exception):
        tsk.mp_selfjoin(X, [100], 1)       # m < 2
    with pytest.raises(Exception):
        tsk.set_tile_rows(12)


def test_nonfinite_input_is_reported(tsk):
    x = np.cumsum(np.random.default_rng(107).normal(size=300)).astype(np.float32)
    x[100] = np.nan
    X = _cuda(x)
    tsk.mp_selfjoin(X, [300], 20)
    with pytest.raises(Exception, match="NONFINITE"):
        tsk.sync()
    tsk.sync()  # the error word was cleared


# --- sketch -------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["bf16", "fp32", "fp64"])
def test_sketch_build_matches_oracle(tsk, precision):
    d, n, k = 37, 3001, 12
    T, _ = synth.water_plant(d, n, 50, 2, seed=108)
    R = synth.gaussian_R(d, k, 109)
    S, stats = tsk.ts_sketch_build(_cuda(T.ravel()), _cuda(R), [n], d, precision=precision)
    tsk.sync()
    Tbar, mu, sigma = o.global_znorm(T)
    st = stats.cpu().numpy()[0]
    np.testing.assert_allclose(st[:, 0], mu, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st[:, 1], sigma, rtol=1e-12, atol=1e-12)
    ref = o.sketch(Tbar, R, bf16=(precision == "bf16"))
    got = S.cpu().numpy().astype(np.float64).reshape(k, n)
    mag = np.abs(R.astype(np.float64)).T @ np.abs(Tbar)
    tol = {"bf16": 2e-6, "fp32": 2e-6, "fp64": 1e-13}[precision]
    assert np.all(np.abs(got - ref) <= tol * mag + 1e-30)


def _exact_stat_streams(d, n, seed):
    """(d, n) float32-exact streams whose mean and std both sides compute exactly (or to an ulp).

    Each stream is a random walk on the grid 2^-10, mirrored about a dyadic centre
    (so the mean is exactly the centre), some centres large (the float32 path's
    |mu| term); stream 3 is constant.
    """
    rng = np.random.default_rng(seed)
    half = n // 2
    T = np.empty((d, n))
    for j in range(d):
        w = np.round(np.cumsum(rng.normal(size=half)) * 2.0 ** 10) / 2.0 ** 10
        w -= np.round(w.mean() * 2.0 ** 10) / 2.0 ** 10
        c = [0.0, 1e4, -3.5, 2048.25, -7777.0][j % 5]
        row = np.concatenate([c + w, c - w[::-1]])
        if n % 2:
            row = np.append(row, c)
        T[j] = row
    T[3] = 5.0
    assert np.array_equal(T.astype(np.float32).astype(np.float64), T)
    return T


@pytest.mark.parametrize("d", [24, 40, 100, 300])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_sketch_bf16_rounding_bit_exact(tsk, d, dtype):
    """With R = I the bf16 sketch returns every rounded sample: each must equal the
    oracle's nearest-even bfloat16 of its float64 z-normalised value, bit for bit
    (ragged batch, odd lengths, large offsets, a constant stream)."""
    series = [_exact_stat_streams(d, n, 120 + n) for n in (4099, 1000, 37)]
    T, lens = tsk.pack_batch([torch.as_tensor(s, dtype=dtype) for s in series])
    R = np.eye(d, dtype=np.float32)
    S, _ = tsk.ts_sketch_build(T.cuda(), _cuda(R), lens, d, precision="bf16")
    tsk.sync()
    got = S.cpu().numpy().astype(np.float64)
    off = 0
    for s in series:
        n = s.shape[1]
        ref = o.bf16_round(o.global_znorm(s)[0])
        g = got[off:off + d * n].reshape(d, n)
        bad = np.argwhere(g != ref)
        assert bad.size == 0, (n, bad[:5], g[tuple(bad[0])], ref[tuple(bad[0])])
        off += d * n


@pytest.mark.parametrize("d", [40, 300])
def test_sketch_bf16_single_series_bit_exact(tsk, d):
    """One float32 series whose rows are 16-byte aligned (the tensor-map staging):
    n = 4100 leaves a last tile of 4 time points and d = 40 a last stage of 8
    rows, both read past the series as zeros; R = I, every rounded sample
    bit-exact against the oracle."""
    T = _exact_stat_streams(d, 4100, 410 + d)
    S, _ = tsk.ts_sketch_build(_cuda(T.ravel()), _cuda(np.eye(d, dtype=np.float32)), [4100], d, precision="bf16")
    tsk.sync()
    got = S.cpu().numpy().astype(np.float64).reshape(d, 4100)
    ref = o.bf16_round(o.global_znorm(T)[0])
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


def test_sketch_bf16_many_units_per_cta_bit_exact(tsk):
    """A batch with several times more sketch work units than resident CTAs (each
    CTA walks many units, prefetching across their boundaries): R = I, every
    rounded sample bit-exact against the oracle."""
    d = 260
    series = [_exact_stat_streams(d, 1000 + 37 * i, 300 + i) for i in range(12)]
    T, lens = tsk.pack_batch([torch.as_tensor(s, dtype=torch.float32) for s in series])
    S, _ = tsk.ts_sketch_build(T.cuda(), _cuda(np.eye(d, dtype=np.float32)), lens, d, precision="bf16")
    tsk.sync()
    got = S.cpu().numpy().astype(np.float64)
    off = 0
    for s in series:
        n = s.shape[1]
        ref = o.bf16_round(o.global_znorm(s)[0])
        g = got[off:off + d * n].reshape(d, n)
        assert np.array_equal(g, ref), np.argwhere(g != ref)[:5]
        off += d * n


@pytest.mark.parametrize("k", [65, 100, 130])
def test_sketch_more_than_64_outputs(tsk, k):
    """k beyond one group of 64 tensor-core outputs (the sketch-quality experiment uses k = ceil(sqrt(d)))."""
    d, n = 300, 1500
    rng = np.random.default_rng(110 + k)
    T = np.cumsum(rng.normal(size=(d, n)), axis=1).astype(np.float32)
    R = synth.count_sketch_R(d, k, 111) if k == 100 else synth.gaussian_R(d, k, 111)
    S, _ = tsk.ts_sketch_build(_cuda(T.ravel()), _cuda(R), [n], d, precision="bf16")
    tsk.sync()
    Tbar, _, _ = o.global_znorm(T)
    ref = o.sketch(Tbar, R, bf16=True)
    got = S.cpu().numpy().astype(np.float64).reshape(k, n)
    mag = np.abs(R.astype(np.float64)).T @ np.abs(Tbar)
    assert np.all(np.abs(got - ref) <= 2e-6 * mag + 1e-30)


def test_sketch_ragged_batch_and_count_sketch(tsk):
    d, k = 9, 3
    rng = np.random.default_rng(110)
    series = [np.cumsum(rng.normal(size=(d, n)), axis=1) for n in (70, 333, 1, 64, 129)]
    series[1][4] = 5.0  # a globally constant stream
    R = synth.count_sketch_R(d, k, 111)
    T, lens = tsk.pack_batch([torch.as_tensor(s, dtype=torch.float32) for s in series])
    S, _ = tsk.ts_sketch_build(T.cuda(), _cuda(R), lens, d)
    tsk.sync()
    got = S.cpu().numpy().astype(np.float64)
    off = 0
    for s in series:
        n = s.shape[1]
        ref = o.sketch(o.global_znorm(s.astype(np.float32))[0], R, bf16=True)
        np.testing.assert_allclose(got[off:off + k * n].reshape(k, n), ref, rtol=0, atol=2e-5)
        off += k * n


def test_update_dims_delete_then_add(tsk):
    d, n, k = 10, 2000, 4
    T, _ = synth.random_walks(d, n, 50, 1, seed=112)
    R = synth.gaussian_R(d, k, 113)
    S, _ = tsk.ts_sketch_build(_cuda(T.ravel()), _cuda(R), [n], d)
    S0 = S.clone()
    dims = [3, 7]
    dirty, _ = tsk.ts_sketch_update_dims(S, _cuda(T[dims].ravel()), [n], R[dims], [-1, -1])
    tsk.sync()
    assert list(dirty) == [1] * k
    keep = [j for j in range(d) if j not in dims]
    ref = o.sketch(o.global_znorm(T[keep])[0], R[keep], bf16=True)
    mag = np.abs(R.astype(np.float64)).T @ np.abs(o.global_znorm(T)[0])
    assert np.all(np.abs(S.cpu().numpy().reshape(k, n) - ref) <= 4e-6 * mag)
    tsk.ts_sketch_update_dims(S, _cuda(T[dims].ravel()), [n], R[dims], [1, 1])
    tsk.sync()
    assert np.all(np.abs((S - S0).cpu().numpy().reshape(k, n)) <= 4e-6 * mag)
    Rc = synth.count_sketch_R(d, k, 114)
    dirty, _ = tsk.ts_sketch_update_dims(S, _cuda(T[[0]].ravel()), [n], Rc[[0]], [1])
    assert int(dirty.sum()) == 1 and dirty[int(np.argmax(np.abs(Rc[0])))] == 1


# --- aggregation / discords -----------------------------------------------------

def test_topk_tie_rules_on_hand_built_profiles(tsk):
    P = np.array([[1, 5, 2, 2, 0, 3, 5, 1], [4, 5, 1, 2, 0, 3, 1, 1], [4, 0, 2, 7, 0, 3, 0, 1]], dtype=np.float32)
    I = np.array([[7, 6, 5, 4, 3, 2, 1, 0], [6] * 8, [1] * 8], dtype=np.int32)
    m = 1  # profile length l = n - m + 1 = 8 with n = 8
    idx, grp, score, nn = tsk.discord_topk(_cuda(P.ravel()), _cuda(I.ravel(), torch.int32), [8], 3, m, 4, 2)
    got = list(zip(idx.cpu().numpy()[0], grp.cpu().numpy()[0], score.cpu().numpy()[0], nn.cpu().numpy()[0]))
    want = o.discord_topk(P.astype(np.float64), I, 4, 2)
    assert [(int(a), int(b), float(c), int(e)) for a, b, c, e in got[:3]] == want
    assert got[3][0] == -1 and np.isnan(got[3][2])


def test_rw_small_fp64_end_to_end(tsk):
    """Random-walk workload (d=8, n=2000, m=100, k=4), float64 throughout: exact and sketched discords."""
    wl = synth.workload(1)
    T = wl.series[0]
    d, n, m, k = wl.d, T.shape[1], wl.m, wl.k
    excl = synth.default_excl(m)
    Tt = _cuda(T.ravel(), torch.float64)
    ex = tsk.exact_discords(Tt, [n], d, m, 3, mp_precision="fp64")
    sk = tsk.sketched_discords(Tt, _cuda(wl.R), [n], d, m, 3, sketch_precision="fp64", mp_precision="fp64")
    tsk.sync()
    P_e, I_e = o.profile_streams(T, m, excl)
    ref_e = o.discord_topk(P_e, I_e, 3, m)
    A_e, _ = o.aggregate(P_e)
    got_e = [(int(a), int(b), float(c), int(e)) for a, b, c, e in
             zip(*(v.cpu().numpy()[0] for v in (ex["idx"], ex["grp"], ex["score"], ex["nn"])))]
    check_discords(got_e, ref_e, A_e)
    for g, r in zip(got_e, ref_e):
        if g[0] == r[0]:
            assert g[2] == pytest.approx(r[2], rel=FP64_REL_TOL)
    ref_s, S_ref, P_s, I_s = o.sketched_discords(T, wl.R, m, excl, 3, m)
    np.testing.assert_allclose(sk["S"].cpu().numpy().reshape(k, n), S_ref, rtol=0, atol=1e-12)
    A_s, _ = o.aggregate(P_s)
    got_s = [(int(a), int(b), float(c), int(e)) for a, b, c, e in
             zip(*(v.cpu().numpy()[0] for v in (sk["idx"], sk["grp"], sk["score"], sk["nn"])))]
    check_discords(got_s, ref_s, A_s)
    Pg = sk["P"].cpu().numpy().reshape(k, n)[:, :n - m + 1]
    np.testing.assert_allclose(Pg, P_s, rtol=FP64_REL_TOL, atol=1e-9)


def test_water_plant_bf16_sketched_path_reduced(tsk):
    """Water-plant-like workload at n = 6000: sketched bf16/fp32 path against the bf16-matched oracle."""
    wl = synth.workload(2, scale=6000 / 50000)
    T = wl.series[0]
    d, n, m, k = wl.d, T.shape[1], wl.m, wl.k
    excl = synth.default_excl(m)
    sk = tsk.sketched_discords(_cuda(T.ravel()), _cuda(wl.R), [n], d, m, 5)
    tsk.sync()
    ref, S_ref, P_ref, I_ref = o.sketched_discords(T, wl.R, m, excl, 5, m, bf16=True)
    S = sk["S"].cpu().numpy().astype(np.float64).reshape(k, n)
    P = sk["P"].cpu().numpy().reshape(k, n)
    I = sk["I"].cpu().numpy().reshape(k, n)
    l = n - m + 1
    for g in range(k):
        # the GPU profile of its own float32 sketch against the oracle of that sketch...
        check_profile(S[g], m, excl, P[g, :l], I[g, :l], rows=np.arange(0, l, 7))
    # ...and against the float64 bf16-matched sketch end to end
    fl = 1e-2 * math.sqrt(2 * m)
    err = np.abs(P[:, :l] - P_ref) / np.maximum(P_ref, fl)
    assert err.max() <= MP_REL_TOL, err.max()
    A_ref, _ = o.aggregate(P_ref)
    got = [(int(a), int(b), float(c), int(e)) for a, b, c, e in
           zip(*(v.cpu().numpy()[0] for v in (sk["idx"], sk["grp"], sk["score"], sk["nn"])))]
    check_discords(got, ref, A_ref)


def test_batched_ragged_series_sketched(tsk):
    """Many uneven series in one launch (the batched-monitoring shape, reduced)."""
    d, m, k = 6, 32, 3
    Ts, _ = synth.batched_random_walks(7, 200, 1500, d, m, seed=115)
    R = synth.gaussian_R(d, k, 116)
    T, lens = tsk.pack_batch([torch.as_tensor(s) for s in Ts])
    sk = tsk.sketched_discords(T.cuda(), _cuda(R), lens, d, m, 2)
    tsk.sync()
    excl = synth.default_excl(m)
    for s, Ts_s in enumerate(Ts):
        ref, S_ref, P_ref, I_ref = o.sketched_discords(Ts_s, R, m, excl, 2, m, bf16=True)
        A_ref, _ = o.aggregate(P_ref)
        got = [(int(a), int(b), float(c), int(e)) for a, b, c, e in
               zip(*(v.cpu().numpy()[s] for v in (sk["idx"], sk["grp"], sk["score"], sk["nn"])))]
        check_discords(got, ref, A_ref)
        for g_, r_ in zip(got, ref):
            assert abs(g_[2] - r_[2]) <= MP_REL_TOL * max(r_[2], 1e-2 * math.sqrt(2 * m))


# --- adjoint --------------------------------------------------------------------

@pytest.mark.parametrize("offset", [0.0, 1e4], ids=["centred", "offset1e4"])
def test_backward_matches_oracle_adjoint(tsk, offset):
    """Adjoint of the summed top-3 scores; with a large offset the dense term
    (-a_j - T_bar_j b_j) / sigma_j must still come from well-centred samples."""
    d, n, m, k, K = 12, 3000, 60, 4, 3
    T, _ = synth.random_walks(d, n, m, 3, seed=117)
    T = (T + offset).astype(T.dtype)
    R = synth.gaussian_R(d, k, 118)
    Tt = _cuda(T.ravel()).requires_grad_(True)
    Rt = _cuda(R).requires_grad_(True)
    scores = tsk.DiscordScores.apply(Tt, Rt, [n], d, m, K)
    scores.sum().backward()
    tsk.sync()
    excl = synth.default_excl(m)
    ref, _, _, _ = o.sketched_discords(T, R, m, excl, K, m)
    got_idx = scores.detach().cpu().numpy()
    np.testing.assert_allclose(got_idx[0], [r[2] for r in ref], rtol=MP_REL_TOL)
    sel = [(i, g, nn) for (i, g, _, nn) in ref]
    dT, dR = o.grad_selected(T, R, sel, m)
    gT = Tt.grad.cpu().numpy().reshape(d, n)
    gR = Rt.grad.cpu().numpy()
    scale_T = np.abs(dT).max()
    np.testing.assert_allclose(gT, dT, rtol=0, atol=1e-3 * scale_T)
    np.testing.assert_allclose(gR, dR, rtol=1e-3, atol=1e-3 * np.abs(dR).max())


def test_close_matches_meet_the_tolerance(tsk):
    """Noisy periodic streams: every window has near-repeats (1 - rho ~ 1e-3), where float32
    keys must still tell neighbours apart to 1e-3 relative in the distance."""
    rng = np.random.default_rng(61)
    m, excl = 40, 10
    xs = []
    for n, noise in ((6000, 0.02), (3000, 0.05), (4500, 0.01)):
        t = np.arange(n)
        xs.append((np.sin(2 * np.pi * t / 50) + 0.5 * np.sin(2 * np.pi * t / 17) + noise * rng.normal(size=n))
                  .astype(np.float32))
    out = _streams(tsk, xs, m, excl)
    for x, (P, I) in zip(xs, out):
        l = len(x) - m + 1
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l], rows=np.arange(0, l, 3))


def test_near_exact_repeats_meet_the_tolerance(tsk):
    """Pure sines with noise 1e-3 and 1e-4 of the signal: every window has dozens of repeats
    whose correlations differ by less than float32 resolves (~1e-6 in rho), and the distances
    sit below the floor, where the bar is absolute.  Those rows are re-scanned exactly."""
    rng = np.random.default_rng(67)
    xs, ms = [], []
    for n, period, noise in ((5000, 100, 1e-3), (4000, 64, 1e-4)):
        t = np.arange(n)
        xs.append((np.sin(2 * np.pi * t / period) + noise * rng.normal(size=n)).astype(np.float32))
    m = 64
    excl = int(math.ceil(m / 4))
    out = _streams(tsk, xs, m, excl)
    for x, (P, I) in zip(xs, out):
        l = len(x) - m + 1
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l], rows=np.arange(0, l, 3))


def test_quiet_windows_between_steps_and_spikes(tsk):
    """Flat stretches with sensor noise next to steps (noise 1e-3 of the step) and between sparse
    spikes (noise 1e-4): windows a thousand times quieter than the stream's loudest, whose keys the
    float32 recurrence cannot order; they are re-scanned from centred values."""
    rng = np.random.default_rng(71)
    n = 6000
    steps = np.repeat(rng.integers(0, 5, n // 50 + 1), 50)[:n].astype(float) + 1e-3 * rng.normal(size=n)
    spikes = np.zeros(n)
    spikes[rng.integers(0, n, 60)] = 1.0
    spikes += 1e-4 * rng.normal(size=n)
    for x, m in ((steps, 64), (spikes, 32)):
        x = x.astype(np.float32)
        excl = int(math.ceil(m / 4))
        (P, I), = _streams(tsk, [x], m, excl)
        l = len(x) - m + 1
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l], rows=np.arange(0, l, 3))


def test_near_ties_just_above_the_floor_are_stable(tsk):
    """A sine with noise 1e-2 (1 - rho ~ 1e-4 with ~100 near-repeats per window, within float32's
    resolution of each other): the same input profiled four times meets the bar every time."""
    rng = np.random.default_rng(72)
    n, m = 6000, 40
    x = (np.sin(2 * np.pi * np.arange(n) / 50) + 1e-2 * rng.normal(size=n)).astype(np.float32)
    excl = int(math.ceil(m / 4))
    l = n - m + 1
    rows = np.arange(0, l, 4)
    for _ in range(4):
        (P, I), = _streams(tsk, [x], m, excl)
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l], rows=rows)
