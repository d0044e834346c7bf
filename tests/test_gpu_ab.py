"""GPU parity of the AB join (Def. 6, train/test form) and Alg. 2 on it, against the oracle."""
import numpy as np
import pytest

from oracle import tsk_oracle as o
from paper_2311_03393_gb300 import synth

from helpers import MP_REL_TOL, check_discords, d_floor, within_mp_tol

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


def _check_ab(a, b, m, P, I, rows=None):
    """GPU AB profile of test stream a against training stream b vs the oracle (ties allowed)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    l = len(a) - m + 1
    rows = np.arange(l) if rows is None else np.asarray(rows)
    P_ref, I_ref = o.abjoin_rows(a, b, m, rows)
    fl = d_floor(m)
    Pg = np.asarray(P, np.float64)[rows]
    Ig = np.asarray(I)[rows]
    err = np.abs(Pg - P_ref) / np.maximum(P_ref, fl)
    good = within_mp_tol(Pg, P_ref, m)
    assert good.all(), (float(err.max()), int(rows[np.argmin(good)]))
    diff = np.flatnonzero(Ig != I_ref)
    if diff.size:
        Za, _, _, _ = o.znorm_windows(a, m)
        Zb, _, _, _ = o.znorm_windows(b, m)
        for r in diff:
            i, j = int(rows[r]), int(Ig[r])
            assert 0 <= j < len(b) - m + 1
            dij = float(np.linalg.norm(Za[i] - Zb[j]))
            assert within_mp_tol(dij, P_ref[r], m) and abs(dij - Pg[r]) <= 1e-4 * max(dij, fl), (i, j, dij, P_ref[r])
    return float(err.max())


def _pack(xs, dtype):
    return torch.cat([torch.as_tensor(np.ascontiguousarray(x)).reshape(-1) for x in xs]).to("cuda", dtype)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_ragged_pairs_both_directions(tsk, dtype):
    """Test longer than train, shorter, equal, tiny; several bands and ragged tails."""
    rng = np.random.default_rng(51)
    m = 50
    la = [3100, 900, 1600, 50, 60]
    lb = [1700, 2600, 1600, 300, 50]
    A = [np.cumsum(rng.normal(size=n)) for n in la]
    B = [np.cumsum(rng.normal(size=n)) for n in lb]
    P_a, I_a, P_b, I_b = tsk.mp_abjoin(_pack(A, dtype), _pack(B, dtype), la, lb, m, train_profile=True)
    tsk.sync()
    P_a, I_a, P_b, I_b = (t.cpu().numpy() for t in (P_a, I_a, P_b, I_b))
    oa = np.concatenate([[0], np.cumsum(la)])
    ob = np.concatenate([[0], np.cumsum(lb)])
    for q in range(len(la)):
        pa, ia = P_a[oa[q]:oa[q + 1]], I_a[oa[q]:oa[q + 1]]
        pb, ib = P_b[ob[q]:ob[q + 1]], I_b[ob[q]:ob[q + 1]]
        l_a, l_b = la[q] - m + 1, lb[q] - m + 1
        assert np.all(np.isnan(pa[l_a:])) and np.all(ia[l_a:] == -1)
        assert np.all(np.isnan(pb[l_b:])) and np.all(ib[l_b:] == -1)
        _check_ab(A[q], B[q], m, pa[:l_a], ia[:l_a])
        _check_ab(B[q], A[q], m, pb[:l_b], ib[:l_b])


def test_constant_windows_self_pair_and_no_train_profile(tsk):
    rng = np.random.default_rng(52)
    m, n = 40, 2500
    sq = np.where((np.arange(n) // 250) % 2 == 0, 0.0, 1.0)
    a = np.where(np.arange(n) < 1200, sq, np.cumsum(rng.normal(size=n)))   # constant windows, then a walk
    b = np.roll(sq, 77)                                                     # constant windows and steps
    x = np.cumsum(rng.normal(size=2000))
    P, I = tsk.mp_abjoin(_pack([a, x], torch.float32), _pack([b, x], torch.float32), [n, 2000], [n, 2000], m)
    tsk.sync()
    P, I = P.cpu().numpy(), I.cpu().numpy()
    _check_ab(a.astype(np.float32), b.astype(np.float32), m, P[:n - m + 1], I[:n - m + 1])
    # a series joined with itself: every window finds itself (distance within the float32 floor)
    px = P[n:n + 2000 - m + 1]
    assert np.all(px <= MP_REL_TOL * d_floor(m) + 1e-2)


def test_close_matches_in_both_directions(tsk):
    """Noisy periodic test and training streams (joint period 850): every window has several
    near-repeats in the other stream, within ~1e-6 of each other in rho and in different bands
    or sides, so the choice among them rests on the near-tie candidates' exact re-scores."""
    rng = np.random.default_rng(57)
    m = 40

    def stream(n, noise, phase):
        t = np.arange(n) + phase
        return (np.sin(2 * np.pi * t / 50) + 0.5 * np.sin(2 * np.pi * t / 17) + noise * rng.normal(size=n)
                ).astype(np.float32)

    A = [stream(4000, 0.01, 0), stream(2600, 0.02, 13)]
    B = [stream(5000, 0.01, 300), stream(3500, 0.005, 7)]
    la, lb = [len(x) for x in A], [len(x) for x in B]
    P_a, I_a, P_b, I_b = tsk.mp_abjoin(_pack(A, torch.float32), _pack(B, torch.float32), la, lb, m,
                                       train_profile=True)
    tsk.sync()
    P_a, I_a, P_b, I_b = (t.cpu().numpy() for t in (P_a, I_a, P_b, I_b))
    oa = np.concatenate([[0], np.cumsum(la)])
    ob = np.concatenate([[0], np.cumsum(lb)])
    for q in range(2):
        l_a, l_b = la[q] - m + 1, lb[q] - m + 1
        _check_ab(A[q], B[q], m, P_a[oa[q]:oa[q] + l_a], I_a[oa[q]:oa[q] + l_a], rows=np.arange(0, l_a, 3))
        _check_ab(B[q], A[q], m, P_b[ob[q]:ob[q] + l_b], I_b[ob[q]:ob[q] + l_b], rows=np.arange(0, l_b, 3))


def test_near_exact_repeats_in_both_directions(tsk):
    """Pure sines with noise 1e-4 in test and training: dozens of near-exact repeats per window
    in the other stream, below float32 resolution; those rows are re-scanned exactly."""
    rng = np.random.default_rng(59)
    m = 64
    A = [(np.sin(2 * np.pi * (np.arange(3000) + 5) / 64) + 1e-4 * rng.normal(size=3000)).astype(np.float32)]
    B = [(np.sin(2 * np.pi * np.arange(3500) / 64) + 1e-4 * rng.normal(size=3500)).astype(np.float32)]
    la, lb = [3000], [3500]
    P_a, I_a, P_b, I_b = tsk.mp_abjoin(_pack(A, torch.float32), _pack(B, torch.float32), la, lb, m,
                                       train_profile=True)
    tsk.sync()
    P_a, I_a, P_b, I_b = (t.cpu().numpy() for t in (P_a, I_a, P_b, I_b))
    l_a, l_b = la[0] - m + 1, lb[0] - m + 1
    _check_ab(A[0], B[0], m, P_a[:l_a], I_a[:l_a], rows=np.arange(0, l_a, 3))
    _check_ab(B[0], A[0], m, P_b[:l_b], I_b[:l_b], rows=np.arange(0, l_b, 3))


def test_sketched_and_exact_ab_discords_match_the_oracle(tsk):
    """Planted window in test only; bf16 sketch of train and test with one R, then Alg. 2 and Alg. 3."""
    d, n, m, k, K = 6, 2400, 40, 3, 3
    rng = np.random.default_rng(53)
    t = np.arange(n)
    train = np.stack([rng.uniform(0.5, 2) * np.sin(2 * np.pi * t / q + rng.uniform(0, 6)) + 0.05 * rng.normal(size=n)
                      for q in (20, 25, 40, 50, 30, 60)])
    test = np.stack([rng.uniform(0.5, 2) * np.sin(2 * np.pi * t / q + rng.uniform(0, 6)) + 0.05 * rng.normal(size=n)
                     for q in (20, 25, 40, 50, 30, 60)])
    test[2, 1500:1500 + m] = rng.normal(size=m)
    R = synth.count_sketch_R(d, k, 6)
    Tt = _pack([test], torch.float32)
    Tr = _pack([train], torch.float32)
    Rt = torch.as_tensor(R).cuda()
    res = tsk.ab_discords(Tt, Tr, [n], [n], d, m, K, R=Rt)
    ex = tsk.ab_discords(Tt, Tr, [n], [n], d, m, K)
    tsk.sync()
    # sketched: the oracle's bf16-matched sketches of both series, then AB profiles and Alg. 2
    ref, Pr, _ = o.ab_discords(test.astype(np.float32), train.astype(np.float32), m, K, m, R=R, bf16=True)
    P = res["P"].cpu().numpy().reshape(k, n)
    A_ref, _ = o.aggregate(Pr)
    Sa = o.sketch(o.global_znorm(test.astype(np.float32))[0], R, bf16=True)
    Sb = o.sketch(o.global_znorm(train.astype(np.float32))[0], R, bf16=True)
    for g in range(k):
        _check_ab(Sa[g], Sb[g], m, P[g, :n - m + 1], res["I"].cpu().numpy().reshape(k, n)[g, :n - m + 1],
                  rows=np.arange(0, n - m + 1, 5))
    got = list(zip(*(res[key].cpu().numpy()[0] for key in ("idx", "grp", "score", "nn"))))
    check_discords(got, ref, A_ref, tie_rel=1e-3)
    assert abs(got[0][0] - 1500) < m
    # exact: the d raw streams
    ref_e, Pe, _ = o.ab_discords(test.astype(np.float32), train.astype(np.float32), m, K, m)
    A_e, _ = o.aggregate(Pe)
    got_e = list(zip(*(ex[key].cpu().numpy()[0] for key in ("idx", "grp", "score", "nn"))))
    check_discords(got_e, ref_e, A_e, tie_rel=1e-3)
    assert got_e[0][1] == 2


def test_float64_ab_join_is_exact(tsk):
    """TSK_MP_FP64: every test and training window's profile value to 1e-9, neighbours exactly."""
    rng = np.random.default_rng(54)
    m = 30
    la, lb = [900, 400], [500, 1300]
    A = [np.cumsum(rng.normal(size=n)) for n in la]
    B = [np.cumsum(rng.normal(size=n)) for n in lb]
    A[1][100:160] = 3.0                                     # constant test windows
    P_a, I_a, P_b, I_b = tsk.mp_abjoin(_pack(A, torch.float64), _pack(B, torch.float64), la, lb, m,
                                       train_profile=True, precision="fp64")
    tsk.sync()
    assert P_a.dtype == torch.float64
    P_a, I_a, P_b, I_b = (t.cpu().numpy() for t in (P_a, I_a, P_b, I_b))
    oa = np.concatenate([[0], np.cumsum(la)])
    ob = np.concatenate([[0], np.cumsum(lb)])
    for q in range(2):
        for (x, y, P, I, off) in ((A[q], B[q], P_a, I_a, oa[q]), (B[q], A[q], P_b, I_b, ob[q])):
            l = len(x) - m + 1
            P_ref, I_ref = o.mp_abjoin(x, y, m)
            np.testing.assert_allclose(P[off:off + l], P_ref, rtol=1e-9, atol=1e-9)
            diff = np.flatnonzero(I[off:off + l] != I_ref)
            if diff.size:  # equal distances (e.g. a constant window against non-constant ones: sqrt(m) each)
                Zx, _, _, _ = o.znorm_windows(x, m)
                Zy, _, _, _ = o.znorm_windows(y, m)
                for i in diff:
                    dij = float(np.linalg.norm(Zx[i] - Zy[I[off + i]]))
                    assert abs(dij - P_ref[i]) <= 1e-9 * max(1.0, P_ref[i]), (i, I[off + i], I_ref[i])
