"""GPU parity of the incremental profile after point updates (Sec. III-C point
updates, followed by the streaming use Sec. III-B names) against the oracle's
whole profile of the updated streams (Def. 6)."""
import numpy as np
import pytest

from oracle import tsk_oracle as o
from paper_2311_03393_gb300 import synth

from helpers import check_profile

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


def _pack(xs):
    return torch.cat([torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)) for x in xs]).cuda()


def _run(tsk, xs, m, excl, changes):
    """Profile xs, apply changes {(stream, t): delta} on the device copy, update; return new P, I and streams."""
    lens = [len(x) for x in xs]
    X = _pack(xs)
    P, I = tsk.mp_selfjoin(X, lens, m, excl)
    before = (P.clone(), I.clone())
    off = np.concatenate([[0], np.cumsum(lens)])
    new = [x.astype(np.float32).copy() for x in xs]
    for (q, t), dl in changes.items():
        new[q][t] = np.float32(new[q][t] + dl)
        X[int(off[q]) + t] = float(new[q][t])
    tsk.mp_selfjoin_update(X, lens, m, P, I, list(changes), excl)
    tsk.sync()
    return new, P.cpu().numpy(), I.cpu().numpy(), before, off


def _rows(l, changes, q, m, stride=5):
    """Rows to compare: every window near a change and a regular sample of the rest."""
    near = [np.arange(max(0, t - 2 * m), min(l, t + m)) for (qq, t) in changes if qq == q]
    return np.unique(np.concatenate(near + [np.arange(0, l, stride)]))


def test_update_matches_the_oracle_profile_of_the_updated_streams(tsk):
    """Few changed windows (< 1.5% of a stream): the incremental path."""
    rng = np.random.default_rng(91)
    m, excl = 64, 16
    xs = [np.cumsum(rng.normal(size=n)) for n in (16000, 3000, 14100)]
    changes = {(0, 1234): 4.0, (0, 1240): -2.5, (2, 3): 3.0, (2, 14099): -5.0}
    new, P, I, before, off = _run(tsk, xs, m, excl, changes)
    for q in (0, 2):
        l = len(new[q]) - m + 1
        check_profile(new[q].astype(np.float64), m, excl, P[off[q]:off[q] + l], I[off[q]:off[q] + l],
                      rows=_rows(l, changes, q, m))
    # a stream without points is left as it was
    np.testing.assert_array_equal(P[off[1]:off[2]], before[0].cpu().numpy()[off[1]:off[2]])
    np.testing.assert_array_equal(I[off[1]:off[2]], before[1].cpu().numpy()[off[1]:off[2]])


def test_update_where_the_change_creates_and_removes_nearest_neighbours(tsk):
    """A planted near-repeat is destroyed: rows whose old neighbour was in the changed windows
    must be re-scanned, and a zero change re-profiles its windows to the same values."""
    rng = np.random.default_rng(92)
    m, excl = 50, 12
    n = 12000
    x = np.cumsum(rng.normal(size=n))
    x[9000:9000 + m] = x[500:500 + m] + 0.01 * rng.normal(size=m)  # near-repeat of window 500 at 9000
    changes = {(0, 9000 + t): float(rng.normal()) * 3.0 for t in range(0, m, 7)}  # destroy it
    changes[(0, 4200)] = 0.0  # a point that does not change anything
    new, P, I, _, _ = _run(tsk, [x], m, excl, changes)
    l = n - m + 1
    rows = np.unique(np.concatenate([_rows(l, changes, 0, m, stride=7), np.arange(450, 560)]))
    check_profile(new[0].astype(np.float64), m, excl, P[:l], I[:l], rows=rows)


def test_many_changes_take_the_whole_profile(tsk):
    """Past ~1.5% changed windows the touched streams are profiled whole; same result."""
    rng = np.random.default_rng(95)
    m, excl = 40, 10
    xs = [np.cumsum(rng.normal(size=n)) for n in (3000, 2500)]
    changes = {(0, int(t)): float(rng.normal()) for t in rng.choice(3000, 40, replace=False)}
    new, P, I, before, off = _run(tsk, xs, m, excl, changes)
    l = len(new[0]) - m + 1
    check_profile(new[0].astype(np.float64), m, excl, P[:l], I[:l], rows=np.arange(0, l, 3))
    np.testing.assert_array_equal(P[off[1]:off[2]], before[0].cpu().numpy()[off[1]:off[2]])


def test_update_of_sketch_streams_after_a_point_update_of_the_series(tsk):
    """ts_sketch_point_update moves every sketch stream at t; the profiles follow incrementally."""
    rng = np.random.default_rng(93)
    d, k, n, m = 7, 3, 12000, 40
    excl = synth.default_excl(m)
    T = np.cumsum(rng.normal(size=(d, n)), axis=1).astype(np.float32)
    R = synth.gaussian_R(d, k, 94)
    Tt = torch.from_numpy(T.ravel()).cuda()
    Rt = torch.from_numpy(R).cuda()
    S, stats = tsk.ts_sketch_build(Tt, Rt, [n], d, precision="fp32")
    P, I = tsk.mp_selfjoin(S, [n] * k, m, excl)
    ups = [(0, 2, 7000, 6.0), (0, 5, 7001, -4.0), (0, 0, n - 1, 3.0)]
    tsk.ts_sketch_point_update(S, stats, Rt, [n], d, *zip(*ups), T=Tt, precision="fp32")
    pts = [(g, t) for g in range(k) for (_, _, t, _) in ups]
    tsk.mp_selfjoin_update(S, [n] * k, m, P, I, pts, excl)
    tsk.sync()
    Sn = S.cpu().numpy().astype(np.float64).reshape(k, n)
    Pn, In = P.cpu().numpy().reshape(k, n), I.cpu().numpy().reshape(k, n)
    l = n - m + 1
    for g in range(k):
        check_profile(Sn[g], m, excl, Pn[g, :l], In[g, :l], rows=_rows(l, pts, g, m, stride=9))


def test_update_with_constant_windows(tsk):
    """Square waves (constant windows), a change inside a flat stretch and one that makes a
    window constant."""
    m, excl = 32, 8
    n = 9000
    t = np.arange(n)
    x = np.where((t // 300) % 2 == 0, 0.0, 1.0) + 0.0
    x[1500:1510] += np.linspace(0, 1, 10)
    changes = {(0, 620): 0.5, (0, 1505): -0.3}
    new, P, I, _, _ = _run(tsk, [x], m, excl, changes)
    l = n - m + 1
    check_profile(new[0].astype(np.float64), m, excl, P[:l], I[:l], rows=_rows(l, changes, 0, m, stride=4))


def test_update_of_near_exact_repeats(tsk):
    """A sine with noise 1e-4: every window has dozens of near-exact repeats; a changed point
    makes the windows over it the only ones far from them, and the rest keep exact choices."""
    rng = np.random.default_rng(96)
    m, excl = 64, 16
    n = 12000
    x = np.sin(2 * np.pi * np.arange(n) / 64) + 1e-4 * rng.normal(size=n)
    changes = {(0, 5000): 0.3, (0, 9100): -0.01}
    new, P, I, _, _ = _run(tsk, [x], m, excl, changes)
    l = n - m + 1
    check_profile(new[0].astype(np.float64), m, excl, P[:l], I[:l], rows=_rows(l, changes, 0, m, stride=6))


def test_update_rejects_points_out_of_range(tsk):
    X = torch.zeros(1000, device="cuda")
    P, I = tsk.mp_selfjoin(torch.randn(1000, device="cuda"), [1000], 20)
    with pytest.raises(Exception):
        tsk.mp_selfjoin_update(X, [1000], 20, P, I, [(0, 1000)])
    with pytest.raises(Exception):
        tsk.mp_selfjoin_update(X, [1000], 20, P, I, [(1, 5)])
