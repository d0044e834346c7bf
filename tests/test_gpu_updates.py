"""GPU parity of the point update of the sketch (Sec. III-C) against the oracle."""
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


def _setup(seed, d=9, k=4, lens=(1500, 700)):
    rng = np.random.default_rng(seed)
    Ts = [np.cumsum(rng.normal(size=(d, n)), axis=1).astype(np.float32) for n in lens]
    R = synth.gaussian_R(d, k, seed + 1)
    ups = [(0, 3, 0, 1.5), (0, 3, 0, -0.25), (0, 8, lens[0] - 1, -3.0), (1, 0, 350, 2.0), (1, 5, 12, 0.75),
           (0, 4, 777, 10.0)]
    return Ts, R, ups


def _apply(Ts, ups):
    """The stored float32 samples after the updates (repeated points merged, deltas summed)."""
    merged = {}
    for s, j, i, dl in ups:
        merged[(s, j, i)] = merged.get((s, j, i), 0.0) + dl
    T2 = [t.copy() for t in Ts]
    for (s, j, i), dl in merged.items():
        T2[s][j, i] = np.float32(np.float64(Ts[s][j, i]) + dl)
    return T2


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_point_update_with_T_keeps_S_the_sketch_of_the_updated_series(tsk, precision):
    Ts, R, ups = _setup(81)
    d, k = R.shape
    lens = [t.shape[1] for t in Ts]
    T = torch.cat([torch.from_numpy(t.ravel()) for t in Ts]).cuda()
    Rt = torch.from_numpy(R).cuda()
    S, stats = tsk.ts_sketch_build(T, Rt, lens, d, precision=precision)
    tsk.ts_sketch_point_update(S, stats, Rt, lens, d, *zip(*ups), T=T, precision=precision)
    tsk.sync()
    T2 = _apply(Ts, ups)
    got_T = T.cpu().numpy()
    np.testing.assert_array_equal(got_T, np.concatenate([t.ravel() for t in T2]))
    got = S.cpu().numpy().astype(np.float64)
    off = 0
    for s, t in enumerate(Ts):
        _, mu, sg = o.global_znorm(t)
        want = o.sketch(o.znorm_with(T2[s], mu, sg), R, bf16=(precision == "bf16"))
        n = t.shape[1]
        mag = np.abs(R.T) @ np.abs(o.znorm_with(T2[s], mu, sg)) + 1.0
        err = np.abs(got[off:off + k * n].reshape(k, n) - want)
        assert np.all(err <= 4e-6 * mag), float((err / mag).max())
        off += k * n


def test_point_update_without_T_is_the_paper_formula(tsk):
    Ts, R, ups = _setup(82)
    d, k = R.shape
    lens = [t.shape[1] for t in Ts]
    T = torch.cat([torch.from_numpy(t.astype(np.float64).ravel()) for t in Ts]).cuda()
    Rt = torch.from_numpy(R).cuda()
    S, stats = tsk.ts_sketch_build(T, Rt, lens, d, precision="fp64")
    tsk.ts_sketch_point_update(S, stats, Rt, lens, d, *zip(*ups), precision="fp64")
    tsk.sync()
    got = S.cpu().numpy()
    off = 0
    for s, t in enumerate(Ts):
        Tb, mu, sg = o.global_znorm(t.astype(np.float64))
        want = o.point_update(o.sketch(Tb, R), R, sg, [(j, i, dl) for (q, j, i, dl) in ups if q == s])
        n = t.shape[1]
        np.testing.assert_allclose(got[off:off + k * n].reshape(k, n), want, rtol=0, atol=1e-11)
        off += k * n


def test_point_update_rejects_bad_input_and_reprofile_matches(tsk):
    Ts, R, ups = _setup(83, lens=(2400,))
    d, k = R.shape
    T = torch.from_numpy(Ts[0].ravel()).cuda()
    Rt = torch.from_numpy(R).cuda()
    S, stats = tsk.ts_sketch_build(T, Rt, [2400], d, precision="fp32")
    with pytest.raises(tsk.api.N.TskError):
        tsk.ts_sketch_point_update(S, stats, Rt, [2400], d, [0], [d], [5], [1.0], T=T, precision="fp32")
    with pytest.raises(tsk.api.N.TskError):
        tsk.ts_sketch_point_update(S, stats, Rt, [2400], d, [0], [1], [5], [1.0], precision="bf16")
    tsk.ts_sketch_point_update(S, stats, Rt, [2400], d, [0, 0], [2, 7], [1000, 1010], [25.0, -25.0], T=T,
                               precision="fp32")
    m = 64
    P, I = tsk.mp_selfjoin(S, [2400] * k, m)
    tsk.sync()
    Sn = S.cpu().numpy().astype(np.float64).reshape(k, 2400)
    l = 2400 - m + 1
    for g in range(k):
        check_profile(Sn[g], m, synth.default_excl(m), P.cpu().numpy()[g * 2400:g * 2400 + l],
                      I.cpu().numpy()[g * 2400:g * 2400 + l], rows=np.arange(900, 1100))
