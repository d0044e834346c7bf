"""Parity at the full workload sizes, on outputs the oracle can compute one by one.

At these sizes the oracle cannot profile every row within a test, so each check
samples rows (plus every reported discord row) and compares them with the
oracle's definition-based rows (Def. 6), computed in spawn-started worker
processes.  The launch configuration is the benchmark's (automatic work units).
"""
import numpy as np
import pytest

from oracle import tsk_oracle as o
from paper_2311_03393_gb300 import synth

from helpers import MP_REL_TOL, d_floor, within_mp_tol
from oracle_pool import pool_profiles, pool_rows

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


def _check_rows(streams_ref, P_gpu, I_gpu, m, excl, picks, seed):
    """Oracle rows of each reference stream vs the GPU profile at the same rows.

    picks[q] = (number of random rows, extra rows) for stream q.  Returns
    {(q, row): oracle P} for every checked row.
    """
    rng = np.random.default_rng(seed)
    jobs = []
    for q, x in enumerate(streams_ref):
        l = len(x) - m + 1
        rows = np.unique(np.concatenate([rng.choice(l, picks[q][0], replace=False),
                                         np.asarray(picks[q][1], dtype=np.int64)])).astype(np.int64)
        jobs.append((np.asarray(x, np.float64), m, excl, rows))
    res = pool_rows(jobs)
    fl = d_floor(m)
    ref = {}
    for q, ((x, _, _, rows), (P_ref, I_ref), Pg, Ig) in enumerate(zip(jobs, res, P_gpu, I_gpu)):
        Pg = np.asarray(Pg, np.float64)[rows]
        Ig = np.asarray(Ig)[rows]
        assert np.all(np.isfinite(P_ref)) and np.all(np.isfinite(Pg))
        err = np.abs(Pg - P_ref) / np.maximum(P_ref, fl)
        good = within_mp_tol(Pg, P_ref, m)
        assert good.all(), (q, float(err.max()), int(rows[np.argmin(good)]))
        diff = np.where(Ig != I_ref)[0]
        if diff.size:  # a different neighbour must be an equally near one
            Z, _, _, _ = o.znorm_windows(x, m)
            for r in diff:
                i, j = int(rows[r]), int(Ig[r])
                assert j >= 0 and abs(i - j) >= excl, (i, j)
                dij = float(np.sqrt(((Z[i] - Z[j]) ** 2).sum()))
                assert within_mp_tol(dij, P_ref[r], m), (i, j, dij, P_ref[r])
        ref.update({(q, int(i)): float(p) for i, p in zip(rows, P_ref)})
    return ref


def _split(t, count, n):
    a = t.cpu().numpy()
    return [a[q * n:(q + 1) * n] for q in range(count)]


@pytest.mark.parametrize("index,K", [(2, 5), (3, 10)], ids=["water_d51_n50000", "traffic_d1024_n100000"])
def test_full_size_sketched_and_exact(tsk, index, K):
    wl = synth.workload(index)
    T = wl.series[0]
    d, n = T.shape
    m, k = wl.m, wl.k
    excl = synth.default_excl(m)
    Tt = torch.from_numpy(np.ascontiguousarray(T.ravel())).cuda()
    sk = tsk.sketched_discords(Tt, torch.from_numpy(wl.R).cuda(), [n], d, m, K)
    ex = tsk.exact_discords(Tt, [n], d, m, K)
    tsk.sync()
    # sketched path against the float64 sketch of the bf16-rounded operands
    S_ref = o.sketch(o.global_znorm(T)[0], wl.R, bf16=True)
    idx, grp, score = (sk[key].cpu().numpy()[0] for key in ("idx", "grp", "score"))
    extra = [[int(i) for i, g in zip(idx, grp) if g == q and i >= 0] for q in range(k)]
    ref = _check_rows(S_ref, _split(sk["P"], k, n), _split(sk["I"], k, n), m, excl,
                      [(24, extra[q]) for q in range(k)], seed=500 + index)
    # the reported scores are the oracle's profile values at the reported rows
    for i, g, s in zip(idx, grp, score):
        if i >= 0:
            pr = ref[(int(g), int(i))]
            assert within_mp_tol(float(s), pr, m), (i, g, s, pr)
    # exact path (one profile per raw dimension) on a sample of dimensions
    rng = np.random.default_rng(600 + index)
    dims = rng.choice(d, min(d, 12), replace=False)
    Pe, Ie = _split(ex["P"], d, n), _split(ex["I"], d, n)
    _check_rows([T[j] for j in dims], [Pe[j] for j in dims], [Ie[j] for j in dims], m, excl,
                [(8, [])] * len(dims), seed=700 + index)


def test_full_size_batched_series(tsk):
    wl = synth.workload(4)
    d, m, k = wl.d, wl.m, wl.k
    excl = synth.default_excl(m)
    T, lens = tsk.pack_batch([torch.as_tensor(s) for s in wl.series])
    T = T.cuda()
    sk = tsk.sketched_discords(T, torch.from_numpy(wl.R).cuda(), lens, d, m, 1)
    tsk.sync()
    P = sk["P"].cpu().numpy()
    I = sk["I"].cpu().numpy()
    idx = sk["idx"].cpu().numpy()
    grp = sk["grp"].cpu().numpy()
    starts = np.concatenate([[0], np.cumsum([k * n for n in lens])])
    rng = np.random.default_rng(800)
    for s in rng.choice(len(lens), 6, replace=False):
        n = lens[s]
        S_ref = o.sketch(o.global_znorm(wl.series[s])[0], wl.R, bf16=True)
        Ps = [P[starts[s] + g * n: starts[s] + (g + 1) * n] for g in range(k)]
        Is = [I[starts[s] + g * n: starts[s] + (g + 1) * n] for g in range(k)]
        i1, g1 = int(idx[s, 0]), int(grp[s, 0])
        _check_rows(S_ref, Ps, Is, m, excl, [(12, [i1] if g == g1 else []) for g in range(k)],
                    seed=900 + int(s))


def test_full_size_gradient_against_central_differences(tsk):
    """Adjoint of the summed top-3 scores (d=64, n=20000, m=100, k=8) vs float64 central differences."""
    wl = synth.workload(5)
    T = wl.series[0].astype(np.float64)
    d, n = T.shape
    m, k, K = wl.m, wl.k, 3
    excl = synth.default_excl(m)
    R = wl.R.astype(np.float64)
    # the oracle's own forward (whole profiles; rows spread over worker processes)
    S = o.sketch(o.global_znorm(T)[0], R)
    P, I = pool_profiles(list(S), m, excl)
    ref = o.discord_topk(P, I, K, m)
    sel = [(i, g, nn) for (i, g, _, nn) in ref]
    # the GPU forward and adjoint (float32 sketch)
    Tt = torch.from_numpy(np.ascontiguousarray(wl.series[0].ravel())).float().cuda().requires_grad_(True)
    Rt = torch.from_numpy(wl.R).float().cuda().requires_grad_(True)
    scores = tsk.DiscordScores.apply(Tt, Rt, [n], d, m, K)
    scores.sum().backward()
    tsk.sync()
    got = tsk.sketched_discords(Tt.detach(), Rt.detach(), [n], d, m, K, sketch_precision="fp32")
    got_sel = [tuple(int(got[key].cpu().numpy()[0][r]) for key in ("idx", "grp", "nn")) for r in range(K)]
    assert got_sel == sel, (got_sel, sel)
    sc = scores.detach().cpu().numpy()[0]
    for s, (_, _, a, _) in zip(sc, ref):
        assert abs(s - a) <= MP_REL_TOL * a
    gT = Tt.grad.cpu().numpy().reshape(d, n).astype(np.float64)
    gR = Rt.grad.cpu().numpy().astype(np.float64)
    # 200 coordinates of T: 100 inside the selected windows, 100 uniform
    rng = np.random.default_rng(1000)
    support = [(j, t) for (i, g, nn) in sel for t in list(range(i, i + m)) + list(range(nn, nn + m))
               for j in range(d)]
    coords = [support[q] for q in rng.choice(len(support), 100, replace=False)]
    coords += [(int(a), int(b)) for a, b in zip(rng.integers(0, d, 100), rng.integers(0, n, 100))]
    h = 1e-4
    fdT = o.central_difference(lambda X: o.selected_loss(X, R, sel, m), T, coords, h)
    gsel = np.array([gT[c] for c in coords])
    scale = 1e-2 * np.abs(fdT).max()
    rel = np.abs(gsel - fdT) / np.maximum(np.abs(fdT), scale)
    assert rel.max() <= 1e-3, (float(rel.max()), coords[int(np.argmax(rel))])
    cR = [(j, g) for j in range(d) for g in range(k)]
    fdR = o.central_difference(lambda X: o.selected_loss(T, X, sel, m), R, cR, h)
    gRs = np.array([gR[c] for c in cR])
    relR = np.abs(gRs - fdR) / np.maximum(np.abs(fdR), 1e-2 * np.abs(fdR).max())
    assert relR.max() <= 1e-3, float(relR.max())
