"""The synthetic sketch-quality experiment (Sec. IV, "Synthetic Data").

Random-walk series of d dimensions and n samples; the sketched method (Alg. 1
count sketch with k = ceil(sqrt(d)), Alg. 2 on the k sketch streams, Alg. 3 for
the dimension) returns one discord (i*, j*).  Its quality is the rank of the
exact discord score of (i*, j*), the 1NN distance of window i* in dimension j*
(Def. 6), among the scores of every (window, dimension) pair; a trial succeeds
when that rank lies in the top 0.01 %.  The same is reported after the optional
refinement (the top discord of dimension j*'s own profile), and, for the other
reading of the paper's ranked list, the rank of time i* by its exact
multidimensional score max_j P_j[i] (Def. 5) among all windows.  The speedup
compares the sketched path (sketch + k profiles + top-1 + Alg. 3, and with the
refinement) with the exact d-dimensional path (d profiles + top-1), all timed
with CUDA events.

Every step runs through the library's entry points; the random walks are
drawn on the device (cumulative sums of N(0, 1) steps from a seeded torch
generator).

  python -m paper_2311_03393_gb300.experiments --d 250 500 1000 --trials 20
  python -m paper_2311_03393_gb300.experiments scores --d 1000 --trials 100
  python -m paper_2311_03393_gb300.experiments update --workload 3 --points 1 10
  python -m paper_2311_03393_gb300.experiments sketch --d 1024 --n 100000 --k 16
  python -m paper_2311_03393_gb300.experiments dims --d 1024 --n 20000 --m 144 --k 16 --K 10
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import api, synth


def random_walks_device(d: int, n: int, seed: int, device) -> torch.Tensor:
    """(d, n) float32 random walks, flattened stream-major, from a seeded device generator."""
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    steps = torch.randn((d, n), generator=g, device=device, dtype=torch.float32)
    return torch.cumsum(steps, dim=1).reshape(-1).contiguous()


def _timed(fn):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    out = fn()
    b.record()
    b.synchronize()
    return out, a.elapsed_time(b)


def trial(d: int, n: int, m: int, k: int, seed: int, device, top_frac: float = 1e-4,
          sketch_precision: str = "bf16", R=None, sample_all: int = 0) -> dict:
    """One trial: the sketched discord's rank among all exact (window, dimension) scores.

    R: the (d, k) sketch matrix; default a seeded count sketch (Alg. 1).
    sample_all: also return that many exact scores of uniformly drawn
    (window, dimension) pairs (the "all subsequences" set of the score
    distributions).
    """
    excl = api.default_excl(m)
    T = random_walks_device(d, n, seed, device)
    if R is None:
        R = synth.count_sketch_R(d, k, seed + 1)
    R = torch.as_tensor(R, dtype=torch.float32).to(device)
    l = n - m + 1

    def sketched():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        S, _ = api.ts_sketch_build(T, R, [n], d, precision=sketch_precision)
        ev[1].record()
        P, I = api.mp_selfjoin(S, [n] * k, m, excl)
        ev[2].record()
        idx, grp, score, nn = api.discord_topk(P, I, [n], k, m, 1)
        ev[3].record()
        dims = api.dimension_detection(T, R, [n], d, m, idx, grp, excl, gather=True)
        ev[4].record()
        ev[4].synchronize()
        parts = [ev[q].elapsed_time(ev[q + 1]) for q in range(4)]
        return (idx, grp, dims), parts

    def refine(dims):
        return api.refine_dimensions(dims["T_sel"], [n], 1, m, excl)

    def exact():
        return api.exact_discords(T, [n], d, m, 1, excl)

    torch.cuda.synchronize()
    ((idx, grp, dims), parts), t_sk = _timed(sketched)
    ref, t_ref = _timed(lambda: refine(dims))
    ex, t_ex = _timed(exact)
    i_star = int(idx[0, 0])
    j_star = int(dims["dim"][0, 0])
    i_ref = int(ref["idx"][0, 0])
    P = ex["P"].view(d, n)[:, :l]
    allowed = max(1, int(math.floor(top_frac * d * l)))

    def rank_of(i, j):
        return int((P > P[j, i]).sum().item()) + 1

    rank, rank_ref = rank_of(i_star, j_star), rank_of(i_ref, j_star)
    # the other reading of the ranked list: time indices by their multidimensional score (Def. 5)
    A = P.max(dim=0).values
    time_rank = int((A > A[i_star]).sum().item()) + 1
    extra = {}
    if sample_all:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) + 17)
        flat = P.reshape(-1)
        pick = torch.randint(0, flat.numel(), (int(sample_all),), generator=g, device=device)
        extra["all_sample"] = flat[pick].cpu().numpy().astype(np.float64).tolist()
        extra["score_refined"] = float(P[j_star, i_ref])
    return {**extra, "i": i_star, "j": j_star, "score": float(P[j_star, i_star]), "rank": rank, "allowed": allowed,
            "time_rank": time_rank, "time_top_frac": time_rank / l,
            "success": rank <= allowed, "i_refined": i_ref, "rank_refined": rank_ref,
            "success_refined": rank_ref <= allowed, "exact_i": int(ex["idx"][0, 0]),
            "exact_j": int(ex["grp"][0, 0]), "exact_score": float(ex["score"][0, 0]), "sketched_ms": t_sk,
            "sketched_parts_ms": parts, "refine_ms": t_ref, "exact_ms": t_ex}


def sketch_quality(d: int, n: int = 10000, m: int = 100, trials: int = 100, k: int | None = None,
                   seed: int = synth.SEED_BASE, device=None, sketch_precision: str = "bf16") -> dict:
    """Success rate and speedup over `trials` seeded random-walk trials (Sec. IV synthetic data)."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    k = int(math.ceil(math.sqrt(d))) if k is None else int(k)
    # warm the layouts once (the first call builds and uploads them)
    trial(d, n, m, k, seed + 999983, device, sketch_precision=sketch_precision)
    rows = [trial(d, n, m, k, seed + 7919 * t, device, sketch_precision=sketch_precision) for t in range(trials)]
    sk = float(np.median([r["sketched_ms"] for r in rows]))
    ex = float(np.median([r["exact_ms"] for r in rows]))
    rf = float(np.median([r["refine_ms"] for r in rows]))
    parts = np.median(np.array([r["sketched_parts_ms"] for r in rows]), axis=0)
    return {"d": d, "n": n, "m": m, "k": k, "trials": trials, "top_frac": 1e-4,
            "success_rate": float(np.mean([r["success"] for r in rows])),
            "success_rate_refined": float(np.mean([r["success_refined"] for r in rows])),
            "median_rank": float(np.median([r["rank"] for r in rows])),
            "median_rank_refined": float(np.median([r["rank_refined"] for r in rows])),
            "exact_hit_rate": float(np.mean([r["i"] == r["exact_i"] and r["j"] == r["exact_j"] for r in rows])),
            "median_time_rank": float(np.median([r["time_rank"] for r in rows])),
            "time_top1pct_rate": float(np.mean([r["time_top_frac"] <= 0.01 for r in rows])),
            "sketched_ms": sk, "sketched_parts_ms": {"sketch": parts[0], "profiles": parts[1], "topk": parts[2],
                                                     "dims": parts[3]},
            "refine_ms": rf, "exact_ms": ex, "speedup": ex / sk if sk > 0 else None,
            "speedup_with_refinement": ex / (sk + rf) if sk + rf > 0 else None,
            "sketch_precision": sketch_precision}


def _summary(v) -> dict:
    v = np.asarray(v, dtype=np.float64)
    q = np.quantile(v, [0.01, 0.05, 0.25, 0.5, 0.75, 0.95, 0.99])
    return {"count": int(v.size), "mean": float(v.mean()), "std": float(v.std()),
            "quantiles": {f"{p:g}": float(x) for p, x in zip([0.01, 0.05, 0.25, 0.5, 0.75, 0.95, 0.99], q)}}


def score_distribution(d: int = 1000, n: int = 10000, m: int = 100, trials: int = 100, k: int | None = None,
                       seed: int = synth.SEED_BASE, device=None, sample_all: int = 4096,
                       sketch_precision: str = "bf16") -> dict:
    """The discord-score distributions of Sec. IV's synthetic experiment (its density figure, d = 1000).

    Three sets of exact discord scores (1NN distances, Def. 6) over the trials:
    all subsequences (a uniform sample of (window, dimension) pairs per trial),
    the exact discords (Def. 4 top-1 of the exact d-dimensional path) and the
    sketched discords (the exact score of the (i*, j*) the sketched path
    returns, before and after the refinement).  Reported as quantiles, with the
    exact discords' distance from the sketched discords' mean in units of the
    sketched discords' standard deviation (the statistic the paper quotes for
    its real datasets), and each set's distance from the all-subsequence mean.
    """
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    k = int(math.ceil(math.sqrt(d))) if k is None else int(k)
    trial(d, n, m, k, seed + 999983, device, sketch_precision=sketch_precision)
    rows = [trial(d, n, m, k, seed + 7919 * t, device, sketch_precision=sketch_precision, sample_all=sample_all)
            for t in range(trials)]
    allv = np.concatenate([r["all_sample"] for r in rows])
    allv = allv[np.isfinite(allv)]
    ex = np.array([r["exact_score"] for r in rows])
    sk = np.array([r["score"] for r in rows])
    rf = np.array([r["score_refined"] for r in rows])
    sd_sk = float(sk.std()) or float("nan")
    sd_rf = float(rf.std()) or float("nan")
    return {"d": d, "n": n, "m": m, "k": k, "trials": trials, "sketch_precision": sketch_precision,
            "all_subsequences": _summary(allv), "exact_discords": _summary(ex), "sketched_discords": _summary(sk),
            "sketched_refined_discords": _summary(rf),
            "exact_vs_sketched_sd": float((ex.mean() - sk.mean()) / sd_sk),
            "exact_vs_refined_sd": float((ex.mean() - rf.mean()) / sd_rf),
            "sketched_vs_all_sd": float((sk.mean() - allv.mean()) / allv.std()),
            "exact_vs_all_sd": float((ex.mean() - allv.mean()) / allv.std()),
            "sketched_over_exact": float(np.mean(sk / ex)),
            "success_rate": float(np.mean([r["success"] for r in rows])),
            "time_rank_median": float(np.median([r["time_rank"] for r in rows])),
            "time_top_0.01pct_rate": float(np.mean([r["time_rank"] <= max(1, int(1e-4 * (n - m + 1)))
                                                    for r in rows])),
            "time_top_1pct_rate": float(np.mean([r["time_top_frac"] <= 0.01 for r in rows]))}


def sketch_throughput(d: int, n: int, k: int, reps: int = 5, seed: int = synth.SEED_BASE, precision: str = "bf16",
                      device=None) -> dict:
    """Time ts_sketch_build's sketch kernel on one (d, n) random-walk series with a Gaussian R (d x k).

    Reports the kernel's device time per launch (library events) and its
    algorithmic bytes per second, 4 d n (T) + 4 k n (S).
    """
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    T = random_walks_device(d, n, seed, device)
    R = torch.from_numpy(synth.gaussian_R(d, k, seed + 1)).to(device)
    for _ in range(3):
        api.ts_sketch_build(T, R, [n], d, precision=precision)
    api.sync()
    api.profile_enable(True)
    api.profile_read("sketch")
    for _ in range(reps):
        api.ts_sketch_build(T, R, [n], d, precision=precision)
    api.sync()
    ms, launches = api.profile_read("sketch")
    api.profile_enable(False)
    per = ms / max(launches, 1)
    return {"d": d, "n": n, "k": k, "precision": precision, "ms_per_launch": per,
            "gb_per_s": (4.0 * d * n + 4.0 * k * n) / (per / 1e3) / 1e9}


def dims_throughput(d: int, n: int, m: int, k: int, K: int, reps: int = 5, seed: int = synth.SEED_BASE,
                    device=None) -> dict:
    """Time Alg. 3 (the dimension scan) for the K top sketch discords of one random-walk series.

    The series is (d, n) random walks, R a seeded Gaussian d x k (every
    dimension in every group, so each discord scans all d streams), the
    discords those of the bf16 sketch's profiles.  Reports the scan kernel's
    device time per launch (library events) and its FMA rate: each (discord,
    stream) scores every window with an m-sample dot product.
    """
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    excl = api.default_excl(m)
    T = random_walks_device(d, n, seed, device)
    R = torch.from_numpy(synth.gaussian_R(d, k, seed + 1)).to(device)
    S, _ = api.ts_sketch_build(T, R, [n], d, precision="bf16")
    P, I = api.mp_selfjoin(S, [n] * k, m, excl)
    idx, grp, _, _ = api.discord_topk(P, I, [n], k, m, K)
    for _ in range(2):
        api.dimension_detection(T, R, [n], d, m, idx, grp, excl)
    api.sync()
    api.profile_enable(True)
    api.profile_read("dims")
    for _ in range(reps):
        api.dimension_detection(T, R, [n], d, m, idx, grp, excl)
    api.sync()
    ms, launches = api.profile_read("dims")
    api.profile_enable(False)
    per = ms / max(launches, 1)
    found = int((idx[0] >= 0).sum().item())
    fmas = float(found) * d * (n - m + 1) * m
    return {"d": d, "n": n, "m": m, "k": k, "K": K, "discords": found, "ms_per_launch": per,
            "tfma_per_s": fmas / (per / 1e3) / 1e12}


def update_throughput(index: int = 3, points: int = 1, reps: int = 5, seed: int = synth.SEED_BASE,
                      device=None) -> dict:
    """Time the incremental profile after point updates against a full re-profile.

    Workload `index`'s first series is sketched (bf16), its k sketch streams
    profiled; then `points` samples of one dimension change (ts_sketch_point_update
    moves every sketch stream at those times) and the profiles follow with
    mp_selfjoin_update.  Reports both times (CUDA events) and the speedup.
    """
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    wl = synth.workload(index, seed=seed + index)
    T0 = wl.series[0]
    d, n = T0.shape
    m, k = wl.m, wl.k
    excl = api.default_excl(m)
    T = torch.from_numpy(np.ascontiguousarray(T0.ravel())).to(device)
    R = torch.from_numpy(wl.R).to(device)
    S, stats = api.ts_sketch_build(T, R, [n], d, precision="bf16")
    lens = [n] * k
    P, I = api.mp_selfjoin(S, lens, m, excl)
    rng = np.random.default_rng(seed)
    t_full, t_upd = [], []
    for r in range(reps + 1):
        ts = sorted(int(x) for x in rng.integers(0, n, points))
        ups = [(0, int(rng.integers(0, d)), t, float(rng.normal())) for t in ts]
        api.ts_sketch_point_update(S, stats, R, [n], d, *zip(*ups), T=T, precision="bf16")
        pts = [(g, t) for g in range(k) for t in ts]
        _, ms_u = _timed(lambda: api.mp_selfjoin_update(S, lens, m, P, I, pts, excl))
        _, ms_f = _timed(lambda: api.mp_selfjoin(S, lens, m, excl))
        if r:
            t_upd.append(ms_u)
            t_full.append(ms_f)
    mu, mf = float(np.median(t_upd)), float(np.median(t_full))
    return {"workload": wl.name, "streams": k, "n": n, "m": m, "points": points, "update_ms": mu, "full_ms": mf,
            "speedup": mf / mu if mu > 0 else None}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd")
    q = sub.add_parser("quality", help="success rate and speedup over d (the default)")
    q.add_argument("--d", type=int, nargs="+", default=[250, 500, 1000, 2500, 5000, 7500, 10000])
    q.add_argument("--n", type=int, default=10000)
    q.add_argument("--m", type=int, default=100)
    q.add_argument("--trials", type=int, default=100)
    q.add_argument("--seed", type=int, default=synth.SEED_BASE)
    q.add_argument("--sketch-precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    t = sub.add_parser("sketch", help="throughput of the sketch kernel on one series")
    t.add_argument("--d", type=int, default=1024)
    t.add_argument("--n", type=int, default=100000)
    t.add_argument("--k", type=int, default=16)
    t.add_argument("--reps", type=int, default=5)
    t.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    e = sub.add_parser("scores", help="discord-score distributions (all, exact, sketched) at one d")
    e.add_argument("--d", type=int, default=1000)
    e.add_argument("--n", type=int, default=10000)
    e.add_argument("--m", type=int, default=100)
    e.add_argument("--trials", type=int, default=100)
    e.add_argument("--seed", type=int, default=synth.SEED_BASE)
    u = sub.add_parser("update", help="incremental profile after point updates vs a full re-profile")
    u.add_argument("--workload", type=int, default=3)
    u.add_argument("--points", type=int, nargs="+", default=[1, 10])
    u.add_argument("--reps", type=int, default=5)
    a = sub.add_parser("dims", help="time of the Alg. 3 dimension scan on one series")
    a.add_argument("--d", type=int, default=1024)
    a.add_argument("--n", type=int, default=20000)
    a.add_argument("--m", type=int, default=144)
    a.add_argument("--k", type=int, default=16)
    a.add_argument("--K", type=int, default=10)
    a.add_argument("--reps", type=int, default=5)
    argv = list(argv) if argv is not None else None
    import sys
    raw = sys.argv[1:] if argv is None else argv
    if not raw or raw[0].startswith("-"):
        raw = ["quality"] + raw
    args = ap.parse_args(raw)
    if args.cmd == "sketch":
        print(json.dumps(sketch_throughput(args.d, args.n, args.k, args.reps, precision=args.precision)), flush=True)
        return
    if args.cmd == "scores":
        print(json.dumps(score_distribution(args.d, args.n, args.m, args.trials, seed=args.seed)), flush=True)
        return
    if args.cmd == "update":
        for p in args.points:
            print(json.dumps(update_throughput(args.workload, p, args.reps)), flush=True)
        return
    if args.cmd == "dims":
        print(json.dumps(dims_throughput(args.d, args.n, args.m, args.k, args.K, args.reps)), flush=True)
        return
    for d in args.d:
        out = sketch_quality(d, args.n, args.m, args.trials, seed=args.seed, sketch_precision=args.sketch_precision)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
