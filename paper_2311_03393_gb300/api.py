"""Python face of libtsketch: the five C entry points with the same names, over
torch CUDA tensors (torch supplies device memory and the current stream only;
every step of the computation runs in the library's kernels).

Layouts (see include/tsketch.h):
  batch   T is a flat tensor holding n_series series packed back to back, each
          (d, len_s) stream-major; `series_len` lists len_s.
  streams X is a flat tensor of streams packed back to back; `stream_len`
          lists their lengths.  P and I share X's packing.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Sequence

import numpy as np
import torch

from . import _native as N

_CTX: dict = {}


def _ctx(device: torch.device):
    idx = device.index if device.index is not None else torch.cuda.current_device()
    h = _CTX.get(idx)
    if h is None:
        h = C.c_void_p()
        N.check(N.lib().tsk_create(C.byref(h), idx, None), None, "tsk_create")
        _CTX[idx] = h
    N.check(N.lib().tsk_set_stream(h, C.c_void_p(torch.cuda.current_stream(idx).cuda_stream)), h, "tsk_set_stream")
    return h


def context(device=None):
    """The library context used for `device` (created on first use)."""
    return _ctx(torch.device("cuda", device) if isinstance(device, int) or device is None else torch.device(device))


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _i32_array(vals) -> C.Array:
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.int32))
    return a, a.ctypes.data_as(C.c_void_p)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return N.TSK_F32
    if t.dtype == torch.float64:
        return N.TSK_F64
    raise TypeError(f"series must be float32 or float64, got {t.dtype}")


def _need_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("arguments must be contiguous CUDA tensors")


SKETCH_PRECISION = {"bf16": N.TSK_SKETCH_BF16, "fp32": N.TSK_SKETCH_FP32, "fp64": N.TSK_SKETCH_FP64}
MP_PRECISION = {"fp32": N.TSK_MP_FP32, "fp64": N.TSK_MP_FP64}


def default_excl(m: int) -> int:
    return int(math.ceil(m / 4))


def ts_sketch_build(T: torch.Tensor, R: torch.Tensor, series_len: Sequence[int], d: int,
                    precision: str = "bf16", out: torch.Tensor | None = None,
                    stats: torch.Tensor | None = None):
    """Sketch S = R^T T_bar of every series (Sec. III-A, Alg. 1).

    Returns (S, stats): S packed like T with k streams per series (float32, or
    float64 for precision='fp64'); stats float64 (n_series, d, 2) = (mean, std).
    """
    _need_cuda(T, R)
    k = int(R.shape[1])
    ns = len(series_len)
    sdt = torch.float64 if precision == "fp64" else torch.float32
    total = int(sum(series_len))
    if out is None:
        out = torch.empty(k * total, dtype=sdt, device=T.device)
    if stats is None:
        stats = torch.empty((ns, d, 2), dtype=torch.float64, device=T.device)
    Rf = R if R.dtype == torch.float32 else R.float().contiguous()
    lens, lp = _i32_array(series_len)
    h = _ctx(T.device)
    N.check(N.lib().ts_sketch_build(h, _ptr(T), _dtype_code(T), ns, lp, d, _ptr(Rf), k,
                                    SKETCH_PRECISION[precision], _ptr(out), _ptr(stats)), h, "ts_sketch_build")
    return out, stats


def ts_sketch_update_dims(S: torch.Tensor, T_dims: torch.Tensor, series_len: Sequence[int], R_rows,
                          op: Sequence[int], precision: str = "bf16"):
    """Add (op=+1) or delete (op=-1) dimensions of every series in S, in place (Sec. III-C).

    R_rows: (nd, k) projection rows on the host.  Returns (dirty, stats): the
    uint8 mask of sketch streams that changed, and the new dims' (mean, std).
    """
    _need_cuda(S, T_dims)
    Rr = np.ascontiguousarray(np.asarray(R_rows.cpu() if isinstance(R_rows, torch.Tensor) else R_rows,
                                         dtype=np.float32))
    nd, k = Rr.shape
    opa = np.ascontiguousarray(np.asarray(op, dtype=np.int8))
    ns = len(series_len)
    stats = torch.empty((ns, nd, 2), dtype=torch.float64, device=S.device)
    dirty = np.zeros(k, dtype=np.uint8)
    lens, lp = _i32_array(series_len)
    h = _ctx(S.device)
    N.check(N.lib().ts_sketch_update_dims(h, _ptr(S), _ptr(T_dims), _dtype_code(T_dims), ns, lp, nd,
                                          Rr.ctypes.data_as(C.c_void_p), opa.ctypes.data_as(C.c_void_p), k,
                                          SKETCH_PRECISION[precision], _ptr(stats),
                                          dirty.ctypes.data_as(C.c_void_p)), h, "ts_sketch_update_dims")
    return dirty, stats


def ts_sketch_point_update(S: torch.Tensor, stats: torch.Tensor, R: torch.Tensor, series_len: Sequence[int], d: int,
                           series, dims, times, deltas, T: torch.Tensor | None = None, precision: str = "bf16"):
    """Point updates T_j[t] += delta of (series, dim, time, delta) lists, and the sketch by linearity (Sec. III-C).

    With T, T is updated in place too and S stays the sketch of the updated T
    (required for the bf16-matched sketch).  The build's normalisation is kept.
    """
    _need_cuda(S, stats, R)
    if T is not None:
        _need_cuda(T)
    k = int(R.shape[1])
    ns = len(series_len)
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32)) for a in (series, dims, times)]
    dl = np.ascontiguousarray(np.asarray(deltas, dtype=np.float64))
    n_upd = len(dl)
    if any(len(a) != n_upd for a in arrs):
        raise ValueError("series, dims, times and deltas must have the same length")
    Rf = R if R.dtype == torch.float32 else R.float().contiguous()
    lens, lp = _i32_array(series_len)
    h = _ctx(S.device)
    tcode = _dtype_code(T) if T is not None else N.TSK_F32
    N.check(N.lib().ts_sketch_point_update(h, _ptr(S), _ptr(T) if T is not None else None, tcode, ns, lp, d,
                                           _ptr(Rf), k, SKETCH_PRECISION[precision], _ptr(stats), n_upd,
                                           *(a.ctypes.data_as(C.c_void_p) for a in arrs),
                                           dl.ctypes.data_as(C.c_void_p)), h, "ts_sketch_point_update")


def mp_selfjoin(X: torch.Tensor, stream_len: Sequence[int], m: int, excl: int | None = None,
                precision: str = "fp32", mask=None, P: torch.Tensor | None = None,
                I: torch.Tensor | None = None, tile_rows: int | None = None):
    """Self-join matrix profile of every stream (Def. 6).  Returns (P, I) packed like X.

    tile_rows: rows per work unit of the diagonal kernel; None uses the
    autotuner's cached choice for this layout (0, automatic, when untuned).
    """
    _need_cuda(X)
    excl = default_excl(m) if excl is None else int(excl)
    from . import autotune
    rows = autotune.rows_for(stream_len, m, excl) if tile_rows is None else int(tile_rows)
    pdt = torch.float64 if precision == "fp64" else torch.float32
    if P is None:
        P = torch.empty(X.numel(), dtype=pdt, device=X.device)
    if I is None:
        I = torch.empty(X.numel(), dtype=torch.int32, device=X.device)
    lens, lp = _i32_array(stream_len)
    mk = None
    mp = None
    if mask is not None:
        mk = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        mp = mk.ctypes.data_as(C.c_void_p)
    h = _ctx(X.device)
    N.check(N.lib().tsk_set_tile_rows(h, rows), h, "tsk_set_tile_rows")
    N.check(N.lib().mp_selfjoin(h, _ptr(X), _dtype_code(X), len(stream_len), lp, mp, int(m), excl,
                                MP_PRECISION[precision], _ptr(P), _ptr(I)), h, "mp_selfjoin")
    return P, I


def mp_selfjoin_update(X: torch.Tensor, stream_len: Sequence[int], m: int, P: torch.Tensor, I: torch.Tensor,
                       points, excl: int | None = None):
    """Update the self-join profile (P, I) of float32 streams X in place after point changes.

    X already holds the changed samples; P, I are mp_selfjoin's (fp32) output
    for the streams before the change.  points: (stream, time) pairs of the
    samples that changed.  Only the windows covering them, and the windows whose
    nearest neighbour was one of those, are re-profiled (Sec. III-C point
    updates followed incrementally).  Returns (P, I).
    """
    _need_cuda(X, P, I)
    if X.dtype != torch.float32 or P.dtype != torch.float32:
        raise TypeError("mp_selfjoin_update needs float32 streams and a float32 profile")
    excl = default_excl(m) if excl is None else int(excl)
    pts = np.asarray(list(points), dtype=np.int64).reshape(-1, 2)
    qs, qp = _i32_array(pts[:, 0])
    ts, tp = _i32_array(pts[:, 1])
    lens, lp = _i32_array(stream_len)
    h = _ctx(X.device)
    N.check(N.lib().mp_selfjoin_update(h, _ptr(X), len(stream_len), lp, int(m), excl, _ptr(P), _ptr(I),
                                       len(pts), qp, tp), h, "mp_selfjoin_update")
    return P, I


def mp_abjoin(A: torch.Tensor, B: torch.Tensor, len_a: Sequence[int], len_b: Sequence[int], m: int,
              train_profile: bool = False, precision: str = "fp32"):
    """AB-join profiles (Def. 6): each test window of A_q against every window of B_q.

    Returns (P_a, I_a) packed like A, plus (P_b, I_b) packed like B when
    train_profile (each training window's nearest test window).  precision
    'fp64' is the exact float64 mode (P float64).
    """
    _need_cuda(A, B)
    if A.dtype != B.dtype:
        raise ValueError("A and B must share a dtype")
    n = len(len_a)
    if len(len_b) != n:
        raise ValueError("len_a and len_b must have one entry per stream pair")
    dev = A.device
    pdt = torch.float64 if precision == "fp64" else torch.float32
    P_a = torch.empty(A.numel(), dtype=pdt, device=dev)
    I_a = torch.empty(A.numel(), dtype=torch.int32, device=dev)
    P_b = torch.empty(B.numel(), dtype=pdt, device=dev) if train_profile else None
    I_b = torch.empty(B.numel(), dtype=torch.int32, device=dev) if train_profile else None
    la, lap = _i32_array(len_a)
    lb, lbp = _i32_array(len_b)
    h = _ctx(dev)
    N.check(N.lib().mp_abjoin(h, _ptr(A), _ptr(B), _dtype_code(A), n, lap, lbp, int(m), MP_PRECISION[precision],
                              _ptr(P_a), _ptr(I_a), _ptr(P_b) if train_profile else None,
                              _ptr(I_b) if train_profile else None), h, "mp_abjoin")
    return (P_a, I_a, P_b, I_b) if train_profile else (P_a, I_a)


def ab_discords(T_test: torch.Tensor, T_train: torch.Tensor, test_len: Sequence[int], train_len: Sequence[int],
                d: int, m: int, K: int, R: torch.Tensor | None = None, topk_excl: int | None = None,
                sketch_precision: str = "bf16"):
    """Discords of test series against training series (Def. 5 in train/test form, Alg. 2).

    With R both are z-normalised over their own length and sketched with R,
    and the k sketch streams are AB-joined; without R the d raw streams are.
    """
    if R is not None:
        k = int(R.shape[1])
        A, sa = ts_sketch_build(T_test, R, test_len, d, precision=sketch_precision)
        B, sb = ts_sketch_build(T_train, R, train_len, d, precision=sketch_precision)
        g = k
    else:
        A, B, sa, sb, g = T_test, T_train, None, None, d
    la = [n for n in test_len for _ in range(g)]
    lb = [n for n in train_len for _ in range(g)]
    P, I = mp_abjoin(A, B, la, lb, m)
    idx, grp, score, nn = discord_topk(P, I, test_len, g, m, K, topk_excl)
    return {"S_test": A, "S_train": B, "P": P, "I": I, "idx": idx, "grp": grp, "score": score, "nn": nn}


def discord_topk(P: torch.Tensor, I: torch.Tensor, series_len: Sequence[int], group: int, m: int, K: int,
                 topk_excl: int | None = None):
    """Aggregate over each series' `group` streams and rank K discords (Def. 5, Alg. 2).

    Returns (idx, grp, score, nn), each (n_series, K).
    """
    _need_cuda(P, I)
    ns = len(series_len)
    te = int(m) if topk_excl is None else int(topk_excl)
    dev = P.device
    idx = torch.empty((ns, K), dtype=torch.int32, device=dev)
    grp = torch.empty((ns, K), dtype=torch.int32, device=dev)
    nn = torch.empty((ns, K), dtype=torch.int32, device=dev)
    score = torch.empty((ns, K), dtype=P.dtype, device=dev)
    lens, lp = _i32_array(series_len)
    h = _ctx(dev)
    N.check(N.lib().discord_topk(h, _ptr(P), _dtype_code(P), _ptr(I), ns, lp, int(group), int(m), int(K), te,
                                 _ptr(idx), _ptr(grp), _ptr(score), _ptr(nn)), h, "discord_topk")
    return idx, grp, score, nn


def mp_backward(dscore: torch.Tensor, idx, grp, nn, T: torch.Tensor, stats: torch.Tensor, R: torch.Tensor,
                S: torch.Tensor, series_len: Sequence[int], d: int, m: int):
    """Adjoint of the ranked discord scores: returns (dT packed like T, float32; dR (d, k))."""
    _need_cuda(dscore, idx, grp, nn, T, stats, R, S)
    k = int(R.shape[1])
    ns = len(series_len)
    K = int(idx.shape[1])
    dT = torch.empty(T.numel(), dtype=torch.float32, device=T.device)
    dR = torch.empty((d, k), dtype=torch.float32, device=T.device)
    Rf = R if R.dtype == torch.float32 else R.float().contiguous()
    lens, lp = _i32_array(series_len)
    h = _ctx(T.device)
    N.check(N.lib().mp_backward(h, _ptr(dscore), _ptr(idx), _ptr(grp), _ptr(nn), K, _ptr(T), _dtype_code(T),
                                _ptr(stats), _ptr(Rf), _ptr(S), ns, lp, d, k, int(m), _ptr(dT), _ptr(dR)),
            h, "mp_backward")
    return dT, dR


def sync(device=None, timeout_s: float = 0.0) -> None:
    """Wait for the library's work on the current stream; raise on a device-side error."""
    h = context(device)
    N.check(N.lib().tsk_sync(h, float(timeout_s)), h, "tsk_sync")


def launch_count(device=None) -> int:
    """Kernels launched by the library on this device's context so far."""
    return int(N.lib().tsk_launch_count(context(device)))


def profile_enable(on: bool = True, device=None) -> None:
    """Record CUDA events around the matrix-profile and sketch kernels."""
    h = context(device)
    N.check(N.lib().tsk_profile_enable(h, 1 if on else 0), h, "tsk_profile_enable")


def profile_read(kernel: str = "mp_diag", device=None) -> tuple:
    """(total device ms, launches) of `kernel` ('mp_diag', 'sketch' or 'dims') since the last read."""
    h = context(device)
    ms = C.c_double()
    n = C.c_int64()
    kid = {"mp_diag": N.TSK_PROF_MP_DIAG, "sketch": N.TSK_PROF_SKETCH, "dims": N.TSK_PROF_DIMS}[kernel]
    N.check(N.lib().tsk_profile_read(h, kid, C.byref(ms), C.byref(n)), h, "tsk_profile_read")
    return float(ms.value), int(n.value)


def set_tile_rows(rows: int, device=None) -> None:
    """Rows per matrix-profile work unit (multiple of 8)."""
    h = context(device)
    N.check(N.lib().tsk_set_tile_rows(h, int(rows)), h, "tsk_set_tile_rows")


def reserve(nbytes: int, device=None) -> None:
    h = context(device)
    N.check(N.lib().tsk_reserve(h, int(nbytes)), h, "tsk_reserve")


# ---------------------------------------------------------------------------
# whole-pipeline helpers
# ---------------------------------------------------------------------------

def pack_batch(series) -> tuple:
    """Pack a list of (d, len_s) arrays/tensors into one flat tensor + lengths (host-side layout)."""
    lens = [int(s.shape[1]) for s in series]
    flat = [torch.as_tensor(s).reshape(-1) for s in series]
    return torch.cat(flat), lens


def sketched_discords(T: torch.Tensor, R: torch.Tensor, series_len: Sequence[int], d: int, m: int, K: int,
                      excl: int | None = None, topk_excl: int | None = None, sketch_precision: str = "bf16",
                      mp_precision: str = "fp32"):
    """Sketch, profile the k sketch streams, rank K discords per series (Alg. 1 then Alg. 2)."""
    k = int(R.shape[1])
    S, stats = ts_sketch_build(T, R, series_len, d, precision=sketch_precision)
    slen = [n for n in series_len for _ in range(k)]
    P, I = mp_selfjoin(S, slen, m, excl, precision=mp_precision)
    idx, grp, score, nn = discord_topk(P, I, series_len, k, m, K, topk_excl)
    return {"S": S, "stats": stats, "P": P, "I": I, "idx": idx, "grp": grp, "score": score, "nn": nn}


def exact_discords(T: torch.Tensor, series_len: Sequence[int], d: int, m: int, K: int,
                   excl: int | None = None, topk_excl: int | None = None, mp_precision: str = "fp32"):
    """Exact multidimensional discords: one profile per raw dimension, max over d (Def. 5)."""
    slen = [n for n in series_len for _ in range(d)]
    P, I = mp_selfjoin(T, slen, m, excl, precision=mp_precision)
    idx, grp, score, nn = discord_topk(P, I, series_len, d, m, K, topk_excl)
    return {"P": P, "I": I, "idx": idx, "grp": grp, "score": score, "nn": nn}


def dimension_detection(T: torch.Tensor, R: torch.Tensor, series_len: Sequence[int], d: int, m: int, idx, grp,
                        excl: int | None = None, all_scores: bool = False, gather: bool = False,
                        T_train: torch.Tensor | None = None, train_len: Sequence[int] | None = None):
    """Alg. 3: the raw dimension behind each sketch discord (idx, grp of discord_topk).

    Self-join form by default; with T_train (and train_len) the train/test
    form: each test window is scored against every window of the training
    stream.  Returns {"dim", "score", "nn"} ([n_series, K]; score float64),
    plus "scores" ([n_series, K, d], NaN outside the group) when all_scores
    and "T_sel" (the chosen streams, packed like a K-stream sketch; with
    T_train also "T_sel_train") when gather.
    """
    _need_cuda(T, R, idx, grp)
    ab = T_train is not None
    if ab:
        _need_cuda(T_train)
        if train_len is None or len(train_len) != len(series_len) or T_train.dtype != T.dtype:
            raise ValueError("T_train needs train_len (one per series) and T's dtype")
    excl = 0 if ab else (default_excl(m) if excl is None else int(excl))
    k = int(R.shape[1])
    ns = len(series_len)
    K = int(idx.shape[1])
    dev = T.device
    dim = torch.empty((ns, K), dtype=torch.int32, device=dev)
    score = torch.empty((ns, K), dtype=torch.float64, device=dev)
    nn = torch.empty((ns, K), dtype=torch.int32, device=dev)
    scores = torch.empty((ns, K, d), dtype=torch.float64, device=dev) if all_scores else None
    T_sel = torch.empty(sum(series_len) * K, dtype=T.dtype, device=dev) if gather else None
    T_sel_t = torch.empty(sum(train_len) * K, dtype=T.dtype, device=dev) if (gather and ab) else None
    Rf = R if R.dtype == torch.float32 else R.float().contiguous()
    lens, lp = _i32_array(series_len)
    tl, tlp = _i32_array(train_len) if ab else (None, None)
    h = _ctx(dev)
    N.check(N.lib().dimension_detection(h, _ptr(T), _dtype_code(T), ns, lp, d, _ptr(Rf), k, int(m), excl, K,
                                        _ptr(idx), _ptr(grp), _ptr(dim), _ptr(score), _ptr(nn),
                                        _ptr(scores) if all_scores else None, _ptr(T_sel) if gather else None,
                                        _ptr(T_train) if ab else None, tlp if ab else None,
                                        _ptr(T_sel_t) if T_sel_t is not None else None),
            h, "dimension_detection")
    out = {"dim": dim, "score": score, "nn": nn}
    if all_scores:
        out["scores"] = scores
    if gather:
        out["T_sel"] = T_sel
        if ab:
            out["T_sel_train"] = T_sel_t
    return out


def refine_dimensions(T_sel: torch.Tensor, series_len: Sequence[int], K: int, m: int, excl: int | None = None,
                      topk_excl: int | None = None, mp_precision: str = "fp32",
                      T_sel_train: torch.Tensor | None = None, train_len: Sequence[int] | None = None):
    """The refinement after Alg. 3: the top-1 discord of each chosen stream's own profile.

    T_sel is dimension_detection(..., gather=True)["T_sel"]; with T_sel_train
    (the train/test form) the profile is the AB join against the chosen
    training stream.  Returns {"idx", "score", "nn"} of shape [n_series, K].
    """
    lens = [n for n in series_len for _ in range(K)]
    if T_sel_train is None:
        P, I = mp_selfjoin(T_sel, lens, m, excl, precision=mp_precision)
    else:
        P, I = mp_abjoin(T_sel, T_sel_train, lens, [n for n in train_len for _ in range(K)], m)
    idx, _, score, nn = discord_topk(P, I, lens, 1, m, 1, topk_excl)
    ns = len(series_len)
    return {"idx": idx.view(ns, K), "score": score.view(ns, K), "nn": nn.view(ns, K), "P": P, "I": I}


class DiscordScores(torch.autograd.Function):
    """Top-K aggregated discord scores of the sketched path, differentiable in T and R.

    forward(T, R, series_len, d, m, K) -> scores (n_series, K); backward uses
    mp_backward with the forward's selections held fixed.
    """

    @staticmethod
    def forward(ctx, T, R, series_len, d, m, K, excl=None, topk_excl=None, sketch_precision="fp32"):
        res = sketched_discords(T, R, series_len, d, m, K, excl, topk_excl, sketch_precision=sketch_precision)
        ctx.save_for_backward(T, R, res["stats"], res["S"], res["idx"], res["grp"], res["nn"])
        ctx.meta = (list(series_len), d, m)
        return res["score"].float()

    @staticmethod
    def backward(ctx, g):
        T, R, stats, S, idx, grp, nn = ctx.saved_tensors
        series_len, d, m = ctx.meta
        S32 = S if S.dtype == torch.float32 else S.float().contiguous()
        dT, dR = mp_backward(g.contiguous().float(), idx, grp, nn, T, stats, R, S32, series_len, d, m)
        return dT.to(T.dtype), dR.to(R.dtype), None, None, None, None, None, None, None
