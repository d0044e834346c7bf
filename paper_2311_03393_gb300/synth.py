"""Seeded synthetic workloads for sketched discord mining.

This module only draws random numbers and lays them out: random walks, square
waves, AR(1) processes, periodic sensors, planted discords, and the random
projection matrices R (Gaussian or count sketch).  It holds none of the
method's arithmetic (no z-normalisation, sketching or distance), so both the
CUDA path and the FP64 oracle can be fed from it without sharing any code.

Shapes follow the workloads of the paper's experiments (Sec. IV): multivariate
series T of shape (d, n), stream-major, one row per dimension (Def. 1), with a
subsequence length m.  Planted discords replace a window of one stream by a
sine of period 20 plus N(0, 0.5^2) noise (period 144-scaled variant for the
traffic-like workload).  All generators take an explicit integer seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Workload",
    "plant_positions",
    "random_walks",
    "water_plant",
    "traffic",
    "batched_random_walks",
    "gaussian_R",
    "count_sketch_hashes",
    "count_sketch_R",
    "default_k",
    "default_excl",
    "workload",
    "WORKLOADS",
]

SEED_BASE = 20231106


def default_k(d: int) -> int:
    """k = ceil(sqrt(d)), the sketch size the paper uses (Sec. IV-A)."""
    return int(math.ceil(math.sqrt(d)))


def default_excl(m: int) -> int:
    """Self-join exclusion half-width ceil(m/4) (pairs with |i-j| < excl are trivial matches)."""
    return int(math.ceil(m / 4))


@dataclass
class Workload:
    """One seeded multivariate workload.

    series: list of float arrays, each (d, n_s) stream-major.
    planted: list of (series, stream, start) of the planted discord windows.
    """
    name: str
    series: list
    m: int
    k: int
    R: np.ndarray
    planted: list = field(default_factory=list)
    dtype: str = "f32"

    @property
    def d(self) -> int:
        return int(self.series[0].shape[0])

    @property
    def lengths(self) -> list:
        return [int(s.shape[1]) for s in self.series]


def plant_positions(rng: np.random.Generator, n: int, m: int, count: int) -> list:
    """Seeded discord starts, uniform over [m, n-2m], pairwise at least 2m apart."""
    lo, hi = m, n - 2 * m
    if hi < lo or count == 0:
        return []
    out: list = []
    tries = 0
    while len(out) < count and tries < 100000:
        p = int(rng.integers(lo, hi + 1))
        if all(abs(p - q) >= 2 * m for q in out):
            out.append(p)
        tries += 1
    return sorted(out)


def _discord_shape(rng: np.random.Generator, length: int, period: float) -> np.ndarray:
    t = np.arange(length, dtype=np.float64)
    return np.sin(2.0 * np.pi * t / period) + rng.normal(0.0, 0.5, size=length)


def random_walks(d: int, n: int, m: int, n_discords: int, seed: int, dtype=np.float32,
                 discord_streams=None):
    """Gaussian random walks (cumulative sums of N(0,1) steps) with planted discords.

    Returns (T (d, n), planted [(stream, start)]).
    """
    rng = np.random.default_rng(seed)
    T = np.cumsum(rng.normal(0.0, 1.0, size=(d, n)), axis=1)
    pos = plant_positions(rng, n, m, n_discords)
    planted = []
    for q, p in enumerate(pos):
        if discord_streams is not None:
            j = int(discord_streams[q % len(discord_streams)])
        else:
            j = int(rng.integers(0, d))
        T[j, p:p + m] = _discord_shape(rng, m, 20.0)
        planted.append((j, p))
    return T.astype(dtype), planted


def _ar1_fast(rng: np.random.Generator, rows: int, n: int, phi: float, sd: float) -> np.ndarray:
    """AR(1) x_t = phi x_{t-1} + e_t, e_t ~ N(0, sd^2), started from its stationary law."""
    from scipy.signal import lfilter
    e = rng.normal(0.0, sd, size=(rows, n))
    e[:, 0] /= math.sqrt(max(1e-12, 1.0 - phi * phi))
    return lfilter([1.0], [1.0, -phi], e, axis=1)


def water_plant(d: int, n: int, m: int, n_discords: int, seed: int, dtype=np.float32):
    """Water-plant-like sensors (the shape of the SWaT setting, Sec. IV-D).

    A third each of random walks, square-wave actuators (levels {0,1}, period
    uniform in 500..5000, 50% duty, random phase) and AR(1) (phi=0.95, N(0,1)
    innovations); n_discords planted windows of length m in random streams.
    """
    rng = np.random.default_rng(seed)
    T = np.empty((d, n), dtype=np.float64)
    kinds = np.arange(d) % 3
    t = np.arange(n)
    for j in range(d):
        if kinds[j] == 0:
            T[j] = np.cumsum(rng.normal(0.0, 1.0, size=n))
        elif kinds[j] == 1:
            period = int(rng.integers(500, 5001))
            phase = int(rng.integers(0, period))
            T[j] = (((t + phase) % period) < (period // 2)).astype(np.float64)
        else:
            T[j] = _ar1_fast(rng, 1, n, 0.95, 1.0)[0]
    pos = plant_positions(rng, n, m, n_discords)
    planted = []
    for p in pos:
        j = int(rng.integers(0, d))
        T[j, p:p + m] = _discord_shape(rng, m, 20.0)
        planted.append((j, p))
    return T.astype(dtype), planted


def traffic(d: int, n: int, m: int, n_discords: int, seed: int, dtype=np.float32):
    """Traffic-like sensors: a_j * (sin(2 pi t/144 + phi_j) + AR(1)).

    a_j ~ LogNormal(0, 0.5), phi_j ~ U[0, 2pi), AR(1) with phi=0.95 and
    innovation sd 0.1; discords of length m use the sine+noise shape scaled by a_j.
    """
    rng = np.random.default_rng(seed)
    a = rng.lognormal(0.0, 0.5, size=d)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=d)
    t = np.arange(n, dtype=np.float64)
    T = np.sin(2.0 * np.pi * t[None, :] / 144.0 + ph[:, None])
    T += _ar1_fast(rng, d, n, 0.95, 0.1)
    T *= a[:, None]
    pos = plant_positions(rng, n, m, n_discords)
    planted = []
    for p in pos:
        j = int(rng.integers(0, d))
        T[j, p:p + m] = a[j] * _discord_shape(rng, m, 20.0)
        planted.append((j, p))
    return T.astype(dtype), planted


def batched_random_walks(n_series: int, nmin: int, nmax: int, d: int, m: int, seed: int,
                         dtype=np.float32):
    """Many independent multivariate random-walk series of uneven length.

    Lengths uniform in {nmin..nmax}; one planted discord of length m per series.
    Returns (list of (d, n_s) arrays, planted [(series, stream, start)]).
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(nmin, nmax + 1, size=n_series)
    out, planted = [], []
    for s in range(n_series):
        n = int(lens[s])
        X = np.cumsum(rng.normal(0.0, 1.0, size=(d, n)), axis=1)
        pos = plant_positions(rng, n, m, 1)
        for p in pos:
            j = int(rng.integers(0, d))
            X[j, p:p + m] = _discord_shape(rng, m, 20.0)
            planted.append((s, j, p))
        out.append(X.astype(dtype))
    return out, planted


def gaussian_R(d: int, k: int, seed: int) -> np.ndarray:
    """Dense random projection, entries i.i.d. N(0, 1/k), shape (d, k), FP32."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0 / math.sqrt(k), size=(d, k)).astype(np.float32)


_P31 = 2147483647  # Mersenne prime 2^31 - 1


def count_sketch_hashes(d: int, k: int, seed: int):
    """Draw h: [d] -> [k] and s: [d] -> {-1,+1} from 2-universal families (Sec. III-A).

    h(j) = ((a j + b) mod p) mod k and s(j) = 2 (((c j + e) mod p) mod 2) - 1,
    p = 2^31 - 1, with (a, b, c, e) drawn from the seed.
    """
    rng = np.random.default_rng(seed)
    a, c = (int(v) for v in rng.integers(1, _P31, size=2))
    b, e = (int(v) for v in rng.integers(0, _P31, size=2))
    j = np.arange(d, dtype=np.int64)
    h = ((a * j + b) % _P31) % k
    s = 2 * (((c * j + e) % _P31) % 2) - 1
    return h.astype(np.int64), s.astype(np.int64)


def count_sketch_R(d: int, k: int, seed: int) -> np.ndarray:
    """The count sketch as a (d, k) matrix: R[j, h(j)] = s(j), zero elsewhere."""
    h, s = count_sketch_hashes(d, k, seed)
    R = np.zeros((d, k), dtype=np.float32)
    R[np.arange(d), h] = s
    return R


# ---------------------------------------------------------------------------
# The named workloads (synthetic stand-ins for the paper's data shapes)
# ---------------------------------------------------------------------------

def _wl_rw_small(seed, scale):
    d, n, m, k = 8, 2000, 100, 4
    n = max(4 * m, int(n * scale))
    T, pl = random_walks(d, n, m, 1, seed, dtype=np.float64, discord_streams=[0])
    return Workload("rw_d8_n2000_m100_k4_fp64", [T], m, k, gaussian_R(d, k, seed + 1),
                    [(0, j, p) for j, p in pl], dtype="f64")


def _wl_water(seed, scale):
    d, n, m, k = 51, 50000, 100, 8
    n = max(4 * m, int(n * scale))
    T, pl = water_plant(d, n, m, 5, seed)
    return Workload(f"water_d51_n{n}_m100_k8", [T], m, k, gaussian_R(d, k, seed + 1),
                    [(0, j, p) for j, p in pl])


def _wl_traffic(seed, scale):
    d, n, m, k = 1024, 100000, 144, 16
    n = max(4 * m, int(n * scale))
    T, pl = traffic(d, n, m, 10, seed)
    return Workload(f"traffic_d1024_n{n}_m144_k16", [T], m, k, gaussian_R(d, k, seed + 1),
                    [(0, j, p) for j, p in pl])


def _wl_batched(seed, scale):
    ns, nmin, nmax, d, m, k = 4096, 1000, 32000, 16, 64, 4
    ns = max(1, int(ns * scale))
    Ts, pl = batched_random_walks(ns, nmin, nmax, d, m, seed)
    return Workload(f"batched_{ns}x_d16_n1000-32000_m64_k4", Ts, m, k, gaussian_R(d, k, seed + 1), pl)


def _wl_grad(seed, scale):
    d, n, m, k = 64, 20000, 100, 8
    n = max(4 * m, int(n * scale))
    T, pl = random_walks(d, n, m, 3, seed)
    return Workload(f"grad_rw_d64_n{n}_m100_k8", [T], m, k, gaussian_R(d, k, seed + 1),
                    [(0, j, p) for j, p in pl])


WORKLOADS = {
    1: _wl_rw_small,
    2: _wl_water,
    3: _wl_traffic,
    4: _wl_batched,
    5: _wl_grad,
}


def workload(index: int, seed: int | None = None, scale: float = 1.0) -> Workload:
    """Build named workload `index` (1..5) with the default seed 20231106 + index.

    `scale` shrinks the length n (or the number of series for the batched
    workload) for quick parity cases; scale=1 is the full size.
    """
    if seed is None:
        seed = SEED_BASE + index
    return WORKLOADS[index](seed, scale)
