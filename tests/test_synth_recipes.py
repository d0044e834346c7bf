"""The synthetic inputs follow the recipes the design documents (no GPU).

Seeded generators stand in for the paper's datasets; these checks pin their
shapes and the properties the workload table states, at reduced lengths.
"""
import numpy as np
import pytest

from paper_2311_03393_gb300 import synth


@pytest.mark.parametrize("n,m,count", [(2000, 100, 1), (50000, 100, 5), (100000, 144, 10), (1000, 64, 1)])
def test_planted_positions_are_spread_inside_the_series(n, m, count):
    rng = np.random.default_rng(3)
    pos = synth.plant_positions(rng, n, m, count)
    assert len(pos) == count and pos == sorted(pos)
    assert all(m <= p <= n - 2 * m for p in pos)
    assert all(b - a >= 2 * m for a, b in zip(pos, pos[1:]))


@pytest.mark.parametrize("index,d,m,k", [(1, 8, 100, 4), (2, 51, 100, 8), (3, 1024, 144, 16), (5, 64, 100, 8)])
def test_single_series_workloads_have_the_documented_shapes(index, d, m, k):
    wl = synth.workload(index, scale=0.01)
    assert len(wl.series) == 1 and wl.d == d and wl.m == m and wl.k == k
    assert wl.R.shape == (d, k) and wl.R.dtype == np.float32
    assert wl.series[0].dtype == (np.float64 if index == 1 else np.float32)
    n = wl.lengths[0]
    assert all(m <= p <= n - 2 * m for (_, _, p) in wl.planted)


def test_water_streams_are_walks_square_waves_and_ar1():
    T, planted = synth.water_plant(51, 20000, 100, 5, seed=11)
    hit = np.zeros(T.shape, dtype=bool)
    for j, p in planted:
        hit[j, p:p + 100] = True
    for j in range(51):
        x = T[j][~hit[j]]
        if j % 3 == 1:                                   # square waves: levels {0, 1}, about half on
            assert set(np.unique(x)) <= {0.0, 1.0} and 0.3 < x.mean() < 0.7
        elif j % 3 == 2:                                 # AR(1), phi 0.95, unit innovations: var 1/(1 - 0.95^2)
            assert 4.0 < x.var() < 25.0
    assert len(planted) == 5


def test_traffic_streams_carry_a_period_of_144_and_lognormal_amplitudes():
    T, planted = synth.traffic(64, 14400, 144, 3, seed=12)
    spec = np.abs(np.fft.rfft(T - T.mean(axis=1, keepdims=True), axis=1))
    peak = spec[:, 1:].argmax(axis=1) + 1
    assert np.mean(peak == 14400 // 144) > 0.9          # the daily cycle dominates every stream
    amp = spec[:, 100] / (14400 / 2)
    assert 0.3 < np.median(amp) < 3.0 and amp.std() > 0.1
    assert len(planted) == 3


def test_batched_series_have_uneven_lengths_and_one_discord_each():
    Ts, planted = synth.batched_random_walks(64, 1000, 32000, 16, 64, seed=13)
    lens = [t.shape[1] for t in Ts]
    assert all(1000 <= n <= 32000 for n in lens) and len(set(lens)) > 50
    assert all(t.shape[0] == 16 and t.dtype == np.float32 for t in Ts)
    assert sorted(s for s, _, _ in planted) == list(range(64))


def test_gaussian_R_has_variance_one_over_k():
    R = synth.gaussian_R(4096, 16, seed=14)
    assert abs(R.var() * 16 - 1.0) < 0.02 and abs(R.mean()) < 0.01
