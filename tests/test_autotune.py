"""Host logic of the work-unit autotuner (no GPU: a fake timer stands in for the kernel)."""
import json

import pytest

from paper_2311_03393_gb300 import autotune


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("TSK_TUNE_CACHE", str(path))
    return path


def test_tune_picks_the_fastest_and_caches_it(cache):
    times = {0: 5.0, 2048: 3.0, 3072: 3.5, 4096: 3.0, 6144: 9.0}
    best = autotune.tune(None, [50000] * 8, 100, 25, timer=lambda r: times[r])
    assert best == 2048  # tie with 4096 resolved to the smaller height
    assert autotune.rows_for([50000] * 8, 100, 25, device_name="cpu", sm_count=0) == 2048
    data = json.loads(cache.read_text())
    assert list(data.values()) == [2048]


def test_untuned_layout_uses_the_automatic_rule(cache):
    assert autotune.rows_for([1000] * 3, 64, 16, device_name="cpu", sm_count=0) == 0


def test_layout_buckets_group_similar_sizes_and_separate_different_ones():
    k = lambda lens, m=100, e=25: autotune.layout_key(lens, m, e, "gpu", 152)
    assert k([50000] * 8) == k([50100] * 8)          # same size bucket
    assert k([50000] * 8) != k([50000] * 51)         # more streams
    assert k([50000] * 8) != k([50000] * 8, m=64)    # other subsequence length
    assert k([50000] * 8) != k([200000] * 8)         # 16x more cells
