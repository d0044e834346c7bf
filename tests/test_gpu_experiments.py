"""The synthetic sketch-quality experiment (Sec. IV) runs end to end on the GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_03393_gb300 import build
    build.build()
    from paper_2311_03393_gb300 import experiments
    return experiments


def test_identity_sketch_finds_the_exact_discord(exp):
    """k = d with h(j) = j: the sketched path is the exact path, so every trial succeeds at rank 1."""
    d, n, m = 12, 3000, 50
    dev = torch.device("cuda")
    for seed in (1, 2, 3):
        r = exp.trial(d, n, m, d, seed, dev, sketch_precision="fp32", R=np.eye(d, dtype=np.float32))
        assert r["success"] and r["rank"] == 1
        assert (r["i"], r["j"]) == (r["exact_i"], r["exact_j"])
        assert abs(r["score"] - r["exact_score"]) <= 1e-4 * r["exact_score"]


def test_count_sketch_quality_run(exp):
    out = exp.sketch_quality(256, n=4000, m=100, trials=4)
    assert out["k"] == 16 and 0.0 <= out["success_rate"] <= 1.0
    assert out["median_rank"] >= 1 and out["speedup"] > 1.0
