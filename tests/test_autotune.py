"""Selection logic of the batched autotuner (host only: the timing function
is replaced by a model, so no GPU is needed)."""
import pytest


def test_autotuner_picks_fastest_tile_per_shape_and_one_dense_threshold(monkeypatch, tmp_path):
    torch = pytest.importorskip("torch")
    from paper_2208_06194_gb300 import autotune
    calls = []

    def fake_time(kernel, m, n, b, sx, sy, tol, precision, dense_rank):
        calls.append((m, n, b, dense_rank))
        # small matrices prefer b = 256, large ones b = 512; threshold 32 best overall
        base = m * n / 1e8
        tile = 1.0 if (m <= 8192) == (b == 256) else 1.5
        return base * tile * (1.0 + abs(dense_rank - 32) / 64)

    monkeypatch.setattr(autotune, "_time_one", fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda i=0: "fake")
    probs = [(4096, 2048, 1, 2), (16384, 8192, 3, 4), (4096, 2048, 5, 6), (6144, 3072, 7, 8)]
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(probs, "laplace3d", 1e-6, 1, cache_path=cache)
    assert res["b"] == [256, 512, 256, 256]
    assert res["dense_rank"] == 32
    n_calls = len(calls)
    res2 = autotune.tune(probs, "laplace3d", 1e-6, 1, cache_path=cache)     # served from the cache
    assert res2["b"] == res["b"] and res2["dense_rank"] == 32
    assert len(calls) == n_calls + 1                                        # only the warm-up ran again
