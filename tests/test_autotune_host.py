"""Host logic of the autotuner (no GPU): which launch shapes are valid, how a
shape is applied without passing through an invalid intermediate, and the
bucketed workload signature that keys the cache."""
import pytest

autotune = pytest.importorskip("paper_2412_19420_gb300.autotune")


def test_valid_shapes():
    assert autotune.valid({"dfs_threads": 256, "dfs_ctas_per_sm": 4})
    assert autotune.valid({"dfs_threads": 512, "dfs_ctas_per_sm": 2})
    assert not autotune.valid({"dfs_threads": 512, "dfs_ctas_per_sm": 4})
    # the search space holds at least one valid shape per thread count
    for t in autotune.SPACE["dfs_threads"]:
        assert any(autotune.valid({"dfs_threads": t, "dfs_ctas_per_sm": c}) for c in autotune.SPACE["dfs_ctas_per_sm"])
    assert autotune.valid(autotune.DEFAULT)


def test_apply_never_passes_an_invalid_intermediate(monkeypatch):
    calls = []
    state = {"dfs_threads": 256, "dfs_ctas_per_sm": 4}

    def fake_set(ctx, key, value):
        calls.append((key, value))
        state[key] = value
        assert state["dfs_threads"] * state["dfs_ctas_per_sm"] <= 1024, (key, value, dict(state))

    monkeypatch.setattr(autotune.fim, "fim_set_tuning", fake_set)
    autotune.apply(None, {"dfs_threads": 512, "dfs_ctas_per_sm": 2, "split_depth": 4})
    assert calls[0] == ("dfs_ctas_per_sm", 1) and calls[-1] == ("dfs_ctas_per_sm", 2)
    assert state == {"dfs_threads": 512, "dfs_ctas_per_sm": 2, "split_depth": 4}
    with pytest.raises(ValueError):
        autotune.apply(None, {"dfs_threads": 512, "dfs_ctas_per_sm": 4})


def test_signature_buckets_by_log2():
    a = autotune.signature("single", 1_000_000, 1000, 10_000_000, 1000, 0)
    b = autotune.signature("single", 1_040_000, 1010, 10_400_000, 1010, 0)
    c = autotune.signature("single", 2_100_000, 1000, 10_000_000, 1000, 0)
    assert a == b and a != c
    assert a != autotune.signature("single", 1_000_000, 1000, 10_000_000, 1000, 2)
    assert a != autotune.signature("batched", 1_000_000, 1000, 10_000_000, 1000, 0)
