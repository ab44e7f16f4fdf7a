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


def test_coordinate_search_keeps_only_real_gains(monkeypatch):
    # a fake cost surface: batch_pairs_shape 3 is 10% faster, build block 64
    # 0.5% faster (below the 1% bar), everything else neutral
    state = {}

    def fake_apply(ctx, cfg):
        state.clear()
        state.update(cfg)

    def fake_time(run, repeats):
        t = 10.0
        if state.get("batch_pairs_shape") == 3:
            t *= 0.9
        if state.get("batch_build_block") == 64:
            t *= 0.995
        return t

    monkeypatch.setattr(autotune, "apply", fake_apply)
    monkeypatch.setattr(autotune, "_time_ms", fake_time)
    best, ms, table = autotune._coordinate_search(None, None, autotune.BATCH_SPACE, autotune.BATCH_DEFAULT, 1)
    assert best["batch_pairs_shape"] == 3 and best["batch_build_block"] == 32
    assert abs(ms - 9.0) < 1e-9
    assert state == best  # the chosen shape is the one left applied
    # every knob value was tried from the starting point, and only valid shapes
    tried = {(k, c[k]) for c, _ in table for k in autotune.BATCH_SPACE}
    assert all((k, v) in tried for k, vals in autotune.BATCH_SPACE.items() for v in vals)
    assert all(autotune.valid(c) for c, _ in table)
