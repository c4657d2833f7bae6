"""Autotuner bookkeeping without a GPU: the key groups shapes by
(b, w, arrow blocks, precision) and cached choices are returned as stored."""
import json

from paper_2504_19171_gb300 import autotune as AT


def test_key_groups_arrow_by_blocks():
    assert AT.key_of(256, 2, 1, 0) == AT.key_of(256, 2, 64, 0)
    assert AT.key_of(256, 2, 65, 0) != AT.key_of(256, 2, 64, 0)
    assert AT.key_of(256, 2, 64, 1) != AT.key_of(256, 2, 64, 0)


def test_cached_choice_is_used(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({AT.key_of(512, 3, 100, 1): {"code": 24, "seconds": {"0": 1.0, "24": 0.5}}}))
    t = AT.Autotuner(str(p))
    assert t.best(512, 3, 100, 1) == 24
    assert t.codes_for([(50, 512, 3, 128)], 1) == [24]


def test_candidates_are_valid_tuning_codes():
    from paper_2504_19171_gb300 import stiles as S
    for c in AT.CANDIDATES:
        assert S.stiles_debug_validate(5, 64, 1, 8, S.PLAN_FUSED + 256 * c) == S.STILES_OK


def test_single_regime_has_its_own_key(tmp_path):
    # a long matrix alone and a batch of short ones are tuned separately
    assert AT.key_of(1024, 1, 64, 0, "single") != AT.key_of(1024, 1, 64, 0)
    assert AT.key_of(1024, 1, 64, 0, "single").endswith(":single")
    p = tmp_path / "t.json"
    p.write_text(json.dumps({AT.key_of(1024, 1, 64, 1, "single"): {"code": 3, "grid_per_sm": 1, "seconds": {}},
                             AT.key_of(1024, 1, 64, 1): {"code": 26, "seconds": {}}}))
    t = AT.Autotuner(str(p))
    assert t.best_single(1024, 1, 64, 1) == (3, 1)
    assert t.best(1024, 1, 64, 1) == 26
    assert t.cached(1024, 1, 64, 2) is None


def test_shipped_cache_entries_are_valid():
    from paper_2504_19171_gb300 import stiles as S
    t = AT.Autotuner(AT.default_cache_path())
    for k, e in t.cache.items():
        assert S.stiles_debug_validate(4, 64, 1, 8, S.PLAN_FUSED + 256 * int(e["code"])) == S.STILES_OK, k
        assert int(e.get("grid_per_sm", 2)) in AT.GRID_PER_SM, k


def test_single_regime_keeps_defaults_within_margin():
    # a probe win smaller than the margin does not replace the defaults
    t = {(0, 2): 1.000, (4, 2): 0.998, (1, 1): 1.2}
    assert AT.Autotuner.pick_single(t) == (0, 2)
    t[(26, 2)] = 0.90
    assert AT.Autotuner.pick_single(t) == (26, 2)
