"""The autotuner's persistent cache (host logic only, no GPU): where it
lives, that a saved table reads back, that a damaged file reads as empty,
and that the key tells workloads apart."""
import json

import pytest

from paper_1802_00036_gb300 import tune


@pytest.fixture
def dc_mod():
    from paper_1802_00036_gb300 import build, dc
    build.build()
    return dc


def test_cache_path_follows_the_environment(tmp_path, monkeypatch):
    monkeypatch.setenv("DCGB_TUNE_CACHE", str(tmp_path / "t.json"))
    assert tune.cache_path() == str(tmp_path / "t.json")
    monkeypatch.delenv("DCGB_TUNE_CACHE")
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path / "xdg"))
    assert tune.cache_path() == str(tmp_path / "xdg" / "dcgb" / "autotune.json")


def test_save_then_load(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    data = {"gpu|152|n64|352x1216|0,31,1,1,1,-1,1,0": [16, 5, 160]}
    tune.save_cache(data, path)
    assert tune.load_cache(path) == data
    assert not [p for p in (tmp_path / "sub").iterdir() if ".tmp" in p.name]


@pytest.mark.parametrize("text", ["{not json", "[1, 2, 3]", ""])
def test_damaged_or_foreign_file_reads_empty(tmp_path, text):
    path = tmp_path / "cache.json"
    path.write_text(text)
    assert tune.load_cache(str(path)) == {}
    assert tune.load_cache(str(tmp_path / "missing.json")) == {}


def test_key_separates_workloads(dc_mod):
    base = tune.cache_key("GB300", 152, 64, 352, 1216, dc_mod.params())
    others = [
        tune.cache_key("GB300", 148, 64, 352, 1216, dc_mod.params()),
        tune.cache_key("GB300", 152, 32, 352, 1216, dc_mod.params()),
        tune.cache_key("GB300", 152, 64, 375, 1242, dc_mod.params()),
        tune.cache_key("GB300", 152, 64, 352, 1216, dc_mod.params(blur="bilateral")),
        tune.cache_key("GB300", 152, 64, 352, 1216, dc_mod.params(large_fill=51)),
        tune.cache_key("GB300", 152, 64, 352, 1216, dc_mod.params(extend_top=False)),
        tune.cache_key("other", 152, 64, 352, 1216, dc_mod.params()),
    ]
    assert len({base, *others}) == len(others) + 1
    assert base == tune.cache_key("GB300", 152, 64, 352, 1216, dc_mod.params())
    json.dumps({base: [1, 2, 3]})  # keys are plain strings
