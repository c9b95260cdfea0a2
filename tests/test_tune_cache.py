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


class _Tensor:
    """Stands in for a CUDA tensor: shape, device and a data pointer."""

    def __init__(self, shape):
        self.shape = shape
        self.device = "cuda:0"

    def data_ptr(self):
        return 0


def test_tuned_records_the_size_from_cache_and_from_the_autotuner(dc_mod, tmp_path, monkeypatch):
    # tune.tuned applies a cached tuning (dc_set_tuning) and records it for the
    # frame size (dc_set_class_tuning), as dc_autotune records its own choice;
    # on a miss it runs dc_autotune and caches the result (no GPU: the CUDA
    # and library calls are stood in for)
    import torch
    from types import SimpleNamespace
    monkeypatch.setenv("DCGB_TUNE_CACHE", str(tmp_path / "t.json"))
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev: SimpleNamespace(name="GB300", multi_processor_count=152))
    calls = []
    monkeypatch.setattr(dc_mod, "dc_set_tuning", lambda h, *t: calls.append(("set", t)))
    monkeypatch.setattr(dc_mod, "dc_set_class_tuning", lambda h, H, W, t=None: calls.append(("class", H, W, t)))
    monkeypatch.setattr(dc_mod, "dc_autotune", lambda h, i, o, n, H, W, p, s: (12, 5, 8, 64))
    ctx = SimpleNamespace(h=1)
    inp, out = _Tensor((32, 256, 512)), _Tensor((32, 256, 512))
    t, source = tune.tuned(ctx, inp, out, dc_mod.params(), stream=7)
    assert (t, source) == ((12, 5, 8, 64), "measured") and calls == []
    t, source = tune.tuned(ctx, inp, out, dc_mod.params(), stream=7)
    assert (t, source) == ((12, 5, 8, 64), "cache")
    assert calls == [("set", (12, 5, 8, 64)), ("class", 256, 512, (12, 5, 8, 64))]
