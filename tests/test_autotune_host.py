"""Host logic of the autotuner (no GPU): workload signature and JSON cache."""
import json

from paper_2602_03207_gb300 import autotune


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    assert autotune._load() == {}
    autotune._save({"sig": {"tile": 16, "digit_bits": 9, "ms": 1.0}})
    assert json.load(open(autotune.cache_path()))["sig"]["tile"] == 16
    assert autotune._load()["sig"]["digit_bits"] == 9


def test_signature_depends_on_resolutions(monkeypatch):
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d=None: "GPU")
    a = autotune.signature(10, [{"width": 32, "height": 16}])
    b = autotune.signature(10, [{"width": 16, "height": 32}])
    c = autotune.signature(11, [{"width": 32, "height": 16}])
    assert len({a, b, c}) == 3
