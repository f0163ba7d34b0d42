"""The autotuner's on-disk cache (paper_1301_4019_gb300/tune.py) without a GPU: the library
calls are replaced by fakes, so only the keying, the reuse and the repair logic run."""
import json

import torch

from paper_1301_4019_gb300 import tune


def _fakes(shapes=((128, 2), (512, 1))):
    calls, sets = [], []

    def fake_tune(h, logw, offsets, B=0, B_per_filter=None, reps=3):
        calls.append((logw.dtype, logw.numel()))
        return {"metropolis": shapes[0], "permute": shapes[1]}

    def fake_set(h, kernel, block, ipt):
        if block % 32:
            raise ValueError("bad shape")
        sets.append((kernel, block, ipt))
    return calls, sets, fake_tune, fake_set


def test_cache_key_classes():
    k = tune.cache_key("GB300", torch.float32, 3000, 5)
    assert k == "GB300|metropolis|f32|N2^12|F2^2"
    assert tune.cache_key("GB300", torch.float64, 3000, 5) != k
    assert tune.cache_key("GB300", torch.float32, 2900, 5) == k      # same size class
    assert tune.cache_key("GB300", torch.float32, 6000, 5) != k
    assert tune.cache_key("other", torch.float32, 3000, 5) != k


def test_tune_once_then_reuse(tmp_path):
    calls, sets, ft, fs = _fakes()
    path = str(tmp_path / "c" / "shapes.json")
    lw, off = torch.zeros(3000), torch.tensor([0, 1000, 3000])
    r = tune.autotune_batched(None, lw, off, cache_path=path, gpu="G", _tune=ft, _set=fs)
    assert not r["cached"] and len(calls) == 1 and sets == []
    r = tune.autotune_batched(None, lw, off, cache_path=path, gpu="G", _tune=ft, _set=fs)
    assert r["cached"] and len(calls) == 1
    assert sets == [(0, 128, 2), (2, 512, 1)]
    tune.autotune_batched(None, lw.double(), off, cache_path=path, gpu="G", _tune=ft, _set=fs)
    assert len(calls) == 2 and sets[-2][0] != 1  # binary64: tuned, not taken from binary32
    data = json.load(open(path))
    assert len(data) == 2 and all(set(v) == {"metropolis", "permute"} for v in data.values())


def test_damaged_entry_is_tuned_again(tmp_path):
    calls, sets, ft, fs = _fakes()
    path = tmp_path / "shapes.json"
    lw, off = torch.zeros(100), torch.tensor([0, 100])
    key = tune.cache_key("G", torch.float32, 100, 1)
    path.write_text(json.dumps({key: {"metropolis": [100, 1], "permute": [256, 1]}}))
    r = tune.autotune_batched(None, lw, off, cache_path=str(path), gpu="G", _tune=ft, _set=fs)
    assert not r["cached"] and len(calls) == 1
    assert json.load(open(path))[key]["metropolis"] == [128, 2]
    path.write_text("not json")
    r = tune.autotune_batched(None, lw, off, cache_path=str(path), gpu="G", _tune=ft, _set=fs)
    assert not r["cached"] and len(calls) == 2
