"""Host logic of the autotune cache (no GPU): the shipped GB300 results are
well-formed plan configurations, and a lookup takes the user's cache first,
then the shipped file, and only then runs (and stores) a new search."""
from __future__ import annotations

import json
import os

import pytest

from paper_1707_07263_gb300 import _lib, tune


def _read_json(path):
    with open(path) as f:
        return json.load(f)


def test_shipped_entries_are_well_formed():
    shipped = _read_json(tune.SHIPPED)
    fields = [name for name, _ in _lib.FftPlanConfig._fields_]
    assert shipped
    for k, v in shipped.items():
        if "|many|" in k:
            # uneven batch: GPU | many | count=C | lengths=<digest>, an fft_many_config
            dev, kind, count, digest = k.split("|")
            assert dev and int(count[6:]) >= 1 and len(digest) == len("lengths=") + 16, k
            c = v["config"]
            assert sorted(c) == ["ctas_per_sm", "gap", "lg1"] and 1 <= c["gap"] <= 16 and c["ctas_per_sm"] >= 1, k
            assert len(c["lg1"]) == 4 and all(7 <= c["lg1"][i] <= 8 and 6 <= 13 + i - c["lg1"][i] <= 8
                                              for i in range(4)), k
            assert _lib.FftManyConfig.from_dict(c).as_dict() == c and v["us"] > 0
            continue
        dev, n, batch, prec = k.split("|")
        n, batch, prec = int(n[2:]), int(batch[6:]), int(prec[5:])
        lg = n.bit_length() - 1
        assert dev and n == 1 << lg and batch >= 1 and prec == _lib.FFT_PREC_FP32, k
        c = v["config"]
        assert sorted(c) == sorted(fields), k
        assert v["us"] > 0
        assert c["tma"] in (-1, 0, 1, 2, 3) and c["fused"] in (-1, 0, 1) and c["halves"] in (0, 1, 2)
        assert c["radix"] == 16 or (c["radix"] in (4, 8) and c["npass"] == 1 and c["tma"] == 0), k
        if c["npass"] == 1:
            assert c["lg1"] == lg <= 14, k
        elif c["npass"] == 2:
            assert c["lg1"] + c["lg2"] == lg and c["c1"] >= 1 and c["c2"] >= 1, k
        else:
            assert c["npass"] == 3 and 0 < c["lg1"] + c["lg2"] < lg and min(c["c1"], c["c2"], c["c3"]) >= 1, k
        assert _lib.FftPlanConfig.from_dict(c).as_dict() == c


@pytest.fixture
def fake_tuner(tmp_path, monkeypatch):
    calls = []
    monkeypatch.setenv("GBFFT_TUNE_CACHE", str(tmp_path / "cache" / "tune.json"))
    shipped = tmp_path / "shipped.json"
    shipped.write_text(json.dumps({"dev|n=64|batch=8|prec=0": {"config": {"npass": 1, "lg1": 6}, "us": 1.0}}))
    monkeypatch.setattr(tune, "SHIPPED", str(shipped))
    monkeypatch.setattr(tune, "key", lambda n, batch, prec, device: f"dev|n={n}|batch={batch}|prec={prec}")

    def autotune(n, batch, prec, device):
        calls.append((n, batch, prec))
        return {"npass": 1, "lg1": n.bit_length() - 1, "tma": len(calls)}, 2.0

    monkeypatch.setattr(tune, "autotune", autotune)
    return calls


def test_lookup_order(fake_tuner):
    calls = fake_tuner
    assert tune.tuned_config(64, 8, 0, device="cpu") == {"npass": 1, "lg1": 6}   # shipped
    assert calls == [] and not os.path.exists(tune.cache_path())
    cfg = tune.tuned_config(128, 8, 0, device="cpu")                            # neither: search
    assert calls == [(128, 8, 0)] and cfg["tma"] == 1
    stored = _read_json(tune.cache_path())
    assert stored["dev|n=128|batch=8|prec=0"]["config"] == cfg
    assert tune.tuned_config(128, 8, 0, device="cpu") == cfg and len(calls) == 1  # cached
    cfg2 = tune.tuned_config(64, 8, 0, device="cpu", retune=True)               # forced search
    assert len(calls) == 2 and cfg2["tma"] == 2
    assert tune.tuned_config(64, 8, 0, device="cpu") == cfg2                   # user cache before shipped
    assert os.listdir(os.path.dirname(tune.cache_path())) == ["tune.json"]    # no temporary left


def test_corrupt_cache_is_replaced(fake_tuner):
    path = tune.cache_path()
    os.makedirs(os.path.dirname(path))
    with open(path, "w") as f:
        f.write("{not json")
    cfg = tune.tuned_config(256, 2, 0, device="cpu")
    assert fake_tuner == [(256, 2, 0)]
    assert _read_json(path) == {"dev|n=256|batch=2|prec=0": {"config": cfg, "us": 2.0}}


def test_many_key_is_the_length_list(monkeypatch):
    """The uneven-batch cache key depends on the GPU model and on the exact
    length list (order included), not on anything else."""
    monkeypatch.setattr(tune.torch.cuda, "get_device_name", lambda d=None: "Some GPU")
    a = tune.many_key([256, 512, 8192], 0)
    assert a.startswith("Some_GPU|many|count=3|lengths=")
    assert tune.many_key([256, 512, 8192], 0) == a
    assert tune.many_key([512, 256, 8192], 0) != a
    assert tune.many_key([256, 512], 0) != a
