"""Host logic of the batched-launch autotuner (no GPU): the batch signature,
the staged search and the JSON cache.  Launch timing is replaced by a cost
function of the configuration, so the test checks which candidates the tuner
tries, in which order of stages, and what it keeps."""
import json

import pytest
import torch

import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import autotune


def runs_for(ns, rot=100):
    return [dict(n=n, x=[1] * rot, z=[0] * rot, phi=[0.1] * rot, psi0=torch.zeros(1 << n, dtype=torch.complex64))
            for n in ns]


def test_signature_depends_on_the_work_histogram_only():
    a = runs_for([14, 16, 16, 18])
    b = list(reversed(a))
    s = autotune.signature(a, ps.PS_C64, "GPU")
    assert s == autotune.signature(b, ps.PS_C64, "GPU")
    assert s != autotune.signature(a, ps.PS_C128, "GPU")
    assert s != autotune.signature(a, ps.PS_C64, "other GPU")
    assert s != autotune.signature(runs_for([14, 16, 16, 19]), ps.PS_C64, "GPU")
    # rotation counts enter rounded to two significant digits
    assert autotune.signature(runs_for([14], rot=1001), ps.PS_C64, "GPU") == \
        autotune.signature(runs_for([14], rot=1004), ps.PS_C64, "GPU")
    assert autotune.signature(runs_for([14], rot=1000), ps.PS_C64, "GPU") != \
        autotune.signature(runs_for([14], rot=1200), ps.PS_C64, "GPU")


class FakeBatch:
    made = []

    def __init__(self, runs, dtype=None, cfg=None):
        self.cfg = dict(cfg or {})
        FakeBatch.made.append(self.cfg)

    def close(self):
        pass


def cost(cfg):
    """A made-up launch time with its minimum at lane 16, tile bits 12, single 16."""
    t = 100.0 + abs(cfg["lane_size"] - 16) / 4
    t += 3.0 * abs(cfg.get("tile_bits", 13) - 12)
    t += 0.5 * abs((cfg.get("single_bits") or 14) - 16)
    return t


@pytest.fixture
def fake_device(monkeypatch, tmp_path):
    FakeBatch.made = []
    monkeypatch.setattr(autotune, "Batch", FakeBatch)
    monkeypatch.setattr(autotune, "time_batch", lambda b, reps=2: cost(b.cfg))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "fake GB300")
    monkeypatch.setenv("PS_TUNE_CACHE", str(tmp_path / "tune.json"))
    return tmp_path / "tune.json"


def test_staged_search_and_cache(fake_device):
    runs = runs_for([14, 15, 17, 20, 22])
    res = autotune.tune_batch(runs)
    assert res["cached"] is False
    assert (res["lane_size"], res["tile_bits"], res["single_bits"]) == (16, 12, 16)
    assert res["ms"] == pytest.approx(cost({"lane_size": 16, "tile_bits": 12, "single_bits": 16}))
    # stage 1 tries every lane size alone; stage 2 every tile size at the best lane; stage 3 the single sizes
    tried = [json.dumps(c, sort_keys=True) for c in FakeBatch.made]
    assert len(tried) == len(set(tried))  # each candidate is timed once
    assert [c for c in FakeBatch.made if set(c) == {"lane_size"}] == [{"lane_size": s} for s in autotune.LANE_SIZES]
    stage2 = [c for c in FakeBatch.made if set(c) == {"lane_size", "tile_bits"}]
    assert {c["lane_size"] for c in stage2} == {16}
    assert sorted(c["tile_bits"] for c in stage2) == sorted(autotune.TILE_BITS[ps.PS_C64])
    stage3 = [c for c in FakeBatch.made if "single_bits" in c]
    assert sorted(c["single_bits"] for c in stage3) == sorted(s for s in autotune.SINGLE_BITS if s is not None)
    assert len(res["timings_ms"]) == len(FakeBatch.made)
    # the cache holds the result under the signature; the next call makes no batch
    db = json.loads(fake_device.read_text())
    assert res["signature"] in db and db[res["signature"]]["lane_size"] == 16
    n_made = len(FakeBatch.made)
    again = autotune.tune_batch(runs)
    assert again["cached"] is True and len(FakeBatch.made) == n_made
    assert (again["lane_size"], again["tile_bits"], again["single_bits"]) == (16, 12, 16)
    # without the cache it searches again and finds the same
    fresh = autotune.tune_batch(runs, use_cache=False)
    assert fresh["cached"] is False and len(FakeBatch.made) > n_made
    assert (fresh["lane_size"], fresh["tile_bits"], fresh["single_bits"]) == (16, 12, 16)


def test_default_single_size_is_kept_when_it_wins(fake_device, monkeypatch):
    monkeypatch.setattr(autotune, "time_batch", lambda b, reps=2: cost(b.cfg) + (0.0 if "single_bits" not in b.cfg
                                                                                 else 5.0))
    res = autotune.tune_batch(runs_for([16, 18]), use_cache=False)
    assert "single_bits" not in res
    assert res["ms"] == pytest.approx(cost({"lane_size": 16, "tile_bits": 12}))


def test_complex128_uses_its_tile_sizes(fake_device):
    runs = [dict(r, psi0=r["psi0"].to(torch.complex128)) for r in runs_for([15, 19])]
    res = autotune.tune_batch(runs, dtype=torch.complex128, use_cache=False)
    stage2 = [c["tile_bits"] for c in FakeBatch.made if set(c) == {"lane_size", "tile_bits"}]
    assert sorted(stage2) == sorted(autotune.TILE_BITS[ps.PS_C128])
    assert res["tile_bits"] == 12
