"""Host logic of the batched launch (no GPU): ps_batch_describe.

The batch scheduler decides per run whether its state stays in one CTA's
shared memory, runs on one CTA tile by tile, or goes to a lane of CTAs; which
tile bits it uses; and which lane takes it (longest first onto the least
loaded lane).  Its windows must be exactly those of the single-run scheduler
with the same knobs.
"""
import numpy as np
import pytest

import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs


def runs_for(ns, seed=3, count=600):
    out = []
    for i, n in enumerate(ns):
        x, z, h = inputs.jw_hamiltonian(n, 120 if n >= 8 else 8, seed=seed * 100 + i)
        H = ps.Hamiltonian(n, x, z, h)
        xs, zs, ph = H.qdrift_stream(0.5, count + 37 * i, seed + i)
        out.append(dict(n=n, x=xs, z=zs, phi=ph))
    return out


@pytest.mark.parametrize("dtype", [ps.PS_C64, ps.PS_C128])
def test_kinds_and_tile_bits(dtype):
    ns = [4, 9, 12, 13, 14, 15, 16, 18, 22]
    d = ps.ps_batch_describe(dtype, runs_for(ns), dict(lane_size=16))
    res = 13 if dtype == ps.PS_C64 else 12
    bmax = res
    for n, lane, tb in zip(ns, d["lane_of"], d["tile_bits_of"]):
        if n <= res:
            assert lane == -2 and tb == n
        elif n == res + 1:
            assert lane == -1 and tb == min(bmax, n)
        else:
            assert 0 <= lane < d["lanes"]
            assert tb == min(bmax, max(8, n - 4), n)
    assert d["grid"] == 152 * 3 and d["lanes"] == (152 * 3) // 16


@pytest.mark.parametrize("dtype", [ps.PS_C64, ps.PS_C128])
def test_windows_equal_single_run_schedule(dtype):
    ns = [7, 12, 14, 16, 19]
    runs = runs_for(ns, seed=4)
    d = ps.ps_batch_describe(dtype, runs, dict(lane_size=8, tile_bits=11))
    tot = 0
    amp = 0.0
    for r, tb, nw in zip(runs, d["tile_bits_of"], d["windows_of"]):
        info = ps.ps_plan_describe(r["n"], dtype, r["x"], r["z"], r["phi"],
                                   dict(tile_bits=max(6, int(tb)), group_bits=3,
                                        max_window=32 if dtype == ps.PS_C64 else 24, pair_single=2))
        assert info["windows"] == nw and info["pair_windows"] == 0
        tot += int(nw)
        amp += float(2 ** r["n"]) * int(nw)
    assert d["windows"] == tot
    assert d["amplitude_passes"] == amp
    assert d["rotations"] == sum(len(r["x"]) for r in runs)


def test_lanes_are_filled_longest_first():
    rng = np.random.default_rng(1)
    ns = [int(v) for v in rng.integers(15, 21, size=40)]
    runs = runs_for(ns, seed=5, count=300)
    d = ps.ps_batch_describe(ps.PS_C64, runs, dict(lane_size=64, resident_bits=-1, single_bits=-1), num_sms=16,
                             ctas_per_sm=4)
    lanes = d["lanes"]
    assert lanes == 1 and np.all(d["lane_of"] == 0)
    d = ps.ps_batch_describe(ps.PS_C64, runs, dict(lane_size=4, resident_bits=-1, single_bits=-1), num_sms=16,
                             ctas_per_sm=4)
    lanes = d["lanes"]
    assert lanes == 16
    work = np.array([2.0 ** r["n"] * (int(w) + 1) for r, w in zip(runs, d["windows_of"])])
    load = np.zeros(lanes)
    for w, l in zip(work, d["lane_of"]):
        load[l] += w
    assert d["max_lane_work"] == load.max()
    # greedy longest-first: no lane exceeds the mean by more than one run
    assert load.max() <= work.sum() / lanes + work.max()
    # replay the greedy rule
    order = sorted(range(len(runs)), key=lambda i: (-work[i], i))
    sim = np.zeros(lanes)
    for i in order:
        l = int(np.argmin(sim))
        assert d["lane_of"][i] == l
        sim[l] += work[i]


def test_describe_validation():
    runs = runs_for([10])
    for cfg in [dict(lane_size=3), dict(lane_size=512), dict(tile_bits=7), dict(tile_bits=14),
                dict(resident_bits=14), dict(use_graph=2), dict(wait_ms=-5), dict(test_withhold=2)]:
        with pytest.raises(ps.PsError) as e:
            ps.ps_batch_describe(ps.PS_C64, runs, cfg)
        assert e.value.code == ps.PS_ERR_ARG
    with pytest.raises(ps.PsError):
        ps.ps_batch_describe(ps.PS_C128, runs, dict(tile_bits=13))
    for n in (3, 31):
        with pytest.raises(ps.PsError):
            ps.ps_batch_describe(ps.PS_C64, [dict(n=n, x=[], z=[], phi=[])])
    bad = runs_for([10])
    bad[0]["x"] = np.array(bad[0]["x"], dtype=np.uint64)
    bad[0]["x"][0] = 1 << 10
    with pytest.raises(ps.PsError):
        ps.ps_batch_describe(ps.PS_C64, bad)
    # the timeout test hook needs a lane run in lane 0
    with pytest.raises(ps.PsError):
        ps.ps_batch_describe(ps.PS_C64, runs, dict(test_withhold=1))
    ps.ps_batch_describe(ps.PS_C64, runs_for([16]), dict(test_withhold=1, lane_size=4))


def test_empty_runs_have_no_windows():
    d = ps.ps_batch_describe(ps.PS_C64, [dict(n=12, x=[], z=[], phi=[]), dict(n=20, x=[], z=[], phi=[])])
    assert list(d["windows_of"]) == [0, 0] and d["windows"] == 0
