"""GPU: the batched persistent launch (ps_batch_*) against single runs and the oracle.

Every run of a batch must give the state and overlap that the same rotation
list gives on its own (ps_apply_rotations on a state handle), which the
single-run tests tie to the oracle; small complex128 runs are also compared
with the oracle directly.  The batch uses its own windows (other tile bits,
at most 32 complex64 or 24 complex128 rotations each), so the complex64
comparison allows the rounding of two different schedules: 2e-5 relative L2
for up to ~2000 rotations (sqrt(m) * 1e-7 per schedule, twice).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs

pytestmark = pytest.mark.gpu

TDT = {ps.PS_C128: torch.complex128, ps.PS_C64: torch.complex64}
TOL = {ps.PS_C128: 1e-12, ps.PS_C64: 2e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make_runs(ns, seed, rot_lo=200, rot_hi=1500):
    """Alternating qDRIFT and partially randomised runs on JW-like Hamiltonians."""
    rng = np.random.default_rng(seed)
    runs = []
    for i, n in enumerate(ns):
        L = int(rng.integers(40, 300)) if n >= 8 else 20
        x, z, h = inputs.jw_hamiltonian(n, L, seed=seed * 1000 + i)
        # the rotation streams come from the oracle's sampler, so that every
        # reference the runs are compared with is computed from oracle inputs
        if i % 2 == 0:
            xs, zs, ph = oracle.qdrift_stream(x, z, h, 0.7, int(rng.integers(rot_lo, rot_hi)), seed + i)
        else:
            L_D = max(1, L // 10)
            xs, zs, ph = oracle.partial_stream(x, z, h, L_D, 0.7, 2, int(rng.integers(rot_lo, rot_hi)) // 2, seed + i)
        runs.append(dict(n=n, x=xs, z=zs, phi=ph, host0=inputs.gaussian_state(n, seed * 1000 + 500 + i)))
    return runs


def device_runs(runs, dtype):
    out = []
    for r in runs:
        p0 = torch.as_tensor(r["host0"]).to(TDT[dtype]).cuda()
        out.append(dict(n=r["n"], x=r["x"], z=r["z"], phi=r["phi"], psi0=p0))
    return out


def single_run(r, dtype):
    st = ps.StateVector(r["n"], dtype=TDT[dtype])
    st.load(r["host0"])
    st.apply_rotations(r["x"], r["z"], r["phi"])
    return st.to_numpy()


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_batch_matches_single_runs(dtype):
    # resident (n <= 13 / 12), single-CTA (14 / 13) and lane runs, one empty run
    ns = [6, 9, 12, 13, 14, 15, 16, 17, 18, 12, 15, 16]
    runs = make_runs(ns, seed=21)
    runs.append(dict(n=10, x=[], z=[], phi=[], host0=inputs.gaussian_state(10, 99)))
    b = ps.Batch(device_runs(runs, dtype), dtype=TDT[dtype], cfg=dict(lane_size=8))
    info = b.info
    assert info["resident_runs"] > 0 and info["single_runs"] > 0 and info["lane_runs"] > 0
    g = b.run()
    for i, r in enumerate(runs):
        got = b.states[i].cpu().numpy().astype(np.complex128)
        ref = single_run(r, dtype) if len(r["x"]) else r["host0"]
        assert rel(got, ref) < TOL[dtype], (i, r["n"])
        g_ref = np.vdot(r["host0"], ref)
        assert abs(g[i] - g_ref) < TOL[dtype] * max(1.0, abs(g_ref)), (i, g[i], g_ref)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_batch_smallest_states_vs_oracle(dtype):
    # n = 4 and 5: tiles smaller than one thread's register groups leave most
    # of the CTA without rotation work (one or two active threads)
    runs = make_runs([4, 5, 4, 5, 7], seed=41, rot_lo=50, rot_hi=200)
    b = ps.Batch(device_runs(runs, dtype), dtype=TDT[dtype], cfg=dict(lane_size=8))
    g = b.run()
    for i, r in enumerate(runs):
        ref = oracle.apply(r["host0"], r["x"], r["z"], r["phi"])
        assert rel(b.states[i].cpu().numpy(), ref) < TOL[dtype], (i, r["n"])
        g_ref = oracle.overlap(r["host0"], ref)
        assert abs(g[i] - g_ref) < TOL[dtype] * max(1.0, abs(g_ref)), (i, g[i], g_ref)


def test_batch_complex128_vs_oracle():
    runs = make_runs([8, 11, 13, 14, 16], seed=5, rot_lo=100, rot_hi=300)
    b = ps.Batch(device_runs(runs, ps.PS_C128), dtype=torch.complex128, cfg=dict(lane_size=4))
    g = b.run()
    for i, r in enumerate(runs):
        ref = oracle.apply(r["host0"], r["x"], r["z"], r["phi"])
        assert rel(b.states[i].cpu().numpy(), ref) < 1e-12
        g_ref = oracle.overlap(r["host0"], ref)
        assert abs(g[i] - g_ref) < 1e-12 * max(1.0, abs(g_ref))


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_batch_replay_is_bitwise_deterministic(dtype):
    runs = make_runs([10, 13, 14, 17, 18, 16], seed=8)
    b = ps.Batch(device_runs(runs, dtype), dtype=TDT[dtype], cfg=dict(lane_size=16))
    g1 = b.run()
    s1 = [s.clone() for s in b.states]
    g2 = b.run()
    assert np.array_equal(g1, g2)
    for a, c in zip(s1, b.states):
        assert torch.equal(a, c)


def test_batch_graph_and_plain_launch_agree_bitwise():
    runs = make_runs([12, 15, 17], seed=9)
    dev = device_runs(runs, ps.PS_C64)
    bg = ps.Batch(dev, cfg=dict(lane_size=8, use_graph=1))
    bp = ps.Batch(dev, cfg=dict(lane_size=8, use_graph=-1))
    assert bp.info["graph"] == 0
    g1, g2 = bg.run(), bp.run()
    assert np.array_equal(g1, g2)
    for a, c in zip(bg.states, bp.states):
        assert torch.equal(a, c)


@pytest.mark.parametrize("cfg", [dict(lane_size=1), dict(lane_size=2, tile_bits=8), dict(lane_size=32, tile_bits=10),
                                 dict(lane_size=64, resident_bits=-1, single_bits=-1),
                                 dict(lane_size=8, resident_bits=9, single_bits=16)])
def test_batch_configurations_agree(cfg):
    runs = make_runs([8, 12, 14, 16, 18], seed=10)
    dev = device_runs(runs, ps.PS_C128)
    g = ps.Batch(dev, dtype=torch.complex128, cfg=cfg).run()
    for i, r in enumerate(runs):
        ref = single_run(r, ps.PS_C128)
        assert abs(g[i] - np.vdot(r["host0"], ref)) < 1e-12


def test_batch_without_psi0_evolves_in_place():
    runs = make_runs([11, 15], seed=12)
    states = [torch.as_tensor(r["host0"]).to(torch.complex64).cuda() for r in runs]
    dev = [dict(n=r["n"], x=r["x"], z=r["z"], phi=r["phi"], state=s) for r, s in zip(runs, states)]
    b = ps.Batch(dev, cfg=dict(lane_size=8))
    g = b.run()
    assert np.all(g == 0)
    for r, s in zip(runs, b.states):
        assert rel(s.cpu().numpy(), single_run(r, ps.PS_C64)) < TOL[ps.PS_C64]


def test_batch_rejects_shared_state_and_aliasing():
    runs = make_runs([10, 10], seed=13)
    s = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    dev = [dict(n=10, x=r["x"], z=r["z"], phi=r["phi"], state=s) for r in runs]
    with pytest.raises(ps.PsError) as e:
        ps.Batch(dev)
    assert e.value.code == ps.PS_ERR_ARG
    dev = [dict(n=10, x=runs[0]["x"], z=runs[0]["z"], phi=runs[0]["phi"], state=s, psi0=s)]
    with pytest.raises(ps.PsError):
        ps.Batch(dev)


def test_batch_wait_timeout_returns_status_and_context_survives():
    # The last CTA of lane 0 never arrives at its lane's barrier (test hook),
    # so the other members' bounded waits run out after 200 ms.
    runs = make_runs([16, 16], seed=14)
    dev = device_runs(runs, ps.PS_C64)
    b = ps.Batch(dev, cfg=dict(lane_size=4, wait_ms=200, test_withhold=1, single_bits=-1, resident_bits=-1))
    with pytest.raises(ps.PsError) as e:
        b.run()
    assert e.value.code == ps.PS_ERR_TIMEOUT
    b.close()
    # the context is intact: a normal batch and a single run still work
    g = ps.Batch(dev, cfg=dict(lane_size=4)).run()
    for i, r in enumerate(runs):
        ref = single_run(r, ps.PS_C64)
        assert abs(g[i] - np.vdot(r["host0"], ref)) < 2e-5


def test_batch_config4_shape_sampled_runs():
    """A scaled-down batch of the 512-run shape: n in 14..22, qDRIFT and partial
    runs; every run against its single-run result (complex64) by overlap, and
    three full states."""
    rng = np.random.default_rng(5)
    ns = [int(v) for v in rng.integers(14, 23, size=24)]
    runs = make_runs(ns, seed=31, rot_lo=300, rot_hi=800)
    b = ps.Batch(device_runs(runs, ps.PS_C64), cfg=dict(lane_size=16))
    g = b.run()
    for i, r in enumerate(runs):
        ref = single_run(r, ps.PS_C64)
        assert abs(g[i] - np.vdot(r["host0"], ref)) < 2e-5, (i, r["n"])
        if i < 3:
            assert rel(b.states[i].cpu().numpy(), ref) < 2e-5
