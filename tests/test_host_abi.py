"""Host-side checks of libps that need no GPU.

* the shared library loads and exports every function include/ps.h declares;
* argument validation fails with PS_ERR_ARG before any CUDA call;
* the product-formula streams libps generates on the host, applied by the
  oracle, reproduce the oracle's own Trotter / qDRIFT / partially randomised
  runs bit for bit (same rotations, same order, same angles);
* the scheduler's windows obey the coset construction of Eq. 1 in its
  single-GPU form, checked mask by mask and by applying each window tile by
  tile in tile coordinates (a numpy model of the kernel's index algebra).
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import _lib, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ps_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert not [n for n in names if not hasattr(ps, n)]


def test_abi_version_and_empty_error():
    assert ps.ps_abi_version() == 3
    assert isinstance(ps.ps_last_error(), str)


def test_create_rejects_bad_arguments_without_gpu():
    with pytest.raises(ps.PsError) as e:
        ps.ps_create(10, ps.PS_C64, 0, 0)
    assert e.value.code == _lib.PS_ERR_ARG and "null" in str(e.value)
    with pytest.raises(ps.PsError):
        ps.ps_create(0, ps.PS_C64, 4096, 0)
    with pytest.raises(ps.PsError):
        ps.ps_create(41, ps.PS_C64, 4096, 0)
    with pytest.raises(ps.PsError):
        ps.ps_create(10, 7, 4096, 0)
    with pytest.raises(ps.PsError) as e:
        ps.ps_create(10, ps.PS_C64, 4100, 0)
    assert "aligned" in str(e.value)


def test_hamiltonian_validation():
    with pytest.raises(ps.PsError) as e:
        ps.ps_ham_create(4, [1 << 4], [0], [1.0])
    assert "mask bit" in str(e.value)
    with pytest.raises(ps.PsError):
        ps.ps_ham_create(4, [], [], [])
    with pytest.raises(ps.PsError):
        ps.ps_ham_create(4, [1], [0], [float("nan")])
    h = ps.ps_ham_create(4, [1, 2], [0, 2], [0.5, -1.5])
    assert abs(ps.ps_ham_lambda(h) - 2.0) < 1e-15
    ps.ps_ham_destroy(h)


def test_plan_validation():
    with pytest.raises(ps.PsError) as e:
        ps.ps_plan_describe(8, ps.PS_C64, [1 << 8], [0], [0.1])
    assert "mask bit" in str(e.value)
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(8, ps.PS_C64, [1], [0], [float("inf")])
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"tile_bits": 14})
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(20, ps.PS_C128, [1], [0], [0.1], {"tile_bits": 13})
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"group_bits": 6})
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"max_window": 300})
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"seg_bits": 14})
    with pytest.raises(ps.PsError):
        ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"tile_bits": 10, "seg_bits": 11})
    for bad in (32, 96, 1024):
        with pytest.raises(ps.PsError):
            ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"tile_threads": bad})
    for good in (64, 128, 256, 512):
        ps.ps_plan_describe(20, ps.PS_C64, [1], [0], [0.1], {"tile_threads": good})
    info = ps.ps_plan_describe(20, ps.PS_C64, [], [], [])
    assert info["windows"] == 0


# ------------------------------------------------- streams vs the oracle

def _ham(n, L, seed):
    x, z, h = inputs.jw_hamiltonian(n, L, seed)
    return x, z, h, ps.Hamiltonian(n, x, z, h)


def test_qdrift_stream_matches_oracle_sampler_bit_exact():
    x, z, h, H = _ham(10, 300, 5)
    N, t, seed = 5000, 1.7, 99
    idx = oracle.qdrift_indices(h, seed, 0, N).astype(np.int64)
    xs, zs, phis = H.qdrift_stream(t, N, seed)
    assert np.array_equal(xs, x[idx]) and np.array_equal(zs, z[idx])
    lam = 0.0
    for v in h:  # running sum in term order, as the sampler defines lambda
        lam += abs(float(v))
    tau = lam * t / N
    assert np.array_equal(phis, np.where(h[idx] > 0, tau, -tau))
    # a segment equals the slice of the whole run
    xs2, zs2, ph2 = H.qdrift_stream(t, N, seed, first=1234, count=777)
    assert np.array_equal(xs2, xs[1234:2011]) and np.array_equal(ph2, phis[1234:2011])


def test_streams_applied_by_oracle_reproduce_oracle_drivers():
    n = 6
    x, z, h, H = _ham(n, 20, 8)
    psi = inputs.gaussian_state(n, 9)
    # qDRIFT
    xs, zs, ph = H.qdrift_stream(0.8, 64, 3)
    assert np.array_equal(oracle.apply(psi, xs, zs, ph), oracle.qdrift(psi, x, z, h, 0.8, 64, 3))
    # partially randomised, several steps
    xs, zs, ph = H.partial_stream(5, 0.9, 3, 7, 11)
    assert xs.size == 3 * (5 + 7)
    assert np.array_equal(oracle.apply(psi, xs, zs, ph), oracle.partial(psi, x, z, h, 5, 0.9, 3, 7, 11))
    # its deterministic part is exactly the oracle's split, in term order
    xs, zs, ph = H.partial_stream(6, 1.0, 1, 0, 0)
    det = oracle.partial_split(h, 6)
    assert np.array_equal(xs, x[det]) and np.array_equal(ph, h[det])
    # L_D = L: Trotter
    xs, zs, ph = H.partial_stream(20, 0.9, 2, 4, 1)
    assert np.array_equal(oracle.apply(psi, xs, zs, ph), oracle.trotter(psi, x, z, h, 0.9, 2))


# ------------------------------------------------------------ scheduler

def _parity(v):
    return bin(int(v)).count("1") & 1


def _deposit(H, c, pivots):
    k = int(H) << c
    for p in sorted(pivots):
        k = ((k >> p) << (p + 1)) | (k & ((1 << p) - 1))
    return k


def _check_plan(n, dtype, x, z, phi, tuning=None):
    ex = ps.ps_plan_export(n, dtype, x, z, phi, tuning)
    tun = {"tile_bits": 13 if dtype == ps.PS_C64 else 12, "max_window": 64}
    tun.update(tuning or {})
    B = min(tun["tile_bits"], n)
    cmin = min(tun.get("seg_bits", 4 if dtype == ps.PS_C64 else 3), B)
    wo = ex["window_of"]
    m = len(x)
    assert np.all(np.diff(wo.astype(np.int64)) >= 0) and (m == 0 or wo[0] == 0)
    nw = len(ex["kind"])
    assert m == 0 or wo[-1] == nw - 1
    for w in range(nw):
        members = np.flatnonzero(wo == w)
        assert members.size >= 1 and members.size <= tun["max_window"]
        if ex["kind"][w] == 1:
            assert members.size == 1 and x[members[0]] != 0
            continue
        c, d = int(ex["c"][w]), int(ex["d"][w])
        assert c + d == B
        if B < n:
            assert c >= cmin
        basis = [int(v) for v in ex["basis"][w][:d]]
        tops = [v.bit_length() - 1 for v in basis]
        assert len(set(tops)) == d and all(v & ((1 << c) - 1) == 0 for v in basis)
        for j in members:
            xt, zt = int(ex["xt"][j]), int(ex["zt"][j])
            rebuilt = xt & ((1 << c) - 1)
            for i in range(d):
                if (xt >> (c + i)) & 1:
                    rebuilt ^= basis[i]
            assert rebuilt == int(x[j])
            assert zt & ((1 << c) - 1) == int(z[j]) & ((1 << c) - 1)
            for i in range(d):
                assert (zt >> (c + i)) & 1 == _parity(basis[i] & int(z[j]))
    return ex, B


def _apply_plan_model(n, x, z, phi, ex, B):
    """Apply each tile window coset by coset in tile coordinates (gather form)."""
    psi = inputs.gaussian_state(n, 1)
    out = psi.copy()
    for w in range(len(ex["kind"])):
        members = np.flatnonzero(ex["window_of"] == w)
        if ex["kind"][w] == 1:
            out = oracle.apply(out, x[members], z[members], phi[members])
            continue
        c, d = int(ex["c"][w]), int(ex["d"][w])
        basis = [int(v) for v in ex["basis"][w][:d]]
        pivots = [v.bit_length() - 1 for v in basis]
        t = np.arange(1 << B)
        V = np.zeros(1 << d, dtype=np.int64)
        for s in range(1 << d):
            for i in range(d):
                if (s >> i) & 1:
                    V[s] ^= basis[i]
        for H in range(1 << (n - B)):
            k0 = _deposit(H, c, pivots)
            gidx = k0 ^ V[t >> c] ^ (t & ((1 << c) - 1))
            a = out[gidx].copy()
            for j in members:
                xt, zt = int(ex["xt"][j]), int(ex["zt"][j])
                y = _parity_count = bin(int(x[j]) & int(z[j])).count("1") % 4
                sig = np.array([_parity(tt & zt) ^ _parity(k0 & int(z[j])) for tt in t])
                coef = 1j * np.sin(phi[j]) * (-1j) ** y * (1 - 2 * sig)
                a = np.cos(phi[j]) * a + coef * a[t ^ xt]
            out[gidx] = a
    return psi, out


@pytest.mark.parametrize("dtype", [ps.PS_C64, ps.PS_C128])
def test_scheduler_windows_random_strings(dtype):
    n = 12
    x, z, phi = inputs.random_rotations(n, 200, seed=17)
    _check_plan(n, dtype, x, z, phi, {"tile_bits": 8})
    _check_plan(n, dtype, x, z, phi, {"tile_bits": 6, "max_window": 5})
    _check_plan(n, dtype, x, z, phi)  # B = n: a single tile


def test_scheduler_jw_qdrift_fuses_many_rotations_per_pass():
    n = 30
    xh, zh, hh = inputs.jw_hamiltonian(n, 2000, seed=3)
    H = ps.Hamiltonian(n, xh, zh, hh)
    x, z, phi = H.qdrift_stream(1.0, 20000, 4)
    ex, B = _check_plan(n, ps.PS_C64, x, z, phi)
    info = ps.ps_plan_describe(n, ps.PS_C64, x, z, phi)
    rot_per_pass = info["rotations"] / info["windows"]
    # a 2^13 tile with 128-byte segments leaves 9 basis dimensions; JW strings
    # add at most 2 (weight-2) or 4 (weight-4) new X bits each
    assert rot_per_pass >= 3.0, info
    # greedy maximality: the first rotation of the next window would not fit
    for w in range(len(ex["kind"]) - 1):
        members = np.flatnonzero(ex["window_of"] == w)
        if len(members) == 64:
            continue
        vecs = [int(x[j]) >> 4 for j in members] + [int(x[members[-1] + 1]) >> 4]
        assert _rank(vecs) > B - 4


@pytest.mark.parametrize("seg_bits", [1, 2, 3, 4])
def test_scheduler_seg_bits_bounds_the_window_span(seg_bits):
    # c >= seg_bits in every tile window, the span above c fills the rest of
    # the tile, and every maximal window is one rotation short of B - seg_bits + 1
    n = 24
    xh, zh, hh = inputs.jw_hamiltonian(n, 800, seed=13)
    H = ps.Hamiltonian(n, xh, zh, hh)
    x, z, phi = H.qdrift_stream(1.0, 3000, 14)
    tun = {"seg_bits": seg_bits}
    ex = ps.ps_plan_export(n, ps.PS_C64, x, z, phi, tun)
    B = 13
    for w in range(len(ex["kind"]) - 1):
        assert ex["kind"][w] == 0 and ex["c"][w] >= seg_bits and ex["c"][w] + ex["d"][w] == B
        members = np.flatnonzero(ex["window_of"] == w)
        if len(members) == 32:
            continue
        vecs = [int(x[j]) >> seg_bits for j in members] + [int(x[members[-1] + 1]) >> seg_bits]
        assert _rank(vecs) > B - seg_bits
    rp = [ps.ps_plan_describe(n, ps.PS_C64, x, z, phi, {"seg_bits": s})["windows"] for s in (4, 2)]
    assert rp[1] < rp[0]


def _rank(vecs):
    basis = []
    for v in vecs:
        for b in basis:
            v = min(v, v ^ b)
        if v:
            basis.append(v)
    return len(basis)


@pytest.mark.parametrize("n,B", [(10, 6), (11, 8), (9, 9)])
def test_scheduler_model_matches_oracle(n, B):
    x, z, phi = inputs.random_rotations(n, 40, seed=n + B)
    ex, Bu = _check_plan(n, ps.PS_C64, x, z, phi, {"tile_bits": B, "max_window": 7})
    psi, got = _apply_plan_model(n, x, z, phi, ex, Bu)
    ref = oracle.apply(psi, x, z, phi)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("n,B,seg", [(10, 8, 1), (11, 9, 2), (12, 10, 3), (12, 9, 5), (13, 11, 2)])
def test_scheduler_model_with_segment_sizes(n, B, seg):
    # JW qDRIFT windows at every segment size: the exported windows, applied
    # coset by coset in tile coordinates, reproduce the oracle's evolution
    x, z, h, H = _ham(n, 60, 40 + n + seg)
    xs, zs, ph = H.qdrift_stream(1.0, 240, 41 + seg)
    ex, Bu = _check_plan(n, ps.PS_C64, xs, zs, ph, {"tile_bits": B, "seg_bits": seg, "max_window": 32})
    psi, got = _apply_plan_model(n, xs, zs, ph, ex, Bu)
    ref = oracle.apply(psi, xs, zs, ph)
    assert np.max(np.abs(got - ref)) < 1e-12
    # a smaller segment leaves more of the tile to the span: never fewer rotations per window
    info = ps.ps_plan_describe(n, ps.PS_C64, xs, zs, ph, {"tile_bits": B, "seg_bits": seg})
    if seg < min(4, B):
        wider = ps.ps_plan_describe(n, ps.PS_C64, xs, zs, ph, {"tile_bits": B, "seg_bits": min(4, B)})
        assert info["windows"] <= wider["windows"]


def test_second_order_streams_reproduce_oracle_drivers():
    n = 6
    x, z, h, H = _ham(n, 20, 18)
    psi = inputs.gaussian_state(n, 19)
    # merged symmetric steps: r (2L - 2) + 1 rotations
    xs, zs, ph = H.trotter2_stream(0.9, 3)
    assert xs.size == 3 * (2 * 20 - 2) + 1 == ps.ps_trotter2_length(H.handle, 3)
    assert np.max(np.abs(oracle.apply(psi, xs, zs, ph) - oracle.trotter2(psi, x, z, h, 0.9, 3))) < 1e-13
    # a single term is one rotation over the whole time
    x1, z1, h1, H1 = _ham(n, 1, 5)
    xs, zs, ph = H1.trotter2_stream(0.7, 4)
    assert xs.size == 1 and ph[0] == pytest.approx(0.7 * h1[0], rel=1e-15)
    # second-order partial: halves of the deterministic part around 2 Ns draws
    xs, zs, ph = H.partial2_stream(5, 0.9, 3, 7, 11)
    assert xs.size == 3 * (2 * 5 + 2 * 7) - 2 == ps.ps_partial2_length(H.handle, 5, 3, 7)
    got = oracle.apply(psi, xs, zs, ph)
    assert np.max(np.abs(got - oracle.partial2(psi, x, z, h, 5, 0.9, 3, 7, 11))) < 1e-13
    # reductions: L_D = L is second-order Trotter; L_D = 0, r = 1 is qDRIFT with 2 Ns draws
    xs, zs, ph = H.partial2_stream(20, 0.9, 2, 4, 1)
    assert np.max(np.abs(oracle.apply(psi, xs, zs, ph) - oracle.trotter2(psi, x, z, h, 0.9, 2))) < 1e-13
    xs, zs, ph = H.partial2_stream(0, 0.8, 1, 9, 3)
    q = H.qdrift_stream(0.8, 18, 3)
    assert np.array_equal(xs, q[0]) and np.array_equal(ph, q[2])


def test_lexicographic_sort_matches_oracle_order():
    n = 7
    x, z, h, H = _ham(n, 40, 23)
    H.sort_lexicographic()
    xs, zs, ph = H.trotter_stream(1.0, 1)
    order = oracle.lexicographic_order(n, x, z)
    assert np.array_equal(xs, x[order]) and np.array_equal(zs, z[order]) and np.array_equal(ph, h[order])


def test_split_optimizer_matches_enumeration_with_the_oracle_bound():
    from oracle import learned as OL
    n = 6
    x, z, h, H = _ham(n, 18, 27)
    lam = float(np.abs(h).sum())
    order = OL.split_order(h)
    for eps, a, b in ((1e-3, 1.0, 1.0), (1e-2, 5.0, 0.1), (1e-3, 0.01, 10.0)):
        costs = []
        for L_D in range(0, len(h) + 1):
            C = OL.trotter_bound(n, x, z, h, L_D)
            lam_r = sum(abs(float(h[k])) for k in order[L_D:])
            delta = math.sqrt(eps / C) if C > 0 else math.inf
            cd = 0.0 if (L_D == 0 or math.isinf(delta)) else a * L_D / (eps * delta)
            costs.append(cd + b * lam_r ** 2 / eps ** 2)
        want = int(np.argmin(costs))
        L_D, delta, cost = ps.ps_partial_optimize_split(H.handle, eps, a, b)
        assert L_D == want and cost == pytest.approx(costs[want], rel=1e-12)
    # all-randomised when the deterministic part is expensive, all-deterministic when sampling is
    assert ps.ps_partial_optimize_split(H.handle, 1e-3, 1e6, 1e-6)[0] == 0
    assert ps.ps_partial_optimize_split(H.handle, 1e-3, 1e-6, 1e6)[0] == len(h)
    assert lam > 0



def test_learned_labels_margin_and_bound_steps_match_the_oracle():
    """The arithmetic of the learned step choice sits behind the C ABI:
    Richardson limit, error labels, pick margin and the bound's step count
    against the oracle's versions."""
    from oracle import learned as OL
    rng = np.random.default_rng(90)
    for _ in range(20):
        g = rng.normal(size=3) + 1j * rng.normal(size=3)
        assert abs(ps.ps_richardson3(*g) - OL.richardson3(*g)) < 1e-13 * (1 + np.max(np.abs(g)))
    g = rng.normal(size=9) + 1j * rng.normal(size=9)
    g[4] = 0.3 + 0.1j
    eps, lg = _lib.ps_trotter_error_labels(g, 0.3 + 0.1j, 1e-12)
    eps_o, lg_o = OL.error_labels(g, 0.3 + 0.1j, 1e-12)
    assert np.allclose(eps, eps_o, rtol=1e-15, atol=0) and eps[4] == 0.0
    assert lg.dtype == np.float32 and np.array_equal(lg, lg_o.astype(np.float32))
    for n_rows, q in ((1, 0.8), (7, 0.8), (200, 0.8), (200, 0.5), (201, 0.05), (50, 1.0), (50, 0.0)):
        y = rng.normal(size=n_rows).astype(np.float32)
        pr = rng.normal(size=n_rows).astype(np.float32)
        assert abs(_lib.ps_mlp_margin(y, pr, q) - OL.margin(y, pr, q)) < 1e-12
    with pytest.raises(ps.PsError):
        _lib.ps_mlp_margin(np.zeros(0, np.float32), np.zeros(0, np.float32), 0.8)
    n = 9
    x, z, h = inputs.jw_hamiltonian(n, 60, seed=91)
    H = ps.Hamiltonian(n, x, z, h)
    for t, e in ((0.1, 1e-3), (1.0, 1e-3), (2.5, 1e-2), (1e-6, 10.0)):
        assert _lib.ps_ham_bound_steps(H.handle, t, e) == OL.bound_steps(n, x, z, h, t, e)
    with pytest.raises(ps.PsError):
        _lib.ps_ham_bound_steps(H.handle, 0.0, 1e-3)


def test_shard_moves_reject_bad_arguments_before_any_device_work():
    """ps_shard_pack / ps_shard_unpack validate dtype, slab size, the swapped
    positions and the packed range on the host; none of these calls touches
    the (fake, never dereferenced) pointers."""
    fake_a, fake_b = 1 << 20, 2 << 20
    bad = [
        (10, 7, 0b11, 0, 16),            # dtype
        (0, ps.PS_C64, 0b1, 0, 1),        # s
        (10, ps.PS_C64, 0, 0, 16),        # no swapped position
        (10, ps.PS_C64, 1 << 10, 0, 16),  # a position at or above s
        (10, ps.PS_C64, 0b11, 1000, 100), # range past 2^s
    ]
    for s, dt, lmask, first, count in bad:
        with pytest.raises(ps.PsError):
            _lib.ps_shard_pack(s, dt, lmask, first, count, fake_a, fake_b, None)
        with pytest.raises(ps.PsError):
            _lib.ps_shard_unpack(s, dt, lmask, first, count, fake_a, fake_b, None)
    with pytest.raises(ps.PsError):  # source and destination must differ
        _lib.ps_shard_pack(10, ps.PS_C64, 0b11, 0, 16, fake_a, fake_a, None)
    with pytest.raises(ps.PsError):
        _lib.ps_measure_fma_rate(5)
