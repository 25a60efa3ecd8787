"""GPU parity: libps kernels (through the C ABI) against the CPU oracle.

Tolerances (relative L2 error of amplitudes, relative error of overlaps,
absolute when |g| < 1e-3):
  * complex128 path: 1e-12 (both sides are FP64; they differ only in
    summation order and in the gather vs scatter form of one rotation);
  * complex64 path: 1e-5 for up to a few hundred rotations.  Each rotation
    rounds every amplitude a few times at 2^-24 ~ 6e-8 relative, so after m
    rotations the error grows like sqrt(m) * 1e-7 (3e-6 at m = 1000); longer
    runs are checked against a bound derived the same way.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {ps.PS_C128: 1e-12, ps.PS_C64: 1e-5}
TDT = {ps.PS_C128: torch.complex128, ps.PS_C64: torch.complex64}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rel_scalar(a, b):
    return abs(a - b) / max(abs(b), 1e-3)


def gpu_state(n, dtype, host):
    st = ps.StateVector(n, dtype=TDT[dtype])
    st.load(host)
    return st


def represented(st):
    """The state a handle represents: its stored scale times the stored amplitudes
    (ps_get_state_represented)."""
    return st.to_numpy()


def run_rotations(n, dtype, psi0, x, z, phi, tuning=None):
    st = gpu_state(n, dtype, psi0)
    if tuning:
        st.set_tuning(**tuning)
    st.apply_rotations(x, z, phi)
    out = represented(st)
    ref0 = gpu_state(n, dtype, psi0)
    g = st.overlap(ref0)
    nrm = st.norm2()
    return out, g, nrm


# ------------------------------------------- n = 12, 64 random rotations

TUNINGS = [
    None,
    {"tile_bits": 6},
    {"tile_bits": 8, "group_bits": 1},
    {"tile_bits": 9, "group_bits": 2, "max_window": 5},
    {"tile_bits": 10, "group_bits": 4},
    {"max_window": 1},                      # one rotation per pass: pair kernel
    {"max_window": 1, "pair_single": 2},    # one rotation per pass: tile kernel
    {"tile_bits": 12, "max_window": 64},    # the whole state is one tile
    {"reg_groups": 1, "group_bits": 3},
    {"reg_groups": 2, "group_bits": 4},
    {"reg_groups": 4, "group_bits": 2, "tile_bits": 11},
    {"group_bits": 5, "tile_bits": 9, "max_window": 7},
    {"seg_bits": 1, "tile_bits": 10},       # 2-amplitude segments
    {"seg_bits": 2, "group_bits": 4, "reg_groups": 1, "tile_bits": 11},
    {"seg_bits": 3, "tile_bits": 9},
]


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
@pytest.mark.parametrize("tuning", TUNINGS)
def test_random_rotations_n12_all_amplitudes(dtype, tuning):
    if dtype == ps.PS_C128 and tuning and tuning.get("group_bits") == 5:
        tuning = dict(tuning, group_bits=4)  # complex128 register groups stop at 16 amplitudes
    n = 12
    psi0 = inputs.gaussian_state(n, 0)
    x, z, phi = inputs.random_rotations(n, 64, seed=1)
    ref = oracle.apply(psi0, x, z, phi)
    out, g, nrm = run_rotations(n, dtype, psi0, x, z, phi, tuning)
    assert rel(out, ref) < TOL[dtype]
    assert rel_scalar(g, oracle.overlap(psi0, ref)) < TOL[dtype]
    assert abs(nrm - 1.0) < (1e-13 if dtype == ps.PS_C128 else 1e-5)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9, 14, 17])
def test_small_and_ragged_sizes(dtype, n):
    psi0 = inputs.gaussian_state(n, n)
    x, z, phi = inputs.random_rotations(n, 37, seed=100 + n)
    ref = oracle.apply(psi0, x, z, phi)
    for tuning in (None, {"tile_bits": 6, "max_window": 3}, {"max_window": 1}):
        out, _, _ = run_rotations(n, dtype, psi0, x, z, phi, tuning)
        assert rel(out, ref) < TOL[dtype], (n, tuning)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_edge_rotations(dtype):
    n = 16
    psi0 = inputs.gaussian_state(n, 3)
    top = 1 << (n - 1)
    x = np.array([0, 1, 1, top, top | 1, 0, (1 << n) - 1, 3, 0, top], np.uint64)
    z = np.array([0, 0, 1, 0, top, (1 << n) - 1, (1 << n) - 1, 2, 5, top | 1], np.uint64)
    phi = np.array([0.3, -1.1, 2.0, 0.7, math.pi / 2, -0.2, 1e-9, -math.pi, 0.0, 3.0])
    ref = oracle.apply(psi0, x, z, phi)
    for tuning in (None, {"max_window": 1}, {"max_window": 1, "pair_single": 2}, {"tile_bits": 7}):
        out, _, _ = run_rotations(n, dtype, psi0, x, z, phi, tuning)
        assert rel(out, ref) < TOL[dtype], tuning


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_empty_sequence_is_a_no_op(dtype):
    n = 10
    psi0 = inputs.gaussian_state(n, 4)
    st = gpu_state(n, dtype, psi0)
    before = st.to_numpy()
    st.apply_rotations([], [], [])
    assert np.array_equal(st.to_numpy(), before)


def test_invalid_mask_touches_nothing():
    n = 10
    psi0 = inputs.gaussian_state(n, 5)
    st = gpu_state(n, ps.PS_C128, psi0)
    with pytest.raises(ps.PsError):
        st.apply_rotations([1, 1 << n], [0, 0], [0.1, 0.2])
    assert np.array_equal(st.to_numpy(), psi0)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_fused_equals_rotation_by_rotation(dtype):
    """Eq. 1 in single-GPU form: a fused window equals one pass per rotation.

    The two differ only in where the cos(phi) factors are rounded (once per
    window vs once per rotation), so they agree to a few ulps per rotation;
    the pair kernel and the tile kernel on single-rotation windows run the
    same arithmetic and agree bit for bit."""
    n = 20
    xh, zh, hh = inputs.jw_hamiltonian(n, 500, seed=7)
    H = ps.Hamiltonian(n, xh, zh, hh)
    x, z, phi = oracle.qdrift_stream(xh, zh, hh, 1.0, 400, 8)
    psi0 = inputs.gaussian_state(n, 6)
    fused, _, _ = run_rotations(n, dtype, psi0, x, z, phi)
    unfused, _, _ = run_rotations(n, dtype, psi0, x, z, phi, {"max_window": 1})
    tile_only, _, _ = run_rotations(n, dtype, psi0, x, z, phi, {"max_window": 1, "pair_single": 2})
    assert rel(fused, unfused) < (1e-14 if dtype == ps.PS_C128 else 2e-6)
    assert np.array_equal(unfused, tile_only)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
@pytest.mark.parametrize("tuning", [{"seg_bits": 3}, {"seg_bits": 2, "group_bits": 4, "reg_groups": 1},
                                    {"seg_bits": 3, "group_bits": 4, "reg_groups": 1},
                                    {"group_bits": 5, "reg_groups": 1}, {"seg_bits": 1, "group_bits": 2}, {"seg_bits": 6}])
def test_segment_sizes_and_group_shapes_vs_oracle(dtype, tuning):
    """JW qDRIFT (small angles, even Y counts): windows of the wider span that
    a smaller seg_bits allows, and register rounds of G = 2, 4 and 5 (most of
    them standard rounds), against the oracle."""
    n = 18
    xh, zh, hh = inputs.jw_hamiltonian(n, 400, seed=17)
    H = ps.Hamiltonian(n, xh, zh, hh)
    x, z, phi = oracle.qdrift_stream(xh, zh, hh, 1.0, 500, 18)
    psi0 = inputs.gaussian_state(n, 19)
    ref = oracle.apply(psi0, x, z, phi)
    if dtype == ps.PS_C128 and tuning.get("group_bits") == 5:
        tuning = dict(tuning, group_bits=4)
    out, g, _ = run_rotations(n, dtype, psi0, x, z, phi, tuning)
    assert rel(out, ref) < TOL[dtype]
    assert rel_scalar(g, oracle.overlap(psi0, ref)) < TOL[dtype]


_REF22 = {}


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
@pytest.mark.parametrize("tuning", [{"tile_threads": 64}, {"tile_threads": 128}, {"tile_threads": 128, "reg_groups": 1},
                                    {"tile_threads": 128, "reg_groups": 4}, {"tile_threads": 64, "reg_groups": 4},
                                    {"tile_threads": 256, "reg_groups": 2}])
def test_tile_threads_give_the_same_amplitudes(dtype, tuning):
    """Fewer threads per tile (more register batches per thread) and other
    group counts change only which thread updates which amplitude, never the
    arithmetic: bitwise equal to the default launch, and within tolerance of
    the oracle.  n = 22 gives 2^9 or 2^10 tiles."""
    n = 22
    xh, zh, hh = inputs.jw_hamiltonian(n, 300, seed=23)
    H = ps.Hamiltonian(n, xh, zh, hh)
    x, z, phi = oracle.qdrift_stream(xh, zh, hh, 1.0, 160, 24)
    psi0 = inputs.gaussian_state(n, 25)
    if dtype == ps.PS_C128:
        tuning = dict(tuning, reg_groups=min(tuning.get("reg_groups", 1), 2))
    out, g, _ = run_rotations(n, dtype, psi0, x, z, phi, tuning)
    base, g0, _ = run_rotations(n, dtype, psi0, x, z, phi)
    assert np.array_equal(out, base)
    assert g == g0
    if n not in _REF22:
        _REF22[n] = oracle.apply(psi0, x, z, phi)
    assert rel(out, _REF22[n]) < TOL[dtype]


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_large_angles_use_full_form(dtype):
    """|tan(phi)| > 1 takes the cos/sin form; windows mixing both forms stay exact."""
    n = 14
    x, z, _ = inputs.random_rotations(n, 60, seed=31)
    rng = np.random.default_rng(32)
    phi = np.where(rng.random(60) < 0.5, rng.uniform(-0.6, 0.6, 60), rng.uniform(0.9, 2.3, 60) * rng.choice([-1, 1], 60))
    psi0 = inputs.gaussian_state(n, 33)
    ref = oracle.apply(psi0, x, z, phi)
    for tuning in (None, {"max_window": 1}, {"tile_bits": 8}):
        out, _, nrm = run_rotations(n, dtype, psi0, x, z, phi, tuning)
        assert rel(out, ref) < TOL[dtype]
        assert abs(nrm - 1) < (1e-13 if dtype == ps.PS_C128 else 1e-5)


def test_complex64_norm_does_not_drift_over_long_small_angle_runs():
    """10^5 qDRIFT-sized angles (|phi| ~ 1e-4): cos(phi) rounds to 1 in FP32,
    which would grow the norm by sin^2(phi) per rotation (~1e-3 in total)
    unless the cos factors are carried in FP64 as the stored scale."""
    n = 14
    xh, zh, hh = inputs.jw_hamiltonian(n, 500, seed=9)
    H = ps.Hamiltonian(n, xh, zh, hh)
    N = 100_000
    x, z, phi = oracle.qdrift_stream(xh, zh, hh, 10.0, N, 10)
    assert np.max(np.abs(phi)) > 1e-4
    psi0 = inputs.gaussian_state(n, 11)
    s64 = gpu_state(n, ps.PS_C64, psi0)
    s128 = gpu_state(n, ps.PS_C128, psi0)
    s64.apply_rotations(x, z, phi)
    s128.apply_rotations(x, z, phi)
    # FP64: every rotation has the same |angle|, so the rounding of tan(phi) and
    # cos(phi) biases the norm the same way each time, up to 4 * 2^-53 per
    # rotation (4e-18 here), plus one rounding per carried-factor update
    assert abs(s128.norm2() - 1.0) < N * 4 * 2.0 ** -53
    assert abs(s64.norm2() - 1.0) < 2e-5
    # random-walk rounding error only: sqrt(N) * ~1e-7
    assert rel(represented(s64), represented(s128)) < 1e-4


def test_represented_state_applies_the_carried_scale():
    """ps_get_state_represented returns f * stored in FP64 (complex128), f the
    carried scale: after 2*10^4 small-angle complex64 rotations f differs
    from 1 by more than the complex64 tolerance allows to ignore."""
    n = 12
    xh, zh, hh = inputs.jw_hamiltonian(n, 200, seed=41)
    H = ps.Hamiltonian(n, xh, zh, hh)
    x, z, phi = oracle.qdrift_stream(xh, zh, hh, 20.0, 20_000, 42)
    psi0 = inputs.gaussian_state(n, 43)
    st = gpu_state(n, ps.PS_C64, psi0)
    st.apply_rotations(x[:19_999], z[:19_999], phi[:19_999])
    f = st.scale()
    stored = st.stored_numpy()
    assert stored.dtype == np.complex64
    rep = st.to_numpy()
    assert rep.dtype == np.complex128
    want = np.empty_like(rep)
    want.real = f * stored.real.astype(np.float64)
    want.imag = f * stored.imag.astype(np.float64)
    assert np.array_equal(rep, want)
    ref = oracle.apply(psi0, x[:19_999], z[:19_999], phi[:19_999])
    assert rel(rep, ref) < 1e-4
    if abs(f - 1.0) > 1e-6:
        assert rel(rep, ref) < rel(stored.astype(np.complex128), ref)


def test_complex128_carried_scale_stays_within_its_band():
    """complex128 applies the carried cos(phi) factor only once it leaves
    |f - 1| <= 2^-20: in between the stored amplitudes are the state divided by
    f, and every readout (represented state, norm, overlap) includes it."""
    n = 11
    xh, zh, hh = inputs.jw_hamiltonian(n, 150, seed=44)
    x, z, phi = oracle.qdrift_stream(xh, zh, hh, 0.3, 3000, 45)  # |phi| ~ 1e-4: the factor builds up over many passes
    psi0 = inputs.gaussian_state(n, 46)
    st = gpu_state(n, ps.PS_C128, psi0)
    seen = set()
    for lo in range(0, 3000, 300):
        st.apply_rotations(x[lo:lo + 300], z[lo:lo + 300], phi[lo:lo + 300])
        f = st.scale()
        assert abs(f - 1.0) <= 2.0 ** -20
        seen.add(f != 1.0)
    assert True in seen  # the factor was carried at least once
    ref = oracle.apply(psi0, x, z, phi)
    assert rel(st.to_numpy(), ref) < 1e-12
    assert abs(st.norm2() - 1.0) < 1e-12
    assert rel_scalar(st.overlap(gpu_state(n, ps.PS_C128, psi0)), oracle.overlap(psi0, ref)) < 1e-12


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_plan_apply_equals_apply_rotations(dtype):
    n = 18
    x, z, phi = inputs.random_rotations(n, 120, seed=9)
    psi0 = inputs.gaussian_state(n, 10)
    a, _, _ = run_rotations(n, dtype, psi0, x, z, phi)
    st = gpu_state(n, dtype, psi0)
    plan = ps.Plan(n, dtype, x, z, phi)
    st.apply_plan(plan)
    assert np.array_equal(represented(st), a)
    assert plan.info["rotations"] == 120


# --------------------------------------------------- reductions

@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
@pytest.mark.parametrize("n", [1, 4, 11, 19, 22])
def test_overlap_and_norm(dtype, n):
    a = inputs.gaussian_state(n, 20 + n)
    b = inputs.gaussian_state(n, 40 + n)
    if dtype == ps.PS_C64:
        a = a.astype(np.complex64).astype(np.complex128)
        b = b.astype(np.complex64).astype(np.complex128)
    sa, sb = gpu_state(n, dtype, a), gpu_state(n, dtype, b)
    g = sb.overlap(sa)
    ref = oracle.overlap(a, b)
    assert abs(g - ref) < 1e-14 * math.sqrt(1 << n) + 1e-15
    assert abs(sa.norm2() - oracle.norm2(a)) < 1e-13
    # bitwise reproducible on one device
    assert sb.overlap(sa) == g


# ---------------------------------------- product formulas vs the oracle

@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_trotter_vs_oracle(dtype):
    n = 12
    x, z, h = inputs.jw_hamiltonian(n, 150, seed=2)
    psi0 = inputs.gaussian_state(n, 3)
    H = ps.Hamiltonian(n, x, z, h)
    for t, r in ((0.1, 1), (0.8, 3)):
        st = gpu_state(n, dtype, psi0)
        st.evolve_trotter(H, t, r)
        ref = oracle.trotter(psi0, x, z, h, t, r)
        assert rel(represented(st), ref) < TOL[dtype] * (1 if dtype == ps.PS_C128 else 3)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_qdrift_vs_oracle(dtype):
    n = 13
    x, z, h = inputs.jw_hamiltonian(n, 400, seed=4)
    psi0 = inputs.gaussian_state(n, 5)
    H = ps.Hamiltonian(n, x, z, h)
    st = gpu_state(n, dtype, psi0)
    st.evolve_qdrift(H, 1.0, 300, 77)
    ref = oracle.qdrift(psi0, x, z, h, 1.0, 300, 77)
    assert rel(represented(st), ref) < TOL[dtype]
    g = st.overlap(gpu_state(n, dtype, psi0))
    assert rel_scalar(g, oracle.overlap(psi0, ref)) < TOL[dtype]


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_partial_vs_oracle(dtype):
    n = 12
    x, z, h = inputs.jw_hamiltonian(n, 300, seed=6)
    psi0 = inputs.gaussian_state(n, 7)
    H = ps.Hamiltonian(n, x, z, h)
    st = gpu_state(n, dtype, psi0)
    st.evolve_partial(H, 30, 0.6, 2, 40, 13)
    ref = oracle.partial(psi0, x, z, h, 30, 0.6, 2, 40, 13)
    assert rel(represented(st), ref) < TOL[dtype]


def test_trotter_exact_for_commuting_terms_on_gpu():
    n = 14
    rng = np.random.default_rng(8)
    z = rng.integers(1, 1 << n, 40).astype(np.uint64)
    x = np.zeros_like(z)
    h = rng.normal(size=40)
    psi0 = inputs.gaussian_state(n, 9)
    H = ps.Hamiltonian(n, x, z, h)
    k = np.arange(1 << n, dtype=np.uint64)
    energy = np.zeros(1 << n)
    for zl, hl in zip(z, h):
        par = np.array([bin(int(v)).count("1") & 1 for v in (k & zl)])
        energy += hl * (1 - 2 * par)
    exact = np.exp(1j * 0.9 * energy) * psi0
    for r in (1, 4):
        st = gpu_state(n, ps.PS_C128, psi0)
        st.evolve_trotter(H, 0.9, r)
        assert rel(represented(st), exact) < 1e-12


# ------------------------- full size, launch configuration of the benchmark

N30 = 30
L30 = 10_000


@pytest.fixture(scope="module")
def ham30():
    x, z, h = inputs.jw_hamiltonian(N30, L30, seed=3)
    return x, z, h, ps.Hamiltonian(N30, x, z, h)


def test_n30_forward_then_inverse_returns_initial_state(ham30):
    """P^2 = I makes the reversed sequence with negated angles the exact inverse."""
    xh, zh, hh, _ = ham30
    xs, zs, ph = oracle.qdrift_stream(xh, zh, hh, 1.0, 100_000, 4, first=0, count=3000)
    idx, amp = inputs.determinant_state(N30, seed=11)
    st = ps.StateVector(N30, dtype=torch.complex64)
    st.tensor.zero_()
    st.tensor[torch.as_tensor(idx.astype(np.int64), device="cuda")] = torch.as_tensor(amp, device="cuda").to(
        torch.complex64)
    st.apply_rotations(xs, zs, ph)
    mid_norm = st.norm2()
    st.apply_rotations(xs[::-1].copy(), zs[::-1].copy(), -ph[::-1])
    back = st.tensor[torch.as_tensor(idx.astype(np.int64), device="cuda")].cpu().numpy() * st.scale()
    # FP32: 6000 rotations, sqrt(6000) * ~1e-7 ~ 1e-5
    assert np.max(np.abs(back - amp)) < 5e-5
    assert abs(mid_norm - 1.0) < 5e-5
    del st
    torch.cuda.empty_cache()


def test_stats_count_launches_and_bytes():
    n = 16
    x, z, phi = inputs.random_rotations(n, 50, seed=13)
    st = gpu_state(n, ps.PS_C64, inputs.gaussian_state(n, 14))
    st.set_tuning(kernel_timing=1)
    ps.ps_reset_stats(st.handle)
    st.apply_rotations(x, z, phi)
    info = ps.ps_plan_describe(n, ps.PS_C64, x, z, phi)
    s = st.stats()
    assert s["rotations"] == 50 and s["passes"] == info["windows"]
    assert s["launches"]["tile"] + s["launches"]["pair"] == info["windows"]
    assert s["kernel_ms"]["tile"] + s["kernel_ms"]["pair"] > 0
    assert s["bytes"]["tile"] + s["bytes"]["pair"] == 2 * 8 * (1 << n) * info["windows"]


# ------------------------------------------------------------ second order

@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_trotter2_vs_oracle(dtype):
    n = 11
    x, z, h = inputs.jw_hamiltonian(n, 200, seed=14)
    psi0 = inputs.gaussian_state(n, 15)
    H = ps.Hamiltonian(n, x, z, h)
    st = gpu_state(n, dtype, psi0)
    st.evolve_trotter2(H, 0.9, 3)
    ref = oracle.trotter2(psi0, x, z, h, 0.9, 3)
    assert rel(represented(st), ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_partial2_vs_oracle(dtype):
    n = 12
    x, z, h = inputs.jw_hamiltonian(n, 300, seed=16)
    psi0 = inputs.gaussian_state(n, 17)
    H = ps.Hamiltonian(n, x, z, h)
    st = gpu_state(n, dtype, psi0)
    st.evolve_partial2(H, 30, 0.6, 2, 40, 13)
    ref = oracle.partial2(psi0, x, z, h, 30, 0.6, 2, 40, 13)
    assert rel(represented(st), ref) < TOL[dtype]


def test_lexicographic_order_gives_the_same_commuting_limit_and_changes_only_the_error():
    # reordering terms changes the product formula, not the limit: both orders
    # approach exp(itH) psi, and the sorted order's stream fuses at least as well
    n = 10
    x, z, h = inputs.jw_hamiltonian(n, 120, seed=18)
    psi0 = inputs.gaussian_state(n, 19)
    H = ps.Hamiltonian(n, x, z, h)
    Hs = ps.Hamiltonian(n, x, z, h)
    Hs.sort_lexicographic()
    a = gpu_state(n, ps.PS_C128, psi0)
    b = gpu_state(n, ps.PS_C128, psi0)
    a.evolve_trotter2(H, 0.5, 64)
    b.evolve_trotter2(Hs, 0.5, 64)
    assert rel(represented(a), represented(b)) < 1e-4
    order = oracle.lexicographic_order(n, x, z)
    ref = oracle.trotter2(psi0, x[order], z[order], h[order], 0.5, 2)
    c = gpu_state(n, ps.PS_C128, psi0)
    c.evolve_trotter2(Hs, 0.5, 2)
    assert rel(represented(c), ref) < 1e-12


@pytest.mark.parametrize("order,L_D,Ns", [(1, 40, 0), (2, 40, 0), (1, 6, 5), (2, 6, 3)])
def test_rpe_signal_reuses_state_and_matches_separate_runs(order, L_D, Ns):
    # Z_m = g(delta 2^m) from one continued state equals 2^m steps run from psi0
    n = 9
    x, z, h = inputs.jw_hamiltonian(n, 40, seed=28)
    psi0 = inputs.gaussian_state(n, 29)
    H = ps.Hamiltonian(n, x, z, h)
    p0 = gpu_state(n, ps.PS_C128, psi0)
    work = gpu_state(n, ps.PS_C128, psi0)
    delta, M, seed = 0.07, 5, 31
    Z = ps.ps_rpe_signal(work.handle, p0.handle, H.handle, order, L_D, delta, M, Ns, seed)
    for m in range(M + 1):
        steps = 1 << m
        t = delta * steps
        if order == 1:
            ref = oracle.partial(psi0, x, z, h, L_D, t, steps, Ns, seed)
        else:
            ref = oracle.partial2(psi0, x, z, h, L_D, t, steps, Ns, seed)
        g = np.vdot(psi0, ref)
        assert abs(Z[m] - g) < 1e-12, (m, Z[m], g)


@pytest.mark.parametrize("dtype,tol", [(ps.PS_C128, 1e-11), (ps.PS_C64, 1e-4)])
def test_rpe_signal_and_estimate_recover_the_trotter_eigenphase(dtype, tol):
    """The RPE chain on the GPU: the signal of a state mostly along one
    eigenvector of the first-order step U(delta) (n = 5, dense U from the
    oracle), then ps_rpe_estimate, gives that eigenvector's phase."""
    from oracle import rpe as OR
    n, delta, M = 5, 0.15, 8
    x, z, h = inputs.jw_hamiltonian(n, 16, seed=33, lam=3.0)
    dim = 1 << n
    U = np.zeros((dim, dim), dtype=np.complex128)
    for k in range(dim):
        e = np.zeros(dim, dtype=np.complex128)
        e[k] = 1.0
        U[:, k] = oracle.trotter(e, x, z, h, delta, 1)
    _, vecs = np.linalg.eigh((U + U.conj().T) / 2 + 0.37 * (U - U.conj().T) / 2j)
    v0 = vecs[:, 0]
    theta0 = np.angle(v0.conj() @ U @ v0)
    w = np.random.default_rng(34).normal(size=dim) + 0j
    w -= (v0.conj() @ w) * v0
    w /= np.linalg.norm(w)
    psi0 = np.sqrt(0.85) * v0 + np.sqrt(0.15) * w
    H = ps.Hamiltonian(n, x, z, h)
    p0 = gpu_state(n, dtype, psi0)
    work = gpu_state(n, dtype, psi0)
    Z = ps.ps_rpe_signal(work.handle, p0.handle, H.handle, 1, H.L, delta, M)
    Z_ref = OR.signal(psi0, x, z, h, delta, M)
    assert np.max(np.abs(Z - Z_ref)) < tol
    E, _ = ps.ps_rpe_estimate(Z, delta)
    assert abs(E * delta - theta0) <= np.arcsin(0.15 / 0.85) / 2.0 ** M + 1e-9

