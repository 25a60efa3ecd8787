"""GPU parity at full size, in the launch configuration of the benchmark.

* n = 28: the whole 2^28-amplitude state (4 GiB complex128) after the first
  1000 rotations of the benchmark's qDRIFT generator (10^4 JW-like terms,
  N = 10^5 samples at t = 1, seed 4), starting from a dense Gaussian state,
  compared element by element with the oracle run on all host cores.
* n = 30: the longest prefix of the benchmark stream whose single
  amplitudes the oracle evaluates exactly (26 rotations, all with X masks),
  256 amplitudes compared one by one, relative to each amplitude.
* n = 32 and n = 33 (complex64 and complex128): the amplitude index no
  longer fits 32 bits; 20 rotations whose X masks reach the top qubits.

Tolerances (each amplitude k):
  complex128  |got_k - ref_k| <= 1e-12 max(|ref_k|, floor), relative L2 <= 1e-12;
  complex64   |got_k - ref_k| <= 4 sqrt(m) 1e-7 max(|ref_k|, floor) after m
              rotations, relative L2 <= sqrt(m) 1e-7 (the growth of FP32
              rounding, 2^-24 relative per update, over m rotations).
The floor is 1% of the RMS amplitude for the dense n = 28 state (an
amplitude near zero still carries the absolute rounding of its neighbours'
contributions).  A sampled amplitude is reached from one determinant by
flipping s of the rotations' X masks; its floor is the size of that one path,
|amp_det| max|sin phi|^s.  Where two rotations share an X mask (the same
hopping term drawn twice, or XX and YY on the same qubits) two paths reach
the same state and can cancel almost exactly, and the rounding then scales
with the paths, not with their difference.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs

pytestmark = pytest.mark.gpu

TDT = {ps.PS_C128: torch.complex128, ps.PS_C64: torch.complex64}
N_TERMS = 10_000
HAM_SEED = 3
QDRIFT_SEED = 4
N_SAMPLES = 100_000
T_TOTAL = 1.0


def per_element_ok(got, ref, rel_tol, floor):
    err = np.abs(got - ref)
    bound = rel_tol * np.maximum(np.abs(ref), floor)
    worst = int(np.argmax(err / bound))
    return bool(np.all(err <= bound)), float(err[worst]), float(np.abs(ref[worst]))


def sparse_state_on_gpu(n, dtype, idx, amp):
    st = ps.StateVector(n, dtype=TDT[dtype])
    st.tensor.zero_()
    st.tensor[torch.as_tensor(idx.astype(np.int64), device="cuda")] = torch.as_tensor(amp, device="cuda").to(
        st.tensor.dtype)
    return st


def gather(st, ks):
    """Amplitudes ks of the represented state (stored x carried scale, FP64)."""
    got = st.tensor[torch.as_tensor(ks.astype(np.int64), device="cuda")].cpu().numpy().astype(np.complex128)
    return got * st.scale()


def few_flip_indices(rng, idx, amp, xs, ph, count, max_flips):
    """Basis states reached from a determinant by flipping 0..max_flips of the
    rotations' X masks, and the size of that path, |amp_det| max|sin phi|^s
    (far above the FP32 underflow for the flips allowed)."""
    ks, scale = [], []
    smax = float(np.max(np.abs(np.sin(ph))))
    for i in range(count):
        d = int(rng.integers(len(idx)))
        k = int(idx[d])
        s = i % (max_flips + 1)
        for j in rng.choice(len(xs), size=s, replace=False):
            k ^= int(xs[j])
        ks.append(k)
        scale.append(abs(amp[d]) * smax ** s)
    return np.array(ks, dtype=np.uint64), np.array(scale)


# ------------------------------------------------ n = 28, the whole state

N28 = 28
ROT28 = 1000


@pytest.fixture(scope="module")
def n28_case():
    x, z, h = inputs.jw_hamiltonian(N28, N_TERMS, seed=HAM_SEED)
    xs, zs, ph = oracle.qdrift_stream(x, z, h, T_TOTAL, N_SAMPLES, QDRIFT_SEED, first=0, count=ROT28)
    psi0 = inputs.gaussian_state(N28, 28)
    ref = psi0.copy()
    tmp = np.empty_like(ref)
    used = oracle.set_threads(os.cpu_count() or 1)
    try:
        oracle.apply_inplace(ref, tmp, xs, zs, ph)
    finally:
        oracle.set_threads(1)
    del tmp
    return dict(psi0=psi0, xs=xs, zs=zs, ph=ph, ref=ref, threads=used)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_n28_full_state_1000_qdrift_rotations_vs_oracle(n28_case, dtype):
    c = n28_case
    st = ps.StateVector(N28, dtype=TDT[dtype])
    st.load(c["psi0"])
    st0 = ps.StateVector(N28, dtype=TDT[dtype])
    st0.load(c["psi0"])
    st.apply_rotations(c["xs"], c["zs"], c["ph"])
    g = st.overlap(st0)
    del st0
    got = st.to_numpy()
    del st
    torch.cuda.empty_cache()
    ref = c["ref"]
    m = ROT28
    rms = np.linalg.norm(ref) / math.sqrt(ref.size)
    if dtype == ps.PS_C128:
        l2_tol, el_tol = 1e-12, 1e-12
    else:
        l2_tol, el_tol = math.sqrt(m) * 1e-7, 4 * math.sqrt(m) * 1e-7
    rel_l2 = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert rel_l2 < l2_tol, rel_l2
    ok, err, mag = per_element_ok(got, ref, el_tol, 0.01 * rms)
    assert ok, (err, mag, rms)
    g_ref = oracle.overlap(c["psi0"], ref)
    assert abs(g - g_ref) / abs(g_ref) < l2_tol


# --------------------------------- n = 30, 26-rotation prefix, 256 amplitudes

N30 = 30
PREFIX30 = 26  # the oracle's single-amplitude evaluation takes at most 26 rotations with X masks


@pytest.fixture(scope="module")
def n30_case():
    x, z, h = inputs.jw_hamiltonian(N30, N_TERMS, seed=HAM_SEED)
    xs, zs, ph = oracle.qdrift_stream(x, z, h, T_TOTAL, N_SAMPLES, QDRIFT_SEED, first=0, count=PREFIX30)
    assert np.all(xs != 0)
    idx, amp = inputs.determinant_state(N30, seed=11)
    return dict(xs=xs, zs=zs, ph=ph, idx=idx, amp=amp)


@pytest.mark.parametrize("dtype", [ps.PS_C64, ps.PS_C128])
def test_n30_sampled_amplitudes_vs_oracle(n30_case, dtype):
    """The first 26 rotations of the n = 30 benchmark stream on its
    8-determinant state; 256 amplitudes, each compared relative to itself.
    complex128 samples reach up to all 26 flips (amplitudes down to ~1e-107),
    complex64 samples up to 6 (~1e-25, inside the FP32 normal range)."""
    c = n30_case
    xs, zs, ph, idx, amp = c["xs"], c["zs"], c["ph"], c["idx"], c["amp"]
    st = sparse_state_on_gpu(N30, dtype, idx, amp)
    st.apply_rotations(xs, zs, ph)
    rng = np.random.default_rng(12 + dtype)
    ks, path = few_flip_indices(rng, idx, amp, xs, ph, 256, PREFIX30 if dtype == ps.PS_C128 else 6)
    oracle.set_threads(os.cpu_count() or 1)
    try:
        ref = oracle.amplitudes_sparse(N30, idx, amp, xs, zs, ph, ks)
    finally:
        oracle.set_threads(1)
    got = gather(st, ks)
    assert np.all(np.abs(ref) > 0)
    # most samples sit on a single path: there the bound is relative to the amplitude itself
    assert np.mean(np.abs(ref) > 0.5 * path) > 0.75
    tol = 1e-12 if dtype == ps.PS_C128 else 4 * math.sqrt(PREFIX30) * 1e-7
    ok, err, mag = per_element_ok(got, ref, tol, path)
    assert ok, (err, mag)
    assert abs(st.norm2() - 1.0) < (1e-12 if dtype == ps.PS_C128 else 1e-5)
    del st
    torch.cuda.empty_cache()


# -------------------------------------- n = 32, 33: 64-bit amplitude indices

@pytest.mark.parametrize("n", [32, 33])
@pytest.mark.parametrize("dtype", [ps.PS_C64, ps.PS_C128])
def test_64bit_indices_sampled_amplitudes_vs_oracle(n, dtype):
    """At n = 32 the tile kernel's 32-bit index path ends; at n = 33 only the
    64-bit path runs.  20 rotations of a JW-like qDRIFT stream (angles 10x the
    benchmark's, so that every flip moves amplitude visibly), at least five
    of them with an X bit on one of the top two qubits; 96 amplitudes."""
    x, z, h = inputs.jw_hamiltonian(n, 2000, seed=60 + n)
    xs, zs, ph = oracle.qdrift_stream(x, z, h, 10.0 * T_TOTAL, N_SAMPLES, 61 + n, first=0, count=400)
    top = (1 << (n - 1)) | (1 << (n - 2))
    hi = np.flatnonzero((xs & np.uint64(top)) != 0)[:5]
    lo = np.flatnonzero((xs & np.uint64(top)) == 0)[:15]
    sel = np.sort(np.concatenate([hi, lo]))
    assert len(hi) == 5 and len(sel) == 20
    xs, zs, ph = xs[sel].copy(), zs[sel].copy(), ph[sel].copy()
    idx, amp = inputs.determinant_state(n, seed=62 + n)
    st = sparse_state_on_gpu(n, dtype, idx, amp)
    st.apply_rotations(xs, zs, ph)
    rng = np.random.default_rng(63 + n)
    ks, path = few_flip_indices(rng, idx, amp, xs, ph, 96, 20 if dtype == ps.PS_C128 else 5)
    # amplitudes with the top qubits set are among the samples
    assert np.any(ks >> np.uint64(n - 2))
    oracle.set_threads(os.cpu_count() or 1)
    try:
        ref = oracle.amplitudes_sparse(n, idx, amp, xs, zs, ph, ks)
    finally:
        oracle.set_threads(1)
    got = gather(st, ks)
    tol = 1e-12 if dtype == ps.PS_C128 else 4 * math.sqrt(20) * 1e-7
    ok, err, mag = per_element_ok(got, ref, tol, path)
    assert ok, (err, mag)
    assert abs(st.norm2() - 1.0) < (1e-12 if dtype == ps.PS_C128 else 1e-5)
    del st
    torch.cuda.empty_cache()


# ---------------- the n = 26 Trotter sweep's structure, against the oracle

N_T = 24          # the largest n at which the oracle's 12,000 rotations take about a minute on 16 host cores
T_TERMS = 2000    # the sweep's Hamiltonian: 2000 JW-like terms, seed 2, one-norm 3.5
T_TIMES = (0.1, 0.1 * 2.0 ** 5)   # t_1 and t_16 of 0.1 * 2^(j/3)
T_STEPS = (1, 2)


@pytest.fixture(scope="module")
def trotter_case():
    x, z, h = inputs.jw_hamiltonian(N_T, T_TERMS, seed=2)
    idx, amp = inputs.determinant_state(N_T, seed=21)
    psi0 = np.zeros(1 << N_T, dtype=np.complex128)
    psi0[idx.astype(np.int64)] = amp
    ref = {}
    oracle.set_threads(os.cpu_count() or 1)
    try:
        for t in T_TIMES:
            for r in T_STEPS:
                ref[(t, r)] = oracle.trotter(psi0, x, z, h, t, r)
    finally:
        oracle.set_threads(1)
    return dict(x=x, z=z, h=h, idx=idx, amp=amp, psi0=psi0, ref=ref)


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_trotter_sweep_pairs_vs_oracle(trotter_case, dtype):
    """(r in {1, 2}) x (t_1, t_16) of the first-order Trotter sweep, n = 24:
    whole states and overlaps against the oracle's product formula (Eq. 3)."""
    c = trotter_case
    H = ps.Hamiltonian(N_T, c["x"], c["z"], c["h"])
    st0 = sparse_state_on_gpu(N_T, dtype, c["idx"], c["amp"])
    work = ps.StateVector(N_T, dtype=TDT[dtype])
    for (t, r), ref in c["ref"].items():
        work.copy_from(st0)
        work.evolve_trotter(H, t, r)
        g = work.overlap(st0)
        got = work.to_numpy()
        m = r * T_TERMS
        tol = 1e-12 if dtype == ps.PS_C128 else math.sqrt(m) * 1e-7
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, (t, r)
        g_ref = oracle.overlap(c["psi0"], ref)
        assert abs(g - g_ref) / max(abs(g_ref), 1e-3) < tol, (t, r, g, g_ref)
    del work, st0
    H.close()
    torch.cuda.empty_cache()
