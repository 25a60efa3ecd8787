"""Pins of the CPU oracle against facts it does not compute itself.

Each check below is chosen so that a plausible slip in the oracle -- a wrong
phase, a transposed bit order, a dropped term, a wrong sign of time, a
sampler that ignores a coefficient -- fails at least one of them:

* the paper's worked encoding example (golden file);
* dense Kronecker products of the 2x2 Pauli matrices and matrix exponentials
  from numpy's Hermitian eigendecomposition (a library routine);
* closed-form single-qubit evolutions;
* invariants: unitarity, P^2 = I, exactness of Trotter for commuting terms;
* the first-order Trotter convergence rate;
* published SplitMix64 outputs and the exact expectation of qDRIFT.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2504_17881_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

_PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def letters_of(n, x, z):
    out = []
    for q in range(n):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        out.append("Y" if xb and zb else "X" if xb else "Z" if zb else "I")
    return "".join(out)  # position q = qubit q+1 = bit q


def dense_pauli(n, x, z):
    """Kronecker product with qubit n (most significant bit) as the first factor."""
    s = letters_of(n, x, z)
    m = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        m = np.kron(m, _PAULI[s[q]])
    return m


def expm_herm(h, t):
    """exp(i t H) for Hermitian H via numpy's eigendecomposition."""
    w, v = np.linalg.eigh(h)
    return (v * np.exp(1j * t * w)) @ v.conj().T


def dense_ham(n, x, z, h):
    return sum(hl * dense_pauli(n, int(xl), int(zl)) for xl, zl, hl in zip(x, z, h))


# ---------------------------------------------------------------- encoding

def test_worked_encoding_example_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "pauli_encoding.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for s, p1, p2 in rows:
        assert oracle.pauli_from_string(s) == (int(p1), int(p2))


def test_encoding_rejects_unknown_letters():
    with pytest.raises(ValueError):
        oracle.pauli_from_string("XQZ")


def test_phase_matches_dense_matrix_all_strings_n3():
    n = 3
    for x in range(8):
        for z in range(8):
            p = dense_pauli(n, x, z)
            for k in range(8):
                col = p[:, k]
                nz = np.flatnonzero(np.abs(col) > 0.5)
                assert list(nz) == [k ^ x]
                assert abs(col[k ^ x] - oracle.pauli_phase(x, z, k)) < 1e-15


# ------------------------------------------------------------ one rotation

@pytest.mark.parametrize("n", [1, 2, 3])
def test_rotation_vs_expm_all_strings(n):
    rng = np.random.default_rng(10 + n)
    psi = inputs.gaussian_state(n, 11 + n)
    for x in range(1 << n):
        for z in range(1 << n):
            phi = rng.uniform(-math.pi, math.pi)
            ref = expm_herm(dense_pauli(n, x, z), phi) @ psi
            got = oracle.apply(psi, [x], [z], [phi])
            assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("n", [5, 8])
def test_rotation_sequence_vs_expm_random(n):
    x, z, phi = inputs.random_rotations(n, 12, seed=100 + n)
    psi = inputs.gaussian_state(n, 200 + n)
    ref = psi.copy()
    for xl, zl, pl in zip(x, z, phi):
        ref = expm_herm(dense_pauli(n, int(xl), int(zl)), pl) @ ref
    got = oracle.apply(psi, x, z, phi)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_single_qubit_closed_forms():
    phi = 0.37
    e0 = np.array([1, 0], complex)
    e1 = np.array([0, 1], complex)
    X, Y, Z = (oracle.pauli_from_string(s) for s in "XYZ")
    # <0| exp(i phi X) |0> = cos(phi), <1| ... |0> = i sin(phi)
    out = oracle.apply(e0, [X[0]], [X[1]], [phi])
    assert abs(out[0] - math.cos(phi)) < 1e-15 and abs(out[1] - 1j * math.sin(phi)) < 1e-15
    # exp(i phi Y)|0> = cos|0> - sin|1>,  exp(i phi Y)|1> = sin|0> + cos|1>
    out = oracle.apply(e0, [Y[0]], [Y[1]], [phi])
    assert np.allclose(out, [math.cos(phi), -math.sin(phi)], atol=1e-15)
    out = oracle.apply(e1, [Y[0]], [Y[1]], [phi])
    assert np.allclose(out, [math.sin(phi), math.cos(phi)], atol=1e-15)
    # Z: phases exp(+i phi) on |0>, exp(-i phi) on |1>
    out = oracle.apply(np.array([1, 1], complex) / math.sqrt(2), [Z[0]], [Z[1]], [phi])
    assert np.allclose(out * math.sqrt(2), [np.exp(1j * phi), np.exp(-1j * phi)], atol=1e-15)


def test_identity_string_is_global_phase():
    psi = inputs.gaussian_state(4, 3)
    out = oracle.apply(psi, [0], [0], [0.9])
    assert np.max(np.abs(out - np.exp(0.9j) * psi)) < 1e-15


def test_p_squared_is_identity_and_inverse():
    n = 6
    x, z, phi = inputs.random_rotations(n, 40, seed=5)
    psi = inputs.gaussian_state(n, 6)
    fwd = oracle.apply(psi, x, z, phi)
    back = oracle.apply(fwd, x[::-1], z[::-1], -phi[::-1])
    assert np.max(np.abs(back - psi)) < 1e-13
    # exp(i pi/2 P) = i P, so two of them give -I
    for xl, zl in zip(x[:8], z[:8]):
        twice = oracle.apply(psi, [xl, xl], [zl, zl], [math.pi / 2, math.pi / 2])
        assert np.max(np.abs(twice + psi)) < 1e-14


def test_norm_preserved_over_many_rotations():
    n = 8
    x, z, phi = inputs.random_rotations(n, 10_000, seed=7)
    psi = inputs.gaussian_state(n, 8)
    out = oracle.apply(psi, x, z, phi)
    assert abs(oracle.norm2(out) - 1.0) < 1e-12


def test_overlap_and_norm_vs_numpy():
    a = inputs.gaussian_state(9, 1)
    b = inputs.gaussian_state(9, 2)
    assert abs(oracle.overlap(a, b) - np.vdot(a, b)) < 1e-14
    assert abs(oracle.norm2(a) - np.vdot(a, a).real) < 1e-14


def test_common_suffix_identity_eq1_dense():
    """Eq. (1): prod exp(i phi_l P_l (x) Q) = prod exp(i phi_l P_l) (x) (I+Q)/2 + prod exp(-i phi_l P_l) (x) (I-Q)/2."""
    n_low, n_up = 3, 2
    n = n_low + n_up
    rng = np.random.default_rng(44)
    xq, zq = 0b10, 0b11  # Q = Z (x) Y on the upper qubits
    xs, zs = rng.integers(0, 8, 5), rng.integers(0, 8, 5)
    phis = rng.uniform(-1, 1, 5)
    psi = inputs.gaussian_state(n, 45)
    full_x = [int(xl) | (xq << n_low) for xl in xs]
    full_z = [int(zl) | (zq << n_low) for zl in zs]
    lhs = oracle.apply(psi, full_x, full_z, phis)
    plus = np.eye(1 << n_low, dtype=complex)
    minus = np.eye(1 << n_low, dtype=complex)
    for xl, zl, pl in zip(xs, zs, phis):
        p = dense_pauli(n_low, int(xl), int(zl))
        plus = expm_herm(p, pl) @ plus
        minus = expm_herm(p, -pl) @ minus
    q = dense_pauli(n_up, xq, zq)
    eye_u = np.eye(1 << n_up)
    rhs_op = np.kron((eye_u + q) / 2, plus) + np.kron((eye_u - q) / 2, minus)
    assert np.max(np.abs(lhs - rhs_op @ psi)) < 1e-13


# ----------------------------------------------------------- product formulas

def test_trotter_exact_for_diagonal_hamiltonian_closed_form():
    n = 7
    rng = np.random.default_rng(3)
    z = rng.integers(0, 1 << n, 9).astype(np.uint64)
    x = np.zeros_like(z)
    h = rng.normal(size=9)
    psi = inputs.gaussian_state(n, 4)
    t = 1.3
    k = np.arange(1 << n)
    energy = np.zeros(1 << n)
    for zl, hl in zip(z, h):
        par = np.array([bin(int(kk) & int(zl)).count("1") & 1 for kk in k])
        energy += hl * (1 - 2 * par)
    ref = np.exp(1j * t * energy) * psi
    for r in (1, 3, 8):
        assert np.max(np.abs(oracle.trotter(psi, x, z, h, t, r) - ref)) < 1e-13


def test_trotter_exact_for_commuting_xx_yy_zz():
    n = 4
    terms = ["XXII", "YYII", "ZZII", "IIXX", "IIZZ"]
    xz = [oracle.pauli_from_string(s) for s in terms]
    x = [a for a, _ in xz]
    z = [b for _, b in xz]
    h = [0.7, -0.4, 1.1, 0.3, -0.9]
    psi = inputs.gaussian_state(n, 9)
    t = 0.8
    ref = expm_herm(dense_ham(n, x, z, h), t) @ psi
    for r in (1, 2, 5):
        assert np.max(np.abs(oracle.trotter(psi, x, z, h, t, r) - ref)) < 1e-13


def test_trotter_first_order_convergence_rate():
    n = 6
    x, z, h = inputs.jw_hamiltonian(n, 24, seed=12)
    psi = inputs.gaussian_state(n, 13)
    t = 1.0
    ref = expm_herm(dense_ham(n, x, z, h), t) @ psi
    rs = np.array([8, 16, 32, 64, 128])
    errs = np.array([np.linalg.norm(oracle.trotter(psi, x, z, h, t, int(r)) - ref) for r in rs])
    slope = np.polyfit(np.log(rs), np.log(errs), 1)[0]
    assert -1.1 < slope < -0.9, (slope, errs)


def test_splitmix64_published_outputs():
    # Reference outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014;
    # the reference C implementation's first four outputs).
    got = [int(v) for v in oracle.splitmix64(0, 4)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_qdrift_sampler_frequencies_and_segments():
    h = np.array([0.5, -2.0, 0.0, 1.0, -0.25, 3.0])
    N = 200_000
    idx = oracle.qdrift_indices(h, seed=42, first=0, count=N)
    counts = np.bincount(idx.astype(np.int64), minlength=h.size)
    p = np.abs(h) / np.abs(h).sum()
    assert counts[2] == 0  # a zero coefficient is never drawn
    mask = p > 0
    chi2 = np.sum((counts[mask] - N * p[mask]) ** 2 / (N * p[mask]))
    assert chi2 < 25.0  # 4 degrees of freedom; p ~ 5e-5
    # counter-based: any segment equals the corresponding slice of the full stream
    seg = oracle.qdrift_indices(h, seed=42, first=1234, count=500)
    assert np.array_equal(seg, idx[1234:1734])


def _qdrift_expected_g(psi, x, z, h, t, N):
    """E[U] = (cos tau I + i sin tau H / lambda)^N for qDRIFT with tau = lambda t / N."""
    n = psi.size.bit_length() - 1
    lam = np.abs(h).sum()
    tau = lam * t / N
    m = math.cos(tau) * np.eye(1 << n) + 1j * math.sin(tau) * dense_ham(n, x, z, h) / lam
    return np.vdot(psi, np.linalg.matrix_power(m, N) @ psi)


def test_qdrift_mean_matches_exact_expectation():
    n = 4
    x, z, h = inputs.jw_hamiltonian(n, 6, seed=21)
    psi = inputs.gaussian_state(n, 22)
    t, N, S = 0.9, 6, 3000
    g = np.array([np.vdot(psi, oracle.qdrift(psi, x, z, h, t, N, seed=s)) for s in range(S)])
    want = _qdrift_expected_g(psi, x, z, h, t, N)
    band = 5 * (np.std(g.real) + np.std(g.imag)) / math.sqrt(S)
    assert abs(g.mean() - want) < band, (g.mean(), want, band)
    # the wrong sign of time is far outside the band
    wrong = _qdrift_expected_g(psi, x, z, h, -t, N)
    assert abs(g.mean() - wrong) > 3 * band


def test_qdrift_converges_to_exact_evolution():
    n = 4
    x, z, h = inputs.jw_hamiltonian(n, 6, seed=21)
    psi = inputs.gaussian_state(n, 22)
    t = 0.9
    exact = np.vdot(psi, expm_herm(dense_ham(n, x, z, h), t) @ psi)
    errs = [abs(_qdrift_expected_g(psi, x, z, h, t, N) - exact) for N in (10, 100, 1000)]
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5


def test_partial_split_takes_largest_magnitudes():
    h = np.array([0.1, -3.0, 0.5, 3.0, -0.5, 2.0])
    assert list(oracle.partial_split(h, 3)) == [False, True, False, True, False, True]
    # tie between |0.5| and |-0.5|: the lower index wins
    assert list(oracle.partial_split(h, 4)) == [False, True, True, True, False, True]


def test_partial_reduces_to_trotter_and_qdrift():
    n = 5
    x, z, h = inputs.jw_hamiltonian(n, 10, seed=31)
    psi = inputs.gaussian_state(n, 32)
    a = oracle.partial(psi, x, z, h, L_D=10, t=0.7, r=3, Ns=5, seed=1)
    b = oracle.trotter(psi, x, z, h, 0.7, 3)
    assert np.array_equal(a, b)
    a = oracle.partial(psi, x, z, h, L_D=0, t=0.7, r=1, Ns=17, seed=9)
    b = oracle.qdrift(psi, x, z, h, 0.7, 17, seed=9)
    assert np.array_equal(a, b)


def test_partial_mean_matches_exact_expectation():
    n = 4
    x, z, h = inputs.jw_hamiltonian(n, 8, seed=41)
    psi = inputs.gaussian_state(n, 42)
    L_D, t, r, Ns, S = 3, 0.8, 2, 3, 3000
    det = oracle.partial_split(h, L_D)
    delta = t / r
    step = np.eye(1 << n, dtype=complex)
    for l in range(h.size):
        if det[l]:
            step = expm_herm(dense_pauli(n, int(x[l]), int(z[l])), delta * h[l]) @ step
    hr = np.where(det, 0.0, h)
    lam_r = np.abs(hr).sum()
    tau = lam_r * delta / Ns
    m = math.cos(tau) * np.eye(1 << n) + 1j * math.sin(tau) * dense_ham(n, x, z, hr) / lam_r
    step = np.linalg.matrix_power(m, Ns) @ step
    want = np.vdot(psi, np.linalg.matrix_power(step, r) @ psi)
    g = np.array([np.vdot(psi, oracle.partial(psi, x, z, h, L_D, t, r, Ns, seed=s)) for s in range(S)])
    band = 5 * (np.std(g.real) + np.std(g.imag)) / math.sqrt(S)
    assert abs(g.mean() - want) < band, (g.mean(), want, band)


# ------------------------------------------------------- single amplitudes

def test_sparse_amplitudes_vs_dense_products():
    n = 6
    x, z, phi = inputs.random_rotations(n, 9, seed=51)
    idx, amp = inputs.determinant_state(n, seed=52, ndet=3)
    psi0 = inputs.densify(n, idx, amp)
    ref = psi0.copy()
    for xl, zl, pl in zip(x, z, phi):
        ref = expm_herm(dense_pauli(n, int(xl), int(zl)), pl) @ ref
    ks = np.arange(1 << n, dtype=np.uint64)
    got = oracle.amplitudes_sparse(n, idx, amp, x, z, phi, ks)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_trotter_term_order_first_term_acts_first():
    n = 3
    x, z, h = [0b001, 0b010], [0b100, 0b011], [0.9, -1.3]  # X1 Z3 and Z1 Y2 anticommute
    psi = inputs.gaussian_state(n, 61)
    t = 0.6
    ref = expm_herm(dense_pauli(n, x[1], z[1]), t * h[1]) @ (expm_herm(dense_pauli(n, x[0], z[0]), t * h[0]) @ psi)
    wrong = expm_herm(dense_pauli(n, x[0], z[0]), t * h[0]) @ (expm_herm(dense_pauli(n, x[1], z[1]), t * h[1]) @ psi)
    got = oracle.trotter(psi, x, z, h, t, 1)
    assert np.max(np.abs(got - ref)) < 1e-14
    assert np.max(np.abs(got - wrong)) > 1e-3


# ------------------------------------------------------------ second order

def test_trotter2_exact_for_commuting_terms():
    n = 4
    terms = ["XXII", "YYII", "ZZII", "IIXX", "IIZZ"]
    xz = [oracle.pauli_from_string(s) for s in terms]
    x = [a for a, _ in xz]
    z = [b for _, b in xz]
    h = [0.7, -0.4, 1.1, 0.3, -0.9]
    psi = inputs.gaussian_state(n, 19)
    ref = expm_herm(dense_ham(n, x, z, h), 0.8) @ psi
    for r in (1, 2, 5):
        assert np.max(np.abs(oracle.trotter2(psi, x, z, h, 0.8, r) - ref)) < 1e-13


def test_trotter2_second_order_convergence_rate():
    n = 6
    x, z, h = inputs.jw_hamiltonian(n, 24, seed=12)
    psi = inputs.gaussian_state(n, 13)
    ref = expm_herm(dense_ham(n, x, z, h), 1.0) @ psi
    rs = np.array([4, 8, 16, 32, 64])
    errs = np.array([np.linalg.norm(oracle.trotter2(psi, x, z, h, 1.0, int(r)) - ref) for r in rs])
    slope = np.polyfit(np.log(rs), np.log(errs), 1)[0]
    assert -2.1 < slope < -1.9, (slope, errs)


def test_trotter2_is_time_symmetric():
    # S2(-delta) = S2(delta)^-1 for the symmetric splitting; a first-order
    # product (or a second half in the wrong order) fails this
    n = 5
    x, z, h = inputs.jw_hamiltonian(n, 14, seed=21)
    psi = inputs.gaussian_state(n, 22)
    fwd = oracle.trotter2(psi, x, z, h, 0.9, 3)
    back = oracle.trotter2(fwd, x, z, h, -0.9, 3)
    assert np.max(np.abs(back - psi)) < 1e-13
    back1 = oracle.trotter(oracle.trotter(psi, x, z, h, 0.9, 3), x, z, h, -0.9, 3)
    assert np.max(np.abs(back1 - psi)) > 1e-3


def test_partial2_reduces_to_trotter2_and_qdrift():
    n = 5
    x, z, h = inputs.jw_hamiltonian(n, 10, seed=31)
    psi = inputs.gaussian_state(n, 32)
    a = oracle.partial2(psi, x, z, h, L_D=10, t=0.7, r=3, Ns=5, seed=1)
    assert np.array_equal(a, oracle.trotter2(psi, x, z, h, 0.7, 3))
    # no deterministic part, one step: 2 Ns draws over time t, i.e. qDRIFT with N = 2 Ns
    a = oracle.partial2(psi, x, z, h, L_D=0, t=0.7, r=1, Ns=17, seed=9)
    assert np.array_equal(a, oracle.qdrift(psi, x, z, h, 0.7, 34, seed=9))


def test_partial2_mean_matches_exact_expectation():
    n = 4
    x, z, h = inputs.jw_hamiltonian(n, 8, seed=41)
    psi = inputs.gaussian_state(n, 43)
    L_D, t, r, Ns, S = 3, 0.8, 2, 2, 3000
    det = oracle.partial_split(h, L_D)
    half = 0.5 * t / r
    fwd = np.eye(1 << n, dtype=complex)
    for l in range(h.size):
        if det[l]:
            fwd = expm_herm(dense_pauli(n, int(x[l]), int(z[l])), half * h[l]) @ fwd
    bwd = np.eye(1 << n, dtype=complex)
    for l in reversed(range(h.size)):
        if det[l]:
            bwd = expm_herm(dense_pauli(n, int(x[l]), int(z[l])), half * h[l]) @ bwd
    hr = np.where(det, 0.0, h)
    lam_r = np.abs(hr).sum()
    tau = lam_r * (t / r) / (2 * Ns)
    m = math.cos(tau) * np.eye(1 << n) + 1j * math.sin(tau) * dense_ham(n, x, z, hr) / lam_r
    step = bwd @ np.linalg.matrix_power(m, 2 * Ns) @ fwd
    want = np.vdot(psi, np.linalg.matrix_power(step, r) @ psi)
    g = np.array([np.vdot(psi, oracle.partial2(psi, x, z, h, L_D, t, r, Ns, seed=s)) for s in range(S)])
    band = 5 * (np.std(g.real) + np.std(g.imag)) / math.sqrt(S)
    assert abs(g.mean() - want) < band, (g.mean(), want, band)


def test_lexicographic_order_hand_example():
    # strings written qubit 1 first; the order reads them from qubit n down, I < X < Y < Z
    terms = ["XZ", "ZI", "IY", "YY"]
    xz = [oracle.pauli_from_string(s) for s in terms]
    order = oracle.lexicographic_order(2, [a for a, _ in xz], [b for _, b in xz])
    assert order == [1, 2, 3, 0]


def test_threaded_oracle_gives_the_same_rotations():
    """The OpenMP pragmas only share the element loops among threads: a
    rotation writes every output element once, so the state is bitwise the
    same for any thread count; only the order of the overlap and norm sums
    changes (a few ulps)."""
    n = 14
    psi0 = inputs.gaussian_state(n, 51)
    x, z, phi = inputs.random_rotations(n, 40, seed=52)
    one = oracle.apply(psi0, x, z, phi)
    g1, n1 = oracle.overlap(psi0, one), oracle.norm2(one)
    a1 = oracle.amplitudes_sparse(n, [5, 77], [0.6, 0.8j], x[:12], z[:12], phi[:12], [5, 77, 5 ^ int(x[0])])
    try:
        used = oracle.set_threads(4)
        many = oracle.apply(psi0, x, z, phi)
        g4, n4 = oracle.overlap(psi0, many), oracle.norm2(many)
        a4 = oracle.amplitudes_sparse(n, [5, 77], [0.6, 0.8j], x[:12], z[:12], phi[:12], [5, 77, 5 ^ int(x[0])])
    finally:
        oracle.set_threads(1)
    assert used == (4 if oracle.has_openmp() else 1)
    assert np.array_equal(one, many)
    assert np.array_equal(a1, a4)
    assert abs(g1 - g4) < 1e-14 and abs(n1 - n4) < 1e-14


def test_oracle_streams_are_the_rotations_its_drivers_apply():
    """qdrift_stream / partial_stream list exactly the rotations or_qdrift and
    or_partial apply: applying the listed rotations gives bitwise the same
    state (same angles, same order, same products)."""
    n = 7
    x, z, h = inputs.jw_hamiltonian(n, 50, seed=61)
    psi0 = inputs.gaussian_state(n, 62)
    xs, zs, ph = oracle.qdrift_stream(x, z, h, 0.9, 120, 63)
    assert np.array_equal(oracle.apply(psi0, xs, zs, ph), oracle.qdrift(psi0, x, z, h, 0.9, 120, 63))
    a, b, c = oracle.qdrift_stream(x, z, h, 0.9, 120, 63, first=40, count=30)
    assert np.array_equal(a, xs[40:70]) and np.array_equal(b, zs[40:70]) and np.array_equal(c, ph[40:70])
    for L_D, Ns in ((10, 7), (0, 9), (50, 5)):
        xs, zs, ph = oracle.partial_stream(x, z, h, L_D, 0.8, 3, Ns, 64)
        assert len(ph) == 3 * (L_D + (Ns if L_D < 50 else 0))
        assert np.array_equal(oracle.apply(psi0, xs, zs, ph), oracle.partial(psi0, x, z, h, L_D, 0.8, 3, Ns, 64))
