"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only draws random numbers into arrays; it holds none of the
method's arithmetic.  The paper's Hamiltonians (ruthenium-ligand active
spaces, Methods, "Hamiltonian preparation") and guiding states (a few
Slater determinants of the reference wave function) are not available, so
these generators stand in for them with the same shapes:

* ``jw_hamiltonian`` -- Jordan-Wigner-like Pauli terms: X or Y on 2 or 4
  qubits, an even number of Y factors, a Z chain between the first two (and
  the last two) chosen qubits, log-normal coefficient magnitudes with random
  signs, rescaled to a target one-norm lambda.  The paper reports 875 to
  229,140 terms for 10 to 40 qubits and lambda = 2.6 ... 48.9 (Table S2);
  the default lambda(L) = 3.5 (L / 2000)^0.4735 passes through 3.5 at 2000
  terms and 7.5 at 10^4 terms, comparable to Table S2 at those term counts.
* ``determinant_state`` -- a normalised superposition of a few computational
  basis states of Hamming weight floor(n/2) (half filling), standing in for
  the few-determinant guiding state.
* ``gaussian_state`` -- complex Gaussian amplitudes, normalised.
* ``random_rotations`` -- each qubit I/X/Y/Z uniformly, angles uniform in
  [-pi, pi].

Pauli strings are returned as the bitmask pair (x, z) with qubit q at bit q
(bit set in x for X or Y, in z for Y or Z).
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_state(n: int, seed: int) -> np.ndarray:
    """2^n complex Gaussian amplitudes (real parts drawn first, then imaginary), unit norm."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(1 << n)
    im = rng.standard_normal(1 << n)
    psi = re + 1j * im
    return psi / np.sqrt(np.sum(re * re + im * im))


def random_rotations(n: int, count: int, seed: int):
    """`count` rotations on n qubits: every qubit I, X, Y or Z with probability 1/4 each."""
    rng = np.random.default_rng(seed)
    letters = rng.integers(0, 4, size=(count, n))  # 0=I 1=X 2=Y 3=Z
    weights = (np.uint64(1) << np.arange(n, dtype=np.uint64))
    xbits = ((letters == 1) | (letters == 2)).astype(np.uint64)
    zbits = ((letters == 2) | (letters == 3)).astype(np.uint64)
    x = (xbits * weights).sum(axis=1, dtype=np.uint64)
    z = (zbits * weights).sum(axis=1, dtype=np.uint64)
    phi = rng.uniform(-math.pi, math.pi, size=count)
    return x, z, phi


def default_lambda(L: int) -> float:
    return 3.5 * (L / 2000.0) ** 0.4735


def jw_hamiltonian(n: int, L: int, seed: int, lam: float | None = None, p_two_qubit: float = 0.2,
                   sigma: float = 1.5):
    """L distinct JW-like terms (x, z, h) on n >= 4 qubits with one-norm `lam`."""
    if n < 4:
        raise ValueError("jw_hamiltonian needs n >= 4")
    rng = np.random.default_rng(seed)
    terms: dict[tuple[int, int], float] = {}
    order: list[tuple[int, int]] = []
    attempts = 0
    while len(order) < L:
        attempts += 1
        if attempts > 1000 * L + 10000:
            raise ValueError(f"cannot draw {L} distinct JW-like terms on {n} qubits")
        w = 2 if rng.random() < p_two_qubit else 4
        q = np.sort(rng.choice(n, size=w, replace=False))
        ys = rng.integers(0, 2, size=w)
        if ys.sum() % 2:
            ys[-1] ^= 1  # even number of Y factors, as for a real Hamiltonian
        x = 0
        z = 0
        for qi, y in zip(q, ys):
            x |= 1 << int(qi)
            if y:
                z |= 1 << int(qi)
        for a, b in ((0, 1), (2, 3)) if w == 4 else ((0, 1),):
            for qq in range(int(q[a]) + 1, int(q[b])):
                z |= 1 << qq
        mag = rng.lognormal(0.0, sigma)
        h = mag if rng.random() < 0.5 else -mag
        key = (x, z)
        if key in terms:
            terms[key] += h  # duplicate string: merge coefficients
        else:
            terms[key] = h
            order.append(key)
    xs = np.array([k[0] for k in order], dtype=np.uint64)
    zs = np.array([k[1] for k in order], dtype=np.uint64)
    hs = np.array([terms[k] for k in order], dtype=np.float64)
    target = default_lambda(L) if lam is None else lam
    hs *= target / np.abs(hs).sum()
    return xs, zs, hs


def determinant_state(n: int, seed: int, ndet: int = 8, min_distance: int = 0):
    """Sparse state: (indices, complex amplitudes) of `ndet` distinct half-filled
    basis states, pairwise at Hamming distance >= min_distance when given."""
    rng = np.random.default_rng(seed)
    weight = n // 2
    idx: list[int] = []
    attempts = 0
    restarts = 0
    while len(idx) < ndet:
        attempts += 1
        if attempts > 5000:
            # the determinants drawn so far leave no room: start the set again
            restarts += 1
            if restarts > 100:
                raise ValueError(f"cannot draw {ndet} determinants of {n} qubits at distance >= {min_distance}")
            idx, attempts = [], 0
        bits = rng.choice(n, size=weight, replace=False)
        k = int(sum(1 << int(b) for b in bits))
        if k in idx or any(bin(k ^ j).count("1") < min_distance for j in idx):
            continue
        idx.append(k)
    amp = rng.standard_normal(ndet) + 1j * rng.standard_normal(ndet)
    amp /= np.sqrt(np.sum(np.abs(amp) ** 2))
    return np.array(idx, dtype=np.uint64), amp


def densify(n: int, idx, amp) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[np.asarray(idx, dtype=np.int64)] = amp
    return psi
