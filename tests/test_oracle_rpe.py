"""Robust phase estimation: the oracle against what the method fixes, and
libps's ps_rpe_estimate against the oracle (CPU only).

Pins (Methods, "Data analysis"; RPE after Kimmel et al. 2015):
  * an exact single-frequency signal e^{i 2^m theta} gives theta back for any
    theta in (-pi, pi), at every round;
  * with every round's phase error below pi/3 every branch choice is right,
    so the last estimate is theta plus round M's error over 2^M, exactly;
  * a signal with one dominant component (weight >= 0.85) returns that
    component's phase within asin(rest / dominant) / 2^M;
  * end to end: the first-order Trotter step U(delta) of a 4-qubit JW-like H
    as a dense matrix, its eigenphases from numpy, a state mostly along one
    eigenvector, the oracle's own signal, and the estimate equal to that
    eigenphase.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import rpe as OR
import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs


def exact_signal(theta, M, weight=1.0):
    return weight * np.exp(1j * theta * 2.0 ** np.arange(M + 1))


@pytest.mark.parametrize("theta", [0.0, 0.3, -1.1, 2.9, -3.1, 1e-6])
def test_exact_signal_returns_its_phase(theta):
    M = 10
    E, thetas = OR.rpe_estimate(exact_signal(theta, M, 0.7), 0.25)
    assert all(abs(t - theta) < 1e-12 for t in thetas)
    assert abs(E - theta / 0.25) < 1e-11


def test_branch_choice_is_right_below_pi_over_3():
    rng = np.random.default_rng(3)
    M = 12
    for _ in range(200):
        theta = rng.uniform(-math.pi * 0.9, math.pi * 0.9)
        err = rng.uniform(-1.0, 1.0, size=M + 1) * (math.pi / 3 - 1e-3)
        err[0] = rng.uniform(-1, 1) * min(math.pi / 3 - 1e-3, math.pi - abs(theta) - 1e-3)
        Z = np.exp(1j * (theta * 2.0 ** np.arange(M + 1) + err))
        _, thetas = OR.rpe_estimate(Z, 1.0)
        for m in range(M + 1):
            assert abs(thetas[m] - (theta + err[m] / 2.0 ** m)) < 1e-12, (m, theta)


def test_a_wrong_branch_appears_beyond_pi_over_3():
    # the bound is sharp: errors 2 e_{m-1} - e_m beyond pi flip round m's branch
    theta, M = 0.4, 3
    err = np.array([0.0, 1.2, -1.2, 0.0])  # |2 * 1.2 + 1.2| > pi at m = 2
    Z = np.exp(1j * (theta * 2.0 ** np.arange(M + 1) + err))
    _, thetas = OR.rpe_estimate(Z, 1.0)
    assert abs(thetas[2] - (theta + err[2] / 4)) > 1.0


def test_dominant_component_is_resolved():
    rng = np.random.default_rng(4)
    M = 9
    for _ in range(50):
        th = rng.uniform(-2.5, 2.5, size=4)
        w = np.array([0.85, 0.07, 0.05, 0.03])
        Z = (w[:, None] * np.exp(1j * th[:, None] * 2.0 ** np.arange(M + 1))).sum(axis=0)
        E, _ = OR.rpe_estimate(Z, 1.0)
        assert abs(E - th[0]) <= math.asin(0.15 / 0.85) / 2.0 ** M + 1e-12


def test_trotter_signal_of_a_near_eigenstate_gives_the_eigenphase():
    n, delta, M = 4, 0.2, 7
    x, z, h = inputs.jw_hamiltonian(n, 12, seed=31, lam=3.0)
    dim = 1 << n
    # U(delta) as a dense matrix: the oracle's one-step product formula on basis vectors
    U = np.zeros((dim, dim), dtype=np.complex128)
    for k in range(dim):
        e = np.zeros(dim, dtype=np.complex128)
        e[k] = 1.0
        U[:, k] = oracle.trotter(e, x, z, h, delta, 1)
    assert np.allclose(U.conj().T @ U, np.eye(dim), atol=1e-12)
    # U = exp(i delta H_eff): its eigenvectors from the Hermitian (U + U^+)/2
    # and (U - U^+)/2i, which commute with U
    Hr = (U + U.conj().T) / 2
    Hi = (U - U.conj().T) / 2j
    vals, vecs = np.linalg.eigh(Hr + 0.37 * Hi)  # generic mix separates the eigenphases
    v0 = vecs[:, 0]
    lam = v0.conj() @ U @ v0
    theta0 = np.angle(lam)
    assert abs(abs(lam) - 1.0) < 1e-10 and np.allclose(U @ v0, lam * v0, atol=1e-10)
    rng = np.random.default_rng(5)
    w = rng.normal(size=dim) + 1j * rng.normal(size=dim)
    w -= (v0.conj() @ w) * v0
    w /= np.linalg.norm(w)
    psi0 = math.sqrt(0.85) * v0 + math.sqrt(0.15) * w
    Z = OR.signal(psi0, x, z, h, delta, M)
    E, _ = OR.rpe_estimate(Z, delta)
    assert abs(E * delta - theta0) <= math.asin(0.15 / 0.85) / 2.0 ** M + 1e-10
    # the library's estimator reads the same signal the same way
    E_lib, th_lib = ps.ps_rpe_estimate(Z, delta)
    _, th_or = OR.rpe_estimate(Z, delta)
    assert np.allclose(th_lib, th_or, rtol=0, atol=1e-15) and abs(E_lib - E) < 1e-12


def test_library_estimator_matches_the_oracle_and_validates():
    rng = np.random.default_rng(6)
    for M in (0, 1, 5, 20):
        Z = rng.normal(size=M + 1) + 1j * rng.normal(size=M + 1)
        E_lib, th_lib = ps.ps_rpe_estimate(Z, 0.3)
        E_or, th_or = OR.rpe_estimate(Z, 0.3)
        assert np.allclose(th_lib, th_or, rtol=0, atol=1e-15) and abs(E_lib - E_or) < 1e-13
    with pytest.raises(ps.PsError):
        ps.ps_rpe_estimate([1.0, complex(np.nan, 0)], 0.1)
    with pytest.raises(ps.PsError):
        ps.ps_rpe_estimate([1.0], 0.0)
