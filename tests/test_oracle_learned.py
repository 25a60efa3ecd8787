"""Pins of the learned-step-choice oracle (oracle/learned.py), CPU only.

Each check ties the oracle to something other than itself: dense Pauli
matrices, closed forms of the bound on small Hamiltonians, a hand-computed
feature vector, central finite differences of the loss, and the closed form of
Adam's first step.
"""
import math

import numpy as np
import pytest

from oracle import learned as L

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)


def dense(n, x, z):
    """Dense matrix of the string: qubit q (bit q) is the q-th factor from the right."""
    m = np.ones((1, 1), dtype=complex)
    for q in reversed(range(n)):
        f = {(0, 0): I2, (1, 0): PX, (0, 1): PZ, (1, 1): PY}[((x >> q) & 1, (z >> q) & 1)]
        m = np.kron(m, f)
    return m


def test_anticommutation_matches_dense_matrices():
    n = 2
    for x1 in range(4):
        for z1 in range(4):
            for x2 in range(4):
                for z2 in range(4):
                    A, B = dense(n, x1, z1), dense(n, x2, z2)
                    anti = np.allclose(A @ B, -(B @ A))
                    comm = np.allclose(A @ B, B @ A)
                    assert anti != comm
                    assert L.anticommute(n, x1, z1, x2, z2) == anti
    rng = np.random.default_rng(0)
    for _ in range(60):
        x1, z1, x2, z2 = (int(v) for v in rng.integers(0, 16, size=4))
        A, B = dense(4, x1, z1), dense(4, x2, z2)
        assert L.anticommute(4, x1, z1, x2, z2) == np.allclose(A @ B, -(B @ A))


def test_bound_closed_forms():
    a, b = 0.7, -0.3
    # H = a X + b Z on one qubit: the two terms anticommute
    x, z, h = [1, 0], [0, 1], [a, b]
    assert L.trotter_bound(1, x, z, h) == pytest.approx(8 * abs(a) * abs(b), rel=1e-15)
    # only the larger term deterministic: the randomised-part terms of the bound
    big, small = abs(a), abs(b)
    assert L.trotter_bound(1, x, z, h, L_D=1) == pytest.approx(small * big ** 2 + big * small ** 2, rel=1e-15)
    # everything randomised: lambda_R = lambda and both randomised-part terms vanish
    assert L.trotter_bound(1, x, z, h, L_D=0) == 0.0
    # mutually commuting terms: no deterministic contribution
    assert L.trotter_bound(2, [0, 0, 0], [1, 2, 3], [0.5, -0.2, 0.1]) == 0.0
    # {X1X2, Z1Z2, Y1Y2} commute pairwise
    assert L.trotter_bound(2, [3, 0, 3], [0, 3, 3], [0.4, 0.3, -0.2]) == 0.0


def test_features_hand_example():
    # n = 2: 0.5 X1, -0.25 Z1 Z2, 0.25 Y2; psi = |00>
    n, x, z, h = 2, [1, 0, 2], [0, 3, 2], [0.5, -0.25, 0.25]
    psi = np.zeros(4, dtype=complex)
    psi[0] = 1.0
    t, r = 0.8, 4
    f = L.features(n, x, z, h, t, r, psi)
    lam = 1.0
    # anticommuting pairs: X1 with Z1Z2 (qubit 1: X vs Z), Z1Z2 with Y2 (qubit 2: Z vs Y); X1 and Y2 commute
    C = 4 * (0.5 * 0.25 + 0.25 * (0.5 + 0.25) + 0.25 * 0.25)
    # K on |00>: pair (X1, Z1Z2): h2 h1 <00|Z1Z2 X1|00> = 0 (X1 flips qubit 1);
    # pair (Z1Z2, Y2): h3 h2 <00|Y2 Z1Z2|00> = 0 (Y2 flips qubit 2)
    expect = [math.log(3), math.log(lam), math.log(0.5), math.log(t), math.log(r), math.log(C),
              math.log(C * t * t / r), 0.25, math.log(L.K_FLOOR)]
    # E2 |00> = -(h2 h1 Z1Z2 X1 + h3 h2 Y2 Z1Z2)|00>: Z1Z2 X1|00> = Z1Z2|01> = -|01> (qubit 1 set),
    # Y2 Z1Z2|00> = Y2|00> = i|10>; so E2|00> = -(-0.125 * -1)|01> - (-0.0625 i)|10>
    n2 = 0.125 ** 2 + 0.0625 ** 2
    # K = 0 on |00>: the estimate is the second-order one alone
    expect += [math.log(n2), math.log(n2 * t ** 4 / (2 * r * r)), 0.0]
    assert np.allclose(f, expect, rtol=1e-14, atol=1e-15)


def test_error_coefficient_dense_and_small_time_limit():
    """K against dense commutators, and g_r - g -> -(t^2 / r) K as t -> 0
    (first-order Trotter against the exact exponential of the dense H)."""
    import scipy.linalg
    rng = np.random.default_rng(4)
    n = 3
    x = [1, 3, 6, 2, 5, 0]
    z = [0, 1, 6, 3, 4, 5]
    h = list(rng.normal(size=len(x)))
    psi = rng.normal(size=8) + 1j * rng.normal(size=8)
    psi /= np.linalg.norm(psi)
    P = [dense(n, xv, zv) for xv, zv in zip(x, z)]
    Kd = 0j
    for k in range(len(h)):
        for l in range(k + 1, len(h)):
            Kd += h[l] * h[k] * np.vdot(psi, (P[l] @ P[k] - P[k] @ P[l]) @ psi) / 2
    K = L.error_coefficient(n, x, z, h, psi)
    assert abs(K - Kd) < 1e-13
    E2 = sum(-0.5 * h[l] * h[k] * (P[l] @ P[k] - P[k] @ P[l]) for k in range(len(h)) for l in range(k + 1, len(h)))
    assert L.second_order_norm2(n, x, z, h, psi) == pytest.approx(np.linalg.norm(E2 @ psi) ** 2, rel=1e-13)
    H = sum(hv * Pm for hv, Pm in zip(h, P))
    for r in (1, 3):
        t = 2e-3
        step = np.eye(8, dtype=complex)
        for hv, Pm in zip(h, P):
            step = scipy.linalg.expm(1j * (t / r) * hv * Pm) @ step
        Ur = np.linalg.matrix_power(step, r)
        g_r = np.vdot(psi, Ur @ psi)
        g = np.vdot(psi, scipy.linalg.expm(1j * t * H) @ psi)
        assert abs((g_r - g) * r / t ** 2 + K) < 2e-2 * max(1.0, abs(K))


def rand_params(n_in, width, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    size = sum(int(np.prod(s)) for _, s in L.param_shapes(n_in, width))
    return rng.normal(0, scale, size=size)


def test_backprop_matches_central_differences():
    n_in, width = 3, 6
    p = rand_params(n_in, width, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(7, n_in))
    T = rng.normal(size=7)
    loss, g = L.loss_and_grad(p, X, T, n_in, width)
    eps = 1e-6
    fd = np.zeros_like(p)
    for j in range(len(p)):
        q = p.copy()
        q[j] += eps
        lp, _ = L.loss_and_grad(q, X, T, n_in, width)
        q[j] -= 2 * eps
        lm, _ = L.loss_and_grad(q, X, T, n_in, width)
        fd[j] = (lp - lm) / (2 * eps)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_forward_closed_forms():
    n_in, width = 2, 4
    size = sum(int(np.prod(s)) for _, s in L.param_shapes(n_in, width))
    p = L.unpack(np.zeros(size), n_in, width)
    p["b_out"][0] = 0.37
    X = np.array([[1.0, -2.0], [0.5, 3.0]])
    out, _ = L.forward(L.pack(p, n_in, width), X, n_in, width)
    assert np.allclose(out, 0.37)
    # one path through the first unit of every layer
    p = L.unpack(np.zeros(size), n_in, width)
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][0, 0] = 1.0
    p["w_out"][0] = 1.0
    out, _ = L.forward(L.pack(p, n_in, width), X, n_in, width)
    assert np.allclose(out, np.tanh(np.tanh(np.tanh(X[:, 0]))), rtol=1e-15)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.normal(size=20)
    g = rng.normal(size=20)
    z = np.zeros(20)
    lr, eps = 0.01, 1e-8
    p1, m1, v1 = L.adam_step(p, g, z, z, 1, lr, eps=eps)
    # first step: the bias-corrected moments are g and g^2
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=1e-14, atol=1e-16)
    # a constant gradient moves every parameter by about lr per step
    q, m, v = p, z, z
    for s in range(1, 200):
        q_new, m, v = L.adam_step(q, g, m, v, s, lr, eps=eps)
        step = q - q_new
        q = q_new
    assert np.allclose(step, lr * np.sign(g), rtol=1e-6)


def test_richardson_limit_is_exact_for_the_first_order_error_form():
    """g_r = g + a/r + b/r^2 exactly: the three-run limit is g (closed form),
    for any R; an r^-3 term leaves an error that falls 8x per doubling of R."""
    g, a, b = 0.3 - 0.2j, 1.7 + 0.4j, -2.5 + 1.1j
    for R in (1.0, 8.0, 32.0):
        gr = [g + a / r + b / r ** 2 for r in (R, 2 * R, 4 * R)]
        assert abs(L.richardson3(*gr, R=R) - g) < 1e-13
        assert abs(L.richardson3(*gr) - g) < 1e-12  # the limit does not depend on R
    c = 3.0
    err = []
    for R in (8.0, 16.0, 32.0):
        gr = [g + a / r + b / r ** 2 + c / r ** 3 for r in (R, 2 * R, 4 * R)]
        err.append(abs(L.richardson3(*gr, R=R) - g))
    assert 7.5 < err[0] / err[1] < 8.5 and 7.5 < err[1] / err[2] < 8.5


def test_labels_margin_and_bound_steps_closed_forms():
    # labels: g_r = g_lim + a/r gives log eps = log|a| - log r; the floor caps small errors
    a = 0.02 - 0.01j
    g = [0.5 + a / r for r in (1, 2, 4)] + [0.5 + 1e-20]
    eps, lg = L.error_labels(g, 0.5, 1e-12)
    assert np.allclose(eps[:3], abs(a) / np.array([1, 2, 4]), rtol=1e-14)
    assert np.allclose(lg[:3], math.log(abs(a)) - np.log([1, 2, 4]), rtol=1e-14)
    assert lg[3] == math.log(1e-12)
    # margin: residuals 0..99, the 0.8 quantile at position 79.2; all-negative residuals give 0
    y = np.arange(100, dtype=np.float64)
    assert abs(L.margin(y, np.zeros(100), 0.8) - 79.2) < 1e-12
    assert L.margin(-y - 1, np.zeros(100), 0.8) == 0.0
    # bound steps: H = 0.5 X + 0.25 Z anticommute, C = 4 (0.5 * 0.25 + 0.25 * 0.5) = 1
    assert L.trotter_bound(1, [1, 0], [0, 1], [0.5, 0.25]) == 1.0
    assert L.bound_steps(1, [1, 0], [0, 1], [0.5, 0.25], 1.0, 1e-3) == 32   # ceil(sqrt(1000))
    assert L.bound_steps(1, [1, 0], [0, 1], [0.5, 0.25], 2.0, 1e-3) == 64   # ceil(63.25)
    assert L.bound_steps(1, [1, 0], [0, 1], [0.5, 0.25], 1e-3, 1.0) == 1
