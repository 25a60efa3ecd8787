"""Oracle of the learned step choice (test infrastructure, not product code).

Plain numpy / Python, FP64, written from the definitions:
  * Pauli (anti)commutation from the single-qubit rule: two single-qubit
    Paulis anticommute iff both are non-identity and different; two strings
    anticommute iff an odd number of their qubits do.
  * The analytic bound on the Trotter-error prefactor for the partially
    randomised decomposition (Methods, "Data analysis"; Poulin et al.):
        C <= 4 sum_{l in D} |h_l| sum_{k in D, [P_l, P_k] != 0} |h_k|
             + lambda_R (lambda - lambda_R)^2 + (lambda - lambda_R) lambda_R^2,
    D = the first L_D terms by decreasing |h| (ties keep input order), R the rest.
  * The leading-order coefficient K of the first-order Trotter error of the
    overlap (from the second-order term of the product formula's exponent),
    and the feature vector of a (Hamiltonian, t, r, initial state) query
    (twelve numbers).
  * A tanh multilayer perceptron with a linear scalar output, its mean-squared
    loss, the gradient by backpropagation, and one Adam step (Kingma & Ba).
  * The training labels: the r -> infinity limit of first-order overlaps
    g_r = g + a/r + b/r^2 from three runs (the 3x3 linear system solved
    as written), eps = |g_r - g|, log eps with a floor; the pick margin (a
    quantile of held-out residuals, numpy's); the bound's step count from
    the paper's error model eps = C (t/r)^2.
Only ``tests/`` may import this module.  It shares no code with the CUDA
library.
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 12
K_FLOOR = 1e-6


# ------------------------------------------------------------ Pauli algebra

def single_qubit(x_bit: int, z_bit: int) -> str:
    """Factor on one qubit from its (x, z) bits: I, X, Z or Y."""
    return {(0, 0): "I", (1, 0): "X", (0, 1): "Z", (1, 1): "Y"}[(x_bit, z_bit)]


def anticommute(n: int, x1: int, z1: int, x2: int, z2: int) -> bool:
    """True iff the strings (x1, z1) and (x2, z2) anticommute (qubit by qubit)."""
    odd = 0
    for q in range(n):
        a = single_qubit((x1 >> q) & 1, (z1 >> q) & 1)
        b = single_qubit((x2 >> q) & 1, (z2 >> q) & 1)
        if a != "I" and b != "I" and a != b:
            odd ^= 1
    return odd == 1


def split_order(h) -> list[int]:
    """Term indices by decreasing |h|, ties in input order."""
    return sorted(range(len(h)), key=lambda l: (-abs(float(h[l])), l))


def trotter_bound(n: int, x, z, h, L_D: int | None = None) -> float:
    """The analytic bound on the Trotter-error prefactor (see module docstring)."""
    L = len(h)
    L_D = L if L_D is None else L_D
    order = split_order(h)
    D, R = order[:L_D], order[L_D:]
    lam = sum(abs(float(v)) for v in h)
    lam_R = sum(abs(float(h[k])) for k in R)
    det = 0.0
    for l in D:
        s = 0.0
        for k in D:
            if anticommute(n, int(x[l]), int(z[l]), int(x[k]), int(z[k])):
                s += abs(float(h[k]))
        det += abs(float(h[l])) * s
    return 4.0 * det + lam_R * (lam - lam_R) ** 2 + (lam - lam_R) * lam_R ** 2


def pauli_apply(n: int, x: int, z: int, psi: np.ndarray) -> np.ndarray:
    """P psi from P|k> = i^{popc(x & z)} (-1)^{popc(k & z)} |k ^ x>, basis state by basis state."""
    out = np.zeros_like(psi)
    ph = 1j ** (bin(x & z).count("1") % 4)
    for k in range(1 << n):
        if psi[k] != 0:
            out[k ^ x] += ph * (-1) ** (bin(k & z).count("1") % 2) * psi[k]
    return out


def error_coefficient(n: int, x, z, h, psi: np.ndarray) -> complex:
    """K = sum over pairs k < l (k applied first) of anticommuting terms of
    h_l h_k <psi|P_l P_k|psi>.  One first-order Trotter step of size delta
    is exp(i delta H - (delta^2 / 2) sum_{l>k} h_l h_k [P_l, P_k] + ...),
    and [P_l, P_k] = 2 P_l P_k for anticommuting strings, so for small t
    g_r - g = -(t^2 / r) K + O(t^3 / r)."""
    L = len(h)
    K = 0.0 + 0.0j
    for k in range(L):
        pk = pauli_apply(n, int(x[k]), int(z[k]), psi)
        for l in range(k + 1, L):
            if anticommute(n, int(x[l]), int(z[l]), int(x[k]), int(z[k])):
                K += float(h[l]) * float(h[k]) * np.vdot(psi, pauli_apply(n, int(x[l]), int(z[l]), pk))
    return complex(K)


def second_order_norm2(n: int, x, z, h, psi: np.ndarray) -> float:
    """||E2 psi||^2 with E2 = -(1/2) sum_{l>k} h_l h_k [P_l, P_k] = -sum over
    anticommuting pairs k < l of h_l h_k P_l P_k, the second-order term of one
    Trotter step's exponent.  When K = 0 the overlap error starts at
    (t^4 / (2 r^2)) <psi|E2^2|psi> = -(t^4 / (2 r^2)) ||E2 psi||^2."""
    L = len(h)
    v = np.zeros_like(psi)
    for k in range(L):
        pk = pauli_apply(n, int(x[k]), int(z[k]), psi)
        for l in range(k + 1, L):
            if anticommute(n, int(x[l]), int(z[l]), int(x[k]), int(z[k])):
                v += float(h[l]) * float(h[k]) * pauli_apply(n, int(x[l]), int(z[l]), pk)
    return float(np.vdot(v, v).real)


def features(n: int, x, z, h, t: float, r: int, psi: np.ndarray) -> np.ndarray:
    """Feature vector of the query "first-order Trotter, r steps, time t,
    initial state psi":
      0  log L
      1  log lambda                      (lambda = sum |h|)
      2  log(max |h| / lambda)
      3  log t
      4  log r
      5  log C                           (C = trotter_bound with L_D = L)
      6  log(C t^2 / r)                  (the bound's error scale)
      7  sum over diagonal terms (x = 0) of |h| / lambda
      8  log(max(|K| / lambda^2, K_FLOOR))             (K = error_coefficient)
      9  log(max(||E2 psi||^2 / lambda^4, K_FLOOR))    (second_order_norm2)
     10  log(e1 + e2), e1 = |K| t^2 / r, e2 = ||E2 psi||^2 t^4 / (2 r^2)
                                        (the first- and second-order estimates of the overlap error)
     11  e1 / (e1 + e2)                 (the first-order share; 0 when both vanish)
    """
    hab = [abs(float(v)) for v in h]
    lam = sum(hab)
    C = trotter_bound(n, x, z, h)
    diag = sum(a for a, xv in zip(hab, x) if int(xv) == 0)
    K = abs(error_coefficient(n, x, z, h, psi))
    N2 = second_order_norm2(n, x, z, h, psi)
    e1 = K * t * t / r
    e2 = N2 * t ** 4 / (2.0 * r * r)
    est = math.log(max(e1 + e2, K_FLOOR * lam * lam * t * t / r))
    share = e1 / (e1 + e2) if e1 + e2 > 0 else 0.0
    return np.array([math.log(len(h)), math.log(lam), math.log(max(hab) / lam), math.log(t), math.log(r),
                     math.log(C), math.log(C) + 2.0 * math.log(t) - math.log(r), diag / lam,
                     math.log(max(K / (lam * lam), K_FLOOR)), math.log(max(N2 / lam ** 4, K_FLOOR)), est, share],
                    dtype=np.float64)


# ------------------------------------------------------------------- MLP

def param_shapes(n_in: int, width: int, hidden: int = 3):
    """(name, shape) in the flat parameter order: W1 (width x n_in), b1, then
    W_k (width x width), b_k for the other hidden layers, then w_out (width), b_out (1).
    Weights are out-major: W[o, i] multiplies input i into output o."""
    shapes = [("W1", (width, n_in)), ("b1", (width,))]
    for k in range(2, hidden + 1):
        shapes += [(f"W{k}", (width, width)), (f"b{k}", (width,))]
    shapes += [("w_out", (width,)), ("b_out", (1,))]
    return shapes


def unpack(flat, n_in: int, width: int, hidden: int = 3) -> dict:
    out, at = {}, 0
    for name, shape in param_shapes(n_in, width, hidden):
        size = int(np.prod(shape))
        out[name] = np.asarray(flat[at:at + size], dtype=np.float64).reshape(shape)
        at += size
    assert at == len(flat)
    return out


def pack(p: dict, n_in: int, width: int, hidden: int = 3) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1)
                           for name, _ in param_shapes(n_in, width, hidden)])


def forward(flat, X, n_in: int, width: int, hidden: int = 3):
    """Network output for the rows of X (already standardised) and the
    hidden activations: h_1 = tanh(W1 x + b1), h_k = tanh(W_k h_{k-1} + b_k),
    out = w_out . h_hidden + b_out."""
    p = unpack(flat, n_in, width, hidden)
    X = np.asarray(X, dtype=np.float64)
    hs = []
    a = X
    for k in range(1, hidden + 1):
        a = np.tanh(a @ p[f"W{k}"].T + p[f"b{k}"])
        hs.append(a)
    out = a @ p["w_out"] + p["b_out"][0]
    return out, hs


def loss_and_grad(flat, X, T, n_in: int, width: int, hidden: int = 3):
    """Mean squared error (1/B) sum (out - t)^2 and its gradient by
    backpropagation, in the flat parameter order."""
    p = unpack(flat, n_in, width, hidden)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    out, hs = forward(flat, X, n_in, width, hidden)
    diff = out - T
    loss = float(np.dot(diff, diff) / B)
    g = {}
    d_out = 2.0 * diff / B                              # dL/d out
    g["b_out"] = np.array([d_out.sum()])
    g["w_out"] = hs[-1].T @ d_out
    delta = np.outer(d_out, p["w_out"]) * (1.0 - hs[-1] ** 2)   # dL/d(pre-activation of the last hidden layer)
    for k in range(hidden, 0, -1):
        inp = hs[k - 2] if k >= 2 else X
        g[f"W{k}"] = delta.T @ inp
        g[f"b{k}"] = delta.sum(axis=0)
        if k >= 2:
            delta = (delta @ p[f"W{k}"]) * (1.0 - hs[k - 2] ** 2)
    return loss, pack(g, n_in, width, hidden)


def adam_step(p, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1): returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ------------------------------------------------ labels, margin, bound steps

def richardson3(g_R: complex, g_2R: complex, g_4R: complex, R: float = 1.0) -> complex:
    """g from g_r = g + a/r + b/r^2 at r = R, 2R, 4R: the linear system in
    (g, a, b) solved as written (the result does not depend on R)."""
    rs = np.array([R, 2.0 * R, 4.0 * R])
    A = np.stack([np.ones(3), 1.0 / rs, 1.0 / rs ** 2], axis=1).astype(np.complex128)
    sol = np.linalg.solve(A, np.array([g_R, g_2R, g_4R], dtype=np.complex128))
    return complex(sol[0])


def error_labels(g, g_lim: complex, eps_floor: float):
    """eps_i = |g_i - g_lim| and log(max(eps_i, eps_floor))."""
    eps = np.array([abs(complex(v) - complex(g_lim)) for v in g])
    return eps, np.log(np.maximum(eps, eps_floor))


def margin(y, pred, quantile: float) -> float:
    """The quantile of the residuals y - pred (numpy's default), at least 0."""
    resid = np.asarray(y, np.float64) - np.asarray(pred, np.float64)
    return max(0.0, float(np.quantile(resid, quantile)))


def bound_steps(n: int, x, z, h, t: float, eps: float) -> int:
    """r with C (t/r)^2 = eps rounded up, C the bound with every term deterministic."""
    C = trotter_bound(n, x, z, h)
    return max(1, math.ceil(t * math.sqrt(C / eps)))
