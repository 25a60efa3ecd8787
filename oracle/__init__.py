"""Plain CPU complex128 oracle (test infrastructure, not product code).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` -- a direct,
slow transcription of the definitions in the paper (Results, "Software
implementation"; Methods, "Hamiltonian simulation" and "Data analysis";
Supplementary Methods, "Pauli-string bit representation") -- through ctypes.
It shares no code with the CUDA library in ``paper_2504_17881_gb300``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (no fused multiply-adds) into ``liboracle.so``,
    with OpenMP when the compiler has it (the pragmas are ignored otherwise)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fcx-limited-range", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u64, f64, sz, vp = ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
    i32, u32 = ctypes.c_int, ctypes.c_uint32
    sig = {
        "or_pauli_from_string": (i32, [ctypes.c_char_p, vp, vp]),
        "or_pauli_phase": (None, [u64, u64, u64, vp]),
        "or_rotate": (i32, [i32, vp, vp, u64, u64, f64]),
        "or_apply": (i32, [i32, vp, vp, vp, vp, vp, sz]),
        "or_overlap": (None, [i32, vp, vp, vp]),
        "or_norm2": (f64, [i32, vp]),
        "or_trotter": (i32, [i32, vp, vp, sz, vp, vp, vp, f64, u32]),
        "or_splitmix64_next": (u64, [vp]),
        "or_qdrift_indices": (i32, [sz, vp, u64, u64, u64, vp]),
        "or_qdrift": (i32, [i32, vp, vp, sz, vp, vp, vp, f64, u64, u64]),
        "or_partial_split": (i32, [sz, vp, sz, vp]),
        "or_partial": (i32, [i32, vp, vp, sz, vp, vp, vp, sz, f64, u32, u64, u64]),
        "or_trotter2": (i32, [i32, vp, vp, sz, vp, vp, vp, f64, u32]),
        "or_partial2": (i32, [i32, vp, vp, sz, vp, vp, vp, sz, f64, u32, u64, u64]),
        "or_amplitudes_sparse": (i32, [i32, sz, vp, vp, vp, vp, vp, sz, sz, vp, vp]),
    }
    sig["or_set_threads"] = (i32, [i32])
    sig["or_has_openmp"] = (i32, [])
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    lib.or_set_threads(1)
    _lib = lib
    return lib


def set_threads(nthreads: int) -> int:
    """Threads of the oracle's element loops (1 by default); returns the number in effect."""
    return int(_load().or_set_threads(int(nthreads)))


def has_openmp() -> bool:
    return bool(_load().or_has_openmp())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _state(psi) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128)).copy()
    n = int(a.size).bit_length() - 1
    if a.ndim != 1 or a.size != (1 << n):
        raise ValueError("state must be a 1-D array of 2^n amplitudes")
    return a


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def pauli_from_string(s: str) -> tuple[int, int]:
    x = np.zeros(1, np.uint64)
    z = np.zeros(1, np.uint64)
    _check(_load().or_pauli_from_string(s.encode(), _p(x), _p(z)), "pauli_from_string")
    return int(x[0]), int(z[0])


def pauli_phase(x: int, z: int, k: int) -> complex:
    out = np.zeros(2)
    _load().or_pauli_phase(x, z, k, _p(out))
    return complex(out[0], out[1])


def apply(psi, x, z, phi) -> np.ndarray:
    """Return exp(i phi_{m-1} P_{m-1}) ... exp(i phi_0 P_0) psi (rotation 0 first)."""
    a = _state(psi)
    n = a.size.bit_length() - 1
    x, z, phi = _u64(x), _u64(z), _f64(phi)
    tmp = np.empty_like(a)
    _check(_load().or_apply(n, _p(a), _p(tmp), _p(x), _p(z), _p(phi), x.size), "apply")
    return a


def apply_inplace(psi: np.ndarray, tmp: np.ndarray, x, z, phi) -> None:
    """or_apply on caller-owned complex128 buffers (psi updated in place, tmp scratch)."""
    if psi.dtype != np.complex128 or tmp.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise ValueError("psi and tmp must be contiguous complex128 arrays")
    n = psi.size.bit_length() - 1
    x, z, phi = _u64(x), _u64(z), _f64(phi)
    _check(_load().or_apply(n, _p(psi), _p(tmp), _p(x), _p(z), _p(phi), x.size), "apply")


def overlap(a, b) -> complex:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    out = np.zeros(2)
    _load().or_overlap(a.size.bit_length() - 1, _p(a), _p(b), _p(out))
    return complex(out[0], out[1])


def norm2(a) -> float:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return float(_load().or_norm2(a.size.bit_length() - 1, _p(a)))


def trotter(psi, x, z, h, t: float, r: int) -> np.ndarray:
    a = _state(psi)
    x, z, h = _u64(x), _u64(z), _f64(h)
    tmp = np.empty_like(a)
    _check(_load().or_trotter(a.size.bit_length() - 1, _p(a), _p(tmp), x.size, _p(x), _p(z), _p(h),
                              float(t), int(r)), "trotter")
    return a


def trotter2(psi, x, z, h, t: float, r: int) -> np.ndarray:
    """Second-order symmetric product formula (each factor written out)."""
    a = _state(psi)
    x, z, h = _u64(x), _u64(z), _f64(h)
    tmp = np.empty_like(a)
    _check(_load().or_trotter2(a.size.bit_length() - 1, _p(a), _p(tmp), x.size, _p(x), _p(z), _p(h),
                               float(t), int(r)), "trotter2")
    return a


def lexicographic_order(n: int, x, z) -> list[int]:
    """Term indices sorted by their Pauli strings read from qubit n down to
    qubit 1, letters ordered I < X < Y < Z (ties keep input order)."""
    letter = {(0, 0): "0", (1, 0): "1", (1, 1): "2", (0, 1): "3"}

    def key(l):
        xv, zv = int(x[l]), int(z[l])
        return "".join(letter[((xv >> q) & 1, (zv >> q) & 1)] for q in reversed(range(n)))

    return sorted(range(len(x)), key=lambda l: (key(l), l))


def splitmix64(seed: int, count: int) -> np.ndarray:
    st = np.array([seed], dtype=np.uint64)
    lib = _load()
    return np.array([lib.or_splitmix64_next(_p(st)) for _ in range(count)], dtype=np.uint64)


def qdrift_indices(h, seed: int, first: int, count: int) -> np.ndarray:
    h = _f64(h)
    out = np.zeros(count, np.uint64)
    _check(_load().or_qdrift_indices(h.size, _p(h), seed, first, count, _p(out)), "qdrift_indices")
    return out


def qdrift(psi, x, z, h, t: float, N: int, seed: int) -> np.ndarray:
    a = _state(psi)
    x, z, h = _u64(x), _u64(z), _f64(h)
    tmp = np.empty_like(a)
    _check(_load().or_qdrift(a.size.bit_length() - 1, _p(a), _p(tmp), x.size, _p(x), _p(z), _p(h),
                             float(t), int(N), int(seed)), "qdrift")
    return a


def partial_split(h, L_D: int) -> np.ndarray:
    h = _f64(h)
    out = np.zeros(h.size, np.uint8)
    _check(_load().or_partial_split(h.size, _p(h), L_D, _p(out)), "partial_split")
    return out.astype(bool)


def partial(psi, x, z, h, L_D: int, t: float, r: int, Ns: int, seed: int) -> np.ndarray:
    a = _state(psi)
    x, z, h = _u64(x), _u64(z), _f64(h)
    tmp = np.empty_like(a)
    _check(_load().or_partial(a.size.bit_length() - 1, _p(a), _p(tmp), x.size, _p(x), _p(z), _p(h),
                              int(L_D), float(t), int(r), int(Ns), int(seed)), "partial")
    return a


def partial2(psi, x, z, h, L_D: int, t: float, r: int, Ns: int, seed: int) -> np.ndarray:
    """Second-order partially randomised steps (deterministic halves around 2 Ns draws)."""
    a = _state(psi)
    x, z, h = _u64(x), _u64(z), _f64(h)
    tmp = np.empty_like(a)
    _check(_load().or_partial2(a.size.bit_length() - 1, _p(a), _p(tmp), x.size, _p(x), _p(z), _p(h),
                               int(L_D), float(t), int(r), int(Ns), int(seed)), "partial2")
    return a


def amplitudes_sparse(n: int, idx0, amp0, x, z, phi, ks) -> np.ndarray:
    """<k|U|psi0> for each k in ks, psi0 given by basis indices idx0 and complex amp0."""
    idx0 = _u64(idx0)
    amp0 = np.ascontiguousarray(np.asarray(amp0, dtype=np.complex128)).view(np.float64)
    x, z, phi, ks = _u64(x), _u64(z), _f64(phi), _u64(ks)
    out = np.zeros(2 * ks.size)
    _check(_load().or_amplitudes_sparse(n, idx0.size, _p(idx0), _p(amp0), _p(x), _p(z), _p(phi),
                                        x.size, ks.size, _p(ks), _p(out)), "amplitudes_sparse")
    return out.view(np.complex128)


def _one_norm(h) -> float:
    """Sum of |h| in term order, one FP64 addition at a time (as the C sampler's cdf)."""
    lam = 0.0
    for v in h:
        lam += abs(float(v))
    return lam


def qdrift_stream(x, z, h, t: float, N: int, seed: int, first: int = 0, count: int | None = None):
    """Rotations first .. first + count - 1 of the qDRIFT run or_qdrift applies:
    draw j picks term l with probability |h_l| / lambda (the oracle's own
    sampler) and rotates by sgn(h_l) lambda t / N.  Returns (x, z, phi)."""
    x, z, h = _u64(x), _u64(z), _f64(h)
    count = N - first if count is None else count
    idx = qdrift_indices(h, seed, first, count).astype(np.int64)
    tau = _one_norm(h) * t / N
    return x[idx].copy(), z[idx].copy(), np.where(h[idx] > 0.0, tau, -tau)


def partial_stream(x, z, h, L_D: int, t: float, r: int, Ns: int, seed: int):
    """The rotations or_partial applies: r steps of delta = t / r, each the
    terms of H_D in input order with angle delta h_l, then Ns draws from H_R
    (one SplitMix64 stream through all steps) with angle sgn(h) lambda_R delta / Ns.
    Returns (x, z, phi)."""
    x, z, h = _u64(x), _u64(z), _f64(h)
    is_det = partial_split(h, L_D)
    det = np.flatnonzero(is_det)
    rest = np.flatnonzero(~is_det)
    delta = t / r
    lam_R = _one_norm(h[rest])
    sample = rest.size > 0 and Ns > 0 and lam_R > 0.0
    tau = lam_R * delta / Ns if sample else 0.0
    xs, zs, ph = [], [], []
    for step in range(r):
        xs.append(x[det])
        zs.append(z[det])
        ph.append(delta * h[det])
        if sample:
            m = qdrift_indices(h[rest], seed, step * Ns, Ns).astype(np.int64)
            ls = rest[m]
            xs.append(x[ls])
            zs.append(z[ls])
            ph.append(np.where(h[ls] > 0.0, tau, -tau))
    return np.concatenate(xs), np.concatenate(zs), np.concatenate(ph)
