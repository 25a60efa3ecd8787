"""GB300-native Pauli-rotation state-vector simulator (libps + thin binding).

The hot path of Miller et al., "phase2: Full-State Vector Simulation of
Quantum Time Evolution at Scale" (arXiv:2504.17881): sequences of Pauli
rotations exp(i phi P) on a full 2^n state vector, driven by first-order
Trotter, qDRIFT and the partially randomised product formula, ending in the
overlap <psi|exp(itH)|psi>.  All state arithmetic runs in libps's sm_103a
kernels; this package only marshals arguments.  PyTorch provides device
memory and streams.
"""
from __future__ import annotations

from . import _lib
from ._lib import (PS_C64, PS_C128, PsError, ps_abi_version, ps_apply_rotations, ps_copy_state, ps_create,  # noqa: F401
                   ps_destroy, ps_device_count, ps_evolve_partial, ps_evolve_qdrift, ps_evolve_trotter,
                   ps_get_scale, ps_get_state, ps_get_stats, ps_ham_create, ps_ham_destroy, ps_ham_lambda, ps_last_error, ps_norm,
                   ps_overlap, ps_overlap_noalloc, ps_partial_length, ps_partial_stream, ps_plan_apply, ps_plan_create, ps_plan_describe,
                   ps_plan_destroy, ps_plan_export, ps_plan_get_info, ps_qdrift_stream, ps_reset_stats,
                   ps_set_state, ps_set_tuning)

__all__ = [n for n in dir(_lib) if n.startswith("ps_")] + ["StateVector", "Hamiltonian", "Plan", "PsError",
                                                              "PS_C64", "PS_C128"]


def _torch():
    import torch
    return torch


def _ps_dtype(torch_dtype) -> int:
    torch = _torch()
    if torch_dtype == torch.complex64:
        return PS_C64
    if torch_dtype == torch.complex128:
        return PS_C128
    raise ValueError("state dtype must be torch.complex64 or torch.complex128")


class StateVector:
    """A 2^n state on a CUDA device: a torch tensor plus its libps handle."""

    def __init__(self, n: int, dtype=None, device=None, stream=None, tensor=None):
        torch = _torch()
        if tensor is None:
            dtype = torch.complex64 if dtype is None else dtype
            tensor = torch.empty(1 << n, dtype=dtype, device=device or "cuda")
        if tensor.numel() != (1 << n) or not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("tensor must be a contiguous CUDA tensor of 2^n amplitudes")
        self.n = n
        self.tensor = tensor
        self.dtype = _ps_dtype(tensor.dtype)
        self.stream = stream if stream is not None else torch.cuda.current_stream(tensor.device)
        self.handle = ps_create(n, self.dtype, tensor.data_ptr(), self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            ps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, **kw):
        ps_set_tuning(self.handle, kw or None)

    def load(self, host_array):
        """Copy a host array of 2^n amplitudes into the state (synchronous)."""
        torch = _torch()
        src = torch.as_tensor(host_array).to(self.tensor.dtype).contiguous().pin_memory()
        ps_set_state(self.handle, src.data_ptr())
        self.stream.synchronize()

    def to_numpy(self):
        """Stored amplitudes (the represented state is scale() times these)."""
        torch = _torch()
        dst = torch.empty(self.tensor.numel(), dtype=self.tensor.dtype).pin_memory()
        ps_get_state(self.handle, dst.data_ptr())
        return dst.numpy().copy()

    def scale(self) -> float:
        return ps_get_scale(self.handle)

    def copy_from(self, other: "StateVector"):
        ps_copy_state(self.handle, other.handle)

    def apply_rotations(self, x, z, phi):
        ps_apply_rotations(self.handle, x, z, phi)

    def apply_plan(self, plan: "Plan"):
        ps_plan_apply(self.handle, plan.handle)

    def evolve_trotter(self, ham: "Hamiltonian", t: float, r: int):
        ps_evolve_trotter(self.handle, ham.handle, t, r)

    def evolve_qdrift(self, ham: "Hamiltonian", t: float, N: int, seed: int):
        ps_evolve_qdrift(self.handle, ham.handle, t, N, seed)

    def evolve_partial(self, ham: "Hamiltonian", L_D: int, t: float, r: int, Ns: int, seed: int):
        ps_evolve_partial(self.handle, ham.handle, L_D, t, r, Ns, seed)

    def norm2(self) -> float:
        return ps_norm(self.handle)

    def overlap(self, psi0: "StateVector") -> complex:
        """<psi0|self>."""
        return ps_overlap(psi0.handle, self.handle)

    def stats(self) -> dict:
        return ps_get_stats(self.handle)


class Hamiltonian:
    """Term list H = sum_l h_l P_l held by libps (host memory)."""

    def __init__(self, n: int, x, z, h):
        self.n = n
        self.handle = ps_ham_create(n, x, z, h)

    @property
    def lam(self) -> float:
        return ps_ham_lambda(self.handle)

    def qdrift_stream(self, t: float, N: int, seed: int, first: int = 0, count: int | None = None):
        return ps_qdrift_stream(self.handle, t, N, seed, first, N - first if count is None else count)

    def partial_stream(self, L_D: int, t: float, r: int, Ns: int, seed: int):
        return ps_partial_stream(self.handle, L_D, t, r, Ns, seed)

    def close(self):
        if getattr(self, "handle", None):
            ps_ham_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A rotation sequence scheduled once and resident on the current device."""

    def __init__(self, n: int, dtype: int, x, z, phi, tuning=None):
        self.handle = ps_plan_create(n, dtype, x, z, phi, tuning)
        self.info = ps_plan_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            ps_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
