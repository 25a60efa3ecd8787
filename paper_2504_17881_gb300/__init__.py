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
from ._lib import (PS_C64, PS_C128, PS_ERR_ARG, PS_ERR_TIMEOUT, PsError, ps_abi_version, ps_apply_rotations, ps_copy_state, ps_create,  # noqa: F401
                   ps_destroy, ps_device_count, ps_evolve_partial, ps_evolve_qdrift, ps_evolve_trotter,
                   ps_get_scale, ps_get_state, ps_get_state_represented, ps_measure_fma_rate, ps_get_stats, ps_ham_create, ps_ham_destroy, ps_ham_lambda, ps_last_error, ps_norm,
                   ps_overlap, ps_overlap_noalloc, ps_partial_length, ps_partial_stream, ps_plan_apply, ps_plan_create, ps_plan_describe,
                   ps_plan_destroy, ps_plan_export, ps_plan_get_info, ps_qdrift_stream, ps_reset_stats,
                   ps_set_state, ps_set_tuning, ps_batch_create, ps_batch_launch, ps_batch_wait, ps_batch_run,
                   ps_batch_get_info, ps_batch_destroy, ps_batch_describe, ps_ham_trotter_bound, ps_ham_features,
                   ps_ham_error_coefficient,
                   ps_trotter_stream, ps_trotter_sweep, PS_MLP_FEATURES, ps_mlp_create, ps_mlp_destroy,
                   ps_mlp_num_params, ps_mlp_get_params, ps_mlp_set_params, ps_mlp_get_grads, ps_mlp_set_grads,
                   ps_mlp_set_normalization, ps_mlp_get_normalization, ps_mlp_fit_normalization, ps_mlp_loss_grad,
                   ps_mlp_adam_step, ps_mlp_train, ps_mlp_predict, ps_mlp_pick_r,
                   ps_mlp_pick_r_ensemble, ps_evolve_trotter2, ps_evolve_partial2, ps_trotter2_length,
                   ps_trotter2_stream, ps_partial2_length, ps_partial2_stream, ps_ham_sort_lexicographic,
                   ps_rpe_signal, ps_rpe_estimate, ps_partial_optimize_split, ps_shard_swap_plan, ps_shard_pack,
                   ps_shard_unpack, ps_richardson3,
                   ps_ham_bound_steps, ps_trotter_error_labels, ps_mlp_margin, ps_mlp_predict_ensemble)

__all__ = [n for n in dir(_lib) if n.startswith("ps_")] + ["StateVector", "Hamiltonian", "Plan", "Batch",
                                                              "PsError", "PS_C64", "PS_C128"]


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
        """The represented state (the carried scale applied in FP64), as complex128."""
        torch = _torch()
        dst = torch.empty(self.tensor.numel(), dtype=torch.complex128).pin_memory()
        ps_get_state_represented(self.handle, dst.data_ptr())
        return dst.numpy().copy()

    def stored_numpy(self):
        """The stored amplitudes in the state's dtype (the represented state is scale() times these)."""
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

    def evolve_trotter2(self, ham: "Hamiltonian", t: float, r: int):
        ps_evolve_trotter2(self.handle, ham.handle, t, r)

    def evolve_partial2(self, ham: "Hamiltonian", L_D: int, t: float, r: int, Ns: int, seed: int):
        ps_evolve_partial2(self.handle, ham.handle, L_D, t, r, Ns, seed)

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
        self.L = len(h)
        self.handle = ps_ham_create(n, x, z, h)

    @property
    def lam(self) -> float:
        return ps_ham_lambda(self.handle)

    def trotter_stream(self, t: float, r: int):
        return ps_trotter_stream(self.handle, self.L, t, r)

    def trotter2_stream(self, t: float, r: int):
        return ps_trotter2_stream(self.handle, t, r)

    def partial2_stream(self, L_D: int, t: float, r: int, Ns: int, seed: int):
        return ps_partial2_stream(self.handle, L_D, t, r, Ns, seed)

    def sort_lexicographic(self):
        """Reorder the terms in place (upper qubits first, I < X < Y < Z)."""
        ps_ham_sort_lexicographic(self.handle)

    def trotter_bound(self, L_D: int | None = None) -> float:
        return ps_ham_trotter_bound(self.handle, self.L if L_D is None else L_D)

    def features(self, idx, amp, t: float, r: int):
        """Query features for first-order Trotter from the sparse state sum amp_i |idx_i>."""
        return ps_ham_features(self.handle, idx, amp, t, r)

    def error_coefficient(self, idx, amp):
        """(K, ||E2 psi||^2) of first-order Trotter for the sparse initial state."""
        return ps_ham_error_coefficient(self.handle, idx, amp)

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


class Batch:
    """Independent runs in one persistent launch (libps batches).

    runs: sequence of dicts with n, x, z, phi and optionally psi0 (a CUDA
    tensor, the initial state; shared by runs or not).  Every run gets its own
    output state tensor (``states[i]``); a run without psi0 evolves its state
    tensor in place (fill it before launching).
    """

    def __init__(self, runs, dtype=None, cfg=None, device=None, stream=None):
        torch = _torch()
        dtype = torch.complex64 if dtype is None else dtype
        self.ps_dtype = _ps_dtype(dtype)
        dev = device or "cuda"
        self.states = [r.get("state") if r.get("state") is not None else
                       torch.zeros(1 << int(r["n"]), dtype=dtype, device=dev) for r in runs]
        self.psi0 = [r.get("psi0") for r in runs]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.states[0].device)
        descs = []
        for r, st, p0 in zip(runs, self.states, self.psi0):
            if st.dtype != dtype or (p0 is not None and p0.dtype != dtype):
                raise ValueError("every state and psi0 must have the batch dtype")
            descs.append(dict(n=int(r["n"]), state=st.data_ptr(), psi0=p0.data_ptr() if p0 is not None else 0,
                              x=r["x"], z=r["z"], phi=r["phi"]))
        self.nruns = len(descs)
        self.handle = ps_batch_create(self.ps_dtype, descs, cfg, self.stream.cuda_stream)
        self.info = ps_batch_get_info(self.handle)

    def launch(self):
        ps_batch_launch(self.handle)

    def wait(self):
        return ps_batch_wait(self.handle, self.nruns)

    def run(self):
        """Launch, wait, and return <psi0|psi> per run (complex128 numpy array)."""
        return ps_batch_run(self.handle, self.nruns)

    def close(self):
        if getattr(self, "handle", None):
            ps_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
