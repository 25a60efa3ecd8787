"""ctypes binding of libps (include/ps.h): argument marshalling only.

Every function keeps the C name and raises ``PsError`` (with
``ps_last_error()``) when the C call returns a non-zero status.  Device
memory comes from PyTorch tensors; all state arithmetic runs in libps's CUDA
kernels.  There is no fallback: if ``libps.so`` is missing the import fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libps.so")

PS_OK, PS_ERR_ARG, PS_ERR_OOM, PS_ERR_CUDA, PS_ERR_TIMEOUT, PS_ERR_UNSUPPORTED = range(6)
PS_C64, PS_C128 = 0, 1
PS_KERNEL_TILE, PS_KERNEL_PAIR, PS_KERNEL_REDUCE, PS_KERNEL_OTHER = range(4)
KERNEL_KINDS = ("tile", "pair", "reduce", "other")


class PsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libps error {code}: {msg}")
        self.code = code


class ps_tuning(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int), ("group_bits", ctypes.c_int), ("max_window", ctypes.c_int),
                ("pair_single", ctypes.c_int), ("kernel_timing", ctypes.c_int), ("reg_groups", ctypes.c_int),
                ("seg_bits", ctypes.c_int), ("tile_threads", ctypes.c_int)]


class ps_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 4), ("kernel_ms", ctypes.c_double * 4),
                ("bytes", ctypes.c_double * 4), ("rotations", ctypes.c_uint64), ("passes", ctypes.c_uint64)]


class ps_plan_info(ctypes.Structure):
    _fields_ = [("rotations", ctypes.c_uint64), ("windows", ctypes.c_uint64), ("tile_windows", ctypes.c_uint64),
                ("pair_windows", ctypes.c_uint64), ("subwindows", ctypes.c_uint64),
                ("fast_subwindows", ctypes.c_uint64), ("max_window", ctypes.c_uint64),
                ("tile_bits", ctypes.c_int), ("group_bits", ctypes.c_int)]


class ps_run_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("state", ctypes.c_void_p), ("psi0", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("z", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("count", ctypes.c_size_t)]


class ps_batch_config(ctypes.Structure):
    _fields_ = [("lane_size", ctypes.c_int), ("tile_bits", ctypes.c_int), ("resident_bits", ctypes.c_int),
                ("single_bits", ctypes.c_int), ("use_graph", ctypes.c_int), ("wait_ms", ctypes.c_int),
                ("test_withhold", ctypes.c_int)]


class ps_batch_info(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_uint64), ("lane_runs", ctypes.c_uint64), ("single_runs", ctypes.c_uint64),
                ("resident_runs", ctypes.c_uint64), ("rotations", ctypes.c_uint64), ("windows", ctypes.c_uint64),
                ("amplitude_passes", ctypes.c_double), ("amplitude_rotations", ctypes.c_double),
                ("body_bytes", ctypes.c_uint64), ("smem_bytes", ctypes.c_uint64), ("max_lane_work", ctypes.c_double),
                ("single_work", ctypes.c_double), ("grid", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("lanes", ctypes.c_int), ("lane_size", ctypes.c_int), ("tile_bits", ctypes.c_int),
                ("resident_bits", ctypes.c_int), ("single_bits", ctypes.c_int), ("graph", ctypes.c_int)]


class ps_mlp_train_config(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


PS_MLP_FEATURES = 12

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2504_17881_gb300.build` "
                      "(or __graft_entry__.build()); there is no non-CUDA fallback")
lib = ctypes.CDLL(LIB_PATH)

_vp, _i, _u32, _u64, _sz, _d = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t,
                                ctypes.c_double)
_pp = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "ps_last_error": (ctypes.c_char_p, []),
    "ps_abi_version": (_i, []),
    "ps_device_count": (_i, []),
    "ps_create": (_i, [_i, _i, _vp, _vp, _pp]),
    "ps_destroy": (None, [_vp]),
    "ps_set_state": (_i, [_vp, _vp]),
    "ps_get_state": (_i, [_vp, _vp]),
    "ps_get_state_represented": (_i, [_vp, _vp]),
    "ps_measure_fma_rate": (_i, [_i, ctypes.POINTER(_d)]),
    "ps_copy_state": (_i, [_vp, _vp]),
    "ps_set_tuning": (_i, [_vp, ctypes.POINTER(ps_tuning)]),
    "ps_apply_rotations": (_i, [_vp, _vp, _vp, _vp, _sz]),
    "ps_plan_create": (_i, [_i, _i, _vp, _vp, _vp, _sz, ctypes.POINTER(ps_tuning), _pp]),
    "ps_plan_apply": (_i, [_vp, _vp]),
    "ps_plan_get_info": (_i, [_vp, ctypes.POINTER(ps_plan_info)]),
    "ps_plan_destroy": (None, [_vp]),
    "ps_plan_describe": (_i, [_i, _i, _vp, _vp, _vp, _sz, ctypes.POINTER(ps_tuning), ctypes.POINTER(ps_plan_info)]),
    "ps_plan_export": (_i, [_i, _i, _vp, _vp, _vp, _sz, ctypes.POINTER(ps_tuning), _sz, ctypes.POINTER(_sz), _vp, _vp,
                            _vp, _vp, _vp, _vp, _vp]),
    "ps_norm": (_i, [_vp, ctypes.POINTER(_d)]),
    "ps_get_scale": (_i, [_vp, ctypes.POINTER(_d)]),
    "ps_overlap": (_i, [_vp, _vp, _vp]),
    "ps_overlap_noalloc": (_i, [_i, _i, _vp, _vp, _vp, _vp]),
    "ps_ham_create": (_i, [_i, _sz, _vp, _vp, _vp, _pp]),
    "ps_ham_destroy": (None, [_vp]),
    "ps_ham_lambda": (_d, [_vp]),
    "ps_qdrift_stream": (_i, [_vp, _d, _u64, _u64, _u64, _u64, _vp, _vp, _vp]),
    "ps_partial_length": (_u64, [_vp, _sz, _u32, _u64]),
    "ps_partial_stream": (_i, [_vp, _sz, _d, _u32, _u64, _u64, _vp, _vp, _vp]),
    "ps_evolve_trotter": (_i, [_vp, _vp, _d, _u32]),
    "ps_evolve_qdrift": (_i, [_vp, _vp, _d, _u64, _u64]),
    "ps_evolve_partial": (_i, [_vp, _vp, _sz, _d, _u32, _u64, _u64]),
    "ps_get_stats": (_i, [_vp, ctypes.POINTER(ps_stats)]),
    "ps_reset_stats": (_i, [_vp]),
    "ps_batch_create": (_i, [_i, ctypes.POINTER(ps_run_desc), _sz, ctypes.POINTER(ps_batch_config), _vp, _pp]),
    "ps_batch_launch": (_i, [_vp]),
    "ps_batch_wait": (_i, [_vp, _vp]),
    "ps_batch_run": (_i, [_vp, _vp]),
    "ps_batch_get_info": (_i, [_vp, ctypes.POINTER(ps_batch_info)]),
    "ps_batch_destroy": (None, [_vp]),
    "ps_batch_describe": (_i, [_i, ctypes.POINTER(ps_run_desc), _sz, ctypes.POINTER(ps_batch_config), _i, _i,
                               ctypes.POINTER(ps_batch_info), _vp, _vp, _vp]),
    "ps_evolve_trotter2": (_i, [_vp, _vp, _d, _u32]),
    "ps_evolve_partial2": (_i, [_vp, _vp, _sz, _d, _u32, _u64, _u64]),
    "ps_trotter2_length": (_u64, [_vp, _u32]),
    "ps_trotter2_stream": (_i, [_vp, _d, _u32, _vp, _vp, _vp]),
    "ps_partial2_length": (_u64, [_vp, _sz, _u32, _u64]),
    "ps_partial2_stream": (_i, [_vp, _sz, _d, _u32, _u64, _u64, _vp, _vp, _vp]),
    "ps_ham_sort_lexicographic": (_i, [_vp]),
    "ps_rpe_signal": (_i, [_vp, _vp, _vp, _i, _sz, _d, _u32, _u64, _u64, _vp]),
    "ps_rpe_estimate": (_i, [_vp, _u32, _d, ctypes.POINTER(_d), _vp]),
    "ps_shard_swap_plan": (_i, [_i, _i, _i, _i, _vp, _vp, _vp, _sz, _vp, ctypes.POINTER(_sz), _vp, _vp, _vp, _vp,
                                _vp, _vp]),
    "ps_shard_pack": (_i, [_i, _i, _u64, _u64, _u64, _vp, _vp, _vp]),
    "ps_shard_unpack": (_i, [_i, _i, _u64, _u64, _u64, _vp, _vp, _vp]),
    "ps_partial_optimize_split": (_i, [_vp, _d, _d, _d, ctypes.POINTER(_sz), ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "ps_ham_trotter_bound": (_i, [_vp, _sz, ctypes.POINTER(_d)]),
    "ps_ham_bound_steps": (_i, [_vp, _d, _d, ctypes.POINTER(ctypes.c_uint32)]),
    "ps_richardson3": (_i, [_vp, _vp, _vp, _vp]),
    "ps_trotter_error_labels": (_i, [_vp, _sz, _vp, _d, _vp, _vp]),
    "ps_mlp_margin": (_i, [_vp, _vp, _sz, _d, ctypes.POINTER(_d)]),
    "ps_ham_features": (_i, [_vp, _vp, _vp, _sz, _d, _u32, _vp]),
    "ps_ham_error_coefficient": (_i, [_vp, _vp, _vp, _sz, _vp]),
    "ps_trotter_stream": (_i, [_vp, _d, _u32, _vp, _vp, _vp]),
    "ps_trotter_sweep": (_i, [_vp, _vp, _vp, _d, _d, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u64), _vp]),
    "ps_mlp_create": (_i, [_i, _u64, _vp, _pp]),
    "ps_mlp_destroy": (None, [_vp]),
    "ps_mlp_num_params": (_sz, [_vp]),
    "ps_mlp_get_params": (_i, [_vp, _vp]),
    "ps_mlp_set_params": (_i, [_vp, _vp]),
    "ps_mlp_get_grads": (_i, [_vp, _vp]),
    "ps_mlp_set_grads": (_i, [_vp, _vp]),
    "ps_mlp_set_normalization": (_i, [_vp, _vp, _vp, ctypes.c_float, ctypes.c_float]),
    "ps_mlp_get_normalization": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "ps_mlp_fit_normalization": (_i, [_vp, _vp, _vp, _sz]),
    "ps_mlp_loss_grad": (_i, [_vp, _vp, _vp, _sz, ctypes.POINTER(_d)]),
    "ps_mlp_adam_step": (_i, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "ps_mlp_train": (_i, [_vp, _vp, _vp, _sz, ctypes.POINTER(ps_mlp_train_config), _vp]),
    "ps_mlp_predict": (_i, [_vp, _vp, _sz, _vp]),
    "ps_mlp_pick_r": (_i, [_vp, _vp, _vp, _vp, _sz, _d, _d, _d, _u32, ctypes.POINTER(_u32), _vp]),
    "ps_mlp_pick_r_ensemble": (_i, [_vp, _i, _vp, _vp, _vp, _sz, _d, _d, _d, _u32, ctypes.POINTER(_u32), _vp]),
    "ps_mlp_predict_ensemble": (_i, [_vp, _i, _vp, _sz, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def ps_last_error() -> str:
    return lib.ps_last_error().decode()


def _check(rc: int):
    if rc != PS_OK:
        raise PsError(rc, ps_last_error())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64a(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _f64a(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _tuning(t) -> ps_tuning | None:
    if t is None:
        return None
    if isinstance(t, ps_tuning):
        return t
    return ps_tuning(**{k: int(v) for k, v in dict(t).items()})


def ps_abi_version() -> int:
    return lib.ps_abi_version()


def ps_device_count() -> int:
    return lib.ps_device_count()


def ps_create(n: int, dtype: int, dev_ptr: int, stream: int | None) -> int:
    h = ctypes.c_void_p()
    _check(lib.ps_create(n, dtype, ctypes.c_void_p(dev_ptr), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h.value


def ps_destroy(h: int):
    lib.ps_destroy(ctypes.c_void_p(h))


def ps_set_state(h: int, host_ptr: int):
    _check(lib.ps_set_state(ctypes.c_void_p(h), ctypes.c_void_p(host_ptr)))


def ps_get_state(h: int, host_ptr: int):
    _check(lib.ps_get_state(ctypes.c_void_p(h), ctypes.c_void_p(host_ptr)))


def ps_get_state_represented(h: int, host_ptr: int):
    _check(lib.ps_get_state_represented(ctypes.c_void_p(h), ctypes.c_void_p(host_ptr)))


def ps_measure_fma_rate(dtype: int) -> float:
    """FMA throughput of the current device in TFLOP/s (FP32 for PS_C64, FP64 for PS_C128)."""
    out = _d()
    _check(lib.ps_measure_fma_rate(dtype, ctypes.byref(out)))
    return out.value


def ps_copy_state(dst: int, src: int):
    _check(lib.ps_copy_state(ctypes.c_void_p(dst), ctypes.c_void_p(src)))


def ps_set_tuning(h: int, tuning=None):
    t = _tuning(tuning)
    _check(lib.ps_set_tuning(ctypes.c_void_p(h), ctypes.byref(t) if t is not None else None))


def ps_apply_rotations(h: int, x, z, phi):
    x, z, phi = _u64a(x), _u64a(z), _f64a(phi)
    if not (x.size == z.size == phi.size):
        raise ValueError("x, z and phi must have the same length")
    _check(lib.ps_apply_rotations(ctypes.c_void_p(h), _ptr(x), _ptr(z), _ptr(phi), x.size))


def ps_plan_create(n: int, dtype: int, x, z, phi, tuning=None) -> int:
    x, z, phi = _u64a(x), _u64a(z), _f64a(phi)
    t = _tuning(tuning)
    h = ctypes.c_void_p()
    _check(lib.ps_plan_create(n, dtype, _ptr(x), _ptr(z), _ptr(phi), x.size,
                              ctypes.byref(t) if t is not None else None, ctypes.byref(h)))
    return h.value


def ps_plan_apply(h: int, plan: int):
    _check(lib.ps_plan_apply(ctypes.c_void_p(h), ctypes.c_void_p(plan)))


def _info_dict(info: ps_plan_info) -> dict:
    return {f: getattr(info, f) for f, _ in ps_plan_info._fields_}


def ps_plan_get_info(plan: int) -> dict:
    info = ps_plan_info()
    _check(lib.ps_plan_get_info(ctypes.c_void_p(plan), ctypes.byref(info)))
    return _info_dict(info)


def ps_plan_destroy(plan: int):
    lib.ps_plan_destroy(ctypes.c_void_p(plan))


def ps_plan_describe(n: int, dtype: int, x, z, phi, tuning=None) -> dict:
    x, z, phi = _u64a(x), _u64a(z), _f64a(phi)
    t = _tuning(tuning)
    info = ps_plan_info()
    _check(lib.ps_plan_describe(n, dtype, _ptr(x), _ptr(z), _ptr(phi), x.size,
                                ctypes.byref(t) if t is not None else None, ctypes.byref(info)))
    return _info_dict(info)


def ps_plan_export(n: int, dtype: int, x, z, phi, tuning=None) -> dict:
    x, z, phi = _u64a(x), _u64a(z), _f64a(phi)
    t = _tuning(tuning)
    m = x.size
    maxw = max(1, m)
    nw = ctypes.c_size_t()
    window_of = np.zeros(m, np.uint32)
    xt = np.zeros(m, np.uint32)
    zt = np.zeros(m, np.uint32)
    kind = np.zeros(maxw, np.int32)
    c = np.zeros(maxw, np.int32)
    d = np.zeros(maxw, np.int32)
    basis = np.zeros(16 * maxw, np.uint64)
    _check(lib.ps_plan_export(n, dtype, _ptr(x), _ptr(z), _ptr(phi), m, ctypes.byref(t) if t is not None else None,
                              maxw, ctypes.byref(nw), _ptr(window_of), _ptr(xt), _ptr(zt), _ptr(kind), _ptr(c),
                              _ptr(d), _ptr(basis)))
    w = nw.value
    return {"window_of": window_of, "xt": xt, "zt": zt, "kind": kind[:w], "c": c[:w], "d": d[:w],
            "basis": basis[:16 * w].reshape(w, 16)}


def ps_norm(h: int) -> float:
    out = ctypes.c_double()
    _check(lib.ps_norm(ctypes.c_void_p(h), ctypes.byref(out)))
    return out.value


def ps_get_scale(h: int) -> float:
    out = ctypes.c_double()
    _check(lib.ps_get_scale(ctypes.c_void_p(h), ctypes.byref(out)))
    return out.value


def ps_overlap(h0: int, h: int) -> complex:
    out = (ctypes.c_double * 2)()
    _check(lib.ps_overlap(ctypes.c_void_p(h0), ctypes.c_void_p(h), out))
    return complex(out[0], out[1])


def ps_overlap_noalloc(n: int, dtype: int, psi0_ptr: int, psi_ptr: int, stream: int | None, out_ptr: int):
    """<psi0|psi> of two device buffers into 2 doubles at device address out_ptr (asynchronous)."""
    _check(lib.ps_overlap_noalloc(n, dtype, ctypes.c_void_p(psi0_ptr), ctypes.c_void_p(psi_ptr),
                                  ctypes.c_void_p(stream or 0), ctypes.c_void_p(out_ptr)))


def ps_ham_create(n: int, x, z, h) -> int:
    x, z, hh = _u64a(x), _u64a(z), _f64a(h)
    if not (x.size == z.size == hh.size):
        raise ValueError("x, z and h must have the same length")
    out = ctypes.c_void_p()
    _check(lib.ps_ham_create(n, x.size, _ptr(x), _ptr(z), _ptr(hh), ctypes.byref(out)))
    return out.value


def ps_ham_destroy(ham: int):
    lib.ps_ham_destroy(ctypes.c_void_p(ham))


def ps_ham_lambda(ham: int) -> float:
    return lib.ps_ham_lambda(ctypes.c_void_p(ham))


def ps_qdrift_stream(ham: int, t: float, N: int, seed: int, first: int, count: int):
    x = np.zeros(count, np.uint64)
    z = np.zeros(count, np.uint64)
    phi = np.zeros(count, np.float64)
    _check(lib.ps_qdrift_stream(ctypes.c_void_p(ham), t, N, seed, first, count, _ptr(x), _ptr(z), _ptr(phi)))
    return x, z, phi


def ps_partial_length(ham: int, L_D: int, r: int, Ns: int) -> int:
    return int(lib.ps_partial_length(ctypes.c_void_p(ham), L_D, r, Ns))


def ps_partial_stream(ham: int, L_D: int, t: float, r: int, Ns: int, seed: int):
    m = ps_partial_length(ham, L_D, r, Ns)
    x = np.zeros(max(m, 1), np.uint64)
    z = np.zeros(max(m, 1), np.uint64)
    phi = np.zeros(max(m, 1), np.float64)
    _check(lib.ps_partial_stream(ctypes.c_void_p(ham), L_D, t, r, Ns, seed, _ptr(x), _ptr(z), _ptr(phi)))
    return x[:m], z[:m], phi[:m]


def ps_evolve_trotter(h: int, ham: int, t: float, r: int):
    _check(lib.ps_evolve_trotter(ctypes.c_void_p(h), ctypes.c_void_p(ham), t, r))


def ps_evolve_qdrift(h: int, ham: int, t: float, N: int, seed: int):
    _check(lib.ps_evolve_qdrift(ctypes.c_void_p(h), ctypes.c_void_p(ham), t, N, seed))


def ps_evolve_partial(h: int, ham: int, L_D: int, t: float, r: int, Ns: int, seed: int):
    _check(lib.ps_evolve_partial(ctypes.c_void_p(h), ctypes.c_void_p(ham), L_D, t, r, Ns, seed))


def ps_get_stats(h: int) -> dict:
    s = ps_stats()
    _check(lib.ps_get_stats(ctypes.c_void_p(h), ctypes.byref(s)))
    return {"launches": {k: int(s.launches[i]) for i, k in enumerate(KERNEL_KINDS)},
            "kernel_ms": {k: float(s.kernel_ms[i]) for i, k in enumerate(KERNEL_KINDS)},
            "bytes": {k: float(s.bytes[i]) for i, k in enumerate(KERNEL_KINDS)},
            "rotations": int(s.rotations), "passes": int(s.passes)}


def ps_reset_stats(h: int):
    _check(lib.ps_reset_stats(ctypes.c_void_p(h)))


# ----------------------------------------------------------------- batches

def _batch_config(cfg) -> ps_batch_config | None:
    if cfg is None:
        return None
    if isinstance(cfg, ps_batch_config):
        return cfg
    return ps_batch_config(**{k: int(v) for k, v in dict(cfg).items()})


def _run_descs(runs):
    """runs: sequence of dicts n, state (device pointer or 0), psi0 (pointer or 0/None), x, z, phi.
    Returns the ctypes array and the numpy arrays it points into (kept alive by the caller)."""
    keep = []
    arr = (ps_run_desc * len(runs))()
    for i, r in enumerate(runs):
        x, z, phi = _u64a(r["x"]), _u64a(r["z"]), _f64a(r["phi"])
        if not (len(x) == len(z) == len(phi)):
            raise ValueError("x, z and phi differ in length")
        keep += [x, z, phi]
        arr[i] = ps_run_desc(int(r["n"]), r.get("state") or None, r.get("psi0") or None,
                             x.ctypes.data if len(x) else None, z.ctypes.data if len(z) else None,
                             phi.ctypes.data if len(phi) else None, len(x))
    return arr, keep


def _batch_info_dict(info: ps_batch_info) -> dict:
    return {k: getattr(info, k) for k, _ in ps_batch_info._fields_}


def ps_batch_create(dtype: int, runs, cfg=None, stream: int | None = None) -> int:
    arr, keep = _run_descs(runs)
    h = ctypes.c_void_p()
    c = _batch_config(cfg)
    _check(lib.ps_batch_create(dtype, arr, len(runs), ctypes.byref(c) if c is not None else None,
                               ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    del keep
    return h.value


def ps_batch_launch(b: int):
    _check(lib.ps_batch_launch(ctypes.c_void_p(b)))


def ps_batch_wait(b: int, nruns: int | None = None):
    """Wait; returns the overlaps as a complex128 array when nruns is given."""
    if nruns is None:
        _check(lib.ps_batch_wait(ctypes.c_void_p(b), None))
        return None
    out = np.zeros(2 * nruns, dtype=np.float64)
    _check(lib.ps_batch_wait(ctypes.c_void_p(b), _ptr(out)))
    return out[0::2] + 1j * out[1::2]


def ps_batch_run(b: int, nruns: int):
    out = np.zeros(2 * nruns, dtype=np.float64)
    _check(lib.ps_batch_run(ctypes.c_void_p(b), _ptr(out)))
    return out[0::2] + 1j * out[1::2]


def ps_batch_get_info(b: int) -> dict:
    info = ps_batch_info()
    _check(lib.ps_batch_get_info(ctypes.c_void_p(b), ctypes.byref(info)))
    return _batch_info_dict(info)


def ps_batch_destroy(b: int):
    lib.ps_batch_destroy(ctypes.c_void_p(b))


def ps_batch_describe(dtype: int, runs, cfg=None, num_sms: int = 152, ctas_per_sm: int = 3) -> dict:
    """Host-only schedule of a batch (no GPU): info plus per-run lane, tile bits and windows."""
    arr, keep = _run_descs(runs)
    info = ps_batch_info()
    lane = np.zeros(len(runs), dtype=np.int32)
    tb = np.zeros(len(runs), dtype=np.int32)
    nw = np.zeros(len(runs), dtype=np.uint64)
    c = _batch_config(cfg)
    _check(lib.ps_batch_describe(dtype, arr, len(runs), ctypes.byref(c) if c is not None else None, num_sms,
                                 ctas_per_sm, ctypes.byref(info), _ptr(lane), _ptr(tb), _ptr(nw)))
    del keep
    d = _batch_info_dict(info)
    d.update(lane_of=lane, tile_bits_of=tb, windows_of=nw)
    return d


# ------------------------------------------------------ learned step choice

def ps_ham_trotter_bound(ham: int, L_D: int) -> float:
    out = _d()
    _check(lib.ps_ham_trotter_bound(ctypes.c_void_p(ham), L_D, ctypes.byref(out)))
    return out.value


def ps_ham_bound_steps(ham: int, t: float, eps: float) -> int:
    out = ctypes.c_uint32()
    _check(lib.ps_ham_bound_steps(ctypes.c_void_p(ham), float(t), float(eps), ctypes.byref(out)))
    return int(out.value)


def _c2(g) -> np.ndarray:
    return np.array([complex(g).real, complex(g).imag], dtype=np.float64)


def ps_richardson3(g_R: complex, g_2R: complex, g_4R: complex) -> complex:
    a, b, c = _c2(g_R), _c2(g_2R), _c2(g_4R)
    out = np.zeros(2)
    _check(lib.ps_richardson3(_ptr(a), _ptr(b), _ptr(c), _ptr(out)))
    return complex(out[0], out[1])


def ps_trotter_error_labels(g, g_lim: complex, eps_floor: float):
    """(eps, log eps as float32) of overlaps g against the limit g_lim."""
    gg = np.ascontiguousarray(np.asarray(g, dtype=np.complex128)).view(np.float64)
    n = gg.size // 2
    lim = _c2(g_lim)
    eps = np.zeros(n)
    lg = np.zeros(n, np.float32)
    _check(lib.ps_trotter_error_labels(_ptr(gg), n, _ptr(lim), float(eps_floor), _ptr(eps), _ptr(lg)))
    return eps, lg


def ps_mlp_margin(y, pred, quantile: float) -> float:
    y = np.ascontiguousarray(np.asarray(y, np.float32))
    p = np.ascontiguousarray(np.asarray(pred, np.float32))
    if y.size != p.size:
        raise ValueError("y and pred differ in length")
    out = _d()
    _check(lib.ps_mlp_margin(_ptr(y), _ptr(p), y.size, float(quantile), ctypes.byref(out)))
    return out.value


def _sparse(idx, amp):
    idx = _u64a(idx)
    a = np.asarray(amp, dtype=np.complex128)
    ri = np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1).reshape(-1))
    if len(idx) != len(a):
        raise ValueError("idx and amp differ in length")
    return idx, ri


def ps_ham_features(ham: int, idx, amp, t: float, r: int) -> np.ndarray:
    """Features of the query (t, r) from the sparse initial state sum amp_i |idx_i>."""
    i, a = _sparse(idx, amp)
    out = np.zeros(PS_MLP_FEATURES, dtype=np.float32)
    _check(lib.ps_ham_features(ctypes.c_void_p(ham), _ptr(i), _ptr(a), len(i), t, r, _ptr(out)))
    return out


def ps_ham_error_coefficient(ham: int, idx, amp):
    """(K, ||E2 psi||^2) for the sparse state sum amp_i |idx_i>."""
    i, a = _sparse(idx, amp)
    out = np.zeros(3, dtype=np.float64)
    _check(lib.ps_ham_error_coefficient(ctypes.c_void_p(ham), _ptr(i), _ptr(a), len(i), _ptr(out)))
    return complex(out[0], out[1]), float(out[2])


def ps_trotter_stream(ham: int, L: int, t: float, r: int):
    m = L * r
    x = np.zeros(m, dtype=np.uint64)
    z = np.zeros(m, dtype=np.uint64)
    phi = np.zeros(m, dtype=np.float64)
    _check(lib.ps_trotter_stream(ctypes.c_void_p(ham), t, r, _ptr(x), _ptr(z), _ptr(phi)))
    return x, z, phi


def ps_trotter_sweep(work: int, psi0: int, ham: int, t: float, eps: float, r_max: int):
    """Returns (r, rotations applied, g_r)."""
    r = _u32()
    rot = _u64()
    g = np.zeros(2, dtype=np.float64)
    _check(lib.ps_trotter_sweep(ctypes.c_void_p(work), ctypes.c_void_p(psi0), ctypes.c_void_p(ham), t, eps, r_max,
                                ctypes.byref(r), ctypes.byref(rot), _ptr(g)))
    return int(r.value), int(rot.value), complex(g[0], g[1])


def ps_mlp_create(n_in: int, seed: int, stream: int | None) -> int:
    h = ctypes.c_void_p()
    _check(lib.ps_mlp_create(n_in, seed, ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h.value


def ps_mlp_destroy(m: int):
    lib.ps_mlp_destroy(ctypes.c_void_p(m))


def ps_mlp_num_params(m: int) -> int:
    return int(lib.ps_mlp_num_params(ctypes.c_void_p(m)))


def ps_mlp_get_params(m: int) -> np.ndarray:
    out = np.zeros(ps_mlp_num_params(m), dtype=np.float32)
    _check(lib.ps_mlp_get_params(ctypes.c_void_p(m), _ptr(out)))
    return out


def ps_mlp_set_params(m: int, p):
    a = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
    if a.size != ps_mlp_num_params(m):
        raise ValueError("wrong number of parameters")
    _check(lib.ps_mlp_set_params(ctypes.c_void_p(m), _ptr(a)))


def ps_mlp_get_grads(m: int) -> np.ndarray:
    out = np.zeros(ps_mlp_num_params(m), dtype=np.float32)
    _check(lib.ps_mlp_get_grads(ctypes.c_void_p(m), _ptr(out)))
    return out


def ps_mlp_set_grads(m: int, g):
    g = np.ascontiguousarray(np.asarray(g, np.float32))
    _check(lib.ps_mlp_set_grads(ctypes.c_void_p(m), _ptr(g)))


def ps_mlp_set_normalization(m: int, mu, sigma, y_mu: float, y_sigma: float):
    mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float32))
    sigma = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32))
    _check(lib.ps_mlp_set_normalization(ctypes.c_void_p(m), _ptr(mu), _ptr(sigma), y_mu, y_sigma))


def ps_mlp_get_normalization(m: int, n_in: int):
    mu = np.zeros(n_in, dtype=np.float32)
    sigma = np.zeros(n_in, dtype=np.float32)
    ym = ctypes.c_float()
    ys = ctypes.c_float()
    _check(lib.ps_mlp_get_normalization(ctypes.c_void_p(m), _ptr(mu), _ptr(sigma), ctypes.byref(ym),
                                        ctypes.byref(ys)))
    return mu, sigma, ym.value, ys.value


def ps_mlp_fit_normalization(m: int, x, y):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
    _check(lib.ps_mlp_fit_normalization(ctypes.c_void_p(m), _ptr(x), _ptr(y), len(y)))


def ps_mlp_loss_grad(m: int, x_dev: int, y_dev: int, rows: int) -> float:
    out = _d()
    _check(lib.ps_mlp_loss_grad(ctypes.c_void_p(m), ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), rows,
                                ctypes.byref(out)))
    return out.value


def ps_mlp_adam_step(m: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    _check(lib.ps_mlp_adam_step(ctypes.c_void_p(m), lr, beta1, beta2, eps))


def ps_mlp_train(m: int, x_dev: int, y_dev: int, rows: int, cfg=None) -> np.ndarray:
    c = cfg if isinstance(cfg, ps_mlp_train_config) else ps_mlp_train_config(**(cfg or {}))
    epochs = c.epochs or 200
    out = np.zeros(epochs, dtype=np.float32)
    _check(lib.ps_mlp_train(ctypes.c_void_p(m), ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), rows,
                            ctypes.byref(c), _ptr(out)))
    return out


def ps_mlp_predict(m: int, x_dev: int, rows: int, y_dev: int):
    _check(lib.ps_mlp_predict(ctypes.c_void_p(m), ctypes.c_void_p(x_dev), rows, ctypes.c_void_p(y_dev)))


def ps_mlp_pick_r(m: int, ham: int, idx, amp, t: float, eps: float, margin: float, r_max: int):
    """Returns (r, predictions for r = 1..r_max); r = 0 when none qualifies."""
    i, a = _sparse(idx, amp)
    r = _u32()
    pred = np.zeros(r_max, dtype=np.float32)
    rc = lib.ps_mlp_pick_r(ctypes.c_void_p(m), ctypes.c_void_p(ham), _ptr(i), _ptr(a), len(i), t, eps, margin, r_max,
                           ctypes.byref(r), _ptr(pred))
    if rc not in (PS_OK, PS_ERR_UNSUPPORTED):
        _check(rc)
    return int(r.value), pred


def ps_mlp_predict_ensemble(nets, x_dev_ptr: int, rows: int) -> np.ndarray:
    """Mean of the members' predictions for `rows` device feature rows (host float32)."""
    arr = (ctypes.c_void_p * len(nets))(*nets)
    out = np.zeros(rows, dtype=np.float32)
    _check(lib.ps_mlp_predict_ensemble(arr, len(nets), ctypes.c_void_p(x_dev_ptr), rows, _ptr(out)))
    return out


def ps_mlp_pick_r_ensemble(nets, ham: int, idx, amp, t: float, eps: float, margin: float, r_max: int):
    """Returns (r, mean predictions for r = 1..r_max); r = 0 when none qualifies."""
    i, a = _sparse(idx, amp)
    arr = (ctypes.c_void_p * len(nets))(*nets)
    r = _u32()
    pred = np.zeros(r_max, dtype=np.float32)
    rc = lib.ps_mlp_pick_r_ensemble(arr, len(nets), ctypes.c_void_p(ham), _ptr(i), _ptr(a), len(i), t, eps, margin,
                                    r_max, ctypes.byref(r), _ptr(pred))
    if rc not in (PS_OK, PS_ERR_UNSUPPORTED):
        _check(rc)
    return int(r.value), pred


# ------------------------------------------------------------- second order

def ps_evolve_trotter2(h: int, ham: int, t: float, r: int):
    _check(lib.ps_evolve_trotter2(ctypes.c_void_p(h), ctypes.c_void_p(ham), t, r))


def ps_evolve_partial2(h: int, ham: int, L_D: int, t: float, r: int, Ns: int, seed: int):
    _check(lib.ps_evolve_partial2(ctypes.c_void_p(h), ctypes.c_void_p(ham), L_D, t, r, Ns, seed))


def ps_trotter2_length(ham: int, r: int) -> int:
    return int(lib.ps_trotter2_length(ctypes.c_void_p(ham), r))


def ps_trotter2_stream(ham: int, t: float, r: int):
    m = ps_trotter2_length(ham, r)
    x = np.zeros(m, dtype=np.uint64)
    z = np.zeros(m, dtype=np.uint64)
    phi = np.zeros(m, dtype=np.float64)
    _check(lib.ps_trotter2_stream(ctypes.c_void_p(ham), t, r, _ptr(x), _ptr(z), _ptr(phi)))
    return x, z, phi


def ps_partial2_length(ham: int, L_D: int, r: int, Ns: int) -> int:
    return int(lib.ps_partial2_length(ctypes.c_void_p(ham), L_D, r, Ns))


def ps_partial2_stream(ham: int, L_D: int, t: float, r: int, Ns: int, seed: int):
    m = ps_partial2_length(ham, L_D, r, Ns)
    x = np.zeros(m, dtype=np.uint64)
    z = np.zeros(m, dtype=np.uint64)
    phi = np.zeros(m, dtype=np.float64)
    _check(lib.ps_partial2_stream(ctypes.c_void_p(ham), L_D, t, r, Ns, seed, _ptr(x), _ptr(z), _ptr(phi)))
    return x, z, phi


def ps_ham_sort_lexicographic(ham: int):
    _check(lib.ps_ham_sort_lexicographic(ctypes.c_void_p(ham)))


def ps_rpe_signal(work: int, psi0: int, ham: int, order: int, L_D: int, delta: float, M: int, Ns: int = 0,
                  seed: int = 0) -> np.ndarray:
    """Z_m, m = 0..M, as a complex128 array."""
    out = np.zeros(2 * (M + 1), dtype=np.float64)
    _check(lib.ps_rpe_signal(ctypes.c_void_p(work), ctypes.c_void_p(psi0), ctypes.c_void_p(ham), order, L_D, delta,
                             M, Ns, seed, _ptr(out)))
    return out[0::2] + 1j * out[1::2]


def ps_rpe_estimate(Z, delta: float):
    """(energy, per-round phase estimates) from the complex signal Z_0..Z_M."""
    Z = np.asarray(Z, dtype=np.complex128).ravel()
    if Z.size == 0:
        raise ValueError("the signal needs at least Z_0")
    buf = np.empty(2 * Z.size, dtype=np.float64)
    buf[0::2] = Z.real
    buf[1::2] = Z.imag
    theta = np.zeros(Z.size, dtype=np.float64)
    e = _d()
    _check(lib.ps_rpe_estimate(_ptr(buf), Z.size - 1, delta, ctypes.byref(e), _ptr(theta)))
    return e.value, theta


def ps_partial_optimize_split(ham: int, eps: float, a: float, b: float):
    """(L_D, delta, cost) minimising the partially randomised cost model."""
    L_D = _sz()
    d = _d()
    c = _d()
    _check(lib.ps_partial_optimize_split(ctypes.c_void_p(ham), eps, a, b, ctypes.byref(L_D), ctypes.byref(d),
                                         ctypes.byref(c)))
    return int(L_D.value), d.value, c.value


def ps_shard_swap_plan(n: int, m: int, k_max: int, rank: int, x, z, phi, layout=None):
    """Steps of the qubit-swap schedule for one rank of 2^m:
    (steps, layout) with steps a list of ("exchange", rank-position mask, slab-position mask)
    and ("window", local x, local z, local phi); layout the final one."""
    x, z, phi = _u64a(x), _u64a(z), _f64a(phi)
    cnt = len(phi)
    lay = np.arange(n, dtype=np.int32) if layout is None else np.array(layout, dtype=np.int32, copy=True)
    ns = _sz()
    kind = np.zeros(max(2 * cnt, 1), dtype=np.int32)
    a = np.zeros(max(2 * cnt, 1), dtype=np.uint64)
    b = np.zeros(max(2 * cnt, 1), dtype=np.uint64)
    xo = np.zeros(max(cnt, 1), dtype=np.uint64)
    zo = np.zeros(max(cnt, 1), dtype=np.uint64)
    po = np.zeros(max(cnt, 1), dtype=np.float64)
    _check(lib.ps_shard_swap_plan(n, m, k_max, rank, _ptr(x), _ptr(z), _ptr(phi), cnt, _ptr(lay), ctypes.byref(ns),
                                  _ptr(kind), _ptr(a), _ptr(b), _ptr(xo), _ptr(zo), _ptr(po)))
    steps = []
    for t in range(ns.value):
        if kind[t] == 1:
            steps.append(("exchange", int(a[t]), int(b[t])))
        else:
            lo, hi = int(a[t]), int(b[t])
            steps.append(("window", xo[lo:hi].copy(), zo[lo:hi].copy(), po[lo:hi].copy()))
    return steps, lay


def ps_shard_pack(s: int, dtype: int, lmask: int, first: int, count: int, slab_ptr: int, out_ptr: int,
                  stream: int | None):
    _check(lib.ps_shard_pack(s, dtype, lmask, first, count, ctypes.c_void_p(slab_ptr), ctypes.c_void_p(out_ptr),
                             ctypes.c_void_p(stream or 0)))


def ps_shard_unpack(s: int, dtype: int, lmask: int, first: int, count: int, in_ptr: int, slab_ptr: int,
                    stream: int | None):
    _check(lib.ps_shard_unpack(s, dtype, lmask, first, count, ctypes.c_void_p(in_ptr), ctypes.c_void_p(slab_ptr),
                               ctypes.c_void_p(stream or 0)))

