"""Learned Trotter step choice (the network, its training data, the r pick).

A step count r for first-order Trotter to time t is good when the error of
the overlap, eps(H, t, r) = |g_r(t) - g(t)| with g(t) = <psi|exp(itH)|psi>,
is at most the target (the paper works at eps = 0.001, Methods).  The plain
way to find it is the doubling sweep (``ps_trotter_sweep``): r = 1, 2, 4, ...
until 2 |g_r - g_2r| <= eps, paying for every run on the way.  The learned
way predicts log eps(H, t, r) from twelve features of the query
(``ps_ham_features``) with a small network trained on errors this simulator
measures, and runs only the r it picks; the sweep stays as the fallback and
the judge.

Training rows come from the batched engine: for every Hamiltonian and time,
Trotter runs at r = 1, 2, ..., 64 and at 128 share one persistent launch with
many other (H, t) pairs; g is extrapolated from r = 32, 64, 128 by
three-point Richardson extrapolation in 1/r (first order: g_r = g + a/r +
b/r^2 + ...), and eps = |g_r - g|.

All arithmetic runs in libps (features and bound on the host in C++, the
network's forward, backward and Adam steps in CUDA kernels); this module
arranges the calls.
"""
from __future__ import annotations

import numpy as np

from . import PS_MLP_FEATURES, Batch, Hamiltonian, StateVector, _lib, ps_trotter_sweep

TIMES16 = tuple(0.1 * 2.0 ** (j / 3.0) for j in range(16))  # 0.1 .. 3.2
R_VALUES = (1, 2, 4, 8, 16, 32, 64)
R_EXTRA = 128
EPS_FLOOR = 1e-12


def richardson3(g32: complex, g64: complex, g128: complex) -> complex:
    """The r -> infinity limit of g_r = g + a/r + b/r^2 from r = R, 2R, 4R (ps_richardson3)."""
    return _lib.ps_richardson3(g32, g64, g128)


def initial_state(n: int, seed: int, dtype, device, min_distance: int = 0, ndet: int = 8):
    """The few-determinant guiding state on the device (Methods: a few leading
    determinants stand in for the ground state)."""
    import torch

    from . import inputs
    idx, amp = inputs.determinant_state(n, seed=seed, ndet=ndet, min_distance=min_distance)
    t = torch.zeros(1 << n, dtype=dtype, device=device)
    t[torch.as_tensor(idx.astype(np.int64), device=device)] = torch.as_tensor(amp, device=device).to(dtype)
    return t


class Problem:
    """One Hamiltonian with its initial state (ndet determinants from a seed,
    optionally pairwise at Hamming distance >= min_distance)."""

    def __init__(self, n: int, x, z, h, psi_seed: int, min_distance: int = 0, ndet: int = 8):
        from . import inputs
        self.n, self.x, self.z, self.h = n, np.asarray(x, np.uint64), np.asarray(z, np.uint64), np.asarray(h)
        self.psi_seed = psi_seed
        self.min_distance = min_distance
        self.ndet = ndet
        self.ham = Hamiltonian(n, self.x, self.z, self.h)
        self.det_idx, self.det_amp = inputs.determinant_state(n, seed=psi_seed, ndet=ndet, min_distance=min_distance)

    def state(self, dtype, device="cuda"):
        return initial_state(self.n, self.psi_seed, dtype, device, self.min_distance, self.ndet)

    def features(self, t: float, r: int):
        return self.ham.features(self.det_idx, self.det_amp, t, r)

    @property
    def L(self) -> int:
        return len(self.h)


def synthetic_problems(count: int, seed: int, n_range=(14, 22), L_range=(200, 2000), lam_range=None,
                       far_every: int = 0, far_distance: int = 10):
    """Seeded JW-like Hamiltonians: n uniform in n_range, L uniform in
    L_range, one-norm uniform in lam_range (default: the generator's
    L-dependent one-norm).  With far_every = k, every k-th problem has at
    least 16 qubits and a guiding state of four determinants pairwise at
    Hamming distance >= far_distance, so that no product of two 2- or 4-qubit
    terms connects them (the first-order error coefficient vanishes, as it
    does for eight-determinant states at large n)."""
    from . import inputs
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        lam = None if lam_range is None else float(rng.uniform(lam_range[0], lam_range[1]))
        far = far_every and i % far_every == far_every - 1
        if far:
            n = max(n, 16)
        x, z, h = inputs.jw_hamiltonian(n, L, seed=seed * 7919 + i, lam=lam)
        out.append(Problem(n, x, z, h, psi_seed=seed * 7919 + i, min_distance=far_distance if far else 0,
                           ndet=4 if far else 8))
    return out


def overlaps_by_batch(problems, times, r_values, dtype=None, cfg=None, max_rotations: int = 40_000_000,
                      device="cuda"):
    """g[p][t][r] = <psi_p|U_r(t)|psi_p> for every problem, time and r, from
    batched launches of at most max_rotations rotations each."""
    import torch
    dtype = torch.complex64 if dtype is None else dtype
    jobs = [(pi, ti, r) for pi in range(len(problems)) for ti in range(len(times)) for r in r_values]
    g = {}
    start = 0
    while start < len(jobs):
        chunk, rot = [], 0
        while start < len(jobs):
            pi, ti, r = jobs[start]
            cost = problems[pi].L * r
            if chunk and rot + cost > max_rotations:
                break
            chunk.append(jobs[start])
            rot += cost
            start += 1
        psi0 = {}
        runs = []
        for pi, ti, r in chunk:
            p = problems[pi]
            if pi not in psi0:
                psi0[pi] = p.state(dtype, device)
            x, z, phi = p.ham.trotter_stream(times[ti], r)
            runs.append(dict(n=p.n, x=x, z=z, phi=phi, psi0=psi0[pi]))
        b = Batch(runs, dtype=dtype, cfg=cfg, device=device)
        res = b.run()
        b.close()
        for (pi, ti, r), v in zip(chunk, res):
            g[(pi, ti, r)] = complex(v)
        del runs, b, psi0
    return g


def training_rows(problems, times=TIMES16, r_values=R_VALUES, dtype=None, cfg=None, max_rotations=40_000_000):
    """(features [rows x 10] float32, log eps [rows] float32, info) for every
    problem, time and r in r_values, errors against the Richardson limit of
    r = 32, 64, 128.  The runs are complex128 by default: the errors that
    decide r sit near 1e-3 and below, where complex64 rounding of a
    10^5-rotation run (about 1e-5 in the overlap) would blur them."""
    import torch
    dtype = torch.complex128 if dtype is None else dtype
    rs = tuple(sorted(set(r_values) | {32, 64, R_EXTRA}))
    g = overlaps_by_batch(problems, times, rs, dtype=dtype, cfg=cfg, max_rotations=max_rotations)
    X, y, info = [], [], []
    for pi, p in enumerate(problems):
        for ti, t in enumerate(times):
            g_lim = richardson3(g[(pi, ti, 32)], g[(pi, ti, 64)], g[(pi, ti, R_EXTRA)])
            eps, log_eps = _lib.ps_trotter_error_labels([g[(pi, ti, r)] for r in r_values], g_lim, EPS_FLOOR)
            for k, r in enumerate(r_values):
                X.append(p.features(t, r))
                y.append(log_eps[k])
                info.append((pi, ti, r, float(eps[k])))
    return np.asarray(X, np.float32), np.asarray(y, np.float32), info


class StepPredictor:
    """The FP32 network (three tanh layers of 128) on the current device."""

    def __init__(self, seed: int = 0, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = _lib.ps_mlp_create(PS_MLP_FEATURES, seed, self.stream.cuda_stream)
        self.margin = 0.0

    def close(self):
        if getattr(self, "handle", None):
            _lib.ps_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        return _lib.ps_mlp_get_params(self.handle)

    def set_params(self, p):
        _lib.ps_mlp_set_params(self.handle, p)

    def normalization(self):
        return _lib.ps_mlp_get_normalization(self.handle, PS_MLP_FEATURES)

    def set_normalization(self, mu, sigma, y_mu, y_sigma):
        _lib.ps_mlp_set_normalization(self.handle, mu, sigma, y_mu, y_sigma)

    def fit(self, X, y, epochs=300, batch=256, lr=1e-3, seed=0):
        """Standardise on (X, y) and train; returns the loss of every epoch."""
        import torch
        X = np.ascontiguousarray(np.asarray(X, np.float32))
        y = np.ascontiguousarray(np.asarray(y, np.float32))
        _lib.ps_mlp_fit_normalization(self.handle, X, y)
        xd = torch.as_tensor(X).cuda()
        yd = torch.as_tensor(y).cuda()
        losses = _lib.ps_mlp_train(self.handle, xd.data_ptr(), yd.data_ptr(), len(y),
                                   dict(epochs=epochs, batch=batch, lr=lr, seed=seed))
        torch.cuda.synchronize()
        return losses

    def calibrate_margin(self, X_val, y_val, quantile: float = 0.8) -> float:
        """Margin for pick_r: the given quantile of the held-out residuals
        log eps - prediction (at least 0), so that the prediction plus the
        margin bounds the error in about that fraction of cases."""
        self.margin = _lib.ps_mlp_margin(y_val, self.predict(X_val), quantile)
        return self.margin

    def predict(self, X) -> np.ndarray:
        import torch
        X = np.ascontiguousarray(np.asarray(X, np.float32))
        xd = torch.as_tensor(X).cuda()
        yd = torch.empty(len(X), dtype=torch.float32, device="cuda")
        _lib.ps_mlp_predict(self.handle, xd.data_ptr(), len(X), yd.data_ptr())
        return yd.cpu().numpy()

    def pick_r(self, problem: Problem, t: float, eps: float = 1e-3, margin: float | None = None, r_max: int = 4096):
        """(r, predictions for r = 1..r_max); r = 0 when no r <= r_max
        qualifies.  The margin defaults to the calibrated one."""
        m = self.margin if margin is None else margin
        return _lib.ps_mlp_pick_r(self.handle, problem.ham.handle, problem.det_idx, problem.det_amp, t, eps, m, r_max)

    def save(self, path: str):
        mu, sigma, ym, ys = self.normalization()
        np.savez(path, params=self.params(), mu=mu, sigma=sigma, y_mu=ym, y_sigma=ys, margin=self.margin)

    def load(self, path: str):
        d = np.load(path)
        self.set_params(d["params"])
        self.set_normalization(d["mu"], d["sigma"], float(d["y_mu"]), float(d["y_sigma"]))
        self.margin = float(d["margin"])


class StepEnsemble:
    """Several independently seeded predictors trained on the same rows; the
    prediction is the mean of their predicted log errors (lower variance than
    any one network)."""

    def __init__(self, count: int = 4, seed: int = 0, stream=None):
        self.members = [StepPredictor(seed=seed + 101 * k, stream=stream) for k in range(count)]
        self.margin = 0.0

    def fit(self, X, y, epochs=150, batch=256, lr=2e-3, seed=0):
        return [mb.fit(X, y, epochs=epochs, batch=batch, lr=lr, seed=seed + 7 * k)
                for k, mb in enumerate(self.members)]

    def predict(self, X) -> np.ndarray:
        import torch
        X = np.ascontiguousarray(np.asarray(X, np.float32))
        xd = torch.as_tensor(X).cuda()
        return _lib.ps_mlp_predict_ensemble([mb.handle for mb in self.members], xd.data_ptr(), len(X))

    def calibrate_margin(self, X_val, y_val, quantile: float = 0.8) -> float:
        self.margin = _lib.ps_mlp_margin(y_val, self.predict(X_val), quantile)
        return self.margin

    def pick_r(self, problem: Problem, t: float, eps: float = 1e-3, margin: float | None = None, r_max: int = 4096):
        m = self.margin if margin is None else margin
        return _lib.ps_mlp_pick_r_ensemble([mb.handle for mb in self.members], problem.ham.handle, problem.det_idx,
                                           problem.det_amp, t, eps, m, r_max)

    def close(self):
        for mb in self.members:
            mb.close()


def sweep(problem: Problem, t: float, eps: float = 1e-3, r_max: int = 4096, dtype=None):
    """The plain doubling sweep on one GPU state: (r, rotations applied, g_r)."""
    import torch
    dtype = torch.complex64 if dtype is None else dtype
    psi0 = StateVector(problem.n, tensor=problem.state(dtype))
    work = StateVector(problem.n, dtype=dtype)
    try:
        return ps_trotter_sweep(work.handle, psi0.handle, problem.ham.handle, t, eps, r_max)
    finally:
        work.close()
        psi0.close()


def bound_r(problem: Problem, t: float, eps: float = 1e-3) -> int:
    """Step count from the analytic bound (ps_ham_bound_steps): eps = C delta^2
    with delta = t / r (the paper's error model), so r = ceil(t sqrt(C / eps))."""
    return _lib.ps_ham_bound_steps(problem.ham.handle, t, eps)


def run_error(problem: Problem, t: float, r: int, g_ref: complex, dtype=None) -> float:
    """|g_r - g_ref| for one Trotter run on the GPU."""
    import torch
    dtype = torch.complex64 if dtype is None else dtype
    psi0 = StateVector(problem.n, tensor=problem.state(dtype))
    work = StateVector(problem.n, dtype=dtype)
    try:
        work.copy_from(psi0)
        work.evolve_trotter(problem.ham, t, r)
        return abs(work.overlap(psi0) - g_ref)
    finally:
        work.close()
        psi0.close()


def reference_overlap(problem: Problem, t: float, R: int = 256, dtype=None) -> complex:
    """Richardson limit from r = R, 2R, 4R (one batched launch)."""
    g = overlaps_by_batch([problem], [t], (R, 2 * R, 4 * R), dtype=dtype)
    return richardson3(g[(0, 0, R)], g[(0, 0, 2 * R)], g[(0, 0, 4 * R)])


__all__ = ["StepPredictor", "StepEnsemble", "Problem", "synthetic_problems", "training_rows", "overlaps_by_batch", "sweep",
           "bound_r", "run_error", "reference_overlap", "richardson3", "TIMES16", "R_VALUES"]
