"""GPU: the step-count predictor's kernels against the oracle, and what the
trained network gains over the doubling sweep.

FP32 kernels against the FP64 oracle (oracle/learned.py, pinned by finite
differences and closed forms): outputs to 2e-5 relative, gradients and Adam
updates to 1e-3 relative (the bar for FP32 gradients).
"""
import math

import numpy as np
import pytest
import torch

import paper_2504_17881_gb300 as ps
from oracle import learned as OL
from paper_2504_17881_gb300 import _lib, inputs, learned

pytestmark = pytest.mark.gpu

F = ps.PS_MLP_FEATURES
W = 128


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def random_net(seed, scale=0.15):
    m = learned.StepPredictor(seed=seed)
    rng = np.random.default_rng(seed)
    p = rng.normal(0, scale, size=_lib.ps_mlp_num_params(m.handle)).astype(np.float32)
    m.set_params(p)
    return m, p.astype(np.float64)


def data(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(1.0, 2.0, size=(rows, F)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.3 * X[:, 1] ** 2 - X[:, 5]).astype(np.float32)
    return X, y


def test_param_count_and_init():
    m = learned.StepPredictor(seed=3)
    p = m.params().astype(np.float64)
    assert len(p) == W * F + W + 2 * (W * W + W) + W + 1
    d = OL.unpack(p, F, W)
    assert np.all(d["b1"] == 0) and np.all(d["b2"] == 0) and np.all(d["b3"] == 0) and d["b_out"][0] == 0
    a1 = math.sqrt(6 / (F + W))
    a2 = math.sqrt(6 / (2 * W))
    assert np.max(np.abs(d["W1"])) <= a1 and np.std(d["W1"]) == pytest.approx(a1 / math.sqrt(3), rel=0.1)
    assert np.max(np.abs(d["W2"])) <= a2 and np.std(d["W2"]) == pytest.approx(a2 / math.sqrt(3), rel=0.05)
    # the seed determines the weights
    assert np.array_equal(learned.StepPredictor(seed=3).params(), m.params())
    assert not np.array_equal(learned.StepPredictor(seed=4).params(), m.params())


def test_forward_matches_oracle():
    m, p = random_net(1)
    X, _ = data(333, 2)  # ragged: 10 full CTAs of 32 rows and a tail
    mu = np.linspace(-1, 1, F).astype(np.float32)
    sd = np.linspace(0.5, 2, F).astype(np.float32)
    m.set_normalization(mu, sd, 0.25, 3.0)
    got = m.predict(X)
    Xs = (X.astype(np.float64) - mu) / sd
    out, _ = OL.forward(p, Xs, F, W)
    assert rel(got, 0.25 + 3.0 * out) < 2e-5


def numpy_normalization(X, y):
    """Standardisation constants computed here (FP32, as the network stores
    them), so that the oracle's inputs do not come from the library."""
    mu = X.astype(np.float64).mean(axis=0).astype(np.float32)
    sd = X.astype(np.float64).std(axis=0).astype(np.float32)
    return mu, sd, np.float32(y.astype(np.float64).mean()), np.float32(y.astype(np.float64).std())


def test_loss_and_gradient_match_oracle_backprop():
    m, p = random_net(5)
    X, y = data(300, 6)
    mu, sd, ym, ys = numpy_normalization(X, y)
    m.set_normalization(mu, sd, float(ym), float(ys))
    xd, yd = torch.as_tensor(X).cuda(), torch.as_tensor(y).cuda()
    loss = _lib.ps_mlp_loss_grad(m.handle, xd.data_ptr(), yd.data_ptr(), len(y))
    g = _lib.ps_mlp_get_grads(m.handle).astype(np.float64)
    Xs = (X.astype(np.float64) - mu) / sd
    ts = (y.astype(np.float64) - ym) / ys
    loss_o, g_o = OL.loss_and_grad(p, Xs, ts, F, W)
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert rel(g, g_o) < 1e-3
    # every parameter block on its own
    go, gg = OL.unpack(g_o, F, W), OL.unpack(g, F, W)
    for name in go:
        assert rel(gg[name], go[name]) < 1e-3, name


def test_gradient_matches_finite_differences_of_gpu_loss():
    m, p = random_net(7)
    X, y = data(256, 8)
    _lib.ps_mlp_fit_normalization(m.handle, X, y)
    xd, yd = torch.as_tensor(X).cuda(), torch.as_tensor(y).cuda()
    _lib.ps_mlp_loss_grad(m.handle, xd.data_ptr(), yd.data_ptr(), len(y))
    g = _lib.ps_mlp_get_grads(m.handle).astype(np.float64)
    rng = np.random.default_rng(9)
    for _ in range(3):
        d = rng.normal(size=len(p))
        d /= np.linalg.norm(d)
        h = 3e-3
        m.set_params((p + h * d).astype(np.float32))
        lp = _lib.ps_mlp_loss_grad(m.handle, xd.data_ptr(), yd.data_ptr(), len(y))
        m.set_params((p - h * d).astype(np.float32))
        lm = _lib.ps_mlp_loss_grad(m.handle, xd.data_ptr(), yd.data_ptr(), len(y))
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(float(g @ d), rel=2e-2, abs=1e-4)


def test_adam_steps_match_oracle():
    """Three Adam steps of the kernel against the oracle's, both fed the same
    seeded gradients (set on the device with ps_mlp_set_grads), so neither side
    takes an input from the other."""
    m, p = random_net(11)
    rng = np.random.default_rng(12)
    mo = np.zeros_like(p)
    vo = np.zeros_like(p)
    q = p.copy()
    for step in (1, 2, 3):
        g = rng.normal(0, 0.05, size=p.size).astype(np.float32)
        _lib.ps_mlp_set_grads(m.handle, g)
        _lib.ps_mlp_adam_step(m.handle, 1e-3, 0.9, 0.999, 1e-8)
        q, mo, vo = OL.adam_step(q, g.astype(np.float64), mo, vo, step, 1e-3)
        got = m.params().astype(np.float64)
        # FP32 parameters and moments: a few ulps of the 0.15-sized weights per step
        assert np.max(np.abs(got - q)) < 1e-6 * step, step


def test_training_reduces_loss_and_is_reproducible():
    X, y = data(4096, 13)
    m1 = learned.StepPredictor(seed=1)
    l1 = m1.fit(X, y, epochs=60, batch=256, lr=2e-3, seed=5)
    assert l1[-1] < 0.1 * l1[0]
    m2 = learned.StepPredictor(seed=1)
    l2 = m2.fit(X, y, epochs=60, batch=256, lr=2e-3, seed=5)
    assert np.array_equal(l1, l2) and np.array_equal(m1.params(), m2.params())
    Xt, yt = data(512, 14)
    pred = m1.predict(Xt)
    assert np.sqrt(np.mean((pred - yt) ** 2)) < 0.35 * np.std(yt)


def test_features_and_bound_match_oracle():
    for seed, n, L in ((1, 9, 60), (2, 12, 200)):
        x, z, h = inputs.jw_hamiltonian(n, L, seed=seed)
        idx, amp = inputs.determinant_state(n, seed=seed + 10)
        psi = inputs.densify(n, idx, amp)
        H = ps.Hamiltonian(n, x, z, h)
        K, e2 = H.error_coefficient(idx, amp)
        assert abs(K - OL.error_coefficient(n, x, z, h, psi)) < 1e-12
        assert e2 == pytest.approx(OL.second_order_norm2(n, x, z, h, psi), rel=1e-12)
        for t, r in ((0.1, 1), (1.3, 7), (3.2, 64)):
            assert np.allclose(H.features(idx, amp, t, r), OL.features(n, x, z, h, t, r, psi), rtol=3e-7, atol=1e-6)
        for L_D in (0, L // 10, L):
            assert H.trotter_bound(L_D) == pytest.approx(OL.trotter_bound(n, x, z, h, L_D), rel=1e-12)


NPROB = 480
NHOLD = 48


@pytest.fixture(scope="module")
def trained():
    """An ensemble of four predictors trained on batched-engine errors of
    small problems; the last NHOLD problems are held out to calibrate the
    pick margin."""
    probs = learned.synthetic_problems(NPROB, seed=1000, n_range=(8, 12), L_range=(40, 160), lam_range=(1.5, 5.0))
    times = learned.TIMES16[::2]
    X, y, info = learned.training_rows(probs, times=times)
    cut = (NPROB - NHOLD) * len(times) * len(learned.R_VALUES)
    m = learned.StepEnsemble(count=4, seed=2)
    losses = m.fit(X[:cut], y[:cut], epochs=150, batch=256, lr=2e-3, seed=3)[0]
    m.calibrate_margin(X[cut:], y[cut:], 0.8)
    return m, X, y, losses


def test_training_rows_come_from_consistent_errors(trained):
    m, X, y, losses = trained
    assert X.shape == (NPROB * 8 * 7, ps.PS_MLP_FEATURES)
    # first order: the error falls with r, roughly as 1/r at large r
    e = np.exp(y).reshape(NPROB, 8, 7)
    big = e[:, :, 4] > 1e-6
    slope = np.log(e[:, :, 6] / e[:, :, 4]) / np.log(4.0)
    assert np.median(slope[big]) == pytest.approx(-1.0, abs=0.2)
    # the errors span the target: below and above 1e-3
    assert np.mean(e < 1e-3) > 0.2 and np.mean(e > 1e-3) > 0.2
    assert losses[-1] < 0.1 * losses[0]


def test_learned_pick_gains_over_sweep(trained):
    """On held-out Hamiltonians the network's r reaches the target about as
    well as the sweep's, for a fraction of the rotations.  Both are judged
    against the smallest adequate step count r*, found by running every r up
    to 128 in one batched launch and comparing with the Richardson limit."""
    m = trained[0]
    eps = 1e-3
    probs = learned.synthetic_problems(12, seed=2000, n_range=(10, 12), L_range=(60, 150), lam_range=(1.5, 5.0))
    c128 = torch.complex128
    times = [(0.6, 1.2, 2.4)[i % 3] for i in range(len(probs))]
    rows = []
    for i, (p, t) in enumerate(zip(probs, times)):
        r_sw, rot_sw, _ = learned.sweep(p, t, eps, dtype=c128)
        r_ml, _ = m.pick_r(p, t, eps)
        assert r_ml > 0
        g = learned.overlaps_by_batch([p], [t], tuple(range(1, 129)) + (256, 512, 1024), dtype=c128)
        g_ref = learned.richardson3(g[(0, 0, 256)], g[(0, 0, 512)], g[(0, 0, 1024)])
        err = {r: abs(g[(0, 0, r)] - g_ref) for r in range(1, 129)}
        r_star = next(r for r in range(1, 129) if err[r] <= eps)
        rows.append((r_star, r_sw, rot_sw, r_ml, r_ml * p.L, err[r_ml], err[r_sw], learned.bound_r(p, t, eps)))
    rows = np.array(rows, dtype=np.float64)
    r_star, r_sw, rot_sw, r_ml, rot_ml, err_ml, err_sw, r_bd = rows.T
    print(f"\nmargin {m.margin:.3f}\n r*  sweep  learned  bound   err(learned)  err(sweep)")
    for row in rows:
        print(f"{row[0]:4.0f} {row[1]:6.0f} {row[3]:8.0f} {row[7]:6.0f}   {row[5]:.2e}      {row[6]:.2e}")
    print(f"rotations: learned {rot_ml.sum():.0f}, sweep {rot_sw.sum():.0f} ({rot_ml.sum() / rot_sw.sum():.2f})")
    # the learned r is within a factor 3 of the smallest adequate one in
    # every case (the calibrated margin makes it err on the safe side) ...
    assert np.all(np.abs(np.log2(r_ml / r_star)) <= math.log2(3.0) + 1e-9)
    # ... meets the target in most cases and is never off by more than 2x
    assert np.mean(err_ml <= eps) >= 0.7 and err_ml.max() <= 2 * eps
    # and costs far fewer rotations than the sweep (which runs 1, 2, 4, ..., 2 r_sw)
    assert rot_ml.sum() < 0.35 * rot_sw.sum()
    # the analytic bound asks for many more steps than needed
    assert np.median(r_bd / r_star) > 3
