"""Learned boundary closure: the FP64 MLP reference (pinned by central
finite differences and a closed-form linear limit), the device training and
inference kernels against it, the shadow-chain sample recorder and the
closure in the time step."""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from oracle import closure as C
from paper_1610_05023_b300 import workloads as W


def _weights(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0, C.NPARAM)
    W1, b1, W2, b2, w3, b3 = C.unpack(w)
    w[:C.NH * C.NIN] *= scale / np.sqrt(C.NIN)
    o = C.NH * C.NIN + C.NH
    w[o:o + C.NH * C.NH] *= scale / np.sqrt(C.NH)
    w[o + C.NH * C.NH + C.NH:o + C.NH * C.NH + 2 * C.NH] *= scale / np.sqrt(C.NH)
    return w


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0, (n, C.NIN))
    Y = 0.3 * np.tanh(X[:, 0] - 0.5 * X[:, 1]) + 0.1 * X[:, 2] * X[:, 3] - 0.05 * X[:, 4] + 0.02 * X[:, 5]
    return X, Y


# ---------------------------------------------------------------- CPU pins
def test_oracle_gradient_matches_central_differences():
    w = _weights(1)
    X, Y = _data(2, 40)
    _, g = C.loss_grad(w, X, Y)
    o1 = C.NH * C.NIN
    o2 = o1 + C.NH
    o3 = o2 + C.NH * C.NH
    idx = [0, 7, o1 - 1, o1, o1 + 9, o2, o2 + 777, o3 - 1, o3 + 3, o3 + C.NH + 5, C.NPARAM - 1]
    fd = C.finite_difference_grad(w, X, Y, idx)
    assert np.allclose(g[idx], fd, rtol=1e-6, atol=1e-10)


def test_oracle_forward_linear_limit_and_constant_output():
    """Small weights: tanh(z) = z + O(z^3), so the network reduces to the
    affine map b3 + w3.(W2 (W1 x + b1) + b2).  With W2 = b2 = 0 the hidden
    layer 2 vanishes and the output is b3."""
    eps = 1e-4
    w = eps * np.random.default_rng(3).normal(0.0, 1.0, C.NPARAM)   # every weight and bias small
    w[-1] = 0.3
    X, _ = _data(4, 8)
    W1, b1, W2, b2, w3, b3 = C.unpack(w)
    lin = b3 + (((X @ W1.T + b1) @ W2.T + b2) @ w3)
    assert np.allclose(C.forward(w, X), lin, rtol=0, atol=1e-10 * max(1.0, abs(b3)))
    w0 = w.copy()
    o = C.NH * C.NIN + C.NH
    w0[o:o + C.NH * C.NH + C.NH] = 0.0
    assert np.allclose(C.forward(w0, X), b3, atol=0)


# ---------------------------------------------------------------- GPU
@pytest.mark.gpu
def test_gpu_loss_and_gradient_match_fp64():
    w = _weights(5).astype(np.float32)
    X, Y = _data(6, 3000)
    X, Y = X.astype(np.float32), Y.astype(np.float32)
    L, g = dgh.mlp_loss_grad(w, X, Y)
    Lr, gr = C.loss_grad(w.astype(np.float64), X, Y)
    assert abs(L - Lr) <= 1e-5 * Lr
    assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr)


@pytest.mark.gpu
def test_gpu_inference_matches_fp64_with_bf16_weights():
    import torch
    w = _weights(7).astype(np.float32)
    X, _ = _data(8, 5000)
    X = X.astype(np.float32)
    y = dgh.closure_eval(w, X)           # the correction MLP(x) - MLP(0)
    wb = torch.tensor(w).to(torch.bfloat16).to(torch.float64).numpy()   # the weights the kernel uses
    z = np.zeros((1, C.NIN))
    yr = C.forward(wb, X.astype(np.float64)) - C.forward(wb, z)
    assert np.linalg.norm(y - yr) <= 1e-5 * np.linalg.norm(yr)
    y64 = C.forward(w.astype(np.float64), X.astype(np.float64)) - C.forward(w.astype(np.float64), z)
    assert np.linalg.norm(y - y64) <= 1e-2 * np.linalg.norm(y64)   # BF16 weight rounding
    assert dgh.closure_eval(w, np.zeros((3, C.NIN)))[0] == 0.0


@pytest.mark.gpu
def test_gpu_training_fits_smooth_target():
    X, Y = _data(9, 20000)
    w, hist, mse = dgh.mlp_train(X, Y, steps=1500, batch=2048, lr=2e-3, seed=3)
    var = float(np.var(Y))
    assert mse < 0.05 * var, (mse, var)
    assert np.mean(hist[-100:]) < 0.2 * np.mean(hist[:20])
    # the returned weights take raw features (standardisation folded in)
    yr = C.forward(w.astype(np.float64), X)
    assert abs(np.mean((yr - Y) ** 2) - mse) <= 1e-3 * var + 0.05 * mse


def _solver(P, seed=50):
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.02, seed=seed)
    g = dgh.Solver(VX, EToV, 3, P)
    g.init_gaussian([0.3, 0.2, -0.1], 0.3)
    return g


@pytest.mark.gpu
def test_recorder_shadow_equal_order_gives_zero_targets():
    """A shadow chain of the context's own order reproduces its r^- exactly:
    every recorded target is 0; features are the chain's own values."""
    g = _solver(2)
    g.closure_record(shadow_order=2, every=1, fraction=1.0, max_samples=1 << 20, seed=1)
    g.init_gaussian([0.3, 0.2, -0.1], 0.3)
    g.step(30)
    S = g.closure_samples()
    T, Np2 = g.info["n_tris"], g.info["Np2"]
    assert S.shape == (30 * T * Np2, 7)
    assert np.all(S[:, 6] == 0.0)
    assert np.all(np.isfinite(S)) and np.abs(S[:, 0]).max() > 0


@pytest.mark.gpu
def test_recorder_lower_order_shadow_and_sampling():
    g = _solver(6)
    g.closure_record(shadow_order=2, every=5, fraction=0.25, max_samples=1 << 20, seed=2)
    g.init_gaussian([0.3, 0.2, -0.1], 0.3)
    g.step(60)
    S = g.closure_samples()
    T, Np2 = g.info["n_tris"], g.info["Np2"]
    rows = T * Np2 * 12          # steps 0, 5, ..., 55
    assert 0.2 * rows < S.shape[0] < 0.3 * rows
    assert np.abs(S[:, 6]).max() > 0          # orders 6 and 2 differ once the wave is at the faces
    base = dgh.Solver(*W.kuhn_mesh(3, 1.0, 0.02, seed=50), 3, 6)
    base.init_gaussian([0.3, 0.2, -0.1], 0.3)
    base.step(60)
    assert np.array_equal(base.get_state(3), g.get_state(3))   # the shadow never feeds back


@pytest.mark.gpu
def test_closed_loop_recorder_rows_match_open_loop_rows_at_the_first_step():
    """With the closure on, the recorder takes this chain's features and
    r^-_shadow - r^-_this (closed-loop rows).  Here the correction is zero and
    only the first step is recorded, where every chain still sees the initial
    state: a P = 2 context with a P = 6 shadow must then record the same rows
    as a P = 6 context with a P = 2 shadow (open-loop rows: the shadow's
    features, r^-_this - r^-_shadow).  Same hashed node selection, so the
    same set of rows."""
    w = _weights(16).astype(np.float32)
    w[C.NPARAM - C.NH - 1:] = 0.0      # w3 = 0, b3 = 0: MLP == 0
    a, b = _solver(2), _solver(6)
    a.closure_set_weights(w)
    a.closure_record(shadow_order=6, every=1, fraction=1.0, max_samples=1 << 20, seed=3)
    b.closure_record(shadow_order=2, every=1, fraction=1.0, max_samples=1 << 20, seed=3)
    for g in (a, b):
        g.init_gaussian([0.3, 0.2, -0.1], 0.3)
        g.step(1)
    Sa, Sb = a.closure_samples(), b.closure_samples()
    T, Np2 = a.info["n_tris"], a.info["Np2"]
    assert Sa.shape == Sb.shape == (T * Np2, 7)
    Sa, Sb = Sa[np.lexsort(Sa.T[::-1])], Sb[np.lexsort(Sb.T[::-1])]
    assert np.abs(Sa[:, 6]).max() > 0          # the orders differ at the first stage already
    assert np.allclose(Sa, Sb, rtol=1e-6, atol=1e-6 * np.abs(Sb).max())


@pytest.mark.gpu
def test_closure_train_on_recorded_rows_equals_mlp_train():
    """dgh_closure_train trains on the context's recorded rows exactly as
    dgh_mlp_train on the same rows read back (fixed-order reductions)."""
    g = _solver(6)
    g.closure_record(shadow_order=2, every=2, fraction=0.5, max_samples=1 << 20, seed=4)
    g.init_gaussian([0.3, 0.2, -0.1], 0.3)
    g.step(40)
    S = g.closure_samples()
    w1, h1, f1 = g.closure_train(steps=50, batch=256, lr=1e-3, seed=5)
    w2, h2, f2 = dgh.mlp_train(S[:, :6], S[:, 6], steps=50, batch=256, lr=1e-3, seed=5)
    assert np.array_equal(w1, w2) and np.array_equal(h1, h2) and f1 == f2
    fresh = _solver(2)
    with pytest.raises(dgh.DghError):
        fresh.closure_train(steps=5)               # nothing recorded
    # the homogeneous form on the same rows: the context-free fit, exactly
    wh1, hh1, fh1 = g.closure_train(homogeneous=True, steps=50, batch=256, lr=1e-3, seed=5)
    wh2, hh2, fh2 = dgh.closure_fit_homogeneous(S[:, :6], S[:, 6], steps=50, batch=256, lr=1e-3, seed=5)
    assert wh1.shape == (C.NPARAM + C.NIN + 1,)
    assert np.array_equal(wh1, wh2) and np.array_equal(hh1, hh2) and fh1 == fh2


@pytest.mark.gpu
def test_homogeneous_fit_follows_its_definition():
    """dgh_closure_fit_homogeneous against its definition restated in FP64
    numpy: per-feature RMS scales sigma_i and sigma_y, then dgh_mlp_train on
    the directions x~ / |x~| (x~ = x / sigma) and relative targets
    y / (sigma_y |x~|) of the rows with non-zero features.  The scales agree
    to FP32 rounding; the network equals mlp_train's on those inputs up to
    the last-bit differences that the two summation orders of sigma leave in
    the inputs."""
    X, Y = _data(21, 3000)
    X = X * np.array([1.0, 3.0, 0.5, 2.0, 0.1, 7.0])
    X[::97] = 0.0                                  # rows without a direction are dropped
    kw = dict(steps=40, batch=512, lr=1e-3, seed=9)
    wh, _, _ = dgh.closure_fit_homogeneous(X, Y, **kw)
    Xd, Yd = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
    sx = np.sqrt(np.mean(Xd * Xd, axis=0))
    sy = np.sqrt(np.mean(Yd * Yd))
    assert np.allclose(wh[C.NPARAM:C.NPARAM + C.NIN], 1.0 / sx, rtol=1e-6)
    assert abs(wh[-1] - sy) <= 1e-6 * sy
    Xt = Xd / sx
    s = np.linalg.norm(Xt, axis=1)
    keep = s > 0
    assert keep.sum() == len(X) - len(X[::97])
    w2, _, _ = dgh.mlp_train(Xt[keep] / s[keep, None], Yd[keep] / (sy * s[keep]), **kw)
    assert np.abs(wh[:C.NPARAM] - w2).max() <= 1e-4 * np.abs(w2).max()
    with pytest.raises(dgh.DghError):
        dgh.closure_fit_homogeneous(np.zeros((10, 6)), np.ones(10), steps=2)


@pytest.mark.gpu
def test_closure_zero_output_is_bit_identical_and_output_changes_solution():
    w = _weights(11).astype(np.float32)
    o3 = C.NPARAM - C.NH - 1
    w[o3:] = 0.0                       # w3 = 0, b3 = 0: MLP == 0
    a, b = _solver(2), _solver(2)
    b.closure_set_weights(w)
    a.step(25)
    b.step(25)
    for lv in (3, 2, 1):
        assert np.array_equal(a.get_state(lv), b.get_state(lv))
    c0 = _solver(2)
    w[-1] = 1e-3                       # a constant output is removed by the MLP(0) subtraction
    c0.closure_set_weights(w)
    c0.step(25)
    assert np.array_equal(c0.get_state(3), a.get_state(3))
    w[o3:o3 + C.NH] = 1e-3 * np.random.default_rng(12).normal(size=C.NH)   # a field-dependent correction
    c = _solver(2)
    c.closure_set_weights(w)
    c.step(25)
    d = np.linalg.norm(c.get_state(3) - a.get_state(3))
    assert 0 < d < 1e-1 * np.linalg.norm(a.get_state(3))
    c.closure_set_weights(None)        # disabling restores the plain chain from here on
    assert np.isfinite(c.energy())


@pytest.mark.gpu
def test_closure_gives_no_correction_at_zero_fields():
    """MLP(0) is evaluated once per weight set by the inference code itself,
    so a field-free run stays exactly zero under a closure with arbitrary
    weights (a correction of even one ulp at zero fields would inject a
    nonzero exterior state)."""
    g = _solver(2)
    g.closure_set_weights(_weights(17).astype(np.float32))
    g.init_gaussian([0.3, 0.2, -0.1], 0.3, 0.0)
    g.step(20)
    for lv in (3, 2, 1):
        assert np.all(g.get_state(lv) == 0.0)


@pytest.mark.gpu
def test_homogeneous_form_is_degree_one_and_zero_at_zero():
    w = _weights(13).astype(np.float32)
    rng = np.random.default_rng(14)
    scales = np.concatenate([1.0 / rng.uniform(0.5, 2.0, C.NIN), [0.7]]).astype(np.float32)
    wh = np.concatenate([w, scales])
    X, _ = _data(15, 200)
    y1 = dgh.closure_eval(wh, X)
    y3 = dgh.closure_eval(wh, 3.0 * X)
    assert np.allclose(y3, 3.0 * y1, rtol=1e-5, atol=1e-7)
    assert np.all(dgh.closure_eval(wh, np.zeros((4, C.NIN))) == 0.0)
    # against FP64: sigma_y |x~| MLP(x~ / |x~|) with the BF16-rounded weights
    import torch
    wb = torch.tensor(w).to(torch.bfloat16).to(torch.float64).numpy()
    Xt = X * scales[:C.NIN].astype(np.float64)
    s = np.linalg.norm(Xt, axis=1)
    yr = scales[C.NIN] * s * C.forward(wb, Xt / s[:, None])
    assert np.linalg.norm(y1 - yr) <= 1e-5 * np.linalg.norm(yr)


@pytest.mark.gpu
def test_closed_loop_closure_reflects_less_than_plain_p2():
    """What the trained network gains over the method without it: on the
    evaluation problem of the closure form (40^3 x 6 unjittered tets, N = 4,
    Gaussian pulse of width 0.12 at (0.35, -0.25, 0.30), t in [0, 1.5]), the
    energy-norm error against a large-domain run (80^3 x 6 tets, whose
    boundary cannot reflect back in time) after the wave reaches the faces is
    lower with the closed-loop-trained closure than with plain P = 2.  The
    weights are the ones bench.py --form closure wrote (tests/data)."""
    import math
    import os
    w = np.load(os.path.join(os.path.dirname(__file__), "data", "closure_closed_loop_w.npy"))
    assert w.shape == (C.NPARAM,)
    n, T, sigma, x0 = 40, 1.5, 0.12, [0.35, -0.25, 0.30]
    h = 2.0 / n
    pad = int(math.ceil((T / 2 + 2 * sigma) / h))
    VXs, EToVs = W.kuhn_mesh(n, 1.0, 0.0, seed=0)
    VXl, EToVl = W.kuhn_mesh(n + 2 * pad, 1.0 + pad * h, 0.0, seed=0)
    key = lambda c: [tuple(v) for v in np.round(c / (h / 64.0)).astype(np.int64)]
    where = {k: i for i, k in enumerate(key(VXl[EToVl].mean(axis=1)))}
    inner = np.array([where[k] for k in key(VXs[EToVs].mean(axis=1))])
    ref = dgh.Solver(VXl, EToVl, 4, 0)
    dt = min(ref.info["dt"], dgh.plan(VXs, EToVs, 4, 8)["dt"])
    ref.close()
    nck = 15
    nst = int(math.ceil(T / dt))
    nst += (-nst) % nck
    dt = T / nst
    plain = dgh.Solver(VXs, EToVs, 4, 2, dt=dt)
    closed = dgh.Solver(VXs, EToVs, 4, 2, dt=dt)
    closed.closure_set_weights(w)
    ref = dgh.Solver(VXl, EToVl, 4, 0, dt=dt)
    for g in (plain, closed, ref):
        g.init_gaussian(x0, sigma)
    E0 = plain.energy()
    t_hit = 1.0 - max(abs(v) for v in x0) - 2 * sigma
    worst = {"plain": 0.0, "closed": 0.0}
    for ck in range(1, nck + 1):
        ref.step(nst // nck)
        qr = ref.get_state(3)[inner]
        for name, g in (("plain", plain), ("closed", closed)):
            g.step(nst // nck)
            e = math.sqrt(max(g.error_energy(qr), 0.0) / E0)
            assert math.isfinite(e)
            if ck * T / nck >= t_hit:
                worst[name] = max(worst[name], e)
    for g in (plain, closed, ref):
        g.close()
    assert worst["plain"] > 1e-3                       # plain P = 2 reflects visibly here
    assert worst["closed"] < 0.8 * worst["plain"], worst

