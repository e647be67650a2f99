"""The surrogate network's CUDA kernels (lbs_mlp_*) against the FP64
oracle (oracle/mlp.py): forward, loss, backpropagated gradient, Adam,
bfloat16 inference and ensemble statistics; training reduces the loss.

Tolerances (FP32 kernels against FP64): outputs and loss 1e-5 relative;
gradients 1e-4 of the largest component (sums of up to 256 FP32 products);
bfloat16 inference against the oracle evaluated with the same
bfloat16-rounded weights 1e-4, against the FP32 weights 3e-2 (8-bit
significand)."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu

SHAPE = (5, 128, 3, 2)  # the surrogate: 5 -> 128 -> 128 -> 128 -> 2


def net(E=3, max_batch=512):
    from paper_2311_15242_gb300 import Mlp
    return Mlp(E, *SHAPE, max_batch=max_batch)


def random_params(E, P, seed=0, scale=0.15):
    return np.random.default_rng(seed).normal(0, scale, (E, P)).astype(np.float32)


def bf16_round(a):
    """Round float32 to the nearest bfloat16 (ties to even) and back."""
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_forward_and_gradient_match_oracle():
    E, B = 3, 200
    m = net(E)
    d = M.dims(*SHAPE)
    assert m.P == M.param_count(d) == 34050
    th = random_params(E, m.P)
    m.set_params(th)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(E, B, 5)).astype(np.float32)
    t = rng.normal(size=(E, B, 2)).astype(np.float32)
    y = m.forward(x)
    loss, g = m.gradient(x, t)
    for e in range(E):
        yo, _, _ = M.forward(th[e].astype(np.float64), d, x[e])
        assert np.abs(y[e] - yo).max() <= 1e-5 * np.abs(yo).max()
        Lo, go = M.gradient(th[e].astype(np.float64), d, x[e], t[e])
        assert loss[e] == pytest.approx(Lo, rel=1e-5)
        assert np.abs(g[e] - go).max() <= 1e-4 * np.abs(go).max(), e


def test_adam_steps_match_oracle():
    E = 2
    m = net(E)
    P = m.P
    th = random_params(E, P, seed=2)
    m.set_params(th)
    rng = np.random.default_rng(3)
    ref = th.astype(np.float64)
    mo, vo = np.zeros_like(ref), np.zeros_like(ref)
    for it in range(1, 4):
        g = rng.normal(0, 1e-2, (E, P)).astype(np.float32)
        m.set_grad(g)
        m.adam_step(1e-3, 0.9, 0.999, 1e-8)
        ref, mo, vo = M.adam(ref, g.astype(np.float64), mo, vo, it, 1e-3)
    assert np.abs(m.params() - ref).max() <= 1e-6


def test_bf16_inference_and_ensemble_stats():
    E, n = 5, 300
    m = net(E)
    d = M.dims(*SHAPE)
    th = random_params(E, m.P, seed=4)
    m.set_params(th)
    x = np.random.default_rng(5).normal(size=(n, 5)).astype(np.float32)
    mean16, sd16 = m.predict(x, bf16=True)
    mean32, sd32 = m.predict(x, bf16=False)
    ys16 = [M.forward(bf16_round(th[e]).astype(np.float64), d, x)[0] for e in range(E)]
    ys32 = [M.forward(th[e].astype(np.float64), d, x)[0] for e in range(E)]
    mu16, s16 = M.ensemble_stats(ys16)
    mu32, s32 = M.ensemble_stats(ys32)
    sc = np.abs(mu32).max()
    assert np.abs(mean16 - mu16).max() <= 1e-4 * sc
    assert np.abs(sd16 - s16).max() <= 1e-4 * sc
    assert np.abs(mean32 - mu32).max() <= 1e-5 * sc
    assert np.abs(sd32 - s32).max() <= 1e-5 * sc
    assert np.abs(mean16 - mu32).max() <= 3e-2 * sc


def test_init_is_glorot_uniform():
    m = net(2)
    m.init(7)
    p = m.params()
    d = M.dims(*SHAPE)
    for e in range(2):
        for l, (W, b) in enumerate(M.unpack(p[e].astype(np.float64), d)):
            a = np.sqrt(6.0 / (d[l] + d[l + 1]))
            assert np.abs(W).max() <= a and np.abs(W).max() > 0.9 * a
            assert abs(W.mean()) < 0.1 * a and np.all(b == 0)
    assert not np.array_equal(p[0], p[1])


def test_training_fits_a_smooth_function():
    """Five members trained on minibatches drawn on the device fit
    y = (sin x0 + x1 x2, x3^2 - x4) on 512 points to a small loss, and the
    ensemble spread stays small where there is data."""
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (512, 5)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]) + X[:, 1] * X[:, 2], X[:, 3] ** 2 - X[:, 4]], 1).astype(np.float32)
    m = net(5)
    m.init(11)
    m.set_data(X, Y)
    loss0 = m.train(1, 128, 1e-3, seed=3)
    loss = m.train(3000, 128, 1e-3, seed=3)
    assert loss.max() < 2e-3 * max(loss0.max(), 1e-3) or loss.max() < 1e-4, (loss0, loss)
    mean, sd = m.predict(X[:64], bf16=True)
    assert np.abs(mean - Y[:64]).max() < 0.05
    assert sd.max() < 0.05
