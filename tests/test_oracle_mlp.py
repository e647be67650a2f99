"""Pins of the surrogate-network oracle (oracle/mlp.py) against what the
definitions fix independently of its own code."""
import numpy as np
import pytest

from oracle import mlp as M


def test_silu_special_values():
    assert M.silu(np.array(0.0)) == 0.0
    assert M.dsilu(np.array(0.0)) == 0.5
    # large |z|: SiLU -> z (z >> 0) and -> 0 (z << 0); slope -> 1 and 0
    assert M.silu(np.array(40.0)) == pytest.approx(40.0, rel=1e-15)
    assert abs(M.silu(np.array(-40.0))) < 1e-15
    assert M.dsilu(np.array(40.0)) == pytest.approx(1.0, rel=1e-12)
    # derivative against a central difference at several points
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    assert np.allclose(M.dsilu(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), atol=1e-9)


def test_param_count_of_the_surrogate_shape():
    # 5 -> 128 -> 128 -> 128 -> 2
    assert M.param_count(M.dims(5, 128, 3, 2)) == 34050


@pytest.mark.parametrize("shape", [(3, 7, 2, 2), (5, 16, 3, 2)])
def test_gradient_against_finite_differences(shape):
    """Every component of the backpropagated gradient against a central
    difference of the loss (a dropped term, a transposed weight or a wrong
    activation derivative shows here)."""
    rng = np.random.default_rng(0)
    d = M.dims(*shape)
    P = M.param_count(d)
    theta = rng.normal(0, 0.5, P)
    x = rng.normal(size=(6, d[0]))
    t = rng.normal(size=(6, d[-1]))
    L, g = M.gradient(theta, d, x, t)
    assert L == pytest.approx(M.loss(theta, d, x, t), rel=1e-15)
    h = 1e-6
    num = np.empty(P)
    for k in range(P):
        e = np.zeros(P)
        e[k] = h
        num[k] = (M.loss(theta + e, d, x, t) - M.loss(theta - e, d, x, t)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-9)


def test_linear_case_is_fitted_exactly_by_adam():
    """depth-1 network whose hidden layer is near-linear around 0 cannot be
    exact; instead: the output layer alone of a network whose hidden
    activations are fixed is a least-squares problem.  With the hidden
    weights frozen at zero (SiLU(b) constant), Adam on the output bias
    converges to the mean of the targets."""
    d = M.dims(2, 4, 1, 1)
    P = M.param_count(d)
    theta = np.zeros(P)
    x = np.random.default_rng(1).normal(size=(8, 2))
    t = np.arange(8.0).reshape(8, 1)
    m = np.zeros(P)
    v = np.zeros(P)
    for it in range(1, 3001):
        _, g = M.gradient(theta, d, x, t)
        g[:-1] = 0.0  # only the output bias moves (the rest stays zero)
        theta, m, v = M.adam(theta, g, m, v, it, lr=0.05)
    assert theta[-1] == pytest.approx(t.mean(), abs=1e-6)


def test_adam_first_step_is_lr_times_sign():
    """After one step from m = v = 0 the bias-corrected moments are g and
    g^2, so the update is lr g / (|g| + eps)."""
    g = np.array([3.0, -0.2, 1e-3, 0.0])
    th, m, v = M.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_ensemble_stats():
    ys = np.array([[1.0, 2.0], [3.0, 2.0]])
    mu, sd = M.ensemble_stats(ys)
    assert np.allclose(mu, [2.0, 2.0]) and np.allclose(sd, [1.0, 0.0])
