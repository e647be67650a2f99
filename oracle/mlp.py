"""FP64 CPU oracle of the surrogate network (TEST INFRASTRUCTURE ONLY: only
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it).

The paper has no learned part.  The network follows the standard
definitions, one array operation at a time in float64 numpy:
  - SiLU(z) = z s(z) with the logistic s(z) = 1 / (1 + e^-z)
    (Elfwing, Uchibe & Doya 2018); SiLU'(z) = s(z) (1 + z (1 - s(z)));
  - a member: hidden layers h_l = SiLU(W_l h_{l-1} + b_l), linear output;
  - loss: mean over rows and outputs of (y - t)^2; its gradient by the chain
    rule written out layer by layer (backpropagation);
  - Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.
Parameter vector of a member: per layer W (d_out x d_in, row-major) then b.

Pinned in tests/test_oracle_mlp.py against central finite differences of
the loss, SiLU's special values, Adam's first step (lr * sign(g) up to eps)
and a linear network fitted exactly."""
import numpy as np


def dims(n_in, width, depth, n_out):
    return [n_in] + [width] * depth + [n_out]


def param_count(d):
    return sum(d[l] * d[l - 1] + d[l] for l in range(1, len(d)))


def unpack(theta, d):
    """[(W_1, b_1), ..., (W_L, b_L)] views of one member's vector."""
    out, k = [], 0
    for l in range(1, len(d)):
        W = theta[k:k + d[l] * d[l - 1]].reshape(d[l], d[l - 1])
        k += d[l] * d[l - 1]
        b = theta[k:k + d[l]]
        k += d[l]
        out.append((W, b))
    return out


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(theta, d, x):
    """Outputs (rows x n_out) and the pre-activations of every layer."""
    layers = unpack(np.asarray(theta, np.float64), d)
    h = np.asarray(x, np.float64)
    zs, hs = [], [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = silu(z) if l < len(layers) - 1 else z
        hs.append(h)
    return h, zs, hs


def loss(theta, d, x, t):
    y, _, _ = forward(theta, d, x)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def gradient(theta, d, x, t):
    """(loss, dloss/dtheta) by backpropagation."""
    layers = unpack(np.asarray(theta, np.float64), d)
    y, zs, hs = forward(theta, d, x)
    t = np.asarray(t, np.float64)
    n = y.size
    L = float(np.mean((y - t) ** 2))
    delta = 2.0 * (y - t) / n          # dL/dz of the (linear) output layer
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = delta.T @ hs[l]           # sum over rows of delta_o h_i
        gb = delta.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            delta = (delta @ W) * dsilu(zs[l - 1])
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, g


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t = the step's index, from 1); returns theta, m, v."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def ensemble_stats(ys):
    """Mean and (population) standard deviation over the members (axis 0)."""
    ys = np.asarray(ys, np.float64)
    mu = ys.mean(axis=0)
    return mu, np.sqrt(((ys - mu) ** 2).mean(axis=0))
