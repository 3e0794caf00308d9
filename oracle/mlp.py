"""FP64 oracle of the learned preconditioner's network (test infrastructure).

Model (same parameter order as the library): xh = (f - mu) / sigma,
h1 = tanh(W1 xh + b1), h2 = tanh(W2 h1 + b2), z = w3 . h2 + b3,
D = softplus(z); loss = mean over samples of (log D - t)^2.
Forward and backward are written out layer by layer (chain rule), in numpy.
Pinned by central finite differences in tests/test_oracle_precond.py.
"""
import numpy as np

NF, NH = 8, 64
SIZES = [("mu", (NF,)), ("sigma", (NF,)), ("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)),
         ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
NTRAIN = NPARAM - 2 * NF


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def softplus(z):
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def forward(theta, F):
    """Returns (log D, cache) for feature rows F (n x 8)."""
    P = unpack(theta)
    xh = (np.asarray(F, dtype=np.float64) - P["mu"]) / P["sigma"]
    h1 = np.tanh(xh @ P["W1"].T + P["b1"])
    h2 = np.tanh(h1 @ P["W2"].T + P["b2"])
    z = h2 @ P["w3"] + P["b3"][0]
    sp = softplus(z)
    logD = np.where(z < -20.0, z, np.log(np.maximum(sp, 1e-300)))
    return logD, (P, xh, h1, h2, z, sp)


def loss_and_grad(theta, F, t):
    """Mean squared error of log D against t and its gradient with respect to
    the trained parameters (W1 onwards), in the library's parameter order."""
    logD, (P, xh, h1, h2, z, sp) = forward(theta, F)
    n = F.shape[0]
    err = logD - t
    loss = np.mean(err * err)
    sig = 1.0 / (1.0 + np.exp(-z))
    dlog = np.where(z < -20.0, 1.0, sig / sp)          # d log softplus(z) / dz
    d3 = 2.0 * err * dlog / n                           # d loss / dz
    g_w3 = h2.T @ d3
    g_b3 = np.array([d3.sum()])
    d2 = np.outer(d3, P["w3"]) * (1.0 - h2 * h2)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (1.0 - h1 * h1)
    g_W1 = d1.T @ xh
    g_b1 = d1.sum(axis=0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
    return loss, grad


def init_params(rng, mu, sigma):
    """Xavier-uniform weights, zero biases, given feature standardisation."""
    def xavier(fan_out, fan_in):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_out, fan_in))
    parts = [np.asarray(mu, float), np.asarray(sigma, float), xavier(NH, NF).ravel(), np.zeros(NH),
             xavier(NH, NH).ravel(), np.zeros(NH), xavier(1, NH).ravel(), np.zeros(1)]
    return np.concatenate(parts)


def adam_step(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of the trained parameters (from W1)."""
    theta = np.array(theta, dtype=np.float64)
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta[2 * NF:] -= lr * mh / (np.sqrt(vh) + eps)
    return theta, m, v
