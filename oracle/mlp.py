"""ORACLE — test infrastructure only: FP64 numpy reference of the learned
Newton-guess network (6 -> 64 -> 64 -> 1, tanh hidden layers, linear output)
and of its training step (mean-squared loss, its gradient by the chain rule,
and the Adam update of Kingma & Ba 2015).  It shares no code with the CUDA
kernels; tests compare the kernels' forward pass, loss, gradients and Adam
steps with it, and pin it against finite differences and a closed form.

Parameter vector layout (4673 values): W1[6][64], b1[64], W2[64][64], b2[64],
w3[64], b3.
"""
import numpy as np

NIN, NH = 6, 64
SIZES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(theta, x):
    """Predictions y[n] and the hidden activations for inputs x[n, 6]."""
    P = unpack(theta)
    h1 = np.tanh(x @ P["W1"] + P["b1"])
    h2 = np.tanh(h1 @ P["W2"] + P["b2"])
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (h1, h2)


def loss_grad(theta, x, t):
    """Mean-squared loss mean((y - t)^2) and its gradient in the packed layout."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    P = unpack(theta)
    y, (h1, h2) = forward(theta, x)
    n = len(t)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, P["w3"]) * (1.0 - h2 * h2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"].T) * (1.0 - h1 * h1)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init(seed=0):
    """Glorot-uniform weights, zero biases (a common initialisation)."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shape in SIZES:
        if len(shape) == 2:
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            parts[name] = rng.uniform(-lim, lim, size=shape)
        elif name == "w3":
            lim = np.sqrt(6.0 / (NH + 1))
            parts[name] = rng.uniform(-lim, lim, size=shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts)
