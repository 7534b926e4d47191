"""Pins of the FP64 reference network used to check the training kernels:
the analytic gradient against central finite differences, and one Adam step
against the update written out for a single coordinate."""
import numpy as np

from oracle import mlp as R


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    theta = R.init(seed=1) + 0.01 * rng.normal(size=R.NPARAM)
    x = rng.normal(size=(40, 6))
    t = rng.normal(size=40)
    loss, g = R.loss_grad(theta, x, t)
    idx = rng.choice(R.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [R.NPARAM - 1, 0]])        # include b3 and W1[0][0]
    h = 1e-6
    for i in idx:
        e = np.zeros(R.NPARAM)
        e[i] = h
        fd = (R.loss_grad(theta + e, x, t)[0] - R.loss_grad(theta - e, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), i


def test_adam_step_written_out():
    theta = np.array([1.0, -2.0])
    grad = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    th, m1, v1 = R.adam_step(theta, grad, m, v, 1, lr=0.1)
    # first step: mhat = g, vhat = g^2 -> update = lr * g / (|g| + eps)
    assert np.allclose(th, theta - 0.1 * grad / (np.abs(grad) + 1e-8), rtol=1e-12)
    th2, _, _ = R.adam_step(th, grad, m1, v1, 2, lr=0.1)
    mhat = (0.9 * m1 + 0.1 * grad) / (1 - 0.9 ** 2)
    vhat = (0.999 * v1 + 0.001 * grad ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(th2, th - 0.1 * mhat / (np.sqrt(vhat) + 1e-8), rtol=1e-12)


def test_layout_size():
    assert R.NPARAM == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4673
