"""Learned Newton initial guess: harvest, training and loading (marshalling only).

1. harvest: run the scheme (flat form) with grp_set_harvest on; the flux
   kernel and the repair rounds record the
   network inputs and the converged FP64 target v = ln(p*/p_TR) / (-0.005 s^3)
   (the correction of the two-rarefaction estimate p_TR, normalised by the cube
   of the shock strength s = ln(p_TR / min(pL, pR))) at the interfaces the
   network serves.
2. train: mini-batch Adam on the mean-squared error, every batch through the
   library's FP32 kernels grp_mlp_loss_grad and grp_mlp_adam.
3. load: grp_set_guess_model with the weights and the input box of the data.
torch provides the device memory and the random permutation of the samples.
"""
import math

import numpy as np

from . import grprec

NIN, NH = 6, 64
NPARAM = grprec.GRP_MLP_NPARAM


def harvest(runs, capacity=2_000_000, log2_stride=2, device=0):
    """runs: iterable of (prob, avg, lim_minus, lim_plus, n_steps).  Returns a
    float32 device tensor [n, 8]: 6 inputs, target v, Newton iterations."""
    import torch
    dev = torch.device("cuda", device)
    out = []
    for prob, avg, lm, lp, n_steps in runs:
        left = capacity - sum(int(r.shape[0]) for r in out)
        if left <= 0:
            break
        rec = torch.empty((left, 8), dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        s = grprec.Solver(prob, device=device)
        s.set_launch(grprec.GRP_LAUNCH_FLAT)        # the flat form's repair rounds record too
        s.set_harvest(rec, cnt, log2_stride)
        s.set_initial(avg, lm, lp)
        s.step(n_steps)
        s.get_stats()                               # synchronises
        n = min(int(cnt.item()), left)
        out.append(rec[:n].clone())
        s.close()
    return torch.cat(out) if out else torch.empty((0, 8), dtype=torch.float32, device=dev)


def init_weights(seed=0, device=0):
    """Glorot-uniform weight matrices and output weights, zero biases, as a
    float32 device tensor in the parameter layout of the library."""
    import torch
    g = torch.Generator().manual_seed(seed)

    def uni(shape, fan_in, fan_out):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return (torch.rand(shape, generator=g, dtype=torch.float64) * 2 - 1) * lim

    parts = [uni((NIN, NH), NIN, NH), torch.zeros(NH, dtype=torch.float64),
             uni((NH, NH), NH, NH), torch.zeros(NH, dtype=torch.float64),
             uni((NH,), NH, 1), torch.zeros(1, dtype=torch.float64)]
    w = torch.cat([p.reshape(-1) for p in parts]).to(torch.float32)
    assert w.numel() == NPARAM
    return w.to(torch.device("cuda", device))


def input_box(x, margin=0.05):
    """lo[6], hi[6] of the training inputs, widened by `margin` of each range."""
    import torch
    lo = x.min(dim=0).values
    hi = x.max(dim=0).values
    pad = (hi - lo) * margin
    return torch.cat([lo - pad, hi + pad]).contiguous()


def train(x, t, epochs=800, batch=1024, lr=3e-3, lr_end=1e-5, seed=0, weights=None, verbose=False,
          max_steps=50_000):
    """Mini-batch Adam, learning rate decayed geometrically from lr to lr_end,
    at most max_steps optimizer steps (fewer epochs on large sets).
    x: float32 device [n, 6]; t: float32 device [n].  Returns (weights, losses
    per epoch)."""
    import torch
    dev = x.device
    n = int(x.shape[0])
    w = init_weights(seed, dev.index or 0) if weights is None else weights.clone()
    m = torch.zeros(NPARAM, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    grad = torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.empty(grprec.mlp_work_floats(batch), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(seed)
    nb = max(1, n // batch)
    epochs = max(1, min(epochs, -(-max_steps // nb)))
    decay = (lr_end / lr) ** (1.0 / max(1, epochs * nb - 1))
    step, rate, hist = 0, lr, []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=dev)
        acc = torch.zeros((), dtype=torch.float64, device=dev)
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            xb = x[idx].contiguous()
            tb = t[idx].contiguous()
            grprec.grp_mlp_loss_grad(w, xb, tb, grad, loss, work)
            step += 1
            grprec.grp_mlp_adam(w, grad, m, v, step, rate)
            rate *= decay
            acc += loss[0].double()
        hist.append(float(acc.item()) / nb)
        if verbose:
            print("epoch %3d  mse %.3e" % (ep, hist[-1]))
    return w, hist


def predict(w, x):
    import torch
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    grprec.grp_mlp_forward(w, x.contiguous(), y)
    return y


def states_from_features(x, gamma=1.4):
    """A Riemann problem with the given network inputs (float device [n, 6]):
    the representative with rbar = pbar = 1 and ubar = 0 of the family that the
    scaling and Galilean symmetries map onto one input vector.  Returns
    conserved QL, QR as float64 device [3, n] (rho, m, E)."""
    import torch
    x = x.double()
    cbar = math.sqrt(gamma)
    rl, rr = torch.exp(x[:, 0]), torch.exp(x[:, 1])
    pl, pr = torch.exp(x[:, 2]), torch.exp(x[:, 3])
    ul, ur = x[:, 4] * cbar, x[:, 5] * cbar

    def cons(r, u, p):
        return torch.stack([r, r * u, p / (gamma - 1.0) + 0.5 * r * u * u]).contiguous()
    return cons(rl, ul, pl), cons(rr, ur, pr)


def fit_from_records(records, val_fraction=0.1, seed=0, max_records=120_000, **kw):
    """Split harvested records (a random subset of at most max_records),
    train, and report the validation RMS error of the target v and the input
    box."""
    import torch
    gen = torch.Generator(device=records.device).manual_seed(seed + 1)
    perm = torch.randperm(int(records.shape[0]), generator=gen, device=records.device)[:max_records]
    n = int(perm.shape[0])
    nv = max(1, int(n * val_fraction))
    val, tr = records[perm[:nv]], records[perm[nv:]]
    x, t = tr[:, :6].contiguous(), tr[:, 6].contiguous()
    w, hist = train(x, t, seed=seed, **kw)
    yv = predict(w, val[:, :6].contiguous())
    rms = float(torch.sqrt(torch.mean((yv - val[:, 6]) ** 2)).item())
    return w, input_box(x), dict(train_mse=hist, val_rms=rms, n_train=int(x.shape[0]), n_val=nv)
