"""Learned warm start of the implicit step: data collection from the solver's
own trajectories, tensor-core training and evaluation against the plain
extrapolated guess.

The method of DisMech (arXiv 2311.18126, Sec. III-C) starts Newton from the
previous state; this module trains the library's BF16 MLP (dm_mlp, FP32
accumulation and master weights) to predict, per rod segment, the converged
step from the committed state, the velocities and the natural-curvature
controls of the new step.  Newton still runs to the same tolerance, so the
trajectory is the same to within that tolerance; the network can only change
how many iterations a step takes.  Every operation on device data here is a
library kernel (feature extraction, batch gather/normalisation, column
statistics, forward/backward GEMMs, Adam); torch supplies device memory and
the random minibatch indices.
"""
import time

import numpy as np
import torch

from . import dismech as dmx

N_FEAT = 61      # meaningful input columns of the 64-wide feature rows
N_OUT = 4        # position correction (3, local frame / edge length), twist


def collect(system, n_steps, controls=None, every=1):
    """Runs ``system`` for ``n_steps`` steps and returns (features [T*S, 64],
    targets [T*S, 4]) as CUDA float32 tensors, T = ceil(n_steps / every)
    sampled steps.  ``controls(k)`` (optional) returns the natural curvature
    of the whole batch for step k; it is applied before the features are
    taken, so the features see the controls of the step they predict."""
    S = system.ws_enable()
    T = (n_steps + every - 1) // every
    feats = torch.empty((T, S, 64), dtype=torch.float32, device="cuda")
    tgts = torch.empty((T, S, N_OUT), dtype=torch.float32, device="cuda")
    j = 0
    for k in range(n_steps):
        if controls is not None:
            system.set_natural_curvature(0, system.n_rods, controls(k))
        take = k % every == 0
        if take:
            system.ws_capture_features(feats[j])
        system.step(1, stats=False)
        if take:
            system.ws_capture_targets(tgts[j])
            j += 1
    torch.cuda.synchronize()
    return feats.view(T * S, 64), tgts.view(T * S, N_OUT)


def normalisation(feats, tgts):
    """132 floats: input mean [64], input std [64], output RMS [4] (library
    column-statistics kernel)."""
    fs = torch.empty((2, 64), dtype=torch.float32, device="cuda")
    ts = torch.empty((2, N_OUT), dtype=torch.float32, device="cuda")
    dmx.ws_column_stats(feats, fs)
    dmx.ws_column_stats(tgts, ts)
    torch.cuda.synchronize()
    f = fs.cpu().numpy()
    t = ts.cpu().numpy()
    rms = np.sqrt(t[0] ** 2 + t[1] ** 2)
    rms = np.maximum(rms, 1e-12)
    return np.concatenate([f[0], f[1], rms]).astype(np.float32)


def train(feats, tgts, iters=2000, batch=8192, lr=1e-3, lr_final=3e-5, seed=0,
          norm=None, mlp=None, log_every=0):
    """Trains the warm-start MLP on (features, targets) with Adam and a
    cosine learning-rate decay; returns (mlp, norm, losses)."""
    if norm is None:
        norm = normalisation(feats, tgts)
    if mlp is None:
        mlp = dmx.MLP(N_FEAT, N_OUT, seed=seed)
    norm_d = torch.from_numpy(norm).cuda()
    n = feats.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    X = torch.empty((batch, 64), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((batch, N_OUT), dtype=torch.float32, device="cuda")
    losses = []
    for it in range(iters):
        idx = torch.randint(0, n, (batch,), generator=g, device="cuda", dtype=torch.int64)
        dmx.ws_prepare_batch(feats, tgts, idx, norm_d, X, Y)
        c = 0.5 * (1.0 + np.cos(np.pi * it / max(iters - 1, 1)))
        loss = mlp.train_step(X, Y, lr_final + (lr - lr_final) * c)
        losses.append(loss)
        if log_every and it % log_every == 0:
            print("iter %d loss %.4e" % (it, loss), flush=True)
    return mlp, norm, losses


def validation_loss(mlp, norm, feats, tgts, batch=65536):
    """Mean squared error (normalised targets) of ``mlp`` over the rows of a
    held-out set, by the library's forward kernels."""
    norm_d = torch.from_numpy(norm).cuda()
    n = feats.shape[0]
    tot = 0.0
    cnt = 0
    X = torch.empty((batch, 64), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((batch, N_OUT), dtype=torch.float32, device="cuda")
    out = torch.empty((batch, 64), dtype=torch.float32, device="cuda")
    for s in range(0, n - batch + 1, batch):
        idx = torch.arange(s, s + batch, device="cuda", dtype=torch.int64)
        dmx.ws_prepare_batch(feats, tgts, idx, norm_d, X, Y)
        mlp.forward(X, out)
        tot += float(((out[:, :N_OUT] - Y) ** 2).sum())
        cnt += batch * N_OUT
    return tot / max(cnt, 1)


def run(system, n_steps, controls=None, mlp=None, norm=None):
    """Steps ``system`` ``n_steps`` times with the learned guess (mlp given)
    or the extrapolated one; returns (iterations per step [T, n_systems],
    wall seconds, converged residuals of the last step)."""
    if mlp is not None:
        system.ws_enable()
        system.ws_set_model(mlp, norm)
    its = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_steps):
        if controls is not None:
            system.set_natural_curvature(0, system.n_rods, controls(k))
        system.step(1, stats=True)
        its.append(system.iterations)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    res = system.residual
    if mlp is not None:
        system.ws_set_model(None)
    return np.array(its), wall, res
