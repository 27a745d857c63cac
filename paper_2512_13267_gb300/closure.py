"""Learned-closure workflow over the C ABI: collect (input, stress increment)
pairs from plain coupled macro steps, normalise, train the ensemble on the
GPU, and compare a surrogate-gated run with a plain one.

The closure is not part of the paper; it is this library's surrogate layer.
Inputs: the 16 past velocity gradients (Lxx, Lxy, Lyx, Lyy) of a particle,
oldest first, and its current polymer stress (pi_xx, pi_xy, pi_yy); target:
the increment of (pi_xx, pi_xy, pi_yy) over one macro step.
"""
import time

import numpy as np

from . import lhmm

N_IN = 67
N_OUT = 3
HIST = 16
STRESS_COLS = [0, 3, 1]  # xx, xy, yy in the micro stress layout


def collect_pairs(coupled, n_steps, skip=HIST):
    """Run n_steps plain macro steps (gate off, closure attached) and return
    inputs X (m x 67) and targets T (m x 3); the first `skip` steps only fill
    the gradient history."""
    coupled.enable_gate(False)
    Xs, Ts = [], []
    for k in range(n_steps):
        coupled.step(1, use_graph=True)
        if k < skip:
            continue
        X = coupled.closure_inputs()
        _, st = coupled.exchange()
        T = st[:, STRESS_COLS].astype(np.float32) - X[:, 64:67]
        Xs.append(X)
        Ts.append(T)
    if not Xs:
        return np.zeros((0, N_IN), np.float32), np.zeros((0, N_OUT), np.float32)
    return np.concatenate(Xs), np.concatenate(Ts)


def normalization(X, T, floor=1e-6):
    mean = X.mean(axis=0)
    std = np.maximum(X.std(axis=0), floor)
    scale = np.maximum(T.std(axis=0), floor)
    return mean.astype(np.float32), std.astype(np.float32), scale.astype(np.float32)


def train(closure, X, T, steps, batch=4096, lr=1e-3, weight_decay=1e-4, seed=0, log_every=0):
    """AdamW on bootstrap batches (each member draws its own rows).  Returns the
    per-member loss history (every log_every steps) and the wall time."""
    import torch
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    batch = max(32, min(batch, (n // 32) * 32))
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T, np.float32)).cuda()
    loss = torch.zeros(closure.members, dtype=torch.float32, device="cuda")
    rows_all = torch.from_numpy(
        rng.integers(0, n, size=(min(steps, 64), closure.members, batch)).astype(np.int32)).cuda()
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        rows = rows_all[k % rows_all.shape[0]]
        if k % rows_all.shape[0] == 0 and k > 0:
            rows_all = torch.randint(0, n, rows_all.shape, dtype=torch.int32, device="cuda")
        closure.train_step(Xd, Td, batch, lr, weight_decay, rows_dev=rows, loss_dev=loss)
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append(loss.cpu().numpy().copy())
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def binned_profiles(y, stress6, Ly, nbins=16):
    """y-binned pi_xy and N1 = pi_xx - pi_yy of the fluid particles."""
    k = np.minimum((np.asarray(y) / Ly * nbins).astype(int), nbins - 1)
    cnt = np.maximum(np.bincount(k, minlength=nbins), 1)
    pxy = np.bincount(k, weights=stress6[:, 3], minlength=nbins) / cnt
    n1 = np.bincount(k, weights=stress6[:, 0] - stress6[:, 1], minlength=nbins) / cnt
    return pxy, n1


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
