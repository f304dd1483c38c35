"""Surrogate workflow over the C ABI: data from the method's own patch solves,
ensemble training with the library's training kernels, and the surrogate level
solve with its plain-solve fallback.  Argument marshalling and loop control
only; every computation runs in libmlsd's kernels.
"""
import math
import time

import numpy as np

from . import SUR_FEATURES, SUR_IN, SUR_Q_SCALE, SUR_Y_SCALE, Levels, Surrogate


def make_dataset(lv, level, bases):
    """Plain patch solves of one level for each base set: features X (bfloat16
    [n P][640]) and targets Y = (K - B - Q) SUR_Y_SCALE / tr(B) (FP32 [n P][3])
    on the device, Q the second-order estimate the features carry (mlsd.h)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    P = lv.P
    X = torch.empty(len(bases) * P, SUR_IN, dtype=torch.bfloat16, device=dev)
    Y = torch.empty(len(bases) * P, 3, dtype=torch.float32, device=dev)
    K = torch.empty(P, 3, dtype=torch.float64, device=dev)
    F = torch.empty(P, SUR_FEATURES, dtype=torch.float32, device=dev)
    for i, B in enumerate(bases):
        Bd = torch.as_tensor(np.ascontiguousarray(B), dtype=torch.float64, device=dev)
        lv.solve_level(level, Bd, K)
        lv.features(level, Bd, X[i * P:(i + 1) * P], F)
        tr = (Bd[:, 0] + Bd[:, 2]).unsqueeze(1)
        q = F[:, 582:585].double() / SUR_Q_SCALE            # Q / tr(B)
        Y[i * P:(i + 1) * P] = (((K - Bd) / tr - q) * SUR_Y_SCALE).float()
    if lv.status() != 0:
        raise RuntimeError("patch solves reported an error")
    return X, Y


def train(sur, X, Y, epochs, batch, lr, seed=0, lr_final=None):
    """Adam on mean-squared error, each member on its own shuffles of the data;
    the learning rate decays geometrically to lr_final over the run.  Returns
    the last epoch's mean loss per member."""
    import torch
    n = X.shape[0]
    steps = max(1, n // batch)
    total = epochs * steps
    lr_final = lr if lr_final is None else lr_final
    g = torch.Generator(device=X.device)
    losses = []
    for m in range(sur.members):
        g.manual_seed(seed * 7919 + m)
        t = 0
        last = []
        for ep in range(epochs):
            perm = torch.randperm(n, device=X.device, generator=g)
            for s in range(steps):
                idx = perm[s * batch:(s + 1) * batch]
                xb = X.index_select(0, idx)
                yb = Y.index_select(0, idx)
                r = lr * (lr_final / lr) ** (t / max(1, total - 1))
                want = ep == epochs - 1
                loss = sur.train_step(m, xb, yb, r, want_loss=want)
                if want:
                    last.append(loss)
                t += 1
        losses.append(float(np.mean(last)))
    return losses


def k_error(K, Kref):
    """Per-patch relative Frobenius error of symmetric tensors (K11, K12, K22)."""
    d = K - Kref
    num = np.sqrt(d[:, 0] ** 2 + 2 * d[:, 1] ** 2 + d[:, 2] ** 2)
    den = np.sqrt(Kref[:, 0] ** 2 + 2 * Kref[:, 1] ** 2 + Kref[:, 2] ** 2)
    return num / den
