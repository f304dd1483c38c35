"""Surrogate workflow over the C ABI: data from the method's own patch solves,
ensemble training with the library's training kernels, and the surrogate level
solve with its plain-solve fallback.  Argument marshalling and loop control
only; every computation runs in libmlsd's kernels.
"""
import math
import time

import numpy as np

from . import SUR_IN, Levels, Surrogate


def make_dataset(lv, level, bases):
    """Plain patch solves of one level for each base set: features X (bfloat16
    [n P][640]) and targets Y = asinh((K - B - E) SUR_Y_SCALE / tr(B)) (FP32 [n P][3])
    on the device, E the resummed perturbation series the features carry
    (mlsd.h); all of it in mlsd_surrogate_dataset.  A patch whose explicit solve
    went non-finite (MLSD_ENONFINITE: the step rule's stability bound fell short
    for it) gives no row; any other error raises."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    P = lv.P
    X = torch.empty(len(bases) * P, SUR_IN, dtype=torch.bfloat16, device=dev)
    Y = torch.empty(len(bases) * P, 3, dtype=torch.float32, device=dev)
    for i, B in enumerate(bases):
        Bd = torch.as_tensor(np.ascontiguousarray(B), dtype=torch.float64, device=dev)
        lv.surrogate_dataset(level, Bd, X[i * P:(i + 1) * P], Y[i * P:(i + 1) * P])
    rc = lv.status()
    if rc == -5:                                   # MLSD_ENONFINITE
        keep = torch.isfinite(Y).all(1)
        X, Y = X[keep], Y[keep]
    elif rc != 0:
        raise RuntimeError("patch solves reported error %d" % rc)
    return X, Y


def train(sur, X, Y, epochs, batch, lr, seed=0, lr_final=None, augment=False):
    """Adam on mean-squared error, each member on its own shuffles of the data
    (with augment, of every row's 8 images under the square's symmetries); the
    learning rate decays geometrically to lr_final over the run.  Returns the
    last epoch's mean loss per member (mlsd_surrogate_train)."""
    return sur.train(X, Y, epochs, batch, lr, lr_final=lr_final, seed=seed, augment=augment)


def k_error(K, Kref):
    """Per-patch relative Frobenius error of symmetric tensors (K11, K12, K22)."""
    d = K - Kref
    num = np.sqrt(d[:, 0] ** 2 + 2 * d[:, 1] ** 2 + d[:, 2] ** 2)
    den = np.sqrt(Kref[:, 0] ** 2 + 2 * Kref[:, 1] ** 2 + Kref[:, 2] ** 2)
    return num / den
