"""Surrogate data set from the method's own patch solves (over the C ABI), and
the relative K error the surrogate is judged by.  Argument marshalling only;
every computation of the path runs in libmlsd's kernels (training is
Surrogate.train, mlsd_surrogate_train).
"""
import numpy as np

from . import SUR_IN


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


def k_error(K, Kref):
    """Per-patch relative Frobenius error of symmetric tensors (K11, K12, K22)."""
    d = K - Kref
    num = np.sqrt(d[:, 0] ** 2 + 2 * d[:, 1] ** 2 + d[:, 2] ** 2)
    den = np.sqrt(Kref[:, 0] ** 2 + 2 * Kref[:, 1] ** 2 + Kref[:, 2] ** 2)
    return num / den
