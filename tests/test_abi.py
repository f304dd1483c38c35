"""The C-ABI library loads and exports every entry point include/mlsd.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mlsd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlsd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_documented_calls():
    d = _declared()
    for name in ["mlsd_build_levels", "mlsd_solve_level", "mlsd_effective_diffusivity",
                 "mlsd_macro_step"]:
        assert name in d


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1510_00451_gb300", "libmlsd.so"))
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.mlsd_strerror.restype = ctypes.c_char_p
    assert lib.mlsd_strerror(-1) == b"invalid argument"


def test_invalid_problem_rejected_on_host():
    # argument validation happens before any device work
    import numpy as np
    import paper_1510_00451_gb300 as m
    p = m.mlsd_problem(n_macro=0, kappa=0.1, n_levels=1)
    h = ctypes.c_void_p()
    assert m.lib().mlsd_build_levels(ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert not h.value
    # a mode list that is not Hermitian-complete is rejected too
    k1 = np.array([1], np.int32); k2 = np.array([2], np.int32)
    re_ = np.array([0.5]); im = np.array([0.0])
    e = np.array([1.0, 4.0]); pn = np.array([32], np.int32)
    p = m.mlsd_problem(n_macro=4, kappa=0.1, n_modes=1, k1=k1.ctypes.data, k2=k2.ctypes.data,
                       re=re_.ctypes.data, im=im.ctypes.data, n_levels=1, band_edges=e.ctypes.data,
                       patch_n=pn.ctypes.data, cfl=0.2, t_burn_tau=8.0, t_avg_tau=4.0)
    assert m.lib().mlsd_build_levels(ctypes.byref(p), None, ctypes.byref(h)) == -1


def test_surrogate_calls_reject_bad_arguments_on_host():
    # the symmetry map and the training loop validate before any device work
    import paper_1510_00451_gb300 as m
    L = m.lib()
    fake = ctypes.c_void_p(16)                       # never dereferenced: rejected first
    assert L.mlsd_surrogate_symmetry(fake, fake, 4, 8, fake, fake, None) == -1      # g > 7
    assert L.mlsd_surrogate_symmetry(fake, fake, -1, 0, fake, fake, None) == -1     # n < 0
    assert L.mlsd_surrogate_symmetry(fake, fake, 4, 0, None, None, None) == -1      # no output
    assert L.mlsd_surrogate_symmetry(None, fake, 4, 0, fake, None, None) == -1      # X_out, no X
    # training without a handle
    assert L.mlsd_surrogate_train(None, fake, fake, 1024, 1, 128, ctypes.c_float(1e-3),
                                  ctypes.c_float(1e-3), 0, 1, None, None) == -1


def test_profiling_calls_reject_bad_arguments_on_host():
    # no handle, an unknown profiling mode, no output count: rejected before any work
    import paper_1510_00451_gb300 as m
    L = m.lib()
    n = ctypes.c_int32()
    assert L.mlsd_profile(None, 1) == -1
    assert L.mlsd_profile_collect_classes(None, 1, 4, None, None, None, ctypes.byref(n)) == -1
    assert L.mlsd_profile_collect_classes(None, 1, 0, None, None, None, None) == -1
