"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package only builds input data (mode lists of stream functions, initial
fields, random datasets).  It holds none of the method's arithmetic: no band
decomposition, no patch solve, no closed form.
"""
from .flows import (  # noqa: F401
    Spectrum, cellular_two_scale, cellular_hierarchy, continuous_spectrum,
    shear_x1, shear_x2, shear_diag, gaussian_u0, splitmix64, config_problem, mlp_init,
    random_bases, cellular, step_u0,
)
