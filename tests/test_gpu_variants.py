"""Every thread-block tiling the autotuner may choose, forced one at a time
(MLSD_TILE), against the oracle on the same seeded patches (the "t" tilings keep
the per-cell stencil coefficients in tensor memory)."""
import os
import re

import numpy as np
import pytest

from inputs import flows
from tests._parity import oracle_level, random_spd, rel_l2

pytestmark = pytest.mark.gpu

FP32 = {32: ["4x8", "4x8s", "4x8r", "4x4", "2x8", "2x4", "4x4p", "2x4p", "4x2p"],
        64: ["4x8", "4x8m3", "4x8m3s", "4x8m3r", "4x8m2r", "4x4r", "4x4m2r", "4x4m2s", "4x4", "2x8",
             "8x4", "2x4", "4x4p", "2x4p", "4x2p", "4x8m4t", "4x8m4l"],
        128: ["4x8m3c4", "4x8m3c4s", "4x8m3c4n", "4x8m3c4b", "4x4c4b", "4x8c2", "4x4c4",
              "2x8m2c4b", "2x8m2c4", "4x8m3c4d", "4x8m2c4d", "4x8t", "4x8m2c2bt", "4x8l", "4x8m2c2bl"],
        256: ["4x8c8", "4x8c8s", "4x8m2c8s", "4x8c8n", "4x8m2c8n", "4x8m3c16n", "4x8c8b", "4x8m3c16b",
              "4x4c8b", "4x4c8", "4x8m3c16", "2x8c8b", "2x8c8", "4x8c8d", "4x8m3c16d", "4x8m2c16d",
              "2x8c8d", "4x8c4bt", "4x8m2c8bt", "4x8c4bl", "4x8m2c8bl"]}
FP64 = {32: ["2x4", "4x4"], 64: ["2x4", "4x4"]}
CASES = ([(n, "fp32", t) for n, ts in FP32.items() for t in ts]
         + [(n, "fp64", t) for n, ts in FP64.items() for t in ts])
_REF = {}


def _ref(n, prec, spec, edges, pn, N, B):
    key = (n, prec)
    if key not in _REF:
        _REF[key] = oracle_level(spec, edges, pn, 2, N, B, list(range(N * N)),
                                 n_burn_fixed=90, n_avg_fixed=70, want_w=True)
    return _REF[key]


@pytest.mark.parametrize("n,prec,tile", CASES)
def test_tiling_parity(n, prec, tile, monkeypatch):
    import torch
    import paper_1510_00451_gb300 as mlsd
    monkeypatch.setenv("MLSD_TILE", tile)
    spec = flows.cellular_two_scale(0.8, 0.5, 4)
    edges, pn, N = [1, 4, 8], [n, n], (3 if n <= 64 else 2)
    lv = mlsd.Levels(spec, 0.03, N, edges, pn, n_burn_fixed=90, n_avg_fixed=70, precision=prec)
    info = lv.info(2)
    m = re.fullmatch(r"(\d+x\d+)(?:m\d)?(?:c(\d+))?(p?)([snbdr]?)([tl]?)", tile)
    assert f"{info['tile_bx']}x{info['tile_by']}" == m.group(1) and info["packed"] == (m.group(3) == "p")
    assert info["cluster"] == (int(m.group(2)) if m.group(2) else 1)
    assert info["split"] == {"": 0, "s": 1, "n": 2, "b": 3, "r": 4, "d": 5}[m.group(4)]
    assert info["coef_tmem"] == {"": 0, "t": 1, "l": 2}[m.group(5)]
    B = random_spd(N * N, np.random.default_rng(n), 0.03, 0.1)
    dev = torch.device("cuda:0")
    dtype = torch.float64 if prec == "fp64" else torch.float32
    Kb = torch.tensor(B, dtype=torch.float64, device=dev)
    Ko = torch.zeros_like(Kb)
    w = torch.zeros(N * N, 2, n, n, dtype=dtype, device=dev)
    lv.solve_level(2, Kb, Ko, w)
    assert lv.status() == 0
    K, w = Ko.cpu().numpy(), w.cpu().numpy()
    ktol, wtol = (1e-4, 1e-5) if prec == "fp32" else (1e-10, 1e-10)
    for p, (Kr, wr) in enumerate(_ref(n, prec, spec, edges, pn, N, B)):
        assert rel_l2(K[p], Kr) < ktol, (p, K[p], Kr)
        assert rel_l2(w[p], wr) < wtol
