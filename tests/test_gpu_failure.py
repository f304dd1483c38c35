"""Failure detection without a GPU fault: the bounded device waits.

The cluster-split patch kernels, the tensor-core inference kernels and the
persistent DNS kernels wait on mbarriers with a bound of about a second of SM
clocks; on expiry they latch MLSD_ETIMEOUT in a status word and return.  mlsd_check_wait_timeout runs
each wait helper on an mbarrier that never receives an arrival, with nothing
in flight, so the expiry path runs for real.  The test checks that the status
reports MLSD_ETIMEOUT once, within a few seconds, and that the next ordinary
solve on the same context succeeds and gives the same K as before.
"""
import time

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

MLSD_ETIMEOUT = -4


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_expires_and_the_context_survives(which):
    import torch
    import paper_1510_00451_gb300 as mlsd
    dev = torch.device("cuda:0")
    spec = inputs.cellular_hierarchy(2, 4)
    N = 4
    lv = mlsd.Levels(spec, 0.05, N, [1.0, 4.0, 16.0], [32, 32], n_burn_fixed=20, n_avg_fixed=20)
    K0 = torch.zeros(N * N, 3, dtype=torch.float64, device=dev)
    lv.effective_diffusivity(K0)
    assert lv.status() == 0
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    assert mlsd.lib().mlsd_check_wait_timeout(lv.h, which, stream) == 0
    rc = lv.status()                                   # synchronises
    elapsed = time.perf_counter() - t0
    assert rc == MLSD_ETIMEOUT
    assert 0.05 < elapsed < 20.0
    assert lv.status() == 0                            # reported once, then cleared
    K1 = torch.full_like(K0, float("nan"))
    lv.effective_diffusivity(K1)
    assert lv.status() == 0
    np.testing.assert_array_equal(K1.cpu().numpy(), K0.cpu().numpy())


def test_wait_check_rejects_unknown_kind():
    import torch
    import paper_1510_00451_gb300 as mlsd
    lv = mlsd.Levels(inputs.cellular_hierarchy(1, 4), 0.05, 2, [1.0, 4.0], [32],
                     n_burn_fixed=2, n_avg_fixed=2)
    assert mlsd.lib().mlsd_check_wait_timeout(lv.h, 3, None) == -1
    assert mlsd.lib().mlsd_check_wait_timeout(None, 0, None) == -1
