"""The allocation-free coarse-graining entry point against the allocating one.

mlsd_coarse_grain_noalloc serves callers that cannot allocate device memory;
its scratch is a fixed device array inside the library.  Called through the C
ABI twice in a row on different fields, it must give the same coarse field and
FP64 mass as mlsd_coarse_grain (same tolerance as the other coarse-graining
tests), so nothing from the first call leaks into the second.  Collected last
on purpose; passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    import paper_1510_00451_gb300 as mlsd
    from inputs import flows
    lib = mlsd.lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    nf, N = 512, 64
    rng = np.random.default_rng(12)
    fields = [flows.gaussian_u0(nf, 0.7).astype(np.float32),
              rng.standard_normal((nf, nf)).astype(np.float32)]
    for u_host in fields:
        u = torch.tensor(u_host, device=dev)
        U_ref = torch.zeros(N, N, dtype=torch.float32, device=dev)
        U_new = torch.full((N, N), float("nan"), dtype=torch.float32, device=dev)
        m_ref, m_new = ctypes.c_double(), ctypes.c_double()
        assert lib.mlsd_coarse_grain(nf, u.data_ptr(), N, U_ref.data_ptr(),
                                     ctypes.byref(m_ref), stream) == 0
        assert lib.mlsd_coarse_grain_noalloc(nf, u.data_ptr(), N, U_new.data_ptr(),
                                             ctypes.byref(m_new), stream) == 0
        torch.cuda.synchronize()
        a, b = U_new.cpu().numpy(), U_ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
        assert m_new.value == pytest.approx(m_ref.value, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("nf,N,with_mass", [(512, 64, False), (1024, 256, True), (1024, 256, False)])
def test_noalloc_without_mass_and_at_the_scratch_limit(nf, N, with_mass):
    # without a mass pointer the entry point passes no scratch to the box sums;
    # n_macro = 256 fills the scratch array exactly
    import torch
    import paper_1510_00451_gb300 as mlsd
    lib = mlsd.lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(nf + N)
    for _ in range(2):
        u = torch.tensor(rng.standard_normal((nf, nf)).astype(np.float32), device=dev)
        U_ref = torch.zeros(N, N, dtype=torch.float32, device=dev)
        U_new = torch.full((N, N), float("nan"), dtype=torch.float32, device=dev)
        m_ref, m_new = ctypes.c_double(), ctypes.c_double()
        assert lib.mlsd_coarse_grain(nf, u.data_ptr(), N, U_ref.data_ptr(),
                                     ctypes.byref(m_ref) if with_mass else None, stream) == 0
        assert lib.mlsd_coarse_grain_noalloc(nf, u.data_ptr(), N, U_new.data_ptr(),
                                             ctypes.byref(m_new) if with_mass else None,
                                             stream) == 0
        torch.cuda.synchronize()
        a, b = U_new.cpu().numpy(), U_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
        if with_mass:
            assert m_new.value == pytest.approx(m_ref.value, rel=1e-6, abs=1e-9)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    import paper_1510_00451_gb300 as mlsd
    lib = mlsd.lib()
    u = torch.zeros(1024, 1024, dtype=torch.float32, device="cuda:0")
    U = torch.zeros(512, 512, dtype=torch.float32, device="cuda:0")
    rc = lib.mlsd_coarse_grain_noalloc(1024, u.data_ptr(), 512, U.data_ptr(), None,
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == -1                                   # MLSD_EINVAL: n_macro > 256
