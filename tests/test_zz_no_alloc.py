"""kpp_seed_noalloc: the seeding entry point for callers that cannot
allocate device memory (it uses a fixed scratch array inside the library
instead of a caller workspace).  It must give the same result as kpp_seed on
the same problem, call after call, since every call reuses the same array.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _noalloc(x, K, seed, opts=None):
    N, d = x.shape
    idx = torch.empty(K, dtype=torch.int64, device=DEV)
    d2 = torch.empty(N, dtype=torch.float32, device=DEV)
    phi = torch.empty(1, dtype=torch.float64, device=DEV)
    status = ctypes.c_int32(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = kpp.kpp_seed_noalloc(x.data_ptr(), None, N, d, K, kpp.F32, seed, 0, idx.data_ptr(),
                              d2.data_ptr(), phi.data_ptr(), stream, opts, status)
    return rc, status.value, idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0])


def test_noalloc_matches_kpp_seed_twice_in_a_row():
    for N, d, K, seed in [(200_003, 32, 64, 3), (50_000, 8, 40, 5)]:
        x = torch.from_numpy(datagen.gmm(N, d, 32, seed=N)).to(DEV)
        idx, d2, phi = kpp.seed(x, K, seed, opts={"form": kpp.FORM_PERSISTENT})
        idx, d2, phi = idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0])
        for _ in range(2):  # the second call sees the first call's leftovers
            rc, st, nidx, nd2, nphi = _noalloc(x, K, seed)
            assert rc == kpp.OK and st == kpp.OK
            assert np.array_equal(nidx, idx)
            np.testing.assert_allclose(nd2, d2, rtol=1e-5, atol=0)
            assert abs(nphi - phi) <= 1e-5 * phi
