"""kpp_seed_noalloc: the seeding entry point for callers that cannot
allocate device memory (it uses a fixed scratch array inside the library
instead of a caller workspace).  It runs the same persistent kernel as
kpp_seed, so on the same problem and options it must give bit-identical
results, call after call, although every call reuses the same array.

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
SCRATCH_BYTES = 16 * 1024  # the fixed array's size, stated in include/kpp.h


def _outs(N, K):
    return (torch.full((K,), -7, dtype=torch.int64, device=DEV),
            torch.empty(N, dtype=torch.float32, device=DEV),
            torch.empty(1, dtype=torch.float64, device=DEV))


def _noalloc(x, K, seed, opts=None, outs=None, sync_status=True):
    N, d = x.shape
    idx, d2, phi = outs if outs is not None else _outs(N, K)
    status = ctypes.c_int32(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = kpp.kpp_seed_noalloc(x.data_ptr(), None, N, d, K, kpp.F32, seed, 0, idx.data_ptr(),
                              d2.data_ptr(), phi.data_ptr(), stream, opts,
                              status if sync_status else None)
    return rc, status.value, idx, d2, phi


def _reference(x, K, seed, opts=None):
    o = dict(opts or {}, form=kpp.FORM_PERSISTENT)
    idx, d2, phi = kpp.seed(x, K, seed, opts=o)
    return idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0])


def _same(ref, idx, d2, phi):
    assert np.array_equal(idx.cpu().numpy(), ref[0])
    assert np.array_equal(d2.cpu().numpy(), ref[1])
    assert float(phi.cpu()[0]) == ref[2]


def test_noalloc_matches_kpp_seed_twice_in_a_row():
    for N, d, K, seed in [(200_003, 32, 64, 3), (50_000, 8, 40, 5)]:
        x = torch.from_numpy(datagen.gmm(N, d, 32, seed=N)).to(DEV)
        ref = _reference(x, K, seed)
        for _ in range(2):  # the second call sees the first call's leftovers
            rc, st, idx, d2, phi = _noalloc(x, K, seed)
            assert rc == kpp.OK and st == kpp.OK
            _same(ref, idx, d2, phi)


def test_noalloc_without_status_stays_asynchronous():
    x = torch.from_numpy(datagen.gmm(80_000, 16, 16, seed=4)).to(DEV)
    ref = _reference(x, 24, 9)
    rc, st, idx, d2, phi = _noalloc(x, 24, 9, sync_status=False)
    assert rc == kpp.OK and st == -1  # no status was written back
    torch.cuda.current_stream().synchronize()
    _same(ref, idx, d2, phi)


def test_noalloc_allocates_no_device_memory():
    x = torch.from_numpy(datagen.gmm(100_000, 32, 16, seed=6)).to(DEV)
    outs = _outs(100_000, 32)
    rc, st, *_ = _noalloc(x, 32, 2, outs=outs)  # warm: library loaded, address known
    assert rc == kpp.OK and st == kpp.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc, st, *_ = _noalloc(x, 32, 2, outs=outs)
        assert rc == kpp.OK and st == kpp.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_plans_beyond_the_fixed_scratch():
    """A plan needs 256 + 64 bytes per CTA (rounded up to 256) of scratch:
    more than 252 CTAs do not fit the 16 KiB array.  Such plans arise only
    when several of the 512-thread CTAs can share an SM; the entry point must
    reject exactly those plans, before writing anything."""
    N = 2_500_000
    seen_reject = False
    for d in (2, 4, 8):
        x = torch.from_numpy(datagen.integer_points(N, d, seed=d, n_comp=8)).to(DEV)
        for per_sm in (1, 2, 3, 4):
            opts = {"ctas_per_sm": per_sm, "min_rows_per_cta": 256}
            st, plan = kpp.kpp_describe(N, d, 8, kpp.F32,
                                        dict(opts, form=kpp.FORM_PERSISTENT))
            assert st == kpp.OK
            outs = _outs(N, 8)
            rc, dst, idx, d2, phi = _noalloc(x, 8, 1, opts=opts, outs=outs)
            if plan.workspace_bytes > SCRATCH_BYTES:
                seen_reject = True
                assert plan.grid > 252
                assert rc == kpp.ERR_WORKSPACE and dst == -1
                torch.cuda.synchronize()
                assert bool((idx == -7).all())  # nothing was enqueued
            else:
                assert plan.grid <= 252
                assert rc == kpp.OK and dst == kpp.OK
                _same(_reference(x, 8, 1, opts), idx, d2, phi)
    if not seen_reject:
        # every plan this device makes fits: one 512-thread CTA per SM
        assert torch.cuda.get_device_properties(0).multi_processor_count <= 252
