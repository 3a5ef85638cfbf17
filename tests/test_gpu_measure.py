"""kpp_measure_read, the read-bandwidth probe the benchmark reports beside
the copy bandwidth: a plausible rate from a buffer in L2 and one in HBM,
and its argument checks."""
import ctypes

import pytest
import torch

import paper_1908_02136_gb300 as kpp

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_read_rates_are_plausible():
    hbm = kpp.measure_read_gbs(1 << 30, 3, DEV)
    l2 = kpp.measure_read_gbs(32 << 20, 32, DEV)
    assert 1000.0 < hbm < 12_000.0  # a few TB/s from HBM3e
    assert l2 > hbm                 # a buffer resident in L2 reads faster


def test_argument_checks():
    buf = torch.zeros(1 << 20, dtype=torch.uint8, device=DEV)
    ms = ctypes.c_float(0.0)
    s = kpp._stream_handle(torch.device(DEV))
    assert kpp.kpp_measure_read(buf.data_ptr() + 4, 1024, 1, s, ctypes.byref(ms)) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_measure_read(buf.data_ptr(), 1000, 1, s, ctypes.byref(ms)) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_measure_read(buf.data_ptr(), 1024, 0, s, ctypes.byref(ms)) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_measure_read(None, 1024, 1, s, ctypes.byref(ms)) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_measure_read(buf.data_ptr(), 1024, 2, s, ctypes.byref(ms)) == kpp.OK
    assert ms.value > 0.0
