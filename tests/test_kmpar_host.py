"""Host-side parts of k-means|| (no GPU): the default candidate room, the
workspace sizing of the C ABI and argument checks that fail before any CUDA
call."""
import math

import pytest

import paper_1908_02136_gb300 as kpp


def test_default_candidate_room():
    # c_0 plus, per round, ell + 8 standard deviations of a Bernoulli sum
    # (variance <= ell) and a margin
    for ell in (1.0, 16.0, 512.0, 2048.0):
        for rounds in (0, 1, 5):
            cap = kpp.kmeans_par_cap(ell, rounds)
            assert cap >= 1 + rounds * (ell + 8 * math.sqrt(ell))
            assert cap <= 1 + rounds * (ell + 8 * math.sqrt(ell) + 17)
    assert kpp.kmeans_par_cap(-3.0, 4) == 1 + 4 * 16
    assert kpp.kmeans_par_cap(float("nan"), 2) == 1 + 2 * 16


def test_workspace_size_is_host_arithmetic():
    lib = kpp.load_library()
    assert lib is not None
    # invalid shapes
    assert kpp.kpp_kmeans_par_workspace_size(0, 8, 10) == 0
    assert kpp.kpp_kmeans_par_workspace_size(100, 0, 10) == 0
    assert kpp.kpp_kmeans_par_workspace_size(100, 129, 10) == 0
    assert kpp.kpp_kmeans_par_workspace_size(100, 8, 0) == 0
    assert kpp.kpp_kmeans_par_workspace_size(1 << 31, 8, 10) == 0
    # valid: grows with N, d and the candidate room, 256-byte multiple, and
    # holds at least D^2, labels, picks and flags of every point plus the
    # candidates' rows
    a = kpp.kpp_kmeans_par_workspace_size(10_000, 32, 1000)
    b = kpp.kpp_kmeans_par_workspace_size(20_000, 32, 1000)
    c = kpp.kpp_kmeans_par_workspace_size(10_000, 64, 1000)
    e = kpp.kpp_kmeans_par_workspace_size(10_000, 32, 2000)
    assert a % 256 == 0 and a < b and a < c and a < e
    assert a >= 10_000 * 13 + 1000 * 32 * 4
    # the room is capped at N
    assert (kpp.kpp_kmeans_par_workspace_size(500, 16, 10_000) ==
            kpp.kpp_kmeans_par_workspace_size(500, 16, 500))


def test_tensor_helper_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        kpp.kmeans_par(torch.zeros((10, 4)), 2, 1)
    with pytest.raises(ValueError):
        kpp.kmeans_par(torch.zeros(10), 2, 1)


def test_no_cpu_fallback_anywhere():
    # host tensors are refused before any work: there is no CPU path
    torch = pytest.importorskip("torch")
    x = torch.zeros((100, 4))
    with pytest.raises(ValueError):
        kpp.seed(x, 2, 1)
    with pytest.raises(ValueError):
        kpp.Lloyd(x, 2)
    with pytest.raises(ValueError):
        kpp.kmeans_par(x, 2, 1)
