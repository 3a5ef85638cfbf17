"""FP64 CPU oracle for k-means++ D^2 seeding (arXiv:1908.02136, Algorithm 1).

TEST INFRASTRUCTURE ONLY: the correctness reference the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with ``paper_1908_02136_gb300`` and never calls it.
Besides the seeding it holds one Lloyd iteration (readings L1-L3), the
clustering stage the seeds are for.

The arithmetic lives in ``kpp_oracle.c`` (plain C, serial, FP64, built with
``gcc -O2 -ffp-contract=off``); this module only compiles it and marshals
numpy arrays through ctypes.  The readings of the paper it takes (R1-R6) are
listed at the top of ``kpp_oracle.c``.

Pins: every function here is pinned by ``tests/test_oracle_*.py`` against
something other than itself (numpy's Philox4x64-10, scipy's squared
Euclidean distances, torch's BF16/FP8 conversions, the exact D^2 sampling
law by enumeration, invariants and the k-means++ expected-cost bound).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kpp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkpp_oracle.so")
_lock = threading.Lock()
_lib = None

F32, BF16, FP8_E4M3 = 0, 1, 2
OK, INVALID, DEGENERATE = 0, 1, 5


class Draw(ctypes.Structure):
    """Per-draw record (see kpp_oracle_draw in kpp_oracle.c)."""

    _fields_ = [
        ("own", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("T", ctypes.c_double),
        ("P_before", ctypes.c_double),
        ("P_at", ctypes.c_double),
    ]


DRAW_DTYPE = np.dtype(
    [("own", np.int64), ("t", np.float64), ("T", np.float64),
     ("P_before", np.float64), ("P_at", np.float64)]
)


def build(force: bool = False) -> str:
    """Compile kpp_oracle.c into oracle/_build/libkpp_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
               "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.kpp_oracle_philox4x64_10.argtypes = [P, P, P]
        lib.kpp_oracle_philox4x64_10.restype = None
        lib.kpp_oracle_uniform.argtypes = [ctypes.c_uint64] * 3
        lib.kpp_oracle_uniform.restype = ctypes.c_double
        lib.kpp_oracle_decode_bf16.argtypes = [ctypes.c_uint16]
        lib.kpp_oracle_decode_bf16.restype = ctypes.c_double
        lib.kpp_oracle_decode_e4m3.argtypes = [ctypes.c_uint8]
        lib.kpp_oracle_decode_e4m3.restype = ctypes.c_double
        lib.kpp_oracle_encode_e4m3_sat.argtypes = [ctypes.c_float]
        lib.kpp_oracle_encode_e4m3_sat.restype = ctypes.c_uint8
        lib.kpp_oracle_quantize_bf16.argtypes = [P, ctypes.c_int64, P]
        lib.kpp_oracle_quantize_bf16.restype = None
        lib.kpp_oracle_quantize_fp8.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, P]
        lib.kpp_oracle_quantize_fp8.restype = None
        lib.kpp_oracle_pick.argtypes = [P, ctypes.c_int64, ctypes.c_double, P, P]
        lib.kpp_oracle_pick.restype = ctypes.c_int64
        lib.kpp_oracle_seed.argtypes = [
            P, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_uint64, ctypes.c_uint64, P, ctypes.c_int32, P, P, P, P, P]
        lib.kpp_oracle_seed.restype = ctypes.c_int
        lib.kpp_oracle_seed_mt.argtypes = [
            P, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_uint64, ctypes.c_uint64, P, P, P, ctypes.c_int32]
        lib.kpp_oracle_seed_mt.restype = ctypes.c_int
        lib.kpp_oracle_lloyd_step.argtypes = [
            P, P, ctypes.c_int, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P]
        lib.kpp_oracle_lloyd_step.restype = ctypes.c_int
        U64, I64, I32, D = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.kpp_oracle_uniform_ctr.argtypes = [U64] * 6
        lib.kpp_oracle_uniform_ctr.restype = D
        lib.kpp_oracle_min_update.argtypes = [P, P, ctypes.c_int, I64, I32, P, I64, P, ctypes.c_int]
        lib.kpp_oracle_min_update.restype = D
        lib.kpp_oracle_kmpar_select.argtypes = [P, I64, D, D, U64, U64, I32, P, P, P]
        lib.kpp_oracle_kmpar_select.restype = I64
        lib.kpp_oracle_kmpar_weights.argtypes = [P, P, ctypes.c_int, I64, I32, P, I64, P]
        lib.kpp_oracle_kmpar_weights.restype = None
        lib.kpp_oracle_weighted_seed.argtypes = [P, P, ctypes.c_int, I32, P, I64, P, I32, U64, U64,
                                                 P, I32, P, P]
        lib.kpp_oracle_weighted_seed.restype = ctypes.c_int
        lib.kpp_oracle_kmeans_par.argtypes = [P, P, ctypes.c_int, I64, I32, I32, D, I32, U64, U64,
                                              P, P, I64, P, P]
        lib.kpp_oracle_kmeans_par.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block: counter (4 x u64), key (2 x u64) -> 4 x u64."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().kpp_oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed: int, stream: int, m: int) -> float:
    """The draw u_m in [0, 1) (reading R1)."""
    return _load().kpp_oracle_uniform(seed, stream, m)


def decode_bf16(bits: np.ndarray) -> np.ndarray:
    lib = _load()
    flat = np.ascontiguousarray(bits, dtype=np.uint16).ravel()
    return np.array([lib.kpp_oracle_decode_bf16(int(b)) for b in flat]).reshape(np.shape(bits))


def decode_e4m3(codes: np.ndarray) -> np.ndarray:
    lib = _load()
    flat = np.ascontiguousarray(codes, dtype=np.uint8).ravel()
    return np.array([lib.kpp_oracle_decode_e4m3(int(b)) for b in flat]).reshape(np.shape(codes))


def encode_e4m3(x: np.ndarray) -> np.ndarray:
    """FP32 values -> E4M3 codes, round to nearest even, saturating at 448."""
    lib = _load()
    flat = np.ascontiguousarray(x, dtype=np.float32).ravel()
    return np.array([lib.kpp_oracle_encode_e4m3_sat(float(v)) for v in flat],
                    dtype=np.uint8).reshape(np.shape(x))


def quantize_bf16(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns (uint16), round to nearest even."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().kpp_oracle_quantize_bf16(_ptr(x), x.size, _ptr(out))
    return out


def quantize_fp8(x: np.ndarray):
    """FP32 [N, d] -> (E4M3 codes uint8 [N, d], FP32 row scales [N])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    N, d = x.shape
    q = np.empty((N, d), dtype=np.uint8)
    s = np.empty(N, dtype=np.float32)
    _load().kpp_oracle_quantize_fp8(_ptr(x), N, d, _ptr(q), _ptr(s))
    return q, s


def pick(d2: np.ndarray, u: float):
    """Inverse-CDF draw (reading R3). Returns (index, t, T); index -1 if T == 0."""
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    t = ctypes.c_double()
    T = ctypes.c_double()
    i = _load().kpp_oracle_pick(_ptr(d2), d2.size, u, ctypes.byref(t), ctypes.byref(T))
    return int(i), t.value, T.value


def _dtype_code(points: np.ndarray, dtype) -> int:
    if dtype is not None:
        return {"f32": F32, "bf16": BF16, "fp8": FP8_E4M3, F32: F32, BF16: BF16,
                FP8_E4M3: FP8_E4M3}[dtype]
    if points.dtype == np.float32:
        return F32
    if points.dtype == np.uint16:
        return BF16
    if points.dtype == np.uint8:
        return FP8_E4M3
    raise TypeError(f"unsupported stored dtype {points.dtype}")


def seed(points: np.ndarray, K: int, seed: int, stream: int = 0, *, dtype=None,
         scales: np.ndarray | None = None, forced: np.ndarray | None = None,
         draws: bool = False, history: bool = False) -> dict:
    """Serial FP64 k-means++ seeding (Algorithm 1 with readings R1-R6).

    ``points`` holds the stored values, row-major [N, d]: float32, or BF16 bit
    patterns (uint16), or E4M3 codes (uint8, with ``scales``).  ``forced``
    replays an index prefix in place of the oracle's own draws.
    Returns a dict with ``idx`` (int64 [K]), ``d2`` (float64 [N]), ``phi``,
    ``status`` and optionally ``draws`` (structured [K]) and ``d2_hist``
    (float64 [K, N]).
    """
    pts = np.ascontiguousarray(points)
    N, d = pts.shape
    code = _dtype_code(pts, dtype)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    fo = None if forced is None else np.ascontiguousarray(forced, dtype=np.int64)
    n_forced = 0 if fo is None else int(fo.size)
    idx = np.empty(K, dtype=np.int64)
    d2 = np.empty(N, dtype=np.float64)
    phi = np.zeros(1, dtype=np.float64)
    dr = np.zeros(K, dtype=DRAW_DTYPE) if draws else None
    hist = np.empty((K, N), dtype=np.float64) if history else None
    st = _load().kpp_oracle_seed(
        _ptr(pts), _ptr(sc), code, N, d, K, seed, stream, _ptr(fo), n_forced,
        _ptr(idx), _ptr(d2), _ptr(phi), _ptr(dr), _ptr(hist))
    if st == INVALID:
        raise ValueError("oracle rejected its arguments")
    out = {"idx": idx, "d2": d2, "phi": float(phi[0]), "status": st}
    if draws:
        out["draws"] = dr
    if history:
        out["d2_hist"] = hist
    return out


def seed_mt(points: np.ndarray, K: int, seed: int, stream: int = 0, *, dtype=None,
            scales: np.ndarray | None = None, threads: int | None = None) -> dict:
    """Multi-threaded FP64 seeding (the CPU baseline on all host cores).

    Algorithm 1 with readings R1-R6, the points split into ``threads``
    contiguous chunks: D^2 bit-identical to ``seed``; the draw's prefix sums
    regrouped at chunk boundaries (identical to ``seed`` on integer data).
    Returns a dict with ``idx``, ``d2``, ``phi``, ``status`` and ``threads``.
    """
    pts = np.ascontiguousarray(points)
    N, d = pts.shape
    code = _dtype_code(pts, dtype)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    nt = int(threads or os.cpu_count() or 1)
    idx = np.empty(K, dtype=np.int64)
    d2 = np.empty(N, dtype=np.float64)
    phi = np.zeros(1, dtype=np.float64)
    st = _load().kpp_oracle_seed_mt(_ptr(pts), _ptr(sc), code, N, d, K, seed, stream, _ptr(idx),
                                    _ptr(d2), _ptr(phi), nt)
    if st == INVALID:
        raise ValueError("oracle rejected its arguments")
    return {"idx": idx, "d2": d2, "phi": float(phi[0]), "status": st, "threads": min(nt, N)}


def lloyd_step(points: np.ndarray, centres: np.ndarray, *, dtype=None,
               scales: np.ndarray | None = None) -> dict:
    """One FP64 Lloyd iteration (readings L1-L3): assignment to the nearest
    centre, then each centre moved to the mean of its points.

    ``points`` stored values [N, d] (float32, BF16 bits as uint16, or E4M3
    codes as uint8 with ``scales``); ``centres`` [K, d] (cast to float64).
    Returns labels (int32), d2, centres (float64), counts (int64), phi.
    """
    pts = np.ascontiguousarray(points)
    N, d = pts.shape
    code = _dtype_code(pts, dtype)
    C = np.ascontiguousarray(centres, dtype=np.float64)
    K = C.shape[0]
    if C.shape[1] != d:
        raise ValueError("centres must have the points' dimension")
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    labels = np.empty(N, dtype=np.int32)
    d2 = np.empty(N, dtype=np.float64)
    out = np.empty((K, d), dtype=np.float64)
    counts = np.empty(K, dtype=np.int64)
    phi = ctypes.c_double()
    st = _load().kpp_oracle_lloyd_step(_ptr(pts), _ptr(sc), code, N, d, _ptr(C), K, _ptr(labels),
                                       _ptr(d2), _ptr(out), _ptr(counts), ctypes.byref(phi))
    if st != OK:
        raise ValueError(f"kpp_oracle_lloyd_step: status {st}")
    return {"labels": labels, "d2": d2, "centres": out, "counts": counts, "phi": phi.value}


# ---------------------------------------------------------------------------
# k-means|| (readings P1-P4 in kpp_oracle.c).
# ---------------------------------------------------------------------------
def uniform_ctr(seed: int, stream: int, c0: int, c1: int = 0, c2: int = 0, c3: int = 0) -> float:
    """Word 0 of Philox4x64-10 at counter (c0, c1, c2, c3), mapped to [0, 1)."""
    return _load().kpp_oracle_uniform_ctr(seed, stream, c0, c1, c2, c3)


def _stored(points, dtype, scales):
    pts = np.ascontiguousarray(points)
    code = _dtype_code(pts, dtype)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    return pts, code, sc


def min_update(points, centres, D2=None, *, dtype=None, scales=None):
    """D^2 = min(D2, squared distance to the listed centre indices) in FP64;
    D2=None starts from +infinity.  Returns (D2, phi)."""
    pts, code, sc = _stored(points, dtype, scales)
    N, d = pts.shape
    c = np.ascontiguousarray(centres, dtype=np.int64)
    init = D2 is None
    out = np.empty(N, dtype=np.float64) if init else np.array(D2, dtype=np.float64)
    phi = _load().kpp_oracle_min_update(_ptr(pts), _ptr(sc), code, N, d, _ptr(c), c.size,
                                        _ptr(out), 1 if init else 0)
    return out, phi


def kmpar_select(D2, phi: float, ell: float, seed: int, stream: int, r: int):
    """Round r's Bernoulli decisions: (flags uint8, p, u) per point."""
    D = np.ascontiguousarray(D2, dtype=np.float64)
    N = D.size
    flags = np.empty(N, dtype=np.uint8)
    p = np.empty(N, dtype=np.float64)
    u = np.empty(N, dtype=np.float64)
    _load().kpp_oracle_kmpar_select(_ptr(D), N, phi, ell, seed, stream, r, _ptr(flags), _ptr(p),
                                    _ptr(u))
    return flags, p, u


def kmpar_weights(points, cand, *, dtype=None, scales=None):
    """Number of points whose nearest candidate is each candidate."""
    pts, code, sc = _stored(points, dtype, scales)
    N, d = pts.shape
    c = np.ascontiguousarray(cand, dtype=np.int64)
    w = np.empty(c.size, dtype=np.int64)
    _load().kpp_oracle_kmpar_weights(_ptr(pts), _ptr(sc), code, N, d, _ptr(c), c.size, _ptr(w))
    return w


def weighted_seed(points, cand, w, K: int, seed: int, stream: int = 0, *, dtype=None,
                  scales=None, forced=None):
    """Weighted k-means++ over the candidates (P4): (positions, own draws, status)."""
    pts, code, sc = _stored(points, dtype, scales)
    d = pts.shape[1]
    c = np.ascontiguousarray(cand, dtype=np.int64)
    ww = np.ascontiguousarray(w, dtype=np.int64)
    fo = None if forced is None else np.ascontiguousarray(forced, dtype=np.int64)
    out = np.empty(K, dtype=np.int64)
    own = np.empty(K, dtype=np.int64)
    st = _load().kpp_oracle_weighted_seed(_ptr(pts), _ptr(sc), code, d, _ptr(c), c.size, _ptr(ww),
                                          K, seed, stream, _ptr(fo),
                                          0 if fo is None else fo.size, _ptr(out), _ptr(own))
    return out, own, st


def kmeans_par(points, K: int, ell: float, rounds: int, seed: int, stream: int = 0, *,
               dtype=None, scales=None, cand_cap: int | None = None) -> dict:
    """k-means|| (P1-P4): chosen point indices, the candidate list, its weights."""
    pts, code, sc = _stored(points, dtype, scales)
    N, d = pts.shape
    cap = cand_cap if cand_cap is not None else min(N, 1 + int(rounds * ell * 4) + 64)
    idx = np.empty(K, dtype=np.int64)
    cand = np.empty(cap, dtype=np.int64)
    w = np.empty(cap, dtype=np.int64)
    nc = ctypes.c_int64()
    st = _load().kpp_oracle_kmeans_par(_ptr(pts), _ptr(sc), code, N, d, K, float(ell), rounds,
                                       seed, stream, _ptr(idx), _ptr(cand), cap,
                                       ctypes.byref(nc), _ptr(w))
    n = nc.value
    return {"status": st, "idx": idx, "cand": cand[:n].copy(), "w": w[:n].copy()}
