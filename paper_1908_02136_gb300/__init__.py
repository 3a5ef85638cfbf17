"""GB300-native k-means++ D^2 seeding (arXiv:1908.02136) -- Python binding.

A thin ctypes binding over ``libkpp.so`` (C ABI in ``include/kpp.h``).  Every
step of the seeding path runs in the library's CUDA kernels; this module
only marshals arguments.  PyTorch supplies device memory and streams.

Two layers:

* the C entry points under their C names (``kpp_seed``, ``kpp_workspace_size``,
  ``kpp_describe``,
  ``kpp_read_status``, ``kpp_quantize``, ``kpp_seed_host``,
  ``kpp_status_string``, ``kpp_version``), taking raw pointers and sizes;
* tensor helpers (``seed``, ``seed_host``, ``quantize``) that allocate the
  outputs and the workspace with torch and call the entry points on torch's
  current stream.

There is no CPU fallback: if the library cannot be built or loaded, import
of the entry points raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

F32, BF16, FP8_E4M3 = 0, 1, 2
FORM_AUTO, FORM_STREAMED, FORM_PERSISTENT, FORM_RECOMPUTE, FORM_SMALL = 0, 1, 2, 3, 4
(OK, ERR_INVALID_ARG, ERR_CUDA, ERR_LAUNCH, ERR_TIMEOUT, ERR_DEGENERATE,
 ERR_WORKSPACE, ERR_UNSUPPORTED, ERR_CAPACITY, ERR_BOUNDS) = range(10)

_DTYPE_NAMES = {"f32": F32, "fp32": F32, "float32": F32, "bf16": BF16, "bfloat16": BF16,
                "fp8": FP8_E4M3, "e4m3": FP8_E4M3, "fp8_e4m3": FP8_E4M3}


class KppError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {kpp_status_string(status)} (status {status})")


class Options(ctypes.Structure):
    """Mirror of kpp_options."""

    _fields_ = [("form", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("timeout_us", ctypes.c_uint32), ("smem_cache", ctypes.c_int32),
                ("alternate", ctypes.c_int32), ("l2_policy", ctypes.c_int32),
                ("min_rows_per_cta", ctypes.c_int32), ("exact_draws", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class Plan(ctypes.Structure):
    """Mirror of kpp_plan."""

    _fields_ = [("form", ctypes.c_int32), ("grid", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32),
                ("d2_in_smem", ctypes.c_int32), ("rows_per_cta", ctypes.c_int64),
                ("rows_per_segment", ctypes.c_int64), ("cached_rows_per_cta", ctypes.c_int64),
                ("smem_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Problem(ctypes.Structure):
    """Mirror of kpp_problem."""

    _fields_ = [("points", ctypes.c_void_p), ("row_scales", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("d", ctypes.c_int32), ("K", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint64),
                ("indices_out", ctypes.c_void_p), ("d2_out", ctypes.c_void_p),
                ("phi_out", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


class Shard(ctypes.Structure):
    """Mirror of kpp_shard (one process's rows of a point-sharded problem)."""

    _fields_ = [("points", ctypes.c_void_p), ("row_scales", ctypes.c_void_p),
                ("row0", ctypes.c_int64), ("n_local", ctypes.c_int64),
                ("n_global", ctypes.c_int64), ("d", ctypes.c_int32), ("K", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("rank", ctypes.c_int32), ("world", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint64),
                ("indices_out", ctypes.c_void_p), ("d2_out", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


def debug_build() -> bool:
    """True when the environment asks for the KPP_DEBUG build of the library
    (KPP_DEBUG=1): index checks in the kernels, reported as KPP_ERR_BOUNDS."""
    return os.environ.get("KPP_DEBUG", "0") not in ("", "0")


def library_path() -> str:
    return _build.lib_path(debug_build())


def load_library(build_if_stale: bool = True):
    """Load libkpp.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_stale:
            _build.build()
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libkpp.so not built at {path}")
        lib = ctypes.CDLL(path)
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.kpp_status_string.argtypes = [ctypes.c_int]
        lib.kpp_status_string.restype = ctypes.c_char_p
        lib.kpp_version.argtypes = []
        lib.kpp_version.restype = I32
        lib.kpp_workspace_size.argtypes = [I64, I32, I32, ctypes.c_int, P]
        lib.kpp_workspace_size.restype = ctypes.c_size_t
        lib.kpp_describe.argtypes = [I64, I32, I32, ctypes.c_int, P, P]
        lib.kpp_describe.restype = ctypes.c_int
        lib.kpp_seed.argtypes = [P, P, I64, I32, I32, ctypes.c_int, U64, U64, P, I32, P, P, P,
                                 P, ctypes.c_size_t, P, P]
        lib.kpp_seed.restype = ctypes.c_int
        lib.kpp_seed_host.argtypes = [P, P, P, P, I64, I32, I32, ctypes.c_int, U64, U64, P, P, P,
                                      P, P, P, P, ctypes.c_size_t, P, P]
        lib.kpp_seed_host.restype = ctypes.c_int
        lib.kpp_seed_noalloc.argtypes = [P, P, I64, I32, I32, ctypes.c_int, U64, U64, P, P, P,
                                         P, P, P]
        lib.kpp_seed_noalloc.restype = ctypes.c_int
        lib.kpp_batch_workspace_size.argtypes = [P, I32, ctypes.c_int, P]
        lib.kpp_batch_workspace_size.restype = ctypes.c_size_t
        lib.kpp_seed_batched.argtypes = [P, I32, ctypes.c_int, P, ctypes.c_size_t, P, P]
        lib.kpp_seed_batched.restype = ctypes.c_int
        lib.kpp_read_status.argtypes = [P, P]
        lib.kpp_read_status.restype = ctypes.c_int
        lib.kpp_quantize.argtypes = [P, I64, I32, ctypes.c_int, P, P, P]
        lib.kpp_quantize.restype = ctypes.c_int
        lib.kpp_measure_read.argtypes = [P, ctypes.c_size_t, I32, P, P]
        lib.kpp_measure_read.restype = ctypes.c_int
        lib.kpp_shard_exchange_words.argtypes = [I32, ctypes.c_int]
        lib.kpp_shard_exchange_words.restype = I64
        lib.kpp_shard_workspace_size.argtypes = [P, P]
        lib.kpp_shard_workspace_size.restype = ctypes.c_size_t
        lib.kpp_shard_first.argtypes = [P, P, P]
        lib.kpp_shard_first.restype = ctypes.c_int
        lib.kpp_shard_pass.argtypes = [P, I32, P, P, P, P]
        lib.kpp_shard_pass.restype = ctypes.c_int
        lib.kpp_shard_pick.argtypes = [P, I32, P, P, P, P]
        lib.kpp_shard_pick.restype = ctypes.c_int
        lib.kpp_shard_phi.argtypes = [P, I32, P, P]
        lib.kpp_shard_phi.restype = ctypes.c_int
        lib.kpp_tune_workspace_size.argtypes = [I64, I32, I32, ctypes.c_int]
        lib.kpp_tune_workspace_size.restype = ctypes.c_size_t
        lib.kpp_tune.argtypes = [P, P, I64, I32, I32, ctypes.c_int, P, P, P, ctypes.c_size_t, P,
                                 I32, P, P]
        lib.kpp_tune.restype = ctypes.c_int
        lib.kpp_tune_clear.argtypes = []
        lib.kpp_tune_clear.restype = None
        lib.kpp_lloyd_workspace_size.argtypes = [I64, I32, I32]
        lib.kpp_lloyd_workspace_size.restype = ctypes.c_size_t
        lib.kpp_lloyd_prepare.argtypes = [P, I64, I32, I32, P, ctypes.c_size_t, P]
        lib.kpp_lloyd_prepare.restype = ctypes.c_int
        lib.kpp_lloyd_step.argtypes = [P, I64, I32, P, I32, P, P, P, P, P, P, ctypes.c_size_t, P]
        lib.kpp_lloyd_step.restype = ctypes.c_int
        lib.kpp_lloyd_assign.argtypes = [P, I64, I32, I32, P, P, ctypes.c_size_t, P]
        lib.kpp_lloyd_assign.restype = ctypes.c_int
        lib.kpp_kmeans_par_workspace_size.argtypes = [I64, I32, I64]
        lib.kpp_kmeans_par_workspace_size.restype = ctypes.c_size_t
        lib.kpp_kmeans_par.argtypes = [P, I64, I32, I32, ctypes.c_double, I32, U64, U64, I64, P, P,
                                       P, P, P, P, P, P, ctypes.c_size_t, P]
        lib.kpp_kmeans_par.restype = ctypes.c_int
        _lib = lib
        return lib


def _opts_ptr(opts):
    if opts is None:
        return None
    if isinstance(opts, dict):
        o = Options()
        names = {f for f, _ in Options._fields_}
        for k, v in opts.items():
            if k not in names:
                raise KeyError(f"unknown kpp_options field {k!r}")
            setattr(o, k, v)
        opts = o
    return ctypes.byref(opts)


# ---------------------------------------------------------------------------
# C entry points, same names and argument order as include/kpp.h.
# ---------------------------------------------------------------------------
def kpp_status_string(status: int) -> str:
    return load_library().kpp_status_string(int(status)).decode()


def kpp_version() -> int:
    return load_library().kpp_version()


def kpp_workspace_size(N, d, K, dtype, opts=None) -> int:
    return load_library().kpp_workspace_size(N, d, K, dtype, _opts_ptr(opts))


def kpp_describe(N, d, K, dtype, opts=None, plan=None):
    """Returns (status, Plan) for the launch plan kpp_seed would use."""
    plan = plan if plan is not None else Plan()
    st = load_library().kpp_describe(N, d, K, dtype, _opts_ptr(opts), ctypes.byref(plan))
    return st, plan


def kpp_seed(points, row_scales, N, d, K, dtype, seed, stream_id, forced_prefix, n_forced,
             indices_out, d2_out, phi_out, workspace, workspace_bytes, stream, opts=None) -> int:
    return load_library().kpp_seed(points, row_scales, N, d, K, dtype, seed, stream_id,
                                   forced_prefix, n_forced, indices_out, d2_out, phi_out,
                                   workspace, workspace_bytes, stream, _opts_ptr(opts))


def kpp_seed_host(host_points, host_scales, dev_points, dev_scales, N, d, K, dtype, seed,
                  stream_id, host_indices, host_d2, host_phi, dev_indices, dev_d2, dev_phi,
                  workspace, workspace_bytes, stream, opts=None) -> int:
    return load_library().kpp_seed_host(host_points, host_scales, dev_points, dev_scales, N, d,
                                        K, dtype, seed, stream_id, host_indices, host_d2,
                                        host_phi, dev_indices, dev_d2, dev_phi, workspace,
                                        workspace_bytes, stream, _opts_ptr(opts))


def kpp_seed_noalloc(points, row_scales, N, d, K, dtype, seed, stream_id, indices_out, d2_out,
                     phi_out, stream, opts=None, device_status=None) -> int:
    """Seeding with the library's fixed internal scratch (no workspace, no
    allocation); ``device_status`` is a ctypes int32 (or None) that receives
    the device status after a stream synchronisation."""
    ds = None if device_status is None else ctypes.byref(device_status)
    return load_library().kpp_seed_noalloc(points, row_scales, N, d, K, dtype, seed, stream_id,
                                           indices_out, d2_out, phi_out, stream,
                                           _opts_ptr(opts), ds)


def kpp_batch_workspace_size(problems, n, dtype, opts=None) -> int:
    return load_library().kpp_batch_workspace_size(problems, n, dtype, _opts_ptr(opts))


def kpp_seed_batched(problems, n, dtype, workspace, workspace_bytes, stream, opts=None) -> int:
    return load_library().kpp_seed_batched(problems, n, dtype, workspace, workspace_bytes,
                                           stream, _opts_ptr(opts))


def kpp_read_status(workspace, stream) -> int:
    return load_library().kpp_read_status(workspace, stream)


def kpp_quantize(x, N, d, to, out, row_scales, stream) -> int:
    return load_library().kpp_quantize(x, N, d, to, out, row_scales, stream)


def kpp_measure_read(buf, nbytes, reps, stream, ms_out) -> int:
    return load_library().kpp_measure_read(buf, nbytes, reps, stream, ms_out)


def measure_read_gbs(nbytes: int, reps: int, device="cuda") -> float:
    """Read bandwidth (GB/s) of this GPU over a buffer of ``nbytes`` bytes,
    read ``reps`` times after one untimed sweep (``kpp_measure_read``)."""
    import torch

    dev = torch.device(device)
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device=dev)
    ms = ctypes.c_float(0.0)
    st = kpp_measure_read(buf.data_ptr(), buf.numel() * 4, reps, _stream_handle(dev),
                          ctypes.byref(ms))
    if st != OK:
        raise KppError(st, "kpp_measure_read")
    return buf.numel() * 4 / (ms.value * 1e-3) / 1e9


def kpp_shard_exchange_words(d, dtype) -> int:
    return load_library().kpp_shard_exchange_words(d, dtype)


def kpp_shard_workspace_size(shard, opts=None) -> int:
    return load_library().kpp_shard_workspace_size(ctypes.byref(shard), _opts_ptr(opts))


def kpp_shard_first(shard, exchange, stream) -> int:
    return load_library().kpp_shard_first(ctypes.byref(shard), exchange, stream)


def kpp_shard_pass(shard, m, exchange, total_out, stream, opts=None) -> int:
    return load_library().kpp_shard_pass(ctypes.byref(shard), m, exchange, total_out, stream,
                                         _opts_ptr(opts))


def kpp_shard_pick(shard, m, all_totals, exchange, stream, opts=None) -> int:
    return load_library().kpp_shard_pick(ctypes.byref(shard), m, all_totals, exchange, stream,
                                         _opts_ptr(opts))


def kpp_shard_phi(all_totals, world, phi_out, stream) -> int:
    return load_library().kpp_shard_phi(all_totals, world, phi_out, stream)


class PointShard:
    """One shard (a contiguous range of rows) of a point-sharded seeding, on
    the points' GPU, driven by ``multi.seed_sharded``.

    ``points``: this shard's rows [n_local, d] (CUDA, stored as ``dtype``);
    ``row0``: the global index of its first row; ``n_global``: the rows of
    all shards.  Holds the buffers the exchanges carry: ``exchange`` (int64,
    summed over shards), ``total`` (2 floats, gathered into ``totals``).
    After the seeding: ``idx`` (global indices), ``d2`` (this shard's D^2),
    ``phi``; ``status()`` reads the device status.
    """

    def __init__(self, points, row0: int, n_global: int, K: int, seed: int, stream_id: int,
                 rank: int, world: int, *, dtype=None, row_scales=None, opts=None):
        import torch

        n, d = points.shape
        dt = _dtype_code(points, dtype)
        dev = points.device
        self.points, self.row_scales, self.opts, self.world = points, row_scales, opts, world
        self.idx = torch.full((K,), -1, dtype=torch.int64, device=dev)
        self.d2 = torch.empty(n, dtype=torch.float32, device=dev)
        self.phi = torch.zeros(1, dtype=torch.float64, device=dev)
        self.total = torch.zeros(2, dtype=torch.float32, device=dev)
        self.totals = torch.zeros(2 * world, dtype=torch.float32, device=dev)
        words = kpp_shard_exchange_words(d, dt)
        if words <= 0:
            raise KppError(ERR_INVALID_ARG, "kpp_shard_exchange_words")
        self.exchange = torch.zeros(words, dtype=torch.int64, device=dev)
        self.desc = Shard(points.data_ptr(), None if row_scales is None else row_scales.data_ptr(),
                          row0, n, n_global, d, K, dt, rank, world, seed, stream_id,
                          self.idx.data_ptr(), self.d2.data_ptr(), None, 0)
        with torch.cuda.device(dev):
            nb = kpp_shard_workspace_size(self.desc, opts)
        if nb == 0:
            raise KppError(ERR_INVALID_ARG, "kpp_shard_workspace_size")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.desc.workspace, self.desc.workspace_bytes = self.ws.data_ptr(), nb
        self.dev = dev

    def _check(self, st, where):
        if st != OK:
            raise KppError(st, where)

    def first(self):
        self._check(kpp_shard_first(self.desc, self.exchange.data_ptr(),
                                    _stream_handle(self.dev)), "kpp_shard_first")

    def local_pass(self, m: int):
        self._check(kpp_shard_pass(self.desc, m, self.exchange.data_ptr(), self.total.data_ptr(),
                                   _stream_handle(self.dev), self.opts), "kpp_shard_pass")

    def pick(self, m: int):
        self._check(kpp_shard_pick(self.desc, m, self.totals.data_ptr(),
                                   self.exchange.data_ptr(), _stream_handle(self.dev), self.opts),
                    "kpp_shard_pick")

    def finish(self):
        self._check(kpp_shard_phi(self.totals.data_ptr(), self.world, self.phi.data_ptr(),
                                  _stream_handle(self.dev)), "kpp_shard_phi")

    def status(self) -> int:
        return kpp_read_status(self.ws.data_ptr(), _stream_handle(self.dev))


def kpp_tune_workspace_size(N, d, K, dtype) -> int:
    return load_library().kpp_tune_workspace_size(N, d, K, dtype)


def kpp_tune(points, row_scales, N, d, K, dtype, indices_out, d2_out, workspace,
             workspace_bytes, stream, passes, best_out, best_ms_per_pass=None) -> int:
    """``best_out`` is an ``Options`` (filled); ``best_ms_per_pass`` a ctypes
    float or None."""
    ms = None if best_ms_per_pass is None else ctypes.byref(best_ms_per_pass)
    return load_library().kpp_tune(points, row_scales, N, d, K, dtype, indices_out, d2_out,
                                   workspace, workspace_bytes, stream, passes,
                                   ctypes.byref(best_out), ms)


def kpp_tune_clear() -> None:
    load_library().kpp_tune_clear()


def kpp_lloyd_workspace_size(N, d, K) -> int:
    return load_library().kpp_lloyd_workspace_size(N, d, K)


def kpp_lloyd_prepare(points, N, d, K, workspace, workspace_bytes, stream) -> int:
    return load_library().kpp_lloyd_prepare(points, N, d, K, workspace, workspace_bytes, stream)


def kpp_lloyd_assign(centres, N, d, K, labels_out, workspace, workspace_bytes, stream) -> int:
    return load_library().kpp_lloyd_assign(centres, N, d, K, labels_out, workspace,
                                           workspace_bytes, stream)


def kpp_lloyd_step(points, N, d, centres, K, labels_out, d2_out, centres_out, counts_out, phi_out,
                   workspace, workspace_bytes, stream) -> int:
    return load_library().kpp_lloyd_step(points, N, d, centres, K, labels_out, d2_out,
                                         centres_out, counts_out, phi_out, workspace,
                                         workspace_bytes, stream)


def kpp_kmeans_par_workspace_size(N, d, cand_cap) -> int:
    return load_library().kpp_kmeans_par_workspace_size(N, d, cand_cap)


def kpp_kmeans_par(points, N, d, K, ell, rounds, seed, stream_id, cand_cap, idx_out, cand_out,
                   n_cand_out, weights_out, labels_out, d2_out, phi_out, workspace,
                   workspace_bytes, stream) -> int:
    """``n_cand_out``: address of a host int64 (e.g. ``ctypes.addressof``)."""
    return load_library().kpp_kmeans_par(points, N, d, K, ell, rounds, seed, stream_id, cand_cap,
                                         idx_out, cand_out, n_cand_out, weights_out, labels_out,
                                         d2_out, phi_out, workspace, workspace_bytes, stream)


# ---------------------------------------------------------------------------
# Tensor helpers.
# ---------------------------------------------------------------------------
def _dtype_code(points, dtype):
    import torch

    if dtype is not None:
        return _DTYPE_NAMES[dtype] if isinstance(dtype, str) else int(dtype)
    if points.dtype == torch.float32:
        return F32
    if points.dtype in (torch.bfloat16, torch.int16, torch.uint16):
        return BF16
    if points.dtype in (torch.uint8, torch.float8_e4m3fn):
        return FP8_E4M3
    raise TypeError(f"unsupported point dtype {points.dtype}")


def _stream_handle(device):
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def workspace_for(N, d, K, dtype, device, opts=None):
    """A torch uint8 workspace tensor of the size kpp_workspace_size reports."""
    import torch

    with torch.cuda.device(device):
        n = kpp_workspace_size(N, d, K, dtype, opts)
    # 0 means the arguments are rejected; kpp_seed then reports why.
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device)


def seed(points, K: int, seed: int, stream_id: int = 0, *, dtype=None, row_scales=None,
         forced=None, opts=None, workspace=None, out=None, check: bool = True):
    """k-means++ seeding on the GPU through ``kpp_seed``.

    ``points``: CUDA tensor [N, d] of float32, BF16 bits (bfloat16/int16) or
    E4M3 codes (uint8/float8_e4m3fn, with ``row_scales`` float32 [N]).
    Returns ``(idx int64 [K], d2 float32 [N], phi float64 [1])`` on the same
    device.  With ``check`` the stream is synchronised and a device status
    other than OK raises ``KppError`` (degenerate data included); without it
    the call stays asynchronous.
    """
    import torch

    if not points.is_cuda:
        raise ValueError("points must be a CUDA tensor (use seed_host for host data)")
    N, d = points.shape
    dt = _dtype_code(points, dtype)
    dev = points.device
    if out is None:
        idx = torch.empty(K, dtype=torch.int64, device=dev)
        d2 = torch.empty(N, dtype=torch.float32, device=dev)
        phi = torch.empty(1, dtype=torch.float64, device=dev)
    else:
        idx, d2, phi = out
    ws = workspace if workspace is not None else workspace_for(N, d, K, dt, dev, opts)
    fo = None
    if forced is not None:
        fo = torch.as_tensor(forced, dtype=torch.int64, device=dev).contiguous()
    with torch.cuda.device(dev):
        st = kpp_seed(points.data_ptr(), None if row_scales is None else row_scales.data_ptr(),
                      N, d, K, dt, seed, stream_id, None if fo is None else fo.data_ptr(),
                      0 if fo is None else fo.numel(), idx.data_ptr(), d2.data_ptr(),
                      phi.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(dev), opts)
        if st != OK:
            raise KppError(st, "kpp_seed")
        if check:
            st = kpp_read_status(ws.data_ptr(), _stream_handle(dev))
            if st != OK:
                raise KppError(st, "kpp_seed (device)")
    return idx, d2, phi


def tune(points, K: int, *, dtype=None, row_scales=None, passes: int = 0):
    """Autotune ``kpp_seed`` for this shape on the points' device (``kpp_tune``).

    Returns ``(options dict, ms per pass)``.  The choice is also recorded for
    later calls with the same shape whose options leave the knobs at zero.
    """
    import torch

    N, d = points.shape
    dt = _dtype_code(points, dtype)
    dev = points.device
    idx = torch.empty(K, dtype=torch.int64, device=dev)
    d2 = torch.empty(N, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        n = kpp_tune_workspace_size(N, d, K, dt)
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device=dev)
        best = Options()
        ms = ctypes.c_float(0.0)
        st = kpp_tune(points.data_ptr(), None if row_scales is None else row_scales.data_ptr(),
                      N, d, K, dt, idx.data_ptr(), d2.data_ptr(), ws.data_ptr(), ws.numel(),
                      _stream_handle(dev), passes, best, ms)
    if st != OK:
        raise KppError(st, "kpp_tune")
    return {f: getattr(best, f) for f, _ in Options._fields_ if f not in ("reserved", "exact_draws")}, ms.value


class Lloyd:
    """Lloyd iterations on FP32 CUDA points [N, d] with K centres through
    ``kpp_lloyd_prepare`` / ``kpp_lloyd_step``: the workspace holds the
    points' BF16 split, prepared once."""

    def __init__(self, points, K: int):
        import torch

        if not points.is_cuda or points.dtype != torch.float32:
            raise ValueError("points must be a float32 CUDA tensor")
        self.points = points.contiguous()
        self.N, self.d = self.points.shape
        self.K = int(K)
        dev = self.points.device
        with torch.cuda.device(dev):
            n = kpp_lloyd_workspace_size(self.N, self.d, self.K)
            if n == 0:
                raise KppError(ERR_INVALID_ARG, "kpp_lloyd_workspace_size")
            self.ws = torch.empty(n, dtype=torch.uint8, device=dev)
            st = kpp_lloyd_prepare(self.points.data_ptr(), self.N, self.d, self.K,
                                   self.ws.data_ptr(), self.ws.numel(), _stream_handle(dev))
        if st != OK:
            raise KppError(st, "kpp_lloyd_prepare")

    def assign(self, centres, labels=None):
        """Labels int32 [N] of the nearest centre (``kpp_lloyd_assign``)."""
        import torch

        dev = self.points.device
        c = centres.to(device=dev, dtype=torch.float32).contiguous()
        labels = labels if labels is not None else torch.empty(self.N, dtype=torch.int32,
                                                               device=dev)
        with torch.cuda.device(dev):
            st = kpp_lloyd_assign(c.data_ptr(), self.N, self.d, self.K, labels.data_ptr(),
                                  self.ws.data_ptr(), self.ws.numel(), _stream_handle(dev))
        if st != OK:
            raise KppError(st, "kpp_lloyd_assign")
        return labels

    def step(self, centres, check: bool = True):
        """One iteration from ``centres`` [K, d] float32 (CUDA).  Returns
        ``(labels int32 [N], d2 float32 [N], new centres [K, d], counts int64
        [K], phi float64 [1])``."""
        import torch

        dev = self.points.device
        c = centres.to(device=dev, dtype=torch.float32).contiguous()
        labels = torch.empty(self.N, dtype=torch.int32, device=dev)
        d2 = torch.empty(self.N, dtype=torch.float32, device=dev)
        out = torch.empty_like(c)
        counts = torch.empty(self.K, dtype=torch.int64, device=dev)
        phi = torch.empty(1, dtype=torch.float64, device=dev)
        with torch.cuda.device(dev):
            sh = _stream_handle(dev)
            st = kpp_lloyd_step(self.points.data_ptr(), self.N, self.d, c.data_ptr(), self.K,
                                labels.data_ptr(), d2.data_ptr(), out.data_ptr(),
                                counts.data_ptr(), phi.data_ptr(), self.ws.data_ptr(),
                                self.ws.numel(), sh)
            if st != OK:
                raise KppError(st, "kpp_lloyd_step")
            if check:
                st = kpp_read_status(self.ws.data_ptr(), sh)
                if st != OK:
                    raise KppError(st, "kpp_lloyd_step (device)")
        return labels, d2, out, counts, phi


def kmeans_par_cap(ell: float, rounds: int) -> int:
    """Default room for the candidates: c_0 plus, per round, the expected
    ell draws and 8 standard deviations (a round draws a sum of Bernoullis
    with mean <= ell, so its variance is <= ell) and a small margin."""
    import math

    e = max(float(ell), 0.0) if math.isfinite(ell) else 0.0
    return 1 + max(int(rounds), 0) * int(math.ceil(e + 8.0 * math.sqrt(e) + 16.0))


def kmeans_par(points, K: int, seed: int, stream_id: int = 0, *, ell=None, rounds: int = 5,
               cand_cap=None, workspace=None):
    """k-means|| on FP32 CUDA points [N, d] through ``kpp_kmeans_par``
    (``ell`` defaults to 2K).  Returns a dict: ``idx`` int64 [K] (the chosen
    points), ``cand`` int64 [n] (the candidates in list order), ``weights``
    int64 [n], ``labels`` int32 [N] (nearest candidate position), ``d2``
    float32 [N] and ``phi`` float64 [1] after the rounds, ``status``.  A
    degenerate stop (fewer than K weighted candidates) is reported in
    ``status`` with -1 in ``idx``; other errors raise ``KppError``."""
    import torch

    if not points.is_cuda or points.dtype != torch.float32 or points.dim() != 2:
        raise ValueError("points must be a 2-D float32 CUDA tensor")
    x = points.contiguous()
    N, d = x.shape
    ell = float(2 * K if ell is None else ell)
    cap = int(cand_cap if cand_cap is not None else min(N, kmeans_par_cap(ell, rounds)))
    dev = x.device
    with torch.cuda.device(dev):
        if workspace is None:
            n = kpp_kmeans_par_workspace_size(N, d, cap)
            if n == 0:
                raise KppError(ERR_INVALID_ARG, "kpp_kmeans_par_workspace_size")
            workspace = torch.empty(n, dtype=torch.uint8, device=dev)
        idx = torch.empty(K, dtype=torch.int64, device=dev)
        cand = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        w = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        labels = torch.empty(N, dtype=torch.int32, device=dev)
        d2 = torch.empty(N, dtype=torch.float32, device=dev)
        phi = torch.empty(1, dtype=torch.float64, device=dev)
        nc = ctypes.c_int64(0)
        st = kpp_kmeans_par(x.data_ptr(), N, d, int(K), ell, int(rounds), int(seed),
                            int(stream_id), cap, idx.data_ptr(), cand.data_ptr(),
                            ctypes.addressof(nc), w.data_ptr(), labels.data_ptr(), d2.data_ptr(),
                            phi.data_ptr(), workspace.data_ptr(), workspace.numel(),
                            _stream_handle(dev))
    if st not in (OK, ERR_DEGENERATE):
        raise KppError(st, "kpp_kmeans_par")
    n = nc.value
    return {"idx": idx, "cand": cand[:n], "weights": w[:n], "labels": labels, "d2": d2,
            "phi": phi, "status": st}


def seed_host(points_host, K: int, seed: int, stream_id: int = 0, *, dtype=None,
              row_scales_host=None, device="cuda", opts=None, buffers=None):
    """End-to-end seeding from host (ideally pinned) tensors via ``kpp_seed_host``.

    Returns host tensors ``(idx, d2, phi)`` and the device status.
    ``buffers`` may carry reusable device/host buffers from a previous call
    (the dict this function returns as its last element).
    """
    import torch

    N, d = points_host.shape
    dt = _dtype_code(points_host, dtype)
    b = buffers
    if b is None:
        b = {
            "dev_points": torch.empty_like(points_host, device=device),
            "dev_scales": (torch.empty(N, dtype=torch.float32, device=device)
                           if dt == FP8_E4M3 else None),
            "dev_idx": torch.empty(K, dtype=torch.int64, device=device),
            "dev_d2": torch.empty(N, dtype=torch.float32, device=device),
            "dev_phi": torch.empty(1, dtype=torch.float64, device=device),
            "host_idx": torch.empty(K, dtype=torch.int64, pin_memory=True),
            "host_d2": torch.empty(N, dtype=torch.float32, pin_memory=True),
            "host_phi": torch.empty(1, dtype=torch.float64, pin_memory=True),
            "ws": workspace_for(N, d, K, dt, torch.device(device), opts),
        }
    dev = b["dev_idx"].device
    with torch.cuda.device(dev):
        st = kpp_seed_host(
            points_host.data_ptr(),
            None if row_scales_host is None else row_scales_host.data_ptr(),
            b["dev_points"].data_ptr(),
            None if b["dev_scales"] is None else b["dev_scales"].data_ptr(),
            N, d, K, dt, seed, stream_id, b["host_idx"].data_ptr(), b["host_d2"].data_ptr(),
            b["host_phi"].data_ptr(), b["dev_idx"].data_ptr(), b["dev_d2"].data_ptr(),
            b["dev_phi"].data_ptr(), b["ws"].data_ptr(), b["ws"].numel(), _stream_handle(dev),
            opts)
    return b["host_idx"], b["host_d2"], b["host_phi"], st, b


def quantize(x, to: str, *, out=None, row_scales=None):
    """FP32 CUDA points [N, d] -> BF16 bits (int16 tensor) or (E4M3 uint8, scales)."""
    import torch

    N, d = x.shape
    code = _DTYPE_NAMES[to]
    if code == BF16:
        q = out if out is not None else torch.empty((N, d), dtype=torch.int16, device=x.device)
        s = None
    elif code == FP8_E4M3:
        q = out if out is not None else torch.empty((N, d), dtype=torch.uint8, device=x.device)
        s = row_scales if row_scales is not None else torch.empty(N, dtype=torch.float32,
                                                                  device=x.device)
    else:
        raise ValueError(to)
    with torch.cuda.device(x.device):
        st = kpp_quantize(x.data_ptr(), N, d, code, q.data_ptr(),
                          None if s is None else s.data_ptr(), _stream_handle(x.device))
    if st != OK:
        raise KppError(st, "kpp_quantize")
    return q if s is None else (q, s)


def seed_batched(points_list, Ks, seeds, stream_ids=None, *, dtype=None, row_scales=None,
                 opts=None, outs=None, workspace=None, check: bool = True):
    """Batched seeding through ``kpp_seed_batched``.

    ``points_list``: CUDA tensors [N_p, d_p] (same storage type); ``Ks``,
    ``seeds``, ``stream_ids``: per-problem ints.  Returns a list of
    ``(idx, d2, phi)`` and the workspace (reusable for the same batch).
    """
    import torch

    n = len(points_list)
    dev = points_list[0].device
    dt = _dtype_code(points_list[0], dtype)
    stream_ids = list(range(n)) if stream_ids is None else stream_ids
    if outs is None:
        outs = [(torch.empty(K, dtype=torch.int64, device=dev),
                 torch.empty(x.shape[0], dtype=torch.float32, device=dev),
                 torch.empty(1, dtype=torch.float64, device=dev))
                for x, K in zip(points_list, Ks)]
    arr = (Problem * n)()
    for i, (x, K) in enumerate(zip(points_list, Ks)):
        idx, d2, phi = outs[i]
        arr[i].points = x.data_ptr()
        arr[i].row_scales = None if row_scales is None else row_scales[i].data_ptr()
        arr[i].N = x.shape[0]
        arr[i].d = x.shape[1]
        arr[i].K = int(K)
        arr[i].seed = int(seeds[i])
        arr[i].stream_id = int(stream_ids[i])
        arr[i].indices_out = idx.data_ptr()
        arr[i].d2_out = d2.data_ptr()
        arr[i].phi_out = phi.data_ptr()
    with torch.cuda.device(dev):
        if workspace is None:
            # 0 means the problems are rejected; kpp_seed_batched reports why
            nb = kpp_batch_workspace_size(arr, n, dt, opts)
            workspace = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        st = kpp_seed_batched(arr, n, dt, workspace.data_ptr(), workspace.numel(),
                              _stream_handle(dev), opts)
        if st != OK:
            raise KppError(st, "kpp_seed_batched")
        if check:
            st = kpp_read_status(workspace.data_ptr(), _stream_handle(dev))
            if st != OK:
                raise KppError(st, "kpp_seed_batched (device)")
    return outs, workspace
