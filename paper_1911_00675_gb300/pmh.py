"""Thin Python binding of libpmh.so (argument marshalling only).

Every function has the name of the C entry point without the ``pmh_``
prefix and passes raw device pointers of PyTorch tensors plus the current
CUDA stream.  All arithmetic runs in the library's CUDA kernels; if the
shared object is missing or does not load, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpmh.so")

OK, ERR_INVALID_ARG, ERR_BAD_WEIGHT, ERR_ITER_LIMIT, ERR_CUDA, ERR_NO_MEMORY, ERR_UNSUPPORTED = range(7)
V1, V1A, V2, V3, V3A, V4, V3U, V3AU, V4U = range(9)
VARIANTS = {"1": V1, "1a": V1A, "2": V2, "3": V3, "3a": V3A, "4": V4, "3u": V3U, "3au": V3AU, "4u": V4U}
FP64, FP32_RECHECK = 0, 1
TE_INVERSION, TE_REJECTION = 0, 1
SHAPE_WARP, SHAPE_CTA8, SHAPE_QUAD, SHAPE_PAIR, SHAPE_QUAD8, SHAPE_QUAD8L = range(6)
COUNTERS = ("elements", "points32", "points64", "contenders", "resolved", "rounds", "deep", "prefiltered",
            "cyc_pass0", "cyc_first", "cyc_deep", "cyc_refresh", "cyc_finish", "items", "cyc_surv", "cyc_item",
            "cyc_warp", "cyc_barrier", "seq_steps", "seq_points", "redo", "listed",
            "list_hashed", "list_skipped")
EXPORTS = ("pmh_create", "pmh_destroy", "pmh_last_error", "pmh_sketch_batch", "pmh_sketch_batch_host",
           "pmh_last_host_span_ms", "pmh_sketch_batch_noalloc",
           "pmh_set_profiling", "pmh_last_kernel_ms", "pmh_kernel_ms_history", "pmh_last_launches",
           "pmh_set_thresholds", "pmh_set_limits", "pmh_sync_status", "pmh_set_te_sampler", "pmh_set_prefilter",
           "pmh_set_team_shape", "pmh_set_autotune", "pmh_last_team_shapes",
           "pmh_estimate_jp", "pmh_estimate_jp_block", "pmh_estimate_allpairs", "pmh_estimate_pairs", "pmh_merge", "pmh_check_exp1",
           "pmh_check_texp", "pmh_bbit_reduce", "pmh_bbit_allpairs", "pmh_pminhash_batch")

_lib = None
_lock = threading.Lock()


class PmhError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pmh status {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Loads libpmh.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libpmh.so not built ({path}); run paper_1911_00675_gb300/build.py")
            lib = ctypes.CDLL(path)
            vp, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            lib.pmh_create.restype = i32
            lib.pmh_create.argtypes = [ctypes.POINTER(vp), i32]
            lib.pmh_destroy.restype = None
            lib.pmh_destroy.argtypes = [vp]
            lib.pmh_last_error.restype = ctypes.c_char_p
            lib.pmh_last_error.argtypes = [vp]
            lib.pmh_sketch_batch.restype = i32
            lib.pmh_sketch_batch.argtypes = [vp, vp, vp, vp, i64, u32, ctypes.POINTER(i32), i32, i32, u64, vp, vp, vp,
                                             vp, vp]
            lib.pmh_sketch_batch_host.restype = i32
            lib.pmh_sketch_batch_host.argtypes = [vp, vp, vp, vp, i64, u32, ctypes.POINTER(i32), i32, i32, u64, vp, vp,
                                                  vp, i32]
            lib.pmh_last_host_span_ms.restype = i32
            lib.pmh_last_host_span_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)]
            lib.pmh_sketch_batch_noalloc.restype = i32
            lib.pmh_sketch_batch_noalloc.argtypes = [vp, vp, vp, i64, u32, ctypes.POINTER(i32), i32, i32, u64, vp, vp,
                                                     vp, vp, vp]
            lib.pmh_set_profiling.restype = i32
            lib.pmh_set_profiling.argtypes = [vp, i32]
            lib.pmh_last_kernel_ms.restype = i32
            lib.pmh_last_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
            lib.pmh_kernel_ms_history.restype = i32
            lib.pmh_kernel_ms_history.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float),
                                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)]
            lib.pmh_last_launches.restype = i32
            lib.pmh_last_launches.argtypes = [vp, ctypes.POINTER(i32)]
            lib.pmh_set_team_shape.restype = i32
            lib.pmh_set_team_shape.argtypes = [vp, i32, i32]
            lib.pmh_set_autotune.restype = i32
            lib.pmh_set_autotune.argtypes = [vp, i32]
            lib.pmh_last_team_shapes.restype = i32
            lib.pmh_last_team_shapes.argtypes = [vp, ctypes.POINTER(i32)]
            lib.pmh_set_thresholds.restype = i32
            lib.pmh_set_thresholds.argtypes = [vp, ctypes.c_double, ctypes.c_double, i32, i64]
            lib.pmh_set_te_sampler.restype = i32
            lib.pmh_set_te_sampler.argtypes = [vp, i32]
            lib.pmh_set_limits.restype = i32
            lib.pmh_set_limits.argtypes = [vp, u32, i32]
            lib.pmh_set_prefilter.restype = i32
            lib.pmh_set_prefilter.argtypes = [vp, ctypes.c_double]
            lib.pmh_sync_status.restype = i32
            lib.pmh_sync_status.argtypes = [vp, vp, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), vp]
            lib.pmh_estimate_jp.restype = i32
            lib.pmh_estimate_jp.argtypes = [vp, vp, i64, u32, i32, vp, vp]
            lib.pmh_estimate_jp_block.restype = i32
            lib.pmh_estimate_jp_block.argtypes = [vp, vp, i64, vp, i64, u32, vp, i64, vp]
            lib.pmh_estimate_allpairs.restype = i32
            lib.pmh_estimate_allpairs.argtypes = [vp, vp, i64, u32, i32, vp, vp]
            lib.pmh_estimate_pairs.restype = i32
            lib.pmh_estimate_pairs.argtypes = [vp, vp, vp, vp, vp, i64, u32, vp, vp]
            lib.pmh_check_exp1.restype = i32
            lib.pmh_check_exp1.argtypes = [vp, i64, vp, vp]
            lib.pmh_check_texp.restype = i32
            lib.pmh_check_texp.argtypes = [vp, i64, ctypes.c_float, ctypes.c_float, vp, vp]
            lib.pmh_bbit_reduce.restype = i32
            lib.pmh_bbit_reduce.argtypes = [vp, vp, i64, u32, u32, u64, vp, vp]
            lib.pmh_bbit_allpairs.restype = i32
            lib.pmh_bbit_allpairs.argtypes = [vp, vp, i64, u32, u32, i32, vp, vp]
            lib.pmh_pminhash_batch.restype = i32
            lib.pmh_pminhash_batch.argtypes = [vp, vp, vp, vp, i64, u32, u64, vp, vp, vp, vp]
            lib.pmh_merge.restype = i32
            lib.pmh_merge.argtypes = [vp, vp, vp, i64, u32, vp, vp, vp]
            _lib = lib
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(t, name, dtypes, device):
    if t is None:
        return
    if not t.is_cuda or t.device != device:
        raise ValueError(f"{name} must be a CUDA tensor on {device}")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


_I64 = (torch.int64, getattr(torch, "uint64", torch.int64))


class Handle:
    """Owns a pmh_handle bound to one CUDA device."""

    def __init__(self, device: int | None = None):
        lib = load()
        dev = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        rc = lib.pmh_create(ctypes.byref(h), dev)
        if rc:
            raise PmhError(rc, lib.pmh_last_error(None).decode())
        self._h = h
        self.device = torch.device("cuda", dev)

    def close(self):
        if getattr(self, "_h", None):
            load().pmh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, rc):
        if rc:
            raise PmhError(rc, load().pmh_last_error(self._h).decode())

    # -- pmh_sketch_batch ---------------------------------------------------
    def sketch_batch(self, ids, weights, offsets, m: int, variants=("1",), precision: int = FP32_RECHECK,
                     seed: int = 0, out_ids=None, out_q=None, status=None, counters=None, with_q: bool = False,
                     with_status: bool = True, stream=None):
        """Returns (out_ids [V, S, m] int64 view of the uint64 ids, out_q or None, status [V, S] or None)."""
        dev = self.device
        _check(ids, "ids", _I64, dev)
        _check(weights, "weights", (torch.float64,), dev)
        _check(offsets, "offsets", (torch.int64,), dev)
        vs = [VARIANTS[v] if isinstance(v, str) else int(v) for v in variants]
        s = offsets.numel() - 1
        if out_ids is None:
            out_ids = torch.empty((len(vs), s, m), dtype=torch.int64, device=dev)
        if out_q is None and with_q:
            out_q = torch.empty((len(vs), s, m), dtype=torch.float64, device=dev)
        if status is None and with_status:
            status = torch.empty((len(vs), s), dtype=torch.int32, device=dev)
        _check(out_ids, "out_ids", _I64, dev)
        _check(out_q, "out_q", (torch.float64,), dev)
        _check(status, "status", (torch.int32,), dev)
        _check(counters, "counters", _I64, dev)
        if counters is not None and counters.numel() < len(COUNTERS):
            raise ValueError(f"counters needs {len(COUNTERS)} entries")
        arr = (ctypes.c_int32 * len(vs))(*vs)
        rc = load().pmh_sketch_batch(self._h, _ptr(ids), _ptr(weights), _ptr(offsets), s, m, arr, len(vs),
                                     int(precision), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out_ids), _ptr(out_q),
                                     _ptr(status), _ptr(counters), _stream(stream))
        self._raise(rc)
        return out_ids, out_q, status

    # -- pmh_set_profiling / pmh_last_kernel_ms ------------------------------
    # -- pmh_sketch_batch_host ----------------------------------------------
    def sketch_batch_host(self, ids, weights, offsets, m: int, variants=("1",), precision: int = FP32_RECHECK,
                          seed: int = 0, out_ids=None, out_q=None, status=None, with_q: bool = False,
                          with_status: bool = True, chunks: int = 0):
        """Host-buffer sketch (CPU tensors, ideally pinned): returns (out_ids [V, S, m] int64 CPU tensor,
        out_q or None, status or None).  The library copies, sketches and copies back in a pipeline."""
        for t, name, dts in ((ids, "ids", _I64), (weights, "weights", (torch.float64,)), (offsets, "offsets", (torch.int64,))):
            if t.is_cuda or t.dtype not in dts or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CPU tensor of dtype {dts}")
        vs = [VARIANTS[v] if isinstance(v, str) else int(v) for v in variants]
        s = offsets.numel() - 1
        pin = torch.cuda.is_available()
        if out_ids is None:
            out_ids = torch.empty((len(vs), s, m), dtype=torch.int64, pin_memory=pin)
        if out_q is None and with_q:
            out_q = torch.empty((len(vs), s, m), dtype=torch.float64, pin_memory=pin)
        if status is None and with_status:
            status = torch.empty((len(vs), s), dtype=torch.int32, pin_memory=pin)
        arr = (ctypes.c_int32 * len(vs))(*vs)
        rc = load().pmh_sketch_batch_host(self._h, _ptr(ids), _ptr(weights), _ptr(offsets), s, m, arr, len(vs),
                                          int(precision), int(seed) & (2**64 - 1), _ptr(out_ids), _ptr(out_q),
                                          _ptr(status), int(chunks))
        self._raise(rc)
        return out_ids, out_q, status

    def last_host_span_ms(self):
        """(device-side ms from first copy-in to last copy-out, ranges) of the last sketch_batch_host call."""
        ms, k = ctypes.c_float(), ctypes.c_int32()
        self._raise(load().pmh_last_host_span_ms(self._h, ctypes.byref(ms), ctypes.byref(k)))
        return ms.value, k.value

    def set_profiling(self, enable: bool = True):
        self._raise(load().pmh_set_profiling(self._h, 1 if enable else 0))

    def kernel_ms_history(self, max_calls: int):
        """(queue_ms list, sketch_ms list) of up to max_calls most recent profiled calls, oldest first."""
        qa = (ctypes.c_float * max(1, max_calls))()
        ka = (ctypes.c_float * max(1, max_calls))()
        n = ctypes.c_int32()
        self._raise(load().pmh_kernel_ms_history(self._h, int(max_calls), qa, ka, ctypes.byref(n)))
        return list(qa[:n.value]), list(ka[:n.value])

    def last_launches(self) -> int:
        """Kernels launched by the most recent sketch_batch call."""
        n = ctypes.c_int32()
        self._raise(load().pmh_last_launches(self._h, ctypes.byref(n)))
        return n.value

    def set_team_shape(self, family: int = 0, shape: int = -1):
        """Pins the team shape of a family (1..4, 0 = all); -1 lets the handle choose."""
        self._raise(load().pmh_set_team_shape(self._h, int(family), int(shape)))

    def set_autotune(self, enable: int = 1):
        self._raise(load().pmh_set_autotune(self._h, int(enable)))

    def last_team_shapes(self):
        arr = (ctypes.c_int32 * 4)()
        self._raise(load().pmh_last_team_shapes(self._h, arr))
        return list(arr)

    def set_thresholds(self, t_c: float = 3.0, t_c_grid: float = 8.0, rounds: int = 5, grid_min: int = 1 << 20):
        """Work-only tuning of later sketch_batch calls (results never depend on it)."""
        self._raise(load().pmh_set_thresholds(self._h, float(t_c), float(t_c_grid), int(rounds), int(grid_min)))

    def set_limits(self, cap_points: int = 0, max_contenders: int = -1):
        """Iteration cap of warp-cooperative expansion (0 = default) and contender records kept per
        item (-1 = default); an item whose contender log overflows is redone in FP64."""
        self._raise(load().pmh_set_limits(self._h, int(cap_points), int(max_contenders)))

    def set_prefilter(self, list_factor: float = 2.0):
        """Prefilter lists for the first round of sets of at least list_factor * m (ln m + t_c)
        elements (<= 0: off); work only, results never depend on it."""
        self._raise(load().pmh_set_prefilter(self._h, float(list_factor)))

    def set_te_sampler(self, sampler: int = TE_INVERSION):
        """Exp(lambda;0,1) of ProbMinHash3/3a/4 by inversion (default) or by the paper's rejection sampler."""
        self._raise(load().pmh_set_te_sampler(self._h, int(sampler)))

    def sync_status(self, status, stream=None):
        """Waits for the stream, then (first failing status or 0, counts per code [8], first bad index)."""
        _check(status, "status", (torch.int32,), self.device)
        counts = (ctypes.c_int64 * 8)()
        first = ctypes.c_int64()
        rc = load().pmh_sync_status(self._h, _ptr(status), status.numel(), counts, ctypes.byref(first),
                                    _stream(stream))
        if rc in (ERR_CUDA,) or (rc and first.value < 0):
            self._raise(rc)
        return rc, list(counts), first.value

    def last_kernel_ms(self):
        """(queue build ms, sketch kernel ms) of the last profiled pmh_sketch_batch call."""
        a, b = ctypes.c_float(), ctypes.c_float()
        self._raise(load().pmh_last_kernel_ms(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # -- b-bit signatures ---------------------------------------------------
    def bbit_reduce(self, sigs, b: int, seed: int = 0, packed=None, stream=None):
        """Packed b-bit signatures [num_sigs, ceil(m b / 64)] (int64 view of uint64 words)."""
        _check(sigs, "sigs", _I64, self.device)
        n, m = sigs.shape
        words = (m * b + 63) // 64
        if packed is None:
            packed = torch.empty((n, words), dtype=torch.int64, device=self.device)
        self._raise(load().pmh_bbit_reduce(self._h, _ptr(sigs), n, m, int(b), int(seed) & (2**64 - 1), _ptr(packed),
                                           _stream(stream)))
        return packed

    def bbit_allpairs(self, packed, m: int, b: int, upper_only: bool = False, counts=None, stream=None):
        """Equal-field counts of all pairs of packed rows (int16 view of uint16)."""
        _check(packed, "packed", _I64, self.device)
        n = packed.shape[0]
        if counts is None:
            counts = torch.empty((n, n), dtype=torch.int16, device=self.device)
        self._raise(load().pmh_bbit_allpairs(self._h, _ptr(packed), n, int(m), int(b), 1 if upper_only else 0,
                                             _ptr(counts), _stream(stream)))
        return counts

    # -- pmh_estimate_jp ---------------------------------------------------
    def estimate_jp(self, sigs, upper_only: bool = False, counts=None, stream=None):
        """Equal-component counts of all signature pairs (int16 view of uint16); J_P estimate = counts / m."""
        _check(sigs, "sigs", _I64, self.device)
        n, m = sigs.shape
        if counts is None:
            counts = torch.zeros((n, n), dtype=torch.int16, device=self.device)   # uint16 storage
        _check(counts, "counts", (torch.int16, getattr(torch, "uint16", torch.int16)), self.device)
        rc = load().pmh_estimate_jp(self._h, _ptr(sigs), n, m, 1 if upper_only else 0, _ptr(counts), _stream(stream))
        self._raise(rc)
        return counts

    def estimate_jp_block(self, sig_a, sig_b, counts=None, stream=None):
        """Equal-component counts between the rows of two signature tables [na, nb] (int16 view of uint16)."""
        _check(sig_a, "sig_a", _I64, self.device)
        _check(sig_b, "sig_b", _I64, self.device)
        na, m = sig_a.shape
        nb = sig_b.shape[0]
        if sig_b.shape[1] != m:
            raise ValueError("sig_a and sig_b need the same m")
        if counts is None:
            counts = torch.zeros((na, nb), dtype=torch.int16, device=self.device)
        _check(counts, "counts", (torch.int16, getattr(torch, "uint16", torch.int16)), self.device)
        rc = load().pmh_estimate_jp_block(self._h, _ptr(sig_a), na, _ptr(sig_b), nb, m, _ptr(counts), counts.shape[1],
                                          _stream(stream))
        self._raise(rc)
        return counts

    def estimate_allpairs(self, sigs, upper_only: bool = False, counts=None, stream=None):
        """pmh_estimate_allpairs: the same call as estimate_jp under its earlier name."""
        _check(sigs, "sigs", _I64, self.device)
        n, m = sigs.shape
        if counts is None:
            counts = torch.zeros((n, n), dtype=torch.int16, device=self.device)
        _check(counts, "counts", (torch.int16, getattr(torch, "uint16", torch.int16)), self.device)
        rc = load().pmh_estimate_allpairs(self._h, _ptr(sigs), n, m, 1 if upper_only else 0, _ptr(counts),
                                          _stream(stream))
        self._raise(rc)
        return counts

    # -- pmh_estimate_pairs ------------------------------------------------
    def estimate_pairs(self, sig_a, sig_b, pairs_a, pairs_b, counts=None, stream=None):
        _check(sig_a, "sig_a", _I64, self.device)
        _check(sig_b, "sig_b", _I64, self.device)
        _check(pairs_a, "pairs_a", (torch.int64,), self.device)
        _check(pairs_b, "pairs_b", (torch.int64,), self.device)
        m = sig_a.shape[1]
        if counts is None:
            counts = torch.empty(pairs_a.numel(), dtype=torch.int32, device=self.device)
        rc = load().pmh_estimate_pairs(self._h, _ptr(sig_a), _ptr(sig_b), _ptr(pairs_a), _ptr(pairs_b),
                                       pairs_a.numel(), m, _ptr(counts), _stream(stream))
        self._raise(rc)
        return counts

    # -- pmh_pminhash_batch -------------------------------------------------
    def pminhash_batch(self, ids, weights, offsets, m: int, seed: int = 0, out_ids=None, out_q=None, status=None,
                       with_q: bool = False, stream=None):
        """Algorithm P-MinHash on a CSR batch: (out_ids [S, m], out_q or None, status [S])."""
        dev = self.device
        _check(ids, "ids", _I64, dev)
        _check(weights, "weights", (torch.float64,), dev)
        _check(offsets, "offsets", (torch.int64,), dev)
        s = offsets.numel() - 1
        if out_ids is None:
            out_ids = torch.empty((s, m), dtype=torch.int64, device=dev)
        if out_q is None and with_q:
            out_q = torch.empty((s, m), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(s, dtype=torch.int32, device=dev)
        rc = load().pmh_pminhash_batch(self._h, _ptr(ids), _ptr(weights), _ptr(offsets), s, m,
                                       int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out_ids), _ptr(out_q), _ptr(status),
                                       _stream(stream))
        self._raise(rc)
        return out_ids, out_q, status

    # -- pmh_merge ----------------------------------------------------------
    def merge(self, q, z, out_q=None, out_z=None, stream=None):
        _check(q, "q", (torch.float64,), self.device)
        _check(z, "z", _I64, self.device)
        parts, m = q.shape
        if out_q is None:
            out_q = torch.empty(m, dtype=torch.float64, device=self.device)
        if out_z is None:
            out_z = torch.empty(m, dtype=torch.int64, device=self.device)
        rc = load().pmh_merge(self._h, _ptr(q), _ptr(z), parts, m, _ptr(out_q), _ptr(out_z), _stream(stream))
        self._raise(rc)
        return out_q, out_z


_handles: dict[int, Handle] = {}


def handle(device: int | None = None) -> Handle:
    """The process-wide handle of a device (created on first use)."""
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _handles:
        _handles[dev] = Handle(dev)
    return _handles[dev]


def sketch_batch(ids, weights, offsets, m, variants=("1",), precision=FP32_RECHECK, seed=0, **kw):
    return handle(ids.device.index).sketch_batch(ids, weights, offsets, m, variants, precision, seed, **kw)


def sketch_batch_noalloc(ids, weights, offsets, m, variants=("1",), precision=FP32_RECHECK, seed=0, out_ids=None,
                         out_q=None, status=None, counters=None, with_q=False, stream=None):
    """pmh_sketch_batch_noalloc on the tensors' device (no handle, no GPU allocation inside the library).
    Outputs are allocated here only when not given."""
    dev = ids.device
    _check(ids, "ids", _I64, dev)
    _check(weights, "weights", (torch.float64,), dev)
    _check(offsets, "offsets", (torch.int64,), dev)
    vs = [VARIANTS[v] if isinstance(v, str) else int(v) for v in variants]
    s = offsets.numel() - 1
    if out_ids is None:
        out_ids = torch.empty((len(vs), s, m), dtype=torch.int64, device=dev)
    if out_q is None and with_q:
        out_q = torch.empty((len(vs), s, m), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty((len(vs), s), dtype=torch.int32, device=dev)
    _check(out_ids, "out_ids", _I64, dev)
    _check(out_q, "out_q", (torch.float64,), dev)
    _check(status, "status", (torch.int32,), dev)
    _check(counters, "counters", _I64, dev)
    if counters is not None and counters.numel() < len(COUNTERS):
        raise ValueError(f"counters needs {len(COUNTERS)} entries")
    arr = (ctypes.c_int32 * len(vs))(*vs)
    with torch.cuda.device(dev):
        rc = load().pmh_sketch_batch_noalloc(_ptr(ids), _ptr(weights), _ptr(offsets), s, m, arr, len(vs),
                                             int(precision), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out_ids),
                                             _ptr(out_q), _ptr(status), _ptr(counters), _stream(stream))
    if rc:
        raise PmhError(rc, load().pmh_last_error(None).decode())
    return out_ids, out_q, status


def estimate_jp(sigs, upper_only=False, **kw):
    return handle(sigs.device.index).estimate_jp(sigs, upper_only, **kw)


def estimate_allpairs(sigs, upper_only=False, **kw):
    return handle(sigs.device.index).estimate_allpairs(sigs, upper_only, **kw)


def estimate_pairs(sig_a, sig_b, pairs_a, pairs_b, **kw):
    return handle(sig_a.device.index).estimate_pairs(sig_a, sig_b, pairs_a, pairs_b, **kw)


def merge(q, z, **kw):
    return handle(q.device.index).merge(q, z, **kw)


def check_exp1(words, stream=None):
    """FP32 Exp(1) of each uint64 word as the candidate path computes it (CUDA int64 tensor in,
    float32 tensor out)."""
    out = torch.empty(words.numel(), dtype=torch.float32, device=words.device)
    rc = load().pmh_check_exp1(_ptr(words), words.numel(), _ptr(out), _stream(stream))
    if rc:
        raise PmhError(rc, "pmh_check_exp1 failed")
    return out


def check_texp(words, c: float, inv: float, stream=None):
    """FP32 truncated-exponential variate of each uint64 word as the candidate path computes it."""
    out = torch.empty(words.numel(), dtype=torch.float32, device=words.device)
    rc = load().pmh_check_texp(_ptr(words), words.numel(), float(c), float(inv), _ptr(out), _stream(stream))
    if rc:
        raise PmhError(rc, "pmh_check_texp failed")
    return out


def to_u64(t) -> "numpy.ndarray":
    """Host numpy uint64 copy of an int64-viewed id tensor."""
    return t.detach().cpu().numpy().view("uint64")
