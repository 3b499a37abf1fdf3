"""ProbMinHash oracle -- TEST INFRASTRUCTURE ONLY.

A ctypes loader for ``pmh_oracle.c``: a plain single-threaded FP64 C
restatement of the paper's algorithms (ProbMinHash1/1a/2/3/3a/4, brute force,
P-MinHash, exact J_P, the estimator).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline / reference arm
use it; the CUDA library never imports, links or calls anything here.

The shared object is built in-tree under ``oracle/_build`` with
``-ffp-contract=off`` so that no FMA contraction changes the fixed FP64
evaluation order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

V1, V1A, V2, V3, V3A, V4, V3U, V3AU, V4U = range(9)
VARIANTS = {"1": V1, "1a": V1A, "2": V2, "3": V3, "3a": V3A, "4": V4, "3u": V3U, "3au": V3AU, "4u": V4U}
OK, ERR_INVALID_ARG, ERR_BAD_WEIGHT, ERR_ITER_LIMIT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, u32, dbl, i32 = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double,
                                        ctypes.c_int)
            vp = ctypes.c_void_p
            lib.or_mix64.restype = u64; lib.or_mix64.argtypes = [u64]
            lib.or_key.restype = u64; lib.or_key.argtypes = [u64, u64]
            lib.or_word.restype = u64; lib.or_word.argtypes = [u64, u64]
            lib.or_unif.restype = dbl; lib.or_unif.argtypes = [u64]
            lib.or_exp1.restype = dbl; lib.or_exp1.argtypes = [u64]
            lib.or_texp.restype = dbl; lib.or_texp.argtypes = [u64, dbl, dbl]
            lib.or_uint.restype = u32; lib.or_uint.argtypes = [u64, u32]
            lib.or_tables.restype = i32; lib.or_tables.argtypes = [u32, vp, vp, vp, vp, vp]
            lib.or_track_max_run.restype = i32; lib.or_track_max_run.argtypes = [u32, vp, vp, i64, vp]
            lib.or_offer_run.restype = i32; lib.or_offer_run.argtypes = [u32, vp, vp, vp, i64, vp, vp]
            lib.or_perm_labels.restype = i32; lib.or_perm_labels.argtypes = [u32, u64, u32, vp]
            lib.or_sketch.restype = i32; lib.or_sketch.argtypes = [i32, i32, vp, vp, i64, u32, u64, vp, vp, vp]
            lib.or_sketch_opt.restype = i32
            lib.or_sketch_opt.argtypes = [i32, i32, i32, vp, vp, i64, u32, u64, vp, vp, vp]
            lib.or_near_ties_opt.restype = i64
            lib.or_near_ties_opt.argtypes = [i32, i32, vp, vp, i64, u32, u64, vp, vp, dbl, vp, vp]
            lib.or_texp_rej.restype = dbl
            lib.or_texp_rej.argtypes = [u64, u64, u64, dbl, ctypes.POINTER(ctypes.c_int)]
            lib.or_rej_consts.restype = None
            lib.or_rej_consts.argtypes = [dbl, vp]
            lib.or_sketch_batch.restype = i32
            lib.or_sketch_batch.argtypes = [i32, vp, vp, vp, i64, u32, u64, vp, vp, vp]
            lib.or_near_ties.restype = i64
            lib.or_near_ties.argtypes = [i32, vp, vp, i64, u32, u64, vp, vp, dbl, vp, vp]
            lib.or_pminhash.restype = i32; lib.or_pminhash.argtypes = [vp, vp, i64, u32, u64, vp, vp]
            lib.or_jp.restype = dbl; lib.or_jp.argtypes = [vp, vp, i64, vp, vp, i64]
            lib.or_count_equal.restype = u32; lib.or_count_equal.argtypes = [vp, vp, u32]
            lib.or_count_allpairs.restype = i32; lib.or_count_allpairs.argtypes = [vp, i64, u32, vp]
            lib.or_bbit_code.restype = u64; lib.or_bbit_code.argtypes = [u64, u32, u32, u64]
            lib.or_bbit_reduce.restype = i32; lib.or_bbit_reduce.argtypes = [vp, i64, u32, u32, u64, vp]
            lib.or_bbit_estimate.restype = dbl; lib.or_bbit_estimate.argtypes = [u32, u32, u32]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# -- stream primitives (exposed for pins) -----------------------------------
def mix64(z: int) -> int:
    return _load().or_mix64(z)


def key(elem_id: int, seed: int) -> int:
    return _load().or_key(elem_id, seed)


def word(k: int, j: int) -> int:
    return _load().or_word(k, j)


def unif(w: int) -> float:
    return _load().or_unif(w)


def exp1(w: int) -> float:
    return _load().or_exp1(w)


def texp(w: int, c: float, inv_lambda: float) -> float:
    return _load().or_texp(w, c, inv_lambda)


def uint(w: int, r: int) -> int:
    return _load().or_uint(w, r)


def tables(m: int):
    """(beta[0..m], gamma[0..m], dgamma[0..m], lambda_i[0..m], (lambda3, c3, inv3, delta))."""
    beta, gamma, dgamma, lam = (np.zeros(m + 1) for _ in range(4))
    sc = np.zeros(4)
    rc = _load().or_tables(m, _p(beta), _p(gamma), _p(dgamma), _p(lam), _p(sc))
    if rc:
        raise ValueError(f"or_tables({m}) -> {rc}")
    return beta, gamma, dgamma, lam, tuple(sc)


def track_max_run(m: int, values, leaves):
    """Apply (value, 0-based leaf) updates with the stop-limit tree; root after each."""
    h = _f64(values)
    k = np.ascontiguousarray(leaves, dtype=np.uint32)
    out = np.zeros(len(h))
    rc = _load().or_track_max_run(m, _p(h), _p(k), len(h), _p(out))
    if rc:
        raise ValueError(rc)
    return out


def offer_run(m: int, values, ids, comps):
    """Apply (value, id, 0-based component) offers in order; final (q, z)."""
    h = _f64(values)
    d = _u64(ids)
    k = np.ascontiguousarray(comps, dtype=np.uint32)
    q = np.zeros(m)
    z = np.zeros(m, dtype=np.uint64)
    rc = _load().or_offer_run(m, _p(h), _p(d), _p(k), len(h), _p(q), _p(z))
    if rc:
        raise ValueError(rc)
    return q, z


def perm_labels(m: int, k: int, steps: int):
    out = np.zeros(steps, dtype=np.uint32)
    rc = _load().or_perm_labels(m, k, steps, _p(out))
    if rc:
        raise ValueError(rc)
    return out


# -- sketches ----------------------------------------------------------------
TE_REJECTION = 1   # option flag: Exp(lambda;0,1) by the paper's rejection sampler (ProbMinHash3/3a/4)


def sketch(variant, ids, weights, m: int, seed: int = 0, brute: bool = False, te_rejection: bool = False):
    """Signature of one weighted set.  Returns (q[m], z[m], stats dict); raises on error codes."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    ids = _u64(ids)
    w = _f64(weights)
    q = np.zeros(m)
    z = np.zeros(m, dtype=np.uint64)
    st = np.zeros(5, dtype=np.uint64)
    rc = _load().or_sketch_opt(v, 1 if brute else 0, TE_REJECTION if te_rejection else 0, _p(ids), _p(w), len(ids),
                               m, seed, _p(q), _p(z), _p(st))
    if rc:
        raise OracleError(rc)
    stats = dict(zip(("elements", "points", "updates", "buffer_max", "passes"), (int(x) for x in st)))
    return q, z, stats


def sketch_status(variant, ids, weights, m: int, seed: int = 0) -> int:
    """Status code of a one-set sketch (no exception)."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    ids = _u64(ids)
    w = _f64(weights)
    q = np.zeros(max(m, 1))
    z = np.zeros(max(m, 1), dtype=np.uint64)
    return _load().or_sketch(v, 0, _p(ids), _p(w), len(ids), m, seed, _p(q), _p(z), None)


def sketch_batch(variant, ids, weights, offsets, m: int, seed: int = 0, with_q: bool = True):
    """CSR batch, single-threaded.  Returns (q or None, z, status)."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    ids = _u64(ids)
    w = _f64(weights)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    s = len(off) - 1
    q = np.zeros((s, m)) if with_q else None
    z = np.zeros((s, m), dtype=np.uint64)
    st = np.zeros(s, dtype=np.int32)
    _load().or_sketch_batch(v, _p(ids), _p(w), _p(off), s, m, seed, _p(q) if with_q else None, _p(z), _p(st))
    return q, z, st


def near_ties(variant, ids, weights, m: int, seed: int, q, z, rel: float = 1e-12, te_rejection: bool = False):
    """(flags[m] uint8, runner_up[m]).  Raises if the scan disagrees with (q, z)."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    ids = _u64(ids)
    w = _f64(weights)
    q = _f64(q)
    z = _u64(z)
    flags = np.zeros(m, dtype=np.uint8)
    ru = np.zeros(m)
    rc = _load().or_near_ties_opt(v, TE_REJECTION if te_rejection else 0, _p(ids), _p(w), len(ids), m, seed, _p(q),
                                  _p(z), rel, _p(flags), _p(ru))
    if rc < 0:
        raise OracleError(-rc)
    return flags, ru


def texp_rej(key: int, i: int, vw: int, lam: float):
    """(x, attempts): Exp(lam;0,1) by the rejection sampler for point i of the element with `key`,
    whose value word is vw (attempts = rejection-loop iterations, 0 when the first draw lands in A1)."""
    att = ctypes.c_int()
    x = _load().or_texp_rej(key, i, vw, lam, ctypes.byref(att))
    return x, att.value


def rej_consts(lam: float):
    """(c1, c2, c3) of the rejection sampler for rate lam."""
    out = np.zeros(3)
    _load().or_rej_consts(lam, _p(out))
    return tuple(out)


def pminhash(ids, weights, m: int, seed: int = 0):
    ids = _u64(ids)
    w = _f64(weights)
    q = np.zeros(m)
    z = np.zeros(m, dtype=np.uint64)
    rc = _load().or_pminhash(_p(ids), _p(w), len(ids), m, seed, _p(q), _p(z))
    if rc:
        raise OracleError(rc)
    return q, z


def jp(ids_a, w_a, ids_b, w_b) -> float:
    """Exact probability Jaccard similarity from its definition (O(u^2))."""
    a, wa, b, wb = _u64(ids_a), _f64(w_a), _u64(ids_b), _f64(w_b)
    return _load().or_jp(_p(a), _p(wa), len(a), _p(b), _p(wb), len(b))


def count_equal(za, zb) -> int:
    za, zb = _u64(za), _u64(zb)
    return _load().or_count_equal(_p(za), _p(zb), len(za))


def count_allpairs(sigs) -> np.ndarray:
    s = _u64(sigs)
    n, m = s.shape
    out = np.zeros((n, n), dtype=np.uint32)
    _load().or_count_allpairs(_p(s), n, m, _p(out))
    return out


def bbit_code(z: int, k: int, b: int, seed: int = 0) -> int:
    """b-bit code of component k with winning id z (Algorithm "Reduction to a b-bit signature")."""
    return _load().or_bbit_code(z & (2**64 - 1), k, b, seed & (2**64 - 1))


def bbit_reduce(sigs, b: int, seed: int = 0) -> np.ndarray:
    """b-bit codes of every component of a (num x m) signature array, unpacked (uint64)."""
    s = _u64(sigs)
    n, m = s.shape
    out = np.zeros((n, m), dtype=np.uint64)
    rc = _load().or_bbit_reduce(_p(s), n, m, b, seed & (2**64 - 1), _p(out))
    if rc:
        raise OracleError(rc)
    return out


def bbit_estimate(count: int, m: int, b: int) -> float:
    """Collision-corrected J estimate from the number of equal b-bit codes."""
    return _load().or_bbit_estimate(int(count), m, b)


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}")
        self.code = code
