"""CPU oracle for delegate-centric top-k (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It is independent of the CUDA library: it loads
its own C++ shared library (``drtopk_oracle.cpp``) and never the CUDA one.

Keys travel as their raw 32-bit patterns in ``numpy.uint32`` arrays together
with a dtype code (0 = u32, 1 = i32, 2 = f32); ``as_bits`` converts typed
numpy arrays. Every function cites the passage of the paper it follows in the
C++ source.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, the paper's worked example, closed forms and invariants).
"""

import ctypes
import numpy as np

from . import build as _build

U32, I32, F32 = 0, 1, 2
_DT = {np.dtype(np.uint32): U32, np.dtype(np.int32): I32, np.dtype(np.float32): F32}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        lib.oracle_map_keys.argtypes = [i32, p, i64, p]
        lib.oracle_unmap_keys.argtypes = [i32, p, i64, p]
        lib.oracle_topk.argtypes = [i32, p, i64, i64, p, p]
        lib.oracle_kth.argtypes = [i32, p, i64, i64, p]
        lib.oracle_delegates.argtypes = [p, i64, i32, i32, p, p]
        lib.oracle_delegates.restype = i64
        lib.oracle_threshold.argtypes = [p, p, i64, i64, p]
        lib.oracle_candidates.argtypes = [p, i64, i32, i32, p, p, ctypes.c_uint32,
                                          p, p, i64, p]
        lib.oracle_candidates.restype = i64
        lib.oracle_drtopk.argtypes = [i32, p, i64, i64, i32, i32, p, p, p]
        lib.oracle_alpha_rule4.argtypes = [i64, i64, ctypes.c_double]
        lib.oracle_bottomk.argtypes = [i32, p, i64, i64, p, p]
        lib.oracle_kth_smallest.argtypes = [i32, p, i64, i64, p]
        lib.oracle_topk_merge.argtypes = [i32, p, p, i64, i64, i32, p, p]
        lib.oracle_topk_omp.argtypes = [i32, p, i64, i64, i32, p, p, p]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def as_bits(x):
    """Typed numpy array (uint32 / int32 / float32) -> (raw uint32 bits, dtype code)."""
    x = np.ascontiguousarray(x)
    if x.dtype not in _DT:
        raise TypeError("unsupported dtype %s" % x.dtype)
    return x.view(np.uint32), _DT[x.dtype]


def from_bits(bits, dtype):
    """Raw uint32 bits + dtype code -> typed numpy array."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    return bits.view({U32: np.uint32, I32: np.int32, F32: np.float32}[dtype])


def map_keys(bits, dtype):
    """Order-preserving map of raw key bits to uint32 (reading G13)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    out = np.empty_like(bits)
    if _load().oracle_map_keys(dtype, _ptr(bits), bits.size, _ptr(out)) != 0:
        raise ValueError("bad dtype")
    return out


def unmap_keys(mapped, dtype):
    mapped = np.ascontiguousarray(mapped, dtype=np.uint32)
    out = np.empty_like(mapped)
    if _load().oracle_unmap_keys(dtype, _ptr(mapped), mapped.size, _ptr(out)) != 0:
        raise ValueError("bad dtype")
    return out


def topk(bits, dtype, k):
    """Plain top-k (Sec. 1): (key bits, int32 indices), sorted (key desc, idx asc)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    ok = np.empty(k, np.uint32)
    oi = np.empty(k, np.int32)
    rc = _load().oracle_topk(dtype, _ptr(bits), bits.size, k, _ptr(ok), _ptr(oi))
    if rc != 0:
        raise ValueError("oracle_topk rc=%d" % rc)
    return ok, oi


def kth(bits, dtype, k):
    """Plain k-selection (Sec. 1): raw bits of the k-th largest key."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    out = np.zeros(1, np.uint32)
    rc = _load().oracle_kth(dtype, _ptr(bits), bits.size, k, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_kth rc=%d" % rc)
    return int(out[0])


def bottomk(bits, dtype, k):
    """Plain smallest-k (Sec. 1, Sec. 2): (key bits, int32 indices), sorted
    (key asc, idx asc)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    ok = np.empty(k, np.uint32)
    oi = np.empty(k, np.int32)
    rc = _load().oracle_bottomk(dtype, _ptr(bits), bits.size, k, _ptr(ok), _ptr(oi))
    if rc != 0:
        raise ValueError("oracle_bottomk rc=%d" % rc)
    return ok, oi


def kth_smallest(bits, dtype, k):
    """Raw bits of the k-th smallest key."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    out = np.zeros(1, np.uint32)
    rc = _load().oracle_kth_smallest(dtype, _ptr(bits), bits.size, k, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_kth_smallest rc=%d" % rc)
    return int(out[0])


def topk_merge(bits, gidx, dtype, k, smallest=False):
    """Distributed form's final step (Sec. 4.4): top-k of (key bits, int64
    global index) pairs in any order -> (key bits, int64 global indices)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    gidx = np.ascontiguousarray(gidx, dtype=np.int64)
    ok = np.empty(k, np.uint32)
    og = np.empty(k, np.int64)
    rc = _load().oracle_topk_merge(dtype, _ptr(bits), _ptr(gidx), bits.size, k,
                                   1 if smallest else 0, _ptr(ok), _ptr(og))
    if rc != 0:
        raise ValueError("oracle_topk_merge rc=%d" % rc)
    return ok, og


def topk_omp(bits, dtype, k, threads=0):
    """Multi-core chunked top-k (same result as topk): (keys, idx, threads used)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    ok = np.empty(k, np.uint32)
    oi = np.empty(k, np.int32)
    used = np.zeros(1, np.int32)
    rc = _load().oracle_topk_omp(dtype, _ptr(bits), bits.size, k, threads, _ptr(ok),
                                 _ptr(oi), _ptr(used))
    if rc != 0:
        raise ValueError("oracle_topk_omp rc=%d" % rc)
    return ok, oi, int(used[0])


def delegates(mapped, alpha, beta):
    """Rules 1 and 3: per-subrange top-beta (keys, global idx), shape (S, beta)."""
    mapped = np.ascontiguousarray(mapped, dtype=np.uint32)
    n = mapped.size
    S = (n + (1 << alpha) - 1) >> alpha
    dk = np.zeros(S * beta, np.uint32)
    di = np.zeros(S * beta, np.int64)
    r = _load().oracle_delegates(_ptr(mapped), n, alpha, beta, _ptr(dk), _ptr(di))
    if r != S:
        raise ValueError("oracle_delegates failed")
    return dk.reshape(S, beta), di.reshape(S, beta)


def threshold(dk, di, k):
    """Rule 2: tau = k-th largest delegate (0 when D holds fewer than k)."""
    dk = np.ascontiguousarray(dk, dtype=np.uint32).ravel()
    di = np.ascontiguousarray(di, dtype=np.int64).ravel()
    out = np.zeros(1, np.uint32)
    if _load().oracle_threshold(_ptr(dk), _ptr(di), dk.size, k, _ptr(out)) != 0:
        raise ValueError("bad k")
    return int(out[0])


def candidates(mapped, alpha, beta, dk, di, tau):
    """Rules 1-3 concatenation with filtering: (keys, idx, scanned subranges)."""
    mapped = np.ascontiguousarray(mapped, dtype=np.uint32)
    dk = np.ascontiguousarray(dk, dtype=np.uint32).ravel()
    di = np.ascontiguousarray(di, dtype=np.int64).ravel()
    lib = _load()
    sc = np.zeros(1, np.int64)
    c = lib.oracle_candidates(_ptr(mapped), mapped.size, alpha, beta, _ptr(dk),
                              _ptr(di), tau, None, None, 0, _ptr(sc))
    ck = np.zeros(max(c, 1), np.uint32)
    ci = np.zeros(max(c, 1), np.int64)
    lib.oracle_candidates(_ptr(mapped), mapped.size, alpha, beta, _ptr(dk),
                          _ptr(di), tau, _ptr(ck), _ptr(ci), c, _ptr(sc))
    return ck[:c], ci[:c], int(sc[0])


def drtopk(bits, dtype, k, alpha, beta):
    """The method's four steps (Eq. 1) -> (keys, idx, stats dict)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    ok = np.empty(k, np.uint32)
    oi = np.empty(k, np.int32)
    st = np.zeros(4, np.int64)
    rc = _load().oracle_drtopk(dtype, _ptr(bits), bits.size, k, alpha, beta,
                               _ptr(ok), _ptr(oi), _ptr(st))
    if rc != 0:
        raise ValueError("oracle_drtopk rc=%d" % rc)
    return ok, oi, {"tau": int(st[0]), "candidates": int(st[1]),
                    "scanned": int(st[2]), "subranges": int(st[3])}


def alpha_rule4(n, k, const=3.0):
    """Rule 4 / Eq. 9: floor(1/2 (log2 n - log2 k + const))."""
    return int(_load().oracle_alpha_rule4(n, k, const))
