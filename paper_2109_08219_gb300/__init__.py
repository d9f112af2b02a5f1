"""GB300-native delegate-centric top-k (Dr. Top-k, SC'21, arXiv 2109.08219).

Thin Python binding of the C ABI declared in ``include/drtopk.h``: every
function below marshals its arguments and calls the CUDA library
``_build/libdrtopk.so`` of this package; all work runs in its kernels.
PyTorch is used only for device memory and streams. There is no CPU
fallback: a missing library raises ``DrTopkError``.

Key dtypes: ``"u32"``, ``"i32"``, ``"f32"``. A torch.float32 tensor is f32,
torch.int32 is i32 unless ``dtype="u32"`` is passed (torch has little uint32
arithmetic, so u32 keys usually travel as int32 tensors holding the bits),
torch.uint32 is u32.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdrtopk.so")

U32, I32, F32 = 0, 1, 2
_NAMES = {"u32": U32, "i32": I32, "f32": F32}

STATUS = ["DRTOPK_OK", "DRTOPK_ERR_INVALID", "DRTOPK_ERR_K", "DRTOPK_ERR_DTYPE",
          "DRTOPK_ERR_NOMEM", "DRTOPK_ERR_CUDA", "DRTOPK_ERR_BUDGET",
          "DRTOPK_ERR_TIMEOUT", "DRTOPK_PENDING", "DRTOPK_ERR_INTERNAL"]
NUM_STAGES = 6
STAGE_NAMES = ["delegate", "threshold", "filter", "ties", "second_select", "sort"]
BATCH_PHASES = ["delegate", "threshold", "filter", "second_select", "ties", "sort_output",
                "direct_load", "direct_select", "direct_collect", "direct_sort_output"]


class DrTopkError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__("%s%s" % (name, (" in " + where) if where else ""))


class Stats(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("subranges", ctypes.c_int64), ("tau", ctypes.c_uint32),
                ("kth_mapped", ctypes.c_uint32), ("greater", ctypes.c_int64),
                ("ties_needed", ctypes.c_int64), ("scanned", ctypes.c_int64),
                ("tie_scanned", ctypes.c_int64), ("survivors", ctypes.c_int64),
                ("emitted", ctypes.c_int64), ("error", ctypes.c_uint32),
                ("delegate_path", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in
                ("submitted", "completed", "failed", "batches", "batched_requests",
                 "single_queries", "peak_bytes", "in_use_bytes", "fixed_bytes")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NUM_STAGES),
                ("launches", ctypes.c_int64 * NUM_STAGES)]


_lib = None


def lib():
    """The loaded C library (raises DrTopkError-like OSError when missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("drtopk CUDA library not built: %s (run __graft_entry__.build())"
                          % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.drtopk_status_str.argtypes = [i32]
        L.drtopk_status_str.restype = ctypes.c_char_p
        L.drtopk_plan.argtypes = [i64, i64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                  ctypes.POINTER(ctypes.c_size_t)]
        L.drtopk_kth.argtypes = [p, i32, i64, i64, p, p]
        L.drtopk_topk.argtypes = [p, i32, i64, i64, p, p, p]
        L.drtopk_topk_ex.argtypes = [p, i32, i64, i64, i32, i32, p, p, p,
                                     ctypes.POINTER(Stats), p]
        L.drtopk_delegates.argtypes = [p, i32, i64, i32, i32, p, p, p]
        L.drtopk_topk_ablate.argtypes = [p, i32, i64, i64, i32, i32, i32, p, p,
                                         ctypes.POINTER(Stats), p]
        L.drtopk_topk_host.argtypes = [p, i32, i64, i64, p, p, p]
        L.drtopk_kth_noalloc.argtypes = [p, i32, i64, i64, p, p]
        L.drtopk_kth_noalloc.restype = i32
        L.drtopk_select.argtypes = [p, i32, i64, i64, i32, p, p, p, p]
        L.drtopk_topk_merge.argtypes = [p, p, i32, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), i32, i64, i32, p, p, p]
        L.drtopk_sync_status.argtypes = [p]
        L.drtopk_wait_selftest.argtypes = [ctypes.c_uint32, p]
        L.drtopk_profile_begin.argtypes = []
        L.drtopk_profile_end.argtypes = [ctypes.POINTER(Profile)]
        L.drtopk_launch_count.argtypes = []
        L.drtopk_launch_count.restype = ctypes.c_uint64
        L.drtopk_alloc_count.argtypes = []
        L.drtopk_alloc_count.restype = ctypes.c_uint64
        pi32 = ctypes.POINTER(ctypes.c_int32)
        pi64 = ctypes.POINTER(ctypes.c_int64)
        L.drtopk_batch_plan_create.argtypes = [i32, pi64, pi32, i32, i32, i32,
                                               ctypes.POINTER(p)]
        L.drtopk_batch_plan_run.argtypes = [p, p, p, p, p]
        L.drtopk_batch_plan_status.argtypes = [p, p]
        L.drtopk_batch_plan_params.argtypes = [p, pi32, pi32]
        L.drtopk_batch_plan_destroy.argtypes = [p]
        L.drtopk_batch_plan_phase_cycles.argtypes = [p, ctypes.POINTER(ctypes.c_uint64), i32, p]
        L.drtopk_topk_batched.argtypes = [p, i32, pi64, pi32, i32, p, p, p]
        L.drtopk_batch_limits.argtypes = [pi32, pi64, pi32, pi32, pi32, pi32]
        L.drtopk_server_create_ex.argtypes = [ctypes.c_size_t, i32, i32, i64, ctypes.POINTER(p)]
        L.drtopk_server_submit.argtypes = [p, p, i32, i64, i64, p, p,
                                           ctypes.POINTER(ctypes.c_uint64)]
        L.drtopk_server_poll_ex.argtypes = [p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
        L.drtopk_server_wait.argtypes = [p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
        L.drtopk_server_get_stats.argtypes = [p, ctypes.POINTER(ServerStats)]
        L.drtopk_server_footprint.argtypes = [i32, i64, i64, i32, i64,
                                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i32)]
        L.drtopk_server_destroy.argtypes = [p]
        L.drtopk_tune_get.argtypes = [i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.drtopk_tune_set.argtypes = [i32, i32, i32, i32]
        L.drtopk_autotune_batched.argtypes = [i32, i32, i32, i32, p]
        for fn in ("drtopk_select", "drtopk_topk_merge", "drtopk_sync_status", "drtopk_wait_selftest", "drtopk_plan", "drtopk_kth", "drtopk_topk", "drtopk_topk_ex", "drtopk_topk_ablate",
                   "drtopk_delegates", "drtopk_topk_host", "drtopk_profile_begin",
                   "drtopk_profile_end", "drtopk_batch_plan_create", "drtopk_batch_plan_run",
                   "drtopk_batch_plan_status", "drtopk_batch_plan_params",
                   "drtopk_batch_plan_destroy", "drtopk_batch_plan_phase_cycles",
                   "drtopk_topk_batched", "drtopk_batch_limits", "drtopk_tune_get",
                   "drtopk_tune_set", "drtopk_autotune_batched", "drtopk_server_create_ex",
                   "drtopk_server_submit", "drtopk_server_poll_ex", "drtopk_server_wait",
                   "drtopk_server_get_stats", "drtopk_server_footprint",
                   "drtopk_server_destroy"):
            getattr(L, fn).restype = i32
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        raise DrTopkError(rc, where)


def _dtype_code(t, dtype):
    import torch
    if dtype is not None:
        if dtype not in _NAMES:
            raise ValueError("dtype must be one of u32, i32, f32")
        code = _NAMES[dtype]
        if t.element_size() != 4:
            raise ValueError("keys must be 32-bit")
        return code
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.int32:
        return I32
    if t.dtype == getattr(torch, "uint32", None):
        return U32
    raise ValueError("unsupported key dtype %s" % t.dtype)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def status_str(status):
    return lib().drtopk_status_str(status).decode()


def sync_status(stream=None):
    """Synchronizes the stream and raises DrTopkError when queries on the
    current device reported a device-side error since the last check
    (drtopk_sync_status); the flags are cleared."""
    _check(lib().drtopk_sync_status(_stream(stream)), "drtopk_sync_status")


def wait_selftest(timeout_us, stream=None):
    """Launches the bounded-wait self-test kernel (drtopk_wait_selftest):
    a wait on a phase nothing completes, given up after timeout_us."""
    _check(lib().drtopk_wait_selftest(timeout_us, _stream(stream)), "drtopk_wait_selftest")


def drtopk_plan(n, k):
    """Rule 4 parameter choice: (alpha, beta, workspace_bytes). Host only."""
    a, b, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check(lib().drtopk_plan(n, k, ctypes.byref(a), ctypes.byref(b), ctypes.byref(w)),
           "drtopk_plan")
    return a.value, b.value, w.value


def drtopk_kth(keys, k, out=None, dtype=None, stream=None):
    """k-th largest key of a 1-D CUDA tensor; returns a 1-element tensor."""
    import torch
    code = _dtype_code(keys, dtype)
    if out is None:
        out = torch.empty(1, dtype=keys.dtype, device=keys.device)
    _check(lib().drtopk_kth(_dev(keys), code, keys.numel(), k, _dev(out), _stream(stream)),
           "drtopk_kth")
    return out


def drtopk_kth_noalloc(keys, k, out=None, dtype=None, stream=None):
    """k-th largest key using the library's fixed 64 MiB device scratch: no
    device allocation happens in the call. For callers that may not allocate
    while serving queries. Raises DrTopkError(DRTOPK_ERR_NOMEM) when the
    query needs more scratch than the array holds. Calls that overlap on the
    GPU share the array and race: keep them ordered on one stream."""
    import torch
    code = _dtype_code(keys, dtype)
    if out is None:
        out = torch.empty(1, dtype=keys.dtype, device=keys.device)
    _check(lib().drtopk_kth_noalloc(_dev(keys), code, keys.numel(), k, _dev(out),
                                    _stream(stream)), "drtopk_kth_noalloc")
    return out


def drtopk_topk(keys, k, out_keys=None, out_idx=None, dtype=None, stream=None):
    """Top-k of a 1-D CUDA tensor: (keys, int32 indices), sorted by (key desc,
    index asc); ties go to the smallest index."""
    import torch
    code = _dtype_code(keys, dtype)
    if out_keys is None:
        out_keys = torch.empty(k, dtype=keys.dtype, device=keys.device)
    if out_idx is None:
        out_idx = torch.empty(k, dtype=torch.int32, device=keys.device)
    _check(lib().drtopk_topk(_dev(keys), code, keys.numel(), k, _dev(out_keys), _dev(out_idx),
                             _stream(stream)), "drtopk_topk")
    return out_keys, out_idx


SMALLEST = 1


def drtopk_select(keys, k, smallest=False, want_topk=True, want_kth=False, dtype=None,
                  stream=None):
    """Top-k and / or k-th of a 1-D CUDA tensor by the largest (default) or
    smallest criterion (drtopk_select). Returns (keys, int32 indices, kth),
    None for what was not asked; sorted by (key desc or asc, index asc)."""
    import torch
    code = _dtype_code(keys, dtype)
    ok = oi = ot = None
    if want_topk:
        ok = torch.empty(k, dtype=keys.dtype, device=keys.device)
        oi = torch.empty(k, dtype=torch.int32, device=keys.device)
    if want_kth:
        ot = torch.empty(1, dtype=keys.dtype, device=keys.device)
    _check(lib().drtopk_select(_dev(keys), code, keys.numel(), k, SMALLEST if smallest else 0,
                               _dev(ok) if ok is not None else None,
                               _dev(oi) if oi is not None else None,
                               _dev(ot) if ot is not None else None, _stream(stream)),
           "drtopk_select")
    return ok, oi, ot


def drtopk_topk_merge(keys, idx, part_off, part_base, k, smallest=False, dtype=None,
                      stream=None):
    """Final top-k of gathered per-shard lists (drtopk_topk_merge): keys /
    idx are the concatenated results of drtopk_select on each shard (in
    shard order), part_off the list boundaries (parts + 1) and part_base
    each shard's global index base. Returns (keys, int64 global indices)."""
    import numpy as np
    import torch
    code = _dtype_code(keys, dtype)
    off = np.ascontiguousarray(np.asarray(part_off, dtype=np.int64))
    base = np.ascontiguousarray(np.asarray(part_base, dtype=np.int64))
    if off.size != base.size + 1:
        raise ValueError("part_off needs parts + 1 entries and part_base parts entries")
    if idx.dtype != torch.int32:
        raise ValueError("idx must be int32")
    if keys.numel() < int(off[-1]) or idx.numel() < int(off[-1]):
        raise ValueError("keys / idx shorter than part_off[-1]")
    ok = torch.empty(k, dtype=keys.dtype, device=keys.device)
    og = torch.empty(k, dtype=torch.int64, device=keys.device)
    _check(lib().drtopk_topk_merge(_dev(keys), _dev(idx), code,
                                   off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   base.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   int(base.size), k, SMALLEST if smallest else 0, _dev(ok),
                                   _dev(og), _stream(stream)), "drtopk_topk_merge")
    return ok, og


def drtopk_topk_ex(keys, k, alpha=0, beta=0, want_topk=True, want_kth=True, dtype=None,
                   stats=True, stream=None):
    """Extended query with forced alpha/beta and statistics.

    Returns (out_keys or None, out_idx or None, out_kth or None, stats dict or
    None). With stats=True the call synchronizes the stream."""
    import torch
    code = _dtype_code(keys, dtype)
    ok = oi = ot = None
    if want_topk:
        ok = torch.empty(k, dtype=keys.dtype, device=keys.device)
        oi = torch.empty(k, dtype=torch.int32, device=keys.device)
    if want_kth:
        ot = torch.empty(1, dtype=keys.dtype, device=keys.device)
    st = Stats() if stats else None
    rc = lib().drtopk_topk_ex(_dev(keys), code, keys.numel(), k, alpha, beta,
                              _dev(ok) if ok is not None else None,
                              _dev(oi) if oi is not None else None,
                              _dev(ot) if ot is not None else None,
                              ctypes.byref(st) if st is not None else None, _stream(stream))
    _check(rc, "drtopk_topk_ex")
    return ok, oi, ot, (st.as_dict() if st is not None else None)


ABLATE_NO_FILTER = 1
ABLATE_SKIP_LAST_DIGIT = 2


def drtopk_topk_ablate(keys, k, alpha=0, beta=0, no_filter=False, skip_last_digit=False,
                       dtype=None, stats=True, out_keys=None, out_idx=None, stream=None):
    """Top-k with an ablation of the method (drtopk_topk_ablate): Rule 2's
    filtering off and/or the first select stopped one digit early. Returns
    (out_keys, out_idx, stats dict or None); with stats=True the call
    synchronizes the stream, without it the call is asynchronous (and may
    be captured in a CUDA graph)."""
    import torch
    code = _dtype_code(keys, dtype)
    if out_keys is None:
        out_keys = torch.empty(k, dtype=keys.dtype, device=keys.device)
    if out_idx is None:
        out_idx = torch.empty(k, dtype=torch.int32, device=keys.device)
    st = Stats() if stats else None
    flags = (ABLATE_NO_FILTER if no_filter else 0) | (ABLATE_SKIP_LAST_DIGIT if skip_last_digit else 0)
    _check(lib().drtopk_topk_ablate(_dev(keys), code, keys.numel(), k, alpha, beta, flags,
                                    _dev(out_keys), _dev(out_idx),
                                    ctypes.byref(st) if st is not None else None,
                                    _stream(stream)), "drtopk_topk_ablate")
    return out_keys, out_idx, (st.as_dict() if st is not None else None)


def drtopk_delegates(keys, alpha, beta, dtype=None, stream=None):
    """Delegate pass alone: (mapped delegate keys as int32 bits [S, beta],
    int32 positions [S, beta]); pads are key 0 / index -1."""
    import torch
    code = _dtype_code(keys, dtype)
    n = keys.numel()
    S = (n + (1 << alpha) - 1) >> alpha
    dk = torch.empty(S * beta, dtype=torch.int32, device=keys.device)
    di = torch.empty(S * beta, dtype=torch.int32, device=keys.device)
    _check(lib().drtopk_delegates(_dev(keys), code, n, alpha, beta, _dev(dk), _dev(di),
                                  _stream(stream)), "drtopk_delegates")
    return dk.view(S, beta), di.view(S, beta)


def drtopk_topk_host(keys_np, k, dtype, stream=None):
    """Top-k of a host numpy array (uint32/int32/float32 view given by dtype).
    Returns numpy (keys, int32 indices). Synchronous."""
    import numpy as np
    keys_np = np.ascontiguousarray(keys_np)
    if keys_np.itemsize != 4:
        raise ValueError("keys must be 32-bit")
    ok = np.empty(k, dtype=keys_np.dtype)
    oi = np.empty(k, dtype=np.int32)
    _check(lib().drtopk_topk_host(keys_np.ctypes.data_as(ctypes.c_void_p), _NAMES[dtype],
                                  keys_np.size, k, ok.ctypes.data_as(ctypes.c_void_p),
                                  oi.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "drtopk_topk_host")
    return ok, oi


def drtopk_topk_host_ptr(keys_ptr, n, k, dtype, out_keys_ptr, out_idx_ptr, stream=None):
    """Top-k of a host buffer given by raw pointers (e.g. pinned torch tensors)."""
    _check(lib().drtopk_topk_host(ctypes.c_void_p(keys_ptr), _NAMES[dtype], n, k,
                                  ctypes.c_void_p(out_keys_ptr), ctypes.c_void_p(out_idx_ptr),
                                  _stream(stream)), "drtopk_topk_host")


def profile_begin():
    _check(lib().drtopk_profile_begin(), "drtopk_profile_begin")


def profile_end():
    """Stage times since profile_begin: {stage: (ms_total, count)}."""
    pr = Profile()
    _check(lib().drtopk_profile_end(ctypes.byref(pr)), "drtopk_profile_end")
    return {STAGE_NAMES[i]: (pr.ms[i], pr.launches[i]) for i in range(NUM_STAGES)}


def launch_count():
    return int(lib().drtopk_launch_count())


def alloc_count():
    """Allocations the library has made since it was loaded (drtopk_alloc_count)."""
    return int(lib().drtopk_alloc_count())


# ------------------------------------------------------------------ batched --
def _rows_arrays(row_off, ks):
    import numpy as np
    off = np.ascontiguousarray(np.asarray(row_off, dtype=np.int64))
    kk = np.ascontiguousarray(np.asarray(ks, dtype=np.int32))
    if off.ndim != 1 or kk.ndim != 1 or off.size != kk.size + 1:
        raise ValueError("row_off needs rows + 1 entries and ks rows entries")
    return off, kk


class BatchPlan:
    """A reusable plan of the batched top-k for a fixed row layout
    (drtopk_batch_plan_*). ``row_off`` (rows + 1 offsets) and ``ks`` are host
    sequences; ``run`` launches one kernel and may be graph-captured."""

    def __init__(self, row_off, ks, dtype, alpha=0, beta=0):
        import numpy as np
        self.row_off, self.ks = _rows_arrays(row_off, ks)
        if dtype not in _NAMES:
            raise ValueError("dtype must be one of u32, i32, f32")
        self.dtype = dtype
        self.rows = int(self.ks.size)
        self.out_off = np.concatenate([[0], np.cumsum(self.ks, dtype=np.int64)])
        self._h = ctypes.c_void_p()
        _check(lib().drtopk_batch_plan_create(
            _NAMES[dtype], self.row_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            self.ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self.rows, alpha, beta,
            ctypes.byref(self._h)), "drtopk_batch_plan_create")

    @property
    def total_k(self):
        return int(self.out_off[-1])

    def params(self):
        import numpy as np
        a = np.zeros(self.rows, np.int32)
        b = np.zeros(self.rows, np.int32)
        _check(lib().drtopk_batch_plan_params(
            self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "drtopk_batch_plan_params")
        return a, b

    def run(self, keys, out_keys=None, out_idx=None, stream=None):
        import torch
        if out_keys is None:
            out_keys = torch.empty(self.total_k, dtype=keys.dtype, device=keys.device)
        if out_idx is None:
            out_idx = torch.empty(self.total_k, dtype=torch.int32, device=keys.device)
        if keys.numel() < int(self.row_off[-1]) or out_keys.numel() < self.total_k \
                or out_idx.numel() < self.total_k:
            raise ValueError("buffers smaller than the plan's rows")
        _check(lib().drtopk_batch_plan_run(self._h, _dev(keys), _dev(out_keys), _dev(out_idx),
                                           _stream(stream)), "drtopk_batch_plan_run")
        return out_keys, out_idx

    def status(self, stream=None):
        _check(lib().drtopk_batch_plan_status(self._h, _stream(stream)),
               "drtopk_batch_plan_status")

    def phase_cycles(self, reset=False, stream=None):
        """Cycles per step of the batched kernel, summed over CTAs and runs:
        a dict over BATCH_PHASES."""
        out = (ctypes.c_uint64 * len(BATCH_PHASES))()
        _check(lib().drtopk_batch_plan_phase_cycles(self._h, out, 1 if reset else 0,
                                                    _stream(stream)),
               "drtopk_batch_plan_phase_cycles")
        return {name: int(v) for name, v in zip(BATCH_PHASES, out)}

    def close(self):
        if self._h:
            lib().drtopk_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def drtopk_topk_batched(keys, row_off, ks, dtype=None, stream=None):
    """One-shot batched top-k (synchronous). Returns (out_keys, out_idx),
    packed by row: row r owns entries [sum(ks[:r]), sum(ks[:r+1]))."""
    import torch
    off, kk = _rows_arrays(row_off, ks)
    code = _dtype_code(keys, dtype)
    total = int(kk.sum(dtype="int64"))
    out_keys = torch.empty(total, dtype=keys.dtype, device=keys.device)
    out_idx = torch.empty(total, dtype=torch.int32, device=keys.device)
    if keys.numel() < int(off[-1]):
        raise ValueError("keys shorter than row_off[-1]")
    _check(lib().drtopk_topk_batched(
        _dev(keys), code, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        kk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(kk.size), _dev(out_keys),
        _dev(out_idx), _stream(stream)), "drtopk_topk_batched")
    return out_keys, out_idx


def batch_limits():
    """Limits of the batched path (drtopk_batch_limits) as a dict."""
    mk, mr, dm, do, md, oc = (ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(),
                              ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32())
    _check(lib().drtopk_batch_limits(ctypes.byref(mk), ctypes.byref(mr), ctypes.byref(dm),
                                     ctypes.byref(do), ctypes.byref(md), ctypes.byref(oc)),
           "drtopk_batch_limits")
    return {"max_k": mk.value, "max_row": mr.value, "direct_max": dm.value,
            "direct_max_onchip": do.value, "max_delegates": md.value,
            "onchip_candidates": oc.value}


def tune_get(log2n, log2k):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().drtopk_tune_get(log2n, log2k, ctypes.byref(a), ctypes.byref(b)),
           "drtopk_tune_get")
    return a.value, b.value


def tune_set(log2n, log2k, alpha, beta):
    _check(lib().drtopk_tune_set(log2n, log2k, alpha, beta), "drtopk_tune_set")


def autotune_batched(dtype, min_log2n, max_log2n, rows_per_shape=152, stream=None):
    """Measures (alpha, beta) per shape bucket and fills the tuning table."""
    _check(lib().drtopk_autotune_batched(_NAMES[dtype], min_log2n, max_log2n, rows_per_shape,
                                         _stream(stream)), "drtopk_autotune_batched")


# ------------------------------------------------------------------- server --
SERVER_PLAIN = 1
PENDING = 8


def server_footprint(n, k, dtype="f32", flags=0, batch_max_n=0):
    """(bytes counted against the budget, batched?) of a request. Host only."""
    b, bt = ctypes.c_size_t(), ctypes.c_int()
    _check(lib().drtopk_server_footprint(_NAMES[dtype], n, k, flags, batch_max_n,
                                         ctypes.byref(b), ctypes.byref(bt)),
           "drtopk_server_footprint")
    return b.value, bool(bt.value)


class Server:
    """Continuous-batching top-k server (drtopk_server_*). Requests are
    device tensors owned by the caller; keep them alive until done."""

    def __init__(self, hbm_budget_bytes, device=0, plain=False, batch_max_n=0):
        self._h = ctypes.c_void_p()
        _check(lib().drtopk_server_create_ex(hbm_budget_bytes, device,
                                             SERVER_PLAIN if plain else 0, batch_max_n,
                                             ctypes.byref(self._h)), "drtopk_server_create")

    def submit(self, keys, k, out_keys, out_idx, dtype=None):
        t = ctypes.c_uint64()
        _check(lib().drtopk_server_submit(self._h, _dev(keys), _dtype_code(keys, dtype),
                                          keys.numel(), k, _dev(out_keys), _dev(out_idx),
                                          ctypes.byref(t)), "drtopk_server_submit")
        return t.value

    def poll(self, ticket):
        """None while pending, else the latency in microseconds (raises on
        a failed request)."""
        lat = ctypes.c_double()
        rc = lib().drtopk_server_poll_ex(self._h, ticket, ctypes.byref(lat))
        if rc == PENDING:
            return None
        _check(rc, "drtopk_server_poll")
        return lat.value

    def wait(self, ticket):
        lat = ctypes.c_double()
        _check(lib().drtopk_server_wait(self._h, ticket, ctypes.byref(lat)), "drtopk_server_wait")
        return lat.value

    def stats(self):
        st = ServerStats()
        _check(lib().drtopk_server_get_stats(self._h, ctypes.byref(st)), "drtopk_server_get_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            lib().drtopk_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
