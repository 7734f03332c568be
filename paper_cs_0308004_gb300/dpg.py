"""Python binding of the C ABI in include/dpg.h (argument marshalling only).

Every computation runs in the CUDA kernels of libdpg.so; PyTorch supplies
device memory and the current stream.  If the library has not been built the
import fails: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdpg.so")

# status codes (dpg_status)
OK, EINVAL, ERANGE, ENOMEM, ECUDA, ETIMEOUT, EBUSY = range(7)

# key-pointer pair layout used by the sort path: key bytes, zero padding,
# int32 rid at byte 12; 16 bytes per pair
PAIR_BYTES = 16
PAIR_RID_OFF = 12

# every symbol include/dpg.h declares, with its ctypes signature
_P, _S, _U64, _I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "dpg_ctx_create": ([ctypes.POINTER(ctypes.c_void_p), _I], _I),
    "dpg_ctx_destroy": ([_P], None),
    "dpg_strerror": ([_I], ctypes.c_char_p),
    "dpg_last_error": ([_P], ctypes.c_char_p),
    "dpg_retrieve": ([_P, _P, _S, _S, _S, _P, _P, _P], _I),
    "dpg_retrieve_direct": ([_P, _P, _S, _S, _S, _P, _P, _P], _I),
    "dpg_sort_copy": ([_P, _P, _S, _S, _S, _P, _S, _S, _P, _P], _I),
    "dpg_sort_copy_direct": ([_P, _P, _S, _S, _S, _P, _S, _S, _P, _P], _I),
    "dpg_sync": ([_P, _P], _I),
    "dpg_kernel_launches": ([_P], _U64),
    "dpg_retrieve_host": ([_P, _P, _S, _S, _S, _P, _P, _P], _I),
    "dpg_sort_copy_host": ([_P, _P, _S, _S, _S, _P, _S, _S, _P, _P], _I),
    "dpg_trace_enable": ([_P, _I], None),
    "dpg_trace_reset": ([_P], None),
    "dpg_trace_count": ([_P], _S),
    "dpg_trace_get": ([_P, _S, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_uint64)], _I),
    "dpg_retrieve_noalloc": ([_P, _S, _S, _S, _P, _P, _P], _I),
    "dpg_sort_keyptr": ([_P, _P, _S, _S, _S, _P, _P], _I),
    "dpg_sort_records": ([_P, _P, _S, _S, _S, _P, _P], _I),
    "dpg_fk_join": ([_P, _P, _S, _S, _S, _P, _S, _S, _S, _P, _I, _P], _I),
    "dpg_retrieve_batch": ([_P, _P, _S, _P], _I),
    "dpg_server_create": ([ctypes.POINTER(ctypes.c_void_p), _I, _I, _S], _I),
    "dpg_server_submit": ([_P, _P, ctypes.POINTER(ctypes.c_uint64)], _I),
    "dpg_server_result": ([_P, ctypes.c_uint64, _I, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t),
                           ctypes.POINTER(ctypes.c_double)], _I),
    "dpg_server_release": ([_P, ctypes.c_uint64], _I),
    "dpg_server_held_bytes": ([_P], _S),
    "dpg_server_destroy": ([_P], None),
    "dpg_tune": ([_P, _P, _S, _S, _S, _P, _S, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "dpg_last_plan": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I)], None),
    "dpg_run_batch": ([_P, _P, _S, _P], _I),
    "dpg_set_wait_limit": ([_P, ctypes.c_double], _I),
    "dpg_check_wait": ([_P, _P], _I),
    "dpg_inject_alloc_failure": ([_P, _I], _I),
}

JOIN_MODES = {"move": 0, "sort": 1, "direct": 2}


class Job(ctypes.Structure):
    """struct dpg_job (include/dpg.h)."""
    _fields_ = [("kind", ctypes.c_int), ("join_mode", ctypes.c_int),
                ("src", ctypes.c_void_p), ("n_src", ctypes.c_size_t), ("rec_bytes", ctypes.c_size_t),
                ("n", ctypes.c_size_t), ("rids", ctypes.c_void_p),
                ("fact", ctypes.c_void_p), ("n_fact", ctypes.c_size_t), ("fact_bytes", ctypes.c_size_t),
                ("fk_off", ctypes.c_size_t), ("dim", ctypes.c_void_p), ("n_dim", ctypes.c_size_t),
                ("dim_bytes", ctypes.c_size_t), ("pk_off", ctypes.c_size_t)]


class BatchItem(ctypes.Structure):
    """struct dpg_batch_item (include/dpg.h)."""
    _fields_ = [("job", Job), ("out", ctypes.c_void_p)]


class Request(ctypes.Structure):
    """struct dpg_request (include/dpg.h)."""
    _fields_ = [("src", ctypes.c_void_p), ("n_src", ctypes.c_size_t), ("rec_bytes", ctypes.c_size_t),
                ("n", ctypes.c_size_t), ("rids", ctypes.c_void_p), ("dst", ctypes.c_void_p)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`"
                          " (the CUDA library has no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


class DpgError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {lib.dpg_strerror(status).decode()}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class DpgRangeError(DpgError, IndexError):
    pass


def _stream_handle(stream, device) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _need_cuda(t: torch.Tensor, name: str, device: torch.device):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library works on device memory only)")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, the context on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _table(t: torch.Tensor, name: str) -> tuple[int, int]:
    if t.dtype != torch.uint8 or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D uint8 tensor (records x bytes)")
    return t.shape[0], t.shape[1]


class Context:
    """Owns a dpg_ctx (scratch memory and the asynchronous error word)."""

    def __init__(self, device: int | torch.device | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device if isinstance(device, int) else device.index)
        h = ctypes.c_void_p()
        self._check(lib.dpg_ctx_create(ctypes.byref(h), self.device.index), "dpg_ctx_create", h=None)
        self._h = h

    # -- plumbing
    def _check(self, status: int, what: str, h=0):
        if status != OK:
            handle = self._h if h == 0 else h
            detail = lib.dpg_last_error(handle).decode() if handle else ""
            cls = DpgRangeError if status == ERANGE else DpgError
            raise cls(status, what, detail)

    def close(self):
        if getattr(self, "_h", None):
            lib.dpg_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def kernel_launches(self) -> int:
        return int(lib.dpg_kernel_launches(self._h))

    # -- failure detection
    def set_wait_limit(self, seconds: float):
        """Limit of every device wait on another CTA's flag (seconds of SM clock)."""
        self._check(lib.dpg_set_wait_limit(self._h, float(seconds)), "dpg_set_wait_limit")

    def check_wait(self, stream=None):
        """Enqueue one bounded wait on a flag nothing sets (the next sync reports the timeout)."""
        self._check(lib.dpg_check_wait(self._h, _stream_handle(stream, self.device)), "dpg_check_wait")

    def inject_alloc_failure(self, count: int = 1):
        """Make the next `count` device allocations of this context fail (DPG_ENOMEM)."""
        self._check(lib.dpg_inject_alloc_failure(self._h, int(count)), "dpg_inject_alloc_failure")

    # -- operations
    def _retrieve(self, fn, src, rids, out, stream):
        _need_cuda(src, "src", self.device)
        _need_cuda(rids, "rids", self.device)
        if rids.dtype != torch.int32 or rids.dim() != 1:
            raise ValueError("rids must be a 1-D int32 tensor")
        n_src, rec = _table(src, "src")
        n = rids.shape[0]
        if out is None:
            out = torch.empty((n, rec), dtype=torch.uint8, device=self.device)
        _need_cuda(out, "out", self.device)
        if tuple(out.shape) != (n, rec) or out.dtype != torch.uint8:
            raise ValueError("out must be a uint8 tensor of shape (len(rids), record bytes)")
        st = fn(self._h, src.data_ptr(), n_src, rec, n, rids.data_ptr(), out.data_ptr(),
                _stream_handle(stream, self.device))
        self._check(st, fn.__name__)
        return out

    def retrieve(self, src: torch.Tensor, rids: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """dst[i] = src[rids[i]] by distribute-probe-gather (asynchronous; call sync())."""
        return self._retrieve(lib.dpg_retrieve, src, rids, out, stream)

    def retrieve_direct(self, src: torch.Tensor, rids: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """The same result by the plain one-pass gather (baseline)."""
        return self._retrieve(lib.dpg_retrieve_direct, src, rids, out, stream)

    def _sort_copy(self, fn, pairs, src, rid_off, out, stream):
        _need_cuda(pairs, "pairs", self.device)
        _need_cuda(src, "src", self.device)
        n, stride = _table(pairs, "pairs")
        n_src, rec = _table(src, "src")
        if out is None:
            out = torch.empty((n, rec), dtype=torch.uint8, device=self.device)
        _need_cuda(out, "out", self.device)
        if tuple(out.shape) != (n, rec) or out.dtype != torch.uint8:
            raise ValueError("out must be a uint8 tensor of shape (pairs, record bytes)")
        st = fn(self._h, pairs.data_ptr(), stride, rid_off, n, src.data_ptr(), n_src, rec, out.data_ptr(),
                _stream_handle(stream, self.device))
        self._check(st, fn.__name__)
        return out

    def sort_copy(self, pairs, src, rid_off: int = PAIR_RID_OFF, out=None, stream=None):
        """Copy phase of a key-pointer sort (§3): dst[i] = src[rid of pairs[i]]."""
        return self._sort_copy(lib.dpg_sort_copy, pairs, src, rid_off, out, stream)

    def sort_copy_direct(self, pairs, src, rid_off: int = PAIR_RID_OFF, out=None, stream=None):
        return self._sort_copy(lib.dpg_sort_copy_direct, pairs, src, rid_off, out, stream)

    def sort_keyptr(self, src: torch.Tensor, key_bytes: int = 10, out: torch.Tensor | None = None, stream=None):
        """§3 phases 1-2: sorted (n_src, 16) uint8 key-pointer pairs of src."""
        _need_cuda(src, "src", self.device)
        n_src, rec = _table(src, "src")
        if out is None:
            out = torch.empty((n_src, PAIR_BYTES), dtype=torch.uint8, device=self.device)
        _need_cuda(out, "out", self.device)
        if tuple(out.shape) != (n_src, PAIR_BYTES) or out.dtype != torch.uint8:
            raise ValueError("out must be a uint8 tensor of shape (records, 16)")
        st = lib.dpg_sort_keyptr(self._h, src.data_ptr(), n_src, rec, key_bytes, out.data_ptr(),
                                 _stream_handle(stream, self.device))
        self._check(st, "dpg_sort_keyptr")
        return out

    def sort_records(self, src: torch.Tensor, key_bytes: int = 10, out: torch.Tensor | None = None, stream=None):
        """The whole §3 sort: records in (key, rid) order."""
        _need_cuda(src, "src", self.device)
        n_src, rec = _table(src, "src")
        if out is None:
            out = torch.empty((n_src, rec), dtype=torch.uint8, device=self.device)
        _need_cuda(out, "out", self.device)
        if tuple(out.shape) != (n_src, rec) or out.dtype != torch.uint8:
            raise ValueError("out must be a uint8 tensor shaped like src")
        st = lib.dpg_sort_records(self._h, src.data_ptr(), n_src, rec, key_bytes, out.data_ptr(),
                                  _stream_handle(stream, self.device))
        self._check(st, "dpg_sort_records")
        return out

    def fk_join(self, fact: torch.Tensor, dim: torch.Tensor, mode: str = "move", fk_off: int = 0, pk_off: int = 0,
                out: torch.Tensor | None = None, stream=None):
        """Foreign-key join (§4.2.1): rows fact || dim[fk], by DPG-move, DPG-sort or direct."""
        _need_cuda(fact, "fact", self.device)
        _need_cuda(dim, "dim", self.device)
        n_fact, fb = _table(fact, "fact")
        n_dim, db = _table(dim, "dim")
        if out is None:
            out = torch.empty((n_fact, fb + db), dtype=torch.uint8, device=self.device)
        _need_cuda(out, "out", self.device)
        if tuple(out.shape) != (n_fact, fb + db) or out.dtype != torch.uint8:
            raise ValueError("out must be a uint8 tensor of shape (fact rows, fact bytes + dim bytes)")
        st = lib.dpg_fk_join(self._h, fact.data_ptr(), n_fact, fb, fk_off, dim.data_ptr(), n_dim, db, pk_off,
                             out.data_ptr(), JOIN_MODES[mode], _stream_handle(stream, self.device))
        self._check(st, "dpg_fk_join")
        return out

    def retrieve_batch(self, requests, stream=None):
        """Batched retrieval.  requests: list of (src, rids, out) device tensors,
        or (src, n_src, rids, out) to let a request see only the first n_src
        records of src.  Asynchronous; call sync()."""
        arr = (Request * max(1, len(requests)))()
        for k, req in enumerate(requests):
            if len(req) == 3:
                src, rids, out = req
                n_src = src.shape[0]
            else:
                src, n_src, rids, out = req
            for t, nm in ((src, "src"), (rids, "rids"), (out, "out")):
                _need_cuda(t, nm, self.device)
            _, rec = _table(src, "src")
            if rids.dtype != torch.int32 or tuple(out.shape) != (rids.shape[0], rec) or out.dtype != torch.uint8:
                raise ValueError("each request needs int32 rids and a uint8 out of shape (len(rids), record bytes)")
            arr[k] = Request(src.data_ptr(), n_src, rec, rids.shape[0], rids.data_ptr(), out.data_ptr())
        st = lib.dpg_retrieve_batch(self._h, ctypes.cast(arr, ctypes.c_void_p), len(requests),
                                    _stream_handle(stream, self.device))
        self._check(st, "dpg_retrieve_batch")

    def run_batch(self, items, stream=None):
        """One persistent launch over a batch of retrievals and DPG-move joins.
        items: ("retrieve", src, rids, out[, n_src]) or ("join", fact, dim, out[, fk_off, pk_off]),
        device tensors.  Asynchronous; call sync()."""
        arr = (BatchItem * max(1, len(items)))()
        for k, it in enumerate(items):
            if it[0] == "retrieve":
                src, rids, out = it[1:4]
                n_src = it[4] if len(it) > 4 else src.shape[0]
                for t, nm in ((src, "src"), (rids, "rids"), (out, "out")):
                    _need_cuda(t, nm, self.device)
                _, rec = _table(src, "src")
                if rids.dtype != torch.int32 or tuple(out.shape) != (rids.shape[0], rec) or out.dtype != torch.uint8:
                    raise ValueError("a retrieval needs int32 rids and a uint8 out of shape (len(rids), record bytes)")
                arr[k].job = Job(kind=0, src=src.data_ptr(), n_src=n_src, rec_bytes=rec, n=rids.shape[0],
                                 rids=rids.data_ptr())
            elif it[0] == "join":
                fact, dim, out = it[1:4]
                fk_off = it[4] if len(it) > 4 else 0
                pk_off = it[5] if len(it) > 5 else 0
                for t, nm in ((fact, "fact"), (dim, "dim"), (out, "out")):
                    _need_cuda(t, nm, self.device)
                n_fact, fb = _table(fact, "fact")
                n_dim, db = _table(dim, "dim")
                if tuple(out.shape) != (n_fact, fb + db) or out.dtype != torch.uint8:
                    raise ValueError("a join needs a uint8 out of shape (fact rows, fact bytes + dim bytes)")
                arr[k].job = Job(kind=1, join_mode=JOIN_MODES["move"], fact=fact.data_ptr(), n_fact=n_fact,
                                 fact_bytes=fb, fk_off=fk_off, dim=dim.data_ptr(), n_dim=n_dim, dim_bytes=db,
                                 pk_off=pk_off)
            else:
                raise ValueError(f"unknown batch item kind {it[0]!r}")
            arr[k].out = out.data_ptr()
        st = lib.dpg_run_batch(self._h, ctypes.cast(arr, ctypes.c_void_p), len(items),
                               _stream_handle(stream, self.device))
        self._check(st, "dpg_run_batch")

    def tune(self, src: torch.Tensor, rids: torch.Tensor, out: torch.Tensor | None = None,
             rid_stride: int = 4, rid_off: int = 0, stream=None):
        """Time the candidate plans on this data and cache the fastest; returns (variant, seg_log2).
        rids: an int32 array (rid_stride 4) or uint8 key-pointer pairs (rid_stride 16, rid_off 12)."""
        _need_cuda(src, "src", self.device)
        _need_cuda(rids, "rids", self.device)
        n_src, rec = _table(src, "src")
        n = rids.shape[0]
        if out is None:
            out = torch.empty((n, rec), dtype=torch.uint8, device=self.device)
        v, sl = ctypes.c_int(), ctypes.c_int()
        st = lib.dpg_tune(self._h, src.data_ptr(), n_src, rec, n, rids.data_ptr() + rid_off, rid_stride,
                          out.data_ptr(), _stream_handle(stream, self.device), ctypes.byref(v), ctypes.byref(sl))
        self._check(st, "dpg_tune")
        return v.value, sl.value

    def last_plan(self):
        v, sl = ctypes.c_int(), ctypes.c_int()
        lib.dpg_last_plan(self._h, ctypes.byref(v), ctypes.byref(sl))
        return v.value, sl.value

    # -- host buffers (copies in and out happen inside the library)
    @staticmethod
    def _host(t, name):
        if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor (pinned for full copy speed)")

    def retrieve_host(self, src: torch.Tensor, rids: torch.Tensor, out: torch.Tensor, stream=None):
        """Host-memory retrieval: copy in, DPG on the device, copy out; synchronous."""
        for t, nm in ((src, "src"), (rids, "rids"), (out, "out")):
            self._host(t, nm)
        n_src, rec = _table(src, "src")
        st = lib.dpg_retrieve_host(self._h, src.data_ptr(), n_src, rec, rids.shape[0], rids.data_ptr(),
                                   out.data_ptr(), _stream_handle(stream, self.device))
        self._check(st, "dpg_retrieve_host")
        return out

    def sort_copy_host(self, pairs: torch.Tensor, src: torch.Tensor, out: torch.Tensor,
                       rid_off: int = PAIR_RID_OFF, stream=None):
        for t, nm in ((pairs, "pairs"), (src, "src"), (out, "out")):
            self._host(t, nm)
        n, stride = _table(pairs, "pairs")
        n_src, rec = _table(src, "src")
        st = lib.dpg_sort_copy_host(self._h, pairs.data_ptr(), stride, rid_off, n, src.data_ptr(), n_src, rec,
                                    out.data_ptr(), _stream_handle(stream, self.device))
        self._check(st, "dpg_sort_copy_host")
        return out

    # -- kernel tracing (CUDA events around every launch)
    def trace(self, on: bool = True):
        lib.dpg_trace_enable(self._h, 1 if on else 0)

    def trace_reset(self):
        lib.dpg_trace_reset(self._h)

    def trace_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last trace_reset."""
        out = {}
        for i in range(lib.dpg_trace_count(self._h)):
            name, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_uint64()
            self._check(lib.dpg_trace_get(self._h, i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt)),
                        "dpg_trace_get")
            out[name.value.decode()] = (ms.value, cnt.value)
        return out

    def sync(self, stream=None):
        """Wait for the stream; raise the first asynchronous error (bad rid, timeout)."""
        self._check(lib.dpg_sync(self._h, _stream_handle(stream, self.device)), "dpg_sync")


class _DeviceBytes:
    """A device buffer seen by torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


class Server:
    """Request loop with HBM-budget admission (dpg_server_* in include/dpg.h)."""

    def __init__(self, device: int = 0, slots: int = 4, budget_bytes: int = 8 << 30):
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        st = lib.dpg_server_create(ctypes.byref(h), device, slots, budget_bytes)
        if st != OK:
            raise DpgError(st, "dpg_server_create")
        self._h = h
        self._shapes = {}
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            lib.dpg_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _submit(self, job: Job, shape, keep) -> int:
        t = ctypes.c_uint64()
        st = lib.dpg_server_submit(self._h, ctypes.byref(job), ctypes.byref(t))
        if st != OK:
            raise DpgError(st, "dpg_server_submit")
        self._shapes[t.value] = shape
        self._keep[t.value] = keep          # the tables must outlive the job
        return t.value

    def submit_retrieve(self, src: torch.Tensor, rids: torch.Tensor, n_src: int | None = None) -> int:
        n_src_all, rec = _table(src, "src")
        job = Job(kind=0, src=src.data_ptr(), n_src=n_src_all if n_src is None else n_src, rec_bytes=rec,
                  n=rids.shape[0], rids=rids.data_ptr())
        return self._submit(job, (rids.shape[0], rec), (src, rids))

    def submit_join(self, fact: torch.Tensor, dim: torch.Tensor, mode: str = "move", fk_off: int = 0,
                    pk_off: int = 0) -> int:
        n_fact, fb = _table(fact, "fact")
        n_dim, db = _table(dim, "dim")
        job = Job(kind=1, join_mode=JOIN_MODES[mode], fact=fact.data_ptr(), n_fact=n_fact, fact_bytes=fb,
                  fk_off=fk_off, dim=dim.data_ptr(), n_dim=n_dim, dim_bytes=db, pk_off=pk_off)
        return self._submit(job, (n_fact, fb + db), (fact, dim))

    def result(self, ticket: int, wait: bool = True):
        """(status, result tensor viewing server memory or None, latency ms); None while pending."""
        p, nbytes, lat = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_double()
        st = lib.dpg_server_result(self._h, ticket, 1 if wait else 0, ctypes.byref(p), ctypes.byref(nbytes),
                                   ctypes.byref(lat))
        if st == EBUSY and not wait:
            return None
        shape = self._shapes[ticket]
        out = None
        if p.value and shape[0] * shape[1]:
            out = torch.as_tensor(_DeviceBytes(p.value, shape), device=self.device)
        return st, out, lat.value

    def release(self, ticket: int):
        lib.dpg_server_release(self._h, ticket)
        self._shapes.pop(ticket, None)
        self._keep.pop(ticket, None)

    @property
    def held_bytes(self) -> int:
        return int(lib.dpg_server_held_bytes(self._h))
