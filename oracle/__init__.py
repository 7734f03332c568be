"""ORACLE — test infrastructure only.

Python wrappers over oracle.c: a plain CPU statement of what the record
retrieval path computes (Cooperman, Ma, Nguyen, cs/0308004).  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA library and never imports it.

Every function returns numpy arrays and raises ``OracleRangeError`` when a rid
or foreign key lies outside its table (status 2 in oracle.c), in which case
nothing was written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PAIR_BYTES = 16   # key-pointer pair: key bytes, zero padding, int32 rid at byte 12
PAIR_RID_OFF = 12


class OracleRangeError(ValueError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (plain -O2; every function
    single-threaded but oracle_retrieve_threads, the multi-core CPU figure)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    subprocess.run(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp"],
                   check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


# argument kinds: pointers and sizes, in order (u = uint64 size, p = pointer)
_KINDS = {
    "oracle_retrieve": "puuupp",
    "oracle_retrieve_threads": "puuuppu",
    "oracle_dpg_phases": "puuupupppp",
    "oracle_sort_keyptr": "puuup",
    "oracle_sort_copy": "puuupuup",
    "oracle_fk_join_nested": "puuupuuupup",
    "oracle_fk_join_move": "puuupuuup",
    "oracle_fk_join_sorted": "puuupuuup",
    "oracle_fk_join_order": "puuuup",
}


def configure(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Attach the C signatures to a loaded oracle library."""
    for name, kinds in _KINDS.items():
        f = getattr(lib, name)
        f.argtypes = [ctypes.c_void_p if k == "p" else ctypes.c_uint64 for k in kinds]
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(ctypes.CDLL(build()))
    return _lib


def use_library(lib):
    """Swap the loaded library (the mutation tests plant mistakes this way);
    returns the previous one."""
    global _lib
    with _lock:
        prev, _lib = _lib, lib
    return prev


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check(rc: int, what: str):
    if rc == 2:
        raise OracleRangeError(f"{what}: rid or key out of range")
    if rc:
        raise ValueError(f"{what}: status {rc}")


def _records(src: np.ndarray) -> tuple[np.ndarray, int, int]:
    src = np.ascontiguousarray(src)
    assert src.dtype == np.uint8 and src.ndim == 2
    return src, src.shape[0], src.shape[1]


def retrieve(src: np.ndarray, rids: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
    """dst[i] = src[rids[i]] (§2); src is (N, rec) uint8, rids int32."""
    src, n_src, rec = _records(src)
    rids = np.ascontiguousarray(rids, dtype=np.int32)
    n = rids.size
    dst = np.empty((n, rec), dtype=np.uint8) if out is None else out
    _check(_load().oracle_retrieve(_p(src), n_src, rec, n, _p(rids), _p(dst)), "retrieve")
    return dst


def dpg_phases(src: np.ndarray, rids: np.ndarray, run_len: int):
    """Figure 1's three phases with 0-based runs of run_len records.

    Returns (rid_runs: list of int32 arrays, internal_runs: list of (k, rec)
    arrays, dst).  Small inputs only (memory grows as runs x n).
    """
    src, n_src, rec = _records(src)
    rids = np.ascontiguousarray(rids, dtype=np.int32)
    n = rids.size
    num_runs = (n_src + run_len - 1) // run_len
    rid_runs = np.empty(max(n, 1), dtype=np.int32)
    sizes = np.zeros(max(num_runs, 1), dtype=np.uint64)
    internal = np.empty((max(n, 1), rec), dtype=np.uint8)
    dst = np.empty((n, rec), dtype=np.uint8)
    _check(_load().oracle_dpg_phases(_p(src), n_src, rec, n, _p(rids), run_len, _p(rid_runs),
                                     _p(sizes), _p(internal), _p(dst)), "dpg_phases")
    runs, inter, pos = [], [], 0
    for j in range(num_runs):
        k = int(sizes[j])
        runs.append(rid_runs[pos:pos + k].copy())
        inter.append(internal[pos:pos + k].copy())
        pos += k
    return runs, inter, dst


def sort_keyptr(src: np.ndarray, key_bytes: int = 10) -> np.ndarray:
    """§3 phases 1-2: key-pointer pairs of every record, sorted (ties by rid).

    Returns an (N, 16) uint8 array of pairs (key, zero pad, int32 rid at 12).
    """
    src, n_src, rec = _records(src)
    pairs = np.empty((n_src, PAIR_BYTES), dtype=np.uint8)
    _check(_load().oracle_sort_keyptr(_p(src), n_src, rec, key_bytes, _p(pairs)), "sort_keyptr")
    return pairs


def pair_rids(pairs: np.ndarray, rid_off: int = PAIR_RID_OFF) -> np.ndarray:
    return np.ascontiguousarray(pairs[:, rid_off:rid_off + 4]).view("<i4").reshape(-1)


def retrieve_threads(src: np.ndarray, rids: np.ndarray, threads: int, out: np.ndarray | None = None) -> np.ndarray:
    """retrieve() on `threads` host threads (contiguous ranges of destination
    slots, every rid checked first): the benchmark's multi-core CPU figure."""
    src, n_src, rec = _records(src)
    rids = np.ascontiguousarray(rids, dtype=np.int32)
    n = rids.size
    dst = np.empty((n, rec), dtype=np.uint8) if out is None else out
    _check(_load().oracle_retrieve_threads(_p(src), n_src, rec, n, _p(rids), _p(dst), threads), "retrieve_threads")
    return dst


def sort_copy(pairs: np.ndarray, src: np.ndarray, rid_off: int = PAIR_RID_OFF) -> np.ndarray:
    """§3 phase 3: copy records into the order of the sorted pairs."""
    src, n_src, rec = _records(src)
    pairs = np.ascontiguousarray(pairs)
    n, stride = pairs.shape
    dst = np.empty((n, rec), dtype=np.uint8)
    _check(_load().oracle_sort_copy(_p(pairs), stride, rid_off, n, _p(src), n_src, rec, _p(dst)),
           "sort_copy")
    return dst


def sort_records(src: np.ndarray, key_bytes: int = 10) -> np.ndarray:
    """The whole §3 sort: records ordered by key, equal keys by record index."""
    return sort_copy(sort_keyptr(src, key_bytes), src)


def fk_join_nested(fact: np.ndarray, dim: np.ndarray, fk_off: int = 0, pk_off: int = 0) -> np.ndarray:
    """Textbook nested-loop equi-join (fact order, then dimension order)."""
    fact, nf, fb = _records(fact)
    dim, nd, db = _records(dim)
    cap = nf  # a foreign key join emits at most one row per fact row
    out = np.empty((max(cap, 1), fb + db), dtype=np.uint8)
    rows = ctypes.c_uint64(0)
    _check(_load().oracle_fk_join_nested(_p(fact), nf, fb, fk_off, _p(dim), nd, db, pk_off,
                                         _p(out), cap, ctypes.addressof(rows)), "fk_join_nested")
    if rows.value > cap:
        raise ValueError("more join rows than fact rows: dimension keys are not unique")
    return out[:rows.value]


def fk_join_move(fact: np.ndarray, dim: np.ndarray, fk_off: int = 0, pk_off: int = 0) -> np.ndarray:
    """DPG-move join result (§4.2.1): out[i] = fact[i] || dim[fk_i]."""
    fact, nf, fb = _records(fact)
    dim, nd, db = _records(dim)
    out = np.empty((nf, fb + db), dtype=np.uint8)
    _check(_load().oracle_fk_join_move(_p(fact), nf, fb, fk_off, _p(dim), nd, db, pk_off, _p(out)),
           "fk_join_move")
    return out


def fk_join_sorted(fact: np.ndarray, dim: np.ndarray, fk_off: int = 0, pk_off: int = 0) -> np.ndarray:
    """DPG-sort join result (§4.2.1): rows in (fk, fact row) order."""
    fact, nf, fb = _records(fact)
    dim, nd, db = _records(dim)
    out = np.empty((nf, fb + db), dtype=np.uint8)
    _check(_load().oracle_fk_join_sorted(_p(fact), nf, fb, fk_off, _p(dim), nd, db, pk_off, _p(out)),
           "fk_join_sorted")
    return out


def fk_join_order(fact: np.ndarray, n_dim: int, fk_off: int = 0) -> np.ndarray:
    """Fact row indices in DPG-sort join order (fk, then row; §4.2.1), int64."""
    fact, nf, fb = _records(fact)
    order = np.empty(nf, dtype=np.uint64)
    _check(_load().oracle_fk_join_order(_p(fact), nf, fb, fk_off, n_dim, _p(order)), "fk_join_order")
    return order.view(np.int64)
