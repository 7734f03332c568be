"""Seeded synthetic inputs for the record-retrieval path.

This module is shared by the tests, bench.py and the scripts that write
golden values.  It holds none of the retrieval method's arithmetic: it makes
source tables, rid sequences and foreign-key columns from SplitMix64 streams
(see synth.c for the exact stream definitions) and nothing else.

Workload recipes (sizes and distributions follow the paper's workloads:
the Datamation-style file of 100-byte records with 10-byte keys, §3 and §5.1;
the foreign-key join relations of §4.2 and §5.3):

* ``plain_retrieval``: N records of ``rec`` bytes filled from stream seed 1,
  rids = Fisher-Yates permutation of [0, N) from seed 2.
* ``sort_file``: N records of ``rec`` bytes from seed 3; the key is bytes 0..9.
* ``fk_tables``: dimension rows (int64 primary key = row index, the rest
  random bytes from sub-stream A of seed 4) and fact rows (int32 foreign key at
  offset 0, the rest random bytes from sub-stream D); foreign keys are Zipf(s)
  ranks (sub-stream B) pushed through a Fisher-Yates shuffle of the ids
  (sub-stream C).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so beside it (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-lm", "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:3] + ["-fopenmp"] + base[3:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, p = ctypes.c_uint64, ctypes.c_void_p
            lib.synth_splitmix64_at.argtypes = [u64, u64]
            lib.synth_splitmix64_at.restype = u64
            lib.synth_stream_seed.argtypes = [u64, u64]
            lib.synth_stream_seed.restype = u64
            lib.synth_fill_bytes.argtypes = [p, u64, u64]
            lib.synth_permutation_i32.argtypes = [p, u64, u64]
            lib.synth_uniform_i32.argtypes = [p, u64, u64, u64]
            lib.synth_uniform_f64.argtypes = [p, u64, u64]
            lib.synth_zipf_i32.argtypes = [p, u64, u64, ctypes.c_double, u64]
            lib.synth_zipf_i32.restype = ctypes.c_int
            lib.synth_take_i32.argtypes = [p, p, p, u64]
            lib.synth_batch_rids.argtypes = [p, p, p, p, p, u64, u64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def splitmix64_at(seed: int, k: int) -> int:
    return int(_load().synth_splitmix64_at(seed, k))


def stream_seed(seed: int, stream: int) -> int:
    return int(_load().synth_stream_seed(seed, stream))


def random_bytes(nbytes: int, seed: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty(nbytes, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size == nbytes
    _load().synth_fill_bytes(_ptr(out), nbytes, seed)
    return out


def records(n: int, rec: int, seed: int) -> np.ndarray:
    """n records of rec bytes, record-major, as a (n, rec) uint8 array."""
    return random_bytes(n * rec, seed).reshape(n, rec)


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    _load().synth_permutation_i32(_ptr(out), n, seed)
    return out


def uniform_ids(n: int, m: int, seed: int) -> np.ndarray:
    """n ids drawn uniformly with replacement from [0, m)."""
    out = np.empty(n, dtype=np.int32)
    _load().synth_uniform_i32(_ptr(out), n, m, seed)
    return out


def uniform_f64(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform_f64(_ptr(out), n, seed)
    return out


def zipf_ranks(n: int, k: int, s: float, seed: int) -> np.ndarray:
    """n 0-based ranks from Zipf(s) over k ranks (inverse CDF)."""
    out = np.empty(n, dtype=np.int32)
    rc = _load().synth_zipf_i32(_ptr(out), n, k, float(s), seed)
    if rc:
        raise RuntimeError(f"synth_zipf_i32 failed ({rc})")
    return out


def take(idx: np.ndarray, table: np.ndarray) -> np.ndarray:
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    table = np.ascontiguousarray(table, dtype=np.int32)
    out = np.empty(idx.size, dtype=np.int32)
    _load().synth_take_i32(_ptr(out), _ptr(idx), _ptr(table), idx.size)
    return out


def batch_rids(n: np.ndarray, n_src: np.ndarray, kind: np.ndarray, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Rid lists of a batch (see synth_batch_rids): returns (all rids, offsets)."""
    n = np.ascontiguousarray(n, dtype=np.uint64)
    n_src = np.ascontiguousarray(n_src, dtype=np.uint64)
    kind = np.ascontiguousarray(kind, dtype=np.uint8)
    offset = np.zeros(n.size, dtype=np.uint64)
    if n.size:
        offset[1:] = np.cumsum(n)[:-1]
    out = np.empty(int(n.sum()), dtype=np.int32)
    _load().synth_batch_rids(_ptr(out), _ptr(offset), _ptr(n), _ptr(n_src), _ptr(kind), n.size, seed)
    return out, offset


# ---------------------------------------------------------------- workloads

def plain_retrieval(n: int = 1_000_000, rec: int = 100, src_seed: int = 1, rid_seed: int = 2):
    """Source file of n records and a permutation rid sequence."""
    return records(n, rec, src_seed), permutation(n, rid_seed)


def sort_file(n: int = 10_000_000, rec: int = 100, seed: int = 3) -> np.ndarray:
    """n records of rec bytes; the sort key is bytes [0, 10) of each record."""
    return records(n, rec, seed)


BATCH_RECS = (8, 16, 32, 64, 100, 128, 256)


def batch_requests(count: int = 4096, n_min: float = 1e3, n_max: float = 1.6e7, seed: int = 5,
                   perm_share: float = 0.7):
    """Request shapes of the batched-retrieval workload: record counts
    log-uniform in [n_min, n_max], record sizes uniform over BATCH_RECS, rids
    a permutation of [0, n) (perm_share of the requests) or uniform draws from
    [0, n).  Returns (n, rec, kind) arrays; draws come from sub-streams
    1000+ of `seed` so they do not overlap the rid streams."""
    u = uniform_f64(count, stream_seed(seed, 1000))
    n = np.floor(np.exp(np.log(n_min) + u * (np.log(n_max) - np.log(n_min)))).astype(np.uint64)
    r = uniform_ids(count, len(BATCH_RECS), stream_seed(seed, 1001))
    rec = np.array(BATCH_RECS, dtype=np.uint64)[r]
    kind = (uniform_f64(count, stream_seed(seed, 1002)) < perm_share).astype(np.uint8)
    return n, rec, kind


def fk_tables(n_dim: int, n_fact: int, dim_bytes: int = 64, fact_bytes: int = 16,
              zipf_s: float = 0.8, seed: int = 4):
    """Dimension and fact tables for the foreign-key joins.

    dim row d: int64 little-endian primary key d at offset 0, then random bytes.
    fact row i: int32 little-endian foreign key at offset 0, then random bytes.
    Foreign keys: pi[z_i] with z_i ~ Zipf(s) over n_dim ranks, pi a shuffle.
    """
    assert dim_bytes >= 8 and fact_bytes >= 4
    dim = records(n_dim, dim_bytes, stream_seed(seed, 0))
    dim[:, :8] = np.arange(n_dim, dtype="<i8").view(np.uint8).reshape(n_dim, 8)
    ranks = zipf_ranks(n_fact, n_dim, zipf_s, stream_seed(seed, 1))
    pi = permutation(n_dim, stream_seed(seed, 2))
    fk = take(ranks, pi)
    fact = records(n_fact, fact_bytes, stream_seed(seed, 3))
    fact[:, :4] = fk.astype("<i4").view(np.uint8).reshape(n_fact, 4)
    return dim, fact, fk
