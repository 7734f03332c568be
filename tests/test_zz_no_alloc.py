"""dpg_retrieve_noalloc: the allocation-free entry point, for callers that
cannot allocate device memory when they call (a caching allocator holds all
free memory, a memory-capped region, a plug-in that must not allocate).

It is called here through the C ABI with ctypes and must give, on two calls in
a row, byte-for-byte the output of dpg_retrieve on the same inputs.  The file
name makes pytest collect it last; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_cs_0308004_gb300 import dpg
    f = dpg.lib.dpg_retrieve_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return dpg, f


def test_noalloc_matches_dpg_retrieve_twice():
    dpg, f = _lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    cases = [(700_001, 100, synth.permutation(700_001, 2)),
             (300_000, 16, synth.uniform_ids(1_000_003, 300_000, 5))]
    with dpg.Context(0) as ctx:
        for n_src, rec, rids in cases:
            src = torch.from_numpy(synth.records(n_src, rec, 1)).to(dev)
            d_rids = torch.from_numpy(rids).to(dev)
            want = ctx.retrieve(src, d_rids)
            ctx.sync()
            for _ in range(2):       # two calls in a row share the static scratch
                out = torch.full((rids.size, rec), 0xA5, dtype=torch.uint8, device=dev)
                st = f(src.data_ptr(), n_src, rec, rids.size, d_rids.data_ptr(), out.data_ptr(),
                       stream.cuda_stream)
                assert st == 0, dpg.lib.dpg_strerror(st)
                assert torch.equal(out, want)


def test_noalloc_limits_and_bad_rid():
    dpg, f = _lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    src = torch.from_numpy(synth.records(1000, 8, 1)).to(dev)
    too_many = torch.zeros((1 << 21) + 1, dtype=torch.int32, device=dev)
    out = torch.empty((too_many.numel(), 8), dtype=torch.uint8, device=dev)
    assert f(src.data_ptr(), 1000, 8, too_many.numel(), too_many.data_ptr(), out.data_ptr(), stream) == dpg.EINVAL
    rids = np.arange(500, dtype=np.int32)
    rids[77] = 1000
    d_rids = torch.from_numpy(rids).to(dev)
    out = torch.full((500, 8), 7, dtype=torch.uint8, device=dev)
    assert f(src.data_ptr(), 1000, 8, 500, d_rids.data_ptr(), out.data_ptr(), stream) == dpg.ERANGE
    assert bool((out == 7).all())
