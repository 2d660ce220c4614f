"""The allocation-free CoCo level build against hc_build_index (needs a GPU).

hc_coco_levels_noalloc serves callers that cannot let the library allocate
device memory (their device memory is reserved up front by another
allocator, or their request path must never call an allocator).  It writes
only into buffers the caller passes, using a fixed scratch array inside the
library.  These tests call it through the C ABI on keys sorted by
hc_build_index and require the exact V1, O1, V2 and l1 that hc_build_index
produced, on two calls in a row (the second smaller than the first, so stale
scratch from the first call would show).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    return hc


def _relation(n, seed):
    rng = np.random.default_rng(seed)
    hi = 1 << 21
    pairs = datagen.directed_set(rng.integers(0, hi, size=(int(n * 1.05) + 8, 2)).astype(np.uint32))[:n]
    return datagen.scatter_order(pairs, seed)


def _noalloc(hc, keys, n):
    import torch

    lib = hc._lib.load()
    v1 = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    o1 = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    v2 = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    st = lib.hc_coco_levels_noalloc(ctypes.c_void_p(keys.data_ptr() if n else 0), n, ctypes.c_void_p(v1.data_ptr()),
                                    ctypes.c_void_p(o1.data_ptr()), ctypes.c_void_p(v2.data_ptr()),
                                    ctypes.c_void_p(info.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    hc._lib.check(st, "hc_coco_levels_noalloc")
    torch.cuda.synchronize()
    return v1, o1, v2, info.cpu().numpy()


def _compare(hc, n, seed):
    import torch

    pairs = _relation(n, seed)
    d = torch.from_numpy(pairs.view(np.int32)).cuda()
    ix = hc.build_index(d, 0)  # the existing entry point
    keys = ix.keys().clone()
    v1, o1, v2, info = _noalloc(hc, keys, ix.n)
    l1 = int(info[0])
    assert int(info[1]) == 0
    assert l1 == ix.l1
    assert torch.equal(v1[:l1], ix.v1())
    assert torch.equal(o1[:l1 + 1], ix.o1())
    assert torch.equal(v2[:ix.n], ix.v2())


def test_two_calls_in_a_row_match_build_index(hc):
    _compare(hc, 3_000_001, 1)   # 733 tiles, ragged last tile
    _compare(hc, 70_001, 2)      # fewer tiles than the call before


def test_limit_and_small_cases(hc):
    import torch

    lib = hc._lib.load()
    z = ctypes.c_void_p(0)
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.hc_coco_levels_noalloc(p, (1 << 24) + 1, p, p, p, p, z)
    assert st == 5  # HC_ERR_CAPACITY, rejected before any device work
    assert b"exceeds" in lib.hc_last_error()
    _compare(hc, 1, 3)
    _compare(hc, 4096, 4)
    v1, o1, v2, info = _noalloc(hc, torch.zeros(1, dtype=torch.int64, device="cuda"), 0)
    assert info.tolist() == [0, 0] and o1.cpu().tolist() == [0]
