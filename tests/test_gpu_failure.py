"""Bounded device waits that run out, on a GPU, without faulting it.

Every decoupled look-back (radix passes, run-boundary scan, device scans)
waits for status words of earlier tiles with a time limit (a library
parameter, hc_set_wait_limit_ns).  These tests make such a wait run out on
purpose: a testing flag of hc_build_index keeps the first tile of a step from
ever publishing its status word (a flag that nothing sets), so the tiles
after it wait until the limit, record DEV_ERR_TIMEOUT and return.  The host
must then report HC_ERR_TIMEOUT, return no index, and leave the context
usable: the next build and join on the same device are correct.
"""
import time

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    return hc


def dev(arr):
    import torch

    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint32).view(np.int32)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module")
def rel():
    """A multi-tile relation: 200,000 rows span 33 radix tiles and 49 scan tiles."""
    rng = np.random.default_rng(17)
    return datagen.scatter_order(datagen.directed_set(rng.integers(0, 1 << 20, size=(220_000, 2)).astype(np.uint32))
                                 [:200_000], 4)


def _check_index(hc, ix, pairs, ao):
    v1, o1, v2 = oracle.coco_build(pairs, ao)
    assert ix.l1 == v1.shape[0]
    assert np.array_equal(u32(ix.v1()), v1)
    assert np.array_equal(u32(ix.o1()).astype(np.uint64), o1)
    assert np.array_equal(u32(ix.v2()), v2)


@pytest.mark.parametrize("step", ["sort", "scan"])
@pytest.mark.parametrize("limit_ns", [20_000_000, 0])
def test_wait_runs_out_and_context_survives(hc, rel, step, limit_ns):
    import torch

    prev = hc.set_wait_limit_ns(limit_ns)
    try:
        t0 = time.perf_counter()
        with pytest.raises(hc.HoneycombError) as e:
            hc.build_index(dev(rel), 0, test_stall=step)
        elapsed = time.perf_counter() - t0
    finally:
        hc.set_wait_limit_ns(prev)
    assert e.value.status == 4  # HC_ERR_TIMEOUT
    assert elapsed < 20.0
    torch.cuda.synchronize()  # no fault is pending on the device
    # the same device goes on working: a normal build and a join are exact
    for ao in (0, 1):
        _check_index(hc, hc.build_index(dev(rel), ao), rel, ao)
    ep = datagen.orient_lt(datagen.rmat_graph(10, 8, 3))
    ix = hc.build_index(dev(ep), 0)
    cnt, _, _ = oracle.gj_count(3, list(hc.TRIANGLE.atoms), [ep] * 3)
    assert hc.run_join(hc.TRIANGLE, [ix] * 3, shares=[2, 2, 1]).count == cnt


def test_single_tile_has_nothing_to_wait_for(hc):
    """A relation of one tile has no look-back: the stall flags change nothing."""
    rng = np.random.default_rng(2)
    pairs = datagen.directed_set(rng.integers(0, 5000, size=(3000, 2)).astype(np.uint32))
    prev = hc.set_wait_limit_ns(0)
    try:
        for step in ("sort", "scan"):
            _check_index(hc, hc.build_index(dev(pairs), 0, test_stall=step), pairs, 0)
    finally:
        hc.set_wait_limit_ns(prev)


def test_default_limit_builds_are_unaffected(hc, rel):
    assert hc.set_wait_limit_ns(2_000_000_000) == 2_000_000_000
    _check_index(hc, hc.build_index(dev(rel), 1), rel, 1)
