"""Joins whose tuples are delivered to host memory (hc_run_join_to_host).

The search runs as several launches over consecutive ranges of its work
items; each launch's part of the output pool is compacted on the device and
copied to the host while the next launch runs.  The host rows must be the
oracle's tuples exactly (as a set: the row order is not fixed), for every
query shape, shares, pinned and pageable buffers, and the capacity error must
report the exact count.
"""
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


def sorted_rows(a):
    return a[np.lexsort(a.T[::-1])] if a.shape[0] else a


def _indexes(hc, q, rels):
    cache, ixs = {}, []
    for j, r in enumerate(rels):
        key = (id(r), q.attr_order(j))
        if key not in cache:
            cache[key] = hc.build_index(dev(r), q.attr_order(j))
        ixs.append(cache[key])
    return ixs


@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_CLIQUE", "TWO_TRIANGLE"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_rows_equal_oracle(hc, qname, pinned):
    import torch

    q = getattr(hc, qname)
    sym = datagen.rmat_graph(11, 8, 31)
    rel = sym if qname == "FOUR_CYCLE" else datagen.orient_lt(sym)
    rels = [rel] * len(q.atoms)
    ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
    ixs = _indexes(hc, q, rels)
    for sh in ([1] * q.n_vars, [4] + [1] * (q.n_vars - 1), [2] * q.n_vars):
        for slack in (0, 1000):
            out = torch.empty((ref.shape[0] + slack, q.n_vars), dtype=torch.int32, pin_memory=pinned)
            n = hc.run_join_to_host(q, ixs, out, shares=sh, item_grain=7)
            assert n == ref.shape[0], sh
            got = out[:n].numpy().view(np.uint32)
            assert np.array_equal(sorted_rows(got), sorted_rows(ref)), (sh, slack)


def test_capacity_error_reports_the_count(hc):
    import torch

    ep = datagen.orient_lt(datagen.rmat_graph(10, 8, 4))
    q = hc.TRIANGLE
    cnt, _, _ = oracle.gj_count(3, list(q.atoms), [ep] * 3)
    assert cnt > 10
    ixs = _indexes(hc, q, [ep] * 3)
    for cap in (0, 1, cnt - 1):
        out = torch.empty((cap, 3), dtype=torch.int32, pin_memory=True)
        with pytest.raises(hc.HoneycombError) as e:
            hc.run_join_to_host(q, ixs, out)
        assert e.value.status == 5
    # a buffer of exactly |Q| rows
    out = torch.empty((cnt, 3), dtype=torch.int32, pin_memory=True)
    assert hc.run_join_to_host(q, ixs, out) == cnt
    ref = oracle.gj_enumerate(3, list(q.atoms), [ep] * 3)
    assert np.array_equal(sorted_rows(out.numpy().view(np.uint32)), sorted_rows(ref))


def test_empty_result_and_empty_relation(hc):
    import torch

    one = np.array([[0, 1]], dtype=np.uint32)
    empty = np.zeros((0, 2), dtype=np.uint32)
    q = hc.TRIANGLE
    out = torch.empty((4, 3), dtype=torch.int32, pin_memory=True)
    assert hc.run_join_to_host(q, _indexes(hc, q, [one, one, one]), out) == 0
    assert hc.run_join_to_host(q, _indexes(hc, q, [empty, one, one]), out) == 0
    out0 = torch.empty((0, 3), dtype=torch.int32)
    assert hc.run_join_to_host(q, _indexes(hc, q, [empty, empty, empty]), out0) == 0


def test_many_segments_large_triangle(hc):
    """Enough work items for every launch segment to hold output, with the
    copies overlapping later launches: the host rows are the device result's
    rows (R-MAT 16 triangle, about 10^6 tuples)."""
    import torch

    ep = datagen.orient_lt(datagen.rmat_graph(16, 16, 9))
    q = hc.TRIANGLE
    ixs = _indexes(hc, q, [ep] * 3)
    r = hc.run_join(q, ixs, mode="materialize", shares=[4, 1, 1])
    out = torch.empty((r.count + 5, 3), dtype=torch.int32, pin_memory=True)
    n = hc.run_join_to_host(q, ixs, out, shares=[4, 1, 1], item_grain=16)
    assert n == r.count
    dev_rows = sorted_rows(r.tuples.cpu().numpy().view(np.uint32))
    assert np.array_equal(sorted_rows(out[:n].numpy().view(np.uint32)), dev_rows)
    cnt, _, _ = oracle.gj_count(3, list(q.atoms), [ep] * 3)
    assert n == cnt
