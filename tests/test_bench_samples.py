"""The bounded samples of the k-ary benchmark workloads are exact (host only).

bench.py counts LW and CT on a sample -- the query restricted to x < fx and
y < fy, with R4 of LW reduced to the rows whose (y, z) occurs in the sampled
R1 -- on the GPU and with the oracle.  The sample must hold exactly the
results of the full query that satisfy the restriction: checked here against
the oracle's full tuples filtered by the restriction, at sizes where the
full join is cheap.
"""
import types

import numpy as np
import pytest

import bench
import oracle

LW_ATOMS = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


def args(**kw):
    a = dict(workload="lw", tensor="dense", lw_n=8, ct_m=8, ct_first="common", seed=2)
    a.update(kw)
    return types.SimpleNamespace(**a)


@pytest.mark.parametrize("kw", [dict(workload="lw", tensor="dense", lw_n=40),
                                dict(workload="lw", tensor="sparse", lw_n=12),
                                dict(workload="ct", tensor="dense", ct_m=20, ct_first="common"),
                                dict(workload="ct", tensor="dense", ct_m=20, ct_first="paper"),
                                dict(workload="ct", tensor="sparse", ct_m=20, ct_first="common")])
def test_sample_equals_restricted_full_result(kw):
    a = args(**kw)
    atoms, rels, desc, closed = bench.tensor_relations(a, 0, None)
    cnt, full = oracle.kgj(4, atoms, rels, tuples=True)
    if closed is not None:
        assert cnt == closed
    sample, sdesc, ((vx, fx), (vy, fy)) = bench.tensor_sample(a, atoms, rels, "cpu")
    got, part = oracle.kgj(4, atoms, sample, tuples=True)
    keep = full[(full[:, vx] < fx) & (full[:, vy] < fy)]
    assert keep.shape[0] < full.shape[0] or full.shape[0] == 0  # the restriction removes results
    assert got == keep.shape[0]
    srt = lambda t: t[np.lexsort(t.T[::-1])] if t.shape[0] else t
    assert np.array_equal(srt(part), srt(keep))
