"""Per-cell work and time (the skew study of Sec. 1, Examples 1-3).

A HyperCube cell is one logical worker; with HC_FLAG_CELL_PROFILE the join
returns, per cell, the work counter restricted to the cell's bindings and the
SM cycles its warps spent on it.  The per-cell work must equal the oracle's
work counter on the cell's restriction of every relation (the rows whose
shares match the cell's coordinates, Sec. 4), and the cells must add up to the
whole join's counter.
"""
import itertools

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


def cell_restriction(q, rels, seeds, shares, coords):
    """Each atom's rows whose values fall in the cell's shares."""
    out = []
    for (a, b), r in zip(q.atoms, rels):
        keep = np.ones(r.shape[0], dtype=bool)
        for col, v in ((0, a), (1, b)):
            if v is None or v < 0 or shares[v] == 1:
                continue
            s = np.array([oracle.share(int(x), seeds[v], shares[v]) for x in r[:, col]], dtype=np.int64)
            keep &= s == coords[v]
        out.append(np.ascontiguousarray(r[keep]))
    return out


@pytest.mark.parametrize("qname,shares", [("TRIANGLE", [2, 2, 1]), ("TRIANGLE", [4, 1, 2]),
                                          ("FOUR_CYCLE", [2, 1, 2, 1]), ("FOUR_CLIQUE", [2, 2, 1, 2])])
def test_cell_work_equals_oracle_per_cell(hc, qname, shares):
    q = getattr(hc, qname)
    sym = datagen.rmat_graph(8, 8, 17)
    rel = sym if qname == "FOUR_CYCLE" else datagen.orient_lt(sym)
    rels = [rel] * len(q.atoms)
    seeds = list(hc.DEFAULT_SEEDS[: q.n_vars])
    ixs = [hc.build_index(dev(r), q.attr_order(j)) for j, r in enumerate(rels)]
    r = hc.run_join(q, ixs, shares=shares, seeds=seeds, cell_profile=True, cell_counts=True)
    prof = r.cell_profile.cpu().numpy()
    assert prof.shape == (int(np.prod(shares)), 2)
    assert int(prof[:, 0].sum()) == r.work
    assert int(r.cell_counts.sum()) == r.count
    strides = [int(np.prod(shares[v + 1:])) for v in range(q.n_vars)]
    for c in range(prof.shape[0]):
        coords = [(c // strides[v]) % shares[v] for v in range(q.n_vars)]
        sub = cell_restriction(q, rels, seeds, shares, coords)
        cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), sub)
        assert int(prof[c, 0]) == work, (c, coords)
        assert int(r.cell_counts[c]) == cnt, (c, coords)
        if cnt > 0:
            assert int(prof[c, 1]) > 0  # the cell's items took time


def test_profile_does_not_change_results(hc):
    ep = datagen.orient_lt(datagen.rmat_graph(11, 16, 5))
    ix = hc.build_index(dev(ep), 0)
    q = hc.TRIANGLE
    cnt, work, _ = oracle.gj_count(3, list(q.atoms), [ep] * 3)
    for sh in ([1, 1, 1], [64, 1, 1], [4, 4, 4]):
        r = hc.run_join(q, [ix] * 3, shares=sh, cell_profile=True, mode="materialize")
        assert r.count == cnt
        if sh == [1, 1, 1]:
            assert r.work == work
        assert int(r.cell_profile[:, 0].sum()) == r.work
