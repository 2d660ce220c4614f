"""Plans chosen by hc_choose_plan (loop order + shares, Sec. 5.3) run through
the C ABI and give the oracle's result (needs a GB300).

The order and shares a plan picks change only the work, never the result:
counts and sorted tuples are compared exactly with the oracle.
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

    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint32).reshape(-1, 2))
    return torch.from_numpy(a.view(np.int32)).cuda()


def sorted_rows(a):
    a = np.asarray(a)
    return a if a.shape[0] == 0 else a[np.lexsort(a.T[::-1])]


def run_with_plan(hc, q, rels, P, **kw):
    """Statistics from attr-order-0 indexes, then the chosen plan's indexes."""
    stat_ix = [hc.build_index(dev(r), 0) for r in rels]
    order, shares = hc.choose_plan(q, stat_ix, P)
    qo = q.with_order(order)
    ixs = [hc.build_index(dev(r), qo.attr_order(j)) for j, r in enumerate(rels)]
    return order, shares, hc.run_join(qo, ixs, shares=shares, **kw)


@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_DIAMOND", "FOUR_CLIQUE", "TWO_TRIANGLE"])
@pytest.mark.parametrize("P", [1, 16, 256])
def test_chosen_plan_matches_oracle(hc, qname, P):
    q = getattr(hc, qname)
    rng = np.random.default_rng(100 + P)
    # relations of different sizes, so that the plan's order differs from the textual one
    rels = []
    for j in range(len(q.atoms)):
        n = int(rng.choice([60, 400, 1500]))
        rels.append(datagen.directed_set(rng.integers(0, 64, size=(n, 2)).astype(np.uint32)))
    ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
    order, shares, r = run_with_plan(hc, q, rels, P, mode="materialize")
    assert r.count == ref.shape[0], (order, shares)
    assert np.array_equal(sorted_rows(r.tuples.cpu().numpy().view(np.uint32)), sorted_rows(ref)), (order, shares)


def test_chosen_plan_on_rmat_counts(hc):
    """R-MAT graph (skewed degrees): triangle on E+, 4-cycle on E, 4-clique on E+."""
    sym = datagen.rmat_graph(10, 8, 33)
    ep = datagen.orient_lt(sym)
    for q, rel in ((hc.TRIANGLE, ep), (hc.FOUR_CYCLE, sym), (hc.FOUR_CLIQUE, ep)):
        rels = [rel] * len(q.atoms)
        cnt, _, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
        for P in (1, 64):
            order, shares, r = run_with_plan(hc, q, rels, P)
            assert r.count == cnt, (q, order, shares)
