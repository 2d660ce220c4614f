"""Parity at the full workload sizes (needs a GB300).

The oracle cannot run these whole joins in test time, so each is checked on
what it can compute exactly:
  * a sample: the query with x restricted to a seeded vertex subset F (a
    selection pushed into the atoms that hold x, Sec. 2), run by both the
    GPU and the oracle on the same restricted relations -- equal counts, and
    for the triangle equal sorted tuples;
  * properties that hold at any size: the full count does not depend on the
    shares (Sec. 5: cell outputs are disjoint and cover Q), the cell counts
    sum to it, and every sampled output tuple satisfies every atom.
Workloads: the triangle on R-MAT scale 22 (edge factor 16) and the 4-clique /
4-cycle on R-MAT scale 20, as used by the benchmark.
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


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def sorted_rows(a):
    return a[np.lexsort(a.T[::-1])] if a.shape[0] else a


def restrict(rel, col, mask):
    return np.ascontiguousarray(rel[mask[rel[:, col]]])


@pytest.fixture(scope="module")
def rmat22():
    sym = datagen.rmat_graph(22, 16, 2, device="cuda")
    ep = datagen.scatter_order(datagen.orient_lt(sym), 2)
    return ep


def test_triangle_rmat22(hc, rmat22):
    import torch

    ep = rmat22
    q = hc.TRIANGLE
    ix = hc.build_index(dev(ep), 0)
    plan = hc.choose_shares(q, [ix] * 3, 1024)
    counts = {}
    for sh in ([1, 1, 1], plan, [32, 32, 1]):
        r = hc.run_join(q, [ix] * 3, shares=sh, cell_counts=True)
        assert int(r.cell_counts.sum()) == r.count
        counts[tuple(sh)] = r.count
    assert len(set(counts.values())) == 1, counts
    total = counts[(1, 1, 1)]

    # sample: x in F (R and T restricted on x; S restricted to the y that
    # R[F] reaches, which cannot change the result)
    nv = int(ep.max()) + 1
    fmask = datagen.vertex_sample_mask(nv, 77, 1.0 / 256)
    r_f = restrict(ep, 0, fmask)
    ys = np.zeros(nv, dtype=bool)
    ys[r_f[:, 1]] = True
    s_f = restrict(ep, 0, ys)
    want_cnt, _, _ = oracle.gj_count(3, list(q.atoms), [r_f, s_f, r_f], nthreads=16)
    ixr, ixs = hc.build_index(dev(r_f), 0), hc.build_index(dev(s_f), 0)
    got = hc.run_join(q, [ixr, ixs, ixr], mode="materialize")
    assert got.count == want_cnt
    want = oracle.gj_enumerate(3, list(q.atoms), [r_f, s_f, r_f])
    assert np.array_equal(sorted_rows(u32(got.tuples)), sorted_rows(want))

    # full materialize: the rows with x in F are exactly the sample's tuples,
    # and sampled rows satisfy every atom
    full = hc.run_join(q, [ix] * 3, shares=plan, mode="materialize", out_capacity=int(total * 1.1) + 1,
                       keep_device=True)
    assert full.count == total and full.tuples.shape[0] == total
    fx = torch.from_numpy(np.nonzero(fmask)[0].astype(np.int64)).cuda()
    sel = torch.isin(full.tuples[:, 0].to(torch.int64), fx)
    assert np.array_equal(sorted_rows(u32(full.tuples[sel])), sorted_rows(want))
    idx = torch.randint(0, total, (200_000,), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    rows = u32(full.tuples[idx]).astype(np.uint64)
    keys = np.sort((ep[:, 0].astype(np.uint64) << np.uint64(32)) | ep[:, 1])
    assert np.all(rows[:, 0] < rows[:, 1]) and np.all(rows[:, 1] < rows[:, 2])
    for a, b in ((0, 1), (1, 2), (0, 2)):
        k = (rows[:, a] << np.uint64(32)) | rows[:, b]
        pos = np.searchsorted(keys, k)
        assert np.all(keys[np.minimum(pos, keys.shape[0] - 1)] == k)


@pytest.fixture(scope="module")
def rmat20():
    sym = datagen.rmat_graph(20, 16, 3, device="cuda")
    return sym


def test_four_clique_rmat20(hc, rmat20):
    sym = rmat20
    ep = datagen.scatter_order(datagen.orient_lt(sym), 3)
    q = hc.FOUR_CLIQUE
    ix = hc.build_index(dev(ep), 0)
    a = hc.run_join(q, [ix] * 6).count
    b = hc.run_join(q, [ix] * 6, shares=hc.choose_shares(q, [ix] * 6, 256)).count
    assert a == b
    nv = int(ep.max()) + 1
    fmask = datagen.vertex_sample_mask(nv, 78, 1.0 / 512)
    # atoms holding x: R1(X,Y), R2(X,Z), R6(X,U)
    rx = restrict(ep, 0, fmask)
    rels = [rx, rx, ep, ep, ep, rx]
    want, _, _ = oracle.gj_count(4, list(q.atoms), rels, nthreads=16)
    ixr = hc.build_index(dev(rx), 0)
    assert hc.run_join(q, [ixr, ixr, ix, ix, ix, ixr]).count == want


def test_four_cycle_rmat20_sample(hc, rmat20):
    sym = datagen.scatter_order(rmat20, 4)
    q = hc.FOUR_CYCLE
    ix = hc.build_index(dev(sym), 0)
    nv = int(sym.max()) + 1
    fmask = datagen.vertex_sample_mask(nv, 79, 1.0 / 32768)
    # atoms holding x: R1(X,Y), R2(X,Z)
    rx = restrict(sym, 0, fmask)
    rels = [rx, rx, sym, sym]
    want, _, _ = oracle.gj_count(4, list(q.atoms), rels, nthreads=16)
    ixr = hc.build_index(dev(rx), 0)
    for sh in ([1, 1, 1, 1], [4, 2, 2, 1]):
        assert hc.run_join(q, [ixr, ixr, ix, ix], shares=sh).count == want
