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


# ---------------------------------------------------------- k-ary relations

LW_ATOMS = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


def lw_sample(rels, fx, fy):
    """LW restricted to x < fx and y < fy (selections pushed into the atoms
    holding x and y); R4(Y,Z,U) keeps the rows whose (y, z) occurs in the
    restricted R1 (an exact semi-join reduction)."""
    r1, r2, r3, r4 = rels
    s1 = r1[(r1[:, 0] < fx) & (r1[:, 1] < fy)]
    s2 = r2[(r2[:, 0] < fx) & (r2[:, 1] < fy)]
    s3 = r3[r3[:, 0] < fx]
    import torch

    k1 = torch.from_numpy((s1[:, 1].astype(np.int64) << 32) | s1[:, 2].astype(np.int64)).cuda()
    k4 = torch.from_numpy((r4[:, 0].astype(np.int64) << 32) | r4[:, 1].astype(np.int64)).cuda()
    s4 = r4[torch.isin(k4, torch.unique(k1)).cpu().numpy()]
    return [np.ascontiguousarray(s) for s in (s1, s2, s3, s4)]


def test_lw_st_dense_512(hc):
    """LW over ST-Dense's four [512]^3 cubes (134 M rows each): 512^4
    results; a sample (x < 2, y < 32) equal to the oracle's."""
    n = 512
    cube = datagen.full_cube(n)
    q = hc.LW
    ixs = [hc.build_kindex(dev(cube), q.level_cols(j)) for j in range(4)]
    assert hc.run_kjoin(q, ixs).count == n ** 4
    del ixs
    sample = lw_sample([cube] * 4, 2, 32)
    want = oracle.kgj(4, LW_ATOMS, sample)
    assert want == 2 * 32 * n * n
    sx = [hc.build_kindex(dev(r), q.level_cols(j)) for j, r in enumerate(sample)]
    assert hc.run_kjoin(q, sx).count == want


def test_lw_st_sparse_512(hc):
    """LW over ST-Sparse's four relations (134 M distinct uniform tuples of
    [5120]^3 each): every output tuple satisfies every atom, and a sample
    (x < 128) equals the oracle's count."""
    rels = datagen.st_sparse(n=512, domain=5120, m=1, m_domain=1, seed=3, device="cuda")[:4]
    q = hc.LW
    ixs = [hc.build_kindex(dev(r), q.level_cols(j)) for j, r in enumerate(rels)]
    r = hc.run_kjoin(q, ixs, mode="materialize")
    t = u32(r.tuples)
    assert t.shape == (r.count, 4)
    assert np.unique(t, axis=0).shape[0] == t.shape[0]
    for (a, rel) in zip(LW_ATOMS, rels):  # rows are sorted, so packed keys (13 bits a value) are too
        keys = (rel[:, 0].astype(np.uint64) << np.uint64(26)) | (rel[:, 1].astype(np.uint64) << np.uint64(13)) | rel[:, 2]
        probe = ((t[:, a[0]].astype(np.uint64) << np.uint64(26)) | (t[:, a[1]].astype(np.uint64) << np.uint64(13))
                 | t[:, a[2]])
        pos = np.minimum(np.searchsorted(keys, probe), keys.shape[0] - 1)
        assert (keys[pos] == probe).all()
    del ixs
    sample = lw_sample(rels, 128, 5120)
    want = oracle.kgj(4, LW_ATOMS, sample)
    sx = [hc.build_kindex(dev(s), q.level_cols(j)) for j, s in enumerate(sample)]
    assert hc.run_kjoin(q, sx).count == want
    # the sample's results are exactly the full result's tuples with x < 128
    assert int((t[:, 0] < 128).sum()) == want
