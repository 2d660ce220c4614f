"""HyperCube shares for k-ary relations through the C ABI (needs a GB300):
the partitioned k-level CoCo (hc_build_kindex_partitioned) against the
oracle's partitioning (Sec. 4, "Preprocessor"), and Generic Join over every
cell (hc_run_kjoin) against the unpartitioned k-ary oracle: the result does
not depend on the shares, and each cell's count is the number of oracle
tuples that hash to it (Sec. 4-5: the cells' outputs are disjoint).

Index arrays, partition starts, counts, work counters and sorted tuples are
integer results and must match exactly.
"""
import itertools

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc(cuda_device):
    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    return hc


def dev(rows):
    import torch

    a = np.ascontiguousarray(np.asarray(rows, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def sorted_rows(a):
    a = np.asarray(a)
    return a if a.shape[0] == 0 else a[np.lexsort(a.T[::-1])]


def distinct_rows(rng, n, k, hi):
    r = rng.integers(0, hi, size=(int(n * 1.2) + 8, k), dtype=np.uint64).astype(np.uint32)
    r = np.unique(r, axis=0)
    rng.shuffle(r)
    return np.ascontiguousarray(r[:n])


def check_partitioned(hc, rows, cols, seeds, shares, packed=None):
    ix = hc.build_kindex(dev(rows), cols, seeds=seeds, shares=shares)
    want = oracle.kpartition(rows, seeds, shares, cols)
    k = rows.shape[1]
    npart = int(np.prod(shares))
    assert ix.n_parts == npart
    for d in range(k):
        assert ix.len[d] == want["V"][d].shape[0], d
        assert np.array_equal(host(ix.v(d)), want["V"][d]), d
    for d in range(k - 1):
        assert np.array_equal(host(ix.o(d)), want["O"][d]), d
    if npart > 1:
        assert np.array_equal(host(ix.bpref()).astype(np.uint64), want["Bpref"])
        assert np.array_equal(host(ix.level0_start()).astype(np.uint64), want["l0start"])
    else:
        assert ix.bpref() is None and ix.level0_start() is None
    if packed is not None:
        assert ix.packed == packed
    return ix


@pytest.mark.parametrize("k,shares", [(1, (5,)), (2, (4, 3)), (2, (1, 7)), (3, (2, 2, 1)), (3, (3, 1, 4)),
                                      (3, (1, 1, 1)), (3, (16, 16, 16))])
@pytest.mark.parametrize("n", [1, 4097, 20011])
def test_partitioned_kindex_matches_oracle(hc, k, shares, n):
    rng = np.random.default_rng(31 * n + k)
    hi = {1: 1 << 20, 2: 5000, 3: 60}[k]
    rows = distinct_rows(rng, n, k, hi)
    seeds = [int(x) for x in rng.integers(1, 1 << 31, size=k)]
    check_partitioned(hc, rows, None, seeds, shares, packed=True)


def test_partitioned_kindex_level_orders(hc):
    rng = np.random.default_rng(9)
    rows = distinct_rows(rng, 9000, 3, 40)
    for cols in itertools.permutations(range(3)):
        check_partitioned(hc, rows, cols, (5, 6, 7), (2, 3, 2))


def test_partitioned_kindex_unpacked(hc):
    """Value bits plus partition bits above 64: the rows are sorted one level
    at a time, then by partition id."""
    rng = np.random.default_rng(10)
    rows = distinct_rows(rng, 12000, 3, 1 << 32)
    check_partitioned(hc, rows, (0, 1, 2), (1, 2, 3), (2, 3, 4), packed=False)
    check_partitioned(hc, rows, (2, 0, 1), (1, 2, 3), (4, 1, 4), packed=False)
    # 64 value bits: packed alone, unpacked once partitioned
    rows2 = distinct_rows(rng, 5000, 2, 1 << 32)
    check_partitioned(hc, rows2, (1, 0), (3, 4), (1, 1), packed=True)
    check_partitioned(hc, rows2, (1, 0), (3, 4), (2, 1), packed=False)


def test_partitioned_kindex_empty_partitions_and_empty_relation(hc):
    rows = np.stack([np.zeros(300, np.uint32), np.arange(300, dtype=np.uint32), np.full(300, 7, np.uint32)], axis=1)
    # columns 0 and 2 are constant: most partitions are empty
    check_partitioned(hc, rows, (0, 1, 2), (3, 4, 5), (4, 2, 4))
    e = hc.build_kindex(dev(np.zeros((0, 3), np.uint32)), seeds=(1, 2, 3), shares=(2, 2, 2))
    assert e.n_parts == 8 and host(e.bpref()).tolist() == [0] * 9 and host(e.level0_start()).tolist() == [0] * 9


def test_partition_worked_example(hc):
    """Sec. 4, Example "partition": R(X,Y,Z) with shares 2x2x1; partition
    (0,1,0) = {(0,4,1), (5,3,9)} starts at B^pref[0,1,0] = 3 with B = 2, and
    partition (1,0,0) is empty (the hash seeds are chosen so that the
    paper's assumed hash values hold)."""
    px, py, pz = 2, 2, 1
    grey_tuples = [(0, 4, 1), (5, 3, 9)]
    sx = next(s for s in range(1, 100000) if all(oracle.share(t[0], s, px) == 0 for t in grey_tuples))
    sy = next(s for s in range(1, 100000) if all(oracle.share(v, s, py) == 1 for v in (1, 4, 5, 3)))
    xs0 = [v for v in range(10, 400) if oracle.share(v, sx, px) == 0][:3]
    xs1 = [v for v in range(10, 400) if oracle.share(v, sx, px) == 1][:2]
    ys0 = [v for v in range(10, 400) if oracle.share(v, sy, py) == 0][:3]
    rel = [(xs0[i], ys0[i], 7 + i) for i in range(3)] + grey_tuples + [(xs1[0], 1, 2), (xs1[1], 4, 6)]
    rows = np.array(rel, dtype=np.uint32)
    ix = hc.build_kindex(dev(rows), seeds=(sx, sy, 77), shares=(px, py, pz))
    b = host(ix.bpref()).astype(np.int64)
    grey = (0 * py + 1) * pz + 0
    empty = (1 * py + 0) * pz + 0
    assert b[grey] == 3 and b[grey + 1] - b[grey] == 2
    assert b[empty + 1] - b[empty] == 0
    # the grey partition's rows, walked from its level-0 range
    l0 = host(ix.level0_start()).astype(np.int64)
    V = [host(ix.v(d)) for d in range(3)]
    O = [host(ix.o(d)) for d in range(2)]
    got = []
    for a in range(l0[grey], l0[grey + 1]):
        for bb in range(O[0][a], O[0][a + 1]):
            for c in range(O[1][bb], O[1][bb + 1]):
                got.append((int(V[0][a]), int(V[1][bb]), int(V[2][c])))
    assert got == sorted(grey_tuples)


# ------------------------------------------------------------------- joins

LW = (4, [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)])
CT = (4, [(0, 1, 2), (0, 1, 3), (0, 2, 3)])


def random_rel(rng, k, dom, density):
    full = np.array(list(itertools.product(range(dom), repeat=k)), dtype=np.uint32).reshape(-1, k)
    keep = rng.random(full.shape[0]) < density
    return np.ascontiguousarray(full[keep])


def oracle_cell_work(nv, atoms, rels, order, vseeds, vshares):
    """Work counter summed over the cells, each cell's Generic Join run by
    the oracle on the partitions its coordinates select."""
    parts = [oracle.kpartition(r, [vseeds[v] for v in a], [vshares[v] for v in a]) for a, r in zip(atoms, rels)]
    total = 0
    for cell in itertools.product(*[range(s) for s in vshares]):
        sub = []
        for a, pt in zip(atoms, parts):
            pid = 0
            for v in a:
                pid = pid * vshares[v] + cell[v]
            sub.append(pt["rt"][int(pt["Bpref"][pid]):int(pt["Bpref"][pid + 1])])
        total += oracle.kgj(nv, atoms, sub, order=order, work=True)[1]
    return total


def run_cells(hc, nv, atoms, rels, vshares, vseeds, order=None, check_work=False, **kw):
    q = hc.KQuery(nv, tuple(tuple(a) for a in atoms), None if order is None else tuple(order))
    per_atom = hc.atom_shares(q, vshares, vseeds)
    ixs = [hc.build_kindex(dev(r), q.level_cols(j), seeds=per_atom[j][0], shares=per_atom[j][1])
           for j, r in enumerate(rels)]
    cnt, tup = oracle.kgj(nv, atoms, rels, order=order, tuples=True)
    rc = hc.run_kjoin(q, ixs, stats=check_work, cell_counts=True, **kw)
    n_cells = int(np.prod(vshares))
    assert rc.count == cnt, (vshares, order, rc.count, cnt)
    assert rc.n_cells == n_cells
    want_cells = np.bincount(oracle.tuple_cells(tup, vseeds, vshares).astype(np.int64), minlength=n_cells) \
        if cnt else np.zeros(n_cells, dtype=np.int64)
    assert np.array_equal(rc.cell_counts.cpu().numpy(), want_cells), vshares
    if check_work:
        assert rc.work == oracle_cell_work(nv, atoms, rels, order, vseeds, vshares), vshares
    rm = hc.run_kjoin(q, ixs, mode="materialize", **kw)
    assert rm.count == cnt
    got = host(rm.tuples)
    assert np.array_equal(sorted_rows(got), sorted_rows(tup)), vshares
    return cnt


@pytest.mark.parametrize("vshares", [(2, 2, 1, 2), (1, 1, 1, 1), (3, 1, 2, 1), (4, 1, 1, 1), (1, 1, 1, 5),
                                     (2, 3, 2, 2), (4, 4, 4, 4)])
def test_lw_share_invariance(hc, vshares):
    """LW (Table "Queries") on random relations: the same result, per-cell
    counts and (summed over cells) work for every share vector, including
    the paper's P = 2x2x1x2 (Example "partition")."""
    nv, atoms = LW
    rng = np.random.default_rng(5)
    rels = [random_rel(rng, 3, 12, 0.45) for _ in atoms]
    seeds = (101, 202, 303, 404)
    small = int(np.prod(vshares)) <= 16
    run_cells(hc, nv, atoms, rels, vshares, seeds, check_work=small)
    run_cells(hc, nv, atoms, rels, vshares, seeds, order=(3, 1, 0, 2))


@pytest.mark.parametrize("vshares", [(2, 2, 1, 2), (1, 3, 3, 1), (8, 1, 1, 1)])
def test_ct_share_invariance(hc, vshares):
    nv, atoms = CT
    rng = np.random.default_rng(6)
    rels = [random_rel(rng, 3, 12, 0.5) for _ in atoms]
    run_cells(hc, nv, atoms, rels, vshares, (7, 8, 9, 10), check_work=True)


@pytest.mark.parametrize("seed", range(2))
def test_mixed_arities_share_invariance(hc, seed):
    """Unary, binary and ternary atoms; a variable bound at a later loop at
    the top level of its atom (R(U) with U last), so top-level lists of
    loops after loop 0 are partitioned too."""
    nv, atoms = 4, [(2, 0, 3), (1, 2), (3,), (1, 0)]
    rng = np.random.default_rng(70 + seed)
    rels = [random_rel(rng, len(a), 9, 0.5) for a in atoms]
    for vshares in ((2, 2, 2, 2), (1, 3, 1, 2), (3, 1, 1, 1)):
        run_cells(hc, nv, atoms, rels, vshares, (3, 5, 7, 9), check_work=True)
        run_cells(hc, nv, atoms, rels, vshares, (3, 5, 7, 9), order=(3, 2, 1, 0))


def test_one_variable_and_dense_cube_cells(hc):
    """n_vars = 1 (loop 0 only) over several cells, and a larger LW over a
    near-full cube whose loop-0 and search span several tiles."""
    rng = np.random.default_rng(12)
    a = np.unique(rng.integers(0, 5000, 3000).astype(np.uint32))[:, None]
    b = np.unique(rng.integers(0, 5000, 3000).astype(np.uint32))[:, None]
    run_cells(hc, 1, [(0,), (0,)], [a, b], (7,), (99,), check_work=True)
    nv, atoms = LW
    rels = [random_rel(rng, 3, 40, 0.8) for _ in atoms]
    run_cells(hc, nv, atoms, rels, (2, 2, 1, 2), (1, 2, 3, 4))


def test_empty_cells_and_relations(hc):
    nv, atoms = LW
    rng = np.random.default_rng(13)
    rels = [random_rel(rng, 3, 6, 0.5) for _ in atoms]
    rels[2] = np.zeros((0, 3), np.uint32)
    assert run_cells(hc, nv, atoms, rels, (2, 2, 2, 2), (1, 2, 3, 4)) == 0
    # more cells than values: most cells empty
    rels = [random_rel(rng, 3, 4, 0.9) for _ in atoms]
    run_cells(hc, nv, atoms, rels, (16, 16, 1, 16), (1, 2, 3, 4))


def test_inconsistent_shares_rejected(hc):
    nv, atoms = LW
    rng = np.random.default_rng(14)
    rels = [random_rel(rng, 3, 6, 0.5) for _ in atoms]
    q = hc.KQuery(nv, tuple(tuple(a) for a in atoms))
    per_atom = hc.atom_shares(q, (2, 2, 1, 2), (1, 2, 3, 4))
    ixs = [hc.build_kindex(dev(r), q.level_cols(j), seeds=per_atom[j][0], shares=per_atom[j][1])
           for j, r in enumerate(rels)]
    # atom 3 partitioned with another seed for Y
    bad = hc.build_kindex(dev(rels[3]), q.level_cols(3), seeds=(9, 3, 4), shares=(2, 1, 2))
    with pytest.raises(hc.HoneycombError) as ei:
        hc.run_kjoin(q, ixs[:3] + [bad])
    assert ei.value.status == 1
    # atom 0 unpartitioned while the others split X, Y
    plain = hc.build_kindex(dev(rels[0]), q.level_cols(0))
    with pytest.raises(hc.HoneycombError):
        hc.run_kjoin(q, [plain] + ixs[1:])
    with pytest.raises(hc.HoneycombError):
        hc.build_kindex(dev(rels[0]), seeds=(1, 2, 3), shares=(0, 1, 1))
    with pytest.raises(hc.HoneycombError):
        hc.build_kindex(dev(rels[0]), seeds=(1, 2, 3), shares=(256, 256, 2))
