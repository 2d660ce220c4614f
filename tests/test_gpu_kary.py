"""k-ary relations through the C ABI (needs a GB300): the k-level CoCo
(hc_build_kindex) against the oracle's levels, and Generic Join over it
(hc_run_kjoin) against the k-ary oracle, element by element.

Index arrays, counts, work counters and sorted tuples are integer results
and must match exactly.
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
    """About n distinct rows of k values below hi (shuffled)."""
    r = rng.integers(0, hi, size=(int(n * 1.2) + 8, k), dtype=np.uint64).astype(np.uint32)
    r = np.unique(r, axis=0)
    rng.shuffle(r)
    return np.ascontiguousarray(r[:n])


def check_index(hc, rows, cols, packed=None):
    ix = hc.build_kindex(dev(rows), cols)
    want = oracle.kcoco(rows, cols)
    k = rows.shape[1]
    assert ix.arity == k and ix.n == rows.shape[0]
    for d in range(k):
        assert ix.len[d] == want["V"][d].shape[0], d
        assert np.array_equal(host(ix.v(d)), want["V"][d]), d
    for d in range(k - 1):
        assert np.array_equal(host(ix.o(d)), want["O"][d]), d
    if packed is not None:
        assert ix.packed == packed
    return ix


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("n", [1, 31, 4095, 4096, 4097, 20011])
def test_kindex_matches_oracle(hc, k, n):
    rng = np.random.default_rng(1000 * k + n)
    hi = {1: 1 << 20, 2: 5000, 3: 60}[k]
    rows = distinct_rows(rng, n, k, hi)
    check_index(hc, rows, None, packed=True)


def test_kindex_level_orders(hc):
    rng = np.random.default_rng(7)
    rows = distinct_rows(rng, 9000, 3, 40)
    for cols in itertools.permutations(range(3)):
        check_index(hc, rows, cols)


def test_kindex_unpacked_and_wide_values(hc):
    """Levels whose value bits exceed 64 are sorted one level at a time."""
    rng = np.random.default_rng(8)
    rows = distinct_rows(rng, 12000, 3, 1 << 32)
    check_index(hc, rows, (0, 1, 2), packed=False)
    check_index(hc, rows, (2, 0, 1), packed=False)
    # few distinct values in the wide columns: long runs under each prefix
    rows2 = np.ascontiguousarray(np.unique(np.stack([
        rng.choice(np.array([0, 0xFFFFFFFF, 0x80000000], dtype=np.uint32), 8000),
        rng.choice(np.array([5, 0xFFFFFFFE], dtype=np.uint32), 8000),
        rng.integers(0, 1 << 32, 8000, dtype=np.uint64).astype(np.uint32)], axis=1), axis=0))
    check_index(hc, rows2, (0, 1, 2), packed=False)
    # 64 bits exactly: still packed
    rows3 = distinct_rows(rng, 5000, 2, 1 << 32)
    check_index(hc, rows3, (1, 0), packed=True)


def test_kindex_constant_columns_and_empty(hc):
    rows = np.stack([np.zeros(300, np.uint32), np.arange(300, dtype=np.uint32), np.full(300, 7, np.uint32)], axis=1)
    check_index(hc, rows, (0, 1, 2))
    check_index(hc, rows, (2, 0, 1))
    e = hc.build_kindex(dev(np.zeros((0, 3), np.uint32)))
    assert e.len == (0, 0, 0) and host(e.o(0)).tolist() == [0] and host(e.o(1)).tolist() == [0]


def test_kindex_duplicates(hc):
    rows = np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3]], dtype=np.uint32)
    with pytest.raises(hc.HoneycombError) as ei:
        hc.build_kindex(dev(rows), check_duplicates=True)
    assert ei.value.status == 6
    hc.build_kindex(dev(rows[:2]), check_duplicates=True)


# ------------------------------------------------------------------- joins

LW_ATOMS = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
CT_ATOMS = [(0, 1, 2), (0, 1, 3), (0, 2, 3)]


def run_both(hc, nv, atoms, rels, order=None, **kw):
    q = hc.KQuery(nv, tuple(tuple(a) for a in atoms), None if order is None else tuple(order))
    ixs = [hc.build_kindex(dev(r), q.level_cols(j)) for j, r in enumerate(rels)]
    cnt, tup, work = oracle.kgj(nv, atoms, rels, order=order, tuples=True, work=True)
    rc = hc.run_kjoin(q, ixs, stats=True, **kw)
    assert rc.count == cnt, (order, rc.count, cnt)
    assert rc.work == work, (order, rc.work, work)
    rm = hc.run_kjoin(q, ixs, mode="materialize", **kw)
    assert rm.count == cnt
    got = host(rm.tuples)
    assert got.shape == (cnt, nv)
    assert np.array_equal(sorted_rows(got), sorted_rows(tup)), order
    return cnt


@pytest.mark.parametrize("name", ["LW", "CT"])
@pytest.mark.parametrize("seed", range(3))
def test_hypergraph_queries_match_oracle(hc, name, seed):
    atoms = LW_ATOMS if name == "LW" else CT_ATOMS
    rng = np.random.default_rng(40 + seed)
    dom = 14
    rels = [distinct_rows(rng, int(rng.choice([300, 900, 1800])), 3, dom) for _ in atoms]
    for order in ((0, 1, 2, 3), (3, 2, 1, 0), (1, 3, 0, 2)):
        run_both(hc, 4, atoms, rels, order)


def test_lw_every_order(hc):
    rng = np.random.default_rng(5)
    rels = [distinct_rows(rng, 700, 3, 11) for _ in LW_ATOMS]
    counts = {run_both(hc, 4, LW_ATOMS, rels, order) for order in itertools.permutations(range(4))}
    assert len(counts) == 1


@pytest.mark.parametrize("seed", range(3))
def test_mixed_arities(hc, seed):
    rng = np.random.default_rng(60 + seed)
    atoms = [(2, 0, 4), (3, 1), (4,), (1, 2, 0), (3, 4)]
    dom = 9
    rels = []
    for a in atoms:
        n = {1: 6, 2: 50, 3: 350}[len(a)]
        rels.append(distinct_rows(rng, n, len(a), dom))
    for order in ((0, 1, 2, 3, 4), (4, 3, 2, 1, 0), (2, 4, 1, 3, 0)):
        run_both(hc, 5, atoms, rels, order)


def test_binary_atoms_match_binary_oracle(hc):
    sym = datagen.random_graph(120, 0.12, 3)
    ep = datagen.orient_lt(sym)
    for nv, atoms, rel in ((3, [(0, 1), (1, 2), (0, 2)], ep), (4, [(0, 1), (0, 2), (1, 3), (2, 3)], sym),
                           (4, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (0, 3)], ep)):
        want, _, _ = oracle.gj_count(nv, atoms, [rel] * len(atoms))
        q = hc.KQuery(nv, tuple(atoms))
        ixs = [hc.build_kindex(dev(rel), q.level_cols(j)) for j in range(len(atoms))]
        assert hc.run_kjoin(q, ixs).count == want


def test_one_and_two_variables(hc):
    rng = np.random.default_rng(9)
    a = distinct_rows(rng, 3000, 1, 5000)
    b = distinct_rows(rng, 2500, 1, 5000)
    run_both(hc, 1, [(0,), (0,)], [a, b])
    r = distinct_rows(rng, 4000, 2, 300)
    s = distinct_rows(rng, 120, 1, 300)
    run_both(hc, 2, [(0, 1), (1,)], [r, s])
    run_both(hc, 2, [(0, 1), (1,)], [r, s], order=(1, 0))


def test_empty_relation_and_no_output(hc):
    cube = datagen.full_cube(6)
    empty = np.zeros((0, 3), dtype=np.uint32)
    assert run_both(hc, 4, LW_ATOMS, [cube, cube, cube, empty]) == 0
    assert run_both(hc, 4, LW_ATOMS, [empty, cube, cube, cube]) == 0
    sets = [np.array([0, 1]), np.array([0, 2]), np.array([1, 2])]
    rels = [datagen.prefixed_square(s.astype(np.uint32), 9) for s in sets]
    assert run_both(hc, 4, CT_ATOMS, rels) == 0


def test_st_dense_small(hc):
    """ST-Dense shapes at reduced size: LW over four [n]^3 cubes is n^4; CT
    over the three prefixed squares is 0 (C22), and m^3 when the middle
    set is widened to {0,1,2}."""
    n, m = 24, 20
    rels = datagen.st_dense(n=n, m=m)
    q = hc.LW
    ixs = [hc.build_kindex(dev(r), q.level_cols(j)) for j, r in enumerate(rels[:4])]
    assert hc.run_kjoin(q, ixs).count == n ** 4
    ixs = [hc.build_kindex(dev(r), hc.CT.level_cols(j)) for j, r in enumerate(rels[4:])]
    assert hc.run_kjoin(hc.CT, ixs).count == 0
    wide = datagen.prefixed_square(np.array([0, 1, 2], dtype=np.uint32), m)
    ixs[1] = hc.build_kindex(dev(wide), hc.CT.level_cols(1))
    assert hc.run_kjoin(hc.CT, ixs).count == m ** 3


def test_st_sparse_small(hc):
    rels = datagen.st_sparse(n=20, domain=60, m=30, m_domain=90, seed=2)
    run_both(hc, 4, LW_ATOMS, rels[:4])
    run_both(hc, 4, CT_ATOMS, rels[4:])


def test_launch_shapes_agree(hc):
    """LW on [64]^3 cubes (262,144 rows each): 64^4 results for every block
    size and work-item grain."""
    cube = datagen.full_cube(64)
    q = hc.LW
    ixs = [hc.build_kindex(dev(cube), q.level_cols(j)) for j in range(4)]
    for bt in (32, 64, 128):
        for grain in (0, 1, 7, 100000):
            r = hc.run_kjoin(q, ixs, block_threads=bt, item_grain=grain)
            assert r.count == 64 ** 4, (bt, grain)


def test_bad_arguments(hc):
    rng = np.random.default_rng(1)
    r3 = distinct_rows(rng, 50, 3, 8)
    q = hc.KQuery(4, ((0, 1, 2), (1, 2, 3)))
    good = [hc.build_kindex(dev(r3), q.level_cols(j)) for j in range(2)]
    hc.run_kjoin(q, good)
    wrong_levels = [hc.build_kindex(dev(r3), (2, 1, 0)), good[1]]
    with pytest.raises(hc.HoneycombError) as ei:
        hc.run_kjoin(q, wrong_levels)
    assert ei.value.status == 1
    r2 = distinct_rows(rng, 50, 2, 8)
    with pytest.raises(hc.HoneycombError) as ei:
        hc.run_kjoin(q, [hc.build_kindex(dev(r2)), good[1]])  # arity differs from the atom's
    assert ei.value.status == 1
    q5 = hc.KQuery(2, tuple([(0, 1)] * 5))  # X in five atoms
    with pytest.raises(hc.HoneycombError) as ei:
        hc.run_kjoin(q5, [hc.build_kindex(dev(r2))] * 5)
    assert ei.value.status == 5
    q7 = hc.KQuery(7, ((0, 1, 2), (3, 4, 5), (6,)))
    with pytest.raises(hc.HoneycombError) as ei:
        hc.run_kjoin(q7, [good[0], good[0], hc.build_kindex(dev(r3[:, :1].copy()))])
    assert ei.value.status == 5


def test_chosen_order_matches_oracle(hc):
    """The order hc_choose_korder picks from the built indexes' statistics
    changes only the work: the result equals the oracle's."""
    rng = np.random.default_rng(77)
    atoms = [(2, 0, 3), (1, 2), (3,), (1, 0)]
    rels = [distinct_rows(rng, n, len(a), 12) for a, n in zip(atoms, (900, 60, 8, 100))]
    q = hc.KQuery(4, tuple(atoms))
    stats = [hc.build_kindex(dev(r)) for r in rels]
    order = hc.choose_korder(q, stats)
    assert sorted(order) == [0, 1, 2, 3]
    run_both(hc, 4, atoms, rels, order)


@pytest.mark.parametrize("seed", range(2))
def test_six_variables(hc, seed):
    """The largest k-ary query (HC_KMAX_VARS = 6 loops): two ternary atoms,
    binary and unary ones, against the oracle under two orders."""
    rng = np.random.default_rng(90 + seed)
    atoms = [(0, 1, 2), (2, 3, 4), (4, 5), (5, 0), (1, 3), (3,)]
    dom = 7
    rels = [distinct_rows(rng, {1: 5, 2: 30, 3: 200}[len(a)], len(a), dom) for a in atoms]
    for order in ((0, 1, 2, 3, 4, 5), (5, 3, 1, 4, 0, 2)):
        run_both(hc, 6, atoms, rels, order)


@pytest.mark.parametrize("pair_min", [1, 4, 0xFFFFFFFF])
def test_last_loop_paths_agree(hc, pair_min):
    """The last loop's per-binding path (warp-wide, 128 candidates an
    iteration) against the flattened one: pair_min 1 sends every last-loop
    binding through it, 0xFFFFFFFF none; counts, work and sorted tuples
    equal the oracle's for LW, CT, mixed arities (a last loop with one list,
    and a top-level list with a position map), two and six variables, and a
    cube whose bindings span several 128-candidate blocks."""
    rng = np.random.default_rng(123)
    rels = [distinct_rows(rng, 1500, 3, 14) for _ in LW_ATOMS]
    run_both(hc, 4, LW_ATOMS, rels, (0, 1, 2, 3), pair_min=pair_min)
    run_both(hc, 4, LW_ATOMS, rels, (3, 1, 0, 2), pair_min=pair_min)
    run_both(hc, 4, CT_ATOMS, rels[:3], (1, 0, 2, 3), pair_min=pair_min)
    atoms = [(2, 0, 4), (3, 1), (4,), (1, 2, 0), (3, 4)]
    mixed = [distinct_rows(rng, {1: 6, 2: 50, 3: 350}[len(a)], len(a), 9) for a in atoms]
    run_both(hc, 5, atoms, mixed, (0, 1, 2, 3, 4), pair_min=pair_min)
    run_both(hc, 5, atoms, mixed, (4, 3, 2, 1, 0), pair_min=pair_min)
    r = distinct_rows(rng, 4000, 2, 300)
    s = distinct_rows(rng, 120, 1, 300)
    run_both(hc, 2, [(0, 1), (1,)], [r, s], pair_min=pair_min)
    run_both(hc, 2, [(0, 1)], [r], pair_min=pair_min)
    six = [(0, 1, 2), (2, 3, 4), (4, 5), (5, 0), (1, 3), (3,)]
    rels6 = [distinct_rows(rng, {1: 5, 2: 30, 3: 200}[len(a)], len(a), 7) for a in six]
    run_both(hc, 6, six, rels6, (5, 3, 1, 4, 0, 2), pair_min=pair_min)
    cube = datagen.full_cube(40)
    sparse = [cube[rng.random(cube.shape[0]) < 0.7] for _ in LW_ATOMS]
    run_both(hc, 4, LW_ATOMS, sparse, pair_min=pair_min)


@pytest.mark.parametrize("pair_min", [0, 1, 0xFFFFFFFF])
def test_dense_runs(hc, pair_min):
    """Lists that hold every integer of their range (ST-Dense cubes, here
    offset by 1000 so that no range starts at 0) are searched by reading the
    one position a value can take; mixed with lists that have gaps, runs of
    exactly 32 values (the per-binding threshold), and materialize mode,
    all against the oracle."""
    rng = np.random.default_rng(321)
    cube = datagen.full_cube(12).astype(np.uint32) + np.uint32(1000)
    holes = cube[rng.random(cube.shape[0]) < 0.8]
    run_both(hc, 4, LW_ATOMS, [cube] * 4, pair_min=pair_min)
    run_both(hc, 4, LW_ATOMS, [cube, holes, cube, holes], pair_min=pair_min)
    run_both(hc, 4, LW_ATOMS, [holes, cube, cube, cube], (2, 0, 3, 1), pair_min=pair_min)
    c32 = np.array(list(itertools.product(range(3), range(3), range(32))), dtype=np.uint32)
    run_both(hc, 4, LW_ATOMS, [c32, c32, c32, c32], pair_min=pair_min)
    run_both(hc, 4, CT_ATOMS, [cube, holes, cube], pair_min=pair_min)
