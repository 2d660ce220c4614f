"""GPU parity against the CPU oracle through the C ABI (needs a GB300).

Integer work throughout: every comparison is exact (bit-exact arrays,
equal counts, equal sorted tuple sets).
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

    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint32).reshape(-1, 2))
    return torch.from_numpy(a.view(np.int32)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def sorted_rows(a):
    a = np.asarray(a)
    if a.shape[0] == 0:
        return a
    return a[np.lexsort(a.T[::-1])]


# ------------------------------------------------------------------ CoCo build

@pytest.mark.parametrize("n", [1, 2, 31, 100, 4095, 4096, 4097, 65537, 300_001])
@pytest.mark.parametrize("ao", [0, 1])
def test_build_index_matches_oracle(hc, n, ao):
    rng = np.random.default_rng(n * 7 + ao)
    hi = 1 << 22 if n > 1000 else 50
    pairs = datagen.directed_set(rng.integers(0, hi, size=(int(n * 1.2) + 2, 2)).astype(np.uint32))[:n]
    pairs = datagen.scatter_order(pairs, n)
    ix = hc.build_index(dev(pairs), ao, check_duplicates=True)
    v1, o1, v2 = oracle.coco_build(pairs, ao)
    assert ix.n == pairs.shape[0] and ix.l1 == v1.shape[0]
    assert ix.max_run == int(np.diff(o1).max())  # the longest run, for run_join's list limit
    assert np.array_equal(u32(ix.v1()), v1)
    assert np.array_equal(u32(ix.o1()).astype(np.uint64), o1)
    assert np.array_equal(u32(ix.v2()), v2)


def test_build_index_full_uint32_range(hc):
    """Values across all 32 bits: eight 8-bit passes."""
    rng = np.random.default_rng(5)
    raw = rng.integers(0, 2**32, size=(200_000, 2), dtype=np.uint64).astype(np.uint32)
    raw[:10] = [[0xFFFFFFFF, 0xFFFFFFFF], [0, 0], [0xFFFFFFFF, 0], [0, 0xFFFFFFFF], [1, 2], [2, 1],
                [0x80000000, 0x7FFFFFFF], [0x7FFFFFFF, 0x80000000], [5, 5], [6, 6]]
    pairs = datagen.scatter_order(datagen.directed_set(raw), 3)
    pairs = np.concatenate([pairs, np.array([[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [9, 9]], dtype=np.uint32)])
    for ao in (0, 1):
        ix = hc.build_index(dev(pairs), ao)
        v1, o1, v2 = oracle.coco_build(pairs, ao)
        assert np.array_equal(u32(ix.v1()), v1)
        assert np.array_equal(u32(ix.o1()).astype(np.uint64), o1)
        assert np.array_equal(u32(ix.v2()), v2)


def test_build_index_single_key_value(hc):
    """All rows equal in both columns but distinct (no radix pass needed)."""
    pairs = np.array([[0, 0]], dtype=np.uint32)
    ix = hc.build_index(dev(pairs), 0)
    assert ix.l1 == 1 and u32(ix.o1()).tolist() == [0, 1] and u32(ix.v2()).tolist() == [0]


def test_build_index_empty(hc):
    import torch

    ix = hc.build_index(torch.zeros((0, 2), dtype=torch.int32, device="cuda"), 0)
    assert ix.n == 0 and ix.l1 == 0 and u32(ix.o1()).tolist() == [0]


def test_build_index_rejects_duplicates(hc):
    pairs = np.array([[1, 2], [3, 4], [1, 2]], dtype=np.uint32)
    with pytest.raises(hc.HoneycombError) as e:
        hc.build_index(dev(pairs), 0, check_duplicates=True)
    assert e.value.status == 6
    with pytest.raises(hc.HoneycombError) as e:
        hc.build_index(dev(pairs), 2)
    assert e.value.status == 1


# ------------------------------------------------------------------ partitioning

@pytest.mark.parametrize("shares", [(1, 1), (2, 3), (4, 4), (1, 16), (16, 1), (32, 32), (256, 256)])
def test_partition_matches_oracle(hc, shares):
    pa, pb = shares
    sym = datagen.rmat_graph(12, 8, 4)
    pairs = datagen.scatter_order(datagen.orient_lt(sym), 2)
    for ao in (0, 1):
        ix = hc.build_index(dev(pairs), ao)
        part = hc.partition_index(ix, 1234, pa, 987654, pb)
        ref = oracle.partition(pairs, ao, 1234, pa, 987654, pb)
        keys = part.keys().cpu().numpy().view(np.uint64)
        got_rt = np.stack([(keys >> np.uint64(32)).astype(np.uint32), (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)], 1)
        assert np.array_equal(got_rt, ref["rt"])
        assert np.array_equal(u32(part.bpref()).astype(np.uint64), ref["Bpref"])
        assert part.l1 == ref["V1"].shape[0]
        assert np.array_equal(u32(part.v1()), ref["V1"])
        assert np.array_equal(u32(part.o1()).astype(np.uint64), ref["O1"])
        assert np.array_equal(u32(part.v2()), ref["rt"][:, 1])
        assert np.array_equal(u32(part.lvl1_start()).astype(np.uint64), ref["lvl1_start"])


# ------------------------------------------------------------------ joins

QUERIES = ["TRIANGLE", "FOUR_CYCLE", "FOUR_DIAMOND", "FOUR_CLIQUE", "TWO_TRIANGLE"]


def _run(hc, q, rels, **kw):
    """Index each atom's relation in the attr order its loop order needs."""
    ixs = []
    cache = {}
    for j, r in enumerate(rels):
        ao = q.attr_order(j)
        key = (id(r), ao)
        if key not in cache:
            cache[key] = hc.build_index(dev(r), ao)
        ixs.append(cache[key])
    return hc.run_join(q, ixs, **kw)


@pytest.mark.parametrize("qname", QUERIES)
def test_counts_and_tuples_small_graphs(hc, qname):
    q = getattr(hc, qname)
    for seed in range(3):
        sym = datagen.random_graph(40 + 10 * seed, 0.2, seed)
        for rel in (sym, datagen.orient_lt(sym)):
            rels = [rel] * len(q.atoms)
            cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
            ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
            for mmin, mratio in ((0, 0), (1, 1 << 30), (0xFFFFFFFF, 1)):
                r = _run(hc, q, rels, mode="materialize", stats=True, merge_min=mmin, merge_ratio=mratio)
                assert r.count == cnt
                assert r.work == work
                assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref))


@pytest.mark.parametrize("qname", QUERIES)
def test_independent_random_relations(hc, qname):
    """Different relations per atom, directed, with empty sub-lists."""
    q = getattr(hc, qname)
    rng = np.random.default_rng(11)
    for case in range(4):
        rels = [datagen.directed_set(rng.integers(0, 30, size=(300, 2)).astype(np.uint32)) for _ in q.atoms]
        cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
        r = _run(hc, q, rels, mode="count", stats=True)
        assert r.count == cnt and r.work == work


@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_CLIQUE", "TWO_TRIANGLE"])
def test_share_invariance_and_cell_counts(hc, qname):
    """Sec. 5: cell outputs are disjoint and cover Q, whatever the shares."""
    q = getattr(hc, qname)
    sym = datagen.rmat_graph(9, 8, 21)
    rel = datagen.orient_lt(sym) if qname != "FOUR_CYCLE" else sym
    rels = [rel] * len(q.atoms)
    ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
    seeds = [17, 29, 31, 37, 41]
    rng = np.random.default_rng(1)
    share_sets = [[1] * q.n_vars, [4] + [1] * (q.n_vars - 1), [2] * q.n_vars]
    for _ in range(3):
        share_sets.append([int(2 ** rng.integers(0, 4)) for _ in range(q.n_vars)])
    for sh in share_sets:
        r = _run(hc, q, rels, shares=sh, seeds=seeds, mode="materialize", cell_counts=True)
        assert r.count == ref.shape[0], sh
        assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), sh
        cells = oracle.tuple_cells(ref, seeds[:q.n_vars], sh)
        want = np.bincount(cells, minlength=int(np.prod(sh))).astype(np.uint64)
        assert np.array_equal(r.cell_counts.cpu().numpy().view(np.uint64), want), sh


@pytest.mark.parametrize("order", list(itertools.permutations(range(4)))[::3])
def test_variable_orders_four_clique(hc, order):
    q = hc.FOUR_CLIQUE.with_order(order)
    sym = datagen.random_graph(36, 0.35, 4)
    rels = [sym] * 6
    cnt, _, _ = oracle.gj_count(4, list(q.atoms), rels, order=order)
    assert _run(hc, q, rels, shares=[2, 1, 2, 1]).count == cnt


@pytest.mark.parametrize("grain,threads", [(1, 32), (7, 64), (64, 128), (4096, 128), (32, 96)])
def test_launch_shapes_agree(hc, grain, threads):
    sym = datagen.rmat_graph(11, 8, 5)
    ep = datagen.orient_lt(sym)
    cnt, _, _ = oracle.gj_count(3, list(hc.TRIANGLE.atoms), [ep] * 3)
    r = _run(hc, hc.TRIANGLE, [ep] * 3, item_grain=grain, block_threads=threads, shares=[4, 2, 1])
    assert r.count == cnt
    # the last loop's two strategies give the same result: never merge, merge
    # whenever both lists are non-empty, and in between
    for mmin, mratio in ((0xFFFFFFFF, 1), (1, 1 << 30), (8, 2)):
        r = _run(hc, hc.TRIANGLE, [ep] * 3, item_grain=grain, block_threads=threads, merge_min=mmin,
                 merge_ratio=mratio, mode="materialize")
        assert r.count == cnt


@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_CLIQUE"])
def test_single_pass_materialize(hc, qname):
    """Pool output: enough room (one pass), and far too little (overflow, then
    the counted items place a second, deterministic pass)."""
    q = getattr(hc, qname)
    sym = datagen.rmat_graph(10, 8, 6)
    rel = datagen.orient_lt(sym) if qname != "FOUR_CYCLE" else sym
    rels = [rel] * len(q.atoms)
    ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
    for cap in (ref.shape[0] + 1, 10 ** 9, 1):
        for sh in ([1] * q.n_vars, [2] * q.n_vars):
            r = _run(hc, q, rels, mode="materialize", out_capacity=cap, shares=sh, cell_counts=True)
            assert r.count == ref.shape[0]
            assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), (cap, sh)
            assert int(r.cell_counts.sum()) == ref.shape[0]


@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_CLIQUE"])
def test_unary_atoms(hc, qname):
    """Unary atoms restrict variables to value sets (selections pushed into
    the query), with and without shares."""
    q = getattr(hc, qname)
    sym = datagen.rmat_graph(10, 8, 8)
    rel = datagen.orient_lt(sym) if qname != "FOUR_CYCLE" else sym
    rng = np.random.default_rng(3)
    for case in range(4):
        extra, rels = [], [rel] * len(q.atoms)
        nun = 1 if qname == "FOUR_CLIQUE" else 2
        for v in rng.choice(q.n_vars, size=nun, replace=False):
            vals = np.unique(rng.integers(0, 1024, size=300)).astype(np.uint32)
            extra.append(((int(v), -1), np.stack([vals, np.zeros_like(vals)], 1)))
        q2 = q.with_atoms([e[0] for e in extra])
        r2 = rels + [e[1] for e in extra]
        ref = oracle.gj_enumerate(q.n_vars, list(q2.atoms), r2)
        for sh in ([1] * q.n_vars, [2] * q.n_vars):
            r = _run(hc, q2, r2, shares=sh, mode="materialize")
            assert r.count == ref.shape[0]
            assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref))


def test_uniform_4096_vertices_32768_edges(hc):
    """The oracle-sized triangle workload: x<y<z over a uniform graph."""
    ep = datagen.uniform_graph(4096, 32768, seed=1)
    cnt, work, _ = oracle.gj_count(3, list(hc.TRIANGLE.atoms), [ep] * 3)
    r = _run(hc, hc.TRIANGLE, [ep] * 3, mode="materialize", stats=True)
    assert r.count == cnt and r.work == work
    ref = oracle.gj_enumerate(3, list(hc.TRIANGLE.atoms), [ep] * 3)
    assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref))


def test_empty_and_degenerate(hc):
    empty = np.zeros((0, 2), dtype=np.uint32)
    one = np.array([[0, 1]], dtype=np.uint32)
    assert _run(hc, hc.TRIANGLE, [empty, empty, empty]).count == 0
    assert _run(hc, hc.TRIANGLE, [one, empty, one]).count == 0
    assert _run(hc, hc.TRIANGLE, [one, one, one], shares=[2, 2, 2]).count == 0
    r = _run(hc, hc.TRIANGLE, [np.array([[0, 1]]), np.array([[1, 2]]), np.array([[0, 2]])], mode="materialize")
    assert r.count == 1 and u32(r.tuples).tolist() == [[0, 1, 2]]


def test_wrong_attr_order_rejected(hc):
    ep = datagen.orient_lt(datagen.random_graph(20, 0.3, 1))
    ix1 = hc.build_index(dev(ep), 1)
    with pytest.raises(hc.HoneycombError) as e:
        hc.run_join(hc.TRIANGLE, [ix1, ix1, ix1])
    assert e.value.status == 1


# ------------------------------------------------------------ query rewriting

@pytest.mark.parametrize("lift_arena", [0, 48, 1])
def test_query_rewriting_four_clique(hc, lift_arena):
    """Sec. 5.1: the last loop of the 4-clique (lists R3[y], R4[z], R6[x]) reads
    R3[y] n R6[x], computed once per y.  Same result as without rewriting, for
    the default arena, one that fits only some batches' lists and one that
    fits none (every batch falls back to the unrewritten loop)."""
    q = hc.FOUR_CLIQUE
    for seed in range(3):
        sym = datagen.random_graph(44 + 8 * seed, 0.32, 70 + seed)
        for rel in (sym, datagen.orient_lt(sym)):
            rels = [rel] * len(q.atoms)
            ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
            for mmin, mratio in ((0, 0), (1, 1 << 30), (0xFFFFFFFF, 1)):
                r = _run(hc, q, rels, lift_arena=lift_arena, merge_min=mmin, merge_ratio=mratio)
                assert r.count == ref.shape[0], (seed, mmin)
                r = _run(hc, q, rels, mode="materialize", lift_arena=lift_arena, merge_min=mmin, merge_ratio=mratio)
                assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), (seed, mmin)
                r = _run(hc, q, rels, mode="materialize", out_capacity=ref.shape[0] + 10, lift_arena=lift_arena,
                         merge_min=mmin, merge_ratio=mratio)
                assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), (seed, mmin)


@pytest.mark.parametrize("order", [(0, 1, 2, 3), (1, 0, 2, 3), (2, 3, 0, 1), (3, 1, 0, 2)])
def test_query_rewriting_orders_shares_and_relations(hc, order):
    """Different relations per atom (the lifted lists differ from the loop's
    own lists), loop orders and HyperCube shares."""
    q = hc.FOUR_CLIQUE.with_order(order)
    rng = np.random.default_rng(sum(order) + 5)
    rels = [datagen.directed_set(rng.integers(0, 40, size=(500, 2)).astype(np.uint32)) for _ in q.atoms]
    cnt, _, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels, order=order)
    for sh in ([1, 1, 1, 1], [2, 2, 1, 1], [1, 2, 2, 2]):
        assert _run(hc, q, rels, shares=sh).count == cnt, sh
        assert _run(hc, q, rels, shares=sh, lift=False).count == cnt, sh
        assert _run(hc, q, rels, shares=sh, lift_arena=24).count == cnt, sh


def test_query_rewriting_rmat_skew(hc):
    """Skewed R-MAT degrees (hub lists larger than the arena in some batches)."""
    q = hc.FOUR_CLIQUE
    ep = datagen.orient_lt(datagen.rmat_graph(11, 16, 12))
    rels = [ep] * len(q.atoms)
    cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
    for arena in (0, 256):
        assert _run(hc, q, rels, lift_arena=arena).count == cnt
    r = _run(hc, q, rels, stats=True)  # the work counter measures the unrewritten loops
    assert r.count == cnt and r.work == work


@pytest.mark.parametrize("n", [0, 1, 5, 4097, 100_000])
def test_build_unary_index_matches_build_index(hc, n):
    """The wait-free unary builder gives the index build_index makes of the
    pairs (value, 0)."""
    rng = np.random.default_rng(n + 3)
    vals = np.unique(rng.integers(0, 1 << 22, size=2 * n + 1).astype(np.uint32))[:n]
    import torch

    d = torch.from_numpy(vals.view(np.int32)).cuda()
    u = hc.build_unary_index(d, int(vals[-1]) if n else 0)
    pairs = np.stack([vals, np.zeros_like(vals)], axis=1)
    ref = hc.build_index(dev(pairs), 0)
    assert (u.n, u.l1, u.max_first, u.max_second) == (ref.n, ref.l1, ref.max_first, ref.max_second)
    if n:
        assert np.array_equal(u32(u.v1()), u32(ref.v1()))
        assert np.array_equal(u32(u.v2()), u32(ref.v2()))
        assert np.array_equal(u.keys().cpu().numpy(), ref.keys().cpu().numpy())
    assert np.array_equal(u32(u.o1()), u32(ref.o1()))
    # as a selection in a join
    sym = datagen.random_graph(60, 0.25, n % 7)
    sel = np.unique(rng.integers(0, 60, size=25).astype(np.uint32))
    q = hc.TRIANGLE.with_atoms([(0, -1)])
    cnt, _, _ = oracle.gj_count(3, list(q.atoms), [sym] * 3 + [np.stack([sel, np.zeros_like(sel)], 1)])
    us = hc.build_unary_index(torch.from_numpy(sel.view(np.int32)).cuda(), int(sel[-1]))
    ix = hc.build_index(dev(sym), 0)
    assert hc.run_join(q, [ix, ix, ix, us]).count == cnt


# ------------------------------------------- sparse 32-bit ids: no position maps

def _sparse_ids(n, seed):
    """An injective map of n vertex ids onto values spread over all 32 bits,
    holding 0, 0xFFFFFFFE and 0xFFFFFFFF, in a scrambled order."""
    rng = np.random.default_rng(seed)
    ids = np.unique(rng.integers(1, 0xFFFFFFFE, size=2 * n + 8, dtype=np.uint64).astype(np.uint32))
    ids = ids[rng.permutation(ids.shape[0])][: n - 3]
    ids = np.concatenate([ids, np.array([0, 0xFFFFFFFE, 0xFFFFFFFF], dtype=np.uint32)])
    return ids[rng.permutation(n)]


@pytest.mark.parametrize("qname", QUERIES)
def test_sparse_ids_without_position_maps(hc, qname):
    """Relations whose values spread over 32 bits (0 and 0xFFFFFFFF included)
    get no V1 position map, so every top-level search is a binary search of
    V1 (whole, or a partition's range).  Counts, work counters and sorted
    tuples equal the oracle's on the same relations, at one share and mixed
    shares, in both output modes."""
    q = getattr(hc, qname)
    sym0 = datagen.rmat_graph(9, 8, 41)
    ids = _sparse_ids(int(sym0.max()) + 1, 5)
    sym = sorted_rows(ids[sym0])
    rel = sym if qname == "FOUR_CYCLE" else np.ascontiguousarray(sym[sym[:, 0] < sym[:, 1]])
    rels = [rel] * len(q.atoms)
    for ao in (0, 1):
        assert hc.build_index(dev(rel), ao).v1pos_n == 0
    cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
    ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
    assert cnt > 0
    r = _run(hc, q, rels, stats=True)
    assert r.count == cnt and r.work == work
    rng = np.random.default_rng(len(qname))
    for sh in ([1] * q.n_vars, [2] * q.n_vars, [4] + [1] * (q.n_vars - 1),
               [int(2 ** rng.integers(0, 3)) for _ in range(q.n_vars)]):
        assert _run(hc, q, rels, shares=sh).count == cnt, sh
        for cap in (0, cnt + 1):
            r = _run(hc, q, rels, shares=sh, mode="materialize", out_capacity=cap)
            assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), (sh, cap)


def test_sparse_ids_top_level_searches(hc):
    """Loops that search a whole top level: the 4-cycle's R1[x] n R3.V1 at
    loop y over a relation of 20,000 sparse values (a multi-step binary search
    of V1), against the oracle, with and without shares on y."""
    rng = np.random.default_rng(8)
    ids = _sparse_ids(20_000, 9)
    rels = [datagen.directed_set(ids[rng.integers(0, 20_000, size=(60_000, 2))]) for _ in range(4)]
    q = hc.FOUR_CYCLE
    cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
    r = _run(hc, q, rels, stats=True)
    assert r.count == cnt and r.work == work
    for sh in ([1, 4, 1, 1], [1, 2, 2, 1], [2, 1, 1, 4]):
        assert _run(hc, q, rels, shares=sh).count == cnt, sh


# ------------------------------------------------------- hub slicing sweep

@pytest.mark.parametrize("qname", ["FOUR_CLIQUE", "FOUR_CYCLE"])
def test_slice_grain_sweep_skewed(hc, qname):
    """Deep queries cut the work of an entry whose loop-3 lists are long into
    slices of about slice_grain candidates.  On a skewed R-MAT graph every
    grain (1, 7, the default 256, and no slicing) gives the oracle's count and
    work counter (one share) and its tuples; shares keep the count."""
    q = getattr(hc, qname)
    sym = datagen.rmat_graph(10, 16, 13)
    rel = sym if qname == "FOUR_CYCLE" else datagen.orient_lt(sym)
    rels = [rel] * len(q.atoms)
    cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
    ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels) if cnt < 3_000_000 else None
    for sg in (1, 7, 0, 0xFFFFFFFF):
        r = _run(hc, q, rels, slice_grain=sg, stats=True)
        assert r.count == cnt and r.work == work, sg
        assert _run(hc, q, rels, slice_grain=sg).count == cnt, sg
        for sh in ([4, 1, 1, 1], [2, 2, 1, 2]):
            assert _run(hc, q, rels, slice_grain=sg, shares=sh).count == cnt, (sg, sh)
        if ref is not None and sg in (1, 7):
            r = _run(hc, q, rels, slice_grain=sg, mode="materialize", out_capacity=cnt + 1)
            assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), sg


# ------------------------------------------------------- bucket directories

@pytest.mark.parametrize("scramble", [True, False])
@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_CLIQUE", "TWO_TRIANGLE"])
def test_directory_thresholds(hc, qname, scramble):
    """List searches through the runs' bucket directories (runs of at least
    dir_min values) give exactly the plain binary search's results: every
    threshold, and none, on R-MAT graphs with scrambled ids (values spread
    evenly over each run's range) and unscrambled ones (hubs on low ids,
    values bunched), with and without shares and position maps."""
    q = getattr(hc, qname)
    sym = datagen.rmat_graph(11, 16, 23, scramble=scramble)
    rel = sym if qname == "FOUR_CYCLE" else datagen.orient_lt(sym)
    if qname == "FOUR_CYCLE":
        rel = rel[: rel.shape[0] // 3]  # keep the oracle's closed walks few enough
        rel = np.ascontiguousarray(rel)
    rels = [rel] * len(q.atoms)
    cnt, work, _ = oracle.gj_count(q.n_vars, list(q.atoms), rels)
    # pair_min: last-loop bindings searched by the whole warp (1: all, the
    # default 32, 0xFFFFFFFF: none, every binding's values flattened)
    for dmin, pmin in ((0, 0), (17, 1), (100, 0xFFFFFFFF), (0xFFFFFFFF, 0), (0xFFFFFFFF, 0xFFFFFFFF)):
        r = _run(hc, q, rels, dir_min=dmin, pair_min=pmin, stats=True)
        assert r.count == cnt and r.work == work, (dmin, pmin)
        assert _run(hc, q, rels, dir_min=dmin, pair_min=pmin).count == cnt, (dmin, pmin)
        for sh in ([2] * q.n_vars, [1, 4] + [1] * (q.n_vars - 2)):
            assert _run(hc, q, rels, dir_min=dmin, pair_min=pmin, shares=sh).count == cnt, (dmin, pmin, sh)
    if cnt < 2_000_000:
        ref = oracle.gj_enumerate(q.n_vars, list(q.atoms), rels)
        for dmin, pmin in ((0, 0), (0, 1), (0xFFFFFFFF, 0xFFFFFFFF)):
            for cap in (0, cnt + 1):
                r = _run(hc, q, rels, dir_min=dmin, pair_min=pmin, mode="materialize", shares=[2] * q.n_vars,
                         out_capacity=cap, merge_min=0xFFFFFFFF)
                assert np.array_equal(sorted_rows(u32(r.tuples)), sorted_rows(ref)), (dmin, pmin, cap)
