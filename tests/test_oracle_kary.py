"""Pins of the k-ary CPU oracle (oracle_kary.c) to facts other than itself.

The queries are the paper's hypergraph queries over ternary relations
(Table "Queries": LW, Loomis-Whitney; CT, Clover-Triangle) plus mixed
arities.  Checks: brute force over every tuple of a tiny domain, closed
forms on full cubes and on relations with prescribed first-attribute sets
(the shapes of Sec. 6's ST-Dense tensors), agreement with the separately
written binary Generic Join oracle on graphs, and the paper's invariant that
the loop order changes the work but not the result (Sec. 5).
"""
import itertools
import os

import numpy as np
import pytest

import datagen
import oracle

# Q(X,Y,Z,U) := R1(X,Y,Z), R2(X,Y,U), R3(X,Z,U), R4(Y,Z,U)   with X=0 Y=1 Z=2 U=3
LW = (4, [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)])
# Q(U,X,Y,Z) := R5(U,X,Y), R6(U,X,Z), R7(U,Y,Z)              with U=0 X=1 Y=2 Z=3
CT = (4, [(0, 1, 2), (0, 1, 3), (0, 2, 3)])


def brute(n_vars, atoms, rels, dom):
    """Every assignment of the variables over range(dom), kept when each
    atom's projection is one of its relation's rows."""
    sets = [set(map(tuple, np.asarray(r, dtype=np.int64).reshape(-1, len(a)).tolist())) for a, r in zip(atoms, rels)]
    out = []
    for t in itertools.product(range(dom), repeat=n_vars):
        if all(tuple(t[v] for v in a) in s for a, s in zip(atoms, sets)):
            out.append(t)
    return np.array(out, dtype=np.uint32).reshape(-1, n_vars)


def random_rel(rng, k, dom, density):
    full = np.array(list(itertools.product(range(dom), repeat=k)), dtype=np.uint32).reshape(-1, k)
    keep = rng.random(full.shape[0]) < density
    return full[keep]


def sorted_rows(a):
    a = np.asarray(a)
    return a if a.shape[0] == 0 else a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("name,query", [("LW", LW), ("CT", CT)])
@pytest.mark.parametrize("seed", range(6))
def test_brute_force_hypergraph(name, query, seed):
    nv, atoms = query
    rng = np.random.default_rng(seed)
    dom = 5
    rels = [random_rel(rng, 3, dom, rng.choice([0.3, 0.6, 0.9])) for _ in atoms]
    want = brute(nv, atoms, rels, dom)
    cnt, got = oracle.kgj(nv, atoms, rels, tuples=True)
    assert cnt == want.shape[0]
    assert np.array_equal(sorted_rows(got), sorted_rows(want))


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_mixed_arity(seed):
    """Atoms of arity 1, 2 and 3 together, columns listing variables out of
    their id order (a transposed column mapping fails here)."""
    rng = np.random.default_rng(100 + seed)
    dom = 5
    nv = 5
    atoms = [(2, 0, 4), (3, 1), (4,), (1, 2, 0), (3, 4)]
    rels = [random_rel(rng, len(a), dom, rng.choice([0.4, 0.7, 0.95])) for a in atoms]
    want = brute(nv, atoms, rels, dom)
    cnt, got = oracle.kgj(nv, atoms, rels, tuples=True)
    assert cnt == want.shape[0]
    assert np.array_equal(sorted_rows(got), sorted_rows(want))


def test_asymmetric_columns_are_not_swapped():
    """R(X,Y,Z) = {(0,1,2)} joined with unary atoms on each variable: exactly
    one output, and it is (0,1,2) in variable-id order, not a permutation."""
    atoms = [(0, 1, 2), (0,), (1,), (2,)]
    rels = [np.array([[0, 1, 2]]), np.array([[0]]), np.array([[1]]), np.array([[2]])]
    for order in itertools.permutations(range(3)):
        cnt, got = oracle.kgj(3, atoms, rels, order=order, tuples=True)
        assert cnt == 1 and got.tolist() == [[0, 1, 2]]
    rels[1] = np.array([[1]])  # X must be 0 in R: no output
    assert oracle.kgj(3, atoms, rels) == 0


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_lw_on_full_cubes(n):
    """Every relation [n]^3: every assignment of (X,Y,Z,U) survives, n^4."""
    cube = datagen.full_cube(n)
    assert cube.shape == (n ** 3, 3)
    assert oracle.kgj(*LW, [cube] * 4) == n ** 4


@pytest.mark.parametrize("s,m", [(1, 4), (2, 6), (3, 5)])
def test_ct_common_first_attribute(s, m):
    """R5, R6, R7 = S x [m] x [m] with the same S: U ranges over S and X, Y,
    Z over [m] freely, |S| m^3."""
    first = np.arange(10, 10 + s, dtype=np.uint32)
    rels = [datagen.prefixed_square(first, m)] * 3
    assert oracle.kgj(*CT, rels) == s * m ** 3


def test_ct_on_st_dense_first_attribute_sets():
    """Sec. 6's last three ST-Dense relations take their first attribute from
    {0,1}, {0,2} and {1,2}.  CT joins all three on that attribute, and the
    three sets have no common value, so the count is 0; widening the middle
    set to {0,1,2} leaves U = 1 and m^3 results."""
    m = 6
    sets = [np.array([0, 1]), np.array([0, 2]), np.array([1, 2])]
    rels = [datagen.prefixed_square(s.astype(np.uint32), m) for s in sets]
    assert oracle.kgj(*CT, rels) == 0
    rels[1] = datagen.prefixed_square(np.array([0, 1, 2], dtype=np.uint32), m)
    assert oracle.kgj(*CT, rels) == m ** 3


def test_st_dense_generator_shapes():
    rels = datagen.st_dense(n=8, m=16)
    assert len(rels) == 7
    for r in rels[:4]:
        assert r.shape == (8 ** 3, 3) and r.dtype == np.uint32
    for r, s in zip(rels[4:], ({0, 1}, {0, 2}, {1, 2})):
        assert r.shape == (2 * 16 * 16, 3)
        assert set(np.unique(r[:, 0]).tolist()) == s
    # [N] is the positive integers up to N, stored as 0 .. N-1
    assert int(rels[0].max()) == 7 and int(rels[4][:, 1:].max()) == 15


def test_st_sparse_generator():
    rels = datagen.st_sparse(n=6, domain=60, m=8, m_domain=80, seed=3)
    assert len(rels) == 7
    for r in rels[:4]:
        assert r.shape == (6 ** 3, 3)
        assert np.unique(r, axis=0).shape[0] == r.shape[0]  # a set
        assert int(r.max()) < 60
    for r, s in zip(rels[4:], ({0, 1}, {0, 2}, {1, 2})):
        assert r.shape == (2 * 8 * 8, 3)
        assert np.unique(r, axis=0).shape[0] == r.shape[0]
        assert set(np.unique(r[:, 0]).tolist()) == s
        for f in s:  # m^2 pairs under each first value
            assert int((r[:, 0] == f).sum()) == 8 * 8
        assert int(r[:, 1:].max()) < 80
    again = datagen.st_sparse(n=6, domain=60, m=8, m_domain=80, seed=3)
    assert all(np.array_equal(a, b) for a, b in zip(rels, again))


@pytest.mark.parametrize("q", ["TRIANGLE", "FOUR_CYCLE", "FOUR_CLIQUE", "TWO_TRIANGLE"])
def test_binary_atoms_match_binary_oracle(q):
    nv, atoms = getattr(oracle, q)
    sym = datagen.random_graph(40, 0.25, 5)
    ep = datagen.orient_lt(sym)
    for rel in (sym, ep):
        want, _, _ = oracle.gj_count(nv, atoms, [rel] * len(atoms))
        assert oracle.kgj(nv, atoms, [rel] * len(atoms)) == want


@pytest.mark.parametrize("name,query", [("LW", LW), ("CT", CT)])
def test_order_invariance(name, query):
    nv, atoms = query
    rng = np.random.default_rng(77)
    rels = [random_rel(rng, 3, 6, 0.5) for _ in atoms]
    ref = None
    for order in itertools.permutations(range(nv)):
        cnt, got = oracle.kgj(nv, atoms, rels, order=order, tuples=True)
        got = sorted_rows(got)
        if ref is None:
            ref = got
        assert cnt == ref.shape[0] and np.array_equal(got, ref), order


def test_empty_relation_and_cap():
    nv, atoms = LW
    cube = datagen.full_cube(3)
    assert oracle.kgj(nv, atoms, [cube, cube, cube, cube[:0]]) == 0
    with pytest.raises(oracle.OracleError):
        oracle.kgj(nv, atoms, [cube] * 4, tuples=True, cap=10)  # 81 > cap


def test_bad_arguments():
    cube = datagen.full_cube(2)
    with pytest.raises(oracle.OracleError):
        oracle.kgj(3, [(0, 0, 1)], [cube])  # a variable twice in one atom
    with pytest.raises(oracle.OracleError):
        oracle.kgj(4, [(0, 1, 2)], [cube])  # U in no atom
    with pytest.raises(oracle.OracleError):
        oracle.kgj(3, [(0, 1, 2)], [cube], order=[0, 0, 1])


# ---------------------------------------------------------------- k-level CoCo

def trie_levels(rows, cols):
    """The k-level trie written out by hand: prefixes of each length as a
    Python set, sorted; a prefix's first child is the first longer prefix
    that extends it."""
    t = sorted(set(tuple(int(r[c]) for c in cols) for r in np.asarray(rows).tolist()))
    k = len(cols)
    prefixes = [sorted(set(p[:d + 1] for p in t)) for d in range(k)]
    V = [[p[d] for p in prefixes[d]] for d in range(k)]
    O = []
    for d in range(k - 1):
        nxt = prefixes[d + 1]
        o = [next(i for i, q in enumerate(nxt) if q[:d + 1] == p) for p in prefixes[d]]
        O.append(o + [len(nxt)])
    return V, O


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_kcoco_matches_hand_trie(k, seed):
    rng = np.random.default_rng(300 + seed)
    rel = random_rel(rng, k, 4 if k == 3 else 7, 0.5)
    for cols in itertools.permutations(range(k)):
        c = oracle.kcoco(rel, cols)
        V, O = trie_levels(rel, cols)
        assert [v.tolist() for v in c["V"]] == V
        assert [o.tolist() for o in c["O"]] == O


def test_kcoco_binary_matches_coco_build():
    """Arity 2 is the binary CoCo of Sec. 4, built by the separately written
    oracle.c; both attribute orders."""
    rel = datagen.random_graph(60, 0.2, 11)
    for ao in (0, 1):
        v1, o1, v2 = oracle.coco_build(rel, ao)
        c = oracle.kcoco(rel, (0, 1) if ao == 0 else (1, 0))
        assert np.array_equal(c["V"][0], v1) and np.array_equal(c["V"][1], v2)
        assert np.array_equal(c["O"][0].astype(np.uint64), o1)


def test_kcoco_rebuilds_rows_and_empty():
    rng = np.random.default_rng(5)
    rel = random_rel(rng, 3, 6, 0.3)
    c = oracle.kcoco(rel, (2, 0, 1))
    V, O = c["V"], c["O"]
    rows = []
    for a in range(V[0].shape[0]):
        for b in range(O[0][a], O[0][a + 1]):
            for e in range(O[1][b], O[1][b + 1]):
                rows.append((V[0][a], V[1][b], V[2][e]))
    want = sorted(tuple(int(r[c]) for c in (2, 0, 1)) for r in rel.tolist())
    assert [tuple(map(int, r)) for r in rows] == want
    e = oracle.kcoco(np.zeros((0, 3), dtype=np.uint32))
    assert [v.shape[0] for v in e["V"]] == [0, 0, 0] and [o.tolist() for o in e["O"]] == [[0], [0]]


# ------------------------------------------------------------------ work measure

def brute_work(n_vars, atoms, rels, order, dom):
    """Sum over loops i and bindings t of loops 0..i-1 (tuples of the prefix
    query: every atom's bound variables, a prefix of its loop-ordered
    columns, project to some row) of (lists at loop i) * (shortest list),
    a list being the set of values of X_order[i] in the atom's rows that
    agree with t."""
    rank = {v: i for i, v in enumerate(order)}
    sets = [set(map(tuple, np.asarray(r, dtype=np.int64).reshape(-1, len(a)).tolist())) for a, r in zip(atoms, rels)]
    total = 0
    for i in range(n_vars):
        bound = order[:i]
        x = order[i]
        for t in itertools.product(range(dom), repeat=i):
            val = dict(zip(bound, t))
            ok = True
            for a, s in zip(atoms, sets):
                idx = [c for c in range(len(a)) if rank[a[c]] < i]
                if idx and not any(all(row[c] == val[a[c]] for c in idx) for row in s):
                    ok = False
                    break
            if not ok:
                continue
            lens = []
            for a, s in zip(atoms, sets):
                if x not in a:
                    continue
                cx = a.index(x)
                idx = [c for c in range(len(a)) if rank[a[c]] < i]
                lens.append(len({row[cx] for row in s if all(row[c] == val[a[c]] for c in idx)}))
            total += len(lens) * min(lens)
    return total


@pytest.mark.parametrize("name,query", [("LW", LW), ("CT", CT), ("mixed", (4, [(2, 0, 3), (1, 2), (3,), (1, 0)]))])
@pytest.mark.parametrize("seed", range(3))
def test_work_measure_brute_force(name, query, seed):
    nv, atoms = query
    rng = np.random.default_rng(900 + seed)
    dom = 4
    rels = [random_rel(rng, len(a), dom, rng.choice([0.4, 0.8])) for a in atoms]
    for order in ((0, 1, 2, 3), (3, 1, 0, 2)):
        cnt, work = oracle.kgj(nv, atoms, rels, order=order, work=True)
        assert work == brute_work(nv, atoms, rels, order, dom), order


def test_st_sparse_device_dedup_matches_host():
    """The torch de-duplication path (run here on the CPU device) keeps the
    same keys as the numpy one."""
    a = datagen.st_sparse(n=9, domain=30, m=10, m_domain=25, seed=6)
    b = datagen.st_sparse(n=9, domain=30, m=10, m_domain=25, seed=6, device="cpu")
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("name,query", [("LW", LW), ("CT", CT), ("mixed", (5, [(2, 0, 4), (3, 1), (4,), (1, 2, 0), (3, 4)]))])
def test_threaded_count_equals_sequential(name, query):
    nv, atoms = query
    rng = np.random.default_rng(31)
    rels = [random_rel(rng, len(a), 7, 0.5) for a in atoms]
    for order in (None, tuple(reversed(range(nv)))):
        want = oracle.kgj(nv, atoms, rels, order=order, work=True)
        for t in (2, 3, 8, 64, 100):
            assert oracle.kgj(nv, atoms, rels, order=order, work=True, nthreads=t) == want, (order, t)


# ------------------------------------------------------------- partitioning

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = [s.strip() for s in line.split("=", 1)]
            out[k] = [[int(t) for t in r.split()] for r in v.split(";")]
    return out


def test_kpartition_worked_example():
    """Sec. 4, Example "partition" on a ternary R(X,Y,Z) with shares 2x2x1:
    partition (0,1,0) holds (0,4,1), (5,3,9), has B = 2 and starts at
    B^pref = 3; partition (1,0,0) is empty."""
    g = _golden("kpartition_example.txt")
    px, py, pz = g["shares_xyz"][0]
    grey = tuple(g["grey_partition"][0])
    grey_tuples = [tuple(t) for t in g["grey_tuples"]]
    sx = next(s for s in range(1, 100000) if all(oracle.share(t[0], s, px) == grey[0] for t in grey_tuples))
    sy = next(s for s in range(1, 100000) if all(oracle.share(v, s, py) == 1 for v in g["hY_one"][0]))
    hx = lambda v: oracle.share(v, sx, px)
    hy = lambda v: oracle.share(v, sy, py)
    xs0 = [v for v in range(10, 400) if hx(v) == 0][:3]
    xs1 = [v for v in range(10, 400) if hx(v) == 1][:2]
    ys0 = [v for v in range(10, 400) if hy(v) == 0][:3]
    rel = [(xs0[i], ys0[i], 7 + i) for i in range(3)]   # 3 rows in (0,0,0)
    rel += grey_tuples                                     # (0,1,0)
    rel += [(xs1[0], 1, 2), (xs1[1], 4, 6)]                # (1,1,0); (1,0,0) left empty
    part = oracle.kpartition(np.array(rel, dtype=np.uint32), (sx, sy, 77), (px, py, pz))
    pid = (grey[0] * py + grey[1]) * pz + grey[2]
    e = g["empty_partition"][0]
    assert int(part["B"][pid]) == g["B_grey"][0][0]
    assert int(part["Bpref"][pid]) == g["Bpref_grey"][0][0]
    assert int(part["B"][(e[0] * py + e[1]) * pz + e[2]]) == 0
    lo, hi = int(part["Bpref"][pid]), int(part["Bpref"][pid + 1])
    assert sorted(map(tuple, part["rt"][lo:hi].tolist())) == sorted(grey_tuples)


def _expand(V, O, lo, hi):
    """Rows of the trie whose level-0 entries are [lo, hi), in level order."""
    k = len(V)
    rows = []

    def walk(d, e, prefix):
        t = prefix + (int(V[d][e]),)
        if d == k - 1:
            rows.append(t)
            return
        for c in range(int(O[d][e]), int(O[d][e + 1])):
            walk(d + 1, c, t)

    for e in range(lo, hi):
        walk(0, e, ())
    return rows


@pytest.mark.parametrize("k,shares", [(1, (4,)), (2, (3, 2)), (3, (2, 2, 1)), (3, (1, 3, 2)), (3, (4, 1, 1)),
                                      (3, (1, 1, 1))])
@pytest.mark.parametrize("seed", range(3))
def test_kpartition_definition(k, shares, seed):
    """R~ is the input reordered (no replication); B^pref is B's exclusive
    prefix; every row of segment p has partition identifiers whose mixed
    radix (column 0 most significant) is p; the levels of partition p,
    walked from its level-0 range, give back exactly its rows in level
    order."""
    rng = np.random.default_rng(40 + seed)
    rel = random_rel(rng, k, {1: 60, 2: 12, 3: 6}[k], 0.4)
    seeds = [int(x) for x in rng.integers(1, 1 << 31, size=k)]
    for cols in itertools.permutations(range(k)):
        part = oracle.kpartition(rel, seeds, shares, cols)
        n = rel.shape[0]
        rt = part["rt"]
        assert np.array_equal(sorted_rows(rt), sorted_rows(rel))
        pref = part["Bpref"].astype(np.int64)
        assert pref[0] == 0 and pref[-1] == n and np.array_equal(np.diff(pref), part["B"].astype(np.int64))
        l0 = part["l0start"].astype(np.int64)
        assert l0[0] == 0 and l0[-1] == part["V"][0].shape[0] and np.all(np.diff(l0) >= 0)
        assert part["V"][k - 1].shape[0] == n
        for p in range(int(np.prod(shares))):
            seg = rt[pref[p]:pref[p + 1]]
            for row in seg.tolist():
                ids = [oracle.share(row[c], seeds[c], shares[c]) for c in range(k)]
                pid = 0
                for c in range(k):
                    pid = pid * shares[c] + ids[c]
                assert pid == p
            got = _expand(part["V"], part["O"], int(l0[p]), int(l0[p + 1]))
            want = sorted(tuple(int(r[c]) for c in cols) for r in seg.tolist())
            assert got == want, (cols, p)


@pytest.mark.parametrize("vshares", [(2, 2, 1, 2), (3, 1, 2, 1), (1, 1, 1, 1), (2, 3, 2, 2)])
def test_kpartition_cells_partition_the_join(vshares):
    """Sec. 4-5: cell (c_X, c_Y, c_Z, c_U) joins, for each atom, the
    partition its variables' coordinates select; the cells' outputs are
    disjoint and cover the query's result, so the per-cell counts add up to
    the unpartitioned count and each cell's tuples hash to that cell."""
    nv, atoms = LW
    rng = np.random.default_rng(77)
    rels = [random_rel(rng, 3, 7, 0.55) for _ in atoms]
    vseeds = [11, 22, 33, 44]
    parts = [oracle.kpartition(r, [vseeds[v] for v in a], [vshares[v] for v in a]) for a, r in zip(atoms, rels)]
    total = oracle.kgj(nv, atoms, rels)
    acc = 0
    for cell in itertools.product(*[range(s) for s in vshares]):
        sub = []
        for a, pt in zip(atoms, parts):
            pid = 0
            for v in a:
                pid = pid * vshares[v] + cell[v]
            lo, hi = int(pt["Bpref"][pid]), int(pt["Bpref"][pid + 1])
            sub.append(pt["rt"][lo:hi])
        cnt, tup = oracle.kgj(nv, atoms, sub, tuples=True)
        acc += cnt
        if cnt:
            cid = 0
            for v in range(nv):
                cid = cid * vshares[v] + cell[v]
            assert np.all(oracle.tuple_cells(tup, vseeds, vshares) == cid)
    assert acc == total
