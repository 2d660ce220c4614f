"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each check is independent of the oracle's Generic Join code: brute force
over all tuples of the domain, closed forms on complete and complete
bipartite graphs, trace identities computed by integer matrix products,
clique enumeration by networkx, invariants the paper states (order and share
independence), and the paper's worked examples (tests/golden).
"""
import itertools
import math
import os

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
QUERIES = {
    "triangle": oracle.TRIANGLE,
    "four_cycle": oracle.FOUR_CYCLE,
    "four_diamond": oracle.FOUR_DIAMOND,
    "four_clique": oracle.FOUR_CLIQUE,
    "two_triangle": oracle.TWO_TRIANGLE,
}


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = [s.strip() for s in line.split("=", 1)]
            rows = [[int(t) for t in r.split()] for r in v.split(";")]
            out[k] = rows
    return out


def _adj(pairs, nv):
    a = np.zeros((nv, nv), dtype=np.int64)
    if len(pairs):
        a[pairs[:, 0], pairs[:, 1]] = 1
    return a


def brute_force(n_vars, atoms, rels, dom):
    """All tuples of dom^n_vars satisfying every atom (indicator product)."""
    t = np.ones((dom,) * n_vars, dtype=bool)
    for (v0, v1), r in zip(atoms, rels):
        if v1 < 0:  # unary atom: the set of column-0 values
            u = np.zeros(dom, dtype=bool)
            if len(r):
                u[r[:, 0]] = True
            shape = [1] * n_vars
            shape[v0] = dom
            t &= u.reshape(shape)
            continue
        a = np.zeros((dom, dom), dtype=bool)
        if len(r):
            a[r[:, 0], r[:, 1]] = True
        shape = [1] * n_vars
        shape[v0] = dom
        shape[v1] = dom
        if v0 < v1:
            t &= a.reshape(shape)
        else:
            t &= a.T.reshape(shape)
    return np.argwhere(t).astype(np.uint32)


def _sorted_rows(a):
    a = np.asarray(a)
    if a.shape[0] == 0:
        return a
    return a[np.lexsort(a.T[::-1])]


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 8, 13, 24, 40])
def test_complete_graph_closed_forms(n):
    sym = datagen.complete_graph(n)
    ep = datagen.orient_lt(sym)
    c = lambda q, r: oracle.gj_count(*q, [r] * len(q[1]))[0]
    assert c(oracle.TRIANGLE, ep) == math.comb(n, 3)
    assert c(oracle.TRIANGLE, sym) == n * (n - 1) * (n - 2)
    if n <= 24:
        assert c(oracle.FOUR_CLIQUE, ep) == math.comb(n, 4)
        assert c(oracle.FOUR_CLIQUE, sym) == n * (n - 1) * (n - 2) * (n - 3)
        assert c(oracle.FOUR_CYCLE, sym) == (n - 1) ** 4 + (n - 1)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 3), (4, 4), (5, 9), (12, 7)])
def test_complete_bipartite_closed_forms(m, n):
    sym = datagen.complete_bipartite(m, n)
    ep = datagen.orient_lt(sym)
    assert oracle.gj_count(*oracle.TRIANGLE, [ep] * 3)[0] == 0
    assert oracle.gj_count(*oracle.TRIANGLE, [sym] * 3)[0] == 0
    assert oracle.gj_count(*oracle.FOUR_CLIQUE, [ep] * 6)[0] == 0
    assert oracle.gj_count(*oracle.FOUR_CYCLE, [sym] * 4)[0] == 2 * (m * n) ** 2


@pytest.mark.parametrize("seed", range(6))
def test_trace_identities(seed):
    n = 40 + 7 * seed
    sym = datagen.random_graph(n, 0.15 + 0.05 * seed, seed)
    a = _adj(sym, n)
    a3 = a @ a @ a
    a4 = a3 @ a
    ep = datagen.orient_lt(sym)
    assert oracle.gj_count(*oracle.TRIANGLE, [ep] * 3)[0] == np.trace(a3) // 6
    assert oracle.gj_count(*oracle.TRIANGLE, [sym] * 3)[0] == np.trace(a3)
    assert oracle.gj_count(*oracle.FOUR_CYCLE, [sym] * 4)[0] == np.trace(a4)


@pytest.mark.parametrize("seed", range(4))
def test_cliques_against_networkx(seed):
    nx = pytest.importorskip("networkx")
    n = 30 + 5 * seed
    sym = datagen.random_graph(n, 0.3, 100 + seed)
    g = nx.Graph()
    g.add_nodes_from(range(n))
    g.add_edges_from(datagen.orient_lt(sym).tolist())
    sizes = [len(c) for c in nx.enumerate_all_cliques(g)]
    ep = datagen.orient_lt(sym)
    assert oracle.gj_count(*oracle.TRIANGLE, [ep] * 3)[0] == sizes.count(3)
    assert oracle.gj_count(*oracle.FOUR_CLIQUE, [ep] * 6)[0] == sizes.count(4)


def test_uniform_config_against_networkx():
    """The 4,096-vertex / 32,768-edge uniform graph: x<y<z triangles."""
    nx = pytest.importorskip("networkx")
    ep = datagen.uniform_graph(4096, 32768, seed=1)
    assert ep.shape == (32768, 2) and np.all(ep[:, 0] < ep[:, 1])
    g = nx.Graph()
    g.add_edges_from(ep.tolist())
    expect = sum(nx.triangles(g).values()) // 3
    assert oracle.gj_count(*oracle.TRIANGLE, [ep] * 3)[0] == expect


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("name", list(QUERIES))
def test_brute_force_random_relations(name):
    """200 seeded cases of independent random relations per atom."""
    n_vars, atoms = QUERIES[name]
    rng = np.random.default_rng(7 + len(name))
    dom = 6 if n_vars == 5 else 7
    for case in range(200 // len(QUERIES) + 1):
        rels = []
        for _ in atoms:
            p = rng.uniform(0.1, 0.9)
            m = rng.random((dom, dom)) < p
            rels.append(np.argwhere(m).astype(np.uint32))
        expect = brute_force(n_vars, atoms, rels, dom)
        cnt, _, _ = oracle.gj_count(n_vars, atoms, rels)
        assert cnt == expect.shape[0], (name, case)
        got = oracle.gj_enumerate(n_vars, atoms, rels)
        assert np.array_equal(_sorted_rows(got), _sorted_rows(expect)), (name, case)


SPARSE_IDS = np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0xDEADBEEF, 0xFFFFFFFD, 0xFFFFFFFE, 0xFFFFFFFF],
                      dtype=np.uint32)


@pytest.mark.parametrize("name", list(QUERIES))
def test_brute_force_sparse_32bit_ids(name):
    """Values spread over all 32 bits, including 0, 0xFFFFFFFE and 0xFFFFFFFF:
    relations over a small domain are relabelled by an injective map onto
    such ids (monotone, and in a scrambled order); the oracle's result on the
    relabelled relations is the brute-force result on the small domain,
    relabelled the same way."""
    n_vars, atoms = QUERIES[name]
    rng = np.random.default_rng(31 + len(name))
    dom = 6 if n_vars == 5 else 8
    for case in range(12):
        rels = [np.argwhere(rng.random((dom, dom)) < rng.uniform(0.2, 0.8)).astype(np.uint32) for _ in atoms]
        expect = brute_force(n_vars, atoms, rels, dom)
        ids = SPARSE_IDS[:dom] if case % 2 == 0 else rng.permutation(SPARSE_IDS)[:dom]
        mapped = [ids[r] for r in rels]
        cnt, _, _ = oracle.gj_count(n_vars, atoms, mapped)
        assert cnt == expect.shape[0], (name, case)
        got = oracle.gj_enumerate(n_vars, atoms, mapped)
        assert np.array_equal(_sorted_rows(got), _sorted_rows(ids[expect])), (name, case)


@pytest.mark.parametrize("name", ["triangle", "four_cycle", "four_clique"])
def test_brute_force_with_unary_atoms(name):
    """Unary atoms F(X_v) restrict a variable to a set of values."""
    n_vars, atoms = QUERIES[name]
    rng = np.random.default_rng(17)
    dom = 7
    for case in range(20):
        rels = [np.argwhere(rng.random((dom, dom)) < 0.6).astype(np.uint32) for _ in atoms]
        extra = []
        for v in rng.choice(n_vars, size=int(rng.integers(1, n_vars + 1)), replace=False):
            vals = np.unique(rng.integers(0, dom, size=int(rng.integers(0, dom + 1)))).astype(np.uint32)
            extra.append(((int(v), -1), np.stack([vals, np.zeros_like(vals)], 1)))
        a2 = list(atoms) + [e[0] for e in extra]
        r2 = rels + [e[1] for e in extra]
        expect = brute_force(n_vars, a2, r2, dom)
        assert oracle.gj_count(n_vars, a2, r2)[0] == expect.shape[0]
        got = oracle.gj_enumerate(n_vars, a2, r2)
        assert np.array_equal(_sorted_rows(got), _sorted_rows(expect))


def test_unary_first_variable_equals_filter():
    sym = datagen.random_graph(60, 0.2, 3)
    ep = datagen.orient_lt(sym)
    f = np.array([3, 7, 11, 20, 41, 59], dtype=np.uint32)
    unary = np.stack([f, np.zeros_like(f)], 1)
    a = oracle.gj_count(3, list(oracle.TRIANGLE[1]) + [(0, -1)], [ep, ep, ep, unary])[0]
    b = oracle.gj_count(3, list(oracle.TRIANGLE[1]), [ep, ep, ep], filt=f)[0]
    assert a == b


def test_brute_force_empty_and_degenerate():
    n_vars, atoms = oracle.TRIANGLE
    empty = np.zeros((0, 2), dtype=np.uint32)
    one = np.array([[0, 1]], dtype=np.uint32)
    assert oracle.gj_count(n_vars, atoms, [empty] * 3)[0] == 0
    assert oracle.gj_count(n_vars, atoms, [one, empty, one])[0] == 0
    # a single triangle 0-1-2
    r = np.array([[0, 1]], dtype=np.uint32)
    s = np.array([[1, 2]], dtype=np.uint32)
    t = np.array([[0, 2]], dtype=np.uint32)
    assert oracle.gj_enumerate(n_vars, atoms, [r, s, t]).tolist() == [[0, 1, 2]]
    # values at the top of the uint32 range
    big = np.array([[0xFFFFFFFD, 0xFFFFFFFE], [0xFFFFFFFE, 0xFFFFFFFF], [0xFFFFFFFD, 0xFFFFFFFF]],
                   dtype=np.uint32)
    assert oracle.gj_enumerate(n_vars, atoms, [big[:1], big[1:2], big[2:]]).tolist() == [
        [0xFFFFFFFD, 0xFFFFFFFE, 0xFFFFFFFF]]


# ------------------------------------------------------------------- invariants

@pytest.mark.parametrize("name", ["triangle", "four_cycle", "four_clique", "four_diamond"])
def test_order_invariance(name):
    n_vars, atoms = QUERIES[name]
    sym = datagen.random_graph(24, 0.35, 11)
    rels = [sym] * len(atoms)
    base = oracle.gj_count(n_vars, atoms, rels)[0]
    ref = _sorted_rows(oracle.gj_enumerate(n_vars, atoms, rels))
    for order in itertools.permutations(range(n_vars)):
        assert oracle.gj_count(n_vars, atoms, rels, order=order)[0] == base
    for order in list(itertools.permutations(range(n_vars)))[::5]:
        got = _sorted_rows(oracle.gj_enumerate(n_vars, atoms, rels, order=order))
        assert np.array_equal(got, ref)


def test_symmetric_vs_oriented_multiplicity():
    sym = datagen.random_graph(60, 0.2, 5)
    ep = datagen.orient_lt(sym)
    assert oracle.gj_count(*oracle.TRIANGLE, [sym] * 3)[0] == 6 * oracle.gj_count(*oracle.TRIANGLE, [ep] * 3)[0]
    assert oracle.gj_count(*oracle.FOUR_CLIQUE, [sym] * 6)[0] == 24 * oracle.gj_count(*oracle.FOUR_CLIQUE, [ep] * 6)[0]


def test_threads_filter_and_per_top_consistent():
    sym = datagen.rmat_graph(10, 8, 3)
    ep = datagen.orient_lt(sym)
    c1, w1, per = oracle.gj_count(*oracle.TRIANGLE, [ep] * 3, per_top=True)
    c4, w4, _ = oracle.gj_count(*oracle.TRIANGLE, [ep] * 3, nthreads=4)
    assert c1 == c4 and w1 == w4 and int(per.sum()) == c1
    tops = np.unique(ep[:, 0])
    pick = tops[::7]
    cf, _, _ = oracle.gj_count(*oracle.TRIANGLE, [ep] * 3, filt=pick)
    assert cf == int(per[np.searchsorted(tops, pick)].sum())


def test_cells_are_a_disjoint_cover():
    sym = datagen.random_graph(50, 0.25, 9)
    ep = datagen.orient_lt(sym)
    tup = oracle.gj_enumerate(*oracle.TRIANGLE, [ep] * 3)
    shares, seeds = [4, 2, 8], [11, 22, 33]
    cells = oracle.tuple_cells(tup, seeds, shares)
    assert cells.max() < 64
    expect = [[oracle.share(t[v], seeds[v], shares[v]) for v in range(3)] for t in tup[:50]]
    for t, e, c in zip(tup[:50], expect, cells[:50]):
        assert c == (e[0] * shares[1] + e[1]) * shares[2] + e[2]
    assert np.bincount(cells, minlength=64).sum() == tup.shape[0]


# ---------------------------------------------------------------- CoCo / partition

@pytest.mark.parametrize("seed", range(5))
def test_coco_build_matches_library_sort(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 3000))
    pairs = datagen.directed_set(rng.integers(0, 300, size=(n, 2)).astype(np.uint32))
    pairs = datagen.scatter_order(pairs, seed)
    for ao in (0, 1):
        v1, o1, v2 = oracle.coco_build(pairs, ao)
        a, b = (pairs[:, 0], pairs[:, 1]) if ao == 0 else (pairs[:, 1], pairs[:, 0])
        idx = np.lexsort((b, a))
        sa, sb = a[idx], b[idx]
        uv, starts = np.unique(sa, return_index=True)
        assert np.array_equal(v1, uv)
        assert np.array_equal(o1, np.append(starts, len(sa)).astype(np.uint64))
        assert np.array_equal(v2, sb)


def test_coco_join_worked_example():
    g = _golden("coco_join_example.txt")
    r = np.array(g["R"], dtype=np.uint32)
    s = np.array(g["S"], dtype=np.uint32)
    v1r, o1r, v2r = oracle.coco_build(r)
    v1s, o1s, v2s = oracle.coco_build(s)
    i = g["index_of_x2"][0][0]
    assert v1r[i] == 2 and v1s[i] == 2
    assert [int(o1r[i]), int(o1r[i + 1])] == g["range_R"][0]
    assert v2r[o1r[i]:o1r[i + 1]].tolist() == g["sub_R"][0]
    assert v2s[o1s[i]:o1s[i + 1]].tolist() == g["sub_S"][0]
    out = oracle.gj_enumerate(2, [(0, 1), (0, 1)], [r, s])
    assert out.tolist() == [g["join_xy"][0]]


def test_partition_worked_example():
    g = _golden("partition_example.txt")
    px, py = g["shares_xy"][0]
    grey = tuple(g["grey_partition"][0])
    grey_tuples = g["grey_tuples"]
    hy_one = g["hY_one"][0]
    # hash seeds for which the stated hash values hold: h_X(0) = h_X(5) = 0
    # (grey partition has s_X = 0) and h_Y(v) = 1 for the listed v
    sx = next(s for s in range(1, 100000)
              if all(oracle.share(x, s, px) == grey[0] for x, _ in grey_tuples))
    sy = next(s for s in range(1, 100000) if all(oracle.share(v, s, py) == 1 for v in hy_one))
    hx = lambda v: oracle.share(v, sx, px)
    hy = lambda v: oracle.share(v, sy, py)
    xs0 = [v for v in range(6, 400) if hx(v) == 0][:3]
    xs1 = [v for v in range(6, 400) if hx(v) == 1][:2]
    ys0 = [v for v in range(6, 400) if hy(v) == 0][:3]
    rel = [(xs0[0], ys0[0]), (xs0[1], ys0[1]), (xs0[2], ys0[2])]  # 3 tuples in (0,0)
    rel += [tuple(t) for t in grey_tuples]                       # grey (0,1)
    rel += [(xs1[0], 1), (xs1[1], 4)]                            # (1,1); (1,0) left empty
    part = oracle.partition(np.array(rel, dtype=np.uint32), 0, sx, px, sy, py)
    pid = grey[0] * py + grey[1]
    e = g["empty_partition"][0]
    assert int(part["B"][pid]) == g["B_grey"][0][0]
    assert int(part["Bpref"][pid]) == g["Bpref_grey"][0][0]
    assert int(part["B"][e[0] * py + e[1]]) == 0
    lo, hi = int(part["Bpref"][pid]), int(part["Bpref"][pid + 1])
    assert part["rt"][lo:hi].tolist() == sorted(list(t) for t in grey_tuples)


@pytest.mark.parametrize("shares", [(1, 1), (2, 3), (4, 4), (1, 16), (32, 32)])
def test_partition_definition(shares):
    pa, pb = shares
    sym = datagen.rmat_graph(9, 8, 4)
    pairs = datagen.scatter_order(datagen.orient_lt(sym), 1)
    part = oracle.partition(pairs, 1, 123, pa, 456, pb)
    rt = part["rt"]
    n = pairs.shape[0]
    # no replication: exactly the input tuples (in attr order (col1, col0))
    assert rt.shape[0] == n
    assert np.array_equal(_sorted_rows(rt), _sorted_rows(pairs[:, ::-1]))
    pref = part["Bpref"].astype(np.int64)
    assert pref[0] == 0 and pref[-1] == n
    assert np.array_equal(np.diff(pref), part["B"].astype(np.int64))
    for p in range(pa * pb):
        seg = rt[pref[p]:pref[p + 1]]
        for a, b in seg[:20]:
            assert oracle.share(a, 123, pa) * pb + oracle.share(b, 456, pb) == p
        assert np.array_equal(seg, _sorted_rows(seg))
        ls, le = int(part["lvl1_start"][p]), int(part["lvl1_start"][p + 1])
        v1, o1, v2 = oracle.coco_build(seg, 0)
        assert np.array_equal(part["V1"][ls:le], v1)
        assert np.array_equal(part["O1"][ls:le], o1[:-1] + np.uint64(pref[p]))


# ------------------------------------------------------------------- work counter

def _brute_work(n_vars, atoms, rels, dom):
    """Sum over loops i and loop-i bindings of |S| * min list length."""
    first = [a if a[0] < a[1] else (a[1], a[0]) for a in atoms]
    sets = []
    for (v0, v1), r in zip(atoms, rels):
        s = set(map(tuple, r.tolist()))
        sets.append(s if v0 < v1 else {(b, a) for a, b in s})
    total = 0
    for i in range(n_vars):
        srcs = [j for j, (f, s) in enumerate(first) if f == i or s == i]
        for pre in itertools.product(range(dom), repeat=i):
            ok = True
            for j, (f, s) in enumerate(first):
                if f < i and s < i:
                    ok &= (pre[f], pre[s]) in sets[j]
                elif f < i:
                    ok &= any(t[0] == pre[f] for t in sets[j])
            if not ok:
                continue
            lens = []
            for j in srcs:
                f, s = first[j]
                if f == i:
                    lens.append(len({t[0] for t in sets[j]}))
                else:
                    lens.append(sum(1 for t in sets[j] if t[0] == pre[f]))
            total += len(srcs) * min(lens)
    return total


@pytest.mark.parametrize("name", ["triangle", "four_cycle", "four_clique"])
def test_work_counter_brute_force(name):
    n_vars, atoms = QUERIES[name]
    rng = np.random.default_rng(3)
    dom = 6
    for _ in range(6):
        rels = [np.argwhere(rng.random((dom, dom)) < 0.5).astype(np.uint32) for _ in atoms]
        assert oracle.gj_count(n_vars, atoms, rels)[1] == _brute_work(n_vars, atoms, rels, dom)


def test_duplicates_detected_and_hash_vector():
    assert oracle.has_duplicates(np.array([[1, 2], [3, 4], [1, 2]], dtype=np.uint32))
    assert not oracle.has_duplicates(np.array([[1, 2], [2, 1]], dtype=np.uint32))
    # published MurmurHash3 fmix32 values: fmix32(0) = 0, fmix32(1) = 0x514E28B7
    assert oracle.fmix32(0) == 0
    assert oracle.fmix32(1) == 0x514E28B7


def test_arg_errors():
    e = np.array([[0, 1]], dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.gj_count(3, [(0, 1), (1, 1), (0, 2)], [e] * 3)      # atom repeats a variable
    with pytest.raises(oracle.OracleError):
        oracle.gj_count(4, [(0, 1), (1, 2), (0, 2)], [e] * 3)      # variable 3 in no atom
    with pytest.raises(ValueError):
        oracle.gj_count(3, [(0, 1), (1, 2), (0, 2)], [e] * 3, order=[0, 1])
