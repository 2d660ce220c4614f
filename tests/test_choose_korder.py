"""Loop-order choice for k-ary queries (Sec. 5.2-5.3), host only.

hc_kplan_cost estimates Lemma "cost-ub" per loop from statistics-only
indexes; hc_choose_korder keeps the order of least total.  Pins: hand
computations of the estimate on a single ternary atom, equality with the
binary optimizer's level costs (hc_plan_cost, written separately) on binary
atoms where it does not rewrite, the choice against a per-order restatement
with lexicographic ties, and the orders the paper's tensor workloads call
for.  Also the C ABI's argument checks that run before any device work.
"""
import ctypes
import itertools
import math

import pytest

import paper_2502_06715_gb300 as hc


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2502_06715_gb300 import build

    build.build_library()


def test_single_atom_hand_computation():
    # R(X,Y,Z): 100 rows, 4 distinct X, 20 distinct (X,Y); largest values 3, 9, 49
    r = hc.KIndex.from_stats(100, (4, 20, 100), (3, 9, 49))
    q = hc.KQuery(3, ((0, 1, 2),))
    # order X,Y,Z: lists 4, 20/4, 100/20 over 1, 4, 20 bindings
    c = hc.kplan_cost(q, [r])
    assert c["level_cost"] == pytest.approx([4.0, 20.0, 100.0])
    assert c["dom"] == pytest.approx([4.0, 10.0, 50.0])
    # order Z,Y,X: D{Z} = 50 (value range), D{Y,Z} = min(100, 10 * 50) = 100, D{X,Y,Z} = 100
    c = hc.kplan_cost(q.with_order((2, 1, 0)), [r])
    assert c["level_cost"] == pytest.approx([50.0, 100.0, 100.0])


def test_two_lists_hand_computation():
    # R(X,Y), S(Y): loop Y intersects a sub-list of average length 100/10 = 10
    # with S's 30 values over a domain of min(50, 30) = 30
    r = hc.KIndex.from_stats(100, (10, 100), (9, 49))
    s = hc.KIndex.from_stats(30, (30,), (49,))
    q = hc.KQuery(2, ((0, 1), (1,)))
    c = hc.kplan_cost(q, [r, s])
    assert c["dom"] == pytest.approx([10.0, 30.0])
    # loop 0: 1 * 10 * log2(2); loop 1: 2 * (10 * 10) * log2(1 + 300 / 100)
    assert c["level_cost"] == pytest.approx([10.0, 2 * 100 * math.log2(4.0)])


def binary_pair(n, l1, attr_order, max_first, max_second):
    return (hc.Index.from_stats(n, l1, attr_order, max_first, max_second),
            hc.KIndex.from_stats(n, (l1, n), (max_first, max_second), (0, 1) if attr_order == 0 else (1, 0)))


@pytest.mark.parametrize("seed", range(4))
def test_binary_atoms_match_binary_optimizer(seed):
    import random

    rnd = random.Random(seed)
    pairs = [binary_pair(rnd.randint(5_000, 900_000), rnd.randint(100, 4_000), rnd.randint(0, 1),
                         rnd.randint(5_000, 60_000), rnd.randint(5_000, 60_000)) for _ in range(3)]
    bq, kq = hc.TRIANGLE, hc.KQuery(3, hc.TRIANGLE.atoms)
    for order in itertools.permutations(range(3)):
        want = hc.plan_cost(bq.with_order(order), [p[0] for p in pairs], [1, 1, 1])
        got = hc.kplan_cost(kq.with_order(order), [p[1] for p in pairs])
        assert got["level_cost"] == pytest.approx(want["level_cost"][:3], rel=1e-12), order
        assert got["dom"] == pytest.approx(want["dom"][:3], rel=1e-12)
    # 4-cycle under X,Y,Z,U: its last loop has one far list, so no rewriting
    pairs4 = pairs + [binary_pair(300_000, 2_000, 0, 50_000, 50_000)]
    want = hc.plan_cost(hc.FOUR_CYCLE, [p[0] for p in pairs4], [1, 1, 1, 1])
    got = hc.kplan_cost(hc.KQuery(4, hc.FOUR_CYCLE.atoms), [p[1] for p in pairs4])
    assert got["level_cost"] == pytest.approx(want["level_cost"][:4], rel=1e-12)


def restated_order(q, idx):
    best = None
    for perm in itertools.permutations(range(q.n_vars)):
        total = sum(hc.kplan_cost(q.with_order(perm), idx)["level_cost"])
        if best is None or total < best[0] - 1e-9 * max(1.0, abs(best[0])):
            best = (total, perm)
    return best[1]


@pytest.mark.parametrize("seed", range(5))
def test_choice_matches_restatement(seed):
    import random

    rnd = random.Random(50 + seed)
    q = hc.KQuery(5, ((2, 0, 4), (3, 1), (4,), (1, 2, 0), (3, 4)))
    idx = []
    for a in q.atoms:
        k = len(a)
        n = rnd.randint(10_000, 2_000_000)
        ls = sorted(rnd.randint(1, n) for _ in range(k - 1)) + [n]
        idx.append(hc.KIndex.from_stats(n, tuple(ls), tuple(rnd.randint(1_000, 200_000) for _ in range(k)),
                                        tuple(rnd.sample(range(k), k))))
    assert hc.choose_korder(q, idx) == restated_order(q, idx)
    # the given order is ignored
    assert hc.choose_korder(q.with_order((4, 3, 2, 1, 0)), idx) == hc.choose_korder(q, idx)


def test_tensor_workload_orders():
    n, m = 512, 4096
    cube = hc.KIndex.from_stats(n ** 3, (n, n * n, n ** 3), (n - 1, n - 1, n - 1))
    # LW over four equal cubes: every order costs the same, the first is kept
    assert hc.choose_korder(hc.LW, [cube] * 4) == (0, 1, 2, 3)
    # CT over F x [m] x [m], |F| = 2: start from U, whose lists hold 2 values
    sq = [hc.KIndex.from_stats(2 * m * m, (2, 2 * m, 2 * m * m), (f, m - 1, m - 1)) for f in (1, 2, 2)]
    assert hc.choose_korder(hc.CT, sq)[0] == 0


def test_argument_checks_without_device_work():
    lib = hc._lib.load()
    out = ctypes.c_void_p()
    assert lib.hc_build_kindex(None, 0, 4, None, 0, None, ctypes.byref(out)) == 1  # arity 4
    bad_cols = (ctypes.c_uint8 * 3)(0, 0, 1)
    assert lib.hc_build_kindex(None, 0, 3, bad_cols, 0, None, ctypes.byref(out)) == 1
    assert lib.hc_build_kindex(ctypes.c_void_p(16), 0xFFFFFFFF, 3, None, 0, None, ctypes.byref(out)) == 5
    with pytest.raises(hc.HoneycombError):
        hc.KIndex.from_stats(10, (3, 11, 10), (1, 1, 1))  # l_1 > n
    with pytest.raises(hc.HoneycombError):
        hc.KIndex.from_stats(10, (3, 5, 9), (1, 1, 1))  # last level must hold n
    with pytest.raises(hc.HoneycombError):
        hc.KIndex.from_stats(10, (3, 10), (1, 1), (1, 1))

    r3 = hc.KIndex.from_stats(100, (4, 20, 100), (3, 9, 49))
    r2 = hc.KIndex.from_stats(100, (10, 100), (9, 49))
    q = hc.KQuery(4, ((0, 1, 2), (1, 2, 3)))
    for idx, status in (([r3, r3], 1),  # statistics-only indexes hold no data
                        ([hc.KIndex.from_stats(100, (4, 20, 100), (3, 9, 49), (2, 1, 0)), r3], 1),  # level order
                        ([r2, r3], 1)):  # arity differs from the atom's
        with pytest.raises(hc.HoneycombError) as e:
            hc.run_kjoin(q, idx, stream=0)
        assert e.value.status == status
    with pytest.raises(hc.HoneycombError) as e:
        hc.run_kjoin(hc.KQuery(2, tuple([(0, 1)] * 5)), [r2] * 5, stream=0)  # X in five atoms
    assert e.value.status == 5
    with pytest.raises(hc.HoneycombError) as e:
        hc.run_kjoin(hc.KQuery(7, ((0, 1, 2), (3, 4, 5), (6,))), [r3, r3, hc.KIndex.from_stats(5, (5,), (9,))],
                     stream=0)
    assert e.value.status == 5
    with pytest.raises(hc.HoneycombError):
        hc.kplan_cost(hc.KQuery(4, ((0, 1, 2),)), [r3])  # U in no atom


def test_atom_shares_maps_variable_shares_to_columns():
    """Each atom's columns take their variables' shares and seeds (the
    arguments of a partitioned build), default seeds v + 1."""
    import paper_2502_06715_gb300 as hc

    per_atom = hc.atom_shares(hc.LW, (2, 3, 1, 5))
    assert per_atom == [((1, 2, 3), (2, 3, 1)), ((1, 2, 4), (2, 3, 5)), ((1, 3, 4), (2, 1, 5)),
                        ((2, 3, 4), (3, 1, 5))]
    ct = hc.atom_shares(hc.CT, (4, 1, 2, 1), seeds=(9, 8, 7, 6))
    assert ct == [((9, 8, 7), (4, 1, 2)), ((9, 8, 6), (4, 1, 1)), ((9, 7, 6), (4, 2, 1))]
