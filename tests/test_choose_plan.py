"""Joint choice of loop order and shares (Sec. 5.3, "Plan Decision"), host only.

The loop order never changes a join's result (checked on the GPU against the
oracle in test_gpu_plan.py), so these tests pin the decision rule: every
order is tried with the shares hc_choose_shares gives it, the order of least
replicated cost (Eq. "total:cost") at those shares is kept, ties go to the
smaller unpartitioned cost and then to the lexicographically smallest order.
The expected plans are derived here from per-order calls of the library's
estimates (plan_cost, choose_shares), not from hc_choose_plan.
"""
import itertools
import math

import pytest

import paper_2502_06715_gb300 as hc


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2502_06715_gb300 import build

    build.build_library()


def stats(rows, d0, d1, attr_order=0):
    """Statistics-only index of a relation with d0 / d1 distinct values in
    columns 0 / 1 (the index sorts by column `attr_order` first)."""
    first, second = (d0, d1) if attr_order == 0 else (d1, d0)
    return hc.Index.from_stats(rows, first, attr_order, first - 1, second - 1)


def expected_plan(q, idx, P):
    best = None
    for perm in itertools.permutations(range(q.n_vars)):  # lexicographic
        qo = q.with_order(perm)
        sh = hc.choose_shares(qo, idx, P)
        c = hc.plan_cost(qo, idx, sh)
        key = (c["replicated"], sum(c["level_cost"]))
        if best is None or _lt(key, best[0]):
            best = (key, perm, sh)
    return best[1], best[2]


def _lt(a, b):
    def less(x, y):
        return x < y - 1e-9 * max(1.0, abs(y))

    return less(a[0], b[0]) or (not less(b[0], a[0]) and less(a[1], b[1]))


def mixed_relations(q, seed):
    # relations of different sizes and densities, so that orders differ in cost
    import random

    r = random.Random(seed)
    out = []
    for _ in q.atoms:
        d0 = r.choice([1_000, 50_000, 2_000_000])
        d1 = r.choice([1_000, 50_000, 2_000_000])
        rows = r.randint(max(d0, d1), 40 * max(d0, d1))
        out.append(stats(rows, d0, d1))
    return out


@pytest.mark.parametrize("qname", ["TRIANGLE", "FOUR_CYCLE", "FOUR_DIAMOND", "FOUR_CLIQUE", "TWO_TRIANGLE"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_plan_matches_restatement(qname, seed):
    q = getattr(hc, qname)
    idx = mixed_relations(q, seed)
    for P in (1, 64, 1024):
        order, shares = hc.choose_plan(q, idx, P)
        assert (order, shares) == expected_plan(q, idx, P)


def test_order_is_a_permutation_and_shares_multiply_to_P():
    q = hc.FOUR_CLIQUE
    idx = mixed_relations(q, 7)
    for P in (1, 2, 256, 4096):
        order, shares = hc.choose_plan(q, idx, P)
        assert sorted(order) == list(range(q.n_vars))
        assert math.prod(shares) == P or shares == [P if v == order[0] else 1 for v in range(q.n_vars)]


def test_plan_ignores_the_given_order():
    q = hc.TRIANGLE
    idx = mixed_relations(q, 4)
    got = {(o2, tuple(sh)) for o2, sh in (hc.choose_plan(q.with_order(o), idx, 256)
                                          for o in itertools.permutations(range(3)))}
    assert len(got) == 1


def test_small_relation_leads():
    """A triangle whose R(X,Y) is tiny and whose S, T are large: starting the
    loops on R's variables costs far less than starting on Z, and the
    unpartitioned costs of the chosen order are no larger than any other's."""
    q = hc.TRIANGLE
    small = stats(500, 400, 400)
    big = stats(50_000_000, 2_000_000, 2_000_000)
    idx = [small, big, big]
    order, shares = hc.choose_plan(q, idx, 1)
    assert order[0] in (0, 1)
    costs = {o: sum(hc.plan_cost(q.with_order(o), idx, [1, 1, 1])["level_cost"])
             for o in itertools.permutations(range(3))}
    assert costs[order] == pytest.approx(min(costs.values()))


def test_bad_arguments():
    q = hc.TRIANGLE
    idx = mixed_relations(q, 5)
    with pytest.raises(hc._lib.HoneycombError):
        hc.choose_plan(q, idx, 3)  # P not a power of two


def test_ranked_orders_follow_the_estimate():
    """The autotuner's order candidates: every loop order once, cheapest first
    by the summed per-loop estimate that hc_plan_cost reports at shares 1."""
    import itertools

    import paper_2502_06715_gb300 as hc
    from paper_2502_06715_gb300.autotune import ranked_orders

    q = hc.FOUR_CLIQUE
    rels = [hc.Index.from_stats(1_000_000 + 7919 * j, 40_000 + 1013 * j, 0, 2_000_000, 2_000_000)
            for j in range(len(q.atoms))]
    ranked = ranked_orders(q, rels)
    assert sorted(ranked) == sorted(itertools.permutations(range(4)))
    costs = [sum(hc.plan_cost(q.with_order(o), rels, [1] * 4)["level_cost"]) for o in ranked]
    assert costs == sorted(costs)
    # the plan decision's order is among the cheapest by the same estimate
    order, _ = hc.choose_plan(q, rels, 1)
    assert costs[ranked.index(tuple(order))] == costs[0]
