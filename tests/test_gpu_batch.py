"""Batched persistent launch against separate launches and the oracle (GPU)."""
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


def _queries(hc, n, seed):
    """Triangle / 4-clique queries (50/50) on induced subgraphs of one R-MAT graph."""
    sym = datagen.rmat_graph(12, 8, seed)
    ep = datagen.orient_lt(sym)
    rng = np.random.default_rng(seed)
    nv = int(sym.max()) + 1
    qs, rels = [], []
    for i in range(n):
        sub = datagen.induced_by_key(ep, nv, 1000 + i, int(rng.integers(200, 3000)))
        q = hc.TRIANGLE if rng.random() < 0.5 else hc.FOUR_CLIQUE
        qs.append(q)
        rels.append(sub)
    return qs, rels


@pytest.mark.parametrize("n", [1, 7, 40])
def test_batch_matches_separate_and_oracle(hc, n):
    import torch

    qs, rels = _queries(hc, n, 3 + n)
    idx = [hc.build_index(dev(r), 0) for r in rels]
    lists = [[ix] * len(q.atoms) for q, ix in zip(qs, idx)]
    opts = [{"shares": [2] + [1] * (q.n_vars - 1) if i % 3 == 0 else None} for i, q in enumerate(qs)]
    want = [oracle.gj_count(q.n_vars, list(q.atoms), [r] * len(q.atoms))[0] for q, r in zip(qs, rels)]
    sep = [hc.run_join(q, l, **{k: v for k, v in o.items() if v is not None}).count for q, l, o in zip(qs, lists, opts)]
    assert sep == want
    b = hc.Batch(qs, lists, opts)
    b.launch()
    assert b.counts() == want
    # record once as a CUDA graph, then replay twice
    s = torch.cuda.Stream()
    b.capture(s)
    for _ in range(2):
        b.launch(s)
        assert b.counts() == want
    b.free()


def test_batch_of_all_four_shapes(hc):
    """Triangles (two lists per loop), triangles with a selection on y (more
    lists at loop y), 4-cycles and 4-cliques in one batch: one launch over all
    four shape classes; counts equal separate launches and the oracle, also
    replayed as a CUDA graph."""
    import torch

    sym = datagen.rmat_graph(11, 8, 19)
    ep = datagen.orient_lt(sym)
    rng = np.random.default_rng(5)
    ix = hc.build_index(dev(ep), 0)
    ixs = hc.build_index(dev(sym), 0)
    qs, lists, rels = [], [], []
    for i in range(24):
        kind = i % 4
        if kind == 0:
            qs.append(hc.TRIANGLE), lists.append([ix] * 3), rels.append([ep] * 3)
        elif kind == 1:
            vals = np.unique(rng.integers(0, 2048, size=400)).astype(np.uint32)
            sel = np.stack([vals, np.zeros_like(vals)], 1)
            q = hc.TRIANGLE.with_atoms([(1, -1), (1, -1)])
            u = hc.build_index(dev(sel), 0)
            qs.append(q), lists.append([ix] * 3 + [u, u]), rels.append([ep] * 3 + [sel, sel])
        elif kind == 2:
            qs.append(hc.FOUR_CYCLE), lists.append([ixs] * 4), rels.append([sym] * 4)
        else:
            qs.append(hc.FOUR_CLIQUE), lists.append([ix] * 6), rels.append([ep] * 6)
    want = [oracle.gj_count(q.n_vars, list(q.atoms), r)[0] for q, r in zip(qs, rels)]
    opts = [{"shares": [2] + [1] * (q.n_vars - 1)} if i % 5 == 0 else {} for i, q in enumerate(qs)]
    assert [hc.run_join(q, l, **o).count for q, l, o in zip(qs, lists, opts)] == want
    b = hc.Batch(qs, lists, opts)
    b.launch()
    assert b.counts() == want
    s = torch.cuda.Stream()
    b.capture(s)
    for _ in range(2):
        b.launch(s)
        assert b.counts() == want
    b.free()


def test_batch_rejects_five_variable_queries(hc):
    ep = datagen.orient_lt(datagen.random_graph(30, 0.3, 1))
    ix = hc.build_index(dev(ep), 0)
    with pytest.raises(hc.HoneycombError) as e:
        hc.Batch([hc.TRIANGLE, hc.TWO_TRIANGLE], [[ix] * 3, [ix] * 6])
    assert e.value.status == 5


def test_autotuner_picks_a_valid_config(hc, tmp_path):
    """The tuner's choice is one of its candidates and leaves the count unchanged."""
    from paper_2502_06715_gb300.autotune import Tuner

    sym = datagen.rmat_graph(12, 8, 9)
    ep = datagen.orient_lt(sym)
    ix = hc.build_index(dev(ep), 0)
    want = oracle.gj_count(3, list(hc.TRIANGLE.atoms), [ep] * 3)[0]
    path = str(tmp_path / "tune.json")
    t = Tuner(path=path, reps=1)
    cfg = t.tune(hc.TRIANGLE, [ix] * 3, P_list=(4, 16), min_cells=4)
    assert int(np.prod(cfg.shares)) >= 4
    assert hc.run_join(hc.TRIANGLE, [ix] * 3, **cfg.options()).count == want
    # cached: a second tuner reads the file and returns the same choice
    again = Tuner(path=path).tune(hc.TRIANGLE, [ix] * 3, P_list=(4, 16), min_cells=4)
    assert again.shares == cfg.shares and again.item_grain == cfg.item_grain
