"""Serving loop: every result is the same alone and in the mix (GPU).

Requests are the paper's Q1 / Q2 / Q6 shapes over four device-resident
relations, each variable restricted to the request's vertex sample by a
unary atom (a selection pushed into the query).  The concurrent server's
counts must equal the one-at-a-time counts exactly, and the oracle's.
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


def make_requests(hc, rels, n, seed, nv):
    from paper_2502_06715_gb300.serve import Request

    rng = np.random.default_rng(seed)
    names = sorted(rels)
    deg = np.bincount(rels["rmat"][:, 0], minlength=nv)
    pool = np.nonzero(deg <= 64)[0].astype(np.uint32)
    out = []
    for i in range(n):
        u = rng.random()
        base = hc.TRIANGLE if u < 0.6 else (hc.FOUR_CYCLE if u < 0.9 else hc.FOUR_CLIQUE)
        rel_names = tuple(names[k] for k in rng.integers(0, len(names), size=len(base.atoms)))
        size = int(np.exp(rng.uniform(np.log(64), np.log(2048))))
        f = np.unique(rng.choice(pool, size=min(size, pool.shape[0]), replace=False)).astype(np.uint32)
        q = base.with_atoms([(v, None) for v in range(base.n_vars)])
        out.append(Request(i, q, rel_names, f, arrival=float(rng.exponential(0.0005)) * i))
    return out


def test_served_equals_alone_and_oracle(hc):
    import torch

    from paper_2502_06715_gb300.serve import Server, serve_serial

    nv = 1 << 12
    rels = {"rmat": datagen.rmat_graph(12, 8, 5),
            "u20k": datagen.uniform_relation(20000, nv, 6),
            "u5k": datagen.uniform_relation(5000, nv, 7),
            "u1k": datagen.uniform_relation(1000, nv, 8)}
    idx = {k: hc.build_index(torch.from_numpy(v.view(np.int32)).cuda(), 0) for k, v in rels.items()}
    reqs = make_requests(hc, rels, 60, 9, nv)
    srv = Server(idx, budget_bytes=1 << 30, max_inflight=4)
    alone = {o.rid: o.count for o in serve_serial(srv, reqs)}
    mixed = {o.rid: o.count for o in srv.run(reqs)}
    assert mixed == alone
    for r in reqs[:20]:
        un = np.stack([r.restrict, np.zeros_like(r.restrict)], 1)
        want = oracle.gj_count(r.query.n_vars, [(a, -1 if b is None else b) for a, b in r.query.atoms],
                               [rels[n] for n in r.relations] + [un] * r.query.n_vars)[0]
        assert alone[r.rid] == want


def test_admission_respects_budget(hc):
    """With a budget below every footprint, requests still run one at a time."""
    import torch

    from paper_2502_06715_gb300.serve import Server

    nv = 1 << 10
    rels = {"rmat": datagen.rmat_graph(10, 8, 1), "u": datagen.uniform_relation(3000, nv, 2)}
    idx = {k: hc.build_index(torch.from_numpy(v.view(np.int32)).cuda(), 0) for k, v in rels.items()}
    reqs = make_requests(hc, rels, 12, 3, nv)
    out = Server(idx, budget_bytes=1, max_inflight=4).run(reqs)
    assert len(out) == 12
    spans = sorted((o.admitted, o.done) for o in out)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-3  # never two in flight


def test_unrestricted_requests_served(hc):
    """Requests without a selection (the uniform relations joined as they
    are) beside restricted ones: served counts equal the same requests run
    alone, and the unrestricted ones equal the oracle over the relations."""
    import torch

    from paper_2502_06715_gb300.serve import Request, Server, serve_serial

    nv = 1 << 12
    rels = {"rmat": datagen.rmat_graph(12, 8, 5),
            "u20k": datagen.uniform_relation(20000, nv, 6),
            "u5k": datagen.uniform_relation(5000, nv, 7)}
    idx = {k: hc.build_index(torch.from_numpy(v.view(np.int32)).cuda(), 0) for k, v in rels.items()}
    reqs = make_requests(hc, rels, 30, 11, nv)
    rng = np.random.default_rng(12)
    for i in range(30, 50):
        base = (hc.TRIANGLE, hc.FOUR_CYCLE, hc.FOUR_CLIQUE)[i % 3]
        names = tuple(("u20k", "u5k")[k] for k in rng.integers(0, 2, size=len(base.atoms)))
        reqs.append(Request(i, base, names, None, arrival=0.0002 * i))
    srv = Server(idx, budget_bytes=1 << 30, max_inflight=4)
    alone = {o.rid: o.count for o in serve_serial(srv, reqs)}
    mixed = {o.rid: o.count for o in srv.run(reqs)}
    assert mixed == alone
    for r in reqs[30:]:
        want = oracle.gj_count(r.query.n_vars, list(r.query.atoms), [rels[n] for n in r.relations])[0]
        assert alone[r.rid] == want, r.rid
