"""Admission footprints of the serving loop (host only, no GPU).

The server caches one footprint per (query, relations, size class of the
request's selection), computed for the class's largest selection.  Admission
is safe only if that cached figure is never below the footprint of a request
of the class; this is checked against the exact footprint of each request,
with statistics-only indexes standing in for the resident relations.
"""
import numpy as np
import pytest

import paper_2502_06715_gb300 as hc


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2502_06715_gb300 import build

    build.build_library()


def test_cached_footprint_bounds_every_request():
    from paper_2502_06715_gb300.serve import Request, Server

    nv = 1 << 24
    rels = {"rmat": hc.Index.from_stats(258_000_000, 15_000_000, 0, nv - 1, nv - 1),
            "u50M": hc.Index.from_stats(50_000_000, 16_000_000, 0, nv - 1, nv - 1),
            "u1M": hc.Index.from_stats(1_000_000, 950_000, 0, nv - 1, nv - 1)}
    server = Server(rels)
    rng = np.random.default_rng(9)
    names = sorted(rels)
    for i in range(120):
        q = (hc.TRIANGLE, hc.FOUR_CYCLE, hc.FOUR_CLIQUE)[i % 3]
        rel = tuple(names[k] for k in rng.integers(0, len(names), size=len(q.atoms)))
        n = int(rng.integers(1, 140_000))
        vals = np.unique(rng.integers(0, nv, size=n).astype(np.uint32))
        extra = [(v, -1) for v in range(q.n_vars)]
        req = Request(i, q.with_atoms(extra), rel, vals)
        cached = server.footprint(req)
        stand_in = hc.Index.from_stats(vals.shape[0], vals.shape[0], 0, int(vals.max()), 0)
        exact = hc.join_footprint(req.query, server._indexes(req, stand_in))
        assert cached >= exact, (i, cached, exact)
    # the cache is keyed by size class: far fewer entries than requests
    assert len(server._fp) < 120


def test_unrestricted_requests_footprint():
    """A request without a selection joins the resident relations as they
    are: its footprint is the query's over those indexes alone, and asking
    for unary atoms without a selection is refused."""
    from paper_2502_06715_gb300.serve import Request, Server

    nv = 1 << 24
    rels = {"u10M": hc.Index.from_stats(10_000_000, 7_000_000, 0, nv - 1, nv - 1),
            "u1M": hc.Index.from_stats(1_000_000, 950_000, 0, nv - 1, nv - 1)}
    server = Server(rels)
    req = Request(0, hc.TRIANGLE, ("u10M", "u1M", "u10M"), None)
    want = hc.join_footprint(hc.TRIANGLE, [rels["u10M"], rels["u1M"], rels["u10M"]])
    assert server.footprint(req) == want
    bad = Request(1, hc.TRIANGLE.with_atoms([(0, -1)]), ("u10M", "u1M", "u10M"), None)
    with pytest.raises(ValueError):
        server.footprint(bad)
