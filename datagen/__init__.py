"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws and cleans relations; it holds none of the join
method's arithmetic (no trie build, no hashing into shares, no
intersection).  Every generator is deterministic in its seed and
platform-independent: draws come from numpy's PCG64 stream, consumed in
fixed-size chunks, so the x86 host and the Arm GPU host produce the same
relations bit for bit.

Relations are returned as ``(n, 2)`` ``uint32`` arrays of pairs.  The
stand-ins follow the shapes of the paper's graph workloads (Sec. 6,
Table "Dataset Characteristics": sparse/skewed to dense graphs with
millions of vertices and edges): uniform random graphs and R-MAT graphs
with parameters (a, b, c, d) = (0.57, 0.19, 0.19, 0.05).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_CHUNK = 1 << 22  # draws are consumed in fixed chunks so results never depend on memory size

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _unique_u64(keys: np.ndarray, device: str | None = None) -> np.ndarray:
    """Sorted distinct values of a uint64 key array (< 2**63).

    A library sort serves as the de-duplication step.  When ``device`` names
    a CUDA device the sort runs there through torch (same sorted set, only
    faster); the result is always a host numpy array.
    """
    if device is not None and str(device).startswith("cuda"):
        import torch

        t = torch.from_numpy(keys.view(np.int64)).to(device)
        u = torch.unique(t, sorted=True)
        out = u.cpu().numpy().view(np.uint64)
        del t, u
        return out
    return np.unique(keys)


def _pack(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    return (u.astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64)


def _unpack(keys: np.ndarray) -> np.ndarray:
    out = np.empty((keys.shape[0], 2), dtype=np.uint32)
    out[:, 0] = (keys >> np.uint64(32)).astype(np.uint32)
    out[:, 1] = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def scatter_order(pairs: np.ndarray, seed: int) -> np.ndarray:
    """Deterministically reorder rows so that sorted input arrives unsorted.

    Row i moves to position (i * A + B) mod n with A coprime to n: an affine
    bijection, so the multiset of rows is unchanged.
    """
    n = pairs.shape[0]
    if n <= 1:
        return pairs.copy()
    r = _rng(seed ^ 0x5EED5EED)
    a = int(r.integers(n // 3 + 1, n)) | 1
    while math.gcd(a, n) != 1:
        a += 2
    b = int(r.integers(0, n))
    idx = (np.arange(n, dtype=np.uint64) * np.uint64(a) + np.uint64(b)) % np.uint64(n)
    out = np.empty_like(pairs)
    out[idx.astype(np.int64)] = pairs
    return out


def uniform_graph(n_vertices: int, n_edges: int, seed: int) -> np.ndarray:
    """Undirected simple graph: ``n_edges`` distinct pairs (u, v), u < v.

    Pairs u != v are drawn uniformly, canonicalised to (min, max) and kept
    in order of first appearance until ``n_edges`` distinct ones are found.
    Returned sorted by (u, v).
    """
    max_edges = n_vertices * (n_vertices - 1) // 2
    if n_edges > max_edges:
        raise ValueError("more edges requested than the complete graph has")
    rng = _rng(seed)
    found = np.empty(0, dtype=np.uint64)
    first_pos = np.empty(0, dtype=np.int64)
    drawn = 0
    while found.shape[0] < n_edges:
        need = n_edges - found.shape[0]
        k = max(1024, int(need * 1.3))
        u = rng.integers(0, n_vertices, size=k, dtype=np.int64)
        v = rng.integers(0, n_vertices, size=k, dtype=np.int64)
        keep = u != v
        u, v = u[keep], v[keep]
        lo, hi = np.minimum(u, v), np.maximum(u, v)
        keys = _pack(lo, hi)
        allk = np.concatenate([found, keys])
        allpos = np.concatenate([first_pos, drawn + np.arange(keys.shape[0], dtype=np.int64)])
        drawn += keys.shape[0]
        uk, ui = np.unique(allk, return_index=True)
        order = np.argsort(allpos[ui], kind="stable")
        found = uk[order]
        first_pos = allpos[ui][order]
    found = np.sort(found[:n_edges])
    return _unpack(found)


_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build(force: bool = False) -> str:
    """Compile the R-MAT draw helper (plain C, gcc) into ``datagen/_build``."""
    out_dir = os.path.join(_HERE, "_build")
    so = os.path.join(out_dir, "librmat.so")
    src = os.path.join(_HERE, "rmat.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", src, "-o", tmp])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        lib.rmat_fill.restype = ctypes.c_int
        lib.rmat_fill.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_int]
        _LIB = lib
    return _LIB


def rmat_raw(scale: int, edge_factor: int, seed: int, abcd=RMAT_ABCD,
             scramble: bool = True) -> np.ndarray:
    """Raw R-MAT edge list (with self loops and repeats), ``(m, 2)`` uint32.

    m = edge_factor * 2**scale edges.  Each edge descends ``scale`` levels of
    the adjacency quadrants, picking quadrant (0,0), (0,1), (1,0), (1,1) with
    probabilities a, b, c, d (no noise); the 32-bit draws come from a
    counter-based SplitMix64 stream (``rmat.c``).  With ``scramble`` the
    vertex ids go through a seeded random permutation so hubs are not the
    low ids.
    """
    a, b, c, d = abcd
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT probabilities must sum to 1")
    m = edge_factor << scale
    t1 = min(int(a * 2**32), 2**32 - 1)
    t2 = min(int((a + b) * 2**32), 2**32 - 1)
    t3 = min(int((a + b + c) * 2**32), 2**32 - 1)
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    rc = _lib().rmat_fill(src.ctypes.data, dst.ctypes.data, m, scale, int(seed) & (2**64 - 1),
                          t1, t2, t3, max(1, min(64, os.cpu_count() or 1)))
    if rc != 0:
        raise ValueError("rmat_fill rejected its arguments")
    if scramble:
        perm = _rng(seed ^ 0x9E3779B9).permutation(1 << scale).astype(np.uint32)
        src = perm[src]
        dst = perm[dst]
    return np.stack([src, dst], axis=1)


def symmetrize(pairs: np.ndarray, device: str | None = None) -> np.ndarray:
    """Both directions of every pair, self loops removed, de-duplicated, sorted."""
    u, v = pairs[:, 0], pairs[:, 1]
    keep = u != v
    u, v = u[keep], v[keep]
    keys = np.concatenate([_pack(u, v), _pack(v, u)])
    del u, v
    return _unpack(_unique_u64(keys, device))


def directed_set(pairs: np.ndarray, device: str | None = None) -> np.ndarray:
    """The pairs as given, self loops removed, de-duplicated, sorted."""
    keep = pairs[:, 0] != pairs[:, 1]
    return _unpack(_unique_u64(_pack(pairs[keep, 0], pairs[keep, 1]), device))


def orient_lt(sym: np.ndarray) -> np.ndarray:
    """The selection x < y of a relation (predicate pushed into the atom)."""
    return np.ascontiguousarray(sym[sym[:, 0] < sym[:, 1]])


def rmat_graph(scale: int, edge_factor: int, seed: int, device: str | None = None,
               scramble: bool = True) -> np.ndarray:
    """Symmetric, de-duplicated, loop-free R-MAT edge set (sorted pairs)."""
    return symmetrize(rmat_raw(scale, edge_factor, seed, scramble=scramble), device)


def uniform_relation(n_pairs: int, n_vertices: int, seed: int,
                     device: str | None = None) -> np.ndarray:
    """Directed relation of about ``n_pairs`` distinct pairs on ``n_vertices``.

    Pairs are drawn uniformly (self loops removed) and de-duplicated; the
    draw count is inflated by the expected collision rate so the result is
    close to ``n_pairs`` (the exact count is what the caller reads back).
    """
    rng = _rng(seed)
    space = float(n_vertices) * (n_vertices - 1)
    # expected distinct of k draws from `space` values: space*(1-exp(-k/space))
    frac = n_pairs / space
    k = int(math.ceil(-space * math.log1p(-frac))) if frac < 1 else n_pairs
    us, vs = [], []
    for s0 in range(0, k, _CHUNK):
        kk = min(_CHUNK, k - s0)
        us.append(rng.integers(0, n_vertices, size=kk, dtype=np.int64).astype(np.uint32))
        vs.append(rng.integers(0, n_vertices, size=kk, dtype=np.int64).astype(np.uint32))
    pairs = np.stack([np.concatenate(us), np.concatenate(vs)], axis=1)
    return directed_set(pairs, device)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014), vectorised."""
    z = x + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def vertex_sample_mask(n_vertices: int, seed_q: int, frac: float) -> np.ndarray:
    """Seeded vertex subset {v : splitmix64(v ^ seed) < frac * 2**64}."""
    with np.errstate(over="ignore"):
        h = _splitmix64(np.arange(n_vertices, dtype=np.uint64) ^ np.uint64(seed_q))
    thr = np.uint64(min(int(frac * 2.0**64), 2**64 - 1))
    return h < thr


def induced_subgraph(pairs: np.ndarray, n_vertices: int, seed_q: int, target_edges: int,
                     iters: int = 24) -> tuple[np.ndarray, float]:
    """Induced subgraph on a seeded vertex subset sized for ~target_edges.

    The sampled fraction f is found by bisection (edge count grows with f);
    returns the induced pairs and the f used.  The actual edge count is the
    length of the returned array.
    """
    lo, hi = 0.0, 1.0
    best = None
    for _ in range(iters):
        f = 0.5 * (lo + hi)
        mask = vertex_sample_mask(n_vertices, seed_q, f)
        sel = mask[pairs[:, 0]] & mask[pairs[:, 1]]
        cnt = int(sel.sum())
        best = (f, sel)
        if cnt < target_edges:
            lo = f
        else:
            hi = f
        if abs(cnt - target_edges) <= max(1, target_edges // 100):
            break
    f, sel = best
    return np.ascontiguousarray(pairs[sel]), f


MERSENNE31 = (1 << 31) - 1


def vertex_keys(n_vertices: int, seed_q: int) -> np.ndarray:
    """Seeded vertex keys k(v) = (A v + B) mod (2^31 - 1), A, B from the seed.

    Exact in int64 for v < 2^31 (A v < 2^62), so numpy and torch agree.
    """
    r = _rng(seed_q)
    a = int(r.integers(1, MERSENNE31))
    b = int(r.integers(0, MERSENNE31))
    v = np.arange(n_vertices, dtype=np.int64)
    return (v * a + b) % MERSENNE31


def induced_by_key(pairs, n_vertices: int, seed_q: int, target_edges: int):
    """Induced subgraph on {v : k(v) < t} with t chosen for ~target_edges.

    An edge survives iff max(k(u), k(v)) < t, so t is the target-th smallest
    edge key plus one: exactly target_edges edges (fewer on ties or if the
    graph has fewer).  Returns the surviving pairs in input order.  ``pairs``
    may be a numpy array or a torch CUDA tensor (int32 view of the uint32
    pairs); the torch path does the same integer arithmetic on the device.
    """
    if not isinstance(pairs, np.ndarray):
        import torch

        r = _rng(seed_q)
        a = int(r.integers(1, MERSENNE31))
        b = int(r.integers(0, MERSENNE31))
        v = torch.arange(n_vertices, dtype=torch.int64, device=pairs.device)
        k = (v * a + b) % MERSENNE31
        p64 = pairs.to(torch.int64) & 0xFFFFFFFF
        ek = torch.maximum(k[p64[:, 0]], k[p64[:, 1]])
        if target_edges >= pairs.shape[0]:
            return pairs.contiguous()
        t = torch.sort(ek).values[target_edges - 1] + 1
        return pairs[ek < t].contiguous()
    k = vertex_keys(n_vertices, seed_q)
    ek = np.maximum(k[pairs[:, 0]], k[pairs[:, 1]])
    m = pairs.shape[0]
    if target_edges >= m:
        return np.ascontiguousarray(pairs)
    t = np.partition(ek, target_edges - 1)[target_edges - 1] + 1
    return np.ascontiguousarray(pairs[ek < t])


def complete_graph(n: int) -> np.ndarray:
    """All pairs (u, v), u != v, of K_n (symmetric)."""
    u, v = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32), indexing="ij")
    keep = u != v
    return np.stack([u[keep], v[keep]], axis=1)


def complete_bipartite(m: int, n: int) -> np.ndarray:
    """Symmetric K_{m,n} on vertices 0..m-1 (left) and m..m+n-1 (right)."""
    a = np.arange(m, dtype=np.uint32)
    b = np.arange(m, m + n, dtype=np.uint32)
    u, v = np.meshgrid(a, b, indexing="ij")
    left = np.stack([u.ravel(), v.ravel()], axis=1)
    right = left[:, ::-1]
    out = np.concatenate([left, right])
    return out[np.lexsort((out[:, 1], out[:, 0]))]


def random_graph(n: int, p: float, seed: int) -> np.ndarray:
    """Symmetric G(n, p) edge set (sorted, no loops)."""
    rng = _rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    e = np.stack([iu[keep], ju[keep]], axis=1).astype(np.uint32)
    out = np.concatenate([e, e[:, ::-1]])
    return out[np.lexsort((out[:, 1], out[:, 0]))] if out.shape[0] else out.reshape(0, 2)


# --- ternary relations (the tensor workloads of Sec. 6: ST-Dense, ST-Sparse) ---
# The paper writes [N] for the integers 1..N; they are stored here as 0..N-1.


def full_cube(n: int) -> np.ndarray:
    """[n]^3 as an (n^3, 3) uint32 array, lexicographically sorted."""
    g = np.arange(n, dtype=np.uint32)
    a, b, c = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def prefixed_square(first: np.ndarray, m: int) -> np.ndarray:
    """first x [m] x [m]: every value of ``first`` (distinct) with every pair of [m]^2."""
    f = np.unique(np.asarray(first, dtype=np.uint32))
    g = np.arange(m, dtype=np.uint32)
    a, b, c = np.meshgrid(f, g, g, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def _distinct_keys(space: int, n: int, rng: np.random.Generator, device: str | None = None) -> np.ndarray:
    """Exactly ``n`` distinct keys drawn uniformly from [0, space) (< 2^63):
    draws are kept in order of first appearance until ``n`` are found;
    sorted output.  With ``device`` the de-duplication runs through torch on
    that device (the same keys, only faster)."""
    if n > space:
        raise ValueError("more distinct keys requested than the space holds")
    if device is not None:
        return _distinct_keys_torch(space, n, rng, device)
    found = np.empty(0, dtype=np.uint64)
    first_pos = np.empty(0, dtype=np.int64)
    drawn = 0
    while found.shape[0] < n:
        keys = _draw_keys(space, n - found.shape[0], found.shape[0], rng).astype(np.uint64)
        allk = np.concatenate([found, keys])
        allpos = np.concatenate([first_pos, drawn + np.arange(keys.shape[0], dtype=np.int64)])
        drawn += keys.shape[0]
        uk, ui = np.unique(allk, return_index=True)
        order = np.argsort(allpos[ui], kind="stable")
        found = uk[order]
        first_pos = allpos[ui][order]
    return np.sort(found[:n])


def _draw_keys(space: int, need: int, have: int, rng: np.random.Generator) -> np.ndarray:
    """One round of draws, inflated by the expected collision rate."""
    frac = min(0.999, (have + need) / space)
    k = max(1024, int(need * (1.05 - math.log1p(-frac) * 1.1)))
    parts = []
    for s0 in range(0, k, _CHUNK):
        parts.append(rng.integers(0, space, size=min(_CHUNK, k - s0), dtype=np.int64))
    return np.concatenate(parts)


def _distinct_keys_torch(space: int, n: int, rng: np.random.Generator, device) -> np.ndarray:
    import torch

    found = torch.empty(0, dtype=torch.int64, device=device)
    first_pos = torch.empty(0, dtype=torch.int64, device=device)
    drawn = 0
    while found.shape[0] < n:
        keys = torch.from_numpy(_draw_keys(space, n - found.shape[0], found.shape[0], rng)).to(device)
        allk = torch.cat([found, keys])
        allpos = torch.cat([first_pos, drawn + torch.arange(keys.shape[0], dtype=torch.int64, device=device)])
        drawn += keys.shape[0]
        uk, inv = torch.unique(allk, sorted=True, return_inverse=True)
        fp = torch.full((uk.shape[0],), drawn, dtype=torch.int64, device=device)
        fp.scatter_reduce_(0, inv, allpos, reduce="amin")
        order = torch.argsort(fp)
        found = uk[order]
        first_pos = fp[order]
        del allk, allpos, inv, uk, fp, order
    out = torch.sort(found[:n]).values.cpu().numpy().view(np.uint64)
    return out.copy()


def st_dense(n: int = 512, m: int = 4096):
    """ST-Dense (Sec. 6): four relations [n]^3, then three relations
    F x [m] x [m] with first-attribute sets F = {0,1}, {0,2}, {1,2}."""
    cube = full_cube(n)
    return [cube, cube.copy(), cube.copy(), cube.copy()] + \
        [prefixed_square(np.array(f, dtype=np.uint32), m) for f in ((0, 1), (0, 2), (1, 2))]


def st_sparse(n: int = 512, domain: int = 5120, m: int = 4096, m_domain: int = 40960, seed: int = 0,
              device: str | None = None):
    """ST-Sparse (Sec. 6): four relations of n^3 distinct tuples drawn
    uniformly from [domain]^3, then three relations that keep ST-Dense's
    first-attribute sets {0,1}, {0,2}, {1,2} and hold, under each first
    value, m^2 distinct pairs drawn uniformly from [m_domain]^2.  Each
    relation is lexicographically sorted; relation j draws from seed + j.
    ``device`` moves the de-duplication to torch on that device."""
    out = []
    for j in range(4):
        k = _distinct_keys(domain ** 3, n ** 3, _rng(seed + j), device)
        a = (k // np.uint64(domain * domain)).astype(np.uint32)
        b = ((k // np.uint64(domain)) % np.uint64(domain)).astype(np.uint32)
        c = (k % np.uint64(domain)).astype(np.uint32)
        out.append(np.stack([a, b, c], axis=1))
    for j, fs in enumerate(((0, 1), (0, 2), (1, 2))):
        rng = _rng(seed + 4 + j)
        parts = []
        for f in fs:
            k = _distinct_keys(m_domain * m_domain, m * m, rng, device)
            b = (k // np.uint64(m_domain)).astype(np.uint32)
            c = (k % np.uint64(m_domain)).astype(np.uint32)
            parts.append(np.stack([np.full(k.shape[0], f, dtype=np.uint32), b, c], axis=1))
        out.append(np.concatenate(parts))
    return out
