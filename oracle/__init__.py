"""CPU oracle for the HoneyComb hot path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's timed
CPU-baseline leg may import this package.  The product path (the CUDA
library and its binding) never does, and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, compiled with gcc into
``oracle/_build``); this module only marshals numpy arrays.  Functions and
the passages they follow:

* ``coco_build``   -- the CoCo trie of a binary relation (Sec. 4, Fig.
  "cocoindex"): V1 (distinct first values), O1 (run starts, O1[l1] = n), V2.
* ``partition``    -- HyperCube partitioning of one relation (Sec. 4,
  Example "partition"): R~, B, B^pref and the per-partition CoCo.
* ``gj_count`` / ``gj_enumerate`` -- Generic Join of a full conjunctive
  query of binary atoms (Eq. "full:cq", Sec. 2 "Generic Join Algorithm",
  Sec. 5 intersection and level restriction).
* ``tuple_cells``  -- the HyperCube cell of each output tuple (Sec. 5:
  the outputs of different cells are disjoint).
* ``share``        -- h_i(x) mod P_i, read as ((fmix32(x ^ seed) * P) >> 32).
* ``kcoco`` / ``kpartition`` -- the k-level CoCo of a relation of arity 1..3
  (Sec. 4, Fig. "cocoindex"), and its HyperCube partitioning (Sec. 4,
  "Preprocessor", Example "partition"): R~, B, B^pref and one k-level CoCo
  per partition, concatenated.
* ``kgj``          -- Generic Join over atoms of arity 1..3 (``oracle_kary.c``).

A query is ``(n_vars, atoms)`` with ``atoms`` a list of ``(var0, var1)``:
the relation bound to atom j holds pairs whose column 0 is variable var0
and column 1 is variable var1; ``var1 = -1`` makes a unary atom over column
0 (the set of its values).  Output tuples list values in variable-id order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")

OC_ECAP = 3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` and ``oracle_kary.c`` with gcc into ``oracle/_build/liboracle.so``."""
    out_dir = os.path.join(_HERE, "_build")
    so = os.path.join(out_dir, "liboracle.so")
    srcs = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_kary.c")]
    if force or not os.path.exists(so) or any(os.path.getmtime(so) < os.path.getmtime(s) for s in srcs):
        os.makedirs(out_dir, exist_ok=True)
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", *srcs, "-o", tmp])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    lib = ctypes.CDLL(build())
    vp = ctypes.c_void_p
    u64 = ctypes.c_uint64
    lib.oc_fmix32.restype = ctypes.c_uint32
    lib.oc_fmix32.argtypes = [ctypes.c_uint32]
    lib.oc_share.restype = ctypes.c_uint32
    lib.oc_share.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
    lib.oc_has_duplicates.restype = ctypes.c_int
    lib.oc_has_duplicates.argtypes = [vp, u64]
    lib.oc_coco_build.restype = ctypes.c_int
    lib.oc_coco_build.argtypes = [vp, u64, ctypes.c_int, _u32p, _u64p, _u32p, ctypes.POINTER(u64)]
    lib.oc_partition.restype = ctypes.c_int
    lib.oc_partition.argtypes = [vp, u64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint32, _u32p, _u64p, _u64p, _u32p,
                                 _u64p, _u64p, ctypes.POINTER(u64)]
    lib.oc_gj_count.restype = ctypes.c_int
    lib.oc_gj_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp), _u64p, _i32p, _i32p,
                                _i32p, vp, u64, ctypes.c_int, ctypes.POINTER(u64),
                                ctypes.POINTER(u64), vp, u64, ctypes.POINTER(u64)]
    lib.oc_gj_enumerate.restype = ctypes.c_int
    lib.oc_gj_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp), _u64p, _i32p,
                                    _i32p, _i32p, vp, u64, vp, u64, ctypes.POINTER(u64)]
    lib.oc_kgj.restype = ctypes.c_int
    lib.oc_kgj.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.POINTER(vp), _u64p, vp, vp, u64,
                           ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.c_int]
    lib.oc_tuple_cells.restype = ctypes.c_int
    lib.oc_tuple_cells.argtypes = [vp, u64, ctypes.c_int, _u32p, _u32p, _u32p]
    _LIB = lib
    return lib


def _pairs(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    if a.size == 0:
        return np.zeros((0, 2), dtype=np.uint32)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("a relation is an (n, 2) array of pairs")
    return a


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def fmix32(x: int) -> int:
    return int(_lib().oc_fmix32(int(x) & 0xFFFFFFFF))


def share(x: int, seed: int, p: int) -> int:
    """h(x) mod P read as (fmix32(x ^ seed) * P) >> 32."""
    return int(_lib().oc_share(int(x) & 0xFFFFFFFF, int(seed) & 0xFFFFFFFF, int(p)))


def has_duplicates(pairs) -> bool:
    p = _pairs(pairs)
    return bool(_lib().oc_has_duplicates(p.ctypes.data, p.shape[0]))


def coco_build(pairs, attr_order: int = 0):
    """(V1 uint32[l1], O1 uint64[l1+1], V2 uint32[n]) of the relation."""
    p = _pairs(pairs)
    n = p.shape[0]
    v1 = np.zeros(max(n, 1), dtype=np.uint32)
    o1 = np.zeros(n + 1, dtype=np.uint64)
    v2 = np.zeros(max(n, 1), dtype=np.uint32)
    l1 = ctypes.c_uint64(0)
    _check(_lib().oc_coco_build(p.ctypes.data, n, int(attr_order), v1, o1, v2, ctypes.byref(l1)),
           "coco_build")
    l = l1.value
    return v1[:l].copy(), o1[:l + 1].copy(), v2[:n].copy()


def partition(pairs, attr_order: int, seed_a: int, pa: int, seed_b: int, pb: int) -> dict:
    """Partitioned relation and per-partition CoCo (global offsets)."""
    p = _pairs(pairs)
    n = p.shape[0]
    npart = pa * pb
    rt = np.zeros(max(2 * n, 1), dtype=np.uint32)
    hist = np.zeros(npart, dtype=np.uint64)
    pref = np.zeros(npart + 1, dtype=np.uint64)
    v1 = np.zeros(max(n, 1), dtype=np.uint32)
    o1 = np.zeros(n + 1, dtype=np.uint64)
    start = np.zeros(npart + 1, dtype=np.uint64)
    l1 = ctypes.c_uint64(0)
    _check(_lib().oc_partition(p.ctypes.data, n, int(attr_order), seed_a, pa, seed_b, pb, rt, hist,
                               pref, v1, o1, start, ctypes.byref(l1)), "partition")
    l = l1.value
    return {"rt": rt[:2 * n].reshape(n, 2).copy(), "B": hist, "Bpref": pref, "V1": v1[:l].copy(),
            "O1": o1[:l + 1].copy(), "lvl1_start": start}


def _query_args(n_vars, atoms, rels, order):
    na = len(atoms)
    if len(rels) != na:
        raise ValueError("one relation per atom")
    rels = [_pairs(r) for r in rels]
    ptrs = (ctypes.c_void_p * na)(*[r.ctypes.data if r.shape[0] else None for r in rels])
    ns = np.array([r.shape[0] for r in rels], dtype=np.uint64)
    v0 = np.array([a[0] for a in atoms], dtype=np.int32)
    v1 = np.array([a[1] for a in atoms], dtype=np.int32)
    od = np.array(list(range(n_vars)) if order is None else list(order), dtype=np.int32)
    if od.shape[0] != n_vars:
        raise ValueError("order must list every variable once")
    return rels, ptrs, ns, v0, v1, od


def _filter_arg(filt):
    if filt is None:
        return None, None, 0
    f = np.ascontiguousarray(np.unique(np.asarray(filt, dtype=np.uint32)))
    return f, (f.ctypes.data if f.shape[0] else None), f.shape[0]


def gj_count(n_vars: int, atoms, rels, order=None, filt=None, nthreads: int = 1,
             per_top: bool = False):
    """Count of the query; returns (count, work, per_top_counts or None).

    ``filt`` restricts the first loop's variable to the given values
    (selection pushed into the atoms, Eq. "full:cq" remark on predicates).
    ``per_top`` also returns the count for each loop-1 value (ascending).
    """
    rels, ptrs, ns, v0, v1, od = _query_args(n_vars, atoms, rels, order)
    f, fptr, nf = _filter_arg(filt)
    cnt, work, ntop = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    lib = _lib()
    if per_top:
        _check(lib.oc_gj_count(n_vars, len(atoms), ptrs, ns, v0, v1, od, fptr, nf, 1,
                               ctypes.byref(cnt), None, None, 0, ctypes.byref(ntop)), "gj_count")
        buf = np.zeros(max(ntop.value, 1), dtype=np.uint64)
        _check(lib.oc_gj_count(n_vars, len(atoms), ptrs, ns, v0, v1, od, fptr, nf, int(nthreads),
                               ctypes.byref(cnt), ctypes.byref(work), buf.ctypes.data, buf.shape[0],
                               ctypes.byref(ntop)), "gj_count")
        return cnt.value, work.value, buf[:ntop.value].copy()
    _check(lib.oc_gj_count(n_vars, len(atoms), ptrs, ns, v0, v1, od, fptr, nf, int(nthreads),
                           ctypes.byref(cnt), ctypes.byref(work), None, 0, ctypes.byref(ntop)),
           "gj_count")
    return cnt.value, work.value, None


def kcoco(rows, level_cols=None) -> dict:
    """k-level CoCo of a relation of arity k = 1..3 (Sec. 4): the rows
    sorted lexicographically with column level_cols[0] first; for each level
    d, V_d = the level-d value of each distinct prefix of length d+1 (in
    sorted order) and, for d < k-1, O_d[e] = the position in level d+1 of
    prefix e's first child, O_d[l_d] = l_{d+1}; the last level holds every
    row.  Returns {"V": [V_0, ..], "O": [O_0, ..]} as uint32 arrays."""
    r = np.asarray(rows, dtype=np.uint32)
    k = r.shape[1]
    cols = list(range(k)) if level_cols is None else list(level_cols)
    r = r[:, cols]
    if r.shape[0]:
        r = r[np.lexsort(r.T[::-1])]  # a library sort, lexicographic by level 0, 1, ..
    first = []  # per level: the sorted rows' index where each distinct prefix starts
    for d in range(k):
        if r.shape[0] == 0:
            first.append(np.zeros(0, dtype=np.int64))
            continue
        pref = r[:, :d + 1]
        new = np.ones(r.shape[0], dtype=bool)
        new[1:] = np.any(pref[1:] != pref[:-1], axis=1)
        first.append(np.flatnonzero(new))
    V = [r[first[d], d].astype(np.uint32) for d in range(k)]
    O = []
    for d in range(k - 1):
        o = np.searchsorted(first[d + 1], first[d]).astype(np.uint32)
        O.append(np.append(o, np.uint32(first[d + 1].shape[0])))
    return {"V": V, "O": O}


def kpartition(rows, seeds, shares, level_cols=None) -> dict:
    """HyperCube partitioning of a relation of arity k = 1..3 and one
    k-level CoCo per partition (Sec. 4, "Preprocessor").

    Column c of a row has the partition identifier s_c = h_c(x_c) (``share``
    with seeds[c], shares[c]); the row's partition is the mixed-radix number
    of (s_0, .., s_{k-1}), column 0 most significant, so partitions are
    numbered in the lexicographic order of their identifiers.  Returns

    * ``B``       -- rows in each partition;
    * ``Bpref``   -- where each partition starts in R~ (an exclusive prefix
      of B, the reading of B^pref that the paper's example uses: the
      partition (0,1,0) "starts at" B^pref[0,1,0]), with Bpref[np] = n;
    * ``rt``      -- R~: the partitions concatenated in that order, each
      partition's rows sorted in level order (columns in the input order);
    * ``V``, ``O`` -- the levels of every partition's k-level CoCo
      (``kcoco``), concatenated in partition order, O_d shifted to point into
      the concatenated level d+1 (O_d[l_d] = l_{d+1});
    * ``l0start`` -- where each partition's level 0 starts in V_0, with
      l0start[np] = l_0."""
    r = np.asarray(rows, dtype=np.uint32)
    k = r.shape[1]
    cols = list(range(k)) if level_cols is None else list(level_cols)
    shares = [int(x) for x in shares]
    npart = int(np.prod(shares))
    pid = tuple_cells(r, seeds, shares).astype(np.int64) if r.shape[0] else np.zeros(0, dtype=np.int64)
    B = np.bincount(pid, minlength=npart).astype(np.uint64)
    Bpref = np.concatenate([[0], np.cumsum(B)]).astype(np.uint64)
    V = [[] for _ in range(k)]
    O = [[] for _ in range(k - 1)]
    rt = []
    size = [0] * k  # entries of each level before the current partition
    l0start = [0]
    for p in range(npart):
        part = r[pid == p]
        c = kcoco(part, cols)
        if part.shape[0]:
            lv = part[:, cols]
            rt.append(part[np.lexsort(lv.T[::-1])])
        for d in range(k):
            V[d].append(c["V"][d])
        for d in range(k - 1):
            O[d].append(c["O"][d][:-1].astype(np.uint64) + np.uint64(size[d + 1]))
        size = [size[d] + c["V"][d].shape[0] for d in range(k)]
        l0start.append(size[0])
    Vc = [np.concatenate(V[d]).astype(np.uint32) for d in range(k)]
    Oc = [np.append(np.concatenate(O[d]), np.uint64(size[d + 1])).astype(np.uint32) for d in range(k - 1)]
    rt = np.concatenate(rt) if rt else np.zeros((0, k), dtype=np.uint32)
    return {"B": B, "Bpref": Bpref, "rt": rt, "V": Vc, "O": Oc, "l0start": np.array(l0start, dtype=np.uint64)}


def gj_enumerate(n_vars: int, atoms, rels, order=None, filt=None) -> np.ndarray:
    """All output tuples, (count, n_vars) uint32 in variable-id order."""
    rels, ptrs, ns, v0, v1, od = _query_args(n_vars, atoms, rels, order)
    f, fptr, nf = _filter_arg(filt)
    cnt, _, _ = gj_count(n_vars, atoms, rels, order, filt)
    out = np.zeros(max(cnt, 1) * n_vars, dtype=np.uint32)
    nout = ctypes.c_uint64(0)
    _check(_lib().oc_gj_enumerate(n_vars, len(atoms), ptrs, ns, v0, v1, od, fptr, nf,
                                  out.ctypes.data, max(cnt, 1), ctypes.byref(nout)), "gj_enumerate")
    return out[:nout.value * n_vars].reshape(nout.value, n_vars).copy()


def tuple_cells(tuples, seeds, shares) -> np.ndarray:
    """Cell id of each tuple: mixed radix of (s_1..s_n) in variable-id order."""
    t = np.ascontiguousarray(np.asarray(tuples, dtype=np.uint32))
    nv = len(shares)
    t = t.reshape(-1, nv)
    out = np.zeros(max(t.shape[0], 1), dtype=np.uint32)
    _check(_lib().oc_tuple_cells(t.ctypes.data if t.shape[0] else None, t.shape[0], nv,
                                 np.asarray(seeds, dtype=np.uint32),
                                 np.asarray(shares, dtype=np.uint32), out), "tuple_cells")
    return out[:t.shape[0]].copy()


# Query shapes of the paper's Table "Queries" (variables numbered X=0, Y=1,
# Z=2, U=3, V=4 in the table's head order).
TRIANGLE = (3, [(0, 1), (1, 2), (0, 2)])                     # Q1: R(X,Y) S(Y,Z) T(X,Z)
FOUR_CYCLE = (4, [(0, 1), (0, 2), (1, 3), (2, 3)])           # Q2: R1(X,Y) R2(X,Z) R3(Y,U) R4(Z,U)
FOUR_DIAMOND = (4, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2)])  # Q4
FOUR_CLIQUE = (4, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (0, 3)])  # Q6
TWO_TRIANGLE = (5, [(0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)])  # Q8


def kgj(n_vars: int, atoms, rels, order=None, tuples: bool = False, cap: int = 1 << 22, work: bool = False,
        nthreads: int = 1):
    """Generic Join over atoms of arity 1 to 3 (``oracle_kary.c``): atoms[j]
    is a tuple of variable ids, rels[j] an (n, len(atoms[j])) array (a set).
    Returns the output count, or (count, tuples in variable-id order) with
    ``tuples`` (at most ``cap`` of them); with ``work``, (count, work) or
    (count, tuples, work), work being the sum over loops and bindings of
    (number of lists) * (shortest list length).  ``nthreads`` > 1 counts on
    that many threads (ignored with ``tuples``)."""
    na = len(atoms)
    if na != len(rels):
        raise ValueError("one relation per atom")
    arity = np.array([len(a) for a in atoms], dtype=np.int32)
    vars_ = np.zeros(3 * na, dtype=np.int32)
    keep = []
    ptrs = (ctypes.c_void_p * na)()
    ns = np.zeros(na, dtype=np.uint64)
    for j, (a, r) in enumerate(zip(atoms, rels)):
        if not 1 <= len(a) <= 3:
            raise ValueError("atoms of arity 1 to 3")
        vars_[3 * j:3 * j + len(a)] = a
        arr = np.ascontiguousarray(np.asarray(r, dtype=np.uint32).reshape(-1, len(a)))
        keep.append(arr)
        ptrs[j] = arr.ctypes.data if arr.size else None
        ns[j] = arr.shape[0]
    ordv = None
    if order is not None:
        ordv = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    out = np.zeros((cap if tuples else 0, n_vars), dtype=np.uint32)
    cnt = ctypes.c_uint64(0)
    wk = ctypes.c_uint64(0)
    _check(_lib().oc_kgj(n_vars, na, arity, vars_, ptrs, ns,
                         ordv.ctypes.data if ordv is not None else None,
                         out.ctypes.data if tuples else None, cap if tuples else 0, ctypes.byref(cnt),
                         ctypes.byref(wk) if work else None, int(nthreads)), "kgj")
    extra = (wk.value,) if work else ()
    if not tuples:
        return (cnt.value, *extra) if work else cnt.value
    if cnt.value > cap:
        raise OracleError("kgj: more tuples than cap")
    return (cnt.value, out[:cnt.value].copy(), *extra)
