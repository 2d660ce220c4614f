"""Relations of arity 1 to 3 (include/honeycomb_kary.h): the k-level CoCo
index of Sec. 4 and Generic Join over it (Sec. 5), for hypergraph queries
such as the paper's Loomis-Whitney (LW) and Clover-Triangle (CT) queries
(Table "Queries").  Argument marshalling only; the work runs in the
library's CUDA kernels.

    build_kindex(rows, level_cols)     sort + k-level CoCo
    build_kindex(.., seeds, shares)    the same per HyperCube partition (Sec. 4)
    choose_korder(query, indexes)      Sec. 5.2-5.3: loop order of least estimated cost
    run_kjoin(query, indexes, mode)    Generic Join in every HyperCube cell
    atom_shares(query, shares, seeds)  per atom, the seeds and shares of its columns
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Sequence

import torch

from . import Result, _ResultHandle, _alias, _lib, _stream_ptr


@dataclass(frozen=True)
class KQuery:
    """Full conjunctive query over atoms of arity 1..3 (Eq. "full:cq").

    ``atoms[j]`` is the tuple of variables of atom j: column c of its
    relation holds variable atoms[j][c].  ``order`` is the loop order
    (default 0, 1, ...)."""
    n_vars: int
    atoms: tuple
    order: tuple | None = None

    def loop_order(self) -> tuple:
        return tuple(range(self.n_vars)) if self.order is None else tuple(self.order)

    def with_order(self, order) -> "KQuery":
        return KQuery(self.n_vars, self.atoms, tuple(order))

    def level_cols(self, j: int) -> tuple:
        """Columns of atom j in loop order of their variables: the level
        order an index needs for atom j under this query's loop order."""
        rank = {v: i for i, v in enumerate(self.loop_order())}
        a = self.atoms[j]
        return tuple(sorted(range(len(a)), key=lambda c: rank[a[c]]))

    def _c(self) -> _lib.hc_kquery:
        q = _lib.hc_kquery()
        q.n_vars = self.n_vars
        q.n_atoms = len(self.atoms)
        for j, a in enumerate(self.atoms):
            q.atoms[j].arity = len(a)
            for c, v in enumerate(a):
                q.atoms[j].var[c] = v
        for i, v in enumerate(self.loop_order()):
            q.order[i] = v
        return q


# Table "Queries": LW Q(X,Y,Z,U) with X=0, Y=1, Z=2, U=3; CT Q(U,X,Y,Z) with U=0, X=1, Y=2, Z=3.
LW = KQuery(4, ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)))
CT = KQuery(4, ((0, 1, 2), (0, 1, 3), (0, 2, 3)))


class KIndex:
    """A k-level CoCo index (library-owned device memory)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        v = _lib.hc_kindex_view()
        _lib.check(_lib.load().hc_kindex_get_view(self._h, ctypes.byref(v)), "hc_kindex_get_view")
        self.n, self.arity, self.packed = v.n, v.arity, bool(v.packed)
        self.level_cols = tuple(v.level_cols[d] for d in range(v.arity))
        self.len = tuple(int(v.len[d]) for d in range(v.arity))
        self.max_value = tuple(int(v.max_value[d]) for d in range(v.arity))
        self.ms_sort, self.ms_levels = v.ms_sort, v.ms_levels
        self.n_parts = int(v.n_parts) if v.n_parts else 1
        self.shares = tuple(int(v.shares[c]) for c in range(v.arity))
        self.seeds = tuple(int(v.seeds[c]) for c in range(v.arity))
        self._view = v

    @classmethod
    def from_stats(cls, n: int, lengths: Sequence[int], max_value: Sequence[int],
                   level_cols: Sequence[int] | None = None) -> "KIndex":
        """Statistics-only index for planning (no GPU, no data): l_d per
        level (the last is n) and the largest value of each level."""
        k = len(lengths)
        cols = None if level_cols is None else (ctypes.c_uint8 * 3)(*(list(level_cols) + [0] * (3 - k)))
        ls = (ctypes.c_uint64 * 3)(*(list(lengths) + [0] * (3 - k)))
        mv = (ctypes.c_uint32 * 3)(*(list(max_value) + [0] * (3 - k)))
        out = ctypes.c_void_p()
        _lib.check(_lib.load().hc_kindex_from_stats(n, k, cols, ls, mv, ctypes.byref(out)), "hc_kindex_from_stats")
        return cls(out.value)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("index already freed")
        return self._h

    def v(self, d: int) -> torch.Tensor:
        """V_d as an int32 CUDA tensor aliasing the index."""
        return _alias(self._view.d_v[d], (self.len[d],), torch.int32, self)

    def o(self, d: int) -> torch.Tensor:
        """O_d (d < arity-1) as an int32 CUDA tensor aliasing the index."""
        if d >= self.arity - 1:
            raise IndexError("the last level has no offsets")
        return _alias(self._view.d_o[d], (self.len[d] + 1,), torch.int32, self)

    def bpref(self) -> torch.Tensor | None:
        """B^pref (first row of each partition, [n_parts + 1]), or None when
        unpartitioned."""
        if not self._view.d_bpref:
            return None
        return _alias(self._view.d_bpref, (self.n_parts + 1,), torch.int32, self)

    def level0_start(self) -> torch.Tensor | None:
        """First level-0 entry of each partition ([n_parts + 1]), or None
        when unpartitioned."""
        if not self._view.d_level0_start:
            return None
        return _alias(self._view.d_level0_start, (self.n_parts + 1,), torch.int32, self)

    def free(self) -> None:
        if self._h is not None:
            _lib.load().hc_kindex_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_kindex(rows: torch.Tensor, level_cols: Sequence[int] | None = None, check_duplicates: bool = False,
                 stream=None, time_kernels: bool = False, seeds: Sequence[int] | None = None,
                 shares: Sequence[int] | None = None) -> KIndex:
    """k-level CoCo of a relation given as an (n, k) 32-bit CUDA tensor, k = 1..3,
    with level d holding column level_cols[d] (default 0, 1, ..).  With
    ``shares`` (and ``seeds``), one per column, the relation is partitioned
    for HyperCube shares first (Sec. 4) and each partition gets its own
    trie."""
    if not isinstance(rows, torch.Tensor) or not rows.is_cuda or rows.dim() != 2 or rows.element_size() != 4:
        raise TypeError("rows must be an (n, k) 32-bit CUDA tensor")
    r = rows.contiguous()
    k = r.shape[1]
    cols = None
    if level_cols is not None:
        cols = (ctypes.c_uint8 * _lib.HC_KMAX_ARITY)(*([int(c) for c in level_cols] + [0] * (3 - len(level_cols))))
    flags = (_lib.HC_BUILD_CHECK_DUPLICATES if check_duplicates else 0) | (
        _lib.HC_BUILD_TIME_KERNELS if time_kernels else 0)
    out = ctypes.c_void_p()
    ptr = ctypes.c_void_p(r.data_ptr() if r.numel() else 0)
    if shares is None:
        st = _lib.load().hc_build_kindex(ptr, r.shape[0], k, cols, flags, ctypes.c_void_p(_stream_ptr(stream)),
                                         ctypes.byref(out))
        _lib.check(st, "hc_build_kindex")
    else:
        if len(shares) != k:
            raise ValueError("one share per column")
        sd = list(seeds) if seeds is not None else [0] * k
        if len(sd) != k:
            raise ValueError("one seed per column")
        sh = (ctypes.c_uint32 * 3)(*([int(x) for x in shares] + [1] * (3 - k)))
        se = (ctypes.c_uint32 * 3)(*([int(x) & 0xFFFFFFFF for x in sd] + [0] * (3 - k)))
        st = _lib.load().hc_build_kindex_partitioned(ptr, r.shape[0], k, cols, se, sh, flags,
                                                     ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out))
        _lib.check(st, "hc_build_kindex_partitioned")
    return KIndex(out.value)


def atom_shares(query: KQuery, shares: Sequence[int], seeds: Sequence[int] | None = None) -> list:
    """Per atom j, (seeds, shares) of its columns for variable shares
    ``shares[v]`` and seeds ``seeds[v]`` (default v + 1): the arguments of
    build_kindex that partition atom j for the HyperCube cells of these
    shares."""
    sd = list(seeds) if seeds is not None else [v + 1 for v in range(query.n_vars)]
    return [(tuple(sd[v] for v in a), tuple(int(shares[v]) for v in a)) for a in query.atoms]


def _kindex_array(indexes):
    arr = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def kplan_cost(query: KQuery, indexes: Sequence[KIndex]) -> dict:
    """Estimated cost per loop of the query's order, and domain estimates (host only)."""
    q = query._c()
    ptr, keep = _kindex_array(indexes)
    lc = (ctypes.c_double * _lib.HC_MAX_VARS)()
    dm = (ctypes.c_double * _lib.HC_MAX_VARS)()
    _lib.check(_lib.load().hc_kplan_cost(ctypes.byref(q), ptr, lc, dm), "hc_kplan_cost")
    return {"level_cost": list(lc)[:query.n_vars], "dom": list(dm)[:query.n_vars]}


def choose_korder(query: KQuery, indexes: Sequence[KIndex]) -> tuple:
    """Loop order of least estimated cost (host only)."""
    q = query._c()
    ptr, keep = _kindex_array(indexes)
    out = (ctypes.c_uint8 * _lib.HC_MAX_VARS)()
    _lib.check(_lib.load().hc_choose_korder(ctypes.byref(q), ptr, out), "hc_choose_korder")
    return tuple(out[i] for i in range(query.n_vars))


def run_kjoin(query: KQuery, indexes: Sequence[KIndex], mode: str = "count", stats: bool = False,
              item_grain: int = 0, block_threads: int = 0, time_kernels: bool = False, stream=None,
              cell_counts: bool = False, pair_min: int = 0) -> Result:
    """Generic Join of a k-ary query in every HyperCube cell (the shares
    come from the indexes, see build_kindex); tuples (materialize) come back
    as a (count, n_vars) int32 CUDA tensor in variable-id order, in no fixed
    order; ``cell_counts`` adds the count of each cell (int64, cell id = the
    mixed radix of the variables' coordinates, variable 0 most
    significant); ``pair_min``: last-loop bindings with at least this many
    candidates are searched warp-wide (0: the library's 32, 0xFFFFFFFF:
    never)."""
    if len(indexes) != len(query.atoms):
        raise ValueError("one index per atom")
    if mode not in ("count", "materialize"):
        raise ValueError("mode is 'count' or 'materialize'")
    q = query._c()
    arr = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
    prm = _lib.hc_kjoin_params()
    prm.mode = _lib.HC_MODE_COUNT if mode == "count" else _lib.HC_MODE_MATERIALIZE
    prm.flags = ((_lib.HC_FLAG_STATS if stats else 0) | (_lib.HC_FLAG_TIME_KERNELS if time_kernels else 0)
                 | (_lib.HC_FLAG_CELL_COUNTS if cell_counts else 0))
    prm.item_grain = item_grain
    prm.block_threads = block_threads
    prm.pair_min = pair_min
    lib = _lib.load()
    out = ctypes.c_void_p()
    _lib.check(lib.hc_run_kjoin(ctypes.byref(q), ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)),
                                ctypes.byref(prm), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out)),
               "hc_run_kjoin")
    holder = _ResultHandle(out.value)
    v = _lib.hc_result_view()
    _lib.check(lib.hc_result_get(ctypes.c_void_p(holder.h), ctypes.byref(v)), "hc_result_get")
    res = Result(count=v.count, n_cells=v.n_cells, work=v.work, n_items=v.n_items,
                 ms_join_kernel=v.ms_join_kernel, n_join_launches=v.n_join_launches)
    if v.d_cell_counts:
        res.cell_counts = _alias(v.d_cell_counts, (v.n_cells,), torch.int64, holder).clone()
    if v.d_tuples:
        res.tuples = _alias(v.d_tuples, (v.n_tuples, query.n_vars), torch.int32, holder).clone()
    elif mode == "materialize":
        res.tuples = torch.empty((0, query.n_vars), dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    holder.free()
    return res
