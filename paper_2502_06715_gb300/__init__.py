"""GB300-native HoneyComb: Generic Join over CoCo indexes with HyperCube shares.

Python binding of the C ABI (include/honeycomb.h).  The functions here only
marshal arguments: every step of the join runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.

    build_index(pairs, attr_order)            Sec. 4: radix sort + CoCo
    choose_shares(query, indexes, P)          Sec. 5.2-5.3: cost model, plan decision
    run_join(query, indexes, shares, ...)     Sec. 4-5: partitioning + Generic Join
    partition_index(index, ...)               Sec. 4: HyperCube partitioning alone
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Sequence

import torch

from . import _lib
from ._lib import HoneycombError

__all__ = ["Query", "Index", "Partitioned", "Result", "build_index", "choose_shares", "run_join",
           "partition_index", "plan_cost", "HoneycombError", "TRIANGLE", "FOUR_CYCLE", "FOUR_DIAMOND", "FOUR_CLIQUE",
           "TWO_TRIANGLE", "library_path", "kernel_launches", "Batch", "run_join_async", "Pending", "join_footprint"]


def library_path() -> str:
    return _lib.library_path()


def kernel_launches() -> int:
    """Kernels the library has launched in this process (host counter)."""
    return int(_lib.load().hc_kernel_launches())


class _DeviceArray:
    """__cuda_array_interface__ over library-owned device memory."""

    def __init__(self, ptr: int, shape: tuple, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}


def _alias(ptr, shape, dtype: torch.dtype, owner) -> torch.Tensor:
    """A torch tensor aliasing library memory (valid while `owner` lives)."""
    n = 1
    for s in shape:
        n *= s
    if n == 0 or not ptr:
        return torch.empty(shape, dtype=dtype, device="cuda")
    typestr = {torch.int32: "<i4", torch.int64: "<i8"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, tuple(shape), typestr, owner), device="cuda")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass(frozen=True)
class Query:
    """Full conjunctive query of binary atoms (Eq. "full:cq").

    ``atoms[j] = (var0, var1)``: column 0 of atom j's relation holds variable
    var0, column 1 variable var1; ``var1 = None`` (or -1) makes a unary atom
    over column 0.  ``order`` is the Generic Join loop order (default:
    variables 0, 1, ...).
    """
    n_vars: int
    atoms: tuple
    order: tuple | None = None

    def loop_order(self) -> tuple:
        return tuple(range(self.n_vars)) if self.order is None else tuple(self.order)

    def with_order(self, order) -> "Query":
        return Query(self.n_vars, self.atoms, tuple(order))

    def attr_order(self, j: int) -> int:
        """Attribute order an index needs for atom j under the loop order."""
        rank = {v: i for i, v in enumerate(self.loop_order())}
        a, b = self.atoms[j]
        if b is None or b < 0:
            return 0
        return 0 if rank[a] < rank[b] else 1

    def with_atoms(self, extra) -> "Query":
        return Query(self.n_vars, tuple(self.atoms) + tuple(extra), self.order)

    def _c(self) -> _lib.hc_query:
        q = _lib.hc_query()
        q.n_vars = self.n_vars
        q.n_atoms = len(self.atoms)
        for j, (a, b) in enumerate(self.atoms):
            q.atoms[j].var0 = a
            q.atoms[j].var1 = 0xFF if (b is None or b < 0) else b
        for i, v in enumerate(self.loop_order()):
            q.order[i] = v
        return q


# Query shapes of the paper's Table "Queries", variables X=0, Y=1, Z=2, U=3, V=4.
TRIANGLE = Query(3, ((0, 1), (1, 2), (0, 2)))
FOUR_CYCLE = Query(4, ((0, 1), (0, 2), (1, 3), (2, 3)))
FOUR_DIAMOND = Query(4, ((0, 1), (0, 2), (1, 3), (2, 3), (1, 2)))
FOUR_CLIQUE = Query(4, ((0, 1), (0, 2), (1, 3), (2, 3), (1, 2), (0, 3)))
TWO_TRIANGLE = Query(5, ((0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)))


class Index:
    """A CoCo index (library-owned device memory)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        v = _lib.hc_index_view()
        _lib.check(_lib.load().hc_index_get_view(self._h, ctypes.byref(v)), "hc_index_get_view")
        self.n, self.l1, self.attr_order = v.n, v.l1, v.attr_order
        self.max_first, self.max_second = v.max_first, v.max_second
        self.max_run = v.max_run  # rows of the most frequent first-attribute value
        self.v1pos_n = v.v1pos_n  # entries of the V1 position map (0: V1 is searched)
        # device times when built with time_kernels=True (else 0)
        self.ms_radix_passes, self.n_radix_passes, self.ms_boundary = v.ms_radix_passes, v.n_radix_passes, v.ms_boundary
        self._view = v

    @classmethod
    def from_stats(cls, n: int, l1: int, attr_order: int = 0, max_first: int = 0, max_second: int = 0,
                   max_run: int = 0) -> "Index":
        """Statistics-only index for planning (no GPU, no data); ``max_run``,
        the rows of the most frequent first value, is optional (0: unknown)."""
        out = ctypes.c_void_p()
        _lib.check(_lib.load().hc_index_from_stats(n, l1, attr_order, max_first, max_second, max_run,
                                                   ctypes.byref(out)), "hc_index_from_stats")
        return cls(out.value)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("index already freed")
        return self._h

    def v1(self) -> torch.Tensor:
        return _alias(self._view.d_v1, (self.l1,), torch.int32, self)

    def o1(self) -> torch.Tensor:
        return _alias(self._view.d_o1, (self.l1 + 1,), torch.int32, self)

    def v2(self) -> torch.Tensor:
        return _alias(self._view.d_v2, (self.n,), torch.int32, self)

    def keys(self) -> torch.Tensor:
        return _alias(self._view.d_keys, (self.n,), torch.int64, self)

    def free(self) -> None:
        if self._h is not None:
            _lib.load().hc_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _check_pairs(pairs: torch.Tensor) -> torch.Tensor:
    if not isinstance(pairs, torch.Tensor) or not pairs.is_cuda:
        raise TypeError("pairs must be a CUDA tensor of shape (n, 2)")
    if pairs.dtype not in (torch.int32, torch.uint32) or pairs.dim() != 2 or pairs.shape[1] != 2:
        raise TypeError("pairs must be an (n, 2) int32/uint32 tensor")
    return pairs.contiguous()


def build_index(pairs: torch.Tensor, attr_order: int = 0, check_duplicates: bool = False, stream=None,
                time_kernels: bool = False, test_stall: str = "") -> Index:
    """CoCo index of a relation given as an (n, 2) uint32 CUDA tensor.  With
    time_kernels the radix passes and the run-boundary scan are timed with
    CUDA events (Index.ms_radix_passes, n_radix_passes, ms_boundary).
    ``test_stall`` ("sort" or "scan") is for testing the bounded-wait error
    path only: the first tile of that step never publishes its status."""
    p = _check_pairs(pairs)
    out = ctypes.c_void_p()
    stall = {"": 0, "sort": _lib.HC_BUILD_TEST_STALL_SORT, "scan": _lib.HC_BUILD_TEST_STALL_SCAN}[test_stall]
    flags = (_lib.HC_BUILD_CHECK_DUPLICATES if check_duplicates else 0) | (
        _lib.HC_BUILD_TIME_KERNELS if time_kernels else 0) | stall
    st = _lib.load().hc_build_index(ctypes.c_void_p(p.data_ptr() if p.numel() else 0), p.shape[0], attr_order,
                                    flags, ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out))
    _lib.check(st, "hc_build_index")
    return Index(out.value)


def set_wait_limit_ns(ns: int) -> int:
    """Set the limit of every bounded device-side wait of later launches
    (process-wide); returns the previous limit."""
    lib = _lib.load()
    prev = int(lib.hc_wait_limit_ns())
    _lib.check(lib.hc_set_wait_limit_ns(int(ns)), "hc_set_wait_limit_ns")
    return prev


def build_unary_index(values: torch.Tensor, max_value: int | None = None, stream=None) -> Index:
    """Index of a unary relation from its values, strictly ascending, as a 1-D
    uint32 CUDA tensor (int32 storage), without sorting or waiting for the GPU
    (pass ``max_value``, the last value, to avoid reading it back)."""
    if values.dim() != 1 or values.element_size() != 4 or not values.is_cuda:
        raise ValueError("values: a 1-D 32-bit CUDA tensor")
    v = values.contiguous()
    n = v.shape[0]
    if max_value is None:
        max_value = int(v[-1].item()) & 0xFFFFFFFF if n else 0
    out = ctypes.c_void_p()
    st = _lib.load().hc_build_unary_index(ctypes.c_void_p(v.data_ptr() if n else 0), n, int(max_value) & 0xFFFFFFFF,
                                          ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out))
    _lib.check(st, "hc_build_unary_index")
    ix = Index(out.value)
    ix._values = v  # the build reads it on `stream`; kept until the index goes
    return ix


class Partitioned:
    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        v = _lib.hc_partitioned_view()
        _lib.check(_lib.load().hc_partitioned_get_view(self._h, ctypes.byref(v)), "hc_partitioned_get_view")
        self.n, self.l1, self.n_parts, self.pa, self.pb = v.n, v.l1, v.n_parts, v.pa, v.pb
        self._view = v

    def keys(self):
        return _alias(self._view.d_keys, (self.n,), torch.int64, self)

    def bpref(self):
        return _alias(self._view.d_bpref, (self.n_parts + 1,), torch.int32, self)

    def v1(self):
        return _alias(self._view.d_v1, (self.l1,), torch.int32, self)

    def o1(self):
        return _alias(self._view.d_o1, (self.l1 + 1,), torch.int32, self)

    def v2(self):
        return _alias(self._view.d_v2, (self.n,), torch.int32, self)

    def lvl1_start(self):
        return _alias(self._view.d_lvl1_start, (self.n_parts + 1,), torch.int32, self)

    def free(self):
        if self._h is not None:
            _lib.load().hc_partitioned_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def partition_index(index: Index, seed_a: int, pa: int, seed_b: int, pb: int, stream=None) -> Partitioned:
    out = ctypes.c_void_p()
    st = _lib.load().hc_partition_index(index.handle, seed_a & 0xFFFFFFFF, pa, seed_b & 0xFFFFFFFF, pb,
                                        ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out))
    _lib.check(st, "hc_partition_index")
    return Partitioned(out.value)


def _index_array(indexes: Sequence[Index]):
    arr = (ctypes.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def choose_shares(query: Query, indexes: Sequence[Index], P: int = 1024) -> list[int]:
    """Shares per variable id (Sec. 5.3 plan decision)."""
    q = query._c()
    ptr, keep = _index_array(indexes)
    out = (ctypes.c_uint32 * _lib.HC_MAX_VARS)()
    _lib.check(_lib.load().hc_choose_shares(ctypes.byref(q), ptr, P, out), "hc_choose_shares")
    return [int(out[v]) for v in range(query.n_vars)]


def choose_plan(query: Query, indexes: Sequence[Index], P: int = 1024) -> tuple:
    """Loop order and shares together (Sec. 5.3): (order, shares).  Run with
    ``query.with_order(order)`` and, for atom j, an index of attr_order
    ``query.with_order(order).attr_order(j)``."""
    q = query._c()
    ptr, keep = _index_array(indexes)
    order = (ctypes.c_uint8 * _lib.HC_MAX_VARS)()
    shares = (ctypes.c_uint32 * _lib.HC_MAX_VARS)()
    _lib.check(_lib.load().hc_choose_plan(ctypes.byref(q), ptr, P, order, shares), "hc_choose_plan")
    return tuple(int(order[i]) for i in range(query.n_vars)), [int(shares[v]) for v in range(query.n_vars)]


def plan_cost(query: Query, indexes: Sequence[Index], shares: Sequence[int]) -> dict:
    """Estimated per-loop costs, domain sizes and replicated cost (Sec. 5.2)."""
    q = query._c()
    ptr, keep = _index_array(indexes)
    sh = (ctypes.c_uint32 * _lib.HC_MAX_VARS)(*([int(x) for x in shares] + [1] * (_lib.HC_MAX_VARS - len(shares))))
    lc = (ctypes.c_double * _lib.HC_MAX_VARS)()
    dom = (ctypes.c_double * _lib.HC_MAX_VARS)()
    rep = ctypes.c_double()
    _lib.check(_lib.load().hc_plan_cost(ctypes.byref(q), ptr, sh, lc, dom, ctypes.byref(rep)), "hc_plan_cost")
    n = query.n_vars
    return {"level_cost": list(lc)[:n], "dom": list(dom)[:n], "replicated": rep.value}


DEFAULT_SEEDS = (0x9E3779B9, 0x85EBCA6B, 0xC2B2AE35, 0x27D4EB2F, 0x165667B1, 0xD3A2646C, 0xFD7046C5, 0xB55A4F09)


@dataclass
class Result:
    count: int
    n_cells: int
    work: int
    n_items: int
    ms_join_kernel: float = 0.0
    n_join_launches: int = 0
    tuples: torch.Tensor | None = None
    cell_counts: torch.Tensor | None = None
    cell_profile: torch.Tensor | None = None  # (n_cells, 2) int64: work units, SM cycles
    _handle: object = field(default=None, repr=False)


def run_join(query: Query, indexes: Sequence[Index], shares: Sequence[int] | None = None,
             seeds: Sequence[int] | None = None, mode: str = "count", cell_counts: bool = False,
             stats: bool = False, item_grain: int = 0, block_threads: int = 0, stream=None,
             keep_device: bool = False, time_kernels: bool = False, merge_min: int = 0,
             merge_ratio: int = 0, out_capacity: int = 0, slice_grain: int = 0, lift: bool = True,
             lift_arena: int = 0, dir_min: int = 0, pair_min: int = 0, cell_profile: bool = False) -> Result:
    """Evaluate the query.  Tuples (materialize) come back as an
    (count, n_vars) int32 CUDA tensor in variable-id order (a copy, unless
    ``keep_device`` keeps an alias of library memory tied to the result).
    ``lift`` allows the query rewriting of Sec. 5.1 (off with ``stats``);
    ``lift_arena`` sets its device scratch, in words per warp (0: default).
    ``dir_min``: list searches in runs at least this long read the run's
    bucket directory first (0: 16; 0xFFFFFFFF: plain binary search).
    ``cell_profile``: per-cell work units and SM cycles of the warps' work on
    the cell (the skew study of Sec. 1; implies ``stats``).
    ``pair_min``: last-loop bindings whose shorter list has at least this many
    values are searched by the whole warp (0: 32; 0xFFFFFFFF: never)."""
    if len(indexes) != len(query.atoms):
        raise ValueError("one index per atom")
    q = query._c()
    ptr, keep = _index_array(indexes)
    prm = _lib.hc_join_params()
    sh = list(shares) if shares is not None else [1] * query.n_vars
    sd = list(seeds) if seeds is not None else list(DEFAULT_SEEDS)
    for v in range(_lib.HC_MAX_VARS):
        prm.shares[v] = sh[v] if v < len(sh) else 1
        prm.seeds[v] = (sd[v] if v < len(sd) else DEFAULT_SEEDS[v]) & 0xFFFFFFFF
    if mode not in ("count", "materialize"):
        raise ValueError("mode is 'count' or 'materialize'")
    prm.mode = _lib.HC_MODE_COUNT if mode == "count" else _lib.HC_MODE_MATERIALIZE
    prm.flags = ((_lib.HC_FLAG_CELL_COUNTS if cell_counts else 0) | (_lib.HC_FLAG_STATS if stats else 0)
                 | (_lib.HC_FLAG_TIME_KERNELS if time_kernels else 0) | (0 if lift else _lib.HC_FLAG_NO_LIFT)
                 | (_lib.HC_FLAG_CELL_PROFILE if cell_profile else 0))
    prm.lift_arena = int(lift_arena)
    prm.item_grain = item_grain
    prm.block_threads = block_threads
    prm.merge_min = merge_min & 0xFFFFFFFF
    prm.merge_ratio = merge_ratio & 0xFFFFFFFF
    prm.out_capacity = int(out_capacity)
    prm.slice_grain = slice_grain & 0xFFFFFFFF
    prm.dir_min = dir_min & 0xFFFFFFFF
    prm.pair_min = pair_min & 0xFFFFFFFF
    lib = _lib.load()
    out = ctypes.c_void_p()
    _lib.check(lib.hc_run_join(ctypes.byref(q), ptr, ctypes.byref(prm), ctypes.c_void_p(_stream_ptr(stream)),
                               ctypes.byref(out)), "hc_run_join")
    h = out.value
    try:
        v = _lib.hc_result_view()
        _lib.check(lib.hc_result_get(ctypes.c_void_p(h), ctypes.byref(v)), "hc_result_get")
        res = Result(count=v.count, n_cells=v.n_cells, work=v.work, n_items=v.n_items,
                     ms_join_kernel=v.ms_join_kernel, n_join_launches=v.n_join_launches)
        holder = _ResultHandle(h)
        if v.d_tuples:
            t = _alias(v.d_tuples, (v.n_tuples, query.n_vars), torch.int32, holder)
            res.tuples = t if keep_device else t.clone()
        if v.d_cell_counts:
            c = _alias(v.d_cell_counts, (v.n_cells,), torch.int64, holder)
            res.cell_counts = c if keep_device else c.clone()
        if v.d_cell_profile:
            c = _alias(v.d_cell_profile, (v.n_cells, 2), torch.int64, holder)
            res.cell_profile = c if keep_device else c.clone()
        if keep_device:
            res._handle = holder
        else:
            torch.cuda.current_stream().synchronize()
            holder.free()
        return res
    except Exception:
        lib.hc_result_free(ctypes.c_void_p(h))
        raise


def run_join_to_host(query: Query, indexes: Sequence[Index], out: torch.Tensor, stream=None, **options) -> int:
    """Evaluate the query with its tuples delivered into ``out``, a host
    (n, n_vars) int32 tensor (pinned memory lets the copies overlap the
    search), as the C ABI's hc_run_join_to_host.  Returns |Q|; raises
    HoneycombError with status HC_ERR_CAPACITY when |Q| exceeds out's rows.
    ``options`` as for ``run_join`` (mode is materialize)."""
    if len(indexes) != len(query.atoms):
        raise ValueError("one index per atom")
    if out.is_cuda or out.dtype not in (torch.int32, torch.uint32) or out.dim() != 2 or out.shape[1] != query.n_vars:
        raise ValueError("out: a host (n, n_vars) int32 tensor")
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    q = query._c()
    ptr, keep = _index_array(indexes)
    prm = _params(query, mode="materialize", **options)
    cnt = ctypes.c_uint64()
    _lib.check(_lib.load().hc_run_join_to_host(ctypes.byref(q), ptr, ctypes.byref(prm),
                                               ctypes.c_void_p(out.data_ptr() if out.numel() else 0), out.shape[0],
                                               ctypes.byref(cnt), ctypes.c_void_p(_stream_ptr(stream))),
               "hc_run_join_to_host")
    return int(cnt.value)


def _params(query: Query, shares=None, seeds=None, item_grain=0, block_threads=0, merge_min=0, merge_ratio=0,
            slice_grain=0, mode="count", flags=0, out_capacity=0, lift=True, lift_arena=0,
            dir_min=0, pair_min=0) -> _lib.hc_join_params:
    prm = _lib.hc_join_params()
    sh = list(shares) if shares is not None else [1] * query.n_vars
    sd = list(seeds) if seeds is not None else list(DEFAULT_SEEDS)
    for v in range(_lib.HC_MAX_VARS):
        prm.shares[v] = sh[v] if v < len(sh) else 1
        prm.seeds[v] = (sd[v] if v < len(sd) else DEFAULT_SEEDS[v]) & 0xFFFFFFFF
    prm.mode = _lib.HC_MODE_COUNT if mode == "count" else _lib.HC_MODE_MATERIALIZE
    prm.flags = flags | (0 if lift else _lib.HC_FLAG_NO_LIFT)
    prm.lift_arena = int(lift_arena)
    prm.item_grain = item_grain
    prm.block_threads = block_threads
    prm.merge_min = merge_min & 0xFFFFFFFF
    prm.merge_ratio = merge_ratio & 0xFFFFFFFF
    prm.slice_grain = slice_grain & 0xFFFFFFFF
    prm.out_capacity = int(out_capacity)
    prm.dir_min = dir_min & 0xFFFFFFFF
    prm.pair_min = pair_min & 0xFFFFFFFF
    return prm


class Batch:
    """Many count-mode joins in one persistent search launch.

    ``queries[i]`` runs over ``indexes[i]`` (one index per atom) with the
    keyword options ``options[i]`` (shares, seeds, item_grain, merge_min,
    merge_ratio, slice_grain).  ``launch`` enqueues the batch; after
    ``capture(stream)`` launches replay a CUDA graph.  ``counts`` waits.
    """

    def __init__(self, queries, indexes, options=None, stream=None):
        n = len(queries)
        if n == 0 or len(indexes) != n:
            raise ValueError("one index list per query")
        options = options or [{}] * n
        self._keep = list(indexes)
        qarr = (_lib.hc_query * n)(*[q._c() for q in queries])
        flat = [ix.handle.value for lst in indexes for ix in lst]
        for q, lst in zip(queries, indexes):
            if len(lst) != len(q.atoms):
                raise ValueError("one index per atom")
        iarr = (ctypes.c_void_p * len(flat))(*flat)
        parr = (_lib.hc_join_params * n)(*[_params(q, **o) for q, o in zip(queries, options)])
        out = ctypes.c_void_p()
        _lib.check(_lib.load().hc_batch_create(qarr, ctypes.cast(iarr, ctypes.POINTER(ctypes.c_void_p)), parr, n,
                                               ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out)),
                   "hc_batch_create")
        self._h = out
        self.n = n

    def launch(self, stream=None) -> None:
        _lib.check(_lib.load().hc_batch_launch(self._h, ctypes.c_void_p(_stream_ptr(stream))), "hc_batch_launch")

    def capture(self, stream) -> None:
        _lib.check(_lib.load().hc_batch_capture(self._h, ctypes.c_void_p(_stream_ptr(stream))), "hc_batch_capture")

    def counts(self) -> list[int]:
        out = (ctypes.c_uint64 * self.n)()
        _lib.check(_lib.load().hc_batch_counts(self._h, out), "hc_batch_counts")
        return [int(x) for x in out]

    def free(self) -> None:
        if self._h is not None:
            _lib.load().hc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Pending:
    """A count-mode join enqueued without waiting; ``count()`` waits."""

    def __init__(self, h):
        self._h = _ResultHandle(h)

    def count(self) -> int:
        v = _lib.hc_result_view()
        _lib.check(_lib.load().hc_result_get(ctypes.c_void_p(self._h.h), ctypes.byref(v)), "hc_result_get")
        c = int(v.count)
        self._h.free()
        return c


def join_footprint(query: Query, indexes: Sequence[Index], **options) -> int:
    """Upper bound of the device bytes a count-mode join allocates (host only)."""
    q = query._c()
    ptr, keep = _index_array(indexes)
    prm = _params(query, **options)
    out = ctypes.c_uint64()
    _lib.check(_lib.load().hc_join_footprint(ctypes.byref(q), ptr, ctypes.byref(prm), ctypes.byref(out)),
               "hc_join_footprint")
    return int(out.value)


def run_join_async(query: Query, indexes: Sequence[Index], stream=None, **options) -> Pending:
    """Enqueue a count-mode join and return at once (the library waits for
    nothing in count mode); options as for ``run_join``."""
    if len(indexes) != len(query.atoms):
        raise ValueError("one index per atom")
    q = query._c()
    ptr, keep = _index_array(indexes)
    prm = _params(query, **options)
    out = ctypes.c_void_p()
    _lib.check(_lib.load().hc_run_join(ctypes.byref(q), ptr, ctypes.byref(prm), ctypes.c_void_p(_stream_ptr(stream)),
                                       ctypes.byref(out)), "hc_run_join")
    return Pending(out.value)


class _ResultHandle:
    def __init__(self, h):
        self.h = h

    def free(self):
        if self.h:
            _lib.load().hc_result_free(ctypes.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


from .kary import CT, LW, KIndex, KQuery, atom_shares, build_kindex, choose_korder, kplan_cost, run_kjoin  # noqa: E402,E501

__all__ += ["KQuery", "KIndex", "build_kindex", "run_kjoin", "choose_korder", "kplan_cost", "atom_shares", "LW", "CT"]
