"""The C-ABI library builds, loads and exports what include/*.h declares (CPU)."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_06715_gb300 import _lib, build

    build.build_library()
    return _lib.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:hc_status|const char\s*\*|uint32_t|uint64_t)\s+(hc_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hc_build_index", "hc_choose_shares", "hc_run_join", "hc_partition_index",
                     "hc_result_get", "hc_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2502_06715_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hc_\w+)", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    # the binding declares prototypes for exactly the header's functions
    assert set(_lib.SIGNATURES) == _declared()


def test_library_is_sm103a_only():
    from paper_2502_06715_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_calls(lib):
    assert lib.hc_status_str(0) == b"ok"
    assert lib.hc_status_str(4) == b"bounded device wait gave up"
    assert lib.hc_target_sm() == 103


def test_stats_index_rejected_by_join(lib):
    import paper_2502_06715_gb300 as hc

    ix = hc.Index.from_stats(100, 10, 0, 99, 99)
    with pytest.raises(hc.HoneycombError) as e:
        hc.run_join(hc.TRIANGLE, [ix, ix, ix], stream=0)  # rejected before any device work
    assert e.value.status == 1
    bad = hc.Query(3, ((0, 1), (1, 1), (0, 2)))
    with pytest.raises(hc.HoneycombError) as e:
        hc.run_join(bad, [ix, ix, ix], stream=0)
    assert e.value.status == 1
    with pytest.raises(hc.HoneycombError):
        hc.Index.from_stats(10, 11, 0, 1, 1)  # l1 > n


def test_product_path_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2502_06715_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "oracle.c" not in text, path


def test_list_length_limit_is_checked(lib):
    """The search kernels sum up to 32 bindings' candidate counts in 32 bits,
    so a loop whose shortest list can reach 2^27 values is refused with
    HC_ERR_CAPACITY before any device work.  hc_join_footprint plans exactly
    as hc_run_join does and accepts statistics-only indexes, so the check is
    exercised here without a GPU.  In the triangle (order x, y, z) the last
    loop intersects two sub-lists, bounded by the index's longest run."""
    import paper_2502_06715_gb300 as hc

    n, l1 = 1 << 28, 1 << 24
    fits = hc.Index.from_stats(n, l1, 0, n, n, max_run=(1 << 27) - 1)
    over = hc.Index.from_stats(n, l1, 0, n, n, max_run=1 << 27)
    unknown = hc.Index.from_stats(n, l1, 0, n, n)
    assert hc.join_footprint(hc.TRIANGLE, [fits] * 3) > 0
    assert hc.join_footprint(hc.TRIANGLE, [unknown] * 3) > 0
    # loop z reads S[y] and T[x]: only the shorter of the two is iterated
    for ixs in ([over] * 3, [fits, over, over]):
        with pytest.raises(hc.HoneycombError) as e:
            hc.join_footprint(hc.TRIANGLE, ixs)
        assert e.value.status == 5
    for ixs in ([over, fits, over], [over, over, fits]):
        assert hc.join_footprint(hc.TRIANGLE, ixs) > 0
    # a loop whose lists include a top level shorter than the limit is safe:
    # loop y of the triangle reads R[x] and S.V1 (l1 = 2^24 values), and loop
    # z reads S[y] and T[x]; with every atom's key rows below 2^27 only S.V1
    # and sub-lists are iterated
    wide = hc.Index.from_stats(n, (1 << 27) + 5, 0, n, n, max_run=100)
    assert hc.join_footprint(hc.TRIANGLE, [fits, wide, fits]) > 0
    # max_run outside [1, n - l1 + 1] is an argument error
    with pytest.raises(hc.HoneycombError) as e:
        hc.Index.from_stats(100, 10, 0, 99, 99, max_run=92)
    assert e.value.status == 1
    assert hc.Index.from_stats(100, 10, 0, 99, 99, max_run=91).max_run == 91


def test_position_map_never_sized_past_32_bits(lib):
    """A relation holding the value 0xFFFFFFFF gets no V1 position map (its
    length, 2^32, would not fit the map's 32-bit size).  The footprint of a
    partitioned atom counts the map when one is built, so the eligibility
    rule shows in it: max_first 0xFFFFFFFE adds a (2^32 - 1)-entry map for 2^31
    rows, max_first 0xFFFFFFFF adds none."""
    import paper_2502_06715_gb300 as hc

    n = 1 << 31
    q = hc.Query(2, ((0, 1),))
    a = hc.Index.from_stats(n, n >> 1, 0, 0xFFFFFFFE, 7)
    b = hc.Index.from_stats(n, n >> 1, 0, 0xFFFFFFFF, 7)
    fa = hc.join_footprint(q, [a], shares=[2, 1])
    fb = hc.join_footprint(q, [b], shares=[2, 1])
    # (max_first + 1) map entries of 4 bytes, less the V1 directory (16 bytes a
    # row) that a partition without a map needs
    assert fa - fb == 4 * 0xFFFFFFFF - 16 * n


def test_wait_limit_is_a_library_parameter(lib):
    import paper_2502_06715_gb300 as hc

    prev = hc.set_wait_limit_ns(12345)
    try:
        assert prev == 2_000_000_000
        assert lib.hc_wait_limit_ns() == 12345
    finally:
        hc.set_wait_limit_ns(prev)
    assert lib.hc_wait_limit_ns() == prev


def test_serving_selection_is_sorted_and_distinct():
    """The unary builder trusts its values to ascend strictly; the serving
    loop sorts and de-duplicates a request's selection before building it."""
    from paper_2502_06715_gb300.serve import _selection_values

    v = _selection_values([9, 3, 3, 0xFFFFFFFF, 0, 9])
    assert v.dtype == np.uint32 and v.tolist() == [0, 3, 9, 0xFFFFFFFF]
    assert _selection_values([]).shape == (0,)


def test_partitioned_kindex_argument_checks(lib):
    """hc_build_kindex_partitioned refuses bad shares and missing seeds,
    shares or rows before any device work."""
    import ctypes

    out = ctypes.c_void_p()
    seeds = (ctypes.c_uint32 * 3)(1, 2, 3)
    for sh in ((2, 0, 1), (256, 256, 2)):  # a zero share; a product above 65536
        shares = (ctypes.c_uint32 * 3)(*sh)
        assert lib.hc_build_kindex_partitioned(None, 0, 3, None, seeds, shares, 0, None, ctypes.byref(out)) == 1
        assert not out.value
    good = (ctypes.c_uint32 * 3)(2, 2, 1)
    assert lib.hc_build_kindex_partitioned(None, 0, 3, None, None, good, 0, None, ctypes.byref(out)) == 1
    assert lib.hc_build_kindex_partitioned(None, 0, 3, None, seeds, None, 0, None, ctypes.byref(out)) == 1
    assert lib.hc_build_kindex_partitioned(None, 10, 3, None, seeds, good, 0, None, ctypes.byref(out)) == 1
    assert lib.hc_build_kindex_partitioned(None, 0, 4, None, seeds, good, 0, None, ctypes.byref(out)) == 1
