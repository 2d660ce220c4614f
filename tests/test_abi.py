"""The C-ABI library builds, loads and exports what include/*.h declares (CPU)."""
import glob
import os
import re
import subprocess

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
