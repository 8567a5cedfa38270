"""The C-ABI library builds, loads without a GPU and exports what it declares.

No CUDA call is made here; these run on the CPU-only host.
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(INCLUDE):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(sw_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2208_12350_gb300 as swgb
    return swgb.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ["sw_align_batch", "sw_plan_create", "sw_plan_execute", "sw_plan_destroy",
                     "sw_ctx_create", "sw_ctx_destroy", "sw_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2208_12350_gb300 as swgb
    out = subprocess.run(["nm", "-D", "--defined-only", swgb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        assert hasattr(lib, n)
    # the binding wraps every exported sw_ function
    assert set(declared_functions()) <= set(swgb.SIGNATURES)


def test_library_has_no_hard_driver_dependency(lib):
    import paper_2208_12350_gb300 as swgb
    out = subprocess.run(["ldd", swgb.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcuda.so" not in out and "libtorch" not in out


def test_host_side_argument_errors(lib):
    """Argument checks that fail before any CUDA call."""
    import ctypes
    import paper_2208_12350_gb300 as swgb
    # NULL out pointer / NULL ctx are rejected without touching the device
    assert lib.sw_ctx_create(0, None) == swgb.SW_EINVAL
    h = ctypes.c_void_p()
    rc = lib.sw_plan_create(None, None, None, 0, None, 4, -6, -1, 0, 0, ctypes.byref(h))
    assert rc == swgb.SW_EINVAL
    assert b"ctx is NULL" in lib.sw_last_error()
    assert lib.sw_plan_execute(None, None, None, None, None, None, None, None, None) == swgb.SW_EINVAL
    assert lib.sw_ctx_set_tuning(None, -1, 0.5) == swgb.SW_EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2208_12350_gb300 as swgb
    monkeypatch.setattr(swgb, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(swgb, "_lib", None)
    with pytest.raises(ImportError):
        swgb.load()


def test_cigar_capacity_is_host_only(lib):
    """sw_cigar_capacity runs on the host: room per aligned pair, 0 otherwise."""
    import numpy as np
    import paper_2208_12350_gb300 as swgb
    res = np.array([[7, 0, 12],      # scores
                    [4, -1, 30],     # qend
                    [3, -1, 40],     # rend
                    [0, -1, 10],     # qstart
                    [0, -1, 35]], dtype=np.int32)
    off = swgb.sw_cigar_capacity(res)
    assert off.tolist() == [0, 5 + 4, 9, 9 + 21 + 6]
    assert lib.sw_cigar_capacity(None, 3, None) == swgb.SW_EINVAL
    assert lib.sw_traceback(None, None, None, None, None, 0, None, 4, -6, -1, None, None, None,
                            None, None) == swgb.SW_EINVAL


def test_pack_2bit_is_host_only(lib):
    """sw_pack_2bit packs four codes per byte, first in the low bits."""
    import numpy as np
    import paper_2208_12350_gb300 as swgb
    rng = np.random.default_rng(3)
    for n in (0, 1, 3, 4, 5, 1001):
        codes = rng.integers(0, 4, n).astype(np.uint8)
        packed = swgb.sw_pack_2bit(codes)
        assert len(packed) == (n + 3) // 4
        back = ((packed[:, None] >> (2 * np.arange(4))) & 3).astype(np.uint8).reshape(-1)[:n]
        assert np.array_equal(back, codes)
    with pytest.raises(swgb.SwError) as e:
        swgb.sw_pack_2bit(np.array([0, 1, 4], dtype=np.uint8))
    assert e.value.code == swgb.SW_ERANGE
