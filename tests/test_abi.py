"""The C-ABI library builds, loads and exports every function include/gj.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gj.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gj_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_09930_gb300 import _build
    _build.build()
    from paper_1809_09930_gb300 import gj
    return gj.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gj_index_build", "gj_self_join", "gj_free", "gj_last_status", "gj_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1809_09930_gb300 import gj
    so = gj.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(gj_[a-z0-9_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for f in declared_functions():
        assert hasattr(lib, f)
    assert set(gj.EXPORTS) == set(declared_functions())


def header_constants():
    """Every integer #define GJ_... of the header (flags, status codes, limits),
    evaluated (shifts and ors of earlier names)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    vals = {}
    for name, expr in re.findall(r"#define\s+(GJ_[A-Z0-9_]+)\s+([^\n]+)", src):
        expr = expr.strip().replace("1u", "1")
        if not expr or name == "GJ_H":
            continue
        vals[name] = eval(expr, {}, dict(vals))
    return vals


def test_python_constants_match_the_header():
    from paper_1809_09930_gb300 import gj
    consts = header_constants()
    for must in ("GJ_OK", "GJ_ERR_CAPACITY", "GJ_TC_FILTER", "GJ_HOST_BATCHED", "GJ_DEFAULT_FLAGS"):
        assert must in consts
    for name, v in consts.items():
        if hasattr(gj, name):
            assert getattr(gj, name) == v, name
    flags = [n for n in consts if n in ("GJ_REORDER", "GJ_SORTIDU", "GJ_SHORTC", "GJ_TC_FILTER", "GJ_AUTOTUNE",
                                        "GJ_TUNE_FORM", "GJ_HOST_BATCHED")]
    assert len(flags) == 7 and all(hasattr(gj, n) for n in flags)
    bits = [consts[n] for n in flags]
    assert all(b & (b - 1) == 0 for b in bits) and len(set(bits)) == len(bits)   # distinct single bits


def test_host_only_entry_points(lib):
    from paper_1809_09930_gb300 import gj
    assert gj.gj_version().count(".") == 2
    assert gj.gj_status_string(gj.GJ_ERR_CAPACITY).startswith("result larger")
    cfg = gj.gj_config_init()
    assert cfg.flags == gj.GJ_DEFAULT_FLAGS and cfg.k == 0 and cfg.device == -1
    lib.gj_free(None)   # NULL-safe


def test_no_gpu_build_fails_loudly(lib):
    """Without a usable GPU the build reports GJ_ERR_UNSUPPORTED; it never falls
    back to a CPU path."""
    import numpy as np
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    from paper_1809_09930_gb300 import gj
    with pytest.raises(gj.GJError) as e:
        gj.Index(np.zeros((4, 2)), 0.5)
    assert e.value.status == gj.GJ_ERR_UNSUPPORTED


@pytest.mark.parametrize("field,value", [("query_block", 7), ("query_block", 129), ("query_block", -1),
                                         ("tile", 48), ("tile", 16), ("k", 9)])
def test_config_ranges_rejected_before_any_device_call(lib, field, value):
    """Out-of-range settings fail with GJ_ERR_INVALID_ARG (checked on the host,
    before the device is touched, so this runs without a GPU)."""
    import numpy as np
    from paper_1809_09930_gb300 import gj
    cfg = gj.gj_config_init()
    setattr(cfg, field, value)
    with pytest.raises(gj.GJError) as e:
        gj.gj_index_build_ex(np.zeros((16, 8)), 0.5, cfg)
    assert e.value.status == gj.GJ_ERR_INVALID_ARG


def test_config_layout_matches_header(lib):
    """gj_config keeps its size: the new fields took reserved words."""
    import ctypes
    from paper_1809_09930_gb300 import gj
    assert ctypes.sizeof(gj.gj_config) == 4 + 4 + 8 + 8 + 4 + 4 + 4 + 5 * 4   # 56, as before
    assert ctypes.sizeof(gj.gj_tune_result) == 4 * 4 + 8 * 4 + 4 * 2


@pytest.mark.parametrize("n,d,eps,want", [
    (1 << 32, 2, 0.5, "GJ_ERR_TOO_LARGE"),       # pair ids are 32-bit
    (10, 1025, 0.5, "GJ_ERR_TOO_LARGE"),         # d > GJ_MAX_DIMS
    (10, 0, 0.5, "GJ_ERR_INVALID_ARG"),
    (-1, 4, 0.5, "GJ_ERR_INVALID_ARG"),
    (10, 4, 0.0, "GJ_ERR_INVALID_ARG"),
    (10, 4, float("nan"), "GJ_ERR_INVALID_ARG"),
    (10, 4, float("inf"), "GJ_ERR_INVALID_ARG"),
])
def test_build_argument_ranges_rejected_on_the_host(lib, n, d, eps, want):
    """Sizes and eps outside the contract fail before any device work (no GPU
    needed); the points pointer is never read."""
    import ctypes
    from paper_1809_09930_gb300 import gj
    dummy = (ctypes.c_double * 8)()
    cfg = gj.gj_config_init()
    h = lib.gj_index_build_ex(ctypes.cast(dummy, ctypes.c_void_p), n, d, eps, ctypes.byref(cfg))
    assert not h
    assert lib.gj_last_status() == getattr(gj, want)


def test_null_handles_and_buffers_rejected(lib):
    import ctypes
    from paper_1809_09930_gb300 import gj
    cnt = ctypes.c_uint64(0)
    assert lib.gj_self_join(None, None, 0, ctypes.byref(cnt)) == gj.GJ_ERR_INVALID_ARG
    assert lib.gj_join_qe(None, None, 0, None, 0, ctypes.byref(cnt)) == gj.GJ_ERR_INVALID_ARG
    assert lib.gj_neighbor_table(None, None, None, 0, ctypes.byref(cnt)) == gj.GJ_ERR_INVALID_ARG
    assert lib.gj_batch_self_join(None, None, None, None) == gj.GJ_ERR_INVALID_ARG
    assert lib.gj_batch_build(None, 0, None) is None
    assert lib.gj_last_status() == gj.GJ_ERR_INVALID_ARG
    r = gj.gj_tune_result()
    assert lib.gj_autotune(None, 10, 4, 0.5, None, ctypes.byref(r)) == gj.GJ_ERR_INVALID_ARG
    lib.gj_batch_free(None)
