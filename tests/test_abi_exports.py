"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/cascade.h declares; the Python binding covers the same
set under the same names.  No compute calls (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cascade.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cascade_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2411_17729_gb300 import build
    return build()


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("cascade_plan_create", "cascade_forward", "cascade_backward",
                 "cascade_set_system_continuous", "cascade_set_system_discrete",
                 "cascade_set_batch", "cascade_workspace_size", "cascade_get_device_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2411_17729_gb300 import _abi
    bound = {n for n, _, _ in _abi.SIGNATURES}
    assert bound == set(declared_functions())
    lib = _abi.load(libpath)
    assert lib.cascade_status_string(0) == b"ok"
    assert lib.cascade_status_string(5) == b"device wait timed out"


def test_descriptor_layout_matches_header():
    """cascade_desc_t: eight int32 fields, then int64 max_rows, then double eps."""
    from paper_2411_17729_gb300 import _abi
    d = _abi.cascade_desc_t
    assert ctypes.sizeof(d) == 48
    assert d.max_rows.offset == 32 and d.eps.offset == 40
    text = open(HEADER).read()
    block = text[text.index("typedef struct {"):text.index("} cascade_desc_t;")]
    fields = re.findall(r"(int32_t|int64_t|double)\s+([A-Za-z_, ]+);", block)
    flat = [(t, n.strip()) for t, names in fields for n in names.split(",")]
    assert [n for _, n in flat] == [f for f, _ in d._fields_]


def test_plan_create_without_gpu_fails_cleanly(libpath):
    """On a machine without a GPU, plan creation reports CASCADE_ERR_CUDA
    instead of crashing (on a GPU machine it succeeds)."""
    from paper_2411_17729_gb300 import _abi
    lib = _abi.load(libpath)
    plan = _abi.cascade_plan_t()
    d = _abi.cascade_desc_t(m=64, p=1, q=1, nsys=1, N=3, precision=_abi.CASCADE_BF16_SPLIT,
                            max_len=100, flags=0, max_rows=100, eps=0.0)
    st = lib.cascade_plan_create(ctypes.byref(plan), ctypes.byref(d))
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        assert st == _abi.CASCADE_OK
        lib.cascade_plan_destroy(plan)
    else:
        assert st == _abi.CASCADE_ERR_CUDA and not plan.value
    # argument validation happens before any device call
    bad = _abi.cascade_desc_t(m=0, p=1, q=1, nsys=1, N=3, precision=0, max_len=1, flags=0,
                              max_rows=1, eps=0.0)
    assert lib.cascade_plan_create(ctypes.byref(plan), ctypes.byref(bad)) == _abi.CASCADE_ERR_INVALID_ARG
