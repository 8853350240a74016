"""CPU-side checks of the library boundary: it builds for sm_103a, loads, and
exports every function the header declares.  No GPU calls."""
import ctypes
import os
import re

import pytest

from paper_1803_04120_gb300 import _build, sj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "sj.h")).read()
    return sorted(set(re.findall(r"SJ_API\s+[\w\s\*]*?\b(sj_\w+)\s*\(", text)))


def test_header_lists_match_binding():
    assert header_functions() == sorted(sj.ABI_FUNCTIONS)


def test_library_builds_and_exports_every_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_status_names():
    lib = sj.load()
    assert lib.sj_status_str(sj.SJ_EOVERFLOW) == b"SJ_EOVERFLOW"
    cfg = sj.sj_config()
    lib.sj_config_default(ctypes.byref(cfg))
    assert cfg.prec == sj.SJ_PREC_FP32_RECHECK and cfg.unicomp == 1
    assert cfg.min_batches == 3 and cfg.out_cap_bytes == 2 << 30


def test_no_device_is_an_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sj.SJError):
        sj.Context()
