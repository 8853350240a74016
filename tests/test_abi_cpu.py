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


def test_tune_reset_is_host_only():
    # forgetting the tuners' choices touches no device: callable anywhere,
    # any number of times
    sj.sj_tune_reset()
    sj.sj_tune_reset()


def test_no_device_is_an_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sj.SJError):
        sj.Context()


def test_header_is_plain_c_and_struct_sizes_match_the_binding(tmp_path):
    """include/sj.h compiles as C99 (no C++ in the boundary), and the sizes
    of its structs equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include "sj.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu\\n", sizeof(sj_config), sizeof(sj_stats),\n'
        "         sizeof(sj_index_desc), sizeof(sj_job), sizeof(sj_serve_info));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = [ctypes.sizeof(t) for t in (sj.sj_config, sj.sj_stats, sj.sj_index_desc, sj.sj_job,
                                       sj.sj_serve_info)]
    assert got == want


def test_reference_arm_prints_its_json_line():
    """bench.py --impl reference times the CPU oracle and prints one JSON
    line with the contract's keys."""
    import json
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # the same workload description as the GPU arm prints
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == json.loads(json.dumps(bench.bench_config(bench.workload())))
    assert set(line["cpu_baseline"]["build_s"]) == {"2", "3", "4", "5", "6"}
