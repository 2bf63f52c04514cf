"""The C ABI without a GPU: the library loads, exports every function the
header declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

import paper_2202_06929_b300 as frnn
from paper_2202_06929_b300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"FRNN_API\s+[\w\s\*]+?\b(frnn_\w+)\s*\(", src))
    return names


def test_header_declares_the_binding_functions():
    assert declared_functions() == set(_native.ABI_FUNCTIONS)


def test_library_exports_every_declared_symbol():
    lib = frnn.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert frnn.version() >= 10000


def test_status_strings():
    for s in range(9):
        assert frnn.status_string(s) != "unknown status"
    assert frnn.status_string(999) == "unknown status"


def test_null_plan_and_bad_params_rejected_on_host():
    lib = frnn.load()
    c = _native.frnn_csr()
    assert lib.frnn_build_graph(None, None, 10, 3, ctypes.c_float(0.1), 4, None, ctypes.byref(c)) == 1
    off = (ctypes.c_int64 * 2)(0, 10)
    assert lib.frnn_build_graph_batched(None, None, off, 1, 3, ctypes.c_float(0.1), 4, None, ctypes.byref(c)) == 1
    assert lib.frnn_get_last_status(None, None) == 1
    assert lib.frnn_plan_test_stall_next_build(None) == 1
    assert lib.frnn_check_last_build(None, None) == 1
    cid, idx = ctypes.c_int(0), ctypes.c_int64(0)
    assert lib.frnn_get_last_check(None, None, ctypes.byref(cid), ctypes.byref(idx)) == 1
    assert lib.frnn_plan_destroy(None) == 0
    h = ctypes.c_void_p()
    assert lib.frnn_plan_create(ctypes.byref(h), None) == 1
    for bad in [dict(d_max=0), dict(d_max=65), dict(k_max_cap=0), dict(k_max_cap=1025),
                dict(events_max=0), dict(n_max=-1), dict(n_max=1 << 28, k_max_cap=1024)]:
        kw = dict(device=0, d_max=8, n_max=100, events_max=1, k_max_cap=8)
        kw.update(bad)
        prm = _native.frnn_plan_params(**kw)
        assert lib.frnn_plan_create(ctypes.byref(h), ctypes.byref(prm)) == 1, bad


def test_plan_over_its_memory_budget_is_refused_before_any_device_call():
    lib = frnn.load()
    h = ctypes.c_void_p()
    prm = _native.frnn_plan_params(device=0, d_max=8, n_max=100_000, events_max=1, k_max_cap=64)
    need = ctypes.c_uint64(0)
    assert lib.frnn_plan_bytes(ctypes.byref(prm), ctypes.byref(need)) == frnn.FRNN_OK
    prm.mem_budget_bytes = need.value - 1
    assert lib.frnn_plan_create(ctypes.byref(h), ctypes.byref(prm)) == frnn.FRNN_ERR_OOM
    assert not h.value
    # the budget does not change the plan's size
    got = ctypes.c_uint64(0)
    assert lib.frnn_plan_bytes(ctypes.byref(prm), ctypes.byref(got)) == frnn.FRNN_OK and got.value == need.value


def test_plan_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = frnn.load()
    h = ctypes.c_void_p()
    prm = _native.frnn_plan_params(device=0, d_max=8, n_max=100, events_max=1, k_max_cap=8)
    assert lib.frnn_plan_create(ctypes.byref(h), ctypes.byref(prm)) == frnn.FRNN_ERR_CUDA
    assert not h.value


def test_header_compiles_as_c99_and_links(tmp_path):
    """include/frnn.h is a C header: a C99 program includes it (strict,
    pedantic), links against libfrnn.so and calls an entry point that needs no
    GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = frnn.library_path()
    src = tmp_path / "use_frnn.c"
    src.write_text('#include "frnn.h"\n'
                   "int main(void) {\n"
                   "    frnn_plan* p = 0;\n"
                   "    frnn_plan_params prm = {0};\n"
                   "    uint64_t bytes = 0;\n"
                   "    int check = -1;\n"
                   "    int64_t index = 0;\n"
                   "    prm.d_max = 8; prm.n_max = 1000; prm.events_max = 1; prm.k_max_cap = 16;\n"
                   "    prm.flags = FRNN_DEBUG | FRNN_EMIT_D2;\n"
                   "    if (frnn_plan_bytes(&prm, &bytes) != FRNN_OK || bytes == 0) return 2;\n"
                   "    prm.mem_budget_bytes = bytes - 1;\n"
                   "    if (frnn_plan_create(&p, &prm) != FRNN_ERR_OOM || p) return 3;\n"
                   "    if (frnn_check_last_build(p, 0) != FRNN_ERR_INVALID_ARG) return 4;\n"
                   "    if (frnn_get_last_check(p, 0, &check, &index) != FRNN_ERR_INVALID_ARG) return 5;\n"
                   "    if (FRNN_CHECK_COMPLETE != 9 || FRNN_ERR_CHECK != 8) return 6;\n"
                   "    return frnn_plan_test_stall_next_build(p) == FRNN_ERR_INVALID_ARG ? 0 : 1;\n"
                   "}\n")
    exe = tmp_path / "use_frnn"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                    str(src), lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True)
    assert subprocess.run([str(exe)]).returncode == 0
