"""The C-ABI library builds, loads and exports every symbol include/tqp.h declares.

CPU only: no call here launches device work.
"""
import ctypes as C
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tqp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*TQP_API\s+[\w\s\*]*?\b(tqp_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libtqp():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2203_01877_gb300 import build as B
    path = B.build()
    try:
        return C.CDLL(path)
    except OSError as e:  # libcudart missing on a machine without CUDA
        pytest.skip(f"cannot load libtqp.so here: {e}")


def test_header_declares_the_operator_calls():
    names = declared_functions()
    for required in ("tqp_filter", "tqp_hash_join", "tqp_groupby_agg", "tqp_run_plan", "tqp_run_plans",
                     "tqp_ctx_create", "tqp_ctx_destroy", "tqp_ctx_check"):
        assert required in names


def test_every_declared_symbol_is_exported(libtqp):
    missing = [n for n in declared_functions() if not hasattr(libtqp, n)]
    assert not missing, missing


def test_only_api_symbols_are_exported(libtqp):
    import subprocess
    from paper_2203_01877_gb300 import LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(declared_functions())


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the C layout (size and offsets)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import paper_2203_01877_gb300 as tqp
    structs = {"tqp_column": tqp.Column, "tqp_table": tqp.Table, "tqp_pred": tqp.Pred, "tqp_expr": tqp.Expr,
               "tqp_agg": tqp.Agg, "tqp_plan": tqp.Plan, "tqp_result": tqp.Result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tqp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for ln in out:
        if not ln:
            continue
        cname, field, val = ln.split()
        py = structs[cname]
        want = C.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field, val, want)


def test_host_only_calls(libtqp):
    libtqp.tqp_version.restype = C.c_int
    assert libtqp.tqp_version() == 100
    libtqp.tqp_status_string.restype = C.c_char_p
    libtqp.tqp_status_string.argtypes = [C.c_int]
    assert libtqp.tqp_status_string(4) == b"output capacity exceeded"
    # argument validation happens before any CUDA call
    libtqp.tqp_filter.restype = C.c_int
    assert libtqp.tqp_filter(None, None, None, 0, None, None, None, 0, None, None) == 1
    libtqp.tqp_last_error.restype = C.c_char_p
    assert b"ctx" in libtqp.tqp_last_error()
    libtqp.tqp_ctx_destroy.restype = C.c_int
    assert libtqp.tqp_ctx_destroy(None) == 0


def test_tableref_accepts_host_columns_only_on_request():
    """TableRef takes CUDA tensors; a host tensor only with host_ok and only
    when it is pinned (the library then decides where host memory may be read)."""
    torch = pytest.importorskip("torch")
    import paper_2203_01877_gb300 as tqp
    host = torch.zeros(16, dtype=torch.int64)
    with pytest.raises(ValueError):
        tqp.TableRef([host])
    with pytest.raises(ValueError):
        tqp.TableRef([host], host_ok=True)  # pageable, not pinned
