"""CPU-only checks of the C-ABI boundary: the library builds, loads and exports
every entry point include/qk.h declares, and argument checks that need no
device memory reject bad calls.  No compute call runs here (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_07187_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_commands():
    names = declared_functions("qk.h")
    for must in ("qk_add_qubits", "qk_apply_gate", "qk_define_gate_matrix", "qk_define_gate_perm_mulmod",
                 "qk_define_gate_perm_table", "qk_measure", "qk_add_cbits", "qk_apply_rphase_cbits"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for header in os.listdir(os.path.join(ROOT, "include")):
        if not header.endswith(".h"):
            continue
        for name in declared_functions(header):
            assert hasattr(lib, name), f"{name} declared in {header} but not exported"


def test_binding_covers_the_header(lib):
    from paper_1908_07187_gb300 import qk

    assert set(declared_functions("qk.h")) <= set(qk.exported_symbols())


def test_status_strings_and_null_context(lib):
    lib.qk_status_str.restype = ctypes.c_char_p
    assert lib.qk_status_str(0) == b"QK_OK"
    assert lib.qk_status_str(-4) == b"QK_ENOTBIJECTIVE"
    lib.qk_last_error.restype = ctypes.c_char_p
    assert lib.qk_last_error(None) == b"null context"
    assert lib.qk_destroy(None) == -1
    assert lib.qk_flush(None) == -1
    assert lib.qk_num_qubits(None) == -1


def test_create_rejects_bad_precision_without_touching_the_device(lib):
    h = ctypes.c_void_p()
    assert lib.qk_create(ctypes.byref(h), 7, None, None) == -1
    assert lib.qk_create(None, 0, None, None) == -1


def test_create_rejects_bad_options_without_touching_the_device(lib):
    # option checks come before any CUDA call, so they run without a GPU
    from paper_1908_07187_gb300 import qk

    h = ctypes.c_void_p()
    for field, value in (("tile_qubits", 12), ("exec_mode", 5), ("no_tensor_cores", 2)):
        opt = qk.Options()
        setattr(opt, field, value)
        assert lib.qk_create(ctypes.byref(h), 0, None, ctypes.byref(opt)) == -1, field
    opt = qk.Options()
    opt.reserved[3] = 1
    assert lib.qk_create(ctypes.byref(h), 0, None, ctypes.byref(opt)) == -1


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1908_07187_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "qk_oracle" not in src and "liboracle" not in src, f


def test_gate_op_layout_matches_the_header(tmp_path):
    # compile a probe against include/qk.h and compare the C layout of
    # qk_gate_op with the binding's numpy dtype
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    src = tmp_path / "probe.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "qk.h"\n'
        "int main(void) { printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(qk_gate_op),"
        " offsetof(qk_gate_op, target), offsetof(qk_gate_op, np), offsetof(qk_gate_op, controls),"
        " offsetof(qk_gate_op, cond), offsetof(qk_gate_op, params)); return 0; }\n")
    exe = tmp_path / "probe"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    from paper_1908_07187_gb300 import qk

    dt = qk.GATE_OP_DTYPE
    assert got == [dt.itemsize, dt.fields["target"][1], dt.fields["np"][1], dt.fields["controls"][1],
                   dt.fields["cond"][1], dt.fields["params"][1]]
