"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and exports every
function include/stc.h declares; the Python binding declares the same set; the oracle
library exports what its wrapper uses. No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "stc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_10094_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ["stc_create", "stc_destroy", "stc_contract", "stc_count", "stc_linearize", "stc_group_keys",
                 "stc_result_info", "stc_result_data", "stc_result_stats", "stc_result_free",
                 "stc_status_string", "stc_last_error"]:
        assert name in fns


def test_header_is_plain_c():
    """The boundary needs no C++: the header compiles as C99 on its own."""
    import shutil

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-fsyntax-only", "-std=c99", "-Wall", "-Werror", "-x", "c",
                        os.path.join(ROOT, "include", "stc.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_struct_layouts_match_the_binding(tmp_path):
    """The ctypes mirrors of the C structs have the C compiler's field offsets and sizes."""
    import ctypes as C
    import shutil

    from paper_2410_10094_gb300 import binding as B

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"stc_coo": B.stc_coo, "stc_problem": B.stc_problem, "stc_opts": B.stc_opts,
               "stc_stats": B.stc_stats, "stc_server_opts": B.stc_server_opts, "stc_keyed": B.stc_keyed}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "stc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for row in filter(None, out):
        name, field, value = row.split()
        cls = structs[name]
        got = C.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), f"{name}.{field}: ctypes {got}, C {value}"


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (stc_[a-z_0-9]+)$", out, flags=re.M))
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, f"declared in stc.h but not exported: {missing}"
    lib = ctypes.CDLL(libpath)
    for f in header_functions():
        assert getattr(lib, f) is not None


def test_binding_wraps_every_declared_symbol():
    from paper_2410_10094_gb300 import binding

    assert sorted(binding.EXPORTS) == header_functions()


def test_library_is_built_for_sm_103a(libpath):
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_status_strings_without_gpu(libpath):
    from paper_2410_10094_gb300 import binding

    binding.load(libpath)
    assert binding.stc_status_string(0) == "ok"
    assert "coordinate" in binding.stc_status_string(8)


def test_oracle_exports():
    import oracle

    lib = ctypes.CDLL(oracle.build())
    for f in ["oracle_contract", "oracle_ln_key", "oracle_counting_sort", "oracle_first_seen_ids",
              "oracle_group_bounds", "oracle_table_slots"]:
        assert getattr(lib, f) is not None


def test_library_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2410_10094_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "stc_oracle" not in txt, f


def test_missing_library_fails_loudly():
    """Without libstc.so the binding raises: there is no CPU fallback."""
    code = ("import sys; from paper_2410_10094_gb300 import binding as B; B.LIB_PATH = '/nonexistent/libstc.so'\n"
            "try:\n    B.load()\nexcept ImportError as e:\n    print('raised', e); sys.exit(0)\nsys.exit(1)")
    r = subprocess.run([__import__("sys").executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert r.returncode == 0 and "no CPU fallback" in r.stdout, r.stdout + r.stderr


def test_binding_constants_match_the_header():
    """Every enum value and status code of include/stc.h has the same value in the binding."""
    import paper_2410_10094_gb300.binding as b

    src = open(os.path.join(ROOT, "include", "stc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    pairs = dict((name, int(v)) for name, v in re.findall(r"\b(STC_[A-Z_0-9]+)\s*=\s*(\d+)", src))
    assert pairs["STC_ACC_ROWS"] == 4 and pairs["STC_ERR_CANCELLED"] == 10
    for name, v in pairs.items():
        if name.startswith("STC_ERR_") or name == "STC_OK":
            assert b.STATUS_NAMES[v] == name, name
        else:
            assert getattr(b, name[len("STC_"):]) == v, name
