"""The C-ABI library loads and exports every entry point include/gbchfsi.h
declares (no compute calls: this runs without a GPU)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbchfsi.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gbc_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2410_02754_gb300 import gbchfsi
    return gbchfsi.load_library()


def test_header_lists_the_binding_exports():
    from paper_2410_02754_gb300 import gbchfsi
    assert declared_functions() == sorted(gbchfsi.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_string(lib):
    assert lib.gbc_version().decode().startswith("gbchfsi")


def test_bad_arguments_are_rejected_without_a_device(lib):
    h = ct.c_void_p()
    assert lib.gbc_create(None, 0) == 1            # GBC_EINVAL
    assert lib.gbc_create(ct.byref(h), -1) == 1
    assert lib.gbc_last_error(None) == b"null context"
    lib.gbc_destroy(None)                            # NULL-safe


def test_product_path_does_not_reach_the_oracle():
    """No file of the package imports or names the oracle or the input generator."""
    pkg = os.path.join(ROOT, "paper_2410_02754_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\b(import|from)\s+(oracle|synthetic)\b", txt), f


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as pedantic C99 (no C++ types cross the ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "gbchfsi.h"\nint main(void) { return 0; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I" + inc, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
