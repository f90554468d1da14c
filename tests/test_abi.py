"""Host-side checks that need no GPU: the C-ABI library builds, loads and
exports every symbol include/swapmd.h declares, and the product and the oracle
stay independent of each other."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swapmd.h")
PKG = os.path.join(ROOT, "paper_1912_08569_gb300")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^SWP_API\s+[\w\s\*]+?\b(swp_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_08569_gb300 import _abi
    from paper_1912_08569_gb300.build import build

    build()
    return _abi.load_library()


def test_header_declares_the_binding_names():
    from paper_1912_08569_gb300 import _abi

    assert _declared() == sorted(_abi.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(PKG, "libswapmd.so")],
                         capture_output=True, text=True)
    if out.returncode == 0:
        exported = sorted(ln.split()[-1] for ln in out.stdout.splitlines() if " T " in ln)
        assert exported == _declared()


def test_abi_version_needs_no_device(lib):
    from paper_1912_08569_gb300 import _abi

    assert _abi.swp_abi_version() == 6


def test_header_compiles_as_plain_c(tmp_path):
    c = tmp_path / "t.c"
    c.write_text('#include "swapmd.h"\nint main(void){ swp_thermo t; (void)t; return SWP_OK; }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), "-c",
                        str(c), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_thermo_struct_layout_matches_binding():
    import ctypes

    from paper_1912_08569_gb300 import _abi

    # 9 doubles + 4 int64 + 4 int32
    assert ctypes.sizeof(_abi.swp_thermo) == 9 * 8 + 4 * 8 + 4 * 4
    assert _abi.swp_thermo.resident_steps.offset == 9 * 8 + 4 * 8 + 2 * 4


def test_thermo_struct_layout_matches_c(tmp_path):
    """The C compiler's layout of swp_thermo equals the binding's."""
    import ctypes

    from paper_1912_08569_gb300 import _abi

    c = tmp_path / "lay.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "swapmd.h"\n'
                 'int main(void){ printf("%zu %zu %zu\\n", sizeof(swp_thermo), '
                 'offsetof(swp_thermo, state), offsetof(swp_thermo, resident_steps)); return 0; }\n')
    exe = tmp_path / "lay"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()
    assert [int(v) for v in out] == [ctypes.sizeof(_abi.swp_thermo), _abi.swp_thermo.state.offset,
                                     _abi.swp_thermo.resident_steps.offset]


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                yield os.path.join(base, f)


def test_product_does_not_use_the_oracle():
    for p in _py_files(PKG):
        src = open(p).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), p
        assert "swap_oracle" not in src and "liboracle" not in src, p


def test_oracle_does_not_use_the_product():
    for p in _py_files(os.path.join(ROOT, "oracle")):
        src = open(p).read()
        assert "paper_1912_08569_gb300" not in src, p
        assert "swapmd" not in src and "swp_" not in src, p


def test_product_fails_loudly_without_the_library(tmp_path):
    from paper_1912_08569_gb300 import _abi

    with pytest.raises(RuntimeError, match="not built"):
        saved = _abi._lib
        _abi._lib = None
        try:
            _abi.load_library(str(tmp_path / "missing.so"))
        finally:
            _abi._lib = saved
