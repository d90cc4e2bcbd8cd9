"""The C-ABI library builds and exports every entry point include/ihs.h
declares; the Python binding's structures match the header's layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fname in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fname.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fname)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ihs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2006_05874_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_exported(built_lib):
    names = _declared_functions()
    assert "ihs_solve" in names and "ihs_grad" in names and len(names) >= 12
    for name in names:
        assert hasattr(built_lib, name), name


def test_binding_covers_header():
    from paper_2006_05874_gb300 import ihs

    for name in _declared_functions():
        assert name in ihs._SIGNATURES, name


def test_struct_layout_matches_header(tmp_path):
    from paper_2006_05874_gb300 import ihs

    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ihs.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ihs_params), sizeof(ihs_report),'
                   ' offsetof(ihs_report, m_levels), offsetof(ihs_params, seed), offsetof(ihs_params, nested),'
                   ' sizeof(ihs_problem), offsetof(ihs_problem, m_init));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [ctypes.sizeof(ihs.Params), ctypes.sizeof(ihs.Report),
                                     ihs.Report.m_levels.offset, ihs.Params.seed.offset, ihs.Params.nested.offset,
                                     ctypes.sizeof(ihs.Problem), ihs.Problem.m_init.offset]


def test_host_only_calls_without_gpu(built_lib):
    from paper_2006_05874_gb300 import ihs

    assert ihs.version().startswith("ihs-gb300")
    p = ihs.default_params()
    assert p.kind == ihs.SKETCH_SRHT and p.rho == 0.1 and p.m_init == 1
