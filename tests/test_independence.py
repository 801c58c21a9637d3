"""The oracle and the CUDA path share no code: the oracle's C sources include
only the C standard library and each other, the CUDA sources include only
their own headers and CUDA's, and neither Python side imports the other."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
CSRC = os.path.join(ROOT, "paper_2510_07764_gb300", "csrc")
PKG = os.path.join(ROOT, "paper_2510_07764_gb300")


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_oracle_c_includes_only_the_standard_library():
    std = {"math.h", "stdlib.h", "string.h", "complex.h", "stdio.h", "stddef.h", "stdint.h",
           "float.h", "limits.h"}
    for f in sorted(os.listdir(ORACLE)):
        if f.endswith((".c", ".h")):
            for inc in _includes(os.path.join(ORACLE, f)):
                assert inc in std or inc == "ppm_oracle.c", (f, inc)


def test_cuda_sources_include_nothing_from_the_oracle():
    own = set(os.listdir(CSRC)) | {"ppm.h"}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            src = open(os.path.join(CSRC, f)).read()
            # quoted includes are this library's own files; angle brackets are
            # the C++ and CUDA toolkits'
            for inc in re.findall(r'^\s*#\s*include\s*"([^"]+)"', src, re.M):
                assert inc in own, (f, inc)
            for inc in _includes(os.path.join(CSRC, f)):
                assert "oracle" not in inc, (f, inc)


def test_python_sides_do_not_import_each_other():
    imp = re.compile(r"^\s*(?:from|import)\s+([\w.]+)", re.M)
    for f in sorted(os.listdir(PKG)):
        if f.endswith(".py"):
            mods = imp.findall(open(os.path.join(PKG, f)).read())
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), f
    for f in sorted(os.listdir(ORACLE)):
        if f.endswith(".py"):
            mods = imp.findall(open(os.path.join(ORACLE, f)).read())
            assert not any(m.startswith("paper_2510_07764_gb300") for m in mods), (f, mods)
