"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
public header declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2602_19873_gb300 import build as nlbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nl_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_core_entry_points():
    names = _declared()
    for core in ("nl_build", "nl_density_pass", "nl_free"):
        assert core in names


def test_library_exports_every_declared_symbol():
    lib = nlbuild.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b(nl_[a-z0-9_]+)\b", out))
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads_without_gpu():
    import torch  # noqa: F401  (brings the CUDA runtime the library links against)
    lib = ctypes.CDLL(nlbuild.build())
    for name in _declared():
        assert hasattr(lib, name)
    lib.nl_last_error.restype = ctypes.c_char_p
    assert lib.nl_last_error() == b"no error"


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2602_19873_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "nl_oracle" not in txt, f


def test_binding_structs_match_the_header(tmp_path):
    """Sizes and field offsets of the ctypes structs equal those of the C
    structs of include/nl.h, measured by a C program compiled with gcc."""
    import ctypes as C

    from paper_2602_19873_gb300 import nl
    structs = {"nl_box": nl.nl_box, "nl_params": nl.nl_params, "nl_sizes": nl.nl_sizes,
               "nl_hiter_info": nl.nl_hiter_info, "nl_hiter_step": nl.nl_hiter_step}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nl.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
