"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every function include/mirage.h declares (no compute calls without a GPU)."""
import ctypes
import os

import pytest

import synth
from paper_1101_5803_gb300 import binding
from paper_1101_5803_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    path = build()
    assert os.path.exists(path)
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = binding.header_functions()
    for n in ("mirage_create", "mirage_destroy", "mirage_eval_batch", "mirage_lcurve", "mirage_forward"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    for name in binding.header_functions():
        assert hasattr(lib, name), name


def test_binding_loads(lib):
    l2 = binding.load_library()
    assert l2.mirage_eval_batch is not None


def test_struct_layouts_match_header(tmp_path):
    # the binding's ctypes structures against the header as a C compiler lays
    # it out: every struct's size and every field's offset
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [binding.mirage_geom_t, binding.mirage_opts_t, binding.mirage_problem_t]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mirage.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("%zu\\n", sizeof({st.__name__}));')
        for f in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({st.__name__}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(binding.HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = []
    for st in structs:
        want.append(ctypes.sizeof(st))
        want += [getattr(st, f[0]).offset for f in st._fields_]
    assert got == want


def test_header_constants_match_binding():
    import re
    txt = open(binding.HEADER).read()
    assert int(re.search(r"#define MIRAGE_N_PHASE_CLOCKS (\d+)", txt).group(1)) == binding.N_PHASE_CLOCKS
    assert int(re.search(r"#define MIRAGE_MAX_LAM (\d+)", txt).group(1)) == binding.MAX_LAM
    assert int(re.search(r"#define MIRAGE_MAX_KPSF (\d+)", txt).group(1)) == binding.MAX_KPSF
    for name in ("MIRAGE_INTERP_BILINEAR", "MIRAGE_INTERP_NEAREST", "MIRAGE_INTERP_BICUBIC",
                 "MIRAGE_REG_IDENTITY", "MIRAGE_REG_GRADIENT", "MIRAGE_REG_LAPLACIAN"):
        m = re.search(r"#define %s (\d+)" % name, txt)
        assert m and int(m.group(1)) == getattr(binding, name), name
    assert (binding.MIRAGE_INTERP_NEAREST, binding.MIRAGE_INTERP_BICUBIC) == (synth.INTERP_NEAREST,
                                                                              synth.INTERP_BICUBIC)
