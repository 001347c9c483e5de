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


def test_struct_layouts_match_header():
    # mirage_geom_t: 2 ints, 3 doubles, 2 ints, 4 doubles, 4 ints (natural alignment, no padding)
    assert ctypes.sizeof(binding.mirage_geom_t) == 88
    assert ctypes.sizeof(binding.mirage_opts_t) == 40  # double + 8 ints
    assert ctypes.sizeof(binding.mirage_problem_t) == 88 + 32


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
