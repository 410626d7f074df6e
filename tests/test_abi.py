"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/compton.h declares (no compute call is made)."""
import ctypes
import os
import re

import paper_2206_02937_gb300 as cg
from paper_2206_02937_gb300 import buildlib as b

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "compton.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(compton_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = b.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert "compton_bin_pairs" in syms and "compton_scatter_step" in syms
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in compton.h but not exported"
    # the binding declares a signature for each of them
    assert set(syms) <= set(cg.SIGNATURES), set(syms) - set(cg.SIGNATURES)


def test_strerror_without_gpu():
    b.build()
    assert cg.strerror(cg.COMPTON_OK) == "ok"
    assert "range" in cg.strerror(cg.COMPTON_ERANGE)


def test_init_rejects_bad_config_without_touching_the_gpu():
    b.build()
    cfg = cg.compton_config(0, 10, 1.0, 0.05, 1, 0, 1e3, 8.0, 0, 0)  # n_cells = 0
    out = ctypes.c_void_p()
    assert cg.lib().compton_init(ctypes.byref(cfg), ctypes.byref(out)) == cg.COMPTON_EINVAL
    assert cg.lib().compton_init(None, ctypes.byref(out)) == cg.COMPTON_EINVAL
