"""The C-ABI library builds for sm_103a, loads, and exports every function declared in
include/*.h (no compute calls: this runs without a GPU)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_in_headers():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mg_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_1912_08445_gb300 as mg
    lib = mg.load()
    declared = declared_in_headers()
    assert len(declared) >= 25
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(mg.declared_symbols()) <= declared
    # the binding declares a signature for every header function
    assert declared <= set(mg.declared_symbols()) | set(), sorted(declared - set(mg.declared_symbols()))
    # raw symbol lookup through dlsym as well
    raw = ctypes.CDLL(mg.lib_path())
    for n in declared:
        getattr(raw, n)


def test_default_options_and_clean_failure_without_gpu():
    import torch
    import paper_1912_08445_gb300 as mg
    o = mg.default_options()
    assert o.precision == mg.MG_FP64 and abs(o.dshift_frac - 1 / 3) < 1e-16 and o.ng_period == 4
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(mg.MagritteError):
        mg.Context()


def test_invalid_options_rejected():
    import paper_1912_08445_gb300 as mg
    with pytest.raises(mg.MagritteError) as e:
        mg.Context(tol=-1.0)
    assert e.value.code == -1
