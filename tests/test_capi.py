"""The C-ABI library loads and exports every entry point its header declares
(no GPU needed: no compute call is made)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fe2_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    import paper_2305_07030_gb300 as m
    lib = C.CDLL(m.LIB_PATH)
    names = _declared()
    assert {"fe2_batch_create", "fe2_batch_solve", "fe2_batch_stress",
            "fe2_batch_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared but not exported"


def test_opts_defaults():
    import paper_2305_07030_gb300 as m
    o = m.make_opts()
    assert o.tol == 1e-8 and o.max_iter == 10_000_000 and o.dt_safety == 0.9
    assert o.precision == 1 and o.init == 1 and o.lead_iters == -1
    assert C.sizeof(m.Opts) == 72 and o.lead_tol == 1e-2
    assert o.launch == 0 and o.stall_window == 0


def test_errors_are_returned_not_raised_in_c():
    """Without a usable device create fails with a status and a message;
    argument errors are caught before any device call."""
    import paper_2305_07030_gb300 as m
    lib = m._lib
    h = C.c_void_p()
    # n_rve < 1 is rejected
    rc = lib.fe2_batch_create(0, None, None, None, None, None, None, None, None, None,
                              C.byref(h))
    assert rc == 1 and "n_rve" in m.last_error()
    # NULL handles are rejected
    assert lib.fe2_batch_stress(None, None, None, None, None) == 1
    assert lib.fe2_batch_destroy(None) == 0
