"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/discloop.h declares; host-only logic matches the oracle."""
import os
import re

import numpy as np

from oracle import lattice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:dl_status|void|const char\*|long long)\s+(dl_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    import paper_1309_2256_gb300 as dl
    h = dl.lib()
    names = _declared()
    assert {"dl_create", "dl_solve", "dl_contract", "dl_tsm_run"} <= names
    for n in names:
        assert hasattr(h, n), n


def test_momentum_list_matches_oracle():
    import paper_1309_2256_gb300 as dl
    for p2 in (0, 1, 3, 4, 9):
        got = [tuple(int(v) for v in row) for row in dl.dl_momenta(p2)]
        assert got == lattice.momenta(p2)


def test_bad_arguments_are_rejected_without_gpu():
    import ctypes as C
    import paper_1309_2256_gb300 as dl
    h = dl.lib()
    cnt = C.c_int()
    assert h.dl_momenta(-1, C.byref(cnt), None) == dl.DL_ERR_ARG
    assert h.dl_momenta(4, None, None) == dl.DL_ERR_ARG
    out = C.c_void_p()
    odd = (C.c_int * 4)(4, 4, 3, 4)
    assert h.dl_create(C.byref(out), odd, 0, None) == dl.DL_ERR_ARG
    assert h.dl_solve(None, None, None, 1, 0, None, None) == dl.DL_ERR_ARG
    assert h.dl_tsm_run(None, None, None, None, None, None, None) == dl.DL_ERR_ARG
    assert np.isfinite(1.0)
