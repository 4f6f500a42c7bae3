"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/discloop.h declares; host-only logic matches the oracle."""
import os
import re

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


# every call that takes a context or network handle, with that handle NULL and every
# other pointer NULL: a status, never a crash (no GPU needed)
NULL_HANDLE_CALLS = {
    "dl_set_stream": (None, None),
    "dl_load_gauge": (None, None, 0, -1.0, 12, 8),
    "dl_set_params": (None, 0.1, 0.01),
    "dl_noise_z4": (None, 1, 0, 1, None, 0, 0),
    "dl_noise_z4_tdil": (None, 1, 0, 1, None, 0, 0, 0, 1),
    "dl_apply": (None, 0, 0, 1, 1, None, None, None, 0),
    "dl_apply_noalloc": (None, 0, 0, 1, 1, None, None, None, 0),
    "dl_solve": (None, None, None, 1, 0, None, None),
    "dl_contract": (None, 0, None, None, 1, 0, 0, 0, None, 0),
    "dl_contract_slices": (None, 0, None, None, 1, 0, 0, 0, 1, None, 0),
    "dl_hpe_exact": (None, 1, None),
    "dl_tsm_run": (None, None, None, None, None, None, None),
    "dl_load_gauge_lat": (None, 0, None, 0, -1.0, 12, 12),
    "dl_set_params_lat": (None, 0, 0.1, 0.01),
    "dl_batch_loops": (None, None, None, None, None),
    "dl_profile": (None, 1, None),
    "dl_nn_create": (None, 2, 4, 3, None),
    "dl_nn_set_tensor_cores": (None, 1),
    "dl_nn_set_weights": (None, None),
    "dl_nn_get_weights": (None, None),
    "dl_nn_apply": (None, 1, None, None, 0),
    "dl_nn_apply_adjoint": (None, 1, None, None, 0),
    "dl_nn_loss_grad": (None, 1, None, None, 0, None, None),
    "dl_nn_train": (None, None, 1, None, None, 0, None),
    "dl_nn_loss_grad_residual": (None, 1, None, 0, None, None),
    "dl_fgcr_solve": (None, None, None, 1, None, None, 0, None),
    "dl_create_multi": (None, 1, None, 0, None),
    "dl_store_add": (None, None, 1),
    "dl_store_count": (None, None),
}
# calls without a handle argument, or whose NULL handle is a no-op by definition
NO_HANDLE = {"dl_create", "dl_momenta", "dl_kernel_launches", "dl_profile_stencils", "dl_destroy", "dl_nn_destroy", "dl_last_error",
             "dl_nn_weight_count", "dl_store_last_error", "dl_store_open", "dl_store_close", "dl_store_load",
             "dl_store_sources"}


def test_null_handles_are_rejected():
    import paper_1309_2256_gb300 as dl
    h = dl.lib()
    assert set(NULL_HANDLE_CALLS) | NO_HANDLE == _declared()
    for name, args in NULL_HANDLE_CALLS.items():
        assert getattr(h, name)(*args) == dl.DL_ERR_ARG, name
    h.dl_destroy(None)
    h.dl_nn_destroy(None)
    assert h.dl_nn_weight_count(None) == 0
    assert h.dl_last_error(None) is not None
    assert h.dl_profile_stencils(None) == dl.DL_ERR_ARG
