"""ctypes binding of libdiscloop.so: same names as the C ABI (include/discloop.h),
argument marshalling only.  Device buffers are passed as torch tensors (their
data_ptr) or raw integer addresses; host buffers as numpy arrays.  Negative
status codes raise DLError; non-fatal positive codes are returned."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdiscloop.so")

DL_OK, DL_ERR_ARG, DL_ERR_CUDA, DL_ERR_OOM, DL_ERR_STATE, DL_ERR_IO = 0, -1, -2, -3, -4, -5
DL_NOT_CONVERGED, DL_BREAKDOWN = 1, 3
DL_F64, DL_F32, DL_F16, DL_BF16, DL_F64_IEEE = 0, 1, 2, 3, 5
DL_C128, DL_C64 = 0, 1
(DL_OP_M, DL_OP_MDAG, DL_OP_HOP, DL_OP_MHAT, DL_OP_MHAT_DAG, DL_OP_PREP, DL_OP_RECON, DL_OP_BH) = range(8)
DL_EST_STANDARD, DL_EST_ONE_END, DL_EST_GEN, DL_EST_HPE = range(4)
DL_MAX_RHS = 32


class DLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"discloop status {status}: {msg}")
        self.status = status


class dl_solve_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("prec_hi", C.c_int), ("prec_lo", C.c_int),
                ("delta", C.c_double), ("flavour", C.c_int), ("chunk", C.c_int)]


class dl_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int * DL_MAX_RHS), ("resid", C.c_double * DL_MAX_RHS),
                ("true_resid", C.c_double * DL_MAX_RHS), ("reliable_updates", C.c_int), ("max_iters", C.c_int),
                ("seconds", C.c_double)]


class dl_tsm_params(C.Structure):
    _fields_ = [("n_hp", C.c_int), ("n_lp", C.c_int), ("tol_hp", C.c_double), ("tol_lp", C.c_double),
                ("prec_hp_lo", C.c_int), ("prec_lp_lo", C.c_int), ("delta_hp", C.c_double), ("block", C.c_int),
                ("seed", C.c_uint64), ("p2max", C.c_int), ("with_deriv", C.c_int), ("hpe", C.c_int),
                ("max_iter", C.c_int), ("chunk", C.c_int), ("lp_net", C.c_void_p), ("hp_guess", C.c_int), ("hpe_diff", C.c_int),
                ("tdil_dt", C.c_int), ("tdil_t0", C.c_int)]


class dl_tsm_info(C.Structure):
    _fields_ = [("np", C.c_int), ("nd", C.c_int), ("n_est", C.c_int), ("seconds_total", C.c_double),
                ("seconds_hp", C.c_double), ("seconds_lp", C.c_double), ("seconds_contract", C.c_double),
                ("iters_hp", C.c_longlong), ("iters_lp", C.c_longlong), ("not_converged", C.c_int),
                ("block", C.c_int), ("seconds_tune", C.c_double)]


class dl_batch_params(C.Structure):
    _fields_ = [("n", C.c_int), ("tol", C.c_double), ("prec_hi", C.c_int), ("prec_lo", C.c_int),
                ("delta", C.c_double), ("seed", C.c_uint64), ("max_iter", C.c_int), ("tile", C.c_int)]


class dl_batch_info(C.Structure):
    _fields_ = [("tile", C.c_int), ("instances", C.c_int), ("seconds_tune", C.c_double),
                ("seconds_solve", C.c_double), ("seconds_contract", C.c_double), ("iters_max", C.c_int * 16),
                ("resid_max", C.c_double * 16), ("not_converged", C.c_int)]


class dl_nn_train_params(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("seed", C.c_uint64), ("loss", C.c_int)]


class dl_fgcr_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("restart", C.c_int), ("inner_tol", C.c_double),
                ("flavour", C.c_int), ("normal", C.c_int)]


class dl_fgcr_stats(C.Structure):
    _fields_ = [("iters", C.c_int * DL_MAX_RHS), ("cycles", C.c_int * DL_MAX_RHS),
                ("true_resid", C.c_double * DL_MAX_RHS), ("op_applications", C.c_longlong),
                ("nn_applications", C.c_longlong), ("seconds", C.c_double)]


_lib = None

# name -> (restype, argtypes); mirrors include/discloop.h
_SIGS = {
    "dl_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.c_int, C.c_void_p]),
    "dl_destroy": (None, [C.c_void_p]),
    "dl_last_error": (C.c_char_p, [C.c_void_p]),
    "dl_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dl_load_gauge": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int]),
    "dl_set_params": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "dl_noise_z4": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "dl_noise_z4_tdil": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                   C.c_int]),
    "dl_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "dl_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(dl_solve_params),
                           C.POINTER(dl_solve_stats)]),
    "dl_momenta": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_void_p]),
    "dl_contract": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                              C.c_void_p, C.c_int]),
    "dl_contract_slices": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_void_p, C.c_int]),
    "dl_hpe_exact": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "dl_kernel_launches": (C.c_longlong, []),
    "dl_profile_stencils": (C.c_int, [C.c_void_p]),
    "dl_apply_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int]),
    "dl_create_multi": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), C.c_int, C.c_void_p]),
    "dl_load_gauge_lat": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int]),
    "dl_set_params_lat": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double]),
    "dl_batch_loops": (C.c_int, [C.c_void_p, C.POINTER(dl_batch_params), C.c_void_p, C.c_void_p,
                                 C.POINTER(dl_batch_info)]),
    "dl_profile": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "dl_tsm_run": (C.c_int, [C.c_void_p, C.POINTER(dl_tsm_params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.POINTER(dl_tsm_info)]),
    "dl_nn_create": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "dl_nn_destroy": (None, [C.c_void_p]),
    "dl_nn_weight_count": (C.c_longlong, [C.c_void_p]),
    "dl_nn_set_tensor_cores": (C.c_int, [C.c_void_p, C.c_int]),
    "dl_nn_set_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dl_nn_get_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dl_nn_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "dl_nn_apply_adjoint": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "dl_nn_loss_grad": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dl_nn_loss_grad_residual": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dl_nn_train": (C.c_int, [C.c_void_p, C.POINTER(dl_nn_train_params), C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p]),
    "dl_fgcr_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(dl_fgcr_params), C.c_int, C.c_void_p, C.c_void_p,
                                C.c_int, C.POINTER(dl_fgcr_stats)]),
    "dl_store_last_error": (C.c_char_p, []),
    "dl_store_open": (C.c_int, [C.POINTER(C.c_void_p), C.c_char_p, C.c_int64, C.c_int]),
    "dl_store_add": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "dl_store_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "dl_store_close": (C.c_int, [C.c_void_p]),
    "dl_store_load": (C.c_int, [C.c_char_p, C.c_int64, C.c_int64, C.c_void_p]),
    "dl_store_sources": (C.c_int, [C.c_int64, C.c_void_p]),
}


def lib():
    """Load libdiscloop.so (built in-tree by paper_1309_2256_gb300.build); fail loudly if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_1309_2256_gb300.build.build() first "
                              "(there is no fallback implementation)")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(ctx, status):
    if status < 0:
        msg = lib().dl_last_error(ctx).decode() if ctx else "(no context)"
        raise DLError(status, msg)
    return status


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def dl_create(dims, device=0, stream=None):
    h = C.c_void_p()
    d = (C.c_int * 4)(*dims)
    st = lib().dl_create(C.byref(h), d, int(device), _stream_ptr(stream))
    if st < 0:
        raise DLError(st, "dl_create failed (dims must be even and >= 2; CUDA device must exist)")
    return h.value


def dl_destroy(ctx):
    lib().dl_destroy(ctx)


def dl_last_error(ctx):
    return lib().dl_last_error(ctx).decode()


def dl_set_stream(ctx, stream):
    return _check(ctx, lib().dl_set_stream(ctx, _stream_ptr(stream)))


def dl_load_gauge(ctx, links, t_boundary=-1.0, recon_f32=12, recon_f16=8):
    """links: numpy complex128 [T][Z][Y][X][4][3][3] (host) or a CUDA complex128 tensor."""
    on_dev = 0 if isinstance(links, np.ndarray) else 1
    if on_dev == 0:
        links = np.ascontiguousarray(links, dtype=np.complex128)
    return _check(ctx, lib().dl_load_gauge(ctx, _ptr(links), on_dev, float(t_boundary), int(recon_f32), int(recon_f16)))


def dl_set_params(ctx, kappa, amu):
    return _check(ctx, lib().dl_set_params(ctx, float(kappa), float(amu)))


def dl_noise_z4(ctx, seed, first_index, n, out, dtype=DL_C128, quadrant=0):
    return _check(ctx, lib().dl_noise_z4(ctx, int(seed), int(first_index), int(n), _ptr(out), int(dtype), int(quadrant)))


def dl_noise_z4_tdil(ctx, seed, first_index, n, out, t0, dt, dtype=DL_C128, quadrant=0):
    return _check(ctx, lib().dl_noise_z4_tdil(ctx, int(seed), int(first_index), int(n), _ptr(out), int(dtype),
                                              int(quadrant), int(t0), int(dt)))


def dl_apply(ctx, op, prec, flavour, n, inp, aux, out, dtype=DL_C128):
    return _check(ctx, lib().dl_apply(ctx, int(op), int(prec), int(flavour), int(n), _ptr(inp), _ptr(aux), _ptr(out),
                                      int(dtype)))


def dl_solve(ctx, src, sol, n, dtype, params: dl_solve_params, stats: dl_solve_stats | None = None):
    stats = stats if stats is not None else dl_solve_stats()
    st = _check(ctx, lib().dl_solve(ctx, _ptr(src), _ptr(sol), int(n), int(dtype), C.byref(params), C.byref(stats)))
    return st, stats


def dl_momenta(p2max):
    cnt = C.c_int()
    st = lib().dl_momenta(int(p2max), C.byref(cnt), None)
    if st < 0:
        raise DLError(st, "dl_momenta: bad p2max")
    lst = np.zeros(3 * cnt.value, dtype=np.int32)
    lib().dl_momenta(int(p2max), C.byref(cnt), lst.ctypes.data)
    return lst.reshape(-1, 3)


def dl_contract(ctx, est, eta, sol, n, dtype, with_deriv, p2max, out, accumulate=0):
    return _check(ctx, lib().dl_contract(ctx, int(est), _ptr(eta), _ptr(sol), int(n), int(dtype), int(with_deriv),
                                         int(p2max), _ptr(out), int(accumulate)))


def dl_contract_slices(ctx, est, eta, sol, n, dtype, p2max, t0, dt, out, accumulate=0):
    return _check(ctx, lib().dl_contract_slices(ctx, int(est), _ptr(eta), _ptr(sol), int(n), int(dtype), int(p2max),
                                                int(t0), int(dt), _ptr(out), int(accumulate)))


def dl_hpe_exact(ctx, flavour=1):
    out = np.zeros((4, 4), dtype=np.complex128)
    _check(ctx, lib().dl_hpe_exact(ctx, int(flavour), out.ctypes.data))
    return out


def dl_tsm_run(ctx, params: dl_tsm_params, loops=None, obs_hp=None, obs_lp_pair=None, obs_lp=None):
    info = dl_tsm_info()
    st = _check(ctx, lib().dl_tsm_run(ctx, C.byref(params), _ptr(loops), _ptr(obs_hp), _ptr(obs_lp_pair), _ptr(obs_lp),
                                      C.byref(info)))
    return st, info


def dl_profile(ctx, enable=-1):
    """Returns float64 [4 stages][3 precisions][3] = (launches sampled, ms, items)."""
    out = np.zeros((4, 3, 3), dtype=np.float64)
    _check(ctx, lib().dl_profile(ctx, int(enable), out.ctypes.data))
    return out


def dl_profile_stencils():
    """float64 [4 storages][4 epilogues][2 dagger][4] = (launches, timed, ms, items)."""
    out = np.zeros((4, 4, 2, 4), dtype=np.float64)
    st = lib().dl_profile_stencils(out.ctypes.data)
    if st < 0:
        raise DLError(st, "dl_profile_stencils failed")
    return out


def dl_kernel_launches():
    return int(lib().dl_kernel_launches())


def dl_apply_noalloc(ctx, op, prec, flavour, n, inp, aux, out, dtype=DL_C128):
    """dl_apply with its working fields in the library's fixed 64 MiB device array (no allocation)."""
    return _check(ctx, lib().dl_apply_noalloc(ctx, int(op), int(prec), int(flavour), int(n), _ptr(inp), _ptr(aux),
                                              _ptr(out), int(dtype)))


def dl_create_multi(dims_list, device=0, stream=None):
    h = C.c_void_p()
    flat = [int(v) for d in dims_list for v in d]
    arr = (C.c_int * len(flat))(*flat)
    st = lib().dl_create_multi(C.byref(h), len(dims_list), arr, int(device), _stream_ptr(stream))
    if st < 0:
        raise DLError(st, "dl_create_multi failed")
    return h.value


def dl_load_gauge_lat(ctx, lat, links, t_boundary=-1.0, recon_f32=12, recon_f16=12):
    on_dev = 0 if isinstance(links, np.ndarray) else 1
    if on_dev == 0:
        links = np.ascontiguousarray(links, dtype=np.complex128)
    return _check(ctx, lib().dl_load_gauge_lat(ctx, int(lat), _ptr(links), on_dev, float(t_boundary), int(recon_f32),
                                               int(recon_f16)))


def dl_set_params_lat(ctx, lat, kappa, amu):
    return _check(ctx, lib().dl_set_params_lat(ctx, int(lat), float(kappa), float(amu)))


def dl_batch_loops(ctx, params: dl_batch_params, loops=None, sol=None):
    info = dl_batch_info()
    st = _check(ctx, lib().dl_batch_loops(ctx, C.byref(params), _ptr(loops), _ptr(sol), C.byref(info)))
    return st, info


# ---- learned preconditioner ---------------------------------------------------
# A network handle keeps its context for error messages: {"h": address, "ctx": ctx}.

def dl_nn_create(ctx, n_layers, channels, act_prec=DL_BF16):
    h = C.c_void_p()
    _check(ctx, lib().dl_nn_create(ctx, int(n_layers), int(channels), int(act_prec), C.byref(h)))
    return {"h": h.value, "ctx": ctx}


def dl_nn_destroy(nn):
    lib().dl_nn_destroy(nn["h"])


def dl_nn_weight_count(nn):
    return int(lib().dl_nn_weight_count(nn["h"]))


def dl_nn_set_tensor_cores(nn, enable):
    return _check(nn["ctx"], lib().dl_nn_set_tensor_cores(nn["h"], int(enable)))


def dl_nn_set_weights(nn, w):
    w = np.ascontiguousarray(w, dtype=np.complex64)
    assert w.size == dl_nn_weight_count(nn)
    return _check(nn["ctx"], lib().dl_nn_set_weights(nn["h"], w.ctypes.data))


def dl_nn_get_weights(nn):
    w = np.zeros(dl_nn_weight_count(nn), dtype=np.complex64)
    _check(nn["ctx"], lib().dl_nn_get_weights(nn["h"], w.ctypes.data))
    return w


def dl_nn_apply(nn, n, inp, out, dtype=DL_C128):
    return _check(nn["ctx"], lib().dl_nn_apply(nn["h"], int(n), _ptr(inp), _ptr(out), int(dtype)))


def dl_nn_apply_adjoint(nn, n, inp, out, dtype=DL_C128):
    return _check(nn["ctx"], lib().dl_nn_apply_adjoint(nn["h"], int(n), _ptr(inp), _ptr(out), int(dtype)))


def dl_nn_loss_grad(nn, n, eta, s, dtype=DL_C128):
    loss = np.zeros(1, dtype=np.float64)
    grad = np.zeros(dl_nn_weight_count(nn), dtype=np.complex64)
    _check(nn["ctx"], lib().dl_nn_loss_grad(nn["h"], int(n), _ptr(eta), _ptr(s), int(dtype), loss.ctypes.data,
                                            grad.ctypes.data))
    return float(loss[0]), grad


def dl_nn_loss_grad_residual(nn, n, eta, dtype=DL_C128):
    """Residual loss sum_k |M_u N(eta_k) - eta_k|^2 / |eta_k|^2 and its gradient (weight layout)."""
    loss = np.zeros(1, dtype=np.float64)
    grad = np.zeros(dl_nn_weight_count(nn), dtype=np.complex64)
    _check(nn["ctx"], lib().dl_nn_loss_grad_residual(nn["h"], int(n), _ptr(eta), int(dtype), loss.ctypes.data,
                                                     grad.ctypes.data))
    return float(loss[0]), grad


def dl_nn_train(nn, params: dl_nn_train_params, n_pairs, eta, s, dtype=DL_C128):
    hist = np.zeros(max(params.steps, 1), dtype=np.float64)
    _check(nn["ctx"], lib().dl_nn_train(nn["h"], C.byref(params), int(n_pairs), _ptr(eta), _ptr(s), int(dtype),
                                        hist.ctypes.data))
    return hist[:params.steps]


def dl_fgcr_solve(ctx, nn, params: dl_fgcr_params, n, src, sol, dtype=DL_C128):
    stats = dl_fgcr_stats()
    st = _check(ctx, lib().dl_fgcr_solve(ctx, nn["h"] if nn else None, C.byref(params), int(n), _ptr(src), _ptr(sol),
                                         int(dtype), C.byref(stats)))
    return st, stats


# ---- base-2 storage of per-noise loops (host only) ----

def _check_store(status):
    if status < 0:
        raise DLError(status, lib().dl_store_last_error().decode())
    return status


def _as_doubles(values):
    """A host array of float64 or complex128 as a contiguous float64 view."""
    a = np.ascontiguousarray(values)
    if a.dtype == np.complex128:
        return a.view(np.float64)
    if a.dtype != np.float64:
        raise TypeError("sources must be float64 or complex128 host arrays")
    return a


def dl_store_last_error():
    return lib().dl_store_last_error().decode()


def dl_store_open(prefix, n_values, resume=0):
    """Writer handle {"h", "n_values"} for sources of n_values doubles (a complex128
    value counts as two)."""
    h = C.c_void_p()
    _check_store(lib().dl_store_open(C.byref(h), os.fsencode(prefix), int(n_values), int(resume)))
    return {"h": h.value, "n_values": int(n_values)}


def dl_store_add(st, values):
    """values: host float64/complex128 array holding whole sources, in order."""
    a = _as_doubles(values)
    if a.size % st["n_values"]:
        raise ValueError(f"{a.size} doubles is not a whole number of sources of {st['n_values']}")
    return _check_store(lib().dl_store_add(st["h"], a.ctypes.data, a.size // st["n_values"]))


def dl_store_count(st):
    n = C.c_int64()
    _check_store(lib().dl_store_count(st["h"], C.byref(n)))
    return n.value


def dl_store_close(st):
    h, st["h"] = st["h"], None
    return _check_store(lib().dl_store_close(h))


def dl_store_load(prefix, n_values, n):
    out = np.zeros(int(n_values), dtype=np.float64)
    _check_store(lib().dl_store_load(os.fsencode(prefix), int(n_values), int(n), out.ctypes.data))
    return out


def dl_store_sources(n):
    out = np.zeros(int(n), dtype=np.int64)
    _check_store(lib().dl_store_sources(int(n), out.ctypes.data if n else None))
    return out
