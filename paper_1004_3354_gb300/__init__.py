"""Python binding of libedgb, the GB300 exact-diagonalisation C ABI (include/ed.h).

Argument marshalling only: every function below forwards to the C entry point
of the same name; all computation runs in the library's CUDA kernels.  Device
vectors are torch tensors on the context's device (their data_ptr() is passed),
streams are torch.cuda.Stream objects (or None for the current stream).

The library must have been built (``__graft_entry__.build()`` or
``python paper_1004_3354_gb300/_build.py``); importing a function that needs it
raises RuntimeError when libedgb.so is missing.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libedgb.so")

ED_OK, ED_ERR_INVALID, ED_ERR_OOM, ED_ERR_CUDA, ED_ERR_TIMEOUT, ED_ERR_NOT_CONVERGED, ED_ERR_BUSY = range(7)
ED_PREC_FP64, ED_PREC_DF64, ED_PREC_FP32 = 0, 1, 2
ED_SPIN_UP, ED_SPIN_DN = 0, 1
ED_SECTOR_CSR = 1
ED_SECTOR_GENERIC = 2
ED_SECTOR_ACC_DF = 4
ED_MAX_K = 64
PREC_NAMES = {"fp64": ED_PREC_FP64, "df64": ED_PREC_DF64, "fp32": ED_PREC_FP32}
STATUS_NAMES = {0: "ED_OK", 1: "ED_ERR_INVALID", 2: "ED_ERR_OOM", 3: "ED_ERR_CUDA", 4: "ED_ERR_TIMEOUT",
                5: "ED_ERR_NOT_CONVERGED", 6: "ED_ERR_BUSY"}


class EdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ed_model(C.Structure):
    _fields_ = [("n_s", C.c_int), ("T", C.POINTER(C.c_double)), ("U_site", C.POINTER(C.c_double)),
                ("n_orb", C.c_int), ("orb0", C.c_int), ("Up", C.c_double), ("J", C.c_double),
                ("Jsf", C.c_double), ("Jph", C.c_double)]


class ed_sector_info(C.Structure):
    _fields_ = [("n_s", C.c_int), ("n_up", C.c_int), ("n_dn", C.c_int), ("prec", C.c_int),
                ("D_up", C.c_uint64), ("D_dn", C.c_uint64), ("dim", C.c_uint64),
                ("hops_up", C.c_uint64), ("hops_dn", C.c_uint64), ("mix_up", C.c_uint64),
                ("csr_nnz", C.c_uint64), ("table_bytes", C.c_uint64), ("nnz_per_row", C.c_double),
                ("kernel", C.c_int)]


class ed_lanczos_opts(C.Structure):
    _fields_ = [("k", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("check_every", C.c_int),
                ("seed", C.c_uint64), ("v0", C.c_void_p), ("reorth", C.c_int)]


class ed_lanczos_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("n_converged", C.c_int), ("residual", C.c_double * ED_MAX_K),
                ("apply_ms", C.c_double), ("total_ms", C.c_double)]


class ed_trlan_opts(C.Structure):
    _fields_ = [("k", C.c_int), ("tol", C.c_double), ("max_basis", C.c_int), ("keep", C.c_int),
                ("max_iter", C.c_int), ("check_every", C.c_int), ("seed", C.c_uint64), ("v0", C.c_void_p)]


class ed_trlan_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("n_converged", C.c_int),
                ("residual", C.c_double * ED_MAX_K), ("apply_ms", C.c_double), ("total_ms", C.c_double),
                ("basis_bytes", C.c_size_t)]


ED_MAX_TUNE = 16


class ed_tune_result(C.Structure):
    _fields_ = [("n_candidates", C.c_int), ("chosen", C.c_int), ("kernel", C.c_int * ED_MAX_TUNE),
                ("block", C.c_int * ED_MAX_TUNE), ("min_blocks", C.c_int * ED_MAX_TUNE),
                ("ms", C.c_double * ED_MAX_TUNE)]


class ed_batch_tune_result(C.Structure):
    _fields_ = [("n_candidates", C.c_int), ("chosen", C.c_int), ("chunk", C.c_int * ED_MAX_TUNE),
                ("ms_per_step", C.c_double * ED_MAX_TUNE)]


class ed_batch_info(C.Structure):
    _fields_ = [("steps", C.c_int), ("graph_replays", C.c_int), ("n_sectors", C.c_int), ("total_ms", C.c_double)]


class ed_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("prec", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("cf_depth", C.c_int), ("n_w", C.c_int), ("beta", C.c_double),
                ("seed", C.c_uint64), ("pack_dim", C.c_uint64)]


ED_SERVE_MAX_K = 16
ABI_VERSION = 3   # ED_ABI_VERSION of include/ed.h that these structures follow


class ed_request(C.Structure):
    _fields_ = [("model", C.POINTER(ed_model)), ("n_up", C.c_int), ("n_dn", C.c_int), ("want_G", C.c_int),
                ("orbital", C.c_int), ("spin", C.c_int), ("k", C.c_int)]


class ed_result(C.Structure):
    _fields_ = [("status", C.c_int), ("E0", C.c_double), ("iters", C.c_int), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("n_w", C.c_int), ("n_E", C.c_int), ("E", C.c_double * ED_SERVE_MAX_K)]


class ed_server_stats(C.Structure):
    _fields_ = [("queued", C.c_int), ("active", C.c_int), ("done", C.c_int), ("failed", C.c_int),
                ("max_active_seen", C.c_int), ("bytes_in_flight", C.c_size_t), ("n_latency", C.c_int),
                ("latency_p50_ms", C.c_double), ("latency_p99_ms", C.c_double),
                ("queue_p50_ms", C.c_double), ("queue_p99_ms", C.c_double)]


class ed_state(C.Structure):
    _fields_ = [("n_up", C.c_int), ("n_dn", C.c_int), ("E", C.c_double), ("vec", C.c_void_p)]


_lib = None

_SIGS = {
    "ed_last_error": (C.c_int, [C.c_char_p, C.c_size_t]),
    "ed_abi_version": (C.c_int, []),
    "ed_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]),
    "ed_ctx_destroy": (C.c_int, [C.c_void_p]),
    "ed_ctx_bytes_in_use": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "ed_sector_create": (C.c_int, [C.c_void_p, C.POINTER(ed_model), C.c_int, C.c_int, C.c_int, C.c_uint,
                                   C.POINTER(C.c_void_p)]),
    "ed_sector_destroy": (C.c_int, [C.c_void_p]),
    "ed_sector_get_info": (C.c_int, [C.c_void_p, C.POINTER(ed_sector_info)]),
    "ed_sector_basis": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "ed_sector_hops": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_sector_csr_rows": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_apply_h": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_apply_h_host": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_apply_h_csr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_convert": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_uint64, C.c_void_p]),
    "ed_dot": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.POINTER(C.c_double),
                         C.c_void_p]),
    "ed_dot_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "ed_lanczos": (C.c_int, [C.c_void_p, C.POINTER(ed_lanczos_opts), C.c_void_p, C.c_void_p,
                             C.POINTER(ed_lanczos_info), C.c_void_p]),
    "ed_dmft_update": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                 C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                 C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "ed_sector_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(ed_tune_result), C.c_void_p]),
    "ed_sector_set_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "ed_sector_get_variant": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "ed_tune_cache_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "ed_tune_cache_load": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int)]),
    "ed_lanczos_tr": (C.c_int, [C.c_void_p, C.POINTER(ed_trlan_opts), C.c_void_p, C.c_void_p,
                                C.POINTER(ed_trlan_info), C.c_void_p]),
    "ed_greens_cf": (C.c_int, [C.c_void_p, C.POINTER(ed_model), C.c_int, C.c_int, C.POINTER(ed_state),
                               C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p,
                               C.c_void_p, C.c_void_p]),
    "ed_greens_cf_z": (C.c_int, [C.c_void_p, C.POINTER(ed_model), C.c_int, C.c_int, C.POINTER(ed_state),
                                 C.c_double, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_batch_create": (C.c_int, [C.c_void_p, C.POINTER(ed_model), C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                  C.POINTER(C.c_void_p)]),
    "ed_batch_destroy": (C.c_int, [C.c_void_p]),
    "ed_batch_set_chunk": (C.c_int, [C.c_void_p, C.c_int]),
    "ed_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(ed_batch_tune_result), C.c_void_p]),
    "ed_batch_lanczos": (C.c_int, [C.c_void_p, C.POINTER(ed_lanczos_opts), C.c_void_p, C.c_void_p,
                                   C.POINTER(ed_batch_info), C.c_void_p]),
    "ed_server_create": (C.c_int, [C.c_void_p, C.POINTER(ed_server_opts), C.POINTER(C.c_void_p)]),
    "ed_server_destroy": (C.c_int, [C.c_void_p]),
    "ed_submit": (C.c_int, [C.c_void_p, C.POINTER(ed_request), C.POINTER(C.c_uint64)]),
    "ed_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(ed_result), C.c_void_p, C.POINTER(C.c_int)]),
    "ed_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ed_server_stats)]),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load libedgb.so once (RuntimeError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if L.ed_abi_version() != ABI_VERSION:
            raise RuntimeError(f"{LIB_PATH} has ABI version {L.ed_abi_version()}, this binding expects "
                               f"{ABI_VERSION}: rebuild it with __graft_entry__.build()")
        _lib = L
    return _lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().ed_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int, allow=()):
    if status != ED_OK and status not in allow:
        raise EdError(status, last_error())
    return status


def _ptr(t):
    """Address of a torch tensor's or numpy array's data (None stays NULL)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ model
class Model:
    """ed_model plus the host arrays it points to (kept alive here)."""

    def __init__(self, m):
        self.src = m
        self.T = np.ascontiguousarray(m.T, dtype=np.float64)
        self.U = np.ascontiguousarray(m.U_site, dtype=np.float64)
        self.c = ed_model(int(m.n_s), self.T.ctypes.data_as(C.POINTER(C.c_double)),
                          self.U.ctypes.data_as(C.POINTER(C.c_double)), int(m.n_orb),
                          int(getattr(m, "orb0", 0)), float(m.Up), float(m.J), float(m.Jsf), float(m.Jph))


# ---------------------------------------------------------------- context
def ed_ctx_create(device: int = 0, hbm_budget: int = 0):
    h = C.c_void_p()
    check(lib().ed_ctx_create(device, hbm_budget, C.byref(h)))
    return h


def ed_ctx_destroy(ctx):
    return check(lib().ed_ctx_destroy(ctx))


def ed_ctx_bytes_in_use(ctx) -> int:
    v = C.c_size_t()
    check(lib().ed_ctx_bytes_in_use(ctx, C.byref(v)))
    return v.value


def ed_sector_create(ctx, model, n_up: int, n_dn: int, prec=ED_PREC_FP64, flags: int = 0):
    mm = model if isinstance(model, Model) else Model(model)
    h = C.c_void_p()
    check(lib().ed_sector_create(ctx, C.byref(mm.c), n_up, n_dn, PREC_NAMES.get(prec, prec), flags, C.byref(h)))
    return h


def ed_sector_destroy(sec):
    return check(lib().ed_sector_destroy(sec))


def ed_sector_get_info(sec) -> ed_sector_info:
    info = ed_sector_info()
    check(lib().ed_sector_get_info(sec, C.byref(info)))
    return info


def ed_sector_basis(sec, spin: int) -> np.ndarray:
    info = ed_sector_get_info(sec)
    n = info.D_up if spin == ED_SPIN_UP else info.D_dn
    out = np.zeros(n, dtype=np.uint32)
    check(lib().ed_sector_basis(sec, spin, out.ctypes.data_as(C.c_void_p)))
    return out


def ed_sector_hops(sec, spin: int):
    info = ed_sector_get_info(sec)
    D = info.D_up if spin == ED_SPIN_UP else info.D_dn
    nh = info.hops_up if spin == ED_SPIN_UP else info.hops_dn
    ptr = np.zeros(D + 1, dtype=np.uint32)
    tgt = np.zeros(max(nh, 1), dtype=np.uint32)
    val = np.zeros(max(nh, 1), dtype=np.float64)
    check(lib().ed_sector_hops(sec, spin, ptr.ctypes.data_as(C.c_void_p), tgt.ctypes.data_as(C.c_void_p),
                               val.ctypes.data_as(C.c_void_p)))
    return ptr, tgt[:nh], val[:nh]


def ed_sector_csr_rows(sec, row0: int, nrows: int):
    info = ed_sector_get_info(sec)
    rp = np.zeros(nrows + 1, dtype=np.uint64)
    check(lib().ed_sector_csr_rows(sec, row0, nrows, rp.ctypes.data_as(C.c_void_p), None, None))
    nnz = int(rp[-1])
    cols = np.zeros(max(nnz, 1), dtype=np.uint32)
    vals = np.zeros(max(nnz, 1), dtype=np.float64)
    check(lib().ed_sector_csr_rows(sec, row0, nrows, rp.ctypes.data_as(C.c_void_p),
                                   cols.ctypes.data_as(C.c_void_p), vals.ctypes.data_as(C.c_void_p)))
    del info
    return rp.astype(np.int64), cols[:nnz].astype(np.int64), vals[:nnz]


# ------------------------------------------------------------------ apply
def ed_apply_h(sec, x, y, stream=None):
    return check(lib().ed_apply_h(sec, _ptr(x), _ptr(y), _stream(stream)))


def ed_apply_h_host(sec, n_vec, x_host, y_host, stream=None):
    """y = H x for n_vec host vectors (pinned torch tensors or numpy arrays,
    n_vec * dim elements each in the sector's format); returns when y is complete."""
    return check(lib().ed_apply_h_host(sec, int(n_vec), _ptr(x_host), _ptr(y_host), _stream(stream)))


def ed_apply_h_csr(sec, x, y, stream=None):
    return check(lib().ed_apply_h_csr(sec, _ptr(x), _ptr(y), _stream(stream)))


def ed_convert(src, src_prec, dst, dst_prec, n: int, stream=None):
    return check(lib().ed_convert(_ptr(src), PREC_NAMES.get(src_prec, src_prec), _ptr(dst),
                                  PREC_NAMES.get(dst_prec, dst_prec), n, _stream(stream)))


def ed_dot(ctx, x, y, n: int, prec, stream=None) -> float:
    r = C.c_double()
    check(lib().ed_dot(ctx, _ptr(x), _ptr(y), n, PREC_NAMES.get(prec, prec), C.byref(r), _stream(stream)))
    return r.value


def ed_dot_noalloc(x, y, n: int, prec, stream=None) -> float:
    """<x, y> without any device allocation (fixed static scratch; see include/ed.h)."""
    r = C.c_double()
    check(lib().ed_dot_noalloc(_ptr(x), _ptr(y), n, PREC_NAMES.get(prec, prec), C.byref(r), _stream(stream)))
    return r.value


# ---------------------------------------------------------------- Lanczos
def ed_lanczos(sec, k=1, tol=1e-12, max_iter=300, check_every=10, seed=1, v0=None, reorth=True,
               evecs=None, stream=None, allow_not_converged=False):
    """Returns (evals ndarray[k], info, status)."""
    o = ed_lanczos_opts(int(k), float(tol), int(max_iter), int(check_every), int(seed),
                        None if v0 is None else v0.data_ptr(), 1 if reorth else 0)
    ev = np.zeros(k, dtype=np.float64)
    info = ed_lanczos_info()
    st = lib().ed_lanczos(sec, C.byref(o), ev.ctypes.data_as(C.c_void_p), _ptr(evecs), C.byref(info),
                          _stream(stream))
    check(st, allow=(ED_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return ev, info, st


def ed_dmft_update(ctx, G_imp, beta, eps_d, mu, eps, V, e, w, n_fit, stream=None):
    """One DMFT self-consistency update.  G_imp: complex ndarray[n_w] at
    w_n = (2n+1) pi / beta; e, w: band-energy quadrature.  Returns
    (eps_new, V_new, chi2, Sigma, G_loc, Delta_new) with complex ndarrays."""
    def f64(a):
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    g = np.ascontiguousarray(np.asarray(G_imp, dtype=np.complex128)).view(np.float64)
    n_w = g.size // 2
    eps, V, e, w = f64(eps), f64(V), f64(e), f64(w)
    nb = eps.size
    eo, vo = np.zeros(nb), np.zeros(nb)
    outs = [np.zeros(2 * n_w) for _ in range(3)]
    c2 = C.c_double(0.0)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    check(lib().ed_dmft_update(ctx, n_w, float(beta), vp(g), float(eps_d), float(mu), nb, vp(eps), vp(V),
                               e.size, vp(e), vp(w), int(n_fit), vp(eo), vp(vo), C.byref(c2),
                               vp(outs[0]), vp(outs[1]), vp(outs[2]), _stream(stream)))
    cx = [o[0::2] + 1j * o[1::2] for o in outs]
    return eo, vo, c2.value, cx[0], cx[1], cx[2]


def ed_sector_autotune(sec, reps=5, stream=None):
    """Time the fast H*v variants of the sector and keep the fastest; returns
    the ed_tune_result (candidates, times, chosen index)."""
    r = ed_tune_result()
    check(lib().ed_sector_autotune(sec, int(reps), C.byref(r), _stream(stream)))
    return r


def ed_sector_set_variant(sec, variant):
    check(lib().ed_sector_set_variant(sec, int(variant)))


def ed_sector_get_variant(sec):
    v = C.c_int(-1)
    check(lib().ed_sector_get_variant(sec, C.byref(v)))
    return v.value


def ed_tune_cache_save(ctx, path):
    check(lib().ed_tune_cache_save(ctx, os.fsencode(path)))


def ed_tune_cache_load(ctx, path):
    n = C.c_int(0)
    check(lib().ed_tune_cache_load(ctx, os.fsencode(path), C.byref(n)))
    return n.value


def ed_lanczos_tr(sec, k=1, tol=1e-12, max_basis=40, keep=0, max_iter=2000, check_every=5, seed=1, v0=None,
                  evecs=None, stream=None, allow_not_converged=False):
    """Thick-restart Lanczos.  Returns (evals ndarray[k], info, status)."""
    o = ed_trlan_opts(int(k), float(tol), int(max_basis), int(keep), int(max_iter), int(check_every), int(seed),
                      None if v0 is None else v0.data_ptr())
    ev = np.zeros(k, dtype=np.float64)
    info = ed_trlan_info()
    st = lib().ed_lanczos_tr(sec, C.byref(o), ev.ctypes.data_as(C.c_void_p), _ptr(evecs), C.byref(info),
                             _stream(stream))
    check(st, allow=(ED_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return ev, info, st


# --------------------------------------------------------- Green's function
def ed_greens_cf(ctx, model, prec, states, beta, n_w, orbital=0, spin=ED_SPIN_UP, depth=150,
                 boltz_cut=1e-5, want_coeffs=False, stream=None):
    """states: list of (n_up, n_dn, E, device tensor).  Returns G (complex ndarray[n_w])
    and, if asked, the coefficient records (ndarray[kept*2, 2 + 2*depth])."""
    mm = model if isinstance(model, Model) else Model(model)
    arr = (ed_state * len(states))()
    for i, (nu, nd, E, v) in enumerate(states):
        arr[i] = ed_state(int(nu), int(nd), float(E), v.data_ptr())
    G = np.zeros(2 * n_w, dtype=np.float64)
    co = np.zeros(len(states) * 2 * (2 + 2 * depth), dtype=np.float64) if want_coeffs else None
    check(lib().ed_greens_cf(ctx, C.byref(mm.c), PREC_NAMES.get(prec, prec), len(states), arr, float(beta),
                             int(n_w), int(orbital), int(spin), int(depth), float(boltz_cut),
                             G.ctypes.data_as(C.c_void_p),
                             None if co is None else co.ctypes.data_as(C.c_void_p), _stream(stream)))
    Gc = G[0::2] + 1j * G[1::2]
    if want_coeffs:
        return Gc, co.reshape(len(states) * 2, 2 + 2 * depth)
    return Gc


def ed_greens_cf_z(ctx, model, prec, states, z, beta, orbital=0, spin=ED_SPIN_UP, depth=150,
                   boltz_cut=1e-5, want_coeffs=False, stream=None):
    """G(z) at complex frequencies z (array, every Im z > 0), e.g. z = w + i eta
    for the spectral function A(w) = -Im G / pi.  states as in ed_greens_cf."""
    mm = model if isinstance(model, Model) else Model(model)
    arr = (ed_state * len(states))()
    for i, (nu, nd, E, v) in enumerate(states):
        arr[i] = ed_state(int(nu), int(nd), float(E), v.data_ptr())
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128)).view(np.float64)
    n_z = zz.size // 2
    G = np.zeros(2 * n_z, dtype=np.float64)
    co = np.zeros(len(states) * 2 * (2 + 2 * depth), dtype=np.float64) if want_coeffs else None
    check(lib().ed_greens_cf_z(ctx, C.byref(mm.c), PREC_NAMES.get(prec, prec), len(states), arr, float(beta),
                               int(n_z), zz.ctypes.data_as(C.c_void_p), int(orbital), int(spin), int(depth),
                               float(boltz_cut), G.ctypes.data_as(C.c_void_p),
                               None if co is None else co.ctypes.data_as(C.c_void_p), _stream(stream)))
    Gc = G[0::2] + 1j * G[1::2]
    if want_coeffs:
        return Gc, co.reshape(len(states) * 2, 2 + 2 * depth)
    return Gc


def torch_dtype(prec):
    import torch
    p = PREC_NAMES.get(prec, prec)
    return {ED_PREC_FP64: torch.float64, ED_PREC_DF64: torch.float32, ED_PREC_FP32: torch.float32}[p]


def elems_per_value(prec) -> int:
    """torch elements per vector element (DF64 stores {hi, lo} float pairs)."""
    return 2 if PREC_NAMES.get(prec, prec) == ED_PREC_DF64 else 1


# ------------------------------------------------------------ batched sectors
def ed_batch_create(ctx, model, sectors, prec=ED_PREC_FP64):
    """sectors: list of (n_up, n_dn)."""
    mm = model if isinstance(model, Model) else Model(model)
    nu = np.array([a for a, _ in sectors], dtype=np.int32)
    nd = np.array([b for _, b in sectors], dtype=np.int32)
    h = C.c_void_p()
    check(lib().ed_batch_create(ctx, C.byref(mm.c), len(sectors), nu.ctypes.data_as(C.c_void_p),
                                nd.ctypes.data_as(C.c_void_p), PREC_NAMES.get(prec, prec), C.byref(h)))
    h._n = len(sectors)
    return h


def ed_batch_destroy(b):
    return check(lib().ed_batch_destroy(b))


def ed_batch_set_chunk(b, chunk):
    check(lib().ed_batch_set_chunk(b, int(chunk)))


def ed_batch_autotune(b, steps=16, stream=None):
    """Time each sector-packing chunk on a few Lanczos steps; keeps the fastest.
    Returns the ed_batch_tune_result."""
    r = ed_batch_tune_result()
    check(lib().ed_batch_autotune(b, int(steps), C.byref(r), _stream(stream)))
    return r


def ed_batch_lanczos(b, n_sectors, k=8, tol=1e-10, max_iter=300, check_every=10, seed=1, stream=None,
                     allow_not_converged=False):
    """Returns (evals ndarray[n_sectors, k], iters ndarray[n_sectors], info, status)."""
    o = ed_lanczos_opts(int(k), float(tol), int(max_iter), int(check_every), int(seed), None, 1)
    ev = np.zeros(n_sectors * k, dtype=np.float64)
    it = np.zeros(n_sectors, dtype=np.int32)
    info = ed_batch_info()
    st = lib().ed_batch_lanczos(b, C.byref(o), ev.ctypes.data_as(C.c_void_p), it.ctypes.data_as(C.c_void_p),
                                C.byref(info), _stream(stream))
    check(st, allow=(ED_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return ev.reshape(n_sectors, k), it, info, st


# ---------------------------------------------------------------- serving
def ed_server_create(ctx, hbm_budget=0, max_active=8, prec=ED_PREC_FP64, tol=1e-10, max_iter=400, cf_depth=100,
                     n_w=1024, beta=40.0, seed=1, pack_dim=0):
    o = ed_server_opts(int(hbm_budget), int(max_active), PREC_NAMES.get(prec, prec), float(tol), int(max_iter),
                       int(cf_depth), int(n_w), float(beta), int(seed), int(pack_dim))
    h = C.c_void_p()
    check(lib().ed_server_create(ctx, C.byref(o), C.byref(h)))
    h._n_w = int(n_w)
    return h


def ed_server_destroy(srv):
    return check(lib().ed_server_destroy(srv))


def ed_submit(srv, model, n_up, n_dn, want_G=True, orbital=None, spin=ED_SPIN_UP, k=1) -> int:
    mm = model if isinstance(model, Model) else Model(model)
    orb = int(getattr(mm.src, "orb0", 0)) if orbital is None else int(orbital)
    r = ed_request(C.pointer(mm.c), int(n_up), int(n_dn), 1 if want_G else 0, orb, int(spin), int(k))
    t = C.c_uint64()
    check(lib().ed_submit(srv, C.byref(r), C.byref(t)))
    return t.value


def ed_poll(srv, ticket, n_w=None):
    """Returns (done, ed_result or None, G complex ndarray or None)."""
    nw = srv._n_w if n_w is None else n_w
    res = ed_result()
    G = np.zeros(2 * nw, dtype=np.float64)
    done = C.c_int()
    check(lib().ed_poll(srv, int(ticket), C.byref(res), G.ctypes.data_as(C.c_void_p), C.byref(done)))
    if not done.value:
        return False, None, None
    return True, res, (G[0::2] + 1j * G[1::2]) if res.n_w else None


def ed_server_get_stats(srv) -> ed_server_stats:
    st = ed_server_stats()
    check(lib().ed_server_get_stats(srv, C.byref(st)))
    return st
