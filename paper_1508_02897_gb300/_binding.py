"""ctypes binding of libhd.so: the C ABI entry points under the same names.

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  Pointers are passed as integers (``tensor.data_ptr()``), streams as
``torch.cuda.Stream.cuda_stream`` integers.  The library must have been built
(``paper_1508_02897_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as ct
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hd.h")

HD_OK, HD_ERR_INVALID, HD_ERR_OOM, HD_ERR_CUDA, HD_ERR_NOT_CONVERGED, HD_ERR_NUMERIC, HD_ERR_TIMEOUT, HD_PENDING = range(8)
HD_C128, HD_C64, HD_C64_H, HD_C64_B = 0, 1, 2, 3
HD_SYMMETRIC = 0x100
HD_TCORE = 0x200
HD_SMOOTH = 0x400
HD_TF32X3 = 0x800
HD_ARNOLDI_FP64, HD_ARNOLDI_DS = 0, 1
HD_FACTOR_AUTO, HD_FACTOR_SIMT, HD_FACTOR_TCORE = 0, 1, 2
HD_MAX_RESTART = 256
HD_MAX_BLOCK = 128
STATUS_NAMES = {0: "HD_OK", 1: "HD_ERR_INVALID", 2: "HD_ERR_OOM", 3: "HD_ERR_CUDA", 4: "HD_ERR_NOT_CONVERGED",
                5: "HD_ERR_NUMERIC", 6: "HD_ERR_TIMEOUT", 7: "HD_PENDING"}
TIMER_CLASSES = ("factor", "subst", "gather", "matvec", "arnoldi", "other")


class hd_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("npml", ct.c_int32), ("h", ct.c_double),
                ("omega", ct.c_double), ("sigma0_over_omega", ct.c_double), ("pml_power", ct.c_int32)]


class hd_decomp(ct.Structure):
    _fields_ = [("nbx", ct.c_int32), ("nby", ct.c_int32), ("overlap", ct.c_int32),
                ("cut_x", ct.POINTER(ct.c_int32)), ("cut_y", ct.POINTER(ct.c_int32)),
                ("own_global_pml", ct.c_int32)]


class hd_gmres_opts(ct.Structure):
    _fields_ = [("restart", ct.c_int32), ("max_iters", ct.c_int32), ("rtol", ct.c_double), ("use_x0", ct.c_int32),
                ("arnoldi", ct.c_int32), ("graphs", ct.c_int32), ("reorth", ct.c_int32),
                ("precond_steps", ct.c_int32)]


class hd_gmres_stats(ct.Structure):
    _fields_ = [("iters", ct.c_int32), ("restarts", ct.c_int32), ("converged", ct.c_int32), ("status", ct.c_int32),
                ("relres_est", ct.c_double), ("relres_true", ct.c_double), ("t_solve_s", ct.c_double),
                ("second_passes", ct.c_int32), ("second_pass_vecs", ct.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hd_request_info(ct.Structure):
    _fields_ = [("queue_s", ct.c_double), ("run_s", ct.c_double), ("latency_s", ct.c_double),
                ("device_bytes", ct.c_uint64), ("batch", ct.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hd_server_counters(ct.Structure):
    _fields_ = [("queued", ct.c_int32), ("running", ct.c_int32), ("peak_running", ct.c_int32),
                ("completed", ct.c_uint64), ("bytes_in_use", ct.c_uint64), ("peak_bytes_in_use", ct.c_uint64),
                ("budget_bytes", ct.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HDError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed with {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_P = ct.c_void_p
_SIGS = {
    "hd_setup_medium": [ct.POINTER(_P), ct.POINTER(hd_grid), ct.POINTER(hd_decomp), _P, ct.c_int32, _P],
    "hd_query_workspace": [_P, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t),
                           ct.POINTER(ct.c_size_t)],
    "hd_factor_subdomains": [_P, _P, ct.c_size_t, _P, ct.c_size_t, _P],
    "hd_set_factor_path": [_P, ct.c_int32, ct.c_double],
    "hd_factor_report": [_P, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32), _P],
    "hd_matvec": [_P, _P, _P, ct.c_int32, _P],
    "hd_rhs_from_source": [_P, _P, _P, ct.c_int32, _P],
    "hd_apply_precond": [_P, _P, _P, ct.c_int32, _P, ct.c_size_t, _P],
    "hd_apply_ddm": [_P, _P, _P, ct.c_int32, ct.c_int32, _P, ct.c_size_t, _P, ct.c_size_t, _P],
    "hd_gmres_solve": [_P, _P, _P, ct.c_int32, ct.POINTER(hd_gmres_opts), _P, ct.c_size_t, _P, ct.c_size_t,
                       ct.POINTER(hd_gmres_stats), _P],
    "hd_apply_precond_noalloc": [_P, _P, _P, ct.c_int32, _P],
    "hd_query_block_workspace": [_P, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t)],
    "hd_block_gmres_solve": [_P, _P, _P, ct.c_int32, ct.POINTER(hd_gmres_opts), _P, ct.c_size_t, _P, ct.c_size_t,
                             ct.POINTER(hd_gmres_stats), _P],
    "hd_autotune": [_P, _P, _P, _P, ct.c_size_t, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32),
                    ct.POINTER(ct.c_float), _P],
    "hd_set_profiling": [_P, ct.c_int32],
    "hd_get_timers": [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.c_int32, ct.c_int32, _P],
    "hd_check_status": [_P, ct.c_int32, _P],
    "hd_destroy": [_P],
    "hd_server_create": [ct.POINTER(_P), ct.c_size_t, ct.c_int32, ct.c_int32],
    "hd_submit": [_P, ct.POINTER(hd_grid), ct.POINTER(hd_decomp), _P, _P, ct.c_int32, ct.c_int32,
                  ct.POINTER(hd_gmres_opts), _P, ct.POINTER(ct.c_uint64)],
    "hd_poll": [_P, ct.c_uint64, ct.POINTER(hd_gmres_stats), ct.POINTER(hd_request_info), ct.c_int64],
    "hd_server_info": [_P, ct.POINTER(hd_server_counters)],
    "hd_server_destroy": [_P],
    "hd_last_error": [],
    "hd_version": [],
}

_lib = None


def declared_symbols():
    """Names of the functions declared in include/hd.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(hd_\w+)\s*\(", text, flags=re.M)))


def lib():
    """Loads libhd.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhd.so not found at {LIB_PATH}: run paper_1508_02897_gb300.build.build() first")
        L = ct.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ct.c_char_p if name in ("hd_last_error", "hd_version") else ct.c_int
        _lib = L
    return _lib


def _check(fn, rc, allow=()):
    if rc != HD_OK and rc not in allow:
        raise HDError(fn, rc, lib().hd_last_error().decode())
    return rc


def _cuts(cuts):
    if cuts is None:
        return None, None
    arr = (ct.c_int32 * len(cuts))(*[int(c) for c in cuts])
    return arr, ct.cast(arr, ct.POINTER(ct.c_int32))


def hd_setup_medium(nx, ny, npml, h, omega, c_ptr, precision, stream, nbx, nby, overlap, cut_x=None, cut_y=None,
                    own_global_pml=1, sigma0_over_omega=20.0, pml_power=2):
    g = hd_grid(nx, ny, npml, h, omega, sigma0_over_omega, pml_power)
    kx, px = _cuts(cut_x)
    ky, py = _cuts(cut_y)
    d = hd_decomp(nbx, nby, overlap, px, py, own_global_pml)
    ctx = _P()
    _check("hd_setup_medium", lib().hd_setup_medium(ct.byref(ctx), ct.byref(g), ct.byref(d), c_ptr, precision, stream))
    return ctx


def hd_query_workspace(ctx, nrhs, restart):
    f, k, s = ct.c_size_t(), ct.c_size_t(), ct.c_size_t()
    _check("hd_query_workspace", lib().hd_query_workspace(ctx, nrhs, restart, ct.byref(f), ct.byref(k), ct.byref(s)))
    return f.value, k.value, s.value


def hd_factor_subdomains(ctx, factor_ptr, factor_bytes, scratch_ptr, scratch_bytes, stream):
    _check("hd_factor_subdomains", lib().hd_factor_subdomains(ctx, factor_ptr, factor_bytes, scratch_ptr, scratch_bytes, stream))


def hd_set_factor_path(ctx, path, pivot_ratio=0.5):
    _check("hd_set_factor_path", lib().hd_set_factor_path(ctx, int(path), float(pivot_ratio)))


def hd_factor_report(ctx, stream):
    """(boxes kept from the tensor-core factorisation, boxes factorised with partial pivoting)."""
    t, p = ct.c_int32(), ct.c_int32()
    _check("hd_factor_report", lib().hd_factor_report(ctx, ct.byref(t), ct.byref(p), stream))
    return t.value, p.value


def hd_matvec(ctx, x_ptr, y_ptr, nrhs, stream):
    _check("hd_matvec", lib().hd_matvec(ctx, x_ptr, y_ptr, nrhs, stream))


def hd_rhs_from_source(ctx, f_ptr, b_ptr, nrhs, stream):
    _check("hd_rhs_from_source", lib().hd_rhs_from_source(ctx, f_ptr, b_ptr, nrhs, stream))


def hd_apply_precond(ctx, r_ptr, z_ptr, nrhs, scratch_ptr, scratch_bytes, stream):
    _check("hd_apply_precond", lib().hd_apply_precond(ctx, r_ptr, z_ptr, nrhs, scratch_ptr, scratch_bytes, stream))


def hd_apply_ddm(ctx, f_ptr, u_ptr, nrhs, nsteps, work_ptr, work_bytes, scratch_ptr, scratch_bytes, stream):
    _check("hd_apply_ddm", lib().hd_apply_ddm(ctx, f_ptr, u_ptr, nrhs, nsteps, work_ptr, work_bytes, scratch_ptr,
                                              scratch_bytes, stream))


def hd_apply_precond_noalloc(ctx, r_ptr, z_ptr, nrhs, stream):
    """Preconditioner application whose staging lives in the library's fixed 64 MiB array
    (for callers that cannot allocate device memory)."""
    _check("hd_apply_precond_noalloc", lib().hd_apply_precond_noalloc(ctx, r_ptr, z_ptr, nrhs, stream))


def hd_gmres_solve(ctx, b_ptr, x_ptr, nrhs, restart, max_iters, rtol, krylov_ptr, krylov_bytes, scratch_ptr,
                   scratch_bytes, stream, use_x0=0, arnoldi=HD_ARNOLDI_FP64, graphs=0, reorth=0,
                   raise_on_not_converged=False, precond_steps=1):
    o = hd_gmres_opts(restart, max_iters, rtol, use_x0, arnoldi, graphs, reorth, precond_steps)
    st = (hd_gmres_stats * nrhs)()
    allow = () if raise_on_not_converged else (HD_ERR_NOT_CONVERGED,)
    rc = _check("hd_gmres_solve", lib().hd_gmres_solve(ctx, b_ptr, x_ptr, nrhs, ct.byref(o), krylov_ptr, krylov_bytes,
                                                       scratch_ptr, scratch_bytes, st, stream), allow)
    return rc, [s.as_dict() for s in st]


def hd_query_block_workspace(ctx, p, restart):
    """(krylov bytes, scratch bytes) of the block solver for p right-hand sides."""
    k, s = ct.c_size_t(), ct.c_size_t()
    _check("hd_query_block_workspace", lib().hd_query_block_workspace(ctx, p, restart, ct.byref(k), ct.byref(s)))
    return k.value, s.value


def hd_block_gmres_solve(ctx, b_ptr, x_ptr, p, restart, max_iters, rtol, krylov_ptr, krylov_bytes, scratch_ptr,
                         scratch_bytes, stream, use_x0=0):
    o = hd_gmres_opts(restart, max_iters, rtol, use_x0, HD_ARNOLDI_FP64, 0, 0, 1)
    st = (hd_gmres_stats * p)()
    rc = _check("hd_block_gmres_solve", lib().hd_block_gmres_solve(ctx, b_ptr, x_ptr, p, ct.byref(o), krylov_ptr,
                                                                   krylov_bytes, scratch_ptr, scratch_bytes, st,
                                                                   stream), (HD_ERR_NOT_CONVERGED,))
    return rc, [s.as_dict() for s in st]


def hd_autotune(ctx, r_ptr, z_ptr, scratch_ptr, scratch_bytes, stream):
    """Times the substitution launch shapes and keeps the fastest; returns (threads, stages, ms)."""
    t, n, ms = ct.c_int32(), ct.c_int32(), ct.c_float()
    _check("hd_autotune", lib().hd_autotune(ctx, r_ptr, z_ptr, scratch_ptr, scratch_bytes, ct.byref(t), ct.byref(n),
                                            ct.byref(ms), stream))
    return t.value, n.value, ms.value


def hd_set_profiling(ctx, on):
    _check("hd_set_profiling", lib().hd_set_profiling(ctx, int(bool(on))))


def hd_get_timers(ctx, stream, reset=False):
    n = len(TIMER_CLASSES)
    ms = (ct.c_double * n)()
    la = (ct.c_int64 * n)()
    _check("hd_get_timers", lib().hd_get_timers(ctx, ms, la, n, int(reset), stream))
    return {TIMER_CLASSES[i]: (ms[i], la[i]) for i in range(n)}


def hd_check_status(ctx, stream, clear=True):
    return _check("hd_check_status", lib().hd_check_status(ctx, int(clear), stream))


def hd_destroy(ctx):
    _check("hd_destroy", lib().hd_destroy(ctx))


def hd_last_error():
    return lib().hd_last_error().decode()


def hd_version():
    return lib().hd_version().decode()


def hd_server_create(hbm_budget_bytes, max_slots, device=0):
    srv = _P()
    _check("hd_server_create", lib().hd_server_create(ct.byref(srv), int(hbm_budget_bytes), int(max_slots), int(device)))
    return srv


def hd_submit(srv, nx, ny, npml, h, omega, c_ptr, f_ptr, nrhs, precision, restart, max_iters, rtol, x_ptr, nbx, nby,
              overlap, cut_x=None, cut_y=None, own_global_pml=1, arnoldi=HD_ARNOLDI_FP64, sigma0_over_omega=20.0,
              pml_power=2, reorth=0, precond_steps=1):
    """Queues a solve; host buffers (c, f, x) must stay alive until hd_poll reports completion."""
    g = hd_grid(nx, ny, npml, h, omega, sigma0_over_omega, pml_power)
    kx, px = _cuts(cut_x)
    ky, py = _cuts(cut_y)
    d = hd_decomp(nbx, nby, overlap, px, py, own_global_pml)
    o = hd_gmres_opts(restart, max_iters, rtol, 0, arnoldi, 0, reorth, precond_steps)
    t = ct.c_uint64()
    _check("hd_submit", lib().hd_submit(srv, ct.byref(g), ct.byref(d), c_ptr, f_ptr, nrhs, precision, ct.byref(o),
                                        x_ptr, ct.byref(t)))
    return t.value


def hd_poll(srv, ticket, nrhs, timeout_us=-1):
    """Returns (status, stats list, info dict); status HD_PENDING while queued or running."""
    st = (hd_gmres_stats * nrhs)()
    info = hd_request_info()
    rc = lib().hd_poll(srv, ct.c_uint64(ticket), st, ct.byref(info), int(timeout_us))
    if rc == HD_PENDING:
        return rc, None, None
    _check("hd_poll", rc, allow=(HD_ERR_NOT_CONVERGED,))
    return rc, [x.as_dict() for x in st], info.as_dict()


def hd_server_info(srv):
    c = hd_server_counters()
    _check("hd_server_info", lib().hd_server_info(srv, ct.byref(c)))
    return c.as_dict()


def hd_server_destroy(srv):
    _check("hd_server_destroy", lib().hd_server_destroy(srv))
