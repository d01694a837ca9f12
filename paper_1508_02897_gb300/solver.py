"""Python front end of libhd: device memory and streams come from PyTorch,
every computation runs in the library's CUDA kernels through the C ABI."""
from __future__ import annotations

import time
from typing import Optional, Sequence

import numpy as np
import torch

from . import _binding as B


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _storage_flag(prec: int, symmetric: bool, tcore, smoothing: bool = False) -> int:
    """Storage of the S_j^{-1} (tensor-core operand layout, c64 only: ``tcore`` True or
    "tf32" for TF32 planes, "x3" for TF32 hi/lo pairs with FP32-grade products; upper
    tiles; or full) and the optional smoothing function of the sum of local solutions."""
    sm = B.HD_SMOOTH if smoothing else 0
    if tcore:
        if prec != B.HD_C64:
            raise ValueError("tensor-core storage needs precision c64")
        if tcore not in (True, "tf32", "x3"):
            raise ValueError("tcore: False, True / 'tf32' or 'x3'")
        return B.HD_TCORE | (B.HD_TF32X3 if tcore == "x3" else 0) | sm
    return (B.HD_SYMMETRIC if symmetric else 0) | sm


class HelmholtzDDM:
    """One medium on one GPU: PML tables, per-box factors and the solvers.

    Grid: N x N interior cells (h = 1/N) plus npml PML cells per side; vectors
    are complex128 tensors of shape [..., n, n] with n = N + 2 npml (x fastest).
    """

    def __init__(self, N: int, npml: int, omega: float, c, nbx: int, nby: int, overlap: int,
                 precision: str = "c64", cut_x: Optional[Sequence[int]] = None, cut_y: Optional[Sequence[int]] = None,
                 own_global_pml: bool = True, sigma0_over_omega: float = 20.0, pml_power: int = 2,
                 device: str = "cuda", stream: Optional[torch.cuda.Stream] = None, factor: bool = True,
                 symmetric: bool = True, tcore=False, smoothing: bool = False,
                 factor_path: str = "auto", pivot_ratio: float = 0.5):
        if not torch.cuda.is_available():
            raise RuntimeError("HelmholtzDDM needs a CUDA device: there is no CPU path")
        self.N, self.npml, self.n = N, npml, N + 2 * npml
        self.device = torch.device(device)
        self.stream = stream
        self.prec = {"c64": B.HD_C64, "c64h": B.HD_C64_H, "c64b": B.HD_C64_B, "c128": B.HD_C128}[precision]
        c_t = torch.as_tensor(np.asarray(c, dtype=np.float64) if not torch.is_tensor(c) else c,
                              dtype=torch.float64).to(self.device).contiguous()
        assert c_t.shape == (self.n, self.n), f"velocity must be {(self.n, self.n)}"
        self.ctx = B.hd_setup_medium(N, N, npml, 1.0 / N, omega, c_t.data_ptr(),
                                     self.prec | _storage_flag(self.prec, symmetric, tcore, smoothing), self._st(),
                                     nbx, nby, overlap, cut_x, cut_y, int(own_global_pml), sigma0_over_omega,
                                     pml_power)
        fb, _, sb = B.hd_query_workspace(self.ctx, 1, 1)
        self.factor_bytes, self.scratch_bytes = fb, sb
        # workspaces are allocated on the stream the kernels run on, so the caching
        # allocator never hands a replaced buffer out while queued kernels still use it
        with torch.cuda.stream(self.stream):
            self.factor_buf = torch.empty(max(fb, 16), dtype=torch.uint8, device=self.device)
            self.scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device=self.device)
        self._krylov = {}
        self.factored = False
        B.hd_set_factor_path(self.ctx, {"auto": B.HD_FACTOR_AUTO, "simt": B.HD_FACTOR_SIMT,
                                        "tcore": B.HD_FACTOR_TCORE}[factor_path], pivot_ratio)
        if factor:
            self.factor()

    def _st(self) -> int:
        return _stream_ptr(self.stream)

    def factor(self):
        B.hd_factor_subdomains(self.ctx, self.factor_buf.data_ptr(), self.factor_bytes, self.scratch.data_ptr(),
                               self.scratch_bytes, self._st())
        self.factored = True

    def factor_report(self):
        """(boxes kept from the tensor-core factorisation, boxes factorised with partial pivoting)."""
        return B.hd_factor_report(self.ctx, self._st())

    def autotune(self):
        """Picks the substitution launch shape by timing (cached per shape for the process)."""
        r = torch.zeros((self.n, self.n), dtype=torch.complex128, device=self.device)
        z = torch.empty_like(r)
        return B.hd_autotune(self.ctx, r.data_ptr(), z.data_ptr(), self.scratch.data_ptr(), self.scratch_bytes,
                             self._st())

    def _vec(self, x):
        x = torch.as_tensor(x, dtype=torch.complex128, device=self.device).contiguous()
        nrhs = x.numel() // (self.n * self.n)
        assert x.numel() == nrhs * self.n * self.n
        return x, nrhs

    def matvec(self, x):
        x, nrhs = self._vec(x)
        y = torch.empty_like(x)
        B.hd_matvec(self.ctx, x.data_ptr(), y.data_ptr(), nrhs, self._st())
        return y

    def rhs(self, f):
        f, nrhs = self._vec(f)
        b = torch.empty_like(f)
        B.hd_rhs_from_source(self.ctx, f.data_ptr(), b.data_ptr(), nrhs, self._st())
        return b

    def apply_precond(self, r, out=None):
        r, nrhs = self._vec(r)
        z = torch.empty_like(r) if out is None else out
        B.hd_apply_precond(self.ctx, r.data_ptr(), z.data_ptr(), nrhs, self.scratch.data_ptr(), self.scratch_bytes,
                           self._st())
        return z

    def apply_ddm(self, f, steps: int, out=None):
        """Multi-step overlapping DDM (hd_apply_ddm): the sum of `steps` rounds of local
        solves, each round's sources the neighbours' residuals on the owned boxes."""
        f, nrhs = self._vec(f)
        u = torch.empty_like(f) if out is None else out
        _, _, sb = B.hd_query_workspace(self.ctx, nrhs, 1)
        with torch.cuda.stream(self.stream):
            work = torch.empty(2 * f.numel() * 16, dtype=torch.uint8, device=self.device)
            if sb > self.scratch_bytes:
                self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
                self.scratch_bytes = sb
        B.hd_apply_ddm(self.ctx, f.data_ptr(), u.data_ptr(), nrhs, steps, work.data_ptr(), work.numel(),
                       self.scratch.data_ptr(), self.scratch_bytes, self._st())
        return u

    def krylov_workspace(self, restart: int, nrhs: int = 1):
        key = (restart, nrhs)
        if key not in self._krylov:
            _, kb, sb = B.hd_query_workspace(self.ctx, nrhs, restart)
            self._krylov.clear()
            with torch.cuda.stream(self.stream):
                self._krylov[key] = torch.empty(kb, dtype=torch.uint8, device=self.device)
                if sb > self.scratch_bytes:
                    self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
                    self.scratch_bytes = sb
        return self._krylov[key]

    def solve(self, b, restart: int = 50, rtol: float = 1e-8, max_iters: int = 1000, x0=None, out=None,
              arnoldi: str = "auto", graphs: bool = False, reorth: str = "selective", precond_steps: int = 1):
        """FGMRES solve of A x = b.  ``arnoldi``: "fp64", "ds" (double-single
        Gram-Schmidt on the FP32 pipes) or "auto" (ds with FP32 factors, fp64 with c128).
        ``reorth``: "always" (CGS2) or "selective" (second pass only after a cancellation
        of more than a factor 10).  ``precond_steps``: steps of the overlapping DDM used as
        the preconditioner (1: the one-step preconditioner of Eq. (pc))."""
        b, nrhs = self._vec(b)
        if out is not None:
            x = out
            if x0 is not None:   # the solver starts from the contents of x
                x.copy_(self._vec(x0)[0].view_as(x))
        elif x0 is not None:
            x = self._vec(x0)[0].clone()
        else:
            x = torch.empty_like(b)
        kws = self.krylov_workspace(restart, nrhs)
        rc, stats = B.hd_gmres_solve(self.ctx, b.data_ptr(), x.data_ptr(), nrhs, restart, max_iters, rtol,
                                     kws.data_ptr(), kws.numel(), self.scratch.data_ptr(), self.scratch_bytes,
                                     self._st(), use_x0=int(x0 is not None), arnoldi=self._arnoldi(arnoldi),
                                     graphs=int(graphs), reorth={"always": 0, "selective": 1}[reorth],
                                     precond_steps=int(precond_steps))
        return x, stats

    def block_solve(self, b, restart: int = 10, rtol: float = 1e-8, max_iters: int = 1000, x0=None):
        """Block flexible GMRES (hd_block_gmres_solve) of A X = B for the p sources in b
        ([p, n, n]) sharing one Krylov space; `restart` and `max_iters` count block steps."""
        b, p = self._vec(b)
        x = self._vec(x0)[0].clone() if x0 is not None else torch.empty_like(b)
        kb, sb = B.hd_query_block_workspace(self.ctx, p, restart)
        with torch.cuda.stream(self.stream):
            kws = torch.empty(kb, dtype=torch.uint8, device=self.device)
            if sb > self.scratch_bytes:
                self.scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
                self.scratch_bytes = sb
        rc, stats = B.hd_block_gmres_solve(self.ctx, b.data_ptr(), x.data_ptr(), p, restart, max_iters, rtol,
                                           kws.data_ptr(), kb, self.scratch.data_ptr(), self.scratch_bytes,
                                           self._st(), use_x0=int(x0 is not None))
        return x, stats

    def _arnoldi(self, mode: str) -> int:
        if mode == "auto":
            mode = "ds" if self.prec != B.HD_C128 else "fp64"
        return {"fp64": B.HD_ARNOLDI_FP64, "ds": B.HD_ARNOLDI_DS}[mode]

    def set_profiling(self, on: bool = True):
        B.hd_set_profiling(self.ctx, on)

    def timers(self, reset: bool = False):
        return B.hd_get_timers(self.ctx, self._st(), reset)

    def close(self):
        if getattr(self, "ctx", None):
            B.hd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_host(c_host, f_host, N: int, npml: int, omega: float, nbx: int, nby: int, overlap: int,
               restart: int, rtol: float, max_iters: int = 5000, precision: str = "c64", cut_x=None, cut_y=None,
               device: str = "cuda", arnoldi: str = "auto", symmetric: bool = True, reorth: str = "selective",
               tcore: bool = False, smoothing: bool = False):
    """End-to-end solve from host arrays: velocity c [n][n] (float64) and source
    samples f [nrhs][n][n] (complex128), preferably in pinned memory.  Copies in,
    sets up the medium, factorises, forms b = J h^2 f, runs FGMRES and copies the
    solution back.  Returns (x on the host, stats, bytes copied in, bytes out)."""
    dev = torch.device(device)
    c_d = torch.as_tensor(c_host).to(dev, non_blocking=True)
    f_d = torch.as_tensor(f_host).to(dev, non_blocking=True)
    s = HelmholtzDDM(N, npml, omega, c_d, nbx, nby, overlap, precision=precision, cut_x=cut_x, cut_y=cut_y,
                     device=device, symmetric=symmetric, tcore=tcore, smoothing=smoothing)
    b = s.rhs(f_d)
    x, stats = s.solve(b, restart=restart, rtol=rtol, max_iters=max_iters, arnoldi=arnoldi, reorth=reorth)
    x_h = x.to("cpu")
    s.close()
    h2d = c_d.numel() * c_d.element_size() + f_d.numel() * f_d.element_size()
    return x_h, stats, h2d, x_h.numel() * x_h.element_size()


class Server:
    """Continuous-batching solve server (hd_server_*): requests of any grid,
    medium and number of sources run concurrently within an HBM budget."""

    def __init__(self, hbm_budget_bytes: int = 160 << 30, max_slots: int = 4, device: int = 0):
        self.srv = B.hd_server_create(hbm_budget_bytes, max_slots, device)
        self._keep = {}

    def submit(self, c, f, N, npml, omega, nbx, nby, overlap, restart, rtol, max_iters=5000, precision="c64",
               cut_x=None, cut_y=None, arnoldi="auto", symmetric=True, reorth="selective", tcore=False,
               smoothing=False, out=None):
        """c: float64 [n][n], f: complex128 [nrhs][n][n] host arrays (pinned memory, e.g. numpy
        views of pinned torch tensors, makes the copies direct); out: optional host array for
        the solutions, shaped like f.  Returns a ticket."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.complex128)
        if f.ndim == 2:
            f = f[None]
        if out is not None:
            x = out.reshape(f.shape)
            if x.dtype != np.complex128 or not x.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a contiguous complex128 array shaped like f")
        else:
            x = np.empty_like(f)
        prec = {"c64": B.HD_C64, "c64h": B.HD_C64_H, "c64b": B.HD_C64_B, "c128": B.HD_C128}[precision]
        mode = arnoldi if arnoldi != "auto" else ("ds" if prec != B.HD_C128 else "fp64")
        t = B.hd_submit(self.srv, N, N, npml, 1.0 / N, omega, c.ctypes.data, f.ctypes.data, f.shape[0],
                        prec | _storage_flag(prec, symmetric, tcore, smoothing),
                        restart, max_iters, rtol, x.ctypes.data, nbx, nby, overlap, cut_x, cut_y,
                        arnoldi={"fp64": B.HD_ARNOLDI_FP64, "ds": B.HD_ARNOLDI_DS}[mode],
                        reorth={"always": 0, "selective": 1}[reorth])
        self._keep[t] = (c, f, x)
        return t

    def poll(self, ticket, timeout_s=None):
        """(x, stats, info) once done, None while pending (timeout_s None waits forever)."""
        c, f, x = self._keep[ticket]
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        rc, stats, info = B.hd_poll(self.srv, ticket, f.shape[0], us)
        if rc == B.HD_PENDING:
            return None
        del self._keep[ticket]
        return x, stats, info

    def info(self):
        return B.hd_server_info(self.srv)

    def close(self):
        if getattr(self, "srv", None):
            B.hd_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
