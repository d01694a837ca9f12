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


class HelmholtzDDM:
    """One medium on one GPU: PML tables, per-box factors and the solvers.

    Grid: N x N interior cells (h = 1/N) plus npml PML cells per side; vectors
    are complex128 tensors of shape [..., n, n] with n = N + 2 npml (x fastest).
    """

    def __init__(self, N: int, npml: int, omega: float, c, nbx: int, nby: int, overlap: int,
                 precision: str = "c64", cut_x: Optional[Sequence[int]] = None, cut_y: Optional[Sequence[int]] = None,
                 own_global_pml: bool = True, sigma0_over_omega: float = 20.0, pml_power: int = 2,
                 device: str = "cuda", stream: Optional[torch.cuda.Stream] = None, factor: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("HelmholtzDDM needs a CUDA device: there is no CPU path")
        self.N, self.npml, self.n = N, npml, N + 2 * npml
        self.device = torch.device(device)
        self.stream = stream
        self.prec = {"c64": B.HD_C64, "c128": B.HD_C128}[precision]
        c_t = torch.as_tensor(np.asarray(c, dtype=np.float64) if not torch.is_tensor(c) else c,
                              dtype=torch.float64).to(self.device).contiguous()
        assert c_t.shape == (self.n, self.n), f"velocity must be {(self.n, self.n)}"
        self.ctx = B.hd_setup_medium(N, N, npml, 1.0 / N, omega, c_t.data_ptr(), self.prec, self._st(),
                                     nbx, nby, overlap, cut_x, cut_y, int(own_global_pml), sigma0_over_omega,
                                     pml_power)
        fb, _, sb = B.hd_query_workspace(self.ctx, 1, 1)
        self.factor_bytes, self.scratch_bytes = fb, sb
        self.factor_buf = torch.empty(max(fb, 16), dtype=torch.uint8, device=self.device)
        self.scratch = torch.empty(max(sb, 16), dtype=torch.uint8, device=self.device)
        self._krylov = {}
        self.factored = False
        if factor:
            self.factor()

    def _st(self) -> int:
        return _stream_ptr(self.stream)

    def factor(self):
        B.hd_factor_subdomains(self.ctx, self.factor_buf.data_ptr(), self.factor_bytes, self.scratch.data_ptr(),
                               self.scratch_bytes, self._st())
        self.factored = True

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

    def krylov_workspace(self, restart: int):
        if restart not in self._krylov:
            _, kb, _ = B.hd_query_workspace(self.ctx, 1, restart)
            self._krylov.clear()
            self._krylov[restart] = torch.empty(kb, dtype=torch.uint8, device=self.device)
        return self._krylov[restart]

    def solve(self, b, restart: int = 50, rtol: float = 1e-8, max_iters: int = 1000, x0=None, out=None,
              arnoldi: str = "auto"):
        """FGMRES solve of A x = b.  ``arnoldi``: "fp64", "ds" (double-single
        Gram-Schmidt on the FP32 pipes) or "auto" (ds with c64 factors, fp64 with c128)."""
        b, nrhs = self._vec(b)
        if out is not None:
            x = out
        elif x0 is not None:
            x = self._vec(x0)[0].clone()
        else:
            x = torch.empty_like(b)
        kws = self.krylov_workspace(restart)
        rc, stats = B.hd_gmres_solve(self.ctx, b.data_ptr(), x.data_ptr(), nrhs, restart, max_iters, rtol,
                                     kws.data_ptr(), kws.numel(), self.scratch.data_ptr(), self.scratch_bytes,
                                     self._st(), use_x0=int(x0 is not None), arnoldi=self._arnoldi(arnoldi))
        return x, stats

    def _arnoldi(self, mode: str) -> int:
        if mode == "auto":
            mode = "ds" if self.prec == B.HD_C64 else "fp64"
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
               device: str = "cuda", arnoldi: str = "auto"):
    """End-to-end solve from host arrays: velocity c [n][n] (float64) and source
    samples f [nrhs][n][n] (complex128), preferably in pinned memory.  Copies in,
    sets up the medium, factorises, forms b = J h^2 f, runs FGMRES and copies the
    solution back.  Returns (x on the host, stats, bytes copied in, bytes out)."""
    dev = torch.device(device)
    c_d = torch.as_tensor(c_host).to(dev, non_blocking=True)
    f_d = torch.as_tensor(f_host).to(dev, non_blocking=True)
    s = HelmholtzDDM(N, npml, omega, c_d, nbx, nby, overlap, precision=precision, cut_x=cut_x, cut_y=cut_y,
                     device=device)
    b = s.rhs(f_d)
    x, stats = s.solve(b, restart=restart, rtol=rtol, max_iters=max_iters, arnoldi=arnoldi)
    x_h = x.to("cpu")
    s.close()
    h2d = c_d.numel() * c_d.element_size() + f_d.numel() * f_d.element_size()
    return x_h, stats, h2d, x_h.numel() * x_h.element_size()
