"""The oracle's banded direct solver: Python side of ``banded_lu.c``.

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``banded_lu.c`` is plain
C (textbook banded Gaussian elimination with partial pivoting); it is compiled
with the host C compiler into ``oracle/_build/`` on first use, or by
``__graft_entry__.build()``, and called through ctypes, which releases the GIL,
so several boxes factorise in parallel threads.
"""
from __future__ import annotations

import ctypes as ct
import os
import shutil
import subprocess
import tempfile
from typing import Optional

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "banded_lu.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libblu.so")

_lib = None


def build_banded(force: bool = False) -> str:
    """Compiles banded_lu.c into oracle/_build/libblu.so (skipped when up to date)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler found to build the oracle's banded LU")
    os.makedirs(BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD)
    os.close(fd)
    cmd = [cc, "-O2", "-std=c99", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        os.unlink(tmp)
        raise RuntimeError(f"building the oracle's banded LU failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)   # atomic: concurrent builders never load a half-written file
    return LIB


def _load():
    global _lib
    if _lib is None:
        L = ct.CDLL(build_banded())
        dp, ip = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)
        L.blu_factor.argtypes = [ct.c_int, ct.c_int, ct.c_int, dp, ip]
        L.blu_factor.restype = ct.c_int
        L.blu_solve.argtypes = [ct.c_int, ct.c_int, ct.c_int, dp, ip, dp]
        L.blu_solve.restype = None
        _lib = L
    return _lib


def box_order(nx: int, ny: int) -> Optional[np.ndarray]:
    """Unknown ordering of an nx x ny box (unknown (i, j) at j * nx + i) that makes the
    band the shorter side: None keeps x fastest (bandwidth nx); for ny < nx the
    returned permutation lists the old indices in y-fastest order (bandwidth ny)."""
    if nx <= ny:
        return None
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return (j * nx + i).T.ravel()   # new index i * ny + j -> old index j * nx + i


class BandLU:
    """LU factorisation with partial pivoting of a sparse complex matrix in band form.

    ``perm`` (optional) reorders the unknowns first: row and column q of the reordered
    matrix are row and column perm[q] of A.  The band widths kl, ku are those of the
    (reordered) nonzero pattern."""

    def __init__(self, A: sp.spmatrix, perm: Optional[np.ndarray] = None):
        A = sp.coo_matrix(A)
        n = A.shape[0]
        if A.shape != (n, n):
            raise ValueError("square matrix expected")
        self.n, self.perm = n, perm
        r, c = A.row.astype(np.int64), A.col.astype(np.int64)
        if perm is not None:
            inv = np.empty(n, dtype=np.int64)
            inv[perm] = np.arange(n)
            r, c = inv[r], inv[c]
        self.kl = int(max(0, (r - c).max(initial=0)))
        self.ku = int(max(0, (c - r).max(initial=0)))
        ld = 2 * self.kl + self.ku + 1
        ab = np.zeros((n, ld), dtype=np.complex128)
        np.add.at(ab, (r, c - r + self.kl), A.data.astype(np.complex128))
        self.ab = ab
        self.ipiv = np.zeros(n, dtype=np.intc)
        info = _load().blu_factor(n, self.kl, self.ku, self._dp(ab), self.ipiv.ctypes.data_as(ct.POINTER(ct.c_int)))
        if info:
            raise np.linalg.LinAlgError(f"zero pivot at step {info - 1}")

    @staticmethod
    def _dp(a: np.ndarray):
        return a.ctypes.data_as(ct.POINTER(ct.c_double))

    def solve(self, b: np.ndarray) -> np.ndarray:
        b = np.asarray(b, dtype=np.complex128).ravel()
        x = np.ascontiguousarray(b[self.perm] if self.perm is not None else b.copy())
        _load().blu_solve(self.n, self.kl, self.ku, self._dp(self.ab), self.ipiv.ctypes.data_as(ct.POINTER(ct.c_int)),
                          self._dp(x))
        if self.perm is None:
            return x
        out = np.empty_like(x)
        out[self.perm] = x
        return out
