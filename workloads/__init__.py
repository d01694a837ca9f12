"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the method itself: it only lays out the
global grid (cell-centred, x fastest) and draws velocity models, sources and
request traces from ``numpy.random.Generator(PCG64(seed))``.  Both sides of
every parity test read the same arrays produced here.

Grid convention (the paper prints none, Sec. 3 only says "second order finite
difference"): the interior [0,1]^2 holds N x N cells of width h = 1/N; a layer
of ``npml`` cells is added on every side (Sec. 2, the truncated domain Omega), so
the global grid has n = N + 2*npml cells per axis and cell i sits at
x_i = (i - npml + 1/2) h.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Workload", "cell_centres", "velocity_homogeneous", "velocity_three_layer",
    "velocity_random_field", "gaussian_source", "point_source", "make_workload",
    "CONFIGS", "even_cuts", "random_complex", "poisson_trace",
]


def cell_centres(N: int, npml: int) -> np.ndarray:
    """Cell-centre coordinates of the global grid along one axis (length N+2*npml)."""
    n = N + 2 * npml
    return (np.arange(n, dtype=np.float64) - npml + 0.5) / N


def velocity_homogeneous(N: int, npml: int, c0: float = 1.0) -> np.ndarray:
    n = N + 2 * npml
    return np.full((n, n), c0, dtype=np.float64)


def velocity_three_layer(N: int, npml: int, speeds=(1.0, 1.5, 2.0), bounds=(0.33, 0.66)) -> np.ndarray:
    """Horizontal bands: speeds[0] for y < bounds[0], speeds[1] up to bounds[1], speeds[2] above."""
    n = N + 2 * npml
    y = cell_centres(N, npml)
    cy = np.where(y < bounds[0], speeds[0], np.where(y < bounds[1], speeds[1], speeds[2]))
    return np.repeat(cy[:, None], n, axis=1).astype(np.float64)


def velocity_random_field(N: int, npml: int, seed: int, ell: float = 0.05, amp: float = 0.3) -> np.ndarray:
    """c = 1 + amp * clip(g, -1, 1): g is seeded white noise on the global grid,
    convolved (periodic FFT) with exp(-r^2/(2 ell^2)) and renormalised to unit
    sample standard deviation."""
    n = N + 2 * npml
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((n, n))
    h = 1.0 / N
    d = np.minimum(np.arange(n), n - np.arange(n)) * h
    ker = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * ell * ell))
    g = np.fft.irfft2(np.fft.rfft2(noise) * np.fft.rfft2(ker), s=(n, n))
    g = (g - g.mean()) / g.std()
    return (1.0 + amp * np.clip(g, -1.0, 1.0)).astype(np.float64)


def gaussian_source(N: int, npml: int, xs: float, ys: float, width: float) -> np.ndarray:
    """Unit-mass Gaussian exp(-|x-xs|^2/(2 w^2)) / (2 pi w^2) sampled at cell centres."""
    x = cell_centres(N, npml)
    gx = np.exp(-((x - xs) ** 2) / (2.0 * width * width))
    gy = np.exp(-((x - ys) ** 2) / (2.0 * width * width))
    return (gy[:, None] * gx[None, :] / (2.0 * math.pi * width * width)).astype(np.complex128)


def point_source(N: int, npml: int, xs: float, ys: float) -> np.ndarray:
    """Discrete delta 1/(h_x h_y) at the cell nearest to (xs, ys) (Sec. 3 shot)."""
    n = N + 2 * npml
    f = np.zeros((n, n), dtype=np.complex128)
    i = int(np.floor(xs * N)) + npml
    j = int(np.floor(ys * N)) + npml
    f[j, i] = float(N) * float(N)
    return f


def even_cuts(N: int, npml: int, nb: int) -> List[int]:
    """Interior cut points npml = c_0 < ... < c_nb = npml + N, as even as integers allow."""
    return [npml + (i * N) // nb for i in range(nb + 1)]


def random_complex(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


@dataclass
class Workload:
    """One solve: grid, decomposition, medium, source(s) and Krylov settings."""
    name: str
    N: int
    npml: int
    omega: float
    nbx: int
    nby: int
    overlap: int
    c: np.ndarray                      # [n][n] velocity
    f: np.ndarray                      # [nrhs][n][n] complex source samples
    restart: int
    rtol: float
    cut_x: List[int] = field(default_factory=list)
    cut_y: List[int] = field(default_factory=list)
    sigma0_over_omega: float = 20.0
    pml_power: int = 2

    @property
    def n(self) -> int:
        return self.N + 2 * self.npml

    @property
    def h(self) -> float:
        return 1.0 / self.N

    @property
    def nrhs(self) -> int:
        return self.f.shape[0]


def _ppw_omega(N: int, c_min: float, ppw: float = 10.0) -> float:
    # angular frequency giving `ppw` cells per wavelength at the slowest speed
    return 2.0 * math.pi * c_min * N / ppw


def make_workload(name: str, N: Optional[int] = None, nb: Optional[int] = None, seed: Optional[int] = None,
                  nrhs: int = 1, npml: int = 16, overlap: int = 8, medium: Optional[str] = None,
                  restart: Optional[int] = None, rtol: Optional[float] = None,
                  cuts: Optional[Sequence[int]] = None) -> Workload:
    """Build one of the named synthetic workloads (sizes may be overridden for tests).

    tiny       128^2, c = 1, Gaussian (w = 2h) at (0.5, 0.5), 2x2 subdomains, GMRES(50) to 1e-8
    medium     1024^2, three horizontal layers c = 1 / 1.5 / 2, Gaussian at a seeded point, 8x8, GMRES(50) to 1e-8
    precision  4096^2, smooth random medium c = 1 + 0.3 g, Gaussian at a seeded point, 32x32, FGMRES(10) to 1e-6
    batching   1984^2 (owned widths 96 | 14 x 128 | 96), random medium, 64 Gaussian sources, FGMRES(5) to 1e-6
    """
    spec = {
        "tiny": dict(N=128, nb=2, medium="homogeneous", restart=50, rtol=1e-8, seed=0),
        "medium": dict(N=1024, nb=8, medium="three_layer", restart=50, rtol=1e-8, seed=1),
        "precision": dict(N=4096, nb=32, medium="random", restart=10, rtol=1e-6, seed=2),
        "batching": dict(N=1984, nb=16, medium="random", restart=5, rtol=1e-6, seed=3),
    }[name]
    N = N or spec["N"]
    nb = nb or spec["nb"]
    seed = spec["seed"] if seed is None else seed
    medium = medium or spec["medium"]
    restart = restart or spec["restart"]
    rtol = rtol or spec["rtol"]
    if medium == "homogeneous":
        c = velocity_homogeneous(N, npml)
    elif medium == "three_layer":
        c = velocity_three_layer(N, npml)
    elif medium == "random":
        c = velocity_random_field(N, npml, seed)
    else:
        raise ValueError(medium)
    omega = _ppw_omega(N, float(c.min()))
    h = 1.0 / N
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    srcs = []
    for r in range(nrhs):
        if name == "tiny" and nrhs == 1:
            xs, ys = 0.5, 0.5
        else:
            xs, ys = rng.uniform(0.05, 0.95, size=2)
        srcs.append(gaussian_source(N, npml, xs, ys, 2.0 * h))
    f = np.stack(srcs)
    if cuts is not None:
        cut = list(cuts)
    elif name == "batching" and N == 1984 and nb == 16:
        cut = [npml] + [npml + 96 + 128 * i for i in range(15)] + [npml + N]
    else:
        cut = even_cuts(N, npml, nb)
    return Workload(name=name, N=N, npml=npml, omega=omega, nbx=nb, nby=nb, overlap=overlap, c=c, f=f,
                    restart=restart, rtol=rtol, cut_x=list(cut), cut_y=list(cut))


CONFIGS = ("tiny", "medium", "precision", "batching")


def poisson_trace(seed: int, rate: float, duration_s: float, grids=(256, 512, 1024, 2048, 4096),
                  media=("homogeneous", "three_layer", "random"), max_rhs: int = 16):
    """Seeded Poisson arrival trace of solve requests (time, N, medium, nrhs, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            return out
        out.append(dict(t=t, N=int(rng.choice(grids)), medium=str(rng.choice(media)),
                        nrhs=int(rng.integers(1, max_rhs + 1)), seed=int(rng.integers(0, 2**31))))
