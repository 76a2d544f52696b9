"""Seeded synthetic inputs for BSGD-TV: ellipse phantoms, the parallel-beam
projection matrix A (exact Siddon intersection lengths, CSR) and noisy
projections y.

This module is shared by the CPU oracle and by the GPU library's callers
(tests, bench).  It holds no arithmetic of the reconstruction method itself
(Algorithm 1 of the paper takes A and y as given, Sec. 1 Eq. 1); it only makes
the problem instances.  The paper's own data (a fan-beam Shepp-Logan scan,
Sec. 3 Fig. 1) is not available; seeded ellipse phantoms on a parallel-beam
geometry stand in for it.

Conventions
-----------
* image x is n x n, row-major, index ``s*n + t`` (row s from the top);
  pixel (s,t) is centred at ``(t-(n-1)/2, (n-1)/2-s)`` with unit size.
* projection y is angle-major, index ``k*n_bins + d``; angle ``k*pi/n_angles``,
  detector offset ``d-(n_bins-1)/2``.
* phantom: ``n_ellipses`` ellipses drawn with ``numpy.random.default_rng(seed)``,
  per ellipse in the order (cx, cy, a, b, phi, I): centres U(-24,24)*scale,
  semi-axes U(3,20)*scale, rotation U(0,pi), additive intensity U(0,1);
  ``scale = n/64``.  A pixel belongs to an ellipse when its centre satisfies
  ``(x'/a)^2 + (y'/b)^2 <= 1`` in the ellipse frame.
* noise: ``y = A x_true + N(0, sigma^2)``, ``sigma = frac * mean|A x_true|``,
  drawn with ``default_rng(seed + 1)``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon.c")
_LIB = os.path.join(_HERE, "_siddon.so")
_lock = threading.Lock()
_lib = None


def build_siddon(force: bool = False) -> str:
    """Compiles the host Siddon generator (plain C, OpenMP) in place."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_siddon()
            lib = ctypes.CDLL(_LIB)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            f64p = ctypes.POINTER(ctypes.c_double)
            lib.siddon_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p]
            lib.siddon_count.restype = None
            lib.siddon_fill.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i32p, f64p]
            lib.siddon_fill.restype = None
            lib.siddon_ray.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, i32p, f64p]
            lib.siddon_ray.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclasses.dataclass(frozen=True)
class CSR:
    """Host CSR matrix: ``row_ptr`` int64 [rows+1], ``cols`` int32 [nnz], ``vals`` float64 [nnz]."""
    rows: int
    cols_n: int
    row_ptr: np.ndarray
    cols: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.cols, self.row_ptr), shape=(self.rows, self.cols_n))


def siddon_ray(n: int, theta: float, u: float):
    """Columns and lengths of one ray (for tests)."""
    lib = _load()
    cols = np.zeros(2 * n + 2, dtype=np.int32)
    vals = np.zeros(2 * n + 2, dtype=np.float64)
    cnt = lib.siddon_ray(int(n), float(theta), float(u), _ptr(cols, ctypes.c_int32), _ptr(vals, ctypes.c_double))
    return cols[:cnt].copy(), vals[:cnt].copy()


def parallel_beam_csr(n: int, n_angles: int, n_bins: int) -> CSR:
    """Projection matrix A (rows = rays, cols = pixels) of a parallel-beam scan."""
    lib = _load()
    rows = n_angles * n_bins
    row_nnz = np.zeros(rows, dtype=np.int64)
    lib.siddon_count(int(n), int(n_angles), int(n_bins), _ptr(row_nnz, ctypes.c_int64))
    row_ptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(row_nnz, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    cols = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    lib.siddon_fill(int(n), int(n_angles), int(n_bins), _ptr(row_ptr, ctypes.c_int64),
                    _ptr(cols, ctypes.c_int32), _ptr(vals, ctypes.c_double))
    return CSR(rows, n * n, row_ptr, cols, vals)


def parallel_beam_nnz(n: int, n_angles: int, n_bins: int) -> int:
    """Nonzeros of the parallel-beam A, counted without storing it."""
    lib = _load()
    row_nnz = np.zeros(n_angles * n_bins, dtype=np.int64)
    lib.siddon_count(int(n), int(n_angles), int(n_bins), _ptr(row_nnz, ctypes.c_int64))
    return int(row_nnz.sum())


def ellipse_params(n_ellipses: int, seed: int, scale: float) -> np.ndarray:
    """[n_ellipses, 6] array of (cx, cy, a, b, phi, intensity)."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_ellipses, 6), dtype=np.float64)
    for e in range(n_ellipses):
        out[e, 0] = rng.uniform(-24.0, 24.0) * scale
        out[e, 1] = rng.uniform(-24.0, 24.0) * scale
        out[e, 2] = rng.uniform(3.0, 20.0) * scale
        out[e, 3] = rng.uniform(3.0, 20.0) * scale
        out[e, 4] = rng.uniform(0.0, np.pi)
        out[e, 5] = rng.uniform(0.0, 1.0)
    return out


def phantom(n: int, n_ellipses: int, seed: int, scale: float | None = None) -> np.ndarray:
    """Sum-of-ellipses phantom, float64 [n, n].  A pixel gets an ellipse's
    intensity when its centre satisfies (x'/a)^2 + (y'/b)^2 <= 1; the test runs
    only over a bounding box of the ellipse widened by 2 pixels (pixels
    outside it fail the test by a wide margin)."""
    if scale is None:
        scale = n / 64.0
    params = ellipse_params(n_ellipses, seed, scale)
    t = np.arange(n, dtype=np.float64) - 0.5 * (n - 1)
    img = np.zeros((n, n), dtype=np.float64)
    for cx, cy, a, b, phi, inten in params:
        hx = np.sqrt((a * np.cos(phi)) ** 2 + (b * np.sin(phi)) ** 2) + 2.0
        hy = np.sqrt((a * np.sin(phi)) ** 2 + (b * np.cos(phi)) ** 2) + 2.0
        # columns with |x - cx| <= hx, rows with |y - cy| <= hy (y = -t of the row)
        c0 = max(0, int(np.floor(cx - hx + 0.5 * (n - 1))))
        c1 = min(n, int(np.ceil(cx + hx + 0.5 * (n - 1))) + 1)
        r0 = max(0, int(np.floor(-cy - hy + 0.5 * (n - 1))))
        r1 = min(n, int(np.ceil(-cy + hy + 0.5 * (n - 1))) + 1)
        if c0 >= c1 or r0 >= r1:
            continue
        X = t[None, c0:c1]
        Y = (-t)[r0:r1, None]
        dx, dy = X - cx, Y - cy
        xr = dx * np.cos(phi) + dy * np.sin(phi)
        yr = -dx * np.sin(phi) + dy * np.cos(phi)
        img[r0:r1, c0:c1][(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += inten
    return img


def csr_matvec(A: CSR, x: np.ndarray) -> np.ndarray:
    """Plain CSR product used only to synthesise clean projections."""
    return A.to_scipy() @ np.asarray(x, dtype=np.float64).ravel()


def noisy_projections(A: CSR, x_true: np.ndarray, seed: int, frac: float = 0.01) -> np.ndarray:
    y_clean = csr_matvec(A, x_true)
    sigma = frac * float(np.mean(np.abs(y_clean)))
    rng = np.random.default_rng(seed + 1)
    return y_clean + sigma * rng.standard_normal(y_clean.shape[0])


def slice_stack(A: CSR, n: int, n_ellipses: int, slices: int, seed: int = 0,
                frac: float = 0.01):
    """A stack of independent slices through one geometry A (as the slices of
    a parallel-beam volume): slice b is the phantom of seed `seed + b` and its
    projections with 1% Gaussian noise of seed `seed + b`.  Returns
    (X_true [slices, n*n], Y [slices, rows]), float64."""
    X = np.stack([phantom(n, n_ellipses, seed + b).ravel() for b in range(slices)])
    Yc = np.ascontiguousarray(np.asarray(A.to_scipy() @ X.T).T)   # clean projections, [slices, rows]
    Y = np.empty(Yc.shape)
    for b in range(slices):
        sigma = frac * float(np.mean(np.abs(Yc[b])))
        Y[b] = Yc[b] + sigma * np.random.default_rng(seed + b + 1).standard_normal(Yc.shape[1])
    return X, Y


def subset_draws(M: int, N: int, alpha: float, gamma: float, iters: int, seed: int = 0):
    """Random block subsets for the stochastic variant (the draws are inputs of
    the method, not part of it): per iteration max(1, round(gamma*M)) of the M
    row blocks and max(1, round(alpha*N)) of the N column blocks, uniformly
    without replacement, numpy default_rng(seed).  Returns boolean masks
    (row_sel [iters, M], col_sel [iters, N])."""
    rng = np.random.default_rng(seed)
    kM = min(M, max(1, int(round(gamma * M))))
    kN = min(N, max(1, int(round(alpha * N))))
    row_sel = np.zeros((iters, M), dtype=bool)
    col_sel = np.zeros((iters, N), dtype=bool)
    for k in range(iters):
        row_sel[k, rng.choice(M, kM, replace=False)] = True
        col_sel[k, rng.choice(N, kN, replace=False)] = True
    return row_sel, col_sel


@dataclasses.dataclass(frozen=True)
class Workload:
    """One reconstruction problem: geometry, phantom recipe and solver settings."""
    name: str
    n: int
    n_ellipses: int
    n_angles: int
    n_bins: int
    M: int
    N: int
    lam: float
    epochs: int
    fgp_iters: int
    seed: int = 0
    noise: float = 0.01

    @property
    def rows(self) -> int:
        return self.n_angles * self.n_bins


WORKLOADS = {
    # 64x64, 10 ellipses, 60 angles x 91 bins, 4x4 blocks, lambda 0.05, 50 epochs, 20 FGP iterations
    "ellipse64": Workload("ellipse64", 64, 10, 60, 91, 4, 4, 0.05, 50, 20),
    # 512x512, 30 ellipses, 360 angles x 727 bins, 8x8 blocks, lambda 0.02, 200 epochs, 50 FGP iterations
    "ellipse512": Workload("ellipse512", 512, 30, 360, 727, 8, 8, 0.02, 200, 50),
}


@dataclasses.dataclass
class Problem:
    wl: Workload
    A: CSR
    x_true: np.ndarray
    y: np.ndarray


_cache: dict = {}


def make_problem(wl: Workload | str, cache: bool = True) -> Problem:
    """Builds (A, x_true, y) for a workload; cached per process."""
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    key = (wl.n, wl.n_ellipses, wl.n_angles, wl.n_bins, wl.seed, wl.noise)
    if cache and key in _cache:
        A, x_true, y = _cache[key]
        return Problem(wl, A, x_true, y)
    A = parallel_beam_csr(wl.n, wl.n_angles, wl.n_bins)
    x_true = phantom(wl.n, wl.n_ellipses, wl.seed)
    y = noisy_projections(A, x_true, wl.seed, wl.noise)
    if cache:
        _cache[key] = (A, x_true, y)
    return Problem(wl, A, x_true, y)
