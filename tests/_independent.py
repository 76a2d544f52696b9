"""Independent FP64 solvers used to pin the oracle.

They share nothing with ``oracle/``: a different algorithm (Chambolle-Pock
primal-dual, "A first-order primal-dual algorithm for convex problems with
applications to imaging", J. Math. Imaging Vis. 40, 2011) on a gradient
operator written out here from the definition of isotropic TV with forward
differences and a zero-difference (Neumann) border.
"""
import numpy as np


def grad(x):
    """Forward differences (x_{s,t} - x_{s+1,t}, x_{s,t} - x_{s,t+1}), zero on the last row / column."""
    gv = np.zeros_like(x)
    gh = np.zeros_like(x)
    gv[:-1, :] = x[:-1, :] - x[1:, :]
    gh[:, :-1] = x[:, :-1] - x[:, 1:]
    return gv, gh


def grad_adj(gv, gh):
    """Adjoint of `grad`, derived by summation by parts."""
    m, n = gv.shape
    out = np.zeros((m, n))
    out[:-1, :] += gv[:-1, :]
    out[1:, :] -= gv[:-1, :]
    out[:, :-1] += gh[:, :-1]
    out[:, 1:] -= gh[:, :-1]
    return out


def tv_definition(x):
    """Isotropic TV with forward differences and Neumann border, straight from the sum."""
    m, n = x.shape
    total = 0.0
    for s in range(m):
        for t in range(n):
            dv = x[s, t] - x[s + 1, t] if s + 1 < m else 0.0
            dh = x[s, t] - x[s, t + 1] if t + 1 < n else 0.0
            total += np.hypot(dv, dh)
    return total


def _project_ball(gv, gh, radius):
    nrm = np.sqrt(gv * gv + gh * gh)
    scale = np.maximum(1.0, nrm / radius)
    return gv / scale, gh / scale


def cp_denoise(b, tau, iters=20000):
    """argmin_x ||x-b||^2 + 2 tau TV(x) by accelerated Chambolle-Pock (Alg. 2 of
    the 2011 paper, G(x) = ||x-b||^2 is 2-strongly convex)."""
    b = np.asarray(b, dtype=np.float64)
    x = b.copy()
    xbar = x.copy()
    yv = np.zeros_like(b)
    yh = np.zeros_like(b)
    L2 = 8.0
    t = 0.25
    sigma = 1.0 / (L2 * t)
    gamma = 2.0
    for _ in range(iters):
        gv, gh = grad(xbar)
        yv, yh = _project_ball(yv + sigma * gv, yh + sigma * gh, 2.0 * tau)
        x_old = x
        v = x - t * grad_adj(yv, yh)
        x = (v + 2.0 * t * b) / (1.0 + 2.0 * t)
        theta = 1.0 / np.sqrt(1.0 + 2.0 * gamma * t)
        t = theta * t
        sigma = sigma / theta
        xbar = x + theta * (x - x_old)
    return x


def cp_reconstruct(A_dense, y, lam, shape, iters=200000, tol=1e-13):
    """argmin_x ||y - A x||^2 + lam TV(x) by Chambolle-Pock with the data term in
    G (its prox is a dense solve).  A must have full column rank."""
    A = np.asarray(A_dense, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m, n = shape
    AtA = A.T @ A
    Aty = A.T @ y
    umin = float(np.linalg.eigvalsh(AtA).min())
    gamma = 2.0 * umin
    L2 = 8.0
    t = 1.0
    sigma = 1.0 / (L2 * t)
    x = np.linalg.solve(AtA, Aty).reshape(shape)
    xbar = x.copy()
    yv = np.zeros(shape)
    yh = np.zeros(shape)
    eye = np.eye(m * n)
    for k in range(iters):
        gv, gh = grad(xbar)
        yv, yh = _project_ball(yv + sigma * gv, yh + sigma * gh, lam)
        x_old = x
        v = (x - t * grad_adj(yv, yh)).ravel()
        x = np.linalg.solve(2.0 * AtA + eye / t, 2.0 * Aty + v / t).reshape(shape)
        theta = 1.0 / np.sqrt(1.0 + 2.0 * gamma * t)
        t = theta * t
        sigma = sigma / theta
        xbar = x + theta * (x - x_old)
        if k > 100 and np.max(np.abs(x - x_old)) < tol:
            break
    return x
