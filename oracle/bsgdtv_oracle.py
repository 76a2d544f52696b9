"""FP64 reference implementation of BSGD-TV, block by block (test infrastructure).

Paper: Y. Gao, T. Blumensath, "BSGD-TV: A parallel algorithm solving total
variation constrained image reconstruction problems", arXiv 1812.01307.
TV prox solver: A. Beck, M. Teboulle, "Fast gradient-based algorithms for
constrained total variation image denoising and deblurring problems",
IEEE TIP 18(11), 2009 (the method the paper adopts for the TV proximal step of
Algorithm 1).

Readings where the paper is silent or ambiguous (each one is also recorded in
the design notes):
  R1  the TV proximal step is taken as printed: prox weight 2*mu*lambda, so FGP runs with
      tau = mu*lambda, and the algorithm's fixed point minimises
      ||y-Ax||^2 + lambda*TV(x)  (Eq. 1 writes 2*lambda*TV; see F_alg below).
  R2  TV is Beck-Teboulle's isotropic TV_I: forward differences with Neumann
      (zero-difference) border, the discretisation FGP is defined on.
  R3  initialisation: x^0 = 0 and r before the first epoch is y - A x^0 = y,
      so the first epoch's gradient uses r = y.
  R4  the random order of the block pairs is drawn, but the residual and gradient sums
      run in ascending j / i, so the result does not depend on the draw.
  R5  FGP: cold start every epoch, exactly K iterations, P_C = identity.
  R6  lambda = 0 (or K = 0) makes the TV proximal step the identity.
  R7  uneven blocks follow numpy.array_split: the first (L mod M) blocks get
      one extra unit.
  R8  u_max by power iteration on A^T A from the all-ones vector.
  R10 stochastic variant (Sec. 3: only a fraction alpha of the column blocks
      and gamma of the row blocks take part in an iteration): the drawn
      subsets S_I, S_J are inputs; only the pairs in S_I x S_J form their
      block products (from the current x and stored r); r_{I_i}, i in S_I,
      becomes y_{I_i} - sum_j z^j_{I_i} with z^j of unselected j the value
      last computed (0 before the first, consistent with x^0 = 0); x_{J_j},
      j in S_J, gains mu * sum_{i in S_I} g-hat^i_{J_j} (no rescaling); the rest
      of x and r is unchanged; the TV prox then acts on the whole image.
      With every block selected this is exactly Algorithm 1's epoch.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "split_bounds", "partition", "split_blocks", "block_products", "reduce_residual",
    "reduce_gradient", "epoch", "run", "L_op", "Lt_op", "proj_iso", "fgp",
    "tv_iso", "objective", "power_iteration", "descent_condition",
    "to_scipy", "run_subsets",
]


def to_scipy(A) -> sp.csr_matrix:
    """Accepts a scipy matrix or any object with row_ptr/cols/vals (host CSR)."""
    if sp.issparse(A):
        return sp.csr_matrix(A, dtype=np.float64)
    return sp.csr_matrix((np.asarray(A.vals, dtype=np.float64), A.cols, A.row_ptr),
                         shape=(A.rows, A.cols_n))


# ---------------------------------------------------------------- Sec. 2.1 blocks
def split_bounds(units: int, parts: int) -> np.ndarray:
    """Boundaries [parts+1] of `units` split into `parts` contiguous groups (R7)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    q, rem = divmod(int(units), int(parts))
    b = [0]
    for k in range(parts):
        b.append(b[-1] + q + (1 if k < rem else 0))
    return np.asarray(b, dtype=np.int64)


def partition(rows: int, cols: int, M: int, N: int, row_unit: int = 1, col_unit: int = 1):
    """Row blocks I_1..I_M and column blocks J_1..J_N of A (Sec. 2.1).

    Rows are grouped in whole units of `row_unit` (one projection angle = n_bins
    rays) and columns in whole units of `col_unit` (one image row = n pixels),
    so that I_i are contiguous angle groups and J_j contiguous image-row bands.
    """
    if rows % row_unit or cols % col_unit:
        raise ValueError("units must divide the matrix size")
    rb = split_bounds(rows // row_unit, M) * row_unit
    cb = split_bounds(cols // col_unit, N) * col_unit
    return rb, cb


def split_blocks(A, rb, cb):
    """blocks[i][j] = A_{I_i}^{J_j} with block-local column indices (Sec. 2.1)."""
    A = to_scipy(A)
    blocks = []
    for i in range(len(rb) - 1):
        rowblk = A[rb[i]:rb[i + 1], :]
        blocks.append([sp.csr_matrix(rowblk[:, cb[j]:cb[j + 1]]) for j in range(len(cb) - 1)])
    return blocks


def block_products(blocks, rb, cb, x, r, order=None):
    """The block products of Algorithm 1 for every pair (i, j).

    Returns (z, gh) with z[i][j] = A_{I_i}^{J_j} x_{J_j}  (z^j_{I_i}) and
    gh[i][j] = 2 (A_{I_i}^{J_j})^T r_{I_i}  (g-hat^i_{J_j}); `r` is the
    residual from the previous epoch.  `order` is the sequence of pairs drawn;
    every pair reads the same x and r, so the order does not change the values.
    """
    M, N = len(rb) - 1, len(cb) - 1
    if order is None:
        order = [(i, j) for i in range(M) for j in range(N)]
    z = [[None] * N for _ in range(M)]
    gh = [[None] * N for _ in range(M)]
    for i, j in order:
        Aij = blocks[i][j]
        r_I = r[rb[i]:rb[i + 1]]
        x_J = x[cb[j]:cb[j + 1]]
        gh[i][j] = 2.0 * (Aij.T @ r_I)
        z[i][j] = Aij @ x_J
    return z, gh


def reduce_residual(y, z, rb):
    """Residual update of Algorithm 1: r = y - sum_j z^j (ascending j, R4)."""
    r = np.array(y, dtype=np.float64, copy=True)
    for i in range(len(rb) - 1):
        acc = np.zeros(rb[i + 1] - rb[i])
        for zij in z[i]:
            acc = acc + zij
        r[rb[i]:rb[i + 1]] -= acc
    return r


def reduce_gradient(gh, cb, c):
    """Gradient sum of Algorithm 1: g = sum_i g-hat^i (ascending i, R4)."""
    g = np.zeros(c)
    M, N = len(gh), len(cb) - 1
    for j in range(N):
        acc = np.zeros(cb[j + 1] - cb[j])
        for i in range(M):
            acc = acc + gh[i][j]
        g[cb[j]:cb[j + 1]] = acc
    return g


# ------------------------------------------------------------ Beck-Teboulle FGP
def L_op(p, q):
    """L(p,q)_{s,t} = p_{s,t} + q_{s,t} - p_{s-1,t} - q_{s,t-1}, with p, q zero
    outside p:(m-1)xn, q:mx(n-1)  (Beck-Teboulle 2009, Sec. 4)."""
    m, n = p.shape[0] + 1, q.shape[1] + 1
    out = np.zeros((m, n))
    out[:m - 1, :] += p
    out[1:, :] -= p
    out[:, :n - 1] += q
    out[:, 1:] -= q
    return out


def Lt_op(x):
    """Adjoint of L: P_{s,t} = x_{s,t} - x_{s+1,t}, Q_{s,t} = x_{s,t} - x_{s,t+1}."""
    return x[:-1, :] - x[1:, :], x[:, :-1] - x[:, 1:]


def proj_iso(p, q):
    """Projection onto the isotropic dual set: (p,q)/max(1, sqrt(p^2+q^2)) where
    both exist (s<m-1, t<n-1); the border entries p_{s,n-1} and q_{m-1,t}
    are clipped alone by max(1, |.|)."""
    p = p.copy()
    q = q.copy()
    m1, n1 = q.shape[0] - 1, p.shape[1] - 1
    if m1 > 0 and n1 > 0:
        pp = p[:m1, :n1]
        qq = q[:m1, :n1]
        den = np.maximum(1.0, np.sqrt(pp * pp + qq * qq))
        p[:m1, :n1] = pp / den
        q[:m1, :n1] = qq / den
    if p.shape[0] > 0:
        p[:, n1] = p[:, n1] / np.maximum(1.0, np.abs(p[:, n1]))
    if q.shape[1] > 0:
        q[m1, :] = q[m1, :] / np.maximum(1.0, np.abs(q[m1, :]))
    return p, q


def fgp(b, tau: float, K: int, return_dual: bool = False):
    """FGP(b, tau, K) of Beck-Teboulle 2009 for argmin_x ||x-b||^2 + 2 tau TV_I(x),
    unconstrained (P_C = identity, R5).  The TV proximal step of Algorithm 1 calls it with
    tau = mu*lambda (R1)."""
    b = np.asarray(b, dtype=np.float64)
    m, n = b.shape
    p_prev = np.zeros((m - 1, n))
    q_prev = np.zeros((m, n - 1))
    r, s = p_prev.copy(), q_prev.copy()
    t = 1.0
    if tau <= 0.0 or K <= 0:
        out = b.copy()
        return (out, p_prev, q_prev) if return_dual else out
    for _ in range(K):
        u = b - tau * L_op(r, s)
        P, Q = Lt_op(u)
        p, q = proj_iso(r + P / (8.0 * tau), s + Q / (8.0 * tau))
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        beta = (t - 1.0) / t_next
        r = p + beta * (p - p_prev)
        s = q + beta * (q - q_prev)
        p_prev, q_prev, t = p, q, t_next
    out = b - tau * L_op(p_prev, q_prev)
    return (out, p_prev, q_prev) if return_dual else out


def tv_iso(x) -> float:
    """TV_I(x): isotropic, forward differences, Neumann border (R2)."""
    x = np.asarray(x, dtype=np.float64)
    dv = np.zeros_like(x)
    dh = np.zeros_like(x)
    dv[:-1, :] = x[:-1, :] - x[1:, :]
    dh[:, :-1] = x[:, :-1] - x[:, 1:]
    return float(np.sum(np.sqrt(dv * dv + dh * dh)))


# --------------------------------------------------------------- Algorithm 1
def epoch(blocks, rb, cb, y, x, r_prev, mu, lam, fgp_iters, img_shape, rng=None):
    """One epoch of Algorithm 1.  Returns (x_new, r_new, x_hat).

    x: current iterate x^k (flat); r_prev: residual r^{k-1} from the previous
    epoch (its residual update, or y before the first one, R3).
    """
    M, N = len(rb) - 1, len(cb) - 1
    pairs = [(i, j) for i in range(M) for j in range(N)]
    if rng is not None:
        pairs = [pairs[k] for k in rng.permutation(len(pairs))]
    z, gh = block_products(blocks, rb, cb, x, r_prev, pairs)        # block products
    r_new = reduce_residual(y, z, rb)                                 # r = y - sum_j z^j
    g = reduce_gradient(gh, cb, x.shape[0])                           # g = sum_i g-hat^i
    x_hat = x + mu * g                                                # gradient step
    if lam > 0.0 and fgp_iters > 0:                                   # TV prox (R1, R6)
        x_new = fgp(x_hat.reshape(img_shape), mu * lam, fgp_iters).ravel()
    else:
        x_new = x_hat.copy()
    return x_new, r_new, x_hat


def run(A, y, img_shape, M, N, lam, mu, epochs, fgp_iters, row_unit=1, col_unit=1,
        x0=None, r0=None, seed=0, callback=None, row_bounds=None, col_bounds=None):
    """Algorithm 1 for `epochs` epochs from x^0 (default 0) and r^{-1} (default
    y - A x^0, R3).  Explicit block bounds override the unit split.  Returns
    (x, r) after the last epoch."""
    A = to_scipy(A)
    rows, cols = A.shape
    rb, cb = partition(rows, cols, M, N, row_unit, col_unit)
    if row_bounds is not None:
        rb = np.asarray(row_bounds, dtype=np.int64)
    if col_bounds is not None:
        cb = np.asarray(col_bounds, dtype=np.int64)
    blocks = split_blocks(A, rb, cb)
    y = np.asarray(y, dtype=np.float64)
    x = np.zeros(cols) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    r = (y - A @ x) if r0 is None else np.asarray(r0, dtype=np.float64).copy()
    rng = np.random.default_rng(seed)
    for k in range(epochs):
        x_new, r, _ = epoch(blocks, rb, cb, y, x, r, mu, lam, fgp_iters, img_shape, rng)
        if callback is not None:
            callback(k, x, x_new, r)
        x = x_new
    return x, r


def run_subsets(A, y, img_shape, M, N, lam, mu, row_sel, col_sel, fgp_iters, row_unit=1,
                col_unit=1):
    """The stochastic variant of Sec. 3 under reading R10, one iteration per
    row of the boolean masks row_sel [iters, M] and col_sel [iters, N], from
    x^0 = 0 and r = y.  Returns (x, r)."""
    A = to_scipy(A)
    rows, cols = A.shape
    rb, cb = partition(rows, cols, M, N, row_unit, col_unit)
    blocks = split_blocks(A, rb, cb)
    y = np.asarray(y, dtype=np.float64)
    x = np.zeros(cols)
    r = y.copy()
    z = [[np.zeros(rb[i + 1] - rb[i]) for j in range(N)] for i in range(M)]   # last block products
    for sel_i, sel_j in zip(np.asarray(row_sel, dtype=bool), np.asarray(col_sel, dtype=bool)):
        S_I = [i for i in range(M) if sel_i[i]]
        S_J = [j for j in range(N) if sel_j[j]]
        gh = {}
        for i in S_I:                                   # block products of the drawn pairs
            for j in S_J:
                gh[i, j] = 2.0 * (blocks[i][j].T @ r[rb[i]:rb[i + 1]])
                z[i][j] = blocks[i][j] @ x[cb[j]:cb[j + 1]]
        r = r.copy()
        for i in S_I:                                   # residual of the drawn row blocks
            acc = np.zeros(rb[i + 1] - rb[i])
            for j in range(N):
                acc = acc + z[i][j]
            r[rb[i]:rb[i + 1]] = y[rb[i]:rb[i + 1]] - acc
        x_hat = x.copy()
        for j in S_J:                                   # gradient step on the drawn column blocks
            acc = np.zeros(cb[j + 1] - cb[j])
            for i in S_I:
                acc = acc + gh[i, j]
            x_hat[cb[j]:cb[j + 1]] = x[cb[j]:cb[j + 1]] + mu * acc
        if lam > 0.0 and fgp_iters > 0:                 # TV prox on the whole image
            x = fgp(x_hat.reshape(img_shape), mu * lam, fgp_iters).ravel()
        else:
            x = x_hat
    return x, r


# ------------------------------------------------------- step size (Thm. 1)
def power_iteration(A, max_iters: int = 5000, rel_tol: float = 1e-12, v0=None):
    """u_max = largest eigenvalue of A^T A (Theorem 1), by power iteration from
    the all-ones vector (R8).  Returns (u_max, iterations)."""
    A = to_scipy(A)
    v = np.ones(A.shape[1]) if v0 is None else np.asarray(v0, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    u = 0.0
    for it in range(1, max_iters + 1):
        w = A.T @ (A @ v)
        u_new = float(v @ w)          # Rayleigh quotient, ||v|| = 1
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0, it
        v = w / nw
        if it > 1 and abs(u_new - u) <= rel_tol * abs(u_new):
            return u_new, it
        u = u_new
    return u, max_iters


# --------------------------------------------------------- monitoring, Eq. 1
def objective(A, y, x, lam, img_shape):
    """F_alg(x) = ||y - A x||^2 + lambda TV_I(x): the function Algorithm 1 with
    TV proximal step as printed minimises (R1).  Returns (F, ||y-Ax||^2, TV_I(x))."""
    A = to_scipy(A)
    res = np.asarray(y, dtype=np.float64) - A @ np.asarray(x, dtype=np.float64)
    f = float(res @ res)
    tv = tv_iso(np.asarray(x).reshape(img_shape))
    return f + lam * tv, f, tv


def descent_condition(A, y, x_next, x_cur, x_prev, mu):
    """Theorem 2's step condition f(x^{k+1}) < f(x^k) + (x^{k+1}-x^k)^T grad f(x^{k-1})
    + ||x^{k+1}-x^k||^2/(2 mu), with f(x) = ||y - A x||^2.  Returns (lhs, rhs)."""
    A = to_scipy(A)
    y = np.asarray(y, dtype=np.float64)

    def f(v):
        rr = y - A @ v
        return float(rr @ rr)

    grad_prev = -2.0 * (A.T @ (y - A @ x_prev))
    d = x_next - x_cur
    return f(x_next), f(x_cur) + float(d @ grad_prev) + float(d @ d) / (2.0 * mu)

