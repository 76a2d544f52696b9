"""Pins for the oracle's Algorithm 1 against what the paper fixes:
Eq. 3 (stale-gradient recurrence), the fixed point of Sec. 2.2 (least
squares), Theorem 1 and the companion-matrix eigenvalues of its proof,
Theorem 2's descent condition, and an independent solver for lambda > 0."""
import numpy as np
import scipy.sparse as sp
import pytest

import oracle
from paper_1812_01307_gb300 import synth

from _independent import cp_reconstruct, tv_definition


def _problem(n=5, na=30, nb=9, seed=0):
    A = synth.parallel_beam_csr(n, na, nb)
    S = A.to_scipy()
    D = S.toarray()
    rng = np.random.default_rng(seed)
    x_true = rng.uniform(0.0, 1.0, n * n)
    y = D @ x_true + 0.05 * rng.standard_normal(D.shape[0])
    return A, D, y


def test_eq3_recurrence_lambda0():
    """lambda = 0: x^{k+1} = x^k + 2 mu A^T (y - A x^{k-1}) with x^{-1} = x^0 = 0 (Eq. 3)."""
    A, D, y = _problem(8, 12, 13)
    u = np.linalg.eigvalsh(D.T @ D).max()
    mu = 0.9 / (2 * u)
    xs = []
    oracle.run(A, y, (8, 8), 3, 4, 0.0, mu, 25, 0, row_unit=13, col_unit=8,
               callback=lambda k, x, xn, r: xs.append(xn.copy()))
    x_prev = np.zeros(64)
    x_cur = np.zeros(64)
    for k in range(25):
        x_next = x_cur + 2 * mu * D.T @ (y - D @ x_prev)
        assert np.allclose(xs[k], x_next, rtol=1e-12, atol=1e-12 * np.abs(x_next).max())
        x_prev, x_cur = x_cur, x_next


def _modes(D, mu):
    u, V = np.linalg.eigh(D.T @ D)
    disc = np.sqrt((1 - 8 * mu * u).astype(complex))
    return u, V, (1 + disc) / 2, (1 - disc) / 2   # v1, v2 of the proof of Theorem 1


def test_mode_trajectories_follow_companion_eigenvalues():
    """Each eigen-mode of A^T A obeys c_{k+1} = c_k - 2 mu u c_{k-1}, whose
    solution is a v1^k + b v2^k with v1,2 = (1 +- sqrt(1 - 8 mu u))/2."""
    A, D, y = _problem()
    u_all = np.linalg.eigvalsh(D.T @ D)
    mu = 0.9 / (2 * u_all.max())
    x_star = np.linalg.solve(D.T @ D, D.T @ y)
    u, V, v1, v2 = _modes(D, mu)
    assert np.any(8 * mu * u > 1) and np.any(8 * mu * u < 1)   # both regimes present
    traj = []
    oracle.run(A, y, (5, 5), 3, 2, 0.0, mu, 80, 0, row_unit=9, col_unit=5,
               callback=lambda k, x, xn, r: traj.append(V.T @ (xn - x_star)))
    c0 = V.T @ (0 - x_star)          # c^{-1} = c^0 (x^{-1} = x^0 = 0)
    # a + b = c0, a/v1 + b/v2 = c0  ->  solve per mode
    a = c0 * (1 / v2 - 1) / (1 / v2 - 1 / v1)
    b = c0 - a
    for k in range(80):
        pred = (a * v1 ** (k + 1) + b * v2 ** (k + 1)).real
        assert np.allclose(traj[k], pred, rtol=1e-8, atol=1e-9 * np.abs(c0).max())


def test_converges_to_least_squares_theorem1():
    A, D, y = _problem()
    u = np.linalg.eigvalsh(D.T @ D)
    mu = 0.9 / (2 * u.max())
    x_star = np.linalg.solve(D.T @ D, D.T @ y)      # fixed point, Sec. 2.2
    _, _, v1, v2 = _modes(D, mu)
    rate = np.max(np.maximum(np.abs(v1), np.abs(v2)))
    epochs = int(np.ceil(np.log(1e-9) / np.log(rate)))
    assert epochs < 20000
    x, _ = oracle.run(A, y, (5, 5), 3, 2, 0.0, mu, epochs, 0, row_unit=9, col_unit=5)
    assert np.linalg.norm(x - x_star) / np.linalg.norm(x_star) < 1e-8


def test_diverges_outside_theorem1_range():
    A, D, y = _problem()
    u = np.linalg.eigvalsh(D.T @ D)
    mu = 1.1 / (2 * u.max())
    x_star = np.linalg.solve(D.T @ D, D.T @ y)
    errs = []
    oracle.run(A, y, (5, 5), 1, 1, 0.0, mu, 400, 0,
               callback=lambda k, x, xn, r: errs.append(np.linalg.norm(xn - x_star)))
    # envelope growth over 200 epochs (the top mode oscillates: complex roots)
    growth = (max(errs[350:400]) / max(errs[150:200])) ** (1 / 200)
    assert errs[-1] > 1e3 * errs[0]
    assert abs(growth - np.sqrt(2 * mu * u.max())) < 2e-3   # |v|^2 = 2 mu u in the complex case


@pytest.mark.parametrize("n,na,nb", [(5, 30, 9), (8, 12, 13), (6, 7, 11)])
def test_power_iteration_matches_eigvalsh(n, na, nb):
    A = synth.parallel_beam_csr(n, na, nb)
    D = A.to_scipy().toarray()
    u_ref = np.linalg.eigvalsh(D.T @ D).max()
    u, it = oracle.power_iteration(A)
    assert abs(u - u_ref) <= 1e-10 * u_ref
    assert it < 5000


def test_objective_definition():
    A, D, y = _problem()
    rng = np.random.default_rng(1)
    x = rng.standard_normal(25)
    F, f, tv = oracle.objective(A, y, x, 0.3, (5, 5))
    assert np.isclose(f, np.sum((y - D @ x) ** 2), rtol=1e-13)
    assert np.isclose(tv, tv_definition(x.reshape(5, 5)), rtol=1e-13)
    assert np.isclose(F, f + 0.3 * tv, rtol=1e-13)


def test_theorem2_descent_condition_implies_decrease():
    """Where Theorem 2's condition holds, F_alg = f + lambda TV decreases
    (exact prox approximated by many FGP iterations)."""
    A, D, y = _problem()
    u = np.linalg.eigvalsh(D.T @ D).max()
    mu = 0.9 / (2 * u)
    lam = 0.4
    hist = {}

    def cb(k, x, xn, r):
        hist[k] = (x.copy(), xn.copy())

    oracle.run(A, y, (5, 5), 3, 2, lam, mu, 60, 400, row_unit=9, col_unit=5, callback=cb)
    held = 0
    for k in range(1, 60):
        x_prev, x_cur = hist[k - 1]
        _, x_next = hist[k]
        lhs, rhs = oracle.descent_condition(A, y, x_next, x_cur, x_prev, mu)
        if lhs < rhs:
            held += 1
            F_next = oracle.objective(A, y, x_next, lam, (5, 5))[0]
            F_cur = oracle.objective(A, y, x_cur, lam, (5, 5))[0]
            assert F_next <= F_cur + 1e-9 * abs(F_cur)
    assert held >= 10


def test_theorem2_condition_sides_closed_form():
    """The two sides of Theorem 2's condition, pinned without the oracle's own
    expression: f is the quadratic ||y - Ax||^2, so f(x_cur + d) expands
    exactly to f(x_cur) + 2 d^T A^T A x_cur - 2 d^T A^T y + ||A d||^2, and
    lhs - rhs = 2 d^T A^T A (x_cur - x_prev) + ||A d||^2 - ||d||^2 / (2 mu)
    (the gradient grad f(v) = -2 A^T (y - A v) taken at x_prev, not x_cur).
    A dropped term, a wrong sign or the gradient taken at x_cur moves the
    difference by one of these terms, which the random points make nonzero."""
    A, D, y = _problem(6, 14, 11, seed=3)
    rng = np.random.default_rng(7)
    mu = 1.7e-3
    for _ in range(5):
        x_prev, x_cur, x_next = (rng.standard_normal(36) for _ in range(3))
        lhs, rhs = oracle.descent_condition(A, y, x_next, x_cur, x_prev, mu)
        d = x_next - x_cur
        f_cur = float(np.sum((y - D @ x_cur) ** 2))
        f_next = f_cur + 2 * d @ (D.T @ (D @ x_cur)) - 2 * d @ (D.T @ y) + float(np.sum((D @ d) ** 2))
        diff = 2 * d @ (D.T @ (D @ (x_cur - x_prev))) + float(np.sum((D @ d) ** 2)) - d @ d / (2 * mu)
        scale = abs(f_cur) + abs(d @ d / (2 * mu)) + 1.0
        assert abs(lhs - f_next) <= 1e-11 * scale
        assert abs((lhs - rhs) - diff) <= 1e-11 * scale
    # at x_next = x_cur both sides equal f(x_cur): the strict condition fails
    lhs, rhs = oracle.descent_condition(A, y, x_cur, x_cur, x_prev, mu)
    assert lhs == rhs


def test_fixed_point_solves_tv_problem_independently():
    """lambda > 0: the limit of Algorithm 1 (prox weight 2 mu lambda) minimises
    ||y-Ax||^2 + lambda TV(x); checked against Chambolle-Pock."""
    A, D, y = _problem()
    lam = 0.6
    u = np.linalg.eigvalsh(D.T @ D).max()
    mu = 0.9 / (2 * u)
    x, _ = oracle.run(A, y, (5, 5), 3, 2, lam, mu, 1500, 50, row_unit=9, col_unit=5)
    x_cp = cp_reconstruct(D, y, lam, (5, 5)).ravel()
    assert np.linalg.norm(x - x_cp) / np.linalg.norm(x_cp) < 1e-6
    # the other reading of the weight (Eq. 1, 2 lambda TV) is a different point
    x_cp2 = cp_reconstruct(D, y, 2 * lam, (5, 5)).ravel()
    assert np.linalg.norm(x - x_cp2) / np.linalg.norm(x_cp2) > 10 * np.linalg.norm(x - x_cp) / np.linalg.norm(x_cp)


# ------------------------------------------------- stochastic variant (Sec. 3, R10)
def test_subset_draws_sizes_and_determinism():
    R, C = synth.subset_draws(8, 6, 0.5, 0.25, 50, seed=4)
    assert R.shape == (50, 8) and C.shape == (50, 6)
    assert np.all(R.sum(1) == 2) and np.all(C.sum(1) == 3)
    R2, C2 = synth.subset_draws(8, 6, 0.5, 0.25, 50, seed=4)
    assert np.array_equal(R, R2) and np.array_equal(C, C2)
    R3, C3 = synth.subset_draws(3, 3, 0.01, 0.01, 5)       # at least one block each
    assert np.all(R3.sum(1) == 1) and np.all(C3.sum(1) == 1)


def test_subsets_all_selected_is_algorithm1():
    """Every block drawn every iteration: exactly the epochs of Algorithm 1."""
    A = synth.parallel_beam_csr(16, 8, 23)
    y = synth.noisy_projections(A, synth.phantom(16, 4, 0), 0)
    u, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u)
    rs, cs = np.ones((12, 3), bool), np.ones((12, 4), bool)
    xa, ra = oracle.run_subsets(A, y, (16, 16), 3, 4, 0.05, mu, rs, cs, 10, row_unit=23, col_unit=16)
    xb, rb_ = oracle.run(A, y, (16, 16), 3, 4, 0.05, mu, 12, 10, row_unit=23, col_unit=16)
    assert np.array_equal(xa, xb) and np.array_equal(ra, rb_)


def test_subsets_touch_only_the_drawn_blocks():
    """With lambda = 0 one iteration changes x only on the drawn column blocks
    and r only on the drawn row blocks."""
    A = synth.parallel_beam_csr(16, 8, 23)
    y = synth.noisy_projections(A, synth.phantom(16, 4, 1), 1)
    rb, cb = oracle.partition(A.rows, A.cols_n, 4, 4, 23, 16)
    u, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u)
    R = np.array([[True] * 4, [False, True, False, False]])
    C = np.array([[True] * 4, [False, False, True, False]])
    x1, r1 = oracle.run_subsets(A, y, (16, 16), 4, 4, 0.0, mu, R[:1], C[:1], 0, 23, 16)
    x2, r2 = oracle.run_subsets(A, y, (16, 16), 4, 4, 0.0, mu, R, C, 0, 23, 16)
    outside = np.ones(A.cols_n, bool)
    outside[cb[2]:cb[3]] = False
    assert np.array_equal(x1[outside], x2[outside]) and not np.array_equal(x1, x2)
    rows_out = np.ones(A.rows, bool)
    rows_out[rb[1]:rb[2]] = False
    assert np.array_equal(r1[rows_out], r2[rows_out]) and not np.array_equal(r1, r2)


def test_subsets_converge_on_a_consistent_system():
    """lambda = 0 and y = A x_true with A of full column rank: the stochastic
    iteration (stale block products included) reaches x_true."""
    rng = np.random.default_rng(1)
    D = rng.random((48, 16)) * (rng.random((48, 16)) < 0.5)
    x_true = rng.random(16)
    y = D @ x_true
    mu = 0.9 / (2 * np.linalg.eigvalsh(D.T @ D).max())
    for a, g in [(0.5, 0.5), (0.25, 0.75)]:
        R, C = synth.subset_draws(4, 4, a, g, 20000, seed=3)
        x, _ = oracle.run_subsets(sp.csr_matrix(D), y, (4, 4), 4, 4, 0.0, mu, R, C, 0)
        assert np.linalg.norm(x - x_true) <= 1e-10 * np.linalg.norm(x_true)
