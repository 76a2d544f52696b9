"""Pins for the oracle's TV prox (the proximal step of Algorithm 1, solved by
Beck-Teboulle FGP): operator identities, the duality gap, closed forms,
invariances and an independent convex solver."""
import numpy as np
import pytest

import oracle

from _independent import cp_denoise, grad, tv_definition


def test_L_and_Lt_are_adjoint():
    rng = np.random.default_rng(0)
    for m, n in [(5, 7), (1, 4), (6, 1), (2, 2)]:
        p = rng.standard_normal((m - 1, n))
        q = rng.standard_normal((m, n - 1))
        x = rng.standard_normal((m, n))
        P, Q = oracle.Lt_op(x)
        assert np.isclose(np.sum(oracle.L_op(p, q) * x), np.sum(p * P) + np.sum(q * Q), rtol=1e-13, atol=1e-13)


def test_tv_against_definition_and_closed_forms():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 9))
    assert np.isclose(oracle.tv_iso(x), tv_definition(x), rtol=1e-14)
    m, n = 7, 5
    ramp = np.tile(np.arange(n, dtype=float), (m, 1))      # x_{s,t} = t
    assert np.isclose(oracle.tv_iso(ramp), m * (n - 1))
    assert oracle.tv_iso(np.full((4, 4), 3.7)) == 0.0


def test_tv_is_the_support_function_of_the_dual_set():
    # TV_I(x) = max over the isotropic dual set of <L(p,q), x>, attained at the
    # normalised forward differences
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 5))
    P, Q = oracle.Lt_op(x)
    p, q = oracle.proj_iso(1e6 * P, 1e6 * Q)
    assert np.isclose(np.sum(oracle.L_op(p, q) * x), oracle.tv_iso(x), rtol=1e-9)
    for _ in range(20):
        p, q = oracle.proj_iso(rng.standard_normal(P.shape) * 3, rng.standard_normal(Q.shape) * 3)
        assert np.sum(oracle.L_op(p, q) * x) <= oracle.tv_iso(x) + 1e-12


def _primal(x, b, tau):
    return np.sum((x - b) ** 2) + 2 * tau * tv_definition(x)


def _dual(p, q, b, tau):
    return np.sum(b * b) - np.sum((b - tau * oracle.L_op(p, q)) ** 2)


@pytest.mark.parametrize("shape,tau", [((8, 8), 0.3), ((12, 7), 1.0), ((5, 9), 0.05)])
def test_duality_gap_closes(shape, tau):
    rng = np.random.default_rng(4)
    b = rng.standard_normal(shape)
    x, p, q = oracle.fgp(b, tau, 12000, return_dual=True)
    # feasibility of (p, q)
    m1, n1 = shape[0] - 1, shape[1] - 1
    assert np.all(p[:m1, :n1] ** 2 + q[:m1, :n1] ** 2 <= 1 + 1e-12)
    assert np.all(np.abs(p[:, n1]) <= 1 + 1e-12) and np.all(np.abs(q[m1, :]) <= 1 + 1e-12)
    gap = _primal(x, b, tau) - _dual(p, q, b, tau)
    assert gap >= -1e-10
    assert gap < 1e-7 * _primal(x, b, tau)


def test_gap_decreases_with_iterations():
    rng = np.random.default_rng(5)
    b = rng.standard_normal((10, 10))
    gaps = []
    for K in (5, 20, 80, 320):
        x, p, q = oracle.fgp(b, 0.5, K, return_dual=True)
        gaps.append(_primal(x, b, 0.5) - _dual(p, q, b, 0.5))
    assert all(g2 < g1 for g1, g2 in zip(gaps, gaps[1:]))


def test_constant_image_unchanged():
    b = np.full((9, 6), -1.25)
    for K in (1, 7, 50):
        assert np.array_equal(oracle.fgp(b, 0.7, K), b)


def test_sum_and_shift():
    rng = np.random.default_rng(6)
    b = rng.standard_normal((7, 8))
    x = oracle.fgp(b, 0.4, 30)
    assert np.isclose(x.sum(), b.sum(), rtol=0, atol=1e-12)
    assert np.allclose(oracle.fgp(b + 5.0, 0.4, 30), x + 5.0, atol=1e-12)


def test_step_edge_closed_form():
    # top h rows = a, bottom w rows = c (a > c): every column is the 1-D problem
    # h(alpha-a)^2 + w(beta-c)^2 + 2 tau |alpha-beta|, solved by
    # alpha = a - tau/h, beta = c + tau/w while alpha > beta
    m, n, h = 10, 6, 4
    a, c, tau = 2.0, -1.0, 0.9
    b = np.full((m, n), c)
    b[:h] = a
    x = oracle.fgp(b, tau, 4000)
    assert np.allclose(x[:h], a - tau / h, atol=1e-8)
    assert np.allclose(x[h:], c + tau / (m - h), atol=1e-8)
    # large tau merges both levels at the mean
    x = oracle.fgp(b, 50.0, 4000)
    assert np.allclose(x, b.mean(), atol=1e-8)


def test_matches_independent_solver_8x8():
    rng = np.random.default_rng(7)
    b = rng.standard_normal((8, 8)) + np.outer(np.arange(8) > 3, np.ones(8))
    x = oracle.fgp(b, 0.35, 5000)
    x_cp = cp_denoise(b, 0.35, 40000)
    P_fgp, P_cp = _primal(x, b, 0.35), _primal(x_cp, b, 0.35)
    # the primal is 2-strongly convex: P(v) - P(x*) >= ||v - x*||^2, so if the FGP
    # output is the minimiser, CP's iterate lies within sqrt(P_cp - P_fgp) of it
    assert P_fgp <= P_cp + 1e-12 * P_cp
    assert np.sum((x - x_cp) ** 2) <= (P_cp - P_fgp) + 1e-12 * P_cp
    assert np.max(np.abs(x - x_cp)) < 1e-3


def test_zero_iterations_and_zero_weight_are_identity():
    rng = np.random.default_rng(8)
    b = rng.standard_normal((4, 5))
    assert np.array_equal(oracle.fgp(b, 0.3, 0), b)
    assert np.array_equal(oracle.fgp(b, 0.0, 10), b)


def test_eq2_backward_tv_is_rotated_forward_tv():
    # Eq. 2 (backward differences, zero-difference border) equals TV_I of the
    # image rotated by 180 degrees
    rng = np.random.default_rng(9)
    x = rng.standard_normal((5, 6))
    m, n = x.shape
    eq2 = 0.0
    for s in range(m):
        for t in range(n):
            dv = x[s, t] - x[s - 1, t] if s > 0 else 0.0
            dh = x[s, t] - x[s, t - 1] if t > 0 else 0.0
            eq2 += np.hypot(dv, dh)
    assert np.isclose(eq2, oracle.tv_iso(x[::-1, ::-1]), rtol=1e-14)


def test_grad_helper_consistent():
    x = np.arange(12.0).reshape(3, 4)
    gv, gh = grad(x)
    P, Q = oracle.Lt_op(x)
    assert np.array_equal(gv[:-1], P) and np.array_equal(gh[:, :-1], Q)
