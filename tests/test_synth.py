"""Pins for the seeded input generator (Siddon projector, phantom, noise)."""
import numpy as np
import pytest

from paper_1812_01307_gb300 import synth


def _supersampled(n, theta, u, step=2e-4):
    """Brute force: walk the line in tiny steps and add each step to the pixel
    that contains it (pixel (s,t) = [t-n/2, t+1-n/2) x [n/2-s-1, n/2-s))."""
    c, s = np.cos(theta), np.sin(theta)
    if abs(c) < 1e-15:
        c = 0.0
    if abs(s) < 1e-15:
        s = 0.0
    h = n / 2.0
    a = np.arange(-n, n, step) + step / 2
    x = u * c - a * s
    y = u * s + a * c
    inside = (x >= -h) & (x < h) & (y >= -h) & (y < h)
    t = np.floor(x[inside] + h).astype(int)
    row = n - 1 - np.floor(y[inside] + h).astype(int)
    w = np.zeros(n * n)
    np.add.at(w, row * n + t, step)
    return w


@pytest.mark.parametrize("theta,u", [(0.3, 0.37), (1.1, -1.6), (2.0, 0.5), (np.pi / 4, 0.0),
                                     (3.0, 2.2), (0.05, -2.9)])
def test_ray_matches_supersampling(theta, u):
    n = 6
    cols, vals = synth.siddon_ray(n, theta, u)
    dense = np.zeros(n * n)
    dense[cols] = vals
    ref = _supersampled(n, theta, u)
    assert np.max(np.abs(dense - ref)) < 2e-3
    assert np.all(np.diff(cols) > 0)


def test_chord_length_closed_form():
    # a line through the centre of the n x n square at angle theta has chord
    # n / max(|cos|, |sin|)
    n = 8
    for theta in np.linspace(0.01, np.pi - 0.01, 23):
        cols, vals = synth.siddon_ray(n, theta, 0.0)
        expect = n / max(abs(np.cos(theta)), abs(np.sin(theta)))
        assert abs(vals.sum() - expect) < 1e-12 * expect


def test_axis_aligned_rays_follow_half_open_rule():
    n = 6
    # theta = 0: the ray is the vertical line x = u; integer u lies on a grid line
    # and is given to the pixel column on its + side, t = u + n/2.
    for u in range(-3, 3):
        cols, vals = synth.siddon_ray(n, 0.0, float(u))
        assert len(cols) == n
        assert np.all(cols % n == u + n // 2)
        assert np.allclose(vals, 1.0, atol=0, rtol=1e-15)
    cols, _ = synth.siddon_ray(n, 0.0, 3.0)   # on the right border: outside every pixel
    assert len(cols) == 0
    # theta = pi/2: horizontal line y = u goes to the row above it (y-range [u, u+1))
    for u in range(-3, 3):
        cols, vals = synth.siddon_ray(n, np.pi / 2, float(u))
        assert len(cols) == n
        assert np.all(cols // n == n - 1 - (u + n // 2))
        assert np.allclose(vals, 1.0)


def test_matrix_structure_and_conventions():
    A = synth.parallel_beam_csr(8, 12, 13)
    assert A.rows == 12 * 13 and A.cols_n == 64
    assert A.row_ptr[0] == 0 and np.all(np.diff(A.row_ptr) >= 0)
    for r in range(A.rows):
        c = A.cols[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.all((A.cols >= 0) & (A.cols < 64))
    assert np.all(A.vals > 0) and np.all(A.vals <= np.sqrt(2) + 1e-12)
    # row k*n_bins + d is angle k, detector offset d - (n_bins-1)/2
    k, d = 5, 2
    cols, vals = synth.siddon_ray(8, k * np.pi / 12, d - 6.0)
    r = k * 13 + d
    assert np.array_equal(A.cols[A.row_ptr[r]:A.row_ptr[r + 1]], cols)
    assert np.array_equal(A.vals[A.row_ptr[r]:A.row_ptr[r + 1]], vals)


def test_every_pixel_seen_and_nnz_estimate():
    A = synth.parallel_beam_csr(32, 40, 47)
    counts = np.bincount(A.cols, minlength=32 * 32)
    assert counts.min() > 0
    # expected nnz ~ n_angles * n^2 * mean(|cos|+|sin|) = n_angles n^2 4/pi
    est = 40 * 32 * 32 * 4 / np.pi
    assert abs(A.nnz - est) / est < 0.05


def test_phantom_recipe():
    p = synth.ellipse_params(10, 0, 1.0)
    assert p.shape == (10, 6)
    assert np.all(np.abs(p[:, :2]) <= 24) and np.all((p[:, 2:4] >= 3) & (p[:, 2:4] <= 20))
    assert np.all((p[:, 4] >= 0) & (p[:, 4] <= np.pi)) and np.all((p[:, 5] >= 0) & (p[:, 5] <= 1))
    img = synth.phantom(64, 10, 0)
    assert img.shape == (64, 64) and img.min() >= 0
    # a single centred circle of radius 20 covers ~pi 20^2 pixel centres
    rng_free = synth.phantom(128, 0, 0)
    assert rng_free.sum() == 0


def test_noise_level_and_determinism():
    P = synth.make_problem("ellipse64", cache=False)
    y_clean = synth.csr_matvec(P.A, P.x_true)
    sigma = 0.01 * np.mean(np.abs(y_clean))
    e = P.y - y_clean
    assert abs(np.std(e) / sigma - 1.0) < 0.05
    P2 = synth.make_problem("ellipse64", cache=False)
    assert np.array_equal(P.y, P2.y) and np.array_equal(P.A.vals, P2.A.vals)


def test_phantom_bounding_box_equals_whole_grid():
    """The phantom evaluates each ellipse only inside a widened bounding box;
    evaluating every pixel of the grid gives the same image bit for bit."""
    for n, ne, seed in [(64, 10, 0), (37, 4, 1), (128, 10, 2), (9, 3, 3), (200, 25, 4)]:
        params = synth.ellipse_params(ne, seed, n / 64.0)
        t = np.arange(n, dtype=np.float64) - 0.5 * (n - 1)
        X = t[None, :].repeat(n, axis=0)
        Y = (-t)[:, None].repeat(n, axis=1)
        ref = np.zeros((n, n))
        for cx, cy, a, b, phi, inten in params:
            dx, dy = X - cx, Y - cy
            xr = dx * np.cos(phi) + dy * np.sin(phi)
            yr = -dx * np.sin(phi) + dy * np.cos(phi)
            ref[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += inten
        assert np.array_equal(synth.phantom(n, ne, seed), ref)
