"""GPU parity of the stochastic block-subset variant (Sec. 3, reading R10)
against the oracle on the same draws: relative l2 error of x <= 1e-4 after
the run; with every block drawn the GPU iterations equal bsgdtv_run."""
import numpy as np
import pytest

import oracle
from paper_1812_01307_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_01307_gb300 import build
    build.build_library()
    from paper_1812_01307_gb300 import bsgdtv
    bsgdtv.load()
    torch.cuda.set_device(0)
    return bsgdtv


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = {
    # name: (n, n_angles, n_bins, n_ellipses, M, N, alpha, gamma, lambda, iters, K)
    "ellipse64": (64, 60, 91, 10, 4, 4, 0.5, 0.5, 0.05, 40, 20),
    "ragged37": (37, 11, 55, 4, 3, 5, 0.4, 0.67, 0.02, 30, 12),
    "lambda0": (64, 60, 91, 10, 4, 4, 0.25, 0.75, 0.0, 30, 0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_subsets_match_oracle(B, name):
    n, na, nb, ne, M, N, alpha, gamma, lam, iters, K = CASES[name]
    A = synth.parallel_beam_csr(n, na, nb)
    y = synth.noisy_projections(A, synth.phantom(n, ne, 2), 2).astype(np.float32)
    u, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u)
    R, C = synth.subset_draws(M, N, alpha, gamma, iters, seed=9)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y, lam, mu)
        rec.run_subsets(R, C, K)
        x_gpu = rec.x()
    x_ref, _ = oracle.run_subsets(A, y.astype(np.float64), (n, n), M, N, lam, mu, R, C, K,
                                  row_unit=nb, col_unit=n)
    assert rel(x_gpu, x_ref) <= 1e-4, rel(x_gpu, x_ref)


def test_all_blocks_drawn_equals_run(B):
    n, na, nb, ne, M, N = 64, 60, 91, 10, 4, 4
    A = synth.parallel_beam_csr(n, na, nb)
    y = synth.noisy_projections(A, synth.phantom(n, ne, 0), 0).astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y, 0.05)
        rec.run(12, 20)
        x_run = rec.x().copy()
        rec.set_data(y, 0.05)
        rec.run_subsets(np.ones((12, M), bool), np.ones((12, N), bool), 20)
        x_sub = rec.x().copy()
        with pytest.raises(B.BsgdtvError) as e:   # an iteration that draws no column block
            rec.run_subsets(np.ones((2, M), bool), np.zeros((2, N), bool), 20)
        assert e.value.code == -1
    assert rel(x_sub, x_run) <= 1e-6


@pytest.mark.parametrize("fmt", [1, 2])
def test_subsets_in_16_bit_formats(B, fmt):
    """Stored 16-bit formats take whole work items (no split ranges): every
    block drawn equals bsgdtv_run on the same handle, and random draws match
    the oracle run on the operator as stored."""
    from _formats import stored_operator
    n, na, nb, M, N = 64, 60, 91, 4, 4
    A = synth.parallel_beam_csr(n, na, nb)
    y = synth.noisy_projections(A, synth.phantom(n, 10, 0), 0).astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n, fmt=fmt) as rec:
        rec.set_data(y, 0.05)
        mu = rec.params()[0]
        rec.run(10, 20)
        x_run = rec.x().copy()
        rec.set_data(y, 0.05)
        rec.run_subsets(np.ones((10, M), bool), np.ones((10, N), bool), 20)
        assert rel(rec.x(), x_run) <= 1e-6
        rows, cols = synth.subset_draws(M, N, 0.5, 0.5, 25, seed=3)
        rec.set_data(y, 0.05)
        rec.run_subsets(rows, cols, 20)
        x_gpu = rec.x().copy()
    As = stored_operator(A, fmt)
    x_ref, _ = oracle.run_subsets(As, y.astype(np.float64), (n, n), M, N, 0.05, mu, rows, cols, 20,
                                  row_unit=nb, col_unit=n)
    assert rel(x_gpu, x_ref) <= 1e-4
