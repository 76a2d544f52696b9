"""GPU parity of the batched path (B slices sharing one matrix A, each with its
own y_b and lambda_b) against the FP64 oracle run slice by slice with the
block partition of the single-slice workload.

Tolerance: relative l2 error <= 1e-4 per slice after a full FP32
reconstruction (the single-slice bar); <= 1e-5 after the 3 epochs of the
full-size check."""
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
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


GEOM = {
    # name: (n, n_angles, n_bins, n_ellipses, M, N)
    "ellipse64": (64, 60, 91, 10, 4, 4),
    "ragged37": (37, 11, 55, 4, 3, 5),    # rays that miss the image: empty rows of A
}

_cache = {}


def _setup(name, slices):
    key = (name, slices)
    if key not in _cache:
        n, na, nb, ne, M, N = GEOM[name]
        A = synth.parallel_beam_csr(n, na, nb)
        _, Y = synth.slice_stack(A, n, ne, slices, seed=7)
        u, _ = oracle.power_iteration(A)
        _cache[key] = (A, Y.astype(np.float32), 0.9 / (2 * u))
    return _cache[key]


def _lambdas(slices):
    # a spread of weights, with lambda = 0 (identity prox) on every 4th slice
    lam = 0.02 * (1 + np.arange(slices) % 3)
    lam[1::4] = 0.0
    return lam


def _oracle_slice(name, A, y, lam, mu, epochs, K):
    n, na, nb, ne, M, N = GEOM[name]
    x, _ = oracle.run(A, y.astype(np.float64), (n, n), M, N, lam, mu, epochs, K, row_unit=nb,
                      col_unit=n)
    return x


@pytest.mark.parametrize("name,slices,epochs,K,check", [
    ("ellipse64", 1, 30, 20, None),
    ("ellipse64", 5, 30, 20, None),
    ("ellipse64", 33, 12, 20, [0, 1, 2, 31, 32]),        # 16 lanes per nonzero, padded to 64
    ("ellipse64", 70, 8, 20, [0, 5, 63, 64, 69]),        # 32 lanes per nonzero, padded to 128
    ("ragged37", 130, 6, 9, [0, 1, 127, 128, 129]),      # two chunks of 128 slices
])
def test_batch_matches_oracle_per_slice(B, name, slices, epochs, K, check):
    n = GEOM[name][0]
    A, Y, mu = _setup(name, slices)
    lam = _lambdas(slices)
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(epochs, K)
        X = bt.x()
    for b in (range(slices) if check is None else check):
        x_ref = _oracle_slice(name, A, Y[b], lam[b], mu, epochs, K)
        assert rel(X[b], x_ref) <= 1e-4, (b, rel(X[b], x_ref))


def test_batch_prox_multiwave_large_weight(B):
    """40 slices of 130x130 in one FGP launch group: 9 overlapping regions per
    slice, 360 CTAs per launch (several waves), with lambda so large that
    tau = mu * lambda is 0.3 .. 1.2: the duals move far in every iteration,
    so a region reading its halo from a neighbour that already stored the
    next launch's iterates would show.  Every slice vs the oracle."""
    n, na, nb = 130, 12, 185
    A = synth.parallel_beam_csr(n, na, nb)
    slices = 40
    _, Y = synth.slice_stack(A, n, 8, slices, seed=5)
    Y = Y.astype(np.float32)
    u, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u)
    lam = (0.3 + 0.9 * np.arange(slices) / (slices - 1)) / mu
    epochs, K = 3, 30
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(epochs, K)
        X = bt.x()
    for b in range(slices):
        x_ref, _ = oracle.run(A, Y[b].astype(np.float64), (n, n), 2, 3, lam[b], mu, epochs, K,
                              row_unit=nb, col_unit=n)
        assert rel(X[b], x_ref) <= 1e-4, (b, rel(X[b], x_ref))


def test_batch_without_prox_and_device_inputs(B):
    """lambda = 0 everywhere (no prox in the epoch), y and x passed as device tensors."""
    name, slices = "ellipse64", 3
    n = GEOM[name][0]
    A, Y, mu = _setup(name, slices)
    lam = np.zeros(slices)
    out = torch.zeros((slices, n * n), device="cuda")
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(torch.from_numpy(Y).cuda(), lam, mu)
        bt.run(10, 20)
        bt.x(out)
    X = out.cpu().numpy()
    for b in range(slices):
        assert rel(X[b], _oracle_slice(name, A, Y[b], 0.0, mu, 10, 20)) <= 1e-4


def test_batch_slice_equals_single_handle(B):
    """A slice of a batch and a single-slice handle on the same y reach the same x."""
    name, slices = "ellipse64", 4
    n, na, nb, ne, M, N = GEOM[name]
    A, Y, mu = _setup(name, slices)
    lam = np.full(slices, 0.05)
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(20, 20)
        X = bt.x()
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(Y[2], 0.05, mu)
        rec.run(20, 20)
        x1 = rec.x()
    assert rel(X[2], x1) <= 1e-5


def test_batch_deterministic_and_timed(B):
    name, slices = "ellipse64", 33
    n = GEOM[name][0]
    A, Y, mu = _setup(name, slices)
    lam = _lambdas(slices)
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(5, 12)
        X1 = bt.x().copy()
        bt.set_data(Y, lam, mu)
        bt.run(5, 12)
        X2 = bt.x().copy()
        bt.set_data(Y, lam, mu)
        before = B.bsgdtv_launch_count()
        pk, ep = bt.run_timed(5, 12)
        launched = B.bsgdtv_launch_count() - before
        X3 = bt.x().copy()
    assert np.array_equal(X1, X2) and np.array_equal(X1, X3)
    assert 0 < pk < ep
    # per epoch: row pass, column pass, two transposes, one FGP launch (64x64
    # fits one region); plus the transpose of get_x after the loop
    assert launched == 5 * 5


def test_batch_errors(B):
    n = 37
    A, Y, mu = _setup("ragged37", 130)
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_batch_create_csr(A.rows, A.cols_n, n, n, A.row_ptr, A.cols, A.vals, 0)
    assert e.value.code == -1
    bad = A.vals.copy()
    bad[3] = np.inf
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_batch_create_csr(A.rows, A.cols_n, n, n, A.row_ptr, A.cols, bad, 2)
    assert e.value.code == -6
    with B.BatchReconstructor(A, (n, n), 2) as bt:
        with pytest.raises(B.BsgdtvError) as e:
            bt.run(1, 5)
        assert e.value.code == -4
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_data(Y[:2], [0.1, -0.1], mu)
        assert e.value.code == -1
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_data(Y[:2], [0.1, 0.1], 0.0)
        assert e.value.code == -1
        y = Y[:2].copy()
        y[1, 17] = np.nan
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_data(y, [0.1, 0.1], mu)
        assert e.value.code == -6
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_data(torch.from_numpy(y).cuda(), [0.1, 0.1], mu)
        assert e.value.code == -6
        bt.set_data(Y[:2], [0.1, 0.1], mu)      # still usable after the rejections
        bt.run(2, 5)
        assert np.all(np.isfinite(bt.x()))


def test_batch_ellipse512_full_size(B):
    """64 slices of the 512x512 geometry (360 angles x 727 bins, lambda 0.02,
    50 FGP iterations) in the configuration bench.py times: 3 epochs, sampled
    slices against the oracle."""
    wl = synth.WORKLOADS["ellipse512"]
    A = synth.make_problem(wl).A
    slices = 64
    _, Y = synth.slice_stack(A, wl.n, wl.n_ellipses, slices, seed=wl.seed)
    Y = Y.astype(np.float32)
    u, _ = oracle.power_iteration(A, 200, 1e-10)
    mu = 0.9 / (2 * u)
    lam = np.full(slices, wl.lam)
    with B.BatchReconstructor(A, (wl.n, wl.n), slices) as bt:
        bt.set_data(torch.from_numpy(Y).cuda(), lam, mu)
        bt.run(3, wl.fgp_iters)
        X = bt.x()
    for b in (0, 63):
        x_ref, _ = oracle.run(A, Y[b].astype(np.float64), (wl.n, wl.n), wl.M, wl.N, wl.lam, mu, 3,
                              wl.fgp_iters, row_unit=wl.n_bins, col_unit=wl.n)
        assert rel(X[b], x_ref) <= 1e-5, (b, rel(X[b], x_ref))


@pytest.mark.parametrize("fmt,bound", [(2, 2e-3), (3, 2e-2)])
def test_batch_16bit_weights(B, fmt, bound):
    """FP16 / BF16 weights: each slice matches the oracle on the rounded
    operator to 1e-4; the distance to the oracle on the FP64 operator is the
    quantisation error (FP16 <= 2e-3)."""
    from _formats import stored_operator
    name, slices, epochs, K = "ellipse64", 5, 30, 20
    n, na, nb, ne, M, N = GEOM[name]
    A, Y, mu = _setup(name, slices)
    As = stored_operator(A, fmt)
    lam = _lambdas(slices)
    with B.BatchReconstructor(A, (n, n), slices, fmt=fmt) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(epochs, K)
        X = bt.x()
    for b in range(slices):
        x_s = _oracle_slice(name, As, Y[b], lam[b], mu, epochs, K)
        assert rel(X[b], x_s) <= 1e-4, (b, rel(X[b], x_s))
        x_64 = _oracle_slice(name, A, Y[b], lam[b], mu, epochs, K)
        assert rel(X[b], x_64) <= bound


def test_batch_host_y_is_read_before_return(B):
    """Pinned host buffers passed to set_data and set_slice may be overwritten
    as soon as the calls return; a NaN in set_slice's y leaves the slot as it
    was, a NaN in set_data's y leaves the batch without data."""
    name, slices = "ellipse64", 3
    n = GEOM[name][0]
    A, Y, mu = _setup(name, slices)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    lam = np.full(slices, 0.04)
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(Y, lam, mu)
        bt.set_slice(2, Y[0], 0.04)
        bt.run(5, 15)
        X_ref = bt.x().copy()
        pin = torch.empty(Y.size, dtype=torch.float32).pin_memory()
        yp = pin.numpy().reshape(Y.shape)
        yp[:] = Y
        bt.set_data(yp, lam, mu)
        yp[:] = np.nan
        yp[0] = Y[0]
        bt.set_slice(2, yp[0], 0.04)
        yp[0] = np.nan
        bad = Y[1].copy()
        bad[5] = np.nan
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_slice(1, bad, 0.04)       # rejected: slot 1 keeps its data
        assert e.value.code == -6
        bt.run(5, 15)
        assert np.array_equal(bt.x(), X_ref)
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_data(yp, lam, mu)          # NaN everywhere now
        assert e.value.code == -6
        with pytest.raises(B.BsgdtvError) as e:
            bt.run(1, 15)
        assert e.value.code == -4


def test_batch_set_slice_restarts_one_slot(B):
    """A slot restarted mid-run follows Algorithm 1 from its own x^0 = 0 while
    the other slots carry on; the restarted slot's iterates are bit-identical
    to the same request run with every other slot empty."""
    name, slices = "ellipse64", 6
    n = GEOM[name][0]
    A, Y, mu = _setup(name, slices)
    lam = np.full(slices, 0.04)
    A2, Ynew, _ = _setup(name, slices + 1)
    y_new = Ynew[slices]                     # a seventh, different slice
    with B.BatchReconstructor(A, (n, n), slices) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(5, 20)
        bt.set_slice(3, y_new, 0.08)
        bt.run(10, 20)
        X = bt.x()
        x3 = bt.slice_x(3)
        bt.set_slice(1, None, 0.0)          # emptied slot stays zero
        bt.run(2, 20)
        assert not np.any(bt.slice_x(1))
    assert np.array_equal(x3, X[3])
    assert rel(X[3], _oracle_slice(name, A, y_new, 0.08, mu, 10, 20)) <= 1e-4
    for b in (0, 5):
        assert rel(X[b], _oracle_slice(name, A, Y[b], 0.04, mu, 15, 20)) <= 1e-4
    with B.BatchReconstructor(A, (n, n), slices) as alone:
        alone.set_data(np.zeros_like(Y), np.zeros(slices), mu)
        alone.set_slice(3, y_new, 0.08)
        alone.run(10, 20)
        assert np.array_equal(alone.slice_x(3), x3)


def test_batch_autotune_keeps_results(B):
    """The autotuner times the passes' lanes per nonzero and every candidate
    FGP launch shape on the batch's data, restores the state after each trial
    and keeps the fastest; FGP shapes give bit-identical iterates, other
    lanes per nonzero change only the FP32 summation order (<= 1e-6), and a
    tuning applied by hand reproduces the tuned run bit for bit.  130x130
    images (several regions), 16 slices (4 lanes per nonzero; 2 tried)."""
    n, na, nb = 130, 12, 185
    A = synth.parallel_beam_csr(n, na, nb)
    _, Y = synth.slice_stack(A, n, 8, 16, seed=3)
    Y = Y.astype(np.float32)
    u, _ = oracle.power_iteration(A)
    mu, lam = 0.9 / (2 * u), np.full(16, 0.05)
    with B.BatchReconstructor(A, (n, n), 16) as bt:
        bt.set_data(Y, lam, mu)
        bt.run(4, 30)
        X_plain = bt.x().copy()
        bt.set_data(Y, lam, mu)
        bt.run(2, 30)
        chunk, group, ms = bt.autotune(30, 2)
        assert chunk in (3, 4, 5, 6, 8) and 1 <= group <= 16 and ms > 0
        tuned = bt.tuning()
        bt.run(2, 30)
        X_tuned = bt.x().copy()
        bt.set_tuning(3, 2)                  # FGP shape by hand: same bits
        bt.set_pass_lanes(0, 0)
        bt.set_data(Y, lam, mu)
        bt.run(4, 30)
        X_set = bt.x().copy()
        bt.set_tuning(tuned[0], tuned[1])    # the tuned choice by hand: the tuned bits
        bt.set_pass_lanes(tuned[2], tuned[3])
        bt.set_data(Y, lam, mu)
        bt.run(4, 30)
        X_again = bt.x().copy()
        bt.set_pass_lanes(2, 0)              # other lanes: FP32 rounding only
        bt.set_data(Y, lam, mu)
        bt.run(4, 30)
        X_lanes = bt.x().copy()
        with pytest.raises(B.BsgdtvError) as e:
            bt.set_tuning(9, 0)
        assert e.value.code == -1
        for bad in (3, 1):
            with pytest.raises(B.BsgdtvError) as e:
                bt.set_pass_lanes(bad, 0)
            assert e.value.code == -1
    assert np.array_equal(X_plain, X_set)
    assert np.array_equal(X_tuned, X_again)
    for X in (X_tuned, X_lanes):
        for b in range(16):
            assert rel(X[b], X_plain[b]) <= 1e-6


def test_batches_share_one_operator(B):
    """One stored A (an operator) serves batches of different sizes at once;
    each gives the same bits as a batch that owns its copy of A, and the
    operator may be released before the batches that use it."""
    name = "ragged37"
    n, na, nb, ne, M, N = GEOM[name]
    A, Y, mu = _setup(name, 40)
    lam = _lambdas(40)
    op = B.bsgdtv_operator_create_csr(A.rows, A.cols_n, n, n, A.row_ptr, A.cols, A.vals)
    small = B.BatchReconstructor(None, (n, n), 3, operator=op)
    big = B.BatchReconstructor(None, (n, n), 40, operator=op)
    B.bsgdtv_operator_destroy(op)                   # the batches keep it alive
    small.set_data(Y[:3], lam[:3], mu)
    big.set_data(Y, lam, mu)
    small.run(6, 9)
    big.run(6, 9)
    Xs, Xb = small.x(), big.x()
    small.close()
    big.close()
    with B.BatchReconstructor(A, (n, n), 40) as own:
        own.set_data(Y, lam, mu)
        own.run(6, 9)
        Xo = own.x()
    assert np.array_equal(Xb, Xo)
    for b in range(3):
        assert rel(Xs[b], Xo[b]) <= 1e-6
        assert rel(Xs[b], _oracle_slice(name, A, Y[b], lam[b], mu, 6, 9)) <= 1e-4


def test_packed_batch_of_three_geometries(B):
    """Requests of three geometries (64x64, ragged 37x37 with rays missing the
    image, 130x130 over several FGP regions) packed into one handle: every
    epoch stage is one launch over all parts (2 passes, 2 transposes and one
    launch per chunk of FGP iterations, whatever the number of parts), and
    each slot equals the same slot of a batch of its geometry alone bit for
    bit and the oracle within 1e-4."""
    geoms = [(64, 60, 91, 10), (37, 11, 55, 4), (130, 12, 185, 8)]
    slices, epochs, K = 4, 12, 15
    As, Ys, mus, lams = [], [], [], []
    for gi, (n, na, nb, ne) in enumerate(geoms):
        A = synth.parallel_beam_csr(n, na, nb)
        _, Y = synth.slice_stack(A, n, ne, slices, seed=11 + gi)
        u, _ = oracle.power_iteration(A)
        As.append(A)
        Ys.append(Y.astype(np.float32))
        mus.append(0.9 / (2 * u))
        lams.append(np.array([0.05, 0.0, 0.02, 0.1]) * (1 + gi))
    shapes = [(g[0], g[0]) for g in geoms]
    with B.PackedBatch(As, shapes, slices) as pk:
        for k in range(3):
            pk.set_part(k, Ys[k], lams[k], mus[k])
        pk.run(epochs, K)
        Xs = [pk.x(k) for k in range(3)]
        launches = pk.launches_per_epoch(K)
    assert launches == 2 + 2 + (K + 4) // 5           # 5 FGP iterations per launch
    for k, (n, na, nb, ne) in enumerate(geoms):
        with B.BatchReconstructor(As[k], shapes[k], slices) as bt:
            bt.set_data(Ys[k], lams[k], mus[k])
            bt.run(epochs, K)
            assert np.array_equal(bt.x(), Xs[k]), k
        for b in range(slices):
            x_ref, _ = oracle.run(As[k], Ys[k][b].astype(np.float64), (n, n), 1, 1, lams[k][b], mus[k],
                                  epochs, K)
            assert rel(Xs[k][b], x_ref) <= 1e-4, (k, b)
