"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances: partition bounds bit-exact; relative l2 error <= 1e-5 per block
block product; <= 1e-4 on x after a full FP32 reconstruction; the prox
alone <= 1e-5; u_max and the FP64 objective <= 1e-9."""
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


def f32(A):
    """The operator as the GPU stores it (FP32 weights), for FP64 comparisons."""
    return synth.CSR(A.rows, A.cols_n, A.row_ptr, A.cols, A.vals.astype(np.float32).astype(np.float64))


CASES = {
    # name: (n, n_angles, n_bins, M, N)
    "ellipse64": (64, 60, 91, 4, 4),
    "ragged37": (37, 11, 55, 3, 5),     # ragged tiles/bands, rays that miss the image
    "rowbands70": (70, 9, 101, 9, 70),  # one image row per column block
    "wide130": (130, 12, 185, 2, 3),    # several tiles per band
}


def _problem(name):
    n, na, nb, M, N = CASES[name]
    A = synth.parallel_beam_csr(n, na, nb)
    x_true = synth.phantom(n, 10, 0)
    y = synth.noisy_projections(A, x_true, 0)
    return A, x_true, y, n, na, nb, M, N


@pytest.mark.parametrize("name", list(CASES))
def test_partition_bit_exact(B, name):
    A, _, _, n, na, nb, M, N = _problem(name)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rb, cb = rec.partition()
    rb_o, cb_o = oracle.partition(A.rows, A.cols_n, M, N, nb, n)
    assert np.array_equal(rb, rb_o) and np.array_equal(cb, cb_o)


@pytest.mark.parametrize("name", list(CASES))
def test_block_products(B, name):
    A, _, _, n, na, nb, M, N = _problem(name)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(A.cols_n).astype(np.float32)
    r = rng.standard_normal(A.rows).astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        zb = torch.zeros(N * A.rows, device="cuda")
        gb = torch.zeros(M * A.cols_n, device="cuda")
        B.bsgdtv_block_products(rec.h, torch.from_numpy(x).cuda(), torch.from_numpy(r).cuda(), zb, gb)
        zb = zb.cpu().numpy().reshape(N, A.rows)
        gb = gb.cpu().numpy().reshape(M, A.cols_n)
    rb, cb = oracle.partition(A.rows, A.cols_n, M, N, nb, n)
    blocks = oracle.split_blocks(A, rb, cb)
    z, gh = oracle.block_products(blocks, rb, cb, x.astype(np.float64), r.astype(np.float64))
    worst = 0.0
    for i in range(M):
        for j in range(N):
            ez = rel(zb[j, rb[i]:rb[i + 1]], z[i][j])
            eg = rel(gb[i, cb[j]:cb[j + 1]], gh[i][j])
            worst = max(worst, ez, eg)
    assert worst <= 1e-5, worst


def test_block_products_random_csr_explicit_bounds(B):
    import scipy.sparse as sp
    rng = np.random.default_rng(0)
    h, w = 23, 70
    rows, cols = 57, h * w
    dense = (rng.random((rows, cols)) < 0.05) * rng.standard_normal((rows, cols))
    dense[5] = 0.0
    S = sp.csr_matrix(dense)
    S.sort_indices()
    A = synth.CSR(rows, cols, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    rb = np.array([0, 10, 10, 40, 57])
    cb = np.array([0, 3, 11, 23]) * w
    x = rng.standard_normal(cols).astype(np.float32)
    r = rng.standard_normal(rows).astype(np.float32)
    with B.Reconstructor(A, (h, w), 4, 3, row_bounds=rb, col_bounds=cb) as rec:
        zb = torch.zeros(3 * rows, device="cuda")
        gb = torch.zeros(4 * cols, device="cuda")
        B.bsgdtv_block_products(rec.h, torch.from_numpy(x).cuda(), torch.from_numpy(r).cuda(), zb, gb)
        zb = zb.cpu().numpy().reshape(3, rows)
        gb = gb.cpu().numpy().reshape(4, cols)
    blocks = oracle.split_blocks(A, rb, cb)
    z, gh = oracle.block_products(blocks, rb, cb, x.astype(np.float64), r.astype(np.float64))
    for i in range(4):
        for j in range(3):
            assert rel(zb[j, rb[i]:rb[i + 1]], z[i][j]) <= 1e-5
            assert rel(gb[i, cb[j]:cb[j + 1]], gh[i][j]) <= 1e-5


@pytest.mark.parametrize("name", ["ellipse64", "ragged37", "wide130"])
def test_umax_matches_oracle(B, name):
    A, _, _, n, na, nb, M, N = _problem(name)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        u, it = rec.estimate_umax(5000, 1e-12)
    u_ref, it_ref = oracle.power_iteration(f32(A), 5000, 1e-12)
    assert abs(u - u_ref) <= 1e-9 * u_ref
    assert abs(it - it_ref) <= 2


def test_umax_tiny_against_eigvalsh(B):
    A = synth.parallel_beam_csr(6, 40, 11)
    D = f32(A).to_scipy().toarray()
    with B.Reconstructor(A, (6, 6), 2, 2, row_unit=11, col_unit=6) as rec:
        u, _ = rec.estimate_umax(5000, 1e-13)
    assert abs(u - np.linalg.eigvalsh(D.T @ D).max()) <= 1e-9 * u


def _run_both(B, name, lam, epochs, K, mu_from="oracle"):
    A, x_true, y, n, na, nb, M, N = _problem(name)
    u_ref, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u_ref)
    y32 = y.astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(torch.from_numpy(y32).cuda(), lam, mu)
        rec.run(epochs, K)
        x_gpu = rec.x().astype(np.float64)
    x_ref, _ = oracle.run(A, y32.astype(np.float64), (n, n), M, N, lam, mu, epochs, K,
                          row_unit=nb, col_unit=n)
    return x_gpu, x_ref, x_true


def test_full_reconstruction_ellipse64(B):
    """The 64x64 workload end to end: 50 epochs, 20 FGP iterations, lambda 0.05."""
    wl = synth.WORKLOADS["ellipse64"]
    x_gpu, x_ref, x_true = _run_both(B, "ellipse64", wl.lam, wl.epochs, wl.fgp_iters)
    assert rel(x_gpu, x_ref) <= 1e-4
    assert rel(x_ref, x_true) < 0.5       # it does reconstruct


@pytest.mark.parametrize("name,lam,epochs,K", [("ragged37", 0.05, 30, 25), ("wide130", 0.03, 20, 17),
                                               ("rowbands70", 0.0, 25, 10), ("ellipse64", 0.2, 10, 1)])
def test_full_reconstruction_cases(B, name, lam, epochs, K):
    x_gpu, x_ref, _ = _run_both(B, name, lam, epochs, K)
    assert rel(x_gpu, x_ref) <= 1e-4


@pytest.mark.parametrize("shape,tau,K", [((64, 64), 0.3, 20), ((100, 77), 0.5, 50), ((1, 40), 0.4, 10),
                                         ((40, 1), 0.4, 10), ((2, 2), 1.0, 5), ((65, 64), 0.2, 30),
                                         ((64, 65), 0.2, 9), ((200, 130), 0.1, 17), ((37, 91), 2.0, 8)])
def test_tv_prox_matches_oracle(B, shape, tau, K):
    rng = np.random.default_rng(2)
    b = (rng.standard_normal(shape) + (np.arange(shape[0])[:, None] > shape[0] // 2)).astype(np.float32)
    bt = torch.from_numpy(b).cuda()
    xt = torch.empty_like(bt)
    B.bsgdtv_tv_prox(bt, xt, tau, K)
    ref = oracle.fgp(b.astype(np.float64), tau, K)
    assert rel(xt.cpu().numpy(), ref) <= 1e-5


def test_tv_prox_512_full_size(B):
    rng = np.random.default_rng(3)
    b = synth.phantom(512, 30, 0) + 0.05 * rng.standard_normal((512, 512))
    b = b.astype(np.float32)
    bt = torch.from_numpy(b).cuda()
    xt = torch.empty_like(bt)
    B.bsgdtv_tv_prox(bt, xt, 0.02 * 1e-3, 50)
    ref = oracle.fgp(b.astype(np.float64), 0.02 * 1e-3, 50)
    assert rel(xt.cpu().numpy(), ref) <= 1e-5
    B.bsgdtv_tv_prox(bt, xt, 0.5, 50)
    ref = oracle.fgp(b.astype(np.float64), 0.5, 50)
    assert rel(xt.cpu().numpy(), ref) <= 1e-5


def test_tv_prox_multiwave_large_tau(B):
    """1024x1024 with a large weight: each launch of the tiled FGP covers 576
    overlapping 64x64 regions (several waves of CTAs on the GPU), and with
    tau = 0.5 every iteration moves the duals a long way, so a region that
    read a neighbour's halo after that neighbour had already stored the next
    launch's iterates would stand out.  Two weights, 40 and 23 iterations."""
    rng = np.random.default_rng(9)
    b = synth.phantom(1024, 40, 5) + 0.2 * rng.standard_normal((1024, 1024))
    b = b.astype(np.float32)
    bt = torch.from_numpy(b).cuda()
    xt = torch.empty_like(bt)
    for tau, K in ((0.5, 40), (2.0, 23)):
        B.bsgdtv_tv_prox(bt, xt, tau, K)
        ref = oracle.fgp(b.astype(np.float64), tau, K)
        assert rel(xt.cpu().numpy(), ref) <= 1e-5, (tau, K)


def test_tv_prox_degenerate_cases(B):
    b = torch.full((33, 70), -1.25, device="cuda")
    x = torch.empty_like(b)
    B.bsgdtv_tv_prox(b, x, 0.7, 13)
    assert torch.equal(x, b)                       # constant image unchanged
    rng = np.random.default_rng(4)
    b = torch.from_numpy(rng.standard_normal((20, 30)).astype(np.float32)).cuda()
    x1 = torch.empty_like(b)
    B.bsgdtv_tv_prox(b, x1, 0.5, 0)
    assert torch.equal(x1, b)                      # zero iterations: identity
    x2 = torch.empty_like(b)
    B.bsgdtv_tv_prox(b, x2, 0.0, 10)
    assert torch.equal(x2, b)                      # zero weight: identity
    with pytest.raises(B.BsgdtvError):
        B.bsgdtv_tv_prox(b, b, 0.5, 3)             # aliasing rejected


def test_objective_fp64(B):
    A, _, y, n, na, nb, M, N = _problem("ellipse64")
    y32 = y.astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y32, 0.05)
        rec.run(7, 10)
        f, tv = rec.objective()
        x = rec.x().astype(np.float64)
    F, f_ref, tv_ref = oracle.objective(f32(A), y32.astype(np.float64), x, 0.05, (n, n))
    assert abs(f - f_ref) <= 1e-9 * f_ref
    assert abs(tv - tv_ref) <= 1e-9 * tv_ref


def test_run_until_stops_on_the_objective(B):
    """bsgdtv_run_until: checks F = data + lambda TV every 5 epochs and stops
    at the first step whose relative decrease is <= rel_tol; the reported F
    is the handle's FP64 objective at that epoch, the oracle's F of the same
    iterate agrees to 1e-9 and of the oracle's own iterate to 1e-3 (F is a
    small residual there), and the iterates equal a plain run of as many
    epochs, bit for bit."""
    A, _, y, n, na, nb, M, N = _problem("ellipse64")
    y32 = y.astype(np.float32)
    lam, K, c, tol = 0.05, 20, 5, 2e-2   # the oracle's F first moves < 2 % over 5 epochs at 120
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y32, lam)
        mu = rec.params()[0]
        k, F = rec.run_until(400, K, check_every=c, rel_tol=tol)
        x_k = rec.x().copy()
        d, tv = rec.objective()
        assert F == d + lam * tv and c <= k < 400 and k % c == 0

        def F_at(e):
            rec.set_data(y32, lam)
            rec.run(e, K)
            d_, tv_ = rec.objective()
            return d_ + lam * tv_, rec.x().copy()

        f_k, x_again = F_at(k)
        assert f_k == F and np.array_equal(x_again, x_k)
        f_prev, _ = F_at(k - c)
        assert abs(f_prev - f_k) <= tol * f_prev
        if k >= 2 * c:
            f_pp, _ = F_at(k - 2 * c)
            assert abs(f_pp - f_prev) > tol * f_pp
        rec.set_data(y32, lam)
        k0, _ = rec.run_until(7, K, check_every=3, rel_tol=0.0)   # runs to the end: 3 + 3 + 1
        assert k0 == 7
        with pytest.raises(B.BsgdtvError) as e:
            rec.run_until(7, K, check_every=0)
        assert e.value.code == -1
    Fo, _, _ = oracle.objective(f32(A), y32.astype(np.float64), x_k.astype(np.float64), lam, (n, n))
    assert abs(Fo - F) <= 1e-9 * F
    x_ref, _ = oracle.run(A, y32.astype(np.float64), (n, n), M, N, lam, mu, k, K, row_unit=nb, col_unit=n)
    Fr, _, _ = oracle.objective(A, y32.astype(np.float64), x_ref, lam, (n, n))
    assert abs(Fr - F) <= 1e-3 * F


def test_checkpoint_resume(B):
    A, _, y, n, na, nb, M, N = _problem("ragged37")
    y32 = y.astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y32, 0.05)
        rec.run(10, 15)
        xs = np.empty(A.cols_n, np.float32)
        rs = np.empty(A.rows, np.float32)
        assert B.bsgdtv_get_state(rec.h, xs, rs) == 10
        rec.run(10, 15)
        straight = rec.x().copy()
        rec.set_data(y32, 0.05)              # reset, then resume from the checkpoint
        B.bsgdtv_set_state(rec.h, xs, rs, 10)
        rec.run(10, 15)
        resumed = rec.x().copy()
    assert rel(resumed, straight) <= 1e-6
    # r^{k-1} is part of the state (Eq. 3 uses x^{k-1}): resuming with r = y instead
    # gives another trajectory
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y32, 0.05)
        B.bsgdtv_set_state(rec.h, xs, y32, 10)
        rec.run(10, 15)
        wrong = rec.x().copy()
    assert rel(wrong, straight) > 1e-3


def test_errors_and_state(B):
    A, _, y, n, na, nb, M, N = _problem("ragged37")
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        with pytest.raises(B.BsgdtvError) as e:
            rec.run(1, 1)
        assert e.value.code == -4
        bad = y.astype(np.float32)
        bad[3] = np.nan
        with pytest.raises(B.BsgdtvError) as e:
            rec.set_data(bad, 0.1)
        assert e.value.code == -6
        with pytest.raises(B.BsgdtvError) as e:
            rec.set_data(torch.from_numpy(bad).cuda(), 0.1)
        assert e.value.code == -6
        rec.set_data(y.astype(np.float32), 0.1)
        mu, lam, u = rec.params()
        assert lam == 0.1 and u > 0 and abs(mu - 0.9 / (2 * u)) <= 1e-15 * mu
        before = B.bsgdtv_launch_count()
        rec.run(3, 8)
        torch.cuda.synchronize()
        assert B.bsgdtv_launch_count() - before == 3 * 3   # products, reduce/update, one FGP launch


@pytest.mark.parametrize("name", ["ellipse64", "ragged37", "wide130"])
def test_parallel_beam_handle_matches_csr_handle(B, name):
    """bsgdtv_create_parallel_beam builds A on the device for the geometry:
    same partition as a handle built from the FP64 generator's CSR with whole
    angles / image rows as units, block products within 1e-6 of it, epochs
    within 1e-5, and x within 1e-4 of the oracle."""
    A, _, y, n, na, nb, M, N = _problem(name)
    y32 = y.astype(np.float32)
    rng = np.random.default_rng(2)
    x = torch.tensor(rng.random(A.cols_n), dtype=torch.float32, device="cuda")
    r = torch.tensor(rng.standard_normal(A.rows), dtype=torch.float32, device="cuda")
    u, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u)
    out = []
    for src in (A, None):
        with B.Reconstructor(src, (n, n), M, N, row_unit=nb, col_unit=n,
                             parallel_beam=(na, nb)) as rec:
            part = rec.partition()
            info = rec.info()
            zb = torch.zeros(N * A.rows, device="cuda")
            gb = torch.zeros(M * A.cols_n, device="cuda")
            B.bsgdtv_block_products(rec.h, x, r, zb, gb)
            rec.set_data(y32, 0.05, mu)
            rec.run(10, 20)
            out.append((part, info, zb.cpu().numpy(), gb.cpu().numpy(), rec.x().copy()))
    (pc, ic, zc, gc, xc), (pg, ig, zg, gg, xg) = out
    assert all(np.array_equal(a, b) for a, b in zip(pc, pg))
    # the support may differ by weights below 1e-6 (rays grazing pixel corners;
    # test_gpu_matrix_free checks every weight against the FP64 generator)
    assert abs(ig["nnz"] - ic["nnz"]) <= 5e-3 * ic["nnz"]
    assert rel(zg, zc) <= 1e-6 and rel(gg, gc) <= 1e-6
    assert rel(xg, xc) <= 1e-5
    x_ref, _ = oracle.run(A, y32.astype(np.float64), (n, n), M, N, 0.05, mu, 10, 20,
                          row_unit=nb, col_unit=n)
    assert rel(xg, x_ref) <= 1e-4


def test_parallel_beam_handle_512(B):
    """The 512x512 geometry (360 x 727) generated on the device: 2 epochs in
    the bench's configuration within 1e-5 of the CSR-built handle."""
    wl = synth.WORKLOADS["ellipse512"]
    P = synth.make_problem(wl)
    y32 = P.y.astype(np.float32)
    mu = 0.9 / (2 * 1.8e5)
    xs = []
    for src in (P.A, None):
        with B.Reconstructor(src, (wl.n, wl.n), wl.M, wl.N, row_unit=wl.n_bins, col_unit=wl.n,
                             parallel_beam=(wl.n_angles, wl.n_bins)) as rec:
            rec.set_data(y32, wl.lam, mu)
            rec.run(2, wl.fgp_iters)
            xs.append(rec.x().copy())
    assert rel(xs[1], xs[0]) <= 1e-5
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_create_parallel_beam(0, 360, 727, 8, 8)
    assert e.value.code == -1


def test_host_y_is_read_before_set_data_returns(B):
    """A pinned host y may be overwritten as soon as set_data returns (the
    copy has read it by then), and a y with NaN leaves the handle without
    data, even after a successful set_data."""
    A, _, y, n, na, nb, M, N = _problem("wide130")
    y32 = y.astype(np.float32)
    pinned = torch.empty(A.rows, dtype=torch.float32).pin_memory()
    yp = pinned.numpy()
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y32, 0.05)
        rec.run(6, 10)
        x_ref = rec.x().copy()
        yp[:] = y32
        rec.set_data(yp, 0.05)
        yp[:] = np.nan                        # the caller reuses its buffer at once
        rec.run(6, 10)
        assert np.array_equal(rec.x(), x_ref)
        bad = y32.copy()
        bad[-1] = np.inf
        with pytest.raises(B.BsgdtvError) as e:
            rec.set_data(bad, 0.05)
        assert e.value.code == -6
        with pytest.raises(B.BsgdtvError) as e:
            rec.run(1, 10)                    # the rejected y left no data
        assert e.value.code == -4


def test_reconstruct_is_set_data_run_get_x(B):
    """bsgdtv_reconstruct (one call, one synchronisation) gives the iterates of
    set_data + run + get_x bit for bit, from host and from device buffers; a
    pinned y may be reused at once; non-finite y gives BSGDTV_ERR_NONFINITE
    and leaves no data; a short x_out is rejected."""
    A, _, y, n, na, nb, M, N = _problem("wide130")
    y32 = y.astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        u, _ = rec.estimate_umax(500, 1e-10)
        mu = 0.9 / (2 * u)
        rec.set_data(y32, 0.05, mu)
        rec.run(7, 10)
        x_ref = rec.x().copy()
        rec.run(2, 10)                         # move the state on, then start over
        pinned = torch.empty(A.rows, dtype=torch.float32).pin_memory()
        yp = pinned.numpy()
        yp[:] = y32
        out = np.full(A.cols_n + 3, -1.0, dtype=np.float32)
        rec.reconstruct(yp, 0.05, mu, 7, 10, out)
        yp[:] = np.nan
        assert np.array_equal(out[:A.cols_n], x_ref) and np.all(out[A.cols_n:] == -1.0)
        xd = rec.reconstruct(torch.from_numpy(y32).cuda(), 0.05, mu, 7, 10)
        assert np.array_equal(xd.cpu().numpy(), x_ref)
        xo = torch.full((A.cols_n,), -1.0, dtype=torch.float32).pin_memory().numpy()
        rec.reconstruct(y32, 0.05, mu, 7, 10, xo)      # pinned x out: written by a kernel
        assert np.array_equal(xo, x_ref)
        xg = torch.zeros(A.cols_n, dtype=torch.float32).pin_memory().numpy()
        assert np.array_equal(B.bsgdtv_get_x(rec.h, xg), x_ref)
        rec.run(3, 10)                         # the handle holds the data: run continues
        rec.set_data(y32, 0.05, mu)
        rec.run(10, 10)
        x10 = rec.x().copy()
        assert np.array_equal(rec.reconstruct(y32, 0.05, mu, 10, 10), x10)
        assert np.array_equal(rec.reconstruct(y32, 0.05, 0.0, 0, 10), np.zeros(A.cols_n, np.float32))
        bad = y32.copy()
        bad[5] = np.inf
        with pytest.raises(B.BsgdtvError) as e:
            rec.reconstruct(bad, 0.05, mu, 3, 10)
        assert e.value.code == -6
        with pytest.raises(B.BsgdtvError) as e:
            rec.run(1, 10)
        assert e.value.code == -4
        with pytest.raises(B.BsgdtvError) as e:
            rec.reconstruct(y32, 0.05, mu, 3, 10, np.empty(A.cols_n - 1, np.float32))
        assert e.value.code == -1


def test_ellipse512_full_size_epochs(B):
    """The 512x512 workload (360 angles x 727 bins, M = N = 8, lambda 0.02, 50 FGP
    iterations) in the launch configuration bench.py times: 3 epochs vs the oracle."""
    wl = synth.WORKLOADS["ellipse512"]
    P = synth.make_problem(wl)
    A = P.A
    y32 = P.y.astype(np.float32)
    with B.Reconstructor(A, (wl.n, wl.n), wl.M, wl.N, row_unit=wl.n_bins, col_unit=wl.n) as rec:
        u, _ = rec.estimate_umax(200, 1e-10)
        mu = 0.9 / (2 * u)
        rec.set_data(torch.from_numpy(y32).cuda(), wl.lam, mu)
        rec.run(3, wl.fgp_iters)
        x_gpu = rec.x().astype(np.float64)
    x_ref, _ = oracle.run(A, y32.astype(np.float64), (wl.n, wl.n), wl.M, wl.N, wl.lam, mu, 3,
                          wl.fgp_iters, row_unit=wl.n_bins, col_unit=wl.n)
    assert rel(x_gpu, x_ref) <= 1e-5


def test_run_timed_matches_run(B):
    A, _, y, n, na, nb, M, N = _problem("wide130")
    y32 = y.astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
        rec.set_data(y32, 0.05)
        rec.run(6, 12)
        x_plain = rec.x().copy()
        rec.set_data(y32, 0.05)
        pk, ep = B.bsgdtv_run_timed(rec.h, 6, 12)
        x_timed = rec.x().copy()
    assert 0 < pk < ep
    assert rel(x_timed, x_plain) <= 1e-6


def test_epochs_are_deterministic(B):
    """The A^T r tiles are exact integer sums, so repeated runs agree bit for bit."""
    A, _, y, n, na, nb, M, N = _problem("wide130")
    y32 = y.astype(np.float32)
    outs = []
    for _ in range(2):
        with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n) as rec:
            rec.set_data(y32, 0.05)
            rec.run(9, 13)
            outs.append(rec.x().copy())
    assert np.array_equal(outs[0], outs[1])


# ------------------------------------------------------------ stored formats
from _formats import stored_operator  # noqa: E402

FORMATS = {1: "f32_i16", 2: "f16_i16", 3: "bf16_i16"}


@pytest.mark.parametrize("fmt", [1, 2, 3])
@pytest.mark.parametrize("name", ["ellipse64", "ragged37"])
def test_block_products_formats(B, fmt, name):
    """Each stored format computes the block products of its own (rounded)
    operator to FP32 accuracy."""
    A, _, _, n, na, nb, M, N = _problem(name)
    As = stored_operator(A, fmt)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(A.cols_n).astype(np.float32)
    r = rng.standard_normal(A.rows).astype(np.float32)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n, fmt=fmt) as rec:
        zb = torch.zeros(N * A.rows, device="cuda")
        gb = torch.zeros(M * A.cols_n, device="cuda")
        B.bsgdtv_block_products(rec.h, torch.from_numpy(x).cuda(), torch.from_numpy(r).cuda(), zb, gb)
        zb = zb.cpu().numpy().reshape(N, A.rows)
        gb = gb.cpu().numpy().reshape(M, A.cols_n)
    rb, cb = oracle.partition(A.rows, A.cols_n, M, N, nb, n)
    z, gh = oracle.block_products(oracle.split_blocks(As, rb, cb), rb, cb, x.astype(np.float64),
                                  r.astype(np.float64))
    for i in range(M):
        for j in range(N):
            assert rel(zb[j, rb[i]:rb[i + 1]], z[i][j]) <= 1e-5
            assert rel(gb[i, cb[j]:cb[j + 1]], gh[i][j]) <= 1e-5


@pytest.mark.parametrize("fmt,bound", [(1, 1e-4), (2, 2e-3), (3, 2e-2)])
def test_full_reconstruction_formats(B, fmt, bound):
    """64x64 workload end to end per format: x matches the oracle run on the
    rounded operator to 1e-4; its distance to the oracle on the FP64 operator
    is the quantisation error (FP16 weights: <= 2e-3)."""
    wl = synth.WORKLOADS["ellipse64"]
    A, _, y, n, na, nb, M, N = _problem("ellipse64")
    As = stored_operator(A, fmt)
    u_ref, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u_ref)
    y32 = y.astype(np.float32).astype(np.float64)
    with B.Reconstructor(A, (n, n), M, N, row_unit=nb, col_unit=n, fmt=fmt) as rec:
        u, _ = rec.estimate_umax(5000, 1e-12)
        rec.set_data(y32.astype(np.float32), wl.lam, mu)
        rec.run(wl.epochs, wl.fgp_iters)
        x_gpu = rec.x().astype(np.float64)
    u_s, _ = oracle.power_iteration(As, 5000, 1e-12)
    assert abs(u - u_s) <= 1e-9 * u_s
    x_s, _ = oracle.run(As, y32, (n, n), M, N, wl.lam, mu, wl.epochs, wl.fgp_iters, row_unit=nb, col_unit=n)
    x_64, _ = oracle.run(A, y32, (n, n), M, N, wl.lam, mu, wl.epochs, wl.fgp_iters, row_unit=nb, col_unit=n)
    assert rel(x_gpu, x_s) <= 1e-4
    err = rel(x_gpu, x_64)
    print(f"format {FORMATS[fmt]}: x rel err vs FP64 operator {err:.3e}")
    assert err <= bound
