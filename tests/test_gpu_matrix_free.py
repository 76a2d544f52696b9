"""GPU tests of the matrix-free parallel-beam projector: its weights against
the FP64 CSR generator (<= 1e-6 absolute per weight, same support up to
weights below 1e-6), its products and reconstructions against the stored-
matrix batch (<= 1e-5) and the FP64 oracle (<= 1e-4), and its u_max
against the oracle's power iteration."""
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


def _compare_rays(B, n, na, nb, rays):
    A = synth.parallel_beam_csr(n, na, nb)
    got = B.bsgdtv_mf_ray_weights(n, na, nb, rays)
    worst = 0.0
    for r, (c, v) in zip(rays, got):
        lo, hi = A.row_ptr[r], A.row_ptr[r + 1]
        ref = dict(zip(A.cols[lo:hi].tolist(), A.vals[lo:hi].tolist()))
        mine = {}
        for cc, vv in zip(c.tolist(), v.tolist()):
            assert cc not in mine, (r, cc)          # each pixel once per ray
            mine[cc] = vv
        for k in set(ref) | set(mine):
            d = abs(ref.get(k, 0.0) - mine.get(k, 0.0))
            worst = max(worst, d)
            assert d <= 1e-6, (r, k, ref.get(k), mine.get(k))
    return worst


@pytest.mark.parametrize("n,na,nb", [(64, 60, 91), (37, 11, 55), (16, 8, 23), (9, 4, 17)])
def test_mf_weights_equal_generator_small(B, n, na, nb):
    """Every ray of small geometries, even and odd n (half-integer pixel
    corners), axis-parallel rays on grid lines, rays that miss the image."""
    _compare_rays(B, n, na, nb, np.arange(na * nb))


def test_mf_weights_equal_generator_512(B):
    """The 512x512 geometry (360 angles x 727 bins): 4000 sampled rays plus every
    ray of the angles 0 and pi/2 and of the first and last bins."""
    n, na, nb = 512, 360, 727
    rng = np.random.default_rng(3)
    rays = np.unique(np.concatenate([rng.integers(0, na * nb, 4000), np.arange(nb),
                                     180 * nb + np.arange(nb), np.arange(na) * nb,
                                     np.arange(na) * nb + nb - 1]))
    worst = _compare_rays(B, n, na, nb, rays)
    print(f"largest weight difference {worst:.2e}")


GEOM = {"g64": (64, 60, 91, 10), "g37": (37, 11, 55, 4)}


@pytest.mark.parametrize("name,slices,lam", [("g64", 5, 0.05), ("g37", 3, 0.02), ("g64", 70, 0.0)])
def test_mf_batch_matches_stored_batch_and_oracle(B, name, slices, lam):
    n, na, nb, ne = GEOM[name]
    A = synth.parallel_beam_csr(n, na, nb)
    _, Y = synth.slice_stack(A, n, ne, slices, seed=11)
    Y = Y.astype(np.float32)
    u, _ = oracle.power_iteration(A)
    mu = 0.9 / (2 * u)
    lams = np.full(slices, lam)
    epochs, K = 12, 15
    with B.BatchReconstructor(A, (n, n), slices) as st:
        st.set_data(Y, lams, mu)
        st.run(epochs, K)
        Xs = st.x()
    with B.BatchReconstructor(None, (n, n), slices, parallel_beam=(na, nb)) as mf:
        mf.set_data(Y, lams, mu)
        mf.run(epochs, K)
        Xm = mf.x()
    for b in range(slices):
        assert rel(Xm[b], Xs[b]) <= 1e-5, b
    for b in (0, slices - 1):
        x_ref, _ = oracle.run(A, Y[b].astype(np.float64), (n, n), 1, 1, lam, mu, epochs, K)
        assert rel(Xm[b], x_ref) <= 1e-4


def test_mf_umax_matches_oracle(B):
    n, na, nb, _ = GEOM["g64"]
    A = synth.parallel_beam_csr(n, na, nb)
    u_ref, _ = oracle.power_iteration(A, 5000, 1e-12)
    with B.BatchReconstructor(None, (n, n), 4, parallel_beam=(na, nb)) as mf:
        u, it = mf.estimate_umax(5000, 1e-10)
        with pytest.raises(B.BsgdtvError) as e:   # state consumed: set_data first
            mf.run(1, 5)
        assert e.value.code == -4
    assert abs(u - u_ref) <= 1e-5 * u_ref, (u, u_ref, it)
    with B.BatchReconstructor(A, (n, n), 4) as st:
        u2, _ = st.estimate_umax(5000, 1e-10)
    assert abs(u2 - u_ref) <= 1e-5 * u_ref


def test_mf_512_sampled_slices(B):
    """The 512x512 geometry with 4 slices for 3 epochs: matrix-free vs stored."""
    wl = synth.WORKLOADS["ellipse512"]
    A = synth.make_problem(wl).A
    _, Y = synth.slice_stack(A, wl.n, wl.n_ellipses, 4, seed=5)
    Y = Y.astype(np.float32)
    mu, lam = 0.9 / (2 * 1.8e5), np.full(4, wl.lam)
    with B.BatchReconstructor(A, (wl.n, wl.n), 4) as st:
        st.set_data(Y, lam, mu)
        st.run(3, wl.fgp_iters)
        Xs = st.x()
    with B.BatchReconstructor(None, (wl.n, wl.n), 4, parallel_beam=(wl.n_angles, wl.n_bins)) as mf:
        mf.set_data(Y, lam, mu)
        mf.run(3, wl.fgp_iters)
        Xm = mf.x()
    for b in range(4):
        assert rel(Xm[b], Xs[b]) <= 1e-5, b


def test_project_matches_csr_products(B):
    """bsgdtv_batch_project: y = A x per slice, matrix free and stored, vs the
    FP64 CSR product."""
    n, na, nb, ne = GEOM["g37"]
    A = synth.parallel_beam_csr(n, na, nb)
    X = np.stack([synth.phantom(n, ne, s).ravel() for s in range(3)])
    ref = (A.to_scipy() @ X.T).T
    xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    with B.BatchReconstructor(None, (n, n), 3, parallel_beam=(na, nb)) as mf:
        ym = mf.project(xt).cpu().numpy()
    with B.BatchReconstructor(A, (n, n), 3) as st:
        ys = st.project(xt).cpu().numpy()
    for b in range(3):
        assert rel(ym[b], ref[b]) <= 1e-6 and rel(ys[b], ref[b]) <= 1e-6
