"""The allocation-free TV prox entry point (bsgdtv_tv_prox_static).

It exists for callers that cannot allocate device memory when they call in
(a process whose device budget belongs to its own pool allocator, a loop
that cannot afford cudaMalloc's device-wide synchronisation, a runtime that
forbids plugin allocations).  It must give the same result as the allocating
entry point bsgdtv_tv_prox.  Two calls run back to back, with different sizes,
so that a second call sees the shared scratch exactly as the first left it.

This file is named to be collected last.
"""
import numpy as np
import pytest

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


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _image(shape, seed):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(shape) + (np.arange(shape[0])[:, None] > shape[0] // 3)
    return torch.from_numpy(b.astype(np.float32)).cuda()


def test_static_prox_matches_allocating_prox_two_calls(B):
    # first call: the largest accepted image, several launches that pass the
    # dual fields through the scratch; second call: a smaller ragged image
    for shape, tau, iters, seed in [((512, 512), 0.4, 50, 0), ((100, 77), 0.7, 23, 1)]:
        b = _image(shape, seed)
        ref = torch.empty_like(b)
        B.bsgdtv_tv_prox(b, ref, tau, iters)
        out = torch.full_like(b, float("nan"))
        B.bsgdtv_tv_prox_static(b, out, tau, iters)
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= 1e-5


def test_static_prox_rejects_oversize(B):
    b = torch.zeros((513, 512), device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_tv_prox_static(b, x, 0.1, 5)
    assert e.value.code == -1
    b = torch.zeros((8, 8), device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_tv_prox_static(b, x, 0.1, 4097)
    assert e.value.code == -1
