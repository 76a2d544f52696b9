"""The allocation-free TV prox entry point (bsgdtv_tv_prox_static).

It exists for callers that cannot allocate device memory when they call in
(a process whose device budget belongs to its own pool allocator, a loop
that cannot afford cudaMalloc's device-wide synchronisation, a runtime that
forbids plugin allocations).  It must give the same result as the allocating
entry point bsgdtv_tv_prox.  Two calls run back to back, with different sizes,
so that a second call sees the shared scratch exactly as the first left it.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle

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


def test_static_prox_matches_oracle_and_degenerate_paths(B):
    """One call straight against the FP64 oracle (a tiled 300x211 image with a
    large weight), the single-region path (<= 64x64, one launch) and the
    branch that copies b (tau <= 0 or zero iterations)."""
    for shape, tau, iters, seed in [((300, 211), 1.5, 37, 2), ((64, 64), 0.6, 19, 3), ((17, 45), 0.3, 8, 4)]:
        b = _image(shape, seed)
        out = torch.full_like(b, float("nan"))
        B.bsgdtv_tv_prox_static(b, out, tau, iters)
        ref = oracle.fgp(b.cpu().numpy().astype(np.float64), tau, iters)
        assert _rel(out, torch.from_numpy(ref).cuda()) <= 1e-5, shape
    b = _image((40, 33), 5)
    for tau, iters in [(0.0, 10), (-1.0, 10), (0.5, 0)]:
        out = torch.full_like(b, float("nan"))
        B.bsgdtv_tv_prox_static(b, out, tau, iters)
        assert torch.equal(out, b), (tau, iters)


class _DefaultPool:
    """High-water mark of the device's default stream-ordered memory pool
    (the pool cudaMallocAsync draws from), read through the driver API."""
    USED_MEM_HIGH = 8          # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self, device):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def high(self):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


def test_static_prox_allocates_nothing(B):
    """The defining property: after a first call (which may load the library's
    device code, array included), further calls change neither the device's
    free memory nor the default pool's high-water mark, while the allocating
    entry point does raise that mark (so the probe can see an allocation)."""
    b = _image((512, 512), 6)
    out = torch.empty_like(b)
    B.bsgdtv_tv_prox_static(b, out, 0.4, 30)
    torch.cuda.synchronize()
    pool = _DefaultPool(torch.cuda.current_device())
    pool.reset_high()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.bsgdtv_tv_prox_static(b, out, 0.4, 30)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert pool.high() == 0
    ref = torch.empty_like(b)
    B.bsgdtv_tv_prox(b, ref, 0.4, 30)
    assert pool.high() >= 8 * 512 * 512 * 4
    assert torch.equal(out, ref)


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
