"""The TV prox's tiling of an image dimension (host only, through the C ABI).

The prox runs several FGP iterations per launch on 64-pixel regions that
overlap by a halo of (iterations + 1) pixels; only a region's interior is
exact after the launch, because a pixel's value after c iterations depends on
the pixels within c + 1 of it.  These tests check, for many lengths and halos,
the placement the kernel computes (bsgdtv_fgp_tiling runs the same code):

* the interiors tile [0, len) exactly, in order;
* every region lies inside [0, len) on its first pixel and inside its 64 pixels;
* an interior pixel is at least `halo` pixels from any region edge that lies
  inside the image (an edge at the image border needs none: outside the image
  every iterate is zero, which the region reproduces);
* no tiling with fewer regions of the same kind exists (the count is minimal).
"""
import pytest

from paper_1812_01307_gb300 import bsgdtv as B

R = 64


@pytest.fixture(scope="module")
def lib():
    from paper_1812_01307_gb300 import build
    build.build_library()
    B.load()
    return B


LENGTHS = list(range(1, 300)) + [511, 512, 513, 700, 1023, 1024, 1025, 2048, 2897, 4096]


@pytest.mark.parametrize("halo", [1, 2, 5, 6, 7, 9, 10, 11, 13, 16, 31])
def test_interiors_tile_with_full_halos(lib, halo):
    for n in LENGTHS:
        regs = lib.bsgdtv_fgp_tiling(n, halo)
        pos = 0
        for first, lo, hi in regs:
            assert first >= 0 and 0 <= lo < hi <= R, (n, halo, first, lo, hi)
            assert first + lo == pos, (n, halo, "interiors must be contiguous")
            if first > 0:
                assert lo >= halo, (n, halo, first, lo)
            if first + R < n:
                assert hi <= R - halo, (n, halo, first, hi)
            pos = first + hi
        assert pos == n, (n, halo, pos)
        # minimal: edge regions hold at most R - halo interior pixels, the
        # others R - 2 halo
        k = len(regs)
        if n <= R:
            assert k == 1
        else:
            assert 2 * (R - halo) + (k - 2) * (R - 2 * halo) >= n
            assert k == 2 or 2 * (R - halo) + (k - 3) * (R - 2 * halo) < n


def test_counts_of_the_workloads(lib):
    """512 x 512 at 10 iterations per launch (halo 11) takes 12 regions per
    dimension (144 CTAs, one wave on 152 SMs); at 6 iterations (halo 7) 10
    (100 per slice in the batch); 128 x 128 takes 3 up to 15 iterations."""
    assert len(lib.bsgdtv_fgp_tiling(512, 11)) == 12
    assert len(lib.bsgdtv_fgp_tiling(512, 12)) == 13
    assert len(lib.bsgdtv_fgp_tiling(512, 7)) == 10
    assert len(lib.bsgdtv_fgp_tiling(128, 16)) == 3
    assert len(lib.bsgdtv_fgp_tiling(64, 9)) == 1


def test_rejects_bad_arguments(lib):
    for n, h in ((0, 5), (100, 0), (100, 32), (100, -1)):
        with pytest.raises(lib.BsgdtvError):
            lib.bsgdtv_fgp_tiling(n, h)
