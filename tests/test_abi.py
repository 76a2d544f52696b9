"""CPU tests of the C ABI library: it builds, loads, exports every symbol the
header declares, and its host-side bookkeeping (partition bounds, tiled
layout, input validation) is exact.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1812_01307_gb300 import build as build_mod
from paper_1812_01307_gb300 import synth

from _formats import bf16_round

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    build_mod.build_library()
    from paper_1812_01307_gb300 import bsgdtv
    bsgdtv.load()
    return bsgdtv


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bsgdtv_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(B):
    lib = ctypes.CDLL(build_mod.LIB)
    declared = _declared()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(B.exported_symbols())


def test_strerror_and_launch_count(B):
    assert B.bsgdtv_strerror(0) == "ok"
    assert B.bsgdtv_strerror(-6) == "non-finite input"
    assert B.bsgdtv_launch_count() >= 0


@pytest.mark.parametrize("units,M,unit", [(60, 4, 91), (360, 8, 727), (7, 3, 5), (10, 10, 1), (13, 1, 2)])
def test_partition_bounds_match_oracle(B, units, M, unit):
    rows = units * unit
    rb, cb = B.bsgdtv_partition_bounds(rows, 64 * 64, M, 4, unit, 64)
    rb_o, cb_o = oracle.partition(rows, 64 * 64, M, 4, unit, 64)
    assert np.array_equal(rb, rb_o) and np.array_equal(cb, cb_o)


@pytest.mark.parametrize("n,na,nb,M,N,target", [
    (64, 60, 91, 4, 4, 608),      # 64x64 workload: 16-row bands, sub-grouped rows
    (37, 11, 55, 3, 5, 608),      # ragged tiles and bands, rays missing the image
    (70, 9, 101, 9, 70, 100),     # one-row bands, one angle per block
    (8, 5, 13, 1, 1, 1),          # single block
    (130, 6, 185, 2, 3, 50),      # several tiles per band, ragged last tile
])
def test_layout_reassembles_A_exactly(B, n, na, nb, M, N, target):
    A = synth.parallel_beam_csr(n, na, nb)
    st = B.bsgdtv_layout_check(A.rows, A.cols_n, n, n, A.row_ptr, A.cols, A.vals, M, N, nb, n,
                               target_items=target)
    assert st["nnz"] == A.nnz
    # one segment per (row, tile) pair touched
    assert st["segments"] >= np.count_nonzero(np.diff(A.row_ptr))


def test_layout_with_explicit_bounds_and_random_csr(B):
    rng = np.random.default_rng(0)
    h, w = 23, 70
    rows, cols = 57, h * w
    dense = (rng.random((rows, cols)) < 0.05) * rng.standard_normal((rows, cols))
    dense[5] = 0.0                        # empty row
    import scipy.sparse as sp
    S = sp.csr_matrix(dense)
    S.sort_indices()
    rb = np.array([0, 10, 10, 40, 57])    # an empty row block
    cb = np.array([0, 3, 11, 23]) * w
    st = B.bsgdtv_layout_check(rows, cols, h, w, S.indptr.astype(np.int64), S.indices, S.data,
                               4, 3, row_bounds=rb, col_bounds=cb)
    assert st["nnz"] == S.nnz


def _tiny_csr():
    A = synth.parallel_beam_csr(8, 4, 13)
    return A.row_ptr.copy(), A.cols.copy(), A.vals.copy(), A.rows


def test_rejects_unsorted_or_out_of_range_columns(B):
    rp, ci, v, rows = _tiny_csr()
    r = int(np.argmax(np.diff(rp) > 2))
    bad = ci.copy()
    bad[rp[r]], bad[rp[r] + 1] = bad[rp[r] + 1], bad[rp[r]]
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_layout_check(rows, 64, 8, 8, rp, bad, v, 2, 2, 13, 8)
    assert e.value.code == -1
    bad = ci.copy()
    bad[3] = 64
    with pytest.raises(B.BsgdtvError):
        B.bsgdtv_layout_check(rows, 64, 8, 8, rp, bad, v, 2, 2, 13, 8)


def test_rejects_nonfinite_values_and_bad_bounds(B):
    rp, ci, v, rows = _tiny_csr()
    bad = v.copy()
    bad[7] = np.nan
    with pytest.raises(B.BsgdtvError) as e:
        B.bsgdtv_layout_check(rows, 64, 8, 8, rp, ci, bad, 2, 2, 13, 8)
    assert e.value.code == -6
    with pytest.raises(B.BsgdtvError):     # column bands must be whole image rows
        B.bsgdtv_layout_check(rows, 64, 8, 8, rp, ci, v, 2, 2, 13, 8,
                              col_bounds=np.array([0, 20, 64]))
    with pytest.raises(B.BsgdtvError):     # cols != img_h * img_w
        B.bsgdtv_layout_check(rows, 64, 8, 9, rp, ci, v, 2, 2, 13, 8)
    with pytest.raises(B.BsgdtvError):     # more column blocks than image rows
        B.bsgdtv_partition_bounds(rows, 64, 2, 9, 13, 8)


def test_stored_weight_rounding_matches_numpy(B):
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.uniform(0, 1.5, 4000), 10.0 ** rng.uniform(-12, 0.2, 4000),
                           [0.0, 1.0, 1.4142135623730951, 6.1e-5, 5.96e-8, 3e-8, 65504.0, 70000.0,
                            1 + 2 ** -11, 1 + 3 * 2 ** -11, 1 + 2 ** -8, 1 + 3 * 2 ** -8]])
    f32 = np.array([B.bsgdtv_stored_weight(v, B.FMT_F32_I32) for v in vals])
    f16 = np.array([B.bsgdtv_stored_weight(v, B.FMT_F16_I16) for v in vals])
    b16 = np.array([B.bsgdtv_stored_weight(v, B.FMT_BF16_I16) for v in vals])
    assert np.array_equal(f32, vals.astype(np.float32).astype(np.float64))
    with np.errstate(over="ignore"):
        ref16 = vals.astype(np.float16).astype(np.float64)
    assert np.array_equal(f16, ref16)
    assert np.array_equal(b16, bf16_round(vals))


@pytest.mark.parametrize("fmt", [1, 2, 3])
def test_layout_reassembles_in_every_format(B, fmt):
    A = synth.parallel_beam_csr(37, 11, 55)
    st = B.bsgdtv_layout_check(A.rows, A.cols_n, 37, 37, A.row_ptr, A.cols, A.vals, 3, 5, 55, 37,
                               fmt=fmt)
    assert st["nnz"] == A.nnz


def test_batch_device_bytes(B):
    """Host-only size of a batch: grows with slices and with the weight width,
    rejects bad sizes."""
    A = synth.parallel_beam_csr(64, 60, 91)
    f32 = [B.bsgdtv_batch_device_bytes(A.rows, A.cols_n, A.nnz, s) for s in (1, 4, 32, 33, 64, 129)]
    assert all(a <= b for a, b in zip(f32, f32[1:]))
    assert f32[0] > 2 * 8 * A.nnz                       # A twice, 8 bytes per nonzero
    f16 = B.bsgdtv_batch_device_bytes(A.rows, A.cols_n, A.nnz, 4, B.FMT_F16_I16)
    assert f32[1] - f16 == 2 * 2 * A.nnz                # 6 instead of 8 bytes, twice
    assert B.bsgdtv_batch_device_bytes(0, 10, 5, 1) == -1
    assert B.bsgdtv_batch_device_bytes(10, 10, 5, 0) == -1
