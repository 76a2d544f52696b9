"""Python binding of the BSGD-TV C ABI (``include/bsgdtv.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libbsgdtv.so``.  The functions carry the C names.  Device buffers
are passed as CUDA ``torch.Tensor`` objects (PyTorch supplies device memory
and the stream); host buffers as numpy arrays.  There is no fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

_lib = None


class BsgdtvError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def load(path: str | None = None):
    """Loads libbsgdtv.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"BSGD-TV CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "bsgdtv_create_csr": (I32, [ctypes.POINTER(P), I64, I64, I32, I32, P, P, P, I32, I32, I64, I64, P, P, P]),
        "bsgdtv_create_csr_ex": (I32, [ctypes.POINTER(P), I64, I64, I32, I32, P, P, P, I32, I32, I64, I64, P, P, I32, P]),
        "bsgdtv_create_parallel_beam": (I32, [ctypes.POINTER(P), I32, I32, I32, I32, I32, I32, P]),
        "bsgdtv_stored_weight": (ctypes.c_float, [D, I32]),
        "bsgdtv_destroy": (None, [P]),
        "bsgdtv_get_partition": (I32, [P, P, P]),
        "bsgdtv_set_data": (I32, [P, P, I32, D, D]),
        "bsgdtv_estimate_umax": (I32, [P, I32, D, ctypes.POINTER(D), ctypes.POINTER(I32)]),
        "bsgdtv_get_params": (I32, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "bsgdtv_run": (I32, [P, I32, I32]),
        "bsgdtv_run_timed": (I32, [P, I32, I32, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "bsgdtv_run_subsets": (I32, [P, I32, I32, P, P]),
        "bsgdtv_run_subsets_timed": (I32, [P, I32, I32, P, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "bsgdtv_fp32_fma_peak": (I32, [ctypes.POINTER(D), ctypes.POINTER(D)]),
        "bsgdtv_run_until": (I32, [P, I32, I32, I32, D, ctypes.POINTER(I32), ctypes.POINTER(D)]),
        "bsgdtv_get_x": (I32, [P, P, I32, I64]),
        "bsgdtv_reconstruct": (I32, [P, P, I32, D, D, I32, I32, P, I32, I64]),
        "bsgdtv_get_state": (I32, [P, P, P, ctypes.POINTER(I64), I32]),
        "bsgdtv_set_state": (I32, [P, P, P, I64, I32]),
        "bsgdtv_objective": (I32, [P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "bsgdtv_block_products": (I32, [P, P, P, P, P]),
        "bsgdtv_get_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "bsgdtv_tv_prox": (I32, [P, P, I32, I32, D, I32, P]),
        "bsgdtv_tv_prox_static": (I32, [P, P, I32, I32, D, I32, P]),
        "bsgdtv_partition_bounds": (I32, [I64, I64, I32, I32, I64, I64, P, P]),
        "bsgdtv_fgp_tiling": (I32, [I32, I32, I32, P, P, P, P]),
        "bsgdtv_layout_check": (I32, [I64, I64, I32, I32, P, P, P, I32, I32, I64, I64, P, P, I32, I32, P]),
        "bsgdtv_batch_create_csr": (I32, [ctypes.POINTER(P), I64, I64, I32, I32, P, P, P, I32, P]),
        "bsgdtv_batch_create_csr_ex": (I32, [ctypes.POINTER(P), I64, I64, I32, I32, P, P, P, I32, I32, P]),
        "bsgdtv_batch_set_slice": (I32, [P, I32, P, I32, D]),
        "bsgdtv_batch_get_slice_x": (I32, [P, I32, P, I32]),
        "bsgdtv_batch_destroy": (None, [P]),
        "bsgdtv_batch_set_data": (I32, [P, P, I32, P, D]),
        "bsgdtv_batch_run": (I32, [P, I32, I32]),
        "bsgdtv_batch_run_timed": (I32, [P, I32, I32, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "bsgdtv_batch_get_x": (I32, [P, P, I32]),
        "bsgdtv_batch_device_bytes": (I64, [I64, I64, I64, I32, I32]),
        "bsgdtv_operator_create_csr": (I32, [ctypes.POINTER(P), I64, I64, I32, I32, P, P, P, I32, P]),
        "bsgdtv_operator_destroy": (None, [P]),
        "bsgdtv_batch_create_from_operator": (I32, [ctypes.POINTER(P), P, I32, P]),
        "bsgdtv_batch_create_parallel_beam": (I32, [ctypes.POINTER(P), I32, I32, I32, I32, P]),
        "bsgdtv_mf_ray_weights": (I32, [I32, I32, I32, P, I32, I32, P, P, P]),
        "bsgdtv_batch_estimate_umax": (I32, [P, I32, D, ctypes.POINTER(D), ctypes.POINTER(I32)]),
        "bsgdtv_batch_project": (I32, [P, P, P]),
        "bsgdtv_batch_autotune": (I32, [P, I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(D)]),
        "bsgdtv_batch_set_tuning": (I32, [P, I32, I32]),
        "bsgdtv_batch_get_tuning": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "bsgdtv_batch_set_pass_lanes": (I32, [P, I32, I32]),
        "bsgdtv_packed_create": (I32, [ctypes.POINTER(P), P, I32, I32, P]),
        "bsgdtv_packed_set_part": (I32, [P, I32, P, I32, P, D]),
        "bsgdtv_packed_run": (I32, [P, I32, I32]),
        "bsgdtv_packed_get_x": (I32, [P, I32, P, I32]),
        "bsgdtv_packed_launches_per_epoch": (I32, [P, I32, ctypes.POINTER(I64)]),
        "bsgdtv_packed_destroy": (None, [P]),
        "bsgdtv_server_create": (I32, [ctypes.POINTER(P), I64, I32, I32]),
        "bsgdtv_server_destroy": (None, [P]),
        "bsgdtv_server_add_geometry": (I32, [P, I64, I64, I32, I32, P, P, P, I32, I32, D, I32, ctypes.POINTER(I32)]),
        "bsgdtv_server_submit": (I32, [P, I32, P, D, I32, ctypes.POINTER(I64)]),
        "bsgdtv_server_poll": (I32, [P, I64, ctypes.POINTER(I32)]),
        "bsgdtv_server_cancel": (I32, [P, I64]),
        "bsgdtv_server_wait": (I32, [P, I64, D, P, P]),
        "bsgdtv_server_stats": (I32, [P, P]),
        "bsgdtv_server_arm": (I32, [P, I32, D]),
        "bsgdtv_server_set_packing": (I32, [P, I32, D]),
        "bsgdtv_server_set_priority": (I32, [P, I32]),
        "bsgdtv_server_hold": (I32, [P, I32]),
        "bsgdtv_launch_count": (I64, []),
        "bsgdtv_last_error": (ctypes.c_char_p, []),
        "bsgdtv_strerror": (ctypes.c_char_p, [I32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return ["bsgdtv_create_csr", "bsgdtv_create_csr_ex", "bsgdtv_create_parallel_beam", "bsgdtv_stored_weight", "bsgdtv_destroy", "bsgdtv_get_partition", "bsgdtv_set_data",
            "bsgdtv_estimate_umax", "bsgdtv_get_params", "bsgdtv_run", "bsgdtv_run_timed",
            "bsgdtv_run_until", "bsgdtv_get_x", "bsgdtv_reconstruct",
            "bsgdtv_get_state", "bsgdtv_set_state", "bsgdtv_objective", "bsgdtv_block_products",
            "bsgdtv_get_info", "bsgdtv_tv_prox", "bsgdtv_tv_prox_static", "bsgdtv_partition_bounds",
            "bsgdtv_fgp_tiling",
            "bsgdtv_layout_check", "bsgdtv_run_subsets", "bsgdtv_run_subsets_timed",
            "bsgdtv_fp32_fma_peak", "bsgdtv_batch_create_csr", "bsgdtv_batch_destroy",
            "bsgdtv_batch_set_data", "bsgdtv_batch_run", "bsgdtv_batch_run_timed",
            "bsgdtv_batch_get_x", "bsgdtv_batch_create_csr_ex", "bsgdtv_batch_set_slice",
            "bsgdtv_batch_get_slice_x", "bsgdtv_batch_device_bytes", "bsgdtv_server_create",
            "bsgdtv_server_destroy", "bsgdtv_server_add_geometry", "bsgdtv_server_submit",
            "bsgdtv_server_poll", "bsgdtv_server_cancel", "bsgdtv_server_wait", "bsgdtv_server_stats",
            "bsgdtv_server_arm", "bsgdtv_server_set_packing", "bsgdtv_server_set_priority",
            "bsgdtv_server_hold",
            "bsgdtv_batch_create_parallel_beam", "bsgdtv_mf_ray_weights", "bsgdtv_batch_estimate_umax",
            "bsgdtv_batch_project", "bsgdtv_batch_autotune", "bsgdtv_batch_set_tuning",
            "bsgdtv_batch_get_tuning", "bsgdtv_batch_set_pass_lanes", "bsgdtv_operator_create_csr",
            "bsgdtv_operator_destroy", "bsgdtv_batch_create_from_operator",
            "bsgdtv_packed_create", "bsgdtv_packed_set_part", "bsgdtv_packed_run",
            "bsgdtv_packed_get_x", "bsgdtv_packed_launches_per_epoch", "bsgdtv_packed_destroy",
            "bsgdtv_launch_count", "bsgdtv_last_error", "bsgdtv_strerror"]


def _check(rc: int, where: str):
    if rc != 0:
        lib = load()
        msg = lib.bsgdtv_last_error().decode() or lib.bsgdtv_strerror(rc).decode()
        raise BsgdtvError(rc, where, msg)


def _dev_ptr(t, dtype=None, numel=None):
    """Pointer of a contiguous CUDA tensor (checked)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch.Tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype, numel=None):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    if numel is not None and a.size != numel:
        raise ValueError(f"expected {numel} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data)


def _is_tensor(a) -> bool:
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:
        return False


def current_stream():
    """cudaStream_t of torch's current stream (None if CUDA is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


FMT_F32_I32, FMT_F32_I16, FMT_F16_I16, FMT_BF16_I16 = 0, 1, 2, 3
FORMATS = {"f32_i32": FMT_F32_I32, "f32_i16": FMT_F32_I16, "f16_i16": FMT_F16_I16,
           "bf16_i16": FMT_BF16_I16}


# ------------------------------------------------------------------ C names
def bsgdtv_create_csr(rows, cols, img_h, img_w, row_ptr, col_idx, vals, M, N, row_unit=1,
                      col_unit=1, row_bounds=None, col_bounds=None, stream=None, fmt=FMT_F32_I32):
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    if row_ptr.size != rows + 1:
        raise ValueError("row_ptr must have rows+1 entries")
    rb = None if row_bounds is None else np.ascontiguousarray(row_bounds, dtype=np.int64)
    cb = None if col_bounds is None else np.ascontiguousarray(col_bounds, dtype=np.int64)
    h = ctypes.c_void_p()
    rc = lib.bsgdtv_create_csr_ex(ctypes.byref(h), int(rows), int(cols), int(img_h), int(img_w),
                                  _host_ptr(row_ptr, np.int64), _host_ptr(col_idx, np.int32),
                                  _host_ptr(vals, np.float64), int(M), int(N), int(row_unit),
                                  int(col_unit), None if rb is None else _host_ptr(rb, np.int64),
                                  None if cb is None else _host_ptr(cb, np.int64), int(fmt),
                                  stream if stream is not None else current_stream())
    _check(rc, "bsgdtv_create_csr_ex")
    return h


def bsgdtv_create_parallel_beam(n, n_angles, n_bins, M, N, stream=None, fmt=FMT_F32_I32):
    h = ctypes.c_void_p()
    _check(load().bsgdtv_create_parallel_beam(ctypes.byref(h), int(n), int(n_angles), int(n_bins),
                                              int(M), int(N), int(fmt),
                                              stream if stream is not None else current_stream()),
           "bsgdtv_create_parallel_beam")
    return h


def bsgdtv_stored_weight(v, fmt):
    """Host only: the weight as a handle of format `fmt` stores it (as FP32)."""
    return float(load().bsgdtv_stored_weight(float(v), int(fmt)))


def bsgdtv_destroy(h):
    load().bsgdtv_destroy(h)


def bsgdtv_get_partition(h, M, N):
    rb = np.zeros(M + 1, dtype=np.int64)
    cb = np.zeros(N + 1, dtype=np.int64)
    _check(load().bsgdtv_get_partition(h, _host_ptr(rb, np.int64), _host_ptr(cb, np.int64)),
           "bsgdtv_get_partition")
    return rb, cb


def bsgdtv_set_data(h, y, lam, mu=0.0):
    lib = load()
    if _is_tensor(y):
        import torch
        rc = lib.bsgdtv_set_data(h, _dev_ptr(y, torch.float32), 1, float(lam), float(mu))
    else:
        y = np.ascontiguousarray(y, dtype=np.float32)
        rc = lib.bsgdtv_set_data(h, _host_ptr(y, np.float32), 0, float(lam), float(mu))
    _check(rc, "bsgdtv_set_data")


def bsgdtv_estimate_umax(h, max_iters=5000, rel_tol=1e-12):
    u = ctypes.c_double()
    it = ctypes.c_int()
    _check(load().bsgdtv_estimate_umax(h, int(max_iters), float(rel_tol), ctypes.byref(u),
                                       ctypes.byref(it)), "bsgdtv_estimate_umax")
    return u.value, it.value


def bsgdtv_run_until(h, max_epochs, fgp_iters, check_every=10, rel_tol=1e-6):
    done = ctypes.c_int()
    f = ctypes.c_double()
    _check(load().bsgdtv_run_until(h, int(max_epochs), int(fgp_iters), int(check_every),
                                   float(rel_tol), ctypes.byref(done), ctypes.byref(f)),
           "bsgdtv_run_until")
    return done.value, f.value


def bsgdtv_get_params(h):
    mu, lam, u = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().bsgdtv_get_params(h, ctypes.byref(mu), ctypes.byref(lam), ctypes.byref(u)),
           "bsgdtv_get_params")
    return mu.value, lam.value, u.value


def bsgdtv_run(h, epochs, fgp_iters):
    _check(load().bsgdtv_run(h, int(epochs), int(fgp_iters)), "bsgdtv_run")


def bsgdtv_run_timed(h, epochs, fgp_iters):
    """Runs epochs and returns (sum of product-kernel ms, sum of epoch ms)."""
    pk, ep = ctypes.c_double(), ctypes.c_double()
    _check(load().bsgdtv_run_timed(h, int(epochs), int(fgp_iters), ctypes.byref(pk),
                                   ctypes.byref(ep)), "bsgdtv_run_timed")
    return pk.value, ep.value


def bsgdtv_run_subsets(h, row_sel, col_sel, fgp_iters):
    """Stochastic iterations: boolean masks row_sel [iters, M], col_sel [iters, N]."""
    rs = np.ascontiguousarray(row_sel, dtype=np.uint8)
    cs = np.ascontiguousarray(col_sel, dtype=np.uint8)
    if rs.ndim != 2 or cs.ndim != 2 or rs.shape[0] != cs.shape[0]:
        raise ValueError("row_sel [iters, M] and col_sel [iters, N] with the same iters")
    _check(load().bsgdtv_run_subsets(h, int(rs.shape[0]), int(fgp_iters), _host_ptr(rs, np.uint8),
                                     _host_ptr(cs, np.uint8)), "bsgdtv_run_subsets")


def bsgdtv_run_subsets_timed(h, row_sel, col_sel, fgp_iters):
    """bsgdtv_run_subsets returning (device ms of the iterations' kernels,
    host ms spent building and uploading the work-item lists)."""
    rs = np.ascontiguousarray(row_sel, dtype=np.uint8)
    cs = np.ascontiguousarray(col_sel, dtype=np.uint8)
    if rs.ndim != 2 or cs.ndim != 2 or rs.shape[0] != cs.shape[0]:
        raise ValueError("row_sel [iters, M] and col_sel [iters, N] with the same iters")
    dev, prep = ctypes.c_double(), ctypes.c_double()
    _check(load().bsgdtv_run_subsets_timed(h, int(rs.shape[0]), int(fgp_iters), _host_ptr(rs, np.uint8),
                                           _host_ptr(cs, np.uint8), ctypes.byref(dev), ctypes.byref(prep)),
           "bsgdtv_run_subsets_timed")
    return dev.value, prep.value


def bsgdtv_fp32_fma_peak():
    """Measured FP32 FMA throughput of the current device: (scalar, packed) TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().bsgdtv_fp32_fma_peak(ctypes.byref(a), ctypes.byref(b)), "bsgdtv_fp32_fma_peak")
    return a.value, b.value


def bsgdtv_get_info(h):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load().bsgdtv_get_info(h, *[ctypes.byref(a) for a in v]), "bsgdtv_get_info")
    return {"nnz": v[0].value, "segments": v[1].value, "work_items": v[2].value,
            "min_bytes_per_pass": v[3].value}


def bsgdtv_get_x(h, out):
    """Copies x into `out` (CUDA float32 tensor or float32 numpy array)."""
    lib = load()
    if _is_tensor(out):
        import torch
        rc = lib.bsgdtv_get_x(h, _dev_ptr(out, torch.float32), 1, int(out.numel()))
    else:
        rc = lib.bsgdtv_get_x(h, _host_ptr(out, np.float32), 0, int(out.size))
    _check(rc, "bsgdtv_get_x")
    return out


def bsgdtv_reconstruct(h, y, lam, mu, epochs, fgp_iters, out):
    """set_data + run + get_x in one call with one synchronisation; y and
    out are both CUDA float32 tensors or both float32 numpy arrays."""
    lib = load()
    if _is_tensor(y) != _is_tensor(out):
        raise TypeError("y and out must both be CUDA tensors or both numpy arrays")
    if _is_tensor(y):
        import torch
        rc = lib.bsgdtv_reconstruct(h, _dev_ptr(y, torch.float32), 1, float(lam), float(mu), int(epochs),
                                    int(fgp_iters), _dev_ptr(out, torch.float32), 1, int(out.numel()))
    else:
        y = np.ascontiguousarray(y, dtype=np.float32)
        rc = lib.bsgdtv_reconstruct(h, _host_ptr(y, np.float32), 0, float(lam), float(mu), int(epochs),
                                    int(fgp_iters), _host_ptr(out, np.float32), 0, int(out.size))
    _check(rc, "bsgdtv_reconstruct")
    return out


def bsgdtv_get_state(h, x, r):
    lib = load()
    ep = ctypes.c_int64()
    if _is_tensor(x):
        import torch
        rc = lib.bsgdtv_get_state(h, _dev_ptr(x, torch.float32), _dev_ptr(r, torch.float32),
                                  ctypes.byref(ep), 1)
    else:
        rc = lib.bsgdtv_get_state(h, _host_ptr(x, np.float32), _host_ptr(r, np.float32),
                                  ctypes.byref(ep), 0)
    _check(rc, "bsgdtv_get_state")
    return ep.value


def bsgdtv_set_state(h, x, r, epoch):
    lib = load()
    if _is_tensor(x):
        import torch
        rc = lib.bsgdtv_set_state(h, _dev_ptr(x, torch.float32), _dev_ptr(r, torch.float32),
                                  int(epoch), 1)
    else:
        x = np.ascontiguousarray(x, dtype=np.float32)
        r = np.ascontiguousarray(r, dtype=np.float32)
        rc = lib.bsgdtv_set_state(h, _host_ptr(x, np.float32), _host_ptr(r, np.float32),
                                  int(epoch), 0)
    _check(rc, "bsgdtv_set_state")


def bsgdtv_objective(h):
    f, tv = ctypes.c_double(), ctypes.c_double()
    _check(load().bsgdtv_objective(h, ctypes.byref(f), ctypes.byref(tv)), "bsgdtv_objective")
    return f.value, tv.value


def bsgdtv_block_products(h, x, r, z_blocks, g_blocks):
    import torch
    _check(load().bsgdtv_block_products(h, _dev_ptr(x, torch.float32), _dev_ptr(r, torch.float32),
                                        _dev_ptr(z_blocks, torch.float32),
                                        _dev_ptr(g_blocks, torch.float32)),
           "bsgdtv_block_products")


def bsgdtv_tv_prox(b, x, tau, iters, stream=None):
    import torch
    if b.dim() != 2 or x.shape != b.shape:
        raise ValueError("b and x must be matching 2-D tensors")
    _check(load().bsgdtv_tv_prox(_dev_ptr(b, torch.float32), _dev_ptr(x, torch.float32),
                                 int(b.shape[0]), int(b.shape[1]), float(tau), int(iters),
                                 stream if stream is not None else current_stream()),
           "bsgdtv_tv_prox")


def bsgdtv_tv_prox_static(b, x, tau, iters, stream=None):
    """TV prox with no allocation: scratch in a fixed device array inside the
    library (for callers that cannot allocate device memory; at most 262144
    pixels and 4096 iterations; concurrent calls race on the shared array)."""
    import torch
    if b.dim() != 2 or x.shape != b.shape:
        raise ValueError("b and x must be matching 2-D tensors")
    _check(load().bsgdtv_tv_prox_static(_dev_ptr(b, torch.float32), _dev_ptr(x, torch.float32),
                                        int(b.shape[0]), int(b.shape[1]), float(tau), int(iters),
                                        stream if stream is not None else current_stream()),
           "bsgdtv_tv_prox_static")


def bsgdtv_fgp_tiling(length, halo):
    """The prox's regions along one dimension: list of (first, lo, hi)."""
    lib = load()
    n = ctypes.c_int()
    _check(lib.bsgdtv_fgp_tiling(int(length), int(halo), 0, ctypes.byref(n), None, None, None),
           "bsgdtv_fgp_tiling")
    f, lo, hi = (np.zeros(max(n.value, 1), np.int32) for _ in range(3))
    _check(lib.bsgdtv_fgp_tiling(int(length), int(halo), n.value, ctypes.byref(n), _host_ptr(f, np.int32),
                                 _host_ptr(lo, np.int32), _host_ptr(hi, np.int32)), "bsgdtv_fgp_tiling")
    return [(int(f[k]), int(lo[k]), int(hi[k])) for k in range(n.value)]


def bsgdtv_partition_bounds(rows, cols, M, N, row_unit=1, col_unit=1):
    """Host only: default I_i / J_j bounds."""
    rb = np.zeros(M + 1, dtype=np.int64)
    cb = np.zeros(N + 1, dtype=np.int64)
    _check(load().bsgdtv_partition_bounds(int(rows), int(cols), int(M), int(N), int(row_unit),
                                          int(col_unit), _host_ptr(rb, np.int64),
                                          _host_ptr(cb, np.int64)), "bsgdtv_partition_bounds")
    return rb, cb


def bsgdtv_layout_check(rows, cols, img_h, img_w, row_ptr, col_idx, vals, M, N, row_unit=1,
                        col_unit=1, row_bounds=None, col_bounds=None, target_items=608,
                        fmt=FMT_F32_I32):
    """Host only: builds the device layout in host memory and checks it decodes
    back to A.  Returns the layout statistics (raises on failure)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    rb = None if row_bounds is None else np.ascontiguousarray(row_bounds, dtype=np.int64)
    cb = None if col_bounds is None else np.ascontiguousarray(col_bounds, dtype=np.int64)
    stats = np.zeros(6, dtype=np.int64)
    rc = load().bsgdtv_layout_check(int(rows), int(cols), int(img_h), int(img_w),
                                    _host_ptr(row_ptr, np.int64), _host_ptr(col_idx, np.int32),
                                    _host_ptr(vals, np.float64), int(M), int(N), int(row_unit),
                                    int(col_unit), None if rb is None else _host_ptr(rb, np.int64),
                                    None if cb is None else _host_ptr(cb, np.int64), int(fmt),
                                    int(target_items), _host_ptr(stats, np.int64))
    _check(rc, "bsgdtv_layout_check")
    keys = ["nnz", "segments", "slabs", "work_items", "groups", "tiles"]
    return dict(zip(keys, (int(v) for v in stats)))


def bsgdtv_batch_create_csr(rows, cols, img_h, img_w, row_ptr, col_idx, vals, slices,
                            stream=None, fmt=FMT_F32_I32):
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    if row_ptr.size != rows + 1:
        raise ValueError("row_ptr must have rows+1 entries")
    h = ctypes.c_void_p()
    rc = lib.bsgdtv_batch_create_csr_ex(ctypes.byref(h), int(rows), int(cols), int(img_h),
                                        int(img_w), _host_ptr(row_ptr, np.int64),
                                        _host_ptr(col_idx, np.int32), _host_ptr(vals, np.float64),
                                        int(slices), int(fmt),
                                        stream if stream is not None else current_stream())
    _check(rc, "bsgdtv_batch_create_csr_ex")
    return h


def bsgdtv_operator_create_csr(rows, cols, img_h, img_w, row_ptr, col_idx, vals,
                               fmt=FMT_F32_I32, stream=None):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    op = ctypes.c_void_p()
    _check(load().bsgdtv_operator_create_csr(ctypes.byref(op), int(rows), int(cols), int(img_h),
                                             int(img_w), _host_ptr(row_ptr, np.int64),
                                             _host_ptr(col_idx, np.int32),
                                             _host_ptr(vals, np.float64), int(fmt),
                                             stream if stream is not None else current_stream()),
           "bsgdtv_operator_create_csr")
    return op


def bsgdtv_operator_destroy(op):
    load().bsgdtv_operator_destroy(op)


def bsgdtv_batch_create_from_operator(op, slices, stream=None):
    h = ctypes.c_void_p()
    _check(load().bsgdtv_batch_create_from_operator(ctypes.byref(h), op, int(slices),
                                                    stream if stream is not None else current_stream()),
           "bsgdtv_batch_create_from_operator")
    return h


def bsgdtv_batch_destroy(h):
    load().bsgdtv_batch_destroy(h)


def bsgdtv_batch_set_data(h, y, lambdas, mu):
    """y: [slices, rows] float32 (CUDA tensor or numpy); lambdas: [slices]."""
    lib = load()
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    if _is_tensor(y):
        import torch
        rc = lib.bsgdtv_batch_set_data(h, _dev_ptr(y, torch.float32), 1,
                                       _host_ptr(lam, np.float64), float(mu))
    else:
        y = np.ascontiguousarray(y, dtype=np.float32)
        rc = lib.bsgdtv_batch_set_data(h, _host_ptr(y, np.float32), 0, _host_ptr(lam, np.float64),
                                       float(mu))
    _check(rc, "bsgdtv_batch_set_data")


def bsgdtv_batch_run(h, epochs, fgp_iters):
    _check(load().bsgdtv_batch_run(h, int(epochs), int(fgp_iters)), "bsgdtv_batch_run")


def bsgdtv_batch_run_timed(h, epochs, fgp_iters):
    """Runs epochs and returns (sum of product-pass ms, sum of epoch ms)."""
    pk, ep = ctypes.c_double(), ctypes.c_double()
    _check(load().bsgdtv_batch_run_timed(h, int(epochs), int(fgp_iters), ctypes.byref(pk),
                                         ctypes.byref(ep)), "bsgdtv_batch_run_timed")
    return pk.value, ep.value


def bsgdtv_batch_get_x(h, out):
    """Copies every slice's x into `out` ([slices, cols] float32, CUDA tensor or numpy)."""
    lib = load()
    if _is_tensor(out):
        import torch
        rc = lib.bsgdtv_batch_get_x(h, _dev_ptr(out, torch.float32), 1)
    else:
        rc = lib.bsgdtv_batch_get_x(h, _host_ptr(out, np.float32), 0)
    _check(rc, "bsgdtv_batch_get_x")
    return out


def bsgdtv_batch_set_slice(h, b, y, lam):
    """Restarts slice b with projections y (None empties the slot)."""
    lib = load()
    if y is None:
        rc = lib.bsgdtv_batch_set_slice(h, int(b), None, 0, 0.0)
    elif _is_tensor(y):
        import torch
        rc = lib.bsgdtv_batch_set_slice(h, int(b), _dev_ptr(y, torch.float32), 1, float(lam))
    else:
        y = np.ascontiguousarray(y, dtype=np.float32)
        rc = lib.bsgdtv_batch_set_slice(h, int(b), _host_ptr(y, np.float32), 0, float(lam))
    _check(rc, "bsgdtv_batch_set_slice")


def bsgdtv_batch_get_slice_x(h, b, out):
    lib = load()
    if _is_tensor(out):
        import torch
        rc = lib.bsgdtv_batch_get_slice_x(h, int(b), _dev_ptr(out, torch.float32), 1)
    else:
        rc = lib.bsgdtv_batch_get_slice_x(h, int(b), _host_ptr(out, np.float32), 0)
    _check(rc, "bsgdtv_batch_get_slice_x")
    return out


def bsgdtv_batch_create_parallel_beam(n, n_angles, n_bins, slices, stream=None):
    h = ctypes.c_void_p()
    _check(load().bsgdtv_batch_create_parallel_beam(ctypes.byref(h), int(n), int(n_angles),
                                                    int(n_bins), int(slices),
                                                    stream if stream is not None else current_stream()),
           "bsgdtv_batch_create_parallel_beam")
    return h


def bsgdtv_mf_ray_weights(n, n_angles, n_bins, rays, capacity=None):
    """Weights of the matrix-free row pass for the given rays: list of
    (cols int32, vals float32) per ray."""
    rays = np.ascontiguousarray(rays, dtype=np.int64)
    cap = int(capacity or 3 * n + 3)
    cols = np.zeros(rays.size * cap, dtype=np.int32)
    vals = np.zeros(rays.size * cap, dtype=np.float32)
    cnt = np.zeros(rays.size, dtype=np.int32)
    _check(load().bsgdtv_mf_ray_weights(int(n), int(n_angles), int(n_bins), _host_ptr(rays, np.int64),
                                        int(rays.size), cap, _host_ptr(cols, np.int32),
                                        _host_ptr(vals, np.float32), _host_ptr(cnt, np.int32)),
           "bsgdtv_mf_ray_weights")
    return [(cols[i * cap:i * cap + cnt[i]].copy(), vals[i * cap:i * cap + cnt[i]].copy())
            for i in range(rays.size)]


def bsgdtv_batch_estimate_umax(h, max_iters=1000, rel_tol=1e-9):
    u, it = ctypes.c_double(), ctypes.c_int()
    _check(load().bsgdtv_batch_estimate_umax(h, int(max_iters), float(rel_tol), ctypes.byref(u),
                                             ctypes.byref(it)), "bsgdtv_batch_estimate_umax")
    return u.value, it.value


def bsgdtv_batch_project(h, x, y):
    """y = A x for every slice: CUDA float32 tensors x [slices, cols], y [slices, rows]."""
    import torch
    _check(load().bsgdtv_batch_project(h, _dev_ptr(x, torch.float32), _dev_ptr(y, torch.float32)),
           "bsgdtv_batch_project")
    return y


def bsgdtv_batch_set_tuning(h, fgp_chunk=0, fgp_group=0):
    """Applies a known tuning (0 = default for either)."""
    _check(load().bsgdtv_batch_set_tuning(h, int(fgp_chunk), int(fgp_group)), "bsgdtv_batch_set_tuning")


def bsgdtv_batch_autotune(h, fgp_iters, epochs_per_trial=3):
    """Picks the batch's FGP iterations per launch and slices per FGP launch
    group by timing; returns (chunk, group, epoch ms)."""
    c, g, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(load().bsgdtv_batch_autotune(h, int(fgp_iters), int(epochs_per_trial), ctypes.byref(c),
                                        ctypes.byref(g), ctypes.byref(ms)), "bsgdtv_batch_autotune")
    return c.value, g.value, ms.value


def bsgdtv_batch_device_bytes(rows, cols, nnz, slices, fmt=FMT_F32_I32) -> int:
    """Host only: device bytes of a batch of these sizes (-1 on bad sizes)."""
    return int(load().bsgdtv_batch_device_bytes(int(rows), int(cols), int(nnz), int(slices), int(fmt)))


def bsgdtv_server_create(hbm_budget_bytes, fgp_iters, max_tick_epochs=8):
    h = ctypes.c_void_p()
    _check(load().bsgdtv_server_create(ctypes.byref(h), int(hbm_budget_bytes), int(fgp_iters),
                                       int(max_tick_epochs)), "bsgdtv_server_create")
    return h


def bsgdtv_server_destroy(h):
    load().bsgdtv_server_destroy(h)


def bsgdtv_server_add_geometry(h, rows, cols, img_h, img_w, row_ptr, col_idx, vals, fmt, slots, mu,
                               prewarm=1):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    gid = ctypes.c_int()
    _check(load().bsgdtv_server_add_geometry(h, int(rows), int(cols), int(img_h), int(img_w),
                                             _host_ptr(row_ptr, np.int64), _host_ptr(col_idx, np.int32),
                                             _host_ptr(vals, np.float64), int(fmt), int(slots),
                                             float(mu), int(prewarm), ctypes.byref(gid)),
           "bsgdtv_server_add_geometry")
    return gid.value


def bsgdtv_server_submit(h, geom_id, y, lam, epochs):
    y = np.ascontiguousarray(y, dtype=np.float32)
    rid = ctypes.c_int64()
    _check(load().bsgdtv_server_submit(h, int(geom_id), _host_ptr(y, np.float32), float(lam),
                                       int(epochs), ctypes.byref(rid)), "bsgdtv_server_submit")
    return rid.value


def bsgdtv_server_poll(h, request_id):
    st = ctypes.c_int()
    _check(load().bsgdtv_server_poll(h, int(request_id), ctypes.byref(st)), "bsgdtv_server_poll")
    return st.value


def bsgdtv_server_cancel(h, request_id):
    """Cancels a queued or running request (running: at the end of its
    group's current tick)."""
    _check(load().bsgdtv_server_cancel(h, int(request_id)), "bsgdtv_server_cancel")


def bsgdtv_server_wait(h, request_id, out=None, timeout_s=-1.0):
    """Waits for a request; fills `out` (float32 numpy, or None) and returns
    (latency_s, queued_s)."""
    times = np.zeros(2, dtype=np.float64)
    _check(load().bsgdtv_server_wait(h, int(request_id), float(timeout_s),
                                     None if out is None else _host_ptr(out, np.float32),
                                     _host_ptr(times, np.float64)), "bsgdtv_server_wait")
    return float(times[0]), float(times[1])


SERVER_STATS = ["submitted", "completed", "failed", "queued", "running", "groups", "device_bytes",
                "max_running", "ticks", "epochs_run", "slice_epochs", "groups_made", "cancelled",
                "armed_epochs", "wait_timeouts", "packed_groups", "max_parts", "packed_launches"]


def bsgdtv_server_stats(h):
    v = np.zeros(len(SERVER_STATS), dtype=np.int64)
    _check(load().bsgdtv_server_stats(h, _host_ptr(v, np.int64)), "bsgdtv_server_stats")
    return dict(zip(SERVER_STATS, (int(a) for a in v)))


def bsgdtv_launch_count() -> int:
    return int(load().bsgdtv_launch_count())


def bsgdtv_strerror(code: int) -> str:
    return load().bsgdtv_strerror(int(code)).decode()


# ------------------------------------------------------------- convenience
class Reconstructor:
    """Owns one handle: ``Reconstructor(A, img_shape, M, N, ...)`` then
    ``set_data`` / ``run`` / ``x()``.  `A` is any host CSR with row_ptr, cols,
    vals, rows and cols_n attributes."""

    def __init__(self, A, img_shape, M, N, row_unit=1, col_unit=1, row_bounds=None,
                 col_bounds=None, stream=None, fmt=FMT_F32_I32, parallel_beam=None):
        """A = None with parallel_beam = (n_angles, n_bins): A is generated on
        the device for that geometry of the img_shape = (n, n) image."""
        self.img_shape = tuple(img_shape)
        self.M, self.N = int(M), int(N)
        if A is None:
            n = int(img_shape[0])
            if parallel_beam is None or img_shape[1] != n:
                raise ValueError("A = None needs parallel_beam=(n_angles, n_bins) and a square image")
            na, nb = (int(v) for v in parallel_beam)
            self.rows, self.cols = na * nb, n * n
            self.h = bsgdtv_create_parallel_beam(n, na, nb, M, N, stream, fmt)
            return
        self.rows, self.cols = int(A.rows), int(A.cols_n)
        self.h = bsgdtv_create_csr(self.rows, self.cols, img_shape[0], img_shape[1], A.row_ptr,
                                   A.cols, A.vals, M, N, row_unit, col_unit, row_bounds,
                                   col_bounds, stream, fmt)

    def close(self):
        if getattr(self, "h", None) is not None:
            bsgdtv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def partition(self):
        return bsgdtv_get_partition(self.h, self.M, self.N)

    def info(self):
        return bsgdtv_get_info(self.h)

    def estimate_umax(self, max_iters=5000, rel_tol=1e-12):
        return bsgdtv_estimate_umax(self.h, max_iters, rel_tol)

    def set_data(self, y, lam, mu=0.0):
        bsgdtv_set_data(self.h, y, lam, mu)

    def params(self):
        return bsgdtv_get_params(self.h)

    def run(self, epochs, fgp_iters):
        bsgdtv_run(self.h, epochs, fgp_iters)

    def run_until(self, max_epochs, fgp_iters, check_every=10, rel_tol=1e-6):
        """Returns (epochs run, last objective data + lambda TV)."""
        return bsgdtv_run_until(self.h, max_epochs, fgp_iters, check_every, rel_tol)

    def run_subsets(self, row_sel, col_sel, fgp_iters):
        bsgdtv_run_subsets(self.h, row_sel, col_sel, fgp_iters)

    def x(self, out=None):
        if out is None:
            out = np.empty(self.cols, dtype=np.float32)
        return bsgdtv_get_x(self.h, out)

    def reconstruct(self, y, lam, mu, epochs, fgp_iters, out=None):
        """set_data + run + x in one call (one synchronisation)."""
        if out is None:
            if _is_tensor(y):
                import torch
                out = torch.empty(self.cols, dtype=torch.float32, device=y.device)
            else:
                out = np.empty(self.cols, dtype=np.float32)
        return bsgdtv_reconstruct(self.h, y, lam, mu, epochs, fgp_iters, out)

    def objective(self):
        return bsgdtv_objective(self.h)


class BatchReconstructor:
    """Owns one batch handle: B slices sharing the matrix A, each with its own
    y_b and lambda_b; ``set_data(Y, lambdas, mu)`` / ``run`` / ``x()``."""

    def __init__(self, A, img_shape, slices, stream=None, fmt=FMT_F32_I32, parallel_beam=None,
                 operator=None):
        """`A`: host CSR, or None with parallel_beam = (n_angles, n_bins) for
        the matrix-free projector of an img_shape = (n, n) image, or None with
        `operator` (from bsgdtv_operator_create_csr) shared with other batches."""
        self.img_shape = tuple(img_shape)
        self.slices = int(slices)
        if operator is not None:
            n_h, n_w = self.img_shape
            self.rows, self.cols = None, n_h * n_w
            self.h = bsgdtv_batch_create_from_operator(operator, slices, stream)
        elif A is None:
            n = int(img_shape[0])
            na, nb = parallel_beam
            self.rows, self.cols = int(na) * int(nb), n * n
            self.h = bsgdtv_batch_create_parallel_beam(n, na, nb, slices, stream)
        else:
            self.rows, self.cols = int(A.rows), int(A.cols_n)
            self.h = bsgdtv_batch_create_csr(self.rows, self.cols, img_shape[0], img_shape[1],
                                             A.row_ptr, A.cols, A.vals, slices, stream, fmt)

    def close(self):
        if getattr(self, "h", None) is not None:
            bsgdtv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_data(self, Y, lambdas, mu):
        bsgdtv_batch_set_data(self.h, Y, lambdas, mu)

    def run(self, epochs, fgp_iters):
        bsgdtv_batch_run(self.h, epochs, fgp_iters)

    def run_timed(self, epochs, fgp_iters):
        return bsgdtv_batch_run_timed(self.h, epochs, fgp_iters)

    def x(self, out=None):
        if out is None:
            out = np.empty((self.slices, self.cols), dtype=np.float32)
        return bsgdtv_batch_get_x(self.h, out)

    def set_slice(self, b, y, lam):
        bsgdtv_batch_set_slice(self.h, b, y, lam)

    def estimate_umax(self, max_iters=1000, rel_tol=1e-9):
        return bsgdtv_batch_estimate_umax(self.h, max_iters, rel_tol)

    def autotune(self, fgp_iters, epochs_per_trial=3):
        return bsgdtv_batch_autotune(self.h, fgp_iters, epochs_per_trial)

    def set_tuning(self, fgp_chunk=0, fgp_group=0):
        bsgdtv_batch_set_tuning(self.h, fgp_chunk, fgp_group)

    def tuning(self):
        """(FGP iterations per launch, slices per FGP group, row-pass lanes, column-pass lanes)."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(load().bsgdtv_batch_get_tuning(self.h, *[ctypes.byref(a) for a in v]),
               "bsgdtv_batch_get_tuning")
        return tuple(a.value for a in v)

    def set_pass_lanes(self, lanes_row=0, lanes_col=0):
        _check(load().bsgdtv_batch_set_pass_lanes(self.h, int(lanes_row), int(lanes_col)),
               "bsgdtv_batch_set_pass_lanes")

    def project(self, x, y=None):
        """y = A x per slice (CUDA tensors); resets the batch's state."""
        import torch
        if y is None:
            y = torch.empty((self.slices, self.rows), dtype=torch.float32, device=x.device)
        return bsgdtv_batch_project(self.h, x, y)

    def slice_x(self, b, out=None):
        if out is None:
            out = np.empty(self.cols, dtype=np.float32)
        return bsgdtv_batch_get_slice_x(self.h, b, out)


class PackedBatch:
    """Several geometries with `slices` slots each, every epoch stage one
    launch over all of them: ``PackedBatch([A1, A2], [(n1, n1), (n2, n2)],
    slices)``, ``set_part(k, Y_k, lambdas_k, mu_k)``, ``run``, ``x(k)``."""

    def __init__(self, As, img_shapes, slices, fmt=FMT_F32_I32, stream=None):
        import torch
        self.slices = int(slices)
        self.rows = [int(A.rows) for A in As]
        self.cols = [int(A.cols_n) for A in As]
        ops = [bsgdtv_operator_create_csr(A.rows, A.cols_n, shp[0], shp[1], A.row_ptr, A.cols,
                                          A.vals, fmt)
               for A, shp in zip(As, img_shapes)]
        arr = (ctypes.c_void_p * len(ops))(*[op.value for op in ops])
        h = ctypes.c_void_p()
        try:
            _check(load().bsgdtv_packed_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p),
                                               len(ops), self.slices,
                                               stream if stream is not None else current_stream()),
                   "bsgdtv_packed_create")
        finally:
            for op in ops:                      # the parts keep their own references
                bsgdtv_operator_destroy(op)
        self.h = h.value

    def close(self):
        if getattr(self, "h", None) is not None:
            load().bsgdtv_packed_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_part(self, k, Y, lambdas, mu):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        if lam.size != self.slices:
            raise ValueError("one lambda per slot")
        if _is_tensor(Y):
            import torch
            ptr, dev = _dev_ptr(Y, torch.float32, self.slices * self.rows[k]), 1
        else:
            Y = np.ascontiguousarray(Y, dtype=np.float32)
            if Y.size != self.slices * self.rows[k]:
                raise ValueError("Y must hold slices x rows of the part")
            ptr, dev = _host_ptr(Y, np.float32), 0
        _check(load().bsgdtv_packed_set_part(self.h, int(k), ptr, dev, _host_ptr(lam, np.float64),
                                             float(mu)), "bsgdtv_packed_set_part")

    def run(self, epochs, fgp_iters):
        _check(load().bsgdtv_packed_run(self.h, int(epochs), int(fgp_iters)), "bsgdtv_packed_run")

    def x(self, k):
        out = np.empty((self.slices, self.cols[k]), dtype=np.float32)
        _check(load().bsgdtv_packed_get_x(self.h, int(k), _host_ptr(out, np.float32), 0),
               "bsgdtv_packed_get_x")
        return out

    def launches_per_epoch(self, fgp_iters):
        n = ctypes.c_int64()
        _check(load().bsgdtv_packed_launches_per_epoch(self.h, int(fgp_iters), ctypes.byref(n)),
               "bsgdtv_packed_launches_per_epoch")
        return n.value


class Server:
    """Continuous-batching server: ``add_geometry(A, img_shape, mu, ...)`` then
    ``submit(geom, y, lam, epochs)`` from any thread and ``wait(request)``."""

    def __init__(self, hbm_budget_bytes, fgp_iters, max_tick_epochs=8):
        self.h = bsgdtv_server_create(hbm_budget_bytes, fgp_iters, max_tick_epochs)
        self.cols = {}

    def close(self):
        if getattr(self, "h", None) is not None:
            bsgdtv_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def add_geometry(self, A, img_shape, mu, slots=32, fmt=FMT_F32_I32, prewarm=1):
        gid = bsgdtv_server_add_geometry(self.h, A.rows, A.cols_n, img_shape[0], img_shape[1],
                                         A.row_ptr, A.cols, A.vals, fmt, slots, mu, prewarm)
        self.cols[gid] = int(A.cols_n)
        return gid

    def submit(self, geom_id, y, lam, epochs):
        return bsgdtv_server_submit(self.h, geom_id, y, lam, epochs)

    def poll(self, request_id):
        return bsgdtv_server_poll(self.h, request_id)

    def cancel(self, request_id):
        bsgdtv_server_cancel(self.h, request_id)

    def wait(self, request_id, geom_id, timeout_s=-1.0):
        """Returns (x, latency_s, queued_s)."""
        x = np.empty(self.cols[geom_id], dtype=np.float32)
        lat, q = bsgdtv_server_wait(self.h, request_id, x, timeout_s)
        return x, lat, q

    def stats(self):
        return bsgdtv_server_stats(self.h)

    def hold(self, on=True):
        _check(load().bsgdtv_server_hold(self.h, 1 if on else 0), "bsgdtv_server_hold")

    def set_packing(self, max_parts, cost_ratio=4.0):
        _check(load().bsgdtv_server_set_packing(self.h, int(max_parts), float(cost_ratio)),
               "bsgdtv_server_set_packing")

    def set_priority(self, by_size):
        _check(load().bsgdtv_server_set_priority(self.h, int(bool(by_size))),
               "bsgdtv_server_set_priority")

    def arm(self, geom_id, wait_s):
        """Arms an idle group of the geometry for wait_s seconds (device-side
        wait); raises BsgdtvError with code BSGDTV_ERR_TIMEOUT if no request
        arrived meanwhile."""
        _check(load().bsgdtv_server_arm(self.h, int(geom_id), float(wait_s)), "bsgdtv_server_arm")
