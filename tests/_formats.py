"""Stored-weight formats, reproduced independently of the library for the
oracle: the operator the GPU uses for each format, with FP64 entries."""
import numpy as np

from paper_1812_01307_gb300 import synth


def bf16_round(v):
    """Round to nearest even with 8 significant bits (bfloat16), by exact
    scaling of the frexp mantissa and Python's round()."""
    m, e = np.frexp(np.asarray(v, dtype=np.float64))
    q = np.array([round(mm * 256.0) for mm in np.ravel(m)], dtype=np.float64).reshape(np.shape(m))
    return np.ldexp(q / 256.0, e)


def stored_operator(A, fmt):
    """A with its weights rounded as a handle of format `fmt` stores them."""
    if fmt in (0, 1):
        v = A.vals.astype(np.float32).astype(np.float64)
    elif fmt == 2:
        v = A.vals.astype(np.float16).astype(np.float64)
    elif fmt == 3:
        u, inv = np.unique(A.vals, return_inverse=True)
        v = bf16_round(u)[inv]
    else:
        raise ValueError(fmt)
    return synth.CSR(A.rows, A.cols_n, A.row_ptr, A.cols, v)
