"""Stored rows of A with rounded values (oracle side of the stored-matrix variant).

Sec. 4.2 notes that a block A_k may be stored or evaluated; for sizes where all
of A fits in memory it can be kept as a sparse matrix.  Storing it in float32
or bfloat16 changes the matrix the method works with.  This module gives that
matrix exactly, so that the iteration can be checked on the same A:

  float32 value  = round-to-nearest-even of the float64 Joseph weight
  bfloat16 value = round-to-nearest-even of that float32 to 8 significand bits
                   (the upper 16 bits of the float32 after adding
                   0x7FFF + (bit 16), the usual bfloat16 rounding rule)

Row and column order are those of `joseph.rows` (rays in id order, taps in
march order).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import joseph

KINDS = ("f32", "bf16")


def round_values(w: np.ndarray, kind: str) -> np.ndarray:
    """Float64 weights rounded as stored (returned as float64)."""
    w32 = np.asarray(w, dtype=np.float64).astype(np.float32)
    if kind == "f32":
        return w32.astype(np.float64)
    if kind != "bf16":
        raise ValueError(kind)
    bits = w32.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def stored_matrix(g: joseph.Geometry, kind: str) -> sp.csr_matrix:
    """All of A with stored (rounded) values."""
    A = joseph.full_matrix(g)
    A = A.copy()
    A.data = round_values(A.data, kind)
    return A


def stored_rows_fn(A_stored: sp.csr_matrix):
    """Row provider for slim.RowSource over a stored matrix."""
    def rows_fn(ids):
        return A_stored[np.asarray(ids, dtype=np.int64)]
    return rows_fn
