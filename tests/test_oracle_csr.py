"""Pins for the stored-matrix model (float32 / bfloat16 values of A)."""
import numpy as np
import pytest

from oracle import csr, joseph


def test_bf16_rounding_ties_and_library():
    # spacing near 1 is 2^-7: 1 + 2^-8 ties to even (1), 1 + 3*2^-8 ties up to 1 + 2^-6
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 3e-20, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, None, 0.0], dtype=object)
    got = csr.round_values(x, "bf16")
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    torch = pytest.importorskip("torch")
    rs = np.random.default_rng(0)
    v = rs.standard_normal(20000) * 10.0 ** rs.uniform(-3, 3, 20000)
    lib = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(csr.round_values(v, "bf16"), lib)


def test_f32_rounding_is_numpy_cast():
    v = np.random.default_rng(1).standard_normal(1000)
    assert np.array_equal(csr.round_values(v, "f32"), v.astype(np.float32).astype(np.float64))


def test_stored_matrix_keeps_structure():
    g = joseph.Geometry(16, 8, 23)
    A = joseph.full_matrix(g)
    for kind in csr.KINDS:
        S = csr.stored_matrix(g, kind)
        assert np.array_equal(S.indptr, A.indptr) and np.array_equal(S.indices, A.indices)
        assert np.max(np.abs(S.data - A.data) / np.abs(A.data)) <= (2 ** -8 if kind == "bf16" else 2 ** -24)
