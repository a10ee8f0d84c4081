"""The tensor-core product and the triangular inverse of the mixed solve,
against float64 numpy, through the C ABI.

slim_tc_matmul: element-wise |C - C_ref| <= 1e-5 * (|op(A)| |op(B)|) (float32
accumulation over K <= 320; a product of the leading bfloat16 terms alone
would miss by about 4e-3).  Layout flags, ragged M and N, the triangular
masks with garbage in the masked triangle, alpha and beta, on both tile
widths: 128 x 64 for products of fewer 128 x 128 tiles than the GPU has SMs,
128 x 128 from there on (the last two cases, 160 and 165 wide tiles).

slim_chol_inverse: X = L^{-1} of the float32 factor of lambda I + G; its
strict upper triangle is exactly the transpose of the lower; the error to the
float64 inverse, and that of X^T X b as the solution of (lambda I + G) z = b,
stay within a small multiple of kappa(lambda I + G) u32 (the float32
factor's own forward error).
"""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("M,N,K,a_km,b_kn,c_nm,alpha,beta,a_lower,b_lower", [
    (128, 64, 64, 0, 0, 0, 1.0, 0.0, 0, 0),
    (256, 192, 128, 0, 1, 0, 1.0, 0.0, 0, 0),
    (200, 100, 320, 1, 0, 1, 1.0, 0.0, 0, 0),      # ragged tiles, transposed storage
    (300, 70, 192, 1, 1, 0, -1.0, 0.5, 0, 0),      # alpha, beta
    (192, 192, 192, 0, 1, 0, 1.0, 0.0, 1, 0),      # lower-triangular A (masked)
    (192, 130, 192, 0, 1, 1, -1.0, 0.0, 0, 1),     # lower-triangular B (masked)
    (2000, 1250, 64, 0, 1, 0, 1.0, 0.5, 0, 0),     # wide tiles, ragged
    (1900, 1300, 128, 1, 0, 1, -1.0, 0.0, 1, 1),   # wide tiles, both masks, C transposed
])
def test_tc_matmul(sl, M, N, K, a_km, b_kn, c_nm, alpha, beta, a_lower, b_lower):
    rs = np.random.default_rng(M + 7 * N + 13 * K)
    opA = rs.standard_normal((M, K)).astype(np.float32)
    opB = rs.standard_normal((K, N)).astype(np.float32)
    A_st = opA.T.copy() if a_km else opA.copy()          # storage as the flags say
    B_st = opB.copy() if b_kn else opB.T.copy()
    # the masked triangles hold garbage in storage, zeros in the reference
    if a_lower:
        tri = np.tril(np.ones((M, K), bool))
        opA = np.where(tri, opA, 0.0).astype(np.float32)
    if b_lower:
        tri = np.tril(np.ones((K, N), bool))
        opB = np.where(tri, opB, 0.0).astype(np.float32)
    C0 = rs.standard_normal((M, N)).astype(np.float32)
    C_st = C0.T.copy() if c_nm else C0.copy()
    lda = A_st.shape[1]
    ldb = B_st.shape[1]
    ldc = C_st.shape[1]
    At, Bt, Ct = _dev(A_st), _dev(B_st), _dev(C_st)
    sl.tc_matmul(M, N, K, At, lda, a_km, Bt, ldb, b_kn, Ct, ldc, c_nm, alpha, beta,
                 a_lower, b_lower)
    torch.cuda.synchronize()
    got = Ct.cpu().numpy().astype(np.float64)
    got = got.T if c_nm else got
    A64, B64 = opA.astype(np.float64), opB.astype(np.float64)
    want = alpha * (A64 @ B64) + beta * C0.astype(np.float64)
    scale = np.abs(alpha) * (np.abs(A64) @ np.abs(B64)) + np.abs(beta * C0) + 1e-30
    err = np.max(np.abs(got - want) / scale)
    assert err < 1e-5, err


def test_tc_matmul_rejects_bad_arguments(sl):
    x = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    with pytest.raises(sl.SlimError):          # K not a multiple of 64
        sl.tc_matmul(64, 64, 48, x, 64, 0, x, 64, 0, x, 64, 0)
    with pytest.raises(sl.SlimError):          # K-contiguous rows not 16-byte multiples
        sl.tc_matmul(64, 64, 64, x, 66, 0, x, 64, 0, x, 64, 0)


def _spd(p, lam, seed):
    rs = np.random.default_rng(seed)
    B = rs.standard_normal((p, p + 20)) / np.sqrt(p)
    return B @ B.T, lam


def _check_inverse(sl, G, lam):
    p = G.shape[0]
    K = lam * np.eye(p) + G
    X = torch.empty((p, p), dtype=torch.float32, device="cuda")
    sl.chol_inverse(torch.tensor(G, device="cuda"), lam, X)
    torch.cuda.synchronize()
    Xh = X.cpu().numpy().astype(np.float64)
    lo, up = np.tril(Xh), np.triu(Xh, 1)
    assert np.array_equal(up, np.tril(Xh, -1).T)           # X^T above, bit for bit
    L = np.linalg.cholesky(K)
    Xr = sla.solve_triangular(L, np.eye(p), lower=True)
    kK = np.linalg.cond(K)
    # the float32 factor's forward error is bounded by about kappa(K) u32
    err = np.linalg.norm(lo - Xr) / np.linalg.norm(Xr)
    assert err < 20 * kK * U32, (err, kK)
    b = np.random.default_rng(p).standard_normal(p)
    z = lo.T @ (lo @ b)
    zr = np.linalg.solve(K, b)
    ez = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    assert ez < 20 * kK * U32, (ez, kK)
    return err, ez


@pytest.mark.parametrize("p,lam", [(17, 1.0), (64, 1e-1), (100, 1e-1), (364, 1e-2),
                                   (1000, 1.0), (2178, 1e-2)])
def test_chol_inverse_random_spd(sl, p, lam):
    G, lam = _spd(p, lam, p)
    _check_inverse(sl, G, lam)


def test_chol_inverse_tomography_window(sl):
    # the damped Gram matrix of a full 256 x 256 window (p = 2178, kappa 1.5e6)
    import workloads
    from oracle import joseph, slim as oslim
    cfg = workloads.C2
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    ids = np.concatenate([oslim.view_block_ids(g, cfg.seed, k) for k in range(3, 9)])
    M = joseph.rows(g, ids)
    G = (M @ M.T).toarray()
    _check_inverse(sl, G, cfg.lam)
