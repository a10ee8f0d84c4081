"""Pins for the slimTik oracle, Eq. (slimTik) (C_k = L^T L, Sec. 2).

* The Woodbury form (L = diag(l)) equals the direct n x n form at every step,
  in the growing window and after it, with and without the damping ramp, for
  both readings of the Tikhonov count.
* The direct form (any invertible L, reading "window") equals slimLS, Eq. (ram)
  with Eq. (B_k) and C_k = L^T L, applied to the stacked problem of Eq. (TLS1),
  assembled here from the stacked rows [A_i; lam_tik M^{-1/2} L] and [b_i; 0].
* Full memory (r >= k-1), constant damping lambda, any sample sequence:
  (lambda P + k beta P + sum_i A_i^T A_i) x_k = lambda P x_0 + sum_i A_i^T b_i,
  P = L^T L, beta = lam_tik^2 / M (induction as in Appendix A); so one cyclic
  epoch from x_0 = 0 gives the Tikhonov solution of Eq. (TLS1) with the
  regulariser lam_tik^2 + lambda, checked against a least-squares solve of the
  stacked matrix [A; sqrt(lam_tik^2 + lambda) L].
* lam_tik = 0 and L = I: the slimLS step of the slimLS oracle.
* ell = 1, r = 0, L = I: the Sherman-Morrison closed form
  s = (g - a (a.g)/(mu + ||a||^2)) / mu with g = a (a x - b) + beta x.
* The printed count r equals the window count with the damping lowered by
  beta, once the window is full.
Mutations planted in the oracle (here, on the CPU) break these pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import joseph, slim, tik


def _tiny_tomo(N=12, V=10, D=17, seed=5):
    g = joseph.Geometry(N, V, D)
    x_true = workloads.phantom_2d(N, seed, 4)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ x_true, workloads.noise_direction(g.m, seed), 0.01)
    return g, A, b


def _general_L(n, seed):
    # invertible, not diagonal: positive diagonal plus a sparse strictly upper part
    rng = np.random.default_rng(seed)
    U = np.triu(rng.standard_normal((n, n)), 1) * (rng.random((n, n)) < 0.02)
    return np.diag(0.6 + rng.random(n)) + 0.3 * U


def _weights(n, seed):
    return 0.5 + 1.5 * np.random.default_rng(seed).random(n)


@pytest.mark.parametrize("reading", ["window", "printed"])
@pytest.mark.parametrize("ramp", [False, True])
def test_woodbury_equals_direct(reading, ramp):
    g, A, b = _tiny_tomo()
    src = slim.tomo_source(g, b)
    sched = list(slim.view_schedule(g, 4, 9))
    l = _weights(g.n, 1)
    x0 = np.random.default_rng(2).standard_normal(g.n) * 0.1
    kw = dict(r=2, lam=1e-2, lam_tik=0.7, n_blocks=g.n_views, l=l, x0=x0, ramp=ramp,
              reading=reading, eta=0.9)
    xw = [x for _, x, _ in tik.run(src, sched, **kw)]
    xd = [x for _, x, _ in tik.run(src, sched, form="direct", **kw)]
    for k, (a, c) in enumerate(zip(xw, xd), start=1):
        assert np.linalg.norm(a - c) <= 1e-10 * np.linalg.norm(c), k


def _stacked_slimls_step(x, window_blocks, b_new, lam_k, lam_tik, n_blocks, L):
    # slimLS (Eq. ram, Eq. B_k with C_k = L^T L) on the rows of Eq. (TLS1)
    # sampled by W~_k: each block is [A_i; lam_tik M^{-1/2} L], rhs [b_i; 0]
    aug = [np.vstack([B.toarray(), lam_tik / np.sqrt(n_blocks) * L]) for B in window_blocks]
    Mt = np.vstack(aug)
    At = aug[-1]
    bt = np.concatenate([b_new, np.zeros(L.shape[0])])
    H = lam_k * (L.T @ L) + Mt.T @ Mt
    return x - np.linalg.solve(H, At.T @ (At @ x - bt))


def test_direct_form_is_slimls_on_the_stacked_problem():
    g, A, b = _tiny_tomo(seed=6)
    src = slim.tomo_source(g, b)
    sched = list(slim.view_schedule(g, 6, 7))
    L = _general_L(g.n, 3)
    r, lam, lam_tik = 2, 5e-2, 0.8
    x = np.random.default_rng(4).standard_normal(g.n) * 0.1
    xs = [xk for _, xk, _ in tik.run(src, sched, r, lam, lam_tik, g.n_views, x0=x, L=L,
                                     form="direct", ramp=True)]
    window = []
    for k, ids in enumerate(sched, start=1):
        window = (window + [src.rows(ids)])[-(r + 1):]
        x = _stacked_slimls_step(x, window, src.rhs(ids), slim.damping(lam, k, r, True), lam_tik,
                                 g.n_views, L)
        assert np.linalg.norm(xs[k - 1] - x) <= 1e-10 * np.linalg.norm(x), k


def _full_memory_identity(src, A, sched, lam, lam_tik, n_blocks, P, x0, xs):
    beta = lam_tik ** 2 / n_blocks
    H = np.zeros_like(P)
    rhs = lam * (P @ x0)
    worst = 0.0
    for k, (ids, xk) in enumerate(zip(sched, xs), start=1):
        Ak = A[ids].toarray()
        H += Ak.T @ Ak
        rhs = rhs + Ak.T @ src.rhs(ids)
        lhs = (lam * P + k * beta * P + H) @ xk
        worst = max(worst, np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs))
    return worst


@pytest.mark.parametrize("form", ["direct", "woodbury"])
def test_full_memory_identity(form):
    g, A, b = _tiny_tomo(seed=7)
    src = slim.tomo_source(g, b)
    rng = np.random.default_rng(8)
    sched = [g.view_rays(int(v)) for v in rng.integers(0, g.n_views, 8)]   # repeats allowed
    if form == "direct":
        L = _general_L(g.n, 9)
        kw = dict(L=L)
    else:
        l = _weights(g.n, 9)
        L = np.diag(l)
        kw = dict(l=l)
    P = L.T @ L
    lam, lam_tik = 3e-2, 0.6
    x0 = rng.standard_normal(g.n) * 0.1
    xs = [x for _, x, _ in tik.run(src, sched, r=len(sched), lam=lam, lam_tik=lam_tik,
                                   n_blocks=g.n_views, x0=x0, form=form, **kw)]
    assert _full_memory_identity(src, A, sched, lam, lam_tik, g.n_views, P, x0, xs) < 1e-11


@pytest.mark.parametrize("form", ["direct", "woodbury"])
def test_one_epoch_gives_the_tikhonov_solution(form):
    g, A, b = _tiny_tomo(seed=10)
    src = slim.tomo_source(g, b)
    order = np.random.default_rng(11).permutation(g.n_views)
    sched = [g.view_rays(int(v)) for v in order]
    if form == "direct":
        L = _general_L(g.n, 12)
        kw = dict(L=L)
    else:
        l = _weights(g.n, 12)
        L = np.diag(l)
        kw = dict(l=l)
    lam, lam_tik = 1e-3, 0.5
    *_, (_, x_M, _) = tik.run(src, sched, r=g.n_views - 1, lam=lam, lam_tik=lam_tik,
                              n_blocks=g.n_views, form=form, **kw)
    # Eq. (TLS1) with the regulariser lam_tik^2 + lambda, by a least-squares solve
    stacked = np.vstack([A.toarray(), np.sqrt(lam_tik ** 2 + lam) * L])
    want, *_ = np.linalg.lstsq(stacked, np.concatenate([b, np.zeros(g.n)]), rcond=None)
    assert np.linalg.norm(x_M - want) <= 1e-9 * np.linalg.norm(want)


def test_no_tikhonov_term_is_the_slimls_step():
    g, A, b = _tiny_tomo(seed=13)
    src = slim.tomo_source(g, b)
    sched = list(slim.view_schedule(g, 13, 8))
    a = [x for _, x, _ in tik.run(src, sched, 3, 1e-2, 0.0, g.n_views, ramp=True)]
    c = [x for _, x, _ in slim.run(src, sched, 3, 1e-2, ramp=True)]
    for xa, xc in zip(a, c):
        assert np.linalg.norm(xa - xc) <= 1e-12 * np.linalg.norm(xc)


def test_single_row_sherman_morrison():
    A, _, b = workloads.gaussian_problem(3, m=40, n=12)
    src = slim.dense_source(A, b)
    lam, lam_tik, n_blocks = 0.2, 0.9, 40
    beta = lam_tik ** 2 / n_blocks
    mu = lam + beta                                    # r = 0: one block in the window
    sched = [np.array([i]) for i in (3, 17, 3, 8, 30)]
    x = np.zeros(12)
    for (_, xk, _), ids in zip(tik.run(src, sched, 0, lam, lam_tik, n_blocks), sched):
        a = A[ids[0]]
        grad = a * (a @ x - b[ids[0]]) + beta * x
        s = (grad - a * (a @ grad) / (mu + a @ a)) / mu
        x = x - s
        assert np.linalg.norm(xk - x) <= 1e-12 * np.linalg.norm(x)


def test_printed_count_is_the_window_count_with_lower_damping():
    g, A, b = _tiny_tomo(seed=14)
    src = slim.tomo_source(g, b)
    r, lam, lam_tik = 2, 0.2, 0.9
    beta = lam_tik ** 2 / g.n_views
    mem = [src.rows(slim.view_block_ids(g, 14, k)) for k in (1, 2, 3)]
    b_new = src.rhs(slim.view_block_ids(g, 14, 3))
    x = np.random.default_rng(15).standard_normal(g.n) * 0.1
    l = _weights(g.n, 16)
    xp, *_ = tik.step_woodbury(x, mem, b_new, lam, lam_tik, g.n_views, tik.window_count(3, r,
                               "printed"), l)
    xw, *_ = tik.step_woodbury(x, mem, b_new, lam - beta, lam_tik, g.n_views,
                               tik.window_count(3, r, "window"), l)
    assert np.linalg.norm(xp - xw) <= 1e-12 * np.linalg.norm(xw)


def test_planted_mutations_break_the_pins(monkeypatch):
    g, A, b = _tiny_tomo(seed=7)
    src = slim.tomo_source(g, b)
    rng = np.random.default_rng(8)
    sched = [g.view_rays(int(v)) for v in rng.integers(0, g.n_views, 6)]
    l = _weights(g.n, 9)
    P = np.diag(l * l)
    lam, lam_tik = 3e-2, 0.6
    x0 = rng.standard_normal(g.n) * 0.1

    def worst():
        xs = [x for _, x, _ in tik.run(src, sched, r=len(sched), lam=lam, lam_tik=lam_tik,
                                       n_blocks=g.n_views, x0=x0, form="direct", l=l)]
        return _full_memory_identity(src, A, sched, lam, lam_tik, g.n_views, P, x0, xs)

    assert worst() < 1e-11
    real_gradient = tik.gradient
    # the gradient of the Tikhonov rows dropped
    monkeypatch.setattr(tik, "gradient", lambda A_k, r_k, P_, x, beta: A_k.T @ r_k)
    assert worst() > 1e-4
    monkeypatch.setattr(tik, "gradient", real_gradient)
    # the count fixed at r+1 in the growing window
    monkeypatch.setattr(tik, "window_count", lambda k, r, reading="window": r + 1)
    assert worst() > 1e-4


def _bidiag(n, N, seed):
    # the first difference along the image rows plus a multiple of the identity
    rs = np.random.default_rng(seed)
    d0 = 1.0 + 0.5 * rs.random(n)
    d1 = -0.8 * (0.5 + 0.5 * rs.random(n))
    d1[::N] = 0.0                      # no coupling across image rows
    return d0, d1


def test_bidiagonal_matrix_is_the_stated_operator():
    g, A, b = _tiny_tomo()
    d0, d1 = _bidiag(g.n, g.N, 1)
    L = tik.bidiagonal(d0, d1).toarray()
    x = np.random.default_rng(2).standard_normal(g.n)
    want = d0 * x + d1 * np.concatenate([[0.0], x[:-1]])
    assert np.allclose(L @ x, want, rtol=0, atol=1e-15)
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.tril(L, -2), 0)


@pytest.mark.parametrize("lam_tik", [0.0, 0.7])
def test_general_woodbury_equals_direct(lam_tik):
    # the Woodbury algebra with W = (L^T L)^{-1} for a non-diagonal L, step by
    # step against Eq. (slimTik) as written
    g, A, b = _tiny_tomo()
    src = slim.tomo_source(g, b)
    r, lam = 2, 1e-2
    L = tik.bidiagonal(*_bidiag(g.n, g.N, 3))
    x = np.random.default_rng(5).standard_normal(g.n) * 0.1
    mem = []
    for k, ids in enumerate(slim.view_schedule(g, 4, 7), start=1):
        mem = (mem + [src.rows(ids)])[-(r + 1):]
        cnt = tik.window_count(k, r)
        xd, *_ = tik.step_direct(x, mem, src.rhs(ids), lam, lam_tik, g.n_views, cnt, L, 0.9)
        xw, *_ = tik.step_woodbury_general(x, mem, src.rhs(ids), lam, lam_tik, g.n_views, cnt, L,
                                          0.9)
        assert np.linalg.norm(xw - xd) <= 1e-10 * np.linalg.norm(xd), k
        x = xd
