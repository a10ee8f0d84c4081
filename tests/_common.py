"""Shared helpers for the GPU parity tests: seeded inputs and oracle references."""
import numpy as np

import workloads
from oracle import joseph, slim as oslim


def tomo_problem(cfg):
    """(geometry, A (csr), x_true, b) with b = A x_true + noise, all from the oracle side."""
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ x_true, e, cfg.noise)
    return g, A, x_true, b


def oracle_memory(g, seed, k, r, cyclic=False):
    """Row-id blocks of S_k (oldest first) and their ring slots, as the oracle draws them."""
    ks = list(range(max(1, k - r), k + 1))
    return [(kk, (kk - 1) % (r + 1), oslim.view_block_ids(g, seed, kk, cyclic)) for kk in ks]


def oracle_step_from(g, src, seed, k, r, lam, x_prev, ramp=False, eta=1.0, cyclic=False):
    """x_k from x_{k-1} with the memory of step k (Woodbury form, float64)."""
    mem = oracle_memory(g, seed, k, r, cyclic)
    blocks = [src.rows(ids) for _, _, ids in mem]
    lam_k = oslim.damping(lam, k, r, ramp)
    x, r_k, s, z = oslim.step_woodbury(x_prev, blocks, src.rhs(mem[-1][2]), lam_k, eta)
    return x, mem


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))
