"""Learned initial guess for the 256 x 256 workload: training pairs produced by
the method itself, training of the U-Net, and the held-out evaluation of
steps to a relative error with x_0 from the network versus x_0 = 0.

Argument marshalling and loops only: the projector, the iterations, the
network's forward, backward and optimiser all run in the library's kernels.
PyTorch provides device memory for the pairs and the norms of the metric.
"""
from __future__ import annotations

import time

import numpy as np

import workloads

from . import slim as sl


def _stream(torch):
    """Handle of torch's current stream, which must not be the default one:
    the library reads handle 0 as "the context's own stream", whose work
    would not be ordered with the tensors PyTorch forms around it."""
    h = torch.cuda.current_stream().cuda_stream
    if h == 0:
        raise RuntimeError("run the warm-start driver under a non-default torch stream "
                           "(with torch.cuda.stream(torch.cuda.Stream()): ...)")
    return h


def _solver(cfg, torch, lookahead=3):
    """Chosen form on the caller's current stream, so that the library's work
    and the tensors PyTorch forms around it are ordered."""
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, cfg.seed,
                precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED, refine_iters=2,
                use_graph=True, lookahead=lookahead)
    s.set_stream(_stream(torch))
    return s


def make_data(s, cfg, seed, torch):
    """b = A x_true + noise (noise level cfg.noise) for phantom `seed`, on the
    device (the context runs on the caller's stream)."""
    x_true = torch.tensor(workloads.phantom_2d(cfg.N, seed, cfg.n_ellipses), dtype=torch.float32,
                          device="cuda")
    y = torch.zeros(cfg.m, dtype=torch.float32, device="cuda")
    s.project(x_true, y)
    e = torch.tensor(workloads.noise_direction(cfg.m, seed), dtype=torch.float32, device="cuda")
    return y + cfg.noise * torch.linalg.norm(y) * e / torch.linalg.norm(e), x_true


def restart(s, b, torch):
    """Load data b and start the iteration afresh from x = 0."""
    s.set_data(b)
    s.set_x(torch.zeros(s.n, dtype=torch.float32, device="cuda"))
    s.set_iter(0)


def make_pairs(cfg, seeds, epochs, torch, check_every=100, log=None):
    """Inputs A^T b and targets x_E (the method's iterate after `epochs` epochs
    from x_0 = 0, float32 chosen form) for every seed.  Every `check_every`-th
    target is re-run with the float64 form; returns the largest relative
    difference seen."""
    s = _solver(cfg, torch)
    n, steps = cfg.n, epochs * cfg.n_views
    X = torch.empty((len(seeds), n), dtype=torch.float32, device="cuda")
    Y = torch.empty((len(seeds), n), dtype=torch.float32, device="cuda")
    check = None
    worst = 0.0
    t0 = time.perf_counter()
    for i, seed in enumerate(seeds):
        b, _ = make_data(s, cfg, seed, torch)
        restart(s, b, torch)
        s.backproject_data(X[i])
        s.step(steps)
        s.get_x(Y[i])
        if check_every and i % check_every == 0:
            if check is None:
                check = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, cfg.seed)
                check.set_stream(_stream(torch))
            bd = b.double()
            check.set_data(bd)
            check.set_x(torch.zeros(n, dtype=torch.float64, device="cuda"))
            check.set_iter(0)
            check.step(steps)
            x64 = check.get_x()
            worst = max(worst, float(np.linalg.norm(Y[i].double().cpu().numpy() - x64) /
                                     np.linalg.norm(x64)))
        if log and (i + 1) % 200 == 0:
            log(f"pairs {i + 1}/{len(seeds)}  {time.perf_counter() - t0:.1f}s")
    s.close()
    if check is not None:
        check.close()
    return X, Y, worst


def train(net, X, Y, s_in, epochs, batch, lr, torch, seed=0, log=None):
    """Adam on the mean squared error between net(s_in A^T b) and the targets."""
    rng = np.random.default_rng(seed)
    count = X.shape[0]
    losses = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = torch.tensor(rng.permutation(count), device="cuda")
        tot = 0.0
        for j in range(0, count - batch + 1, batch):
            idx = order[j:j + batch]
            xb = (X[idx] * s_in).contiguous()
            yb = Y[idx].contiguous()
            tot += net.train_step(xb.view(-1), yb.view(-1), lr, _stream(torch)) * batch
        losses.append(tot / (count - count % batch))
        if log:
            log(f"epoch {ep + 1}/{epochs}  loss {losses[-1]:.4e}  {time.perf_counter() - t0:.1f}s")
    return losses, time.perf_counter() - t0


def steps_to(s, x_ref, thresholds, max_steps, every, torch):
    """Relative error ||x_k - x_ref|| / ||x_ref|| checked every `every` steps up
    to max_steps: the first step below each threshold, the error at the start,
    the smallest error seen and its step, and the error at the end."""
    xb = torch.empty(s.n, dtype=torch.float32, device="cuda")
    nref = float(torch.linalg.norm(x_ref))
    first = {th: None for th in thresholds}
    k = 0
    s.get_x(xb)
    err = err0 = float(torch.linalg.norm(xb - x_ref)) / nref
    best, best_k = err0, 0
    for th in thresholds:
        if err0 <= th:
            first[th] = 0
    while k < max_steps:
        s.step(every)
        k += every
        s.get_x(xb)
        err = float(torch.linalg.norm(xb - x_ref)) / nref
        if err < best:
            best, best_k = err, k
        for th in thresholds:
            if first[th] is None and err <= th:
                first[th] = k
    return {"first": first, "err0": err0, "best": best, "best_step": best_k, "final": err}


def evaluate(net, cfg, seeds, s_in, max_epochs, thresholds, torch, every=6, log=None):
    """Per held-out seed: steps until ||x_k - x_true|| / ||x_true|| falls below
    each threshold, from x_0 = 0 and from the warm start, within max_epochs;
    the warm start's residual ratio and whether it was used."""
    s = _solver(cfg, torch)
    M = cfg.n_views
    out = []
    t_net = []
    for i, seed in enumerate(seeds):
        b, x_true = make_data(s, cfg, seed, torch)
        rec = {"seed": seed}
        restart(s, b, torch)
        rec["zero"] = steps_to(s, x_true, thresholds, max_epochs * M, every, torch)
        restart(s, b, torch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        used, ratio = s.warm_start(net, s_in, 1.0)
        t_net.append(time.perf_counter() - t0)
        s.set_iter(0)
        rec["warm"] = steps_to(s, x_true, thresholds, max_epochs * M, every, torch)
        rec["used"], rec["ratio"] = used, ratio
        out.append(rec)
        if log and (i + 1) % 20 == 0:
            log(f"eval {i + 1}/{len(seeds)}")
    s.close()
    return out, float(np.median(t_net))


def summarize(recs, thresholds):
    med = lambda v: float(np.median(v)) if len(v) else None
    res = {"thresholds": {}}
    for th in thresholds:
        z = [r["zero"]["first"][th] for r in recs if r["zero"]["first"][th] is not None]
        w = [r["warm"]["first"][th] for r in recs if r["warm"]["first"][th] is not None]
        res["thresholds"][str(th)] = {"median_steps_zero": med(z), "median_steps_warm": med(w),
                                      "reached_zero": len(z), "reached_warm": len(w)}
    for start in ("zero", "warm"):
        res[start] = {k: med([r[start][k] for r in recs])
                      for k in ("err0", "best", "best_step", "final")}
    res["used_fraction"] = float(np.mean([r["used"] for r in recs]))
    res["median_residual_ratio"] = med([r["ratio"] for r in recs])
    return res


def input_scale(X):
    """Scale that brings the back-projections to unit RMS (one constant for all)."""
    rms = float((X * X).mean().sqrt())
    return 1.0 / rms if rms > 0 else 1.0
