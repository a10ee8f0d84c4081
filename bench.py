#!/usr/bin/env python
"""Benchmark of the slimLS hot path on one GB300 (or N replicas).

Metric: sampled rows/s (ell rows per step) of the chosen form on the
256x256 / 180-view / 363-bin workload (r = 5, lambda = 1e-3), next to the
plain float64 form on the same seeds, plus time-to-accuracy of both.

  chosen form: float32 projector/residual/scatter, float64 Gram, float32 tiled
               Cholesky + float64-residual refinement, one CUDA graph per step
  plain form:  float64 everywhere, float64 tiled Cholesky, per-kernel launches

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
stream the library launches on, with a 256 MiB write between steps to flush
L2 (129 MB).  Per-phase times come from the library's own event records
inside the same timed steps.  One JSON line on rank 0.

`--impl reference` times the FP64 CPU oracle (the reference arm) instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "sampled rows/s & time to 1e-2 rel. error: plain FP64 vs chosen form, 1 GB300"
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2          # measured: 1.19 TFLOP/s FP64 FMA at 152 SMs
NUM_SMS = 152
MAX_SM_MHZ = 2070.0


def workload_of(name):
    cfg = {"precision-256": workloads.C2, "plain-64": workloads.C1}[name]
    desc = (f"{cfg.name}: {cfg.N}x{cfg.N} image (n={cfg.n}), {cfg.n_views} views x {cfg.det} bins "
            f"(m={cfg.m}), one view per block (ell={cfg.ell}), r={cfg.r}, lambda={cfg.lam:g}, "
            f"seed {cfg.seed}, 10 random ellipses, 1% noise")
    return cfg, desc


# --------------------------------------------------------------------------- CPU oracle leg
def cpu_leg(args):
    """Times the FP64 oracle (single BLAS thread); prints one JSON object."""
    from oracle import joseph, slim as oslim
    cfg, _ = workload_of(args.workload)
    g = joseph.Geometry(cfg.N, cfg.n_views, cfg.det)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    A = joseph.full_matrix(g)
    b = workloads.add_noise(A @ x_true, e, cfg.noise)
    src = oslim.tomo_source(g, b)
    sched = oslim.view_schedule(g, cfg.seed, 10 ** 9)
    runner = oslim.run(src, sched, cfg.r, cfg.lam)
    for _ in range(args.cpu_warmup):
        next(runner)
    t0 = time.perf_counter()
    steps = 0
    while True:
        next(runner)
        steps += 1
        el = time.perf_counter() - t0
        if (args.cpu_steps and steps >= args.cpu_steps) or (not args.cpu_steps and el >= args.cpu_seconds):
            break
    el = time.perf_counter() - t0
    print(json.dumps({"rows_per_s": cfg.ell * steps / el, "steps": steps, "seconds": el,
                      "warmup": args.cpu_warmup}))


def run_cpu_leg(args, steps=0, warmup=None, threads=1):
    """The oracle leg in a subprocess with `threads` BLAS/OpenMP threads."""
    t = str(threads)
    env = dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload", args.workload,
           "--cpu-seconds", str(args.cpu_seconds), "--cpu-steps", str(steps),
           "--cpu-warmup", str(args.r_warm if warmup is None else warmup)]
    res = subprocess.run(cmd, capture_output=True, text=True, env=env)
    if res.returncode != 0:
        raise RuntimeError("cpu leg failed:\n" + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------------------- GPU helpers
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def make_b(sl, cfg, x_true, e):
    """b = A x_true + noise, with A x_true from the library's projector (float64)."""
    import torch
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, cfg.seed)
    xt = torch.tensor(x_true, dtype=torch.float64, device="cuda")
    y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()   # inputs filled on torch's stream; the context has its own
    s.project(xt, y)
    torch.cuda.synchronize()
    clean = y.cpu().numpy()
    s.close()
    return workloads.add_noise(clean, e, cfg.noise)


CHOSEN_SOLVER = "mixed_inv"   # set from --solver
# slimTik runs the triangular-sweep solve (the inverse forms take no slimTik
# terms), pipelined as that solve is fastest: six steps ahead, one
# factorisation CTA per SM
SWEEP_LOOKAHEAD, SWEEP_CTAS = 6, 1

FORM_OF_SOLVER = {
    "mixed_inv": ("float32 tiled Cholesky, its inverse L^-1 formed on the tcgen05 tensor cores "
                  "(float32-accurate split-bfloat16 products), the solves as products with L^-1, "
                  "2 float64-residual refinements"),
    "mixed": "float32 tiled Cholesky + triangular sweeps, 2 float64-residual refinements",
    "mixed_tc": ("float32 Cholesky and its inverse on the tcgen05 tensor cores, the solves as "
                 "products with L^-1, 3 float64-residual refinements"),
}


def make_form(sl, cfg, form, seed, lookahead=0, ctas_per_sm=0, decay_after=0):
    """chosen: float32 projector/residual/scatter, float64 Gram, float32 factor
    (solved through its tensor-core inverse, or as --solver says when
    pipelined) refined against the float64 Gram; chosen_fp64_factor: the same
    pipeline with the float64 factor and solves the scope names (no
    refinement needed); plain: float64 everywhere, one kernel per phase, no
    graph."""
    if form in ("chosen", "chosen_fp64_factor"):
        mixed = form == "chosen"
        inverse = {"mixed_tc": sl.SLIM_SOLVE_MIXED_TC, "mixed_inv": sl.SLIM_SOLVE_MIXED_INV}
        solver = ((inverse[CHOSEN_SOLVER] if CHOSEN_SOLVER in inverse and lookahead
                   else sl.SLIM_SOLVE_MIXED) if mixed else sl.SLIM_SOLVE_FP64)
        refine = (3 if solver == sl.SLIM_SOLVE_MIXED_TC else 2) if mixed else 0
        return sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, seed,
                       precision=sl.SLIM_PREC_FP32, solver=solver,
                       refine_iters=refine, use_graph=True, lookahead=lookahead,
                       ctas_per_sm=ctas_per_sm, decay_after=decay_after)
    return sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, seed,
                   precision=sl.SLIM_PREC_FP64, solver=sl.SLIM_SOLVE_FP64, use_graph=False,
                   decay_after=decay_after)


def timed_steps(s, K, W, flush, stream, snapshot_every=0, snap_dtype=None, accum_last=0):
    """Run W untimed then K timed steps; returns (ms per step list, phase-ms sums, snapshots)."""
    import torch
    s.set_stream(stream.cuda_stream)
    s.set_timing(True)
    for i in range(W):
        flush.fill_(i)
        s.step(1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    per = []
    phases = None
    snaps = []
    xs = None
    xbuf = torch.empty(s.n, dtype=snap_dtype or torch.float64, device="cuda") if (
        snapshot_every or accum_last) else None
    for i in range(K):
        flush.fill_(i + W)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))
        ph, _ = s.get_timing()
        phases = ph if phases is None else {k: phases[k] + ph[k] for k in ph}
        if snapshot_every and (i + 1) % snapshot_every == 0:
            s.get_x(xbuf)
            snaps.append((i + 1, float(sum(per)), xbuf.double().clone()))
        if accum_last and i >= K - accum_last:
            s.get_x(xbuf)
            xs = xbuf.double().clone() if xs is None else xs + xbuf.double()
    s.set_timing(False)
    return per, phases, snaps, xs


def timed_region(s, K, W, flush, stream, snapshot_every=0, snap_dtype=None):
    """Pipelined form: W untimed steps, a synchronisation, then K steps timed as
    one region on the caller's stream (an event after every step, no
    synchronisation inside, the L2 flush between steps inside the region).
    The region ends once the caller's stream has joined every stream of the
    context, so it holds exactly K steps of the whole pipeline: K iterate
    chains, and K geometry chains and factorisations (the D prepared during
    the warm-up are matched by the D prepared ahead at the end).  The
    factorisation launches and iterate chains of the region are timed by the
    library's launch log.
    Returns (ms per step list, launch log, snapshots, region ms)."""
    import torch
    s.set_stream(stream.cuda_stream)
    s.set_timing(True)
    for i in range(W):
        flush.fill_(i)
        s.step(1)
    s.sync()
    s.launch_log()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 2)]
    snaps = []
    evs[0].record(stream)
    for i in range(K):
        flush.fill_(i + W)
        s.step(1)
        evs[i + 1].record(stream)
        if snapshot_every and (i + 1) % snapshot_every == 0:
            xb = torch.empty(s.n, dtype=snap_dtype or torch.float32, device="cuda")
            s.get_x(xb)
            snaps.append((i + 1, xb))
    s.join(stream.cuda_stream)
    evs[-1].record(stream)
    evs[-1].synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(K)]
    region_ms = evs[0].elapsed_time(evs[-1])
    f_ms, x_ms, n = s.launch_log()
    s.set_timing(False)
    cum = np.cumsum(per)
    snaps = [(k, float(cum[k - 1]), x.double()) for k, x in snaps]
    return per, {"factor_launch_ms": f_ms, "iterate_chain_ms": x_ms, "chains": n}, snaps, region_ms


def chol_flops(p):
    return p ** 3 / 3.0


def roofline_of(phases_ms, K, p, ell, N, form, clocks_mhz):
    """Roofline of the dominant phase (largest share of step time)."""
    tot = {k: v / K for k, v in phases_ms.items()}
    dom = max(tot, key=tot.get)
    t = tot[dom] * 1e-3
    if dom in ("factor",):
        flops = chol_flops(p)
        if form == "chosen":
            peak = NUM_SMS * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
            note = "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz"
        else:
            peak = NUM_SMS * FP64_FMA_PER_SM_CLK * 2 * MAX_SM_MHZ * 1e6 / 1e12
            note = "FP64 FMA: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz"
        ach = flops / t / 1e12
        return {"kernel": "chol_factor_kernel", "phase": dom, "bound": "alu", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "algorithmic": f"p^3/3 = {flops:.4g} flop per launch (p = {p})",
                "peak_source": note, "share_of_step": tot[dom] / sum(tot.values())}
    if dom == "solve":
        # triangular solves + refinement residuals: bytes of L (read twice per solve) and G
        es = 4 if form == "chosen" else 8
        solves = 3 if form == "chosen" else 1
        byts = solves * 2 * (p * p / 2) * es + (2 * p * p * 8 if form == "chosen" else 0)
        ach = byts / t / 1e9
        peak = hbm_peak()
        return {"kernel": "chol_fwd/bwd_kernel", "phase": dom, "bound": "hbm", "achieved": ach,
                "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "algorithmic": f"{byts:.4g} bytes per step", "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                "share_of_step": tot[dom] / sum(tot.values())}
    byts = {"forward_residual": ell * 2 * N * (4 + 12), "gram_update": (ell * 6) * 2 * N * 12,
            "scatter": ell * 6 * 2 * N * 20, "form_k": p * p * 12}.get(dom, 0)
    ach = byts / t / 1e9
    return {"kernel": dom, "phase": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak(),
            "unit": "GB/s", "frac": ach / hbm_peak(), "traffic": None,
            "algorithmic": f"{byts} bytes per step", "peak_source": "MEASURED_PEAKS.json hbm_gbs",
            "share_of_step": tot[dom] / sum(tot.values())}


def traffic_from_profiles(kernel):
    """dram bytes per launch recorded from an ncu capture (profiles/traffic.json), or
    None when the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get("kernels", {}).get(kernel)
    if not rec:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update(open(os.path.join(ROOT, "paper_1912_07962_gb300", "csrc", f), "rb").read())
    return rec["bytes"] if h.hexdigest() == rec["sha256"] else None


def tta_block(sl, cfg, b, flush, stream, epochs, thresholds, lookahead=0, ctas_per_sm=0,
              decay_after=0):
    """Time to relative-error thresholds, plain float64 form against the chosen
    form, on the same seed (the same blocks).  The reference x_ref is the
    pre-registered fallback reading of the time-to-accuracy reference: the
    mean of the float64 iterates over the final epoch of the plain run (the
    float64 GPU iterates, which match the float64 oracle's per step to 1e-12;
    the oracle itself takes about 0.4 s per step here).  `decay_after` > 0
    runs both forms with the decaying damping of the end of Sec. 3,
    lambda_k = lambda k / K after step K; x_ref is then that run's own
    final-epoch mean."""
    import torch
    M = cfg.n_views
    steps = epochs * M
    every = max(1, M // 10)
    out = {}
    res = {}
    x_ref = None
    for form in ("plain", "chosen"):
        s = make_form(sl, cfg, form, cfg.seed, lookahead=lookahead if form == "chosen" else 0,
                      ctas_per_sm=ctas_per_sm if form == "chosen" else 0,
                      decay_after=decay_after)
        s.set_data(b if form == "plain" else b.astype(np.float32))
        if form == "chosen" and lookahead:
            per, _, snaps, _ = timed_region(s, steps, 0, flush, stream, snapshot_every=every)
        else:
            per, _, snaps, xs = timed_steps(s, steps, 0, flush, stream, snapshot_every=every,
                                            snap_dtype=torch.float64 if form == "plain" else torch.float32,
                                            accum_last=M if form == "plain" else 0)
        if form == "plain":
            x_ref = xs / M
        res[form] = (per, snaps)
        s.close()
    nref = float(torch.linalg.norm(x_ref))
    for form, (per, snaps) in res.items():
        errs = [(k, ms, float(torch.linalg.norm(x - x_ref)) / nref) for k, ms, x in snaps]
        first = {}
        for th in thresholds:
            hit = next(((k, ms) for k, ms, e in errs if e <= th), None)
            first[str(th)] = None if hit is None else {"steps": hit[0], "seconds": hit[1] * 1e-3}
        kmin, msmin, emin = min(errs, key=lambda t: t[2])
        out[form] = {"first_below": first, "min_err": emin, "min_err_step": kmin,
                     "seconds_to_min_err": msmin * 1e-3, "seconds_total": sum(per) * 1e-3,
                     "steps_total": len(per)}
    common = [th for th in thresholds
              if out["plain"]["first_below"][str(th)] and out["chosen"]["first_below"][str(th)]]
    if common:
        th = min(common)
        tp = out["plain"]["first_below"][str(th)]["seconds"]
        tc = out["chosen"]["first_below"][str(th)]["seconds"]
        out["smallest_common_threshold"] = {"threshold": th, "plain_s": tp, "chosen_s": tc,
                                            "speedup": tp / tc}
    out["reference"] = (f"x_ref = mean of the float64 GPU iterates (plain form, per-step parity "
                        f"1e-12 with the float64 oracle) over epoch {epochs} (steps "
                        f"{(epochs - 1) * M + 1}..{epochs * M}), same seed")
    out["damping"] = ("constant lambda" if not decay_after else
                      f"lambda_k = lambda k / {decay_after} after step {decay_after} (1/k decay)")
    if out["plain"]["first_below"].get("0.01") is None:
        out["why_not_1e-2"] = ("the iterates jitter about their limit at a level set by the "
                               "damping (the horizon of Theorem 3.1(ii)); the 1/k decay shrinks "
                               "it only as 1/sqrt(k), so 1e-2 of the final-epoch mean is not "
                               "reached within the run")
    out["eval_every_steps"] = every
    return out


def l2_flush(flush, i):
    """Evict L2 before a timed HBM stream: write a buffer twice the L2's size,
    then read it back, so that the lines left in L2 are clean (a dirty line
    left by the write would be written back during the timed pass and take
    HBM bandwidth from it)."""
    flush.fill_(i)
    flush.sum()


def csr_block(sl, cfg, flush, stream, reps=20):
    """Full-A passes over the stored matrix (HBM streams): y = A x through the CSR
    and x += A^T y through the CSC copy, float32 and bfloat16 values."""
    import torch
    out = {}
    hbm = hbm_peak()
    for kind, mode, vs in (("f32", sl.A_CSR_F32, 4), ("bf16", sl.A_CSR_BF16, 2)):
        s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, cfg.seed,
                    precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED, a_mode=mode)
        s.set_stream(stream.cuda_stream)
        nnz = int(s.get_csr()[1].size)
        x = torch.rand(cfg.n, dtype=torch.float32, device="cuda")
        y = torch.rand(cfg.m, dtype=torch.float32, device="cuda")
        res = {"nnz": nnz}
        for name, fn, byts in (
                ("forward", lambda: s.project(x, y),
                 nnz * (4 + vs) + (cfg.m + 1) * 4 + cfg.n * 4 + cfg.m * 4),
                ("transpose", lambda: s.backproject(y, x),
                 nnz * (4 + vs) + (cfg.n + 1) * 4 + cfg.m * 4 + 2 * cfg.n * 4)):
            for i in range(3):
                l2_flush(flush, i)
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            tot = 0.0
            for i in range(reps):
                l2_flush(flush, i)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            ms = tot / reps
            gbs = byts / (ms * 1e-3) / 1e9
            res[name] = {"ms": ms, "algorithmic_bytes": byts, "GB_s": gbs, "frac_of_measured_hbm": gbs / hbm}
        out[kind] = res
        s.close()
    out["note"] = ("one pass over all 180 views; bytes = index + value arrays + row/col pointers + "
                   "vector reads/writes; L2 flushed between passes (256 MiB write, then a read of it "
                   "so that no dirty line is written back inside the timed pass); peak = measured "
                   "copy bandwidth")
    return out


def lsqr_block(sl, cfg, b, flush, stream, K, W, tol=1e-6, max_iter=5000):
    """The step of Eq. (slimLSstep) by LSQR instead of the Woodbury form, on
    the same workload: float64 iterate, each step timed alone with events
    after an L2 flush; iterations per step from the library.  Algorithmic
    bytes of one LSQR iteration: the window's tap rows read twice (pixel +
    float64 weight, 12 B per tap slot), the gathered v and the scattered
    M^T u (8 B per stored tap each), and the n-vectors of the two element
    passes (v, w, s, tmp: 9 reads or writes of 8 B per pixel)."""
    import torch
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, cfg.seed,
                precision=sl.SLIM_PREC_FP64, solver=sl.SLIM_SOLVE_LSQR, lsqr_max_iter=max_iter,
                lsqr_tol=tol)
    s.set_stream(stream.cuda_stream)
    s.set_data(b)
    for i in range(W):
        flush.fill_(i)
        s.step(1)
    torch.cuda.synchronize()
    ms, its = [], []
    for i in range(K):
        flush.fill_(i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(s.lsqr_info()[0])
    s.close()
    tot_ms, tot_it = sum(ms), sum(its)
    taps = 2 * cfg.N
    stored = 0.85 * taps          # stored taps per ray (about 2N x 0.85 for this geometry)
    p = (cfg.r + 1) * cfg.ell
    byts = p * taps * 12 * 2 + p * stored * 8 * 2 + cfg.n * 8 * 9
    gbs = byts * tot_it / (tot_ms * 1e-3) / 1e9
    hbm = hbm_peak()
    return {"workload": f"{cfg.name}, step by LSQR to ||M^T r - lambda s|| <= {tol:g} ||M^T c||",
            "rows_per_s": cfg.ell * K / (tot_ms * 1e-3), "ms_per_step": tot_ms / K,
            "iterations_per_step": tot_it / K, "iterations_min_max": [min(its), max(its)],
            "us_per_iteration": tot_ms * 1e3 / max(tot_it, 1), "steps": K, "warmup": W,
            "algorithmic_bytes_per_iteration": byts, "GB_s": gbs,
            "frac_of_measured_hbm": gbs / hbm,
            "note": ("one cooperative launch per step (two grid-wide sums per iteration); the "
                     "window's taps and vectors are L2-resident, so the fraction is of the HBM "
                     "copy peak for scale only")}


def tik_block(sl, cfg, b, flush, stream, K, W, lam_tik=1.0, lookahead=6, ctas_per_sm=1):
    """slimTik (Eq. slimTik, C_k = diag(c)) on the same workload, against
    slimLS in the same form and timing: float32 iterate, float64 Gram
    M C^{-1} M^T, float32 tiled Cholesky + 2 float64-residual refinements;
    one CUDA graph per step (lookahead 0, each step timed alone, with its
    phases) and the pipelined form (the headline's timing: K steps in one
    region after W warm-up steps).  c is seeded uniform in [0.5, 2];
    beta = lam_tik^2 / A_v."""
    c = 0.5 + 1.5 * np.random.default_rng(cfg.seed).random(cfg.n)
    out = {"workload": f"{cfg.name}, slimTik with lam_tik = {lam_tik:g}, C_k = diag(c)",
           "steps": K, "warmup": W}
    for name, lt in (("slimls", 0.0), ("slimtik", lam_tik)):
        row = {}
        for la in (0, lookahead):
            s = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, cfg.r, cfg.lam, cfg.seed,
                        precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED, refine_iters=2,
                        use_graph=True, tik_lambda=lt, lookahead=la,
                        ctas_per_sm=ctas_per_sm if la else 0)
            s.set_data(b.astype(np.float32))
            if lt > 0:
                s.set_c_diag(c)
            if la:
                _, _, _, reg = timed_region(s, K, W, flush, stream)
                row[f"lookahead_{la}"] = {"rows_per_s": cfg.ell * K / (reg * 1e-3),
                                          "ms_per_step": reg / K}
            else:
                per, ph, _, _ = timed_steps(s, K, W, flush, stream)
                row["lookahead_0"] = {"rows_per_s": cfg.ell * K / (sum(per) * 1e-3),
                                      "ms_per_step": sum(per) / K,
                                      "phase_ms": {k: v / K for k, v in ph.items()},
                                      "kernels_per_step": s.kernels_per_step()}
            s.close()
        out[name] = row
    for key in out["slimls"]:
        out[f"overhead_{key}"] = (out["slimtik"][key]["ms_per_step"] /
                                  out["slimls"][key]["ms_per_step"] - 1.0)
    return out


def sensitivity_block(sl, flush, stream, reps=5, K=30, W=3, memory=10):
    """Step-size sensitivity of slimLS (r = 0), sg and olbfgs (the comparison of
    Sec. 4.1, here on the synthetic 64x64 tomography workload): the relative
    reconstruction error to the phantom x_true after one epoch (60 view
    blocks) for alpha = 1e-5 .. 1e3, the step size of sg and olbfgs and the
    damping 1/lambda of slimLS; median and 5-95th percentiles over `reps`
    block sequences.  (Against x_LS every method sits near 1 after one epoch:
    this problem is ill-posed and x_LS carries the amplified noise.)  Also the
    device time of one step of each method on the 256x256 workload."""
    import torch
    cfg = workloads.C1
    out = {"workload": f"{cfg.name}: one epoch ({cfg.n_views} view blocks), r = 0, "
                       "error to the phantom", "reps": reps, "olbfgs_memory": memory}
    methods = {"slimls_r0": sl.SLIM_SOLVE_FP64, "sg": sl.SLIM_SOLVE_SG,
               "olbfgs": sl.SLIM_SOLVE_OLBFGS}
    if reps > 0:
        out.update(_sensitivity_sweep(sl, cfg, methods, reps, memory))
    # device time of one step at 256x256 (float64 iterate, each step timed alone)
    big = workloads.C2
    xt2, e2 = workloads.tomo_inputs_2d(big)
    b2 = make_b(sl, big, xt2, e2)
    cost = {}
    for name, solver in methods.items():
        c = sl.Slim(big.N, big.n_views, big.det, big.ell, 0, 1e3, big.seed, solver=solver,
                    olbfgs_memory=memory, use_graph=solver != sl.SLIM_SOLVE_OLBFGS)
        c.set_data(b2)
        per, _, _, _ = timed_steps(c, K, W, flush, stream)
        c.close()
        cost[name] = {"ms_per_step": sum(per) / K, "rows_per_s": big.ell * K / (sum(per) * 1e-3)}
    out["step_cost_256"] = cost
    return out


def _sensitivity_sweep(sl, cfg, methods, reps, memory):
    """The error after one epoch for every method and step size (see
    sensitivity_block)."""
    import torch
    x_true, e = workloads.tomo_inputs_2d(cfg)
    b = make_b(sl, cfg, x_true, e)
    xt = torch.tensor(x_true, dtype=torch.float64, device="cuda")
    n_true = float(torch.linalg.norm(xt))
    alphas = [10.0 ** p for p in range(-5, 4)]
    out = {"alpha": alphas}
    xb = torch.empty(cfg.n, dtype=torch.float64, device="cuda")
    for name, solver in methods.items():
        rows = []
        for alpha in alphas:
            errs = []
            for rep in range(reps):
                c = sl.Slim(cfg.N, cfg.n_views, cfg.det, cfg.ell, 0, 1.0 / alpha, 1000 + rep,
                            solver=solver, olbfgs_memory=memory,
                            use_graph=solver != sl.SLIM_SOLVE_OLBFGS)
                c.set_data(b)
                try:
                    c.step(cfg.n_views)
                    c.get_x(xb)
                    err = float(torch.linalg.norm(xb - xt)) / n_true
                except sl.SlimError:
                    err = float("inf")
                c.close()
                errs.append(err if np.isfinite(err) else float("inf"))
            with np.errstate(invalid="ignore"):   # diverged runs are inf
                q = np.percentile(np.array(errs), [5, 50, 95])

            def fin(v):   # JSON has no infinity: a diverged run reads as null
                return float(v) if np.isfinite(v) else None
            rows.append({"alpha": alpha, "median": fin(q[1]), "p5": fin(q[0]), "p95": fin(q[2]),
                         "diverged": int(sum(not np.isfinite(v) for v in errs))})
        out[name] = rows
    return out


def stream3d_block(sl, flush, stream, K, W, steps_per_view=46):
    """The 3D streaming form at 256^3: float32 volume, random rays from the views
    that have arrived, float64 per-slice solves, one CUDA graph per step."""
    import torch
    cfg = workloads.C4
    x_true = workloads.phantom_3d(cfg.N, cfg.seed, cfg.n_ellipsoids, dtype=np.float32)
    s = sl.Slim(cfg.N, cfg.n_views, cfg.det_u, cfg.ell, cfg.r, cfg.lam, cfg.seed,
                precision=sl.SLIM_PREC_FP32, dim=3, det_v=cfg.det_v, kind=sl.SLIM_BLOCKS_STREAM,
                steps_per_view=steps_per_view, use_graph=True)
    xt = torch.tensor(x_true, device="cuda")
    y = torch.zeros(cfg.m, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()   # inputs filled on torch's stream; the context has its own
    s.project(xt, y)
    torch.cuda.synchronize()
    # the matrix-free full-view pass y = A x over all m rays (the scope's
    # projector roofline case): timed alone after an L2 flush, on the
    # context's stream; algorithmic bytes 4 B per float32 tap gathered (2 live
    # taps per step, N steps per ray) plus 4 B per ray written
    full = None
    s.set_stream(stream.cuda_stream)
    reps = 3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    for i in range(reps):
        l2_flush(flush, i)
        ev[2 * i].record(stream)
        s.project(xt, y)
        ev[2 * i + 1].record(stream)
    ev[-1].synchronize()
    ms = min(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps))
    byts = cfg.m * cfg.N * 2 * 4 + cfg.m * 4
    full = {"rays": cfg.m, "ms": ms, "algorithmic_bytes": byts, "GB_s": byts / (ms * 1e-3) / 1e9,
            "frac_of_measured_hbm": byts / (ms * 1e-3) / 1e9 / hbm_peak(),
            "note": ("best of 3 passes after an L2 flush; the float32 volume (67 MB) fits the "
                     "129 MB L2, so most tap gathers hit L2 and the fraction is of HBM by the "
                     "scope's byte count, not DRAM traffic")}
    e = torch.tensor(workloads.noise_direction(cfg.m, cfg.seed), dtype=torch.float32, device="cuda")
    b = y + cfg.noise * torch.linalg.norm(y) * e / torch.linalg.norm(e)
    torch.cuda.synchronize()     # b is formed on torch's stream, copied on the context's
    del xt, e, y
    s.set_data(b)
    per, ph, _, _ = timed_steps(s, K, W, flush, stream)
    s.close()
    t = sum(per) * 1e-3
    phases = {k: v / K for k, v in ph.items()}
    names = {"sample": "sample", "forward_residual": "ray march + residual",
             "gram_update": "slice lists + same-slice Gram pairs", "factor": "per-slice float64 solves",
             "scatter": "scatter into the volume"}
    dom = max(phases, key=phases.get)
    # algorithmic bytes of the ray march and the scatter (2 taps per step, N steps per ray)
    taps_new = cfg.ell * 2 * cfg.N
    taps_all = (cfg.r + 1) * cfg.ell * 2 * cfg.N
    alg = {"forward_residual": taps_new * (4 + 4 + 8),       # x gather + ring index + weight
           "scatter": taps_all * (4 + 8 + 8)}                 # ring index + weight + x RMW
    rl = None
    if dom in alg:
        gbs = alg[dom] / (phases[dom] * 1e-3) / 1e9
        rl = {"phase": dom, "bound": "hbm", "achieved": gbs, "peak": hbm_peak(), "unit": "GB/s",
              "frac": gbs / hbm_peak(), "algorithmic": f"{alg[dom]} bytes per step"}
    return {"workload": f"{cfg.name}: {cfg.N}^3 volume, {cfg.n_views} views x {cfg.det_v}x{cfg.det_u} "
                        f"detector (m={cfg.m}), ell={cfg.ell} random rays from arrived views "
                        f"(one view every {steps_per_view} steps), r={cfg.r}, lambda={cfg.lam:g}",
            "rows_per_s": cfg.ell * K / t, "ms_per_step": t / K * 1e3, "steps": K, "warmup": W,
            "phases_ms": {names.get(k, k): v for k, v in phases.items()}, "dominant": names.get(dom, dom),
            "roofline": rl, "full_view_pass": full}


def frames3d_block(sl, flush, stream, K, W, r_values=(0, 4), steps_per_view=46):
    """3D with views from random directions (Sec. 4.3's geometry) at 256^3:
    360 directions uniform on the sphere, a 368 x 368 detector, ell = 2048
    random rays from the arrived views; float32 volume, float64 Gram from the
    voxel lists, float32 tiled Cholesky + 2 float64 refinements (the window's
    rays cross every slice, so the Gram matrix is dense in general), one CUDA
    graph per step.  r = 0 is the paper's 3D setting, r = 4 the memory of the
    streaming workload (p = 10,240)."""
    import torch
    cfg = workloads.C4R
    fr = workloads.random_frames(cfg.n_views, cfg.seed)
    x_true = workloads.phantom_3d(cfg.N, cfg.seed, cfg.n_ellipsoids, dtype=np.float32)
    out = {"workload": f"{cfg.name}: {cfg.N}^3 volume, {cfg.n_views} random directions x "
                       f"{cfg.det_v}x{cfg.det_u} detector (m={cfg.m}), ell={cfg.ell} random rays "
                       f"from arrived views (one view every {steps_per_view} steps), "
                       f"lambda={cfg.lam:g}", "steps": K, "warmup": W}
    b = None
    for r in r_values:
        s = sl.Slim(cfg.N, cfg.n_views, cfg.det_u, cfg.ell, r, cfg.lam, cfg.seed,
                    precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED, refine_iters=2,
                    dim=3, det_v=cfg.det_v, kind=sl.SLIM_BLOCKS_STREAM,
                    steps_per_view=steps_per_view, use_graph=True, frames=fr)
        if b is None:
            xt = torch.tensor(x_true, device="cuda")
            y = torch.zeros(cfg.m, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()   # inputs filled on torch's stream; the context has its own
            s.project(xt, y)
            torch.cuda.synchronize()
            e = torch.tensor(workloads.noise_direction(cfg.m, cfg.seed), dtype=torch.float32,
                             device="cuda")
            b = y + cfg.noise * torch.linalg.norm(y) * e / torch.linalg.norm(e)
            torch.cuda.synchronize()
            del xt, e, y
        s.set_data(b)
        per, ph, _, _ = timed_steps(s, K, W, flush, stream)
        s.close()
        t = sum(per) * 1e-3
        p = (r + 1) * cfg.ell
        phases = {k: v / K for k, v in ph.items()}
        out[f"r{r}"] = {"p": p, "rows_per_s": cfg.ell * K / t, "ms_per_step": t / K * 1e3,
                        "phases_ms": phases, "dominant": max(phases, key=phases.get),
                        "factor_tflops": (p ** 3 / 3) / (phases["factor"] * 1e-3) / 1e12
                        if phases.get("factor") else None}
    return out


def batch_block(sl, flush, stream, K, W, count=96, tune=True):
    """Many uneven 2D problems (random-ray blocks) advancing together: one CUDA
    graph per batch step with a parallel branch per problem and the problems'
    factorisations in one merged launch; tile size and CTAs per SM chosen by
    the autotuner per size class (tune=False: 64-wide tiles, 1 CTA per SM, no
    tuning runs)."""
    import torch
    cfgs = workloads.batch_mix(count)
    t0 = time.perf_counter()
    specs, choices, alone_ms = [], {}, 0.0
    for c in cfgs:
        sp = dict(N=c.N, n_views=c.n_views, det=c.det, ell=c.ell, r=c.r, lam=c.lam, seed=c.seed,
                  kind=sl.SLIM_BLOCKS_RAYS, precision=sl.SLIM_PREC_FP32, solver=sl.SLIM_SOLVE_MIXED)
        opt = (sl.autotune_opts(sp, steps=3) if tune else
               dict(tile=64, ctas_per_sm=1, ray_lanes=32, pair_window=32, ms=0.0))
        alone_ms += opt["ms"]
        sp.update(tile=opt["tile"], ctas_per_sm=opt["ctas_per_sm"], ray_lanes=opt["ray_lanes"],
                  pair_window=opt["pair_window"])
        key = f"{opt['tile']}x{opt['ctas_per_sm']} lanes {opt['ray_lanes']} window {opt['pair_window']}"
        choices[key] = choices.get(key, 0) + 1
        specs.append(sp)
    tune_s = time.perf_counter() - t0
    bt = sl.SlimBatch(specs)
    for c, pb in zip(cfgs, bt.problems):
        xt = torch.tensor(workloads.phantom_2d(c.N, c.seed, c.n_ellipses), dtype=torch.float32,
                          device="cuda")
        y = torch.zeros(c.m, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()   # inputs filled on torch's stream; the context has its own
        pb.project(xt, y)
        torch.cuda.synchronize()     # y comes from the problem's stream, b is formed on torch's
        e = torch.tensor(workloads.noise_direction(c.m, c.seed), dtype=torch.float32, device="cuda")
        bb = y + c.noise * torch.linalg.norm(y) * e / torch.linalg.norm(e)
        torch.cuda.synchronize()
        pb.set_data(bb)
    torch.cuda.synchronize()
    bt.set_stream(stream.cuda_stream)
    for i in range(W):
        flush.fill_(i)
        bt.step(1)
    bt.sync()
    per = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(i)
            ev[0].record(stream)
            bt.step(1)
            ev[1].record(stream)
            ev[1].synchronize()
            per.append(ev[0].elapsed_time(ev[1]))
    bt.sync()
    bt.close()
    rows = sum(c.ell for c in cfgs)
    t = sum(per) * 1e-3
    flops = sum(chol_flops((c.r + 1) * c.ell) for c in cfgs)
    return {"workload": f"{count} uneven 2D problems: N in {{128..512}}, views U{{90..360}}, "
                        f"bins ceil(sqrt2 N), ell U{{128..512}} random rays, r U{{2..8}}, "
                        f"lambda log-U[1e-4,1e-2]; float32 x, mixed solve",
            "rows_per_s": rows * K / t, "ms_per_step": t / K * 1e3, "rows_per_step": rows,
            "steps": K, "warmup": W, "factor_flops_per_step": flops,
            "factor_tflops_if_all_time": flops / (t / K) / 1e12,
            # the autotuner's best step time of each problem run alone, summed:
            # the step of the batch if the problems ran one after another
            "one_by_one_ms_per_step": alone_ms if tune else None,
            "autotune": {"choices": choices, "seconds": tune_s,
                         "searched": "tile 32/64 x CTAs per SM 1/2/3, then threads per ray 8/16/32 x "
                                     "pair window 16/32/64"}}


def measured_peaks():
    """The measured peaks of this GPU model (MEASURED_PEAKS.json), or {}."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def hbm_peak():
    """Measured HBM copy bandwidth in GB/s (MEASURED_PEAKS.json), else the
    fallback figure of an earlier GB300 measurement."""
    return float(measured_peaks().get("hbm_gbs", 6800.0))


def unet_flops(sl, n1):
    """Multiply-add flops (x2) of one image through the network with n1 pixels
    at full resolution: each weight is used once per output pixel (conv) or
    per input pixel (tconv).  The training step adds the weight gradient (the
    same contraction) and the input gradient (the same, except for the first
    layer, whose input needs none)."""
    px = {"enc1a": n1, "enc1b": n1, "enc2a": n1 // 4, "enc2b": n1 // 4, "enc3a": n1 // 16,
          "enc3b": n1 // 16, "bota": n1 // 64, "botb": n1 // 64, "up3": n1 // 64, "dec3a": n1 // 16,
          "dec3b": n1 // 16, "up2": n1 // 16, "dec2a": n1 // 4, "dec2b": n1 // 4, "up1": n1 // 4,
          "dec1a": n1, "dec1b": n1, "out": n1}
    per = {name: 2 * int(np.prod(shape)) * px[name] for name, shape, _ in sl.UNET_LAYERS}
    fwd = sum(per.values())
    return {"forward": fwd, "train": 3 * fwd - per["enc1a"]}


def unet_block(sl, flush, stream, reps=10, batch=8):
    """The network alone on the 256 x 256 grid with random weights: one
    forward pass of one image, and one training step (forward, backward, Adam)
    of `batch` images, each timed with events on the launching stream after an
    L2 flush.  Flops are the network's own (see unet_flops); the tensor cores
    execute 3x as many for the float32-accurate operands."""
    import torch
    import workloads
    N = workloads.C2.N
    net = sl.UNet(N, N, max_batch=batch)
    net.set_params(sl.flatten_params(workloads.unet_init(0, sl.UNET_LAYERS)))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(batch * N * N, device="cuda", generator=g)
    t = torch.randn(batch * N * N, device="cuda", generator=g)
    y = torch.empty_like(x)
    sp = stream.cuda_stream

    def timed(fn):
        for _ in range(3):
            fn()
        tot = 0.0
        for i in range(reps):
            flush.fill_(i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    with torch.cuda.stream(stream):
        f_ms = timed(lambda: net.forward(x[:N * N], y[:N * N], sp))
        t_ms = timed(lambda: net.train_step(x, t, 1e-4, sp))
    net.close()
    fl = unet_flops(sl, N * N)
    peak = measured_peaks().get("bf16_tflops")
    f_tf = fl["forward"] / f_ms * 1e-9
    t_tf = batch * fl["train"] / t_ms * 1e-9
    return {"grid": f"{N}x{N}", "forward_ms": f_ms, "forward_gflop": fl["forward"] * 1e-9,
            "forward_tflops": f_tf, "train_batch": batch, "train_step_ms": t_ms,
            "train_gflop": batch * fl["train"] * 1e-9, "train_tflops": t_tf,
            "train_images_per_s": batch / t_ms * 1e3,
            "bf16_peak_tflops": peak, "forward_frac_of_measured_bf16": f_tf / peak if peak else None,
            "note": ("implicit-GEMM convolutions on the tcgen05 tensor cores (bfloat16 operands, "
                     "float32 accumulators in tensor memory); activations as "
                     "3 bfloat16 terms (weight gradients 2 x 2), so the pipe executes 3x the flops "
                     "counted here; L2 flushed before each timed call")}


def warm_start_block(args):
    """Learned initial guess on the 256x256 workload: pairs from the method,
    training of the U-Net in the library's kernels, held-out steps to relative
    error thresholds against the method's own reconstruction."""
    import torch
    from paper_1912_07962_gb300 import slim as sl, warmstart as ws
    cfg = workloads.C2
    train = list(workloads.WARM_TRAIN_SEEDS)[:args.ws_train]
    test = list(workloads.WARM_TEST_SEEDS)[:args.ws_test]
    log = (lambda m: print(m, file=sys.stderr)) if args.ws_verbose else None
    t0 = time.perf_counter()
    X, Y, worst = ws.make_pairs(cfg, train, args.ws_target_epochs, torch, log=log)
    t_pairs = time.perf_counter() - t0
    s_in = ws.input_scale(X)
    net = sl.UNet(cfg.N, cfg.N, max_batch=args.ws_batch)
    net.set_params(sl.flatten_params(workloads.unet_init(0, sl.UNET_LAYERS)))
    losses, t_train = ws.train(net, X, Y, s_in, args.ws_net_epochs, args.ws_batch, args.ws_lr, torch,
                               log=log)
    del X, Y
    # inference time of one forward pass (256x256)
    xin = torch.randn(cfg.n, device="cuda")
    yout = torch.empty_like(xin)
    cur = torch.cuda.current_stream()
    for _ in range(3):
        net.forward(xin, yout, cur.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for _ in range(10):
        net.forward(xin, yout, cur.cuda_stream)
    e1.record(cur)
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 10
    thresholds = [0.5, 0.3, 0.2, 0.15, 0.1]
    recs, t_ws = ws.evaluate(net, cfg, test, s_in, args.ws_eval_epochs, thresholds, torch, log=log)
    net.close()
    fwd_gflop = unet_flops(sl, cfg.n)["forward"] * 1e-9
    summ = ws.summarize(recs, thresholds)
    return {"train_seeds": len(train), "test_seeds": len(test),
            "seeds": (f"train {train[0]}..{train[-1]}, held out {test[0]}..{test[-1]}"),
            "gain": {"warm_x0_err_median": summ["warm"]["err0"],
                     "zero_start_best_err_median": summ["zero"]["best"],
                     "warm_x0_beats_zero_start_best": summ["warm"]["err0"] < summ["zero"]["best"]},
            "target": f"chosen-form iterate after {args.ws_target_epochs} epochs from x0=0",
            "error": "relative error to x_true (the phantom), checked every 6 steps",
            "budget": f"{args.ws_eval_epochs} epochs per start",
            "float64_check_max_rel_diff": worst, "pairs_seconds": t_pairs,
            "net_epochs": args.ws_net_epochs, "batch": args.ws_batch, "lr": args.ws_lr,
            "train_seconds": t_train, "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
            "input_scale": s_in, "forward_ms": fwd_ms, "forward_gflop": fwd_gflop,
            "forward_tflops": fwd_gflop / fwd_ms,
            "warm_start_call_ms_median": t_ws * 1e3,
            "steps_to_threshold": summ}


def e2e_block(sl, cfg, b, K, W, lookahead=0, ctas_per_sm=0):
    """Same metric through the C ABI with host buffers: each step copies b from
    pinned host memory, steps, and reads x back to pinned host memory."""
    import torch
    s = make_form(sl, cfg, "chosen", cfg.seed, lookahead=lookahead, ctas_per_sm=ctas_per_sm)
    bh = torch.tensor(b.astype(np.float32)).pin_memory()
    xh = torch.empty(cfg.n, dtype=torch.float32).pin_memory()
    s.set_data(bh)
    for _ in range(W):
        s.set_data(bh)
        s.step(1)
        s.get_x(xh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        s.set_data(bh)
        s.step(1)
        s.get_x(xh)
    el = time.perf_counter() - t0
    s.close()
    return {"value": cfg.ell * K / el, "unit": "rows/s", "h2d_bytes_per_step": 4 * cfg.m,
            "d2h_bytes_per_step": 4 * cfg.n, "seconds": el, "steps": K,
            "note": ("host clock around K steps, each copying b in from pinned host memory, "
                     "stepping and copying x out (synchronous), no L2 flush between steps")}


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica: independent problems of the same workload."""
    return base + 1000 * rank


def job_throughput(local_seconds: float, units_per_rank: float, world: int, device="cpu"):
    """Whole-job throughput of `world` replicas: the units all ranks processed
    over the slowest rank's time (max over ranks by all-reduce when world > 1).
    Returns (units per second, the max time)."""
    t = float(local_seconds)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt)
    return units_per_rank * world / t, t


def main_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1912_07962_gb300 import build as slbuild
    slbuild.build()
    from paper_1912_07962_gb300 import slim as sl

    cfg, desc = workload_of(args.workload)
    seed = replica_seed(cfg.seed, rank)      # independent replicas
    x_true = workloads.phantom_2d(cfg.N, seed, cfg.n_ellipses)
    e = workloads.noise_direction(cfg.m, seed)
    b = make_b(sl, cfg, x_true, e)
    stream = torch.cuda.Stream()          # the library and the timing events share it
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # plain float64 form
    sp = make_form(sl, cfg, "plain", seed)
    sp.set_data(b)
    per_p, ph_p, _, _ = timed_steps(sp, args.plain_steps, args.warmup, flush, stream)
    sp.close()

    # chosen form: the headline timed region
    sc = make_form(sl, cfg, "chosen", seed, lookahead=args.lookahead,
                   ctas_per_sm=args.factor_ctas_per_sm)
    sc.set_data(b.astype(np.float32))
    clk = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    launch_log = None
    if args.lookahead:
        per_c, launch_log, _, region_ms = timed_region(sc, args.steps, args.warmup, flush, stream)
        per_c = [region_ms / args.steps] * args.steps
    else:
        per_c, ph_c, _, _ = timed_steps(sc, args.steps, args.warmup, flush, stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    kernels = sc.kernels_per_step()
    if args.lookahead:
        # phase breakdown from a short synchronous pass (one step at a time)
        _, ph_c, _, _ = timed_steps(sc, 5, 0, flush, stream)
        ph_c = {k: v * args.steps / 5 for k, v in ph_c.items()}
    sc.close()
    fp64_factor = None
    if args.lookahead and rank == 0 and not args.no_fp64_factor:
        # the same pipelined chosen form with the float64 factor and solves
        sf = make_form(sl, cfg, "chosen_fp64_factor", seed, lookahead=args.lookahead,
                       ctas_per_sm=args.factor_ctas_per_sm)
        sf.set_data(b.astype(np.float32))
        _, llog, _, reg = timed_region(sf, args.steps, args.warmup, flush, stream)
        sf.close()
        fp64_factor = {"rows_per_s": cfg.ell * args.steps / (reg * 1e-3),
                       "ms_per_step": reg / args.steps, "steps": args.steps,
                       "factor_launch_ms": llog["factor_launch_ms"],
                       "iterate_chain_ms": llog["iterate_chain_ms"],
                       "factor_tflops_aggregate": chol_flops(cfg.p) / (reg / args.steps * 1e-3) / 1e12,
                       "form": ("float32 projector/residual/scatter, float64 Gram, float64 tiled "
                                "Cholesky and triangular solves (no refinement), pipelined as "
                                "the headline, same timing")}
    t_p = sum(per_p) * 1e-3
    rows_c, t_c = job_throughput(sum(per_c) * 1e-3, cfg.ell * args.steps, world, device="cuda")
    rows_p = cfg.ell * args.plain_steps / t_p

    if launch_log:
        # pipelined: the factorisation is the kernel with the most device time
        # per step; its launches are timed live over the timed region
        f_s = launch_log["factor_launch_ms"] * 1e-3
        peak = NUM_SMS * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
        ach = chol_flops(cfg.p) / f_s / 1e12
        rl = {"kernel": "chol_factor_kernel", "phase": "factor", "bound": "alu", "achieved": ach,
              "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
              "algorithmic": f"p^3/3 = {chol_flops(cfg.p):.4g} flop per launch (p = {cfg.p})",
              "peak_source": "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz",
              "launch_ms": launch_log["factor_launch_ms"],
              "iterate_chain_ms": launch_log["iterate_chain_ms"],
              "aggregate_tflops": chol_flops(cfg.p) / (t_c / args.steps) / 1e12,
              "aggregate_note": ("one factorisation per step over the region's time per step: the "
                                 "throughput of the factorisations in flight together"),
              "launches_timed": launch_log["chains"],
              "note": (f"factorisations run up to {args.lookahead} steps ahead of the iterate "
                       "chain, overlapping one another and it; launch_ms is the mean duration "
                       "of one factorisation launch inside the timed region")}
    else:
        rl = roofline_of(ph_c, args.steps, cfg.p, cfg.ell, cfg.N, "chosen", clocks.get("sm_mhz"))
    rl["traffic"] = traffic_from_profiles(rl["kernel"])
    rl_p = roofline_of(ph_p, args.plain_steps, cfg.p, cfg.ell, cfg.N, "plain", None)

    tta = None
    if args.tta_epochs > 0 and rank == 0:
        ths = [0.5, 0.2, 0.1, 0.05, 0.02, 0.01]
        tta = {"constant_damping": tta_block(sl, cfg, b, flush, stream, args.tta_epochs, ths,
                                             lookahead=args.lookahead,
                                             ctas_per_sm=args.factor_ctas_per_sm)}
        if args.tta_decay_after > 0:
            tta["decaying_damping"] = tta_block(sl, cfg, b, flush, stream, args.tta_epochs, ths,
                                                lookahead=args.lookahead,
                                                ctas_per_sm=args.factor_ctas_per_sm,
                                                decay_after=args.tta_decay_after)
    e2e = (e2e_block(sl, cfg, b, args.steps, args.warmup, lookahead=args.lookahead,
                     ctas_per_sm=args.factor_ctas_per_sm)
           if rank == 0 and not args.no_e2e else None)
    csr_pass = (csr_block(sl, cfg, flush, stream, reps=args.csr_reps)
                if rank == 0 and not args.no_csr else None)
    s3d = stream3d_block(sl, flush, stream, args.steps, args.warmup) if rank == 0 and not args.no_3d else None
    batch = (batch_block(sl, flush, stream, args.batch_steps, max(3, args.warmup))
             if rank == 0 and args.batch_steps > 0 else None)
    lsqr_pass = (lsqr_block(sl, cfg, b, flush, stream, args.lsqr_steps, 3)
                 if rank == 0 and args.lsqr_steps > 0 else None)
    sens = (sensitivity_block(sl, flush, stream, reps=args.sens_reps)
            if rank == 0 and args.sens_reps > 0 else None)
    f3d = (frames3d_block(sl, flush, stream, args.frames_steps, 3)
           if rank == 0 and args.frames_steps > 0 else None)
    tik_pass = (tik_block(sl, cfg, b, flush, stream, args.tik_steps, max(3, args.warmup),
                          lookahead=SWEEP_LOOKAHEAD, ctas_per_sm=SWEEP_CTAS)
                if rank == 0 and args.tik_steps > 0 else None)
    warm = warm_start_block(args) if rank == 0 and not args.no_warm_start else None
    unet = (unet_block(sl, flush, stream, reps=args.unet_reps)
            if rank == 0 and not args.no_unet else None)
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        leg = run_cpu_leg(args)
        cpu = {"value": leg["rows_per_s"], "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": (f"{leg['steps']} oracle steps of this workload after {leg['warmup']} "
                          f"untimed warm-up steps, {leg['seconds']:.1f} s, one BLAS thread")}
        ncores = os.cpu_count() or 1
        leg_all = run_cpu_leg(args, threads=ncores)
        cpu_all = {"value": leg_all["rows_per_s"], "unit": "rows/s", "cores": ncores,
                   "kind": "oracle",
                   "sample": (f"{leg_all['steps']} oracle steps after {leg_all['warmup']} "
                              f"warm-up steps, {leg_all['seconds']:.1f} s, {ncores} BLAS threads "
                              "(the dense Cholesky of each step is threaded; the sparse "
                              "products are not)")}
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": rows_c, "unit": "rows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_c / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "form": "chosen: float32 projector/residual/scatter, "
                   "float64 Gram, " + FORM_OF_SOLVER[CHOSEN_SOLVER] + ", "
                   + (f"geometry and factorisation pipelined {args.lookahead} steps ahead of "
                      "the iterate chain (CUDA graphs on three kinds of stream)"
                      if args.lookahead else "one CUDA graph per step"),
                   "lookahead": args.lookahead, "factor_ctas_per_sm": args.factor_ctas_per_sm,
                   "timing": ("one region of K back-to-back steps after a synchronisation, ended "
                              "once every stream of the context has joined the caller's: K "
                              "iterate chains and K factorisations (pipelined steady state; the "
                              "flush writes are inside the region)" if args.lookahead else
                              "each step bracketed by events and synchronised"),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "chosen_fp64_factor": fp64_factor,
        "plain": {"rows_per_s": rows_p, "ms_per_step": t_p / args.plain_steps * 1e3,
                  "steps": args.plain_steps, "dtype": "f64",
                  "phases_ms": {k: v / args.plain_steps for k, v in ph_p.items()},
                  "roofline": rl_p},
        "speedup_vs_plain": rows_c / (rows_p * world),
        "phases_ms": {k: v / args.steps for k, v in ph_c.items()},
        "phases_note": ("one step at a time (synchronous pass); the pipelined region overlaps "
                        "the geometry phases with the iterate chain" if args.lookahead else
                        "per step, inside the timed region"),
        "roofline": rl, "csr_full_pass": csr_pass, "streaming_3d": s3d, "batched": batch, "lsqr": lsqr_pass, "tik": tik_pass, "random_directions_3d": f3d, "step_size_sensitivity": sens, "unet": unet, "warm_start": warm, "tta": tta, "e2e": e2e,
        "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
        "gpu_launches": kernels * args.steps, "kernels_per_step": kernels, "clocks": clocks,
    }
    print(json.dumps(line))


def main_unet(args):
    """The network leg alone (one JSON line), e.g. for a launch list."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    print(json.dumps({"unet": unet_block(sl, flush, stream, reps=args.unet_reps)}))


def main_csr(args):
    """The stored-matrix passes alone (one JSON line), e.g. for a profile."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cfg, _ = workload_of(args.workload)
    print(json.dumps({"csr_full_pass": csr_block(sl, cfg, flush, stream, reps=args.csr_reps)}))


def main_lsqr(args):
    """The LSQR-step form alone (one JSON line), e.g. for a profile."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cfg, _ = workload_of(args.workload)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    b = make_b(sl, cfg, x_true, e)
    print(json.dumps({"lsqr": lsqr_block(sl, cfg, b, flush, stream, args.lsqr_steps, 3)}))


def main_sens(args):
    """The step-size sensitivity of slimLS, sg and olbfgs alone (one JSON line)."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    print(json.dumps({"step_size_sensitivity": sensitivity_block(sl, flush, stream,
                                                                 reps=max(0, args.sens_reps))}))


def main_frames(args):
    """3D with random view directions alone (one JSON line)."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    print(json.dumps({"random_directions_3d": frames3d_block(sl, flush, stream,
                                                             max(1, args.frames_steps), 3)}))


def tc_block(sl, flush, stream, reps=5):
    """The float32-accurate tensor-core product (slim_tc_matmul: three bfloat16
    terms per operand, six term products on tcgen05) and the tensor-core
    factor + inverse (slim_chol_inverse), each through the C ABI with device
    operands, timed with events on the caller's stream after two warm-up calls
    (each call also allocates its few bytes of descriptors and synchronises)."""
    import torch
    peak = float(measured_peaks().get("bf16_tflops", 1900.0))
    out = {"matmul": [], "chol_inverse": []}
    g = torch.Generator(device="cuda").manual_seed(11)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for n in (4096, 8192):
        A = torch.randn(n, n, device="cuda", generator=g)
        B = torch.randn(n, n, device="cuda", generator=g)
        Cm = torch.empty(n, n, device="cuda")
        torch.cuda.synchronize()
        for _ in range(2):
            sl.tc_matmul(n, n, n, A, n, 0, B, n, 0, Cm, n, 0, stream_ptr=stream.cuda_stream)
        ms = []
        for i in range(reps):
            flush.fill_(i)
            ev[0].record(stream)
            sl.tc_matmul(n, n, n, A, n, 0, B, n, 0, Cm, n, 0, stream_ptr=stream.cuda_stream)
            ev[1].record(stream)
            ev[1].synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        t = min(ms)
        # accuracy on a sampled block against float64
        ref = (A[:256].double() @ B[:256].double().T)
        err = float(torch.linalg.norm(Cm[:256, :256].double() - ref[:, :256]) / torch.linalg.norm(ref[:, :256]))
        eff = 2.0 * n ** 3 / (t * 1e-3) / 1e12
        out["matmul"].append({"M=N=K": n, "ms": t, "float32_tflops": eff,
                              "tensor_tflops": 6 * eff, "tensor_frac_of_bf16_peak": 6 * eff / peak,
                              "rel_error_vs_float64": err})
        del A, B, Cm
    for p in (2178, 4104):
        M = torch.randn(p, p + 16, device="cuda", generator=g, dtype=torch.float64) / (p ** 0.5)
        G = M @ M.T
        X = torch.empty(p, p, device="cuda")
        torch.cuda.synchronize()
        for _ in range(2):
            sl.chol_inverse(G, 1e-3, X, stream_ptr=stream.cuda_stream)
        ms = []
        for i in range(reps):
            flush.fill_(i)
            ev[0].record(stream)
            sl.chol_inverse(G, 1e-3, X, stream_ptr=stream.cuda_stream)
            ev[1].record(stream)
            ev[1].synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        t = min(ms)
        out["chol_inverse"].append({"p": p, "ms": t,
                                    "float32_tflops": (2.0 * p ** 3 / 3.0) / (t * 1e-3) / 1e12})
    out["peak"] = {"bf16_tflops": peak, "source": "MEASURED_PEAKS.json (cuBLAS bf16, burst)"}
    out["note"] = ("float32_tflops counts the float32 product's 2MNK (factor + inverse: p^3/3 + p^3/3); "
                   "tensor_tflops the six bfloat16 term products the tensor cores execute")
    return out


def main_tc(args):
    """The tensor-core product and inverse alone (one JSON line)."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    print(json.dumps({"tensor_core": tc_block(sl, flush, stream)}))


def main_batch(args):
    """The batched block alone (one JSON line)."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    print(json.dumps({"batched": batch_block(sl, flush, stream, max(1, args.batch_steps),
                                             max(3, args.warmup),
                                             tune=not args.batch_no_tune)}))


def main_tik(args):
    """slimTik against slimLS alone (one JSON line)."""
    import torch
    from paper_1912_07962_gb300 import build as slbuild, slim as sl
    slbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cfg, _ = workload_of(args.workload)
    x_true, e = workloads.tomo_inputs_2d(cfg)
    b = make_b(sl, cfg, x_true, e)
    print(json.dumps({"tik": tik_block(sl, cfg, b, flush, stream, args.tik_steps,
                                       max(3, args.warmup), lookahead=SWEEP_LOOKAHEAD,
                                       ctas_per_sm=SWEEP_CTAS)}))


def main_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, desc = workload_of(args.workload)
    leg = run_cpu_leg(args, steps=args.steps, warmup=max(args.warmup, 0))
    v = leg["rows_per_s"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": world,
        "steps": leg["steps"], "warmup": args.warmup, "ms_per_step": leg["seconds"] / leg["steps"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "form": "FP64 CPU oracle (numpy/scipy)",
                                        "parallelism": "single process"},
        "cpu_baseline": {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "sample": f"{leg['steps']} oracle steps after {args.warmup} warm-up steps, "
                                   f"one BLAS thread"},
        "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def parse_args(argv=None):
    """The bench's options, with the chosen form's lookahead and factorisation
    CTAs per SM resolved from its solver when not given."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=6)
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision-256", choices=["precision-256", "plain-64"])
    ap.add_argument("--tta-epochs", type=int, default=20)
    ap.add_argument("--tta-decay-after", type=int, default=180,
                    help="also run time-to-accuracy with the 1/k damping decay after this step "
                         "(0: skip)")
    ap.add_argument("--solver", default="mixed_inv", choices=["mixed", "mixed_tc", "mixed_inv"],
                    help="chosen form's solve: through the tensor-core inverse of the tiled "
                         "float32 factor (mixed_inv, the default), through the float32 factor's "
                         "triangular sweeps (mixed), or through the inverse of a tensor-core "
                         "factor (mixed_tc); the inverse forms are pipelined only")
    ap.add_argument("--no-fp64-factor", action="store_true",
                    help="skip the pipelined chosen form with the float64 factor")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-csr", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-unet", action="store_true")
    ap.add_argument("--lsqr-steps", type=int, default=12,
                    help="steps of the LSQR-step form timed on the workload (0: skip)")
    ap.add_argument("--lsqr-only", action="store_true",
                    help="time only the LSQR-step form and print that line")
    ap.add_argument("--tik-steps", type=int, default=30,
                    help="steps of slimTik and slimLS timed side by side (0: skip)")
    ap.add_argument("--sens-reps", type=int, default=5,
                    help="block sequences per step size in the sensitivity sweep (0: skip; with "
                         "--sens-only, 0 times only the step costs)")
    ap.add_argument("--sens-only", action="store_true",
                    help="run only the step-size sensitivity sweep and print that line")
    ap.add_argument("--frames-steps", type=int, default=5,
                    help="timed steps of the random-direction 3D block (0: skip)")
    ap.add_argument("--frames-only", action="store_true",
                    help="run only the random-direction 3D block and print that line")
    ap.add_argument("--tik-only", action="store_true",
                    help="time only slimTik against slimLS and print that line")
    ap.add_argument("--unet-only", action="store_true",
                    help="time only the network (forward and training step) and print that line")
    ap.add_argument("--unet-reps", type=int, default=10)
    ap.add_argument("--csr-only", action="store_true",
                    help="time only the stored-matrix passes and print that line")
    ap.add_argument("--csr-reps", type=int, default=20)
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned initial guess (by default a reduced protocol runs: "
                         "the --ws-* defaults; the full one is --ws-train 2000 --ws-test 200 "
                         "--ws-target-epochs 2 --ws-eval-epochs 2 --ws-net-epochs 10)")
    ap.add_argument("--ws-train", type=int, default=96)
    ap.add_argument("--ws-test", type=int, default=12)
    ap.add_argument("--ws-target-epochs", type=int, default=1)
    ap.add_argument("--ws-eval-epochs", type=int, default=2)
    ap.add_argument("--ws-net-epochs", type=int, default=16)
    ap.add_argument("--ws-batch", type=int, default=8)
    ap.add_argument("--ws-lr", type=float, default=1e-3)
    ap.add_argument("--ws-verbose", action="store_true")
    ap.add_argument("--factor-ctas-per-sm", type=int, default=None,
                    help="persistent factorisation CTAs per SM shared by the factorisations in "
                         "flight (0: library default; default 2 for mixed_inv, else 1)")
    ap.add_argument("--lookahead", type=int, default=None,
                    help="steps the geometry chain runs ahead in the chosen form (0: one chain; "
                         "default 8 for mixed_inv, else 6)")
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="timed steps of the 96-problem batched block (0: skip it)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched block and print that line")
    ap.add_argument("--ws-only", action="store_true",
                    help="run only the learned initial guess block (the --ws-* options) and print that line")
    ap.add_argument("--tc-only", action="store_true",
                    help="time only the tensor-core product and factor inverse and print that line")
    ap.add_argument("--batch-no-tune", action="store_true",
                    help="batched block without the autotuner (64-wide tiles, 1 CTA per SM)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-steps", type=int, default=0)
    ap.add_argument("--cpu-warmup", type=int, default=6)
    ap.add_argument("--cpu-leg", action="store_true")
    args = ap.parse_args(argv)
    # measured best per solve: the inverse form's short iterate chain leaves the
    # step to the factorisations in flight, which gain from a longer lookahead
    # and a second CTA per SM; the triangular sweeps' chain does not
    if args.lookahead is None:
        args.lookahead = 8 if args.solver == "mixed_inv" else 6
    if args.factor_ctas_per_sm is None:
        args.factor_ctas_per_sm = 2 if args.solver == "mixed_inv" else 1
    args.r_warm = workload_of(args.workload)[0].r + 1
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    return args


def main():
    args = parse_args()
    global CHOSEN_SOLVER
    CHOSEN_SOLVER = args.solver
    if args.cpu_leg:
        cpu_leg(args)
    elif args.impl == "reference":
        main_reference(args)
    elif args.unet_only:
        main_unet(args)
    elif args.csr_only:
        main_csr(args)
    elif args.lsqr_only:
        main_lsqr(args)
    elif args.tik_only:
        main_tik(args)
    elif args.sens_only:
        main_sens(args)
    elif args.frames_only:
        main_frames(args)
    elif args.batch_only:
        main_batch(args)
    elif args.tc_only:
        main_tc(args)
    elif args.ws_only:
        import torch
        from paper_1912_07962_gb300 import build as slbuild
        slbuild.build()
        with torch.cuda.stream(torch.cuda.Stream()):
            print(json.dumps({"warm_start": warm_start_block(args)}))
    else:
        main_gpu(args)


if __name__ == "__main__":
    main()
