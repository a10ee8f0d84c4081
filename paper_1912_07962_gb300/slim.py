"""ctypes binding of libslim.so with the names of the C ABI (include/slim.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Device arrays are passed as torch CUDA tensors (their data_ptr()), host arrays
as numpy arrays or CPU tensors.  Loading fails loudly when the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslim.so")

SLIM_OK, SLIM_EINVAL, SLIM_ENOMEM, SLIM_ECUDA, SLIM_ENOTPD, SLIM_ETIMEOUT, SLIM_ESTATE, \
    SLIM_ENOTSUP = range(8)
STATUS_NAMES = ["SLIM_OK", "SLIM_EINVAL", "SLIM_ENOMEM", "SLIM_ECUDA", "SLIM_ENOTPD",
                "SLIM_ETIMEOUT", "SLIM_ESTATE", "SLIM_ENOTSUP"]
SLIM_F32, SLIM_F64 = 0, 1
SLIM_PREC_FP64, SLIM_PREC_FP32 = 0, 1
SLIM_SOLVE_FP64, SLIM_SOLVE_MIXED, SLIM_SOLVE_LSQR, SLIM_SOLVE_SG, SLIM_SOLVE_OLBFGS = 0, 1, 2, 3, 4
SLIM_SOLVE_MIXED_TC = 5
SLIM_SOLVE_MIXED_INV = 6
SLIM_BLOCKS_VIEWS, SLIM_BLOCKS_RAYS, SLIM_BLOCKS_STREAM = 0, 1, 2

# every function the header declares (checked by the CPU test suite)
EXPORTS = [
    "slim_create", "slim_destroy", "slim_last_error", "slim_set_stream", "slim_set_data",
    "slim_set_x", "slim_get_x", "slim_step", "slim_sync", "slim_set_ref", "slim_run",
    "slim_get_iter", "slim_set_iter", "slim_checkpoint", "slim_restore", "slim_get_memory",
    "slim_get_sizes", "slim_project", "slim_backproject", "slim_damped_solve",
    "slim_set_timing", "slim_get_timing", "slim_damped_solve_noalloc", "slim_get_csr",
    "slim_autotune", "slim_batch_create", "slim_batch_ctx", "slim_batch_step", "slim_batch_sync",
    "slim_batch_set_stream", "slim_batch_destroy", "slim_get_launch_log",
    "slim_unet_param_count", "slim_unet_create", "slim_unet_destroy", "slim_unet_set_params",
    "slim_unet_get_params", "slim_unet_get_grads", "slim_unet_forward", "slim_unet_train_step",
    "slim_warm_start", "slim_backproject_data", "slim_unet_conv3x3", "slim_unet_conv3x3_grad",
    "slim_unet_tconv2x2", "slim_unet_tconv2x2_grad", "slim_get_lsqr_info", "slim_set_c_diag",
    "slim_selftest_wait", "slim_join_stream", "slim_tc_matmul", "slim_chol_inverse",
    "slim_set_tik_bidiag",
]
A_MATRIX_FREE, A_CSR_F32, A_CSR_BF16 = 0, 1, 2
NOALLOC_MAX_P = 1024
PHASES = ["sample", "forward_residual", "gram_update", "form_k", "factor", "solve", "scatter"]


class slim_geometry(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_side", C.c_int), ("n_views", C.c_int),
                ("det_u", C.c_int), ("det_v", C.c_int), ("angles", C.POINTER(C.c_double)),
                ("a_mode", C.c_int), ("precision", C.c_int), ("frames", C.POINTER(C.c_double))]


class slim_blocks(C.Structure):
    _fields_ = [("kind", C.c_int), ("ell", C.c_int), ("seed", C.c_ulonglong),
                ("steps_per_view", C.c_int), ("with_replacement", C.c_int), ("cyclic", C.c_int)]


class slim_step_opts(C.Structure):
    _fields_ = [("eta", C.c_double), ("ramp", C.c_int), ("solver", C.c_int),
                ("refine_iters", C.c_int), ("use_graph", C.c_int), ("tile", C.c_int),
                ("ctas_per_sm", C.c_int), ("lookahead", C.c_int), ("lsqr_max_iter", C.c_int),
                ("lsqr_tol", C.c_double), ("tik_lambda", C.c_double), ("tik_reading", C.c_int),
                ("decay_after", C.c_int), ("olbfgs_memory", C.c_int), ("ray_lanes", C.c_int),
                ("pair_window", C.c_int)]


class SlimError(RuntimeError):
    def __init__(self, code, msg):
        self.code = code
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else str(code)
        super().__init__(f"{name}: {msg}")


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libslim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libslim.so not built ({path}); run paper_1912_07962_gb300.build")
    lib = C.CDLL(path)
    P, VP, I, SZ, D, LL = C.POINTER, C.c_void_p, C.c_int, C.c_size_t, C.c_double, C.c_longlong
    sig = {
        "slim_create": ([P(slim_geometry), P(slim_blocks), I, D, P(slim_step_opts), P(VP)], I),
        "slim_destroy": ([VP], None),
        "slim_last_error": ([VP], C.c_char_p),
        "slim_set_stream": ([VP, VP], I),
        "slim_set_data": ([VP, VP, SZ, I, I], I),
        "slim_set_x": ([VP, VP, SZ, I, I], I),
        "slim_get_x": ([VP, VP, SZ, I, I], I),
        "slim_step": ([VP, I], I),
        "slim_sync": ([VP], I),
        "slim_join_stream": ([VP, VP], I),
        "slim_tc_matmul": ([I, I, I, VP, LL, I, VP, LL, I, VP, LL, I, C.c_float, C.c_float, I, I,
                            VP], I),
        "slim_chol_inverse": ([VP, I, D, VP, VP], I),
        "slim_set_tik_bidiag": ([VP, VP, VP, SZ, I], I),
        "slim_set_ref": ([VP, VP, SZ, I, I], I),
        "slim_run": ([VP, LL, D, I, P(LL), P(D), P(D)], I),
        "slim_get_iter": ([VP, P(LL)], I),
        "slim_set_iter": ([VP, LL], I),
        "slim_checkpoint": ([VP, VP, P(SZ)], I),
        "slim_restore": ([VP, VP, SZ], I),
        "slim_get_memory": ([VP, VP, VP, VP], I),
        "slim_get_sizes": ([VP, P(LL), P(LL), P(I)], I),
        "slim_project": ([VP, VP, I, VP, VP], I),
        "slim_backproject": ([VP, VP, I, VP, VP], I),
        "slim_damped_solve": ([VP, I, D, VP, VP, VP], I),
        "slim_set_timing": ([VP, I], I),
        "slim_get_timing": ([VP, P(D), I, P(I)], I),
        "slim_damped_solve_noalloc": ([VP, I, D, VP, VP, VP], I),
        "slim_get_csr": ([VP, P(LL), VP, VP, VP], I),
        "slim_autotune": ([P(slim_geometry), P(slim_blocks), I, D, P(slim_step_opts), I,
                           P(slim_step_opts), P(D)], I),
        "slim_batch_create": ([I, P(slim_geometry), P(slim_blocks), P(I), P(D),
                               P(slim_step_opts), P(VP)], I),
        "slim_batch_ctx": ([VP, I, P(VP)], I),
        "slim_batch_step": ([VP, I], I),
        "slim_batch_sync": ([VP], I),
        "slim_batch_set_stream": ([VP, VP], I),
        "slim_batch_destroy": ([VP], None),
        "slim_get_launch_log": ([VP, P(D), P(D), P(LL)], I),
        "slim_unet_param_count": ([P(LL)], I),
        "slim_unet_create": ([I, I, I, P(VP)], I),
        "slim_unet_destroy": ([VP], None),
        "slim_unet_set_params": ([VP, VP, LL], I),
        "slim_unet_get_params": ([VP, VP, LL], I),
        "slim_unet_get_grads": ([VP, VP, LL], I),
        "slim_unet_forward": ([VP, VP, VP, I, VP], I),
        "slim_unet_train_step": ([VP, VP, VP, I, C.c_float, P(D), VP], I),
        "slim_warm_start": ([VP, VP, D, D, P(I), P(D)], I),
        "slim_backproject_data": ([VP, VP], I),
        "slim_unet_conv3x3": ([VP, I, I, I, I, VP, VP, I, I, VP, VP], I),
        "slim_unet_conv3x3_grad": ([VP, VP, I, I, I, I, VP, I, VP, VP, VP, VP], I),
        "slim_unet_tconv2x2": ([VP, I, I, I, I, VP, VP, I, VP, VP], I),
        "slim_unet_tconv2x2_grad": ([VP, VP, I, I, I, I, VP, I, VP, VP, VP, VP], I),
        "slim_get_lsqr_info": ([VP, P(I), P(D), P(D)], I),
        "slim_set_c_diag": ([VP, VP, C.c_size_t, I, I], I),
        "slim_selftest_wait": ([VP], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(a):
    """(pointer, on_device, dtype code, element count) of a torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        import torch
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        code = {torch.float32: SLIM_F32, torch.float64: SLIM_F64}.get(a.dtype)
        if code is None:
            raise ValueError(f"unsupported dtype {a.dtype}")
        return C.c_void_p(a.data_ptr()), int(a.is_cuda), code, a.numel()
    a = np.ascontiguousarray(a)
    code = {np.dtype(np.float32): SLIM_F32, np.dtype(np.float64): SLIM_F64}.get(a.dtype)
    if code is None:
        raise ValueError(f"unsupported dtype {a.dtype}")
    return C.c_void_p(a.ctypes.data), 0, code, a.size


class Slim:
    """One slimLS problem on the GPU (owns a slim_ctx).

    The arguments map onto slim_geometry, slim_blocks and slim_step_opts of
    include/slim.h, which documents each one.  Beyond the Woodbury step:
      solver        SLIM_SOLVE_LSQR (the step by LSQR; lsqr_max_iter, lsqr_tol),
                    SLIM_SOLVE_SG and SLIM_SOLVE_OLBFGS (the comparators, r = 0;
                    olbfgs_memory), step size alpha_k = 1/lambda_k
      tik_lambda    slimTik's Tikhonov parameter (0: slimLS); tik_reading 0/1 the
                    count of Tikhonov rows (blocks of M_k, or r as printed);
                    C_k = diag(c) through set_c_diag
      decay_after   the 1/k decay of the damping after that step (0: none)
      with_replacement, cyclic  block sampling: False / True selects the random
                    cyclic order of the views, or distinct rays in random-ray blocks
      frames        3D views from arbitrary directions: rows (d, u, v) per view
    """

    def __init__(self, N, n_views, det, ell, r, lam, seed, precision=SLIM_PREC_FP64,
                 solver=SLIM_SOLVE_FP64, refine_iters=2, eta=1.0, ramp=False, use_graph=False,
                 angles=None, a_mode=A_MATRIX_FREE, dim=2, det_v=1, kind=SLIM_BLOCKS_VIEWS,
                 steps_per_view=1, tile=0, ctas_per_sm=0, lookahead=0, lsqr_max_iter=0,
                 lsqr_tol=0.0, tik_lambda=0.0, tik_reading=0, decay_after=0, olbfgs_memory=0,
                 frames=None, with_replacement=True, cyclic=False, ray_lanes=0, pair_window=0,
                 _handle=None):
        lib = load()
        self._lib = lib
        self._angles = None
        self._owned = _handle is None
        self.precision = precision
        self.N, self.n, self.m = N, N ** dim, n_views * det * det_v
        if _handle is not None:      # a context owned by a batch
            self.h = _handle
            n_, m_, p_ = C.c_longlong(), C.c_longlong(), C.c_int()
            lib.slim_get_sizes(self.h, C.byref(n_), C.byref(m_), C.byref(p_))
            self.p = p_.value
            return
        g = slim_geometry(dim, N, n_views, det, det_v, None, a_mode, precision)
        if angles is not None:
            self._angles = np.ascontiguousarray(angles, dtype=np.float64)
            g.angles = self._angles.ctypes.data_as(C.POINTER(C.c_double))
        self._frames = None
        if frames is not None:       # 3D views from arbitrary directions: rows (d, u, v)
            self._frames = np.ascontiguousarray(frames, dtype=np.float64).reshape(-1)
            g.frames = self._frames.ctypes.data_as(C.POINTER(C.c_double))
        blk = slim_blocks(kind, ell, seed, steps_per_view, int(with_replacement), int(cyclic))
        opts = slim_step_opts(eta, int(ramp), solver, refine_iters, int(use_graph), tile, ctas_per_sm,
                              lookahead, lsqr_max_iter, lsqr_tol, tik_lambda, tik_reading,
                              decay_after, olbfgs_memory, ray_lanes, pair_window)
        h = C.c_void_p()
        st = lib.slim_create(C.byref(g), C.byref(blk), r, lam, C.byref(opts), C.byref(h))
        if st != SLIM_OK:
            raise SlimError(st, "slim_create failed")
        self.h = h
        self.precision = precision
        self.N, self.n, self.m = N, N ** dim, n_views * det * det_v
        n, m, p = C.c_longlong(), C.c_longlong(), C.c_int()
        lib.slim_get_sizes(h, C.byref(n), C.byref(m), C.byref(p))
        self.p = p.value

    def _check(self, st):
        if st != SLIM_OK:
            raise SlimError(st, self._lib.slim_last_error(self.h).decode())

    def lsqr_info(self):
        """(iterations, ||M^T(c - M s) - lambda s|| estimate, ||M^T c||) of the last LSQR step."""
        it, res, res0 = C.c_int(), C.c_double(), C.c_double()
        self._check(self._lib.slim_get_lsqr_info(self.h, C.byref(it), C.byref(res), C.byref(res0)))
        return it.value, res.value, res0.value

    def set_tik_bidiag(self, d0, d1=None):
        """C_k = L^T L with L lower bidiagonal on the image vector, (L x)_i =
        d0_i x_i + d1_i x_{i-1}; None restores C_k = I (host arrays, copied)."""
        if d0 is None:
            self._check(self._lib.slim_set_tik_bidiag(self.h, None, None, 0, 0))
            return
        a0 = np.ascontiguousarray(d0, dtype=np.float64)
        a1 = None if d1 is None else np.ascontiguousarray(d1, dtype=np.float64)
        self._check(self._lib.slim_set_tik_bidiag(
            self.h, a0.ctypes.data_as(C.c_void_p),
            None if a1 is None else a1.ctypes.data_as(C.c_void_p), a0.size, 0))

    def set_c_diag(self, c):
        """C_k = diag(c) of Eq. (B_k) (c > 0; slimTik: L^T L with L = diag(sqrt c)).
        None restores C_k = I.  The memory of the steps taken is rebuilt."""
        if c is None:
            self._check(self._lib.slim_set_c_diag(self.h, None, 0, SLIM_F64, 0))
            return
        p, dev, code, cnt = _ptr(c)
        self._check(self._lib.slim_set_c_diag(self.h, p, cnt, code, dev))

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            self._lib.slim_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, b):
        p, dev, code, cnt = _ptr(b)
        self._check(self._lib.slim_set_data(self.h, p, cnt, code, dev))

    def set_x(self, x):
        p, dev, code, cnt = _ptr(x)
        self._check(self._lib.slim_set_x(self.h, p, cnt, code, dev))

    def get_x(self, out=None, dtype=np.float64):
        if out is None:
            out = np.empty(self.n, dtype=dtype)
        p, dev, code, cnt = _ptr(out)
        self._check(self._lib.slim_get_x(self.h, p, cnt, code, dev))
        return out

    def step(self, nsteps=1):
        self._check(self._lib.slim_step(self.h, nsteps))

    def sync(self):
        self._check(self._lib.slim_sync(self.h))

    def join(self, stream_ptr):
        """Make the cudaStream_t `stream_ptr` wait (on the device) for everything
        the context has queued on all its streams, work prepared ahead included."""
        self._check(self._lib.slim_join_stream(self.h, C.c_void_p(stream_ptr)))

    def set_stream(self, stream_ptr):
        """Run the context's work on the cudaStream_t `stream_ptr`.  0 selects
        the context's own stream, not the legacy default stream, so torch's
        default stream (handle 0) cannot be named here: use a side stream."""
        self._check(self._lib.slim_set_stream(self.h, C.c_void_p(stream_ptr)))

    def set_ref(self, x_ref):
        if x_ref is None:
            self._check(self._lib.slim_set_ref(self.h, None, 0, 0, 0))
            return
        p, dev, code, cnt = _ptr(x_ref)
        self._check(self._lib.slim_set_ref(self.h, p, cnt, code, dev))

    def run(self, max_steps, tol=0.0, eval_every=1):
        k, sec, err = C.c_longlong(), C.c_double(), C.c_double()
        self._check(self._lib.slim_run(self.h, max_steps, tol, eval_every, C.byref(k),
                                       C.byref(sec), C.byref(err)))
        return k.value, sec.value, err.value

    def set_timing(self, on=True):
        self._check(self._lib.slim_set_timing(self.h, int(on)))

    def get_timing(self):
        """(per-phase ms of the last step as a dict, kernels per step)."""
        ms = (C.c_double * len(PHASES))()
        k = C.c_int()
        self._check(self._lib.slim_get_timing(self.h, ms, len(PHASES), C.byref(k)))
        return dict(zip(PHASES, list(ms))), k.value

    def backproject_data(self, out):
        """A^T b of the context's data into a float32 device tensor of n entries."""
        self._check(self._lib.slim_backproject_data(self.h, C.c_void_p(out.data_ptr())))
        return out

    def warm_start(self, net, s_in, s_out):
        """x_0 = s_out * net(s_in * A^T b), or 0 when its residual is not below ||b||.
        Returns (used, ||A x_0 - b|| / ||b||)."""
        used, ratio = C.c_int(), C.c_double()
        self._check(self._lib.slim_warm_start(self.h, net.h, s_in, s_out, C.byref(used),
                                              C.byref(ratio)))
        return bool(used.value), ratio.value

    def launch_log(self):
        """(mean factorisation ms, mean iterate-chain ms, iterate chains) since the
        previous call; pipelined form with timing on."""
        f, x, n = C.c_double(), C.c_double(), C.c_longlong()
        self._check(self._lib.slim_get_launch_log(self.h, C.byref(f), C.byref(x), C.byref(n)))
        return f.value, x.value, n.value

    def kernels_per_step(self):
        k = C.c_int()
        self._check(self._lib.slim_get_timing(self.h, None, 0, C.byref(k)))
        return k.value

    def get_iter(self):
        k = C.c_longlong()
        self._check(self._lib.slim_get_iter(self.h, C.byref(k)))
        return k.value

    def set_iter(self, k):
        self._check(self._lib.slim_set_iter(self.h, k))

    def checkpoint(self) -> bytes:
        ln = C.c_size_t()
        self._check(self._lib.slim_checkpoint(self.h, None, C.byref(ln)))
        buf = C.create_string_buffer(ln.value)
        self._check(self._lib.slim_checkpoint(self.h, buf, C.byref(ln)))
        return buf.raw[:ln.value]

    def restore(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self._lib.slim_restore(self.h, buf, len(blob)))

    def get_memory(self):
        ids = np.empty(self.p, dtype=np.int32)
        G = np.empty((self.p, self.p), dtype=np.float64)
        z = np.empty(self.p, dtype=np.float64)
        self._check(self._lib.slim_get_memory(self.h, ids.ctypes.data, G.ctypes.data,
                                              z.ctypes.data))
        return ids, G, z

    def get_csr(self):
        """(row_ptr, col, values as float32) of the stored matrix."""
        nnz = C.c_longlong()
        self._check(self._lib.slim_get_csr(self.h, C.byref(nnz), None, None, None))
        rp = np.empty(self.m + 1, dtype=np.int32)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value, dtype=np.float32)
        self._check(self._lib.slim_get_csr(self.h, C.byref(nnz), rp.ctypes.data, col.ctypes.data,
                                           val.ctypes.data))
        return rp, col, val

    def project(self, x, y, ray_ids=None):
        ids = C.c_void_p(ray_ids.data_ptr()) if ray_ids is not None else None
        cnt = ray_ids.numel() if ray_ids is not None else 0
        self._check(self._lib.slim_project(self.h, ids, cnt, C.c_void_p(x.data_ptr()),
                                           C.c_void_p(y.data_ptr())))

    def backproject(self, y, x, ray_ids=None):
        ids = C.c_void_p(ray_ids.data_ptr()) if ray_ids is not None else None
        cnt = ray_ids.numel() if ray_ids is not None else 0
        self._check(self._lib.slim_backproject(self.h, ids, cnt, C.c_void_p(y.data_ptr()),
                                               C.c_void_p(x.data_ptr())))


def selftest_wait(stream_ptr=0):
    """Status of a bounded device wait made to run out (SLIM_ETIMEOUT expected)."""
    return load().slim_selftest_wait(C.c_void_p(stream_ptr))


def damped_solve(G, lam, rhs, z, stream_ptr=0):
    """(lam I + G) z = rhs on the device (torch float64 CUDA tensors)."""
    lib = load()
    p = rhs.numel()
    st = lib.slim_damped_solve(C.c_void_p(G.data_ptr()), p, lam, C.c_void_p(rhs.data_ptr()),
                               C.c_void_p(z.data_ptr()), C.c_void_p(stream_ptr))
    if st != SLIM_OK:
        raise SlimError(st, "slim_damped_solve failed")


def tc_matmul(M, N, K, A, lda, a_km, B, ldb, b_kn, Cm, ldc, c_nm, alpha=1.0, beta=0.0,
              a_lower=False, b_lower=False, stream_ptr=0):
    """C = alpha op(A) op(B) + beta C on the tensor cores (torch float32 CUDA tensors;
    layouts as slim_tc_matmul documents)."""
    lib = load()
    st = lib.slim_tc_matmul(M, N, K, C.c_void_p(A.data_ptr()), lda, int(a_km),
                            C.c_void_p(B.data_ptr()), ldb, int(b_kn), C.c_void_p(Cm.data_ptr()),
                            ldc, int(c_nm), alpha, beta, int(a_lower), int(b_lower),
                            C.c_void_p(stream_ptr))
    if st != SLIM_OK:
        raise SlimError(st, "slim_tc_matmul failed")


def chol_inverse(G, lam, X, stream_ptr=0):
    """X = L^{-1} (lower) and L^{-T} (strict upper) of the float32 Cholesky factor of
    lam I + G (G torch float64, X torch float32 p x p, CUDA)."""
    lib = load()
    p = G.shape[0]
    st = lib.slim_chol_inverse(C.c_void_p(G.data_ptr()), p, lam, C.c_void_p(X.data_ptr()),
                               C.c_void_p(stream_ptr))
    if st != SLIM_OK:
        raise SlimError(st, "slim_chol_inverse failed")


def damped_solve_noalloc(G, lam, rhs, z, stream_ptr=0):
    """(lam I + G) z = rhs without device allocation (p <= NOALLOC_MAX_P); torch
    float64 CUDA tensors.  Scratch is a static device array shared by all calls."""
    lib = load()
    p = rhs.numel()
    st = lib.slim_damped_solve_noalloc(C.c_void_p(G.data_ptr()), p, lam,
                                       C.c_void_p(rhs.data_ptr()), C.c_void_p(z.data_ptr()),
                                       C.c_void_p(stream_ptr))
    if st != SLIM_OK:
        raise SlimError(st, "slim_damped_solve_noalloc failed")


def problem_structs(specs):
    """ctypes arrays (geometry, blocks, r, lambda, step options) for a list of
    dicts with keys N, n_views, det, ell, r, lam, seed and optional precision,
    solver, kind, use_graph, tile, ctas_per_sm, refine_iters, ray_lanes, pair_window."""
    n = len(specs)
    G = (slim_geometry * n)()
    B = (slim_blocks * n)()
    R = (C.c_int * n)()
    L = (C.c_double * n)()
    S = (slim_step_opts * n)()
    for i, sp in enumerate(specs):
        G[i] = slim_geometry(2, sp["N"], sp["n_views"], sp["det"], 1, None, 0, sp.get("precision", 0))
        B[i] = slim_blocks(sp.get("kind", SLIM_BLOCKS_RAYS), sp["ell"], sp["seed"], 1,
                           int(sp.get("with_replacement", True)), int(sp.get("cyclic", False)))
        R[i] = sp["r"]
        L[i] = sp["lam"]
        S[i] = slim_step_opts(1.0, 0, sp.get("solver", 0), sp.get("refine_iters", 2), 0,
                              sp.get("tile", 0), sp.get("ctas_per_sm", 0), sp.get("lookahead", 0))
        S[i].ray_lanes = sp.get("ray_lanes", 0)
        S[i].pair_window = sp.get("pair_window", 0)
    return G, B, R, L, S


def autotune_opts(spec, steps=3):
    """The autotuner's choice for a problem spec (dict as in problem_structs):
    a dict of tile, ctas_per_sm, ray_lanes, pair_window and the step time ms."""
    lib = load()
    G, B, R, L, S = problem_structs([spec])
    best = slim_step_opts()
    ms = C.c_double()
    st = lib.slim_autotune(C.byref(G[0]), C.byref(B[0]), R[0], L[0], C.byref(S[0]), steps,
                           C.byref(best), C.byref(ms))
    if st != SLIM_OK:
        raise SlimError(st, "slim_autotune failed")
    return {"tile": best.tile, "ctas_per_sm": best.ctas_per_sm, "ray_lanes": best.ray_lanes,
            "pair_window": best.pair_window, "ms": ms.value}


def autotune(spec, steps=3):
    """Best (tile, ctas_per_sm) for a problem spec (dict as in problem_structs)."""
    lib = load()
    G, B, R, L, S = problem_structs([spec])
    best = slim_step_opts()
    ms = C.c_double()
    st = lib.slim_autotune(C.byref(G[0]), C.byref(B[0]), R[0], L[0], C.byref(S[0]), steps,
                           C.byref(best), C.byref(ms))
    if st != SLIM_OK:
        raise SlimError(st, "slim_autotune failed")
    return best.tile, best.ctas_per_sm, ms.value


class SlimBatch:
    """Many independent problems advancing together (one CUDA graph launch per step)."""

    def __init__(self, specs):
        lib = load()
        self._lib = lib
        G, B, R, L, S = problem_structs(specs)
        self._keep = (G, B, R, L, S)
        h = C.c_void_p()
        st = lib.slim_batch_create(len(specs), G, B, R, L, S, C.byref(h))
        if st != SLIM_OK:
            raise SlimError(st, "slim_batch_create failed")
        self.h = h
        self.problems = []
        for i, sp in enumerate(specs):
            ch = C.c_void_p()
            lib.slim_batch_ctx(h, i, C.byref(ch))
            self.problems.append(Slim(sp["N"], sp["n_views"], sp["det"], sp["ell"], sp["r"], sp["lam"],
                                      sp["seed"], precision=sp.get("precision", 0), _handle=ch))

    def step(self, nsteps=1):
        st = self._lib.slim_batch_step(self.h, nsteps)
        if st != SLIM_OK:
            raise SlimError(st, "slim_batch_step failed")

    def sync(self):
        st = self._lib.slim_batch_sync(self.h)
        if st != SLIM_OK:
            raise SlimError(st, "slim_batch_sync failed")

    def set_stream(self, stream_ptr):
        st = self._lib.slim_batch_set_stream(self.h, C.c_void_p(stream_ptr))
        if st != SLIM_OK:
            raise SlimError(st, "slim_batch_set_stream failed")

    def close(self):
        if getattr(self, "h", None):
            for pb in self.problems:
                pb.h = None
            self._lib.slim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Layers of the warm-start network in the C ABI's parameter order:
# (name, weight shape, kind); convolution weights [out][in][3][3], transposed
# convolutions [in][out][2][2], the final 1x1 [1][32]; each bias follows its weights.
UNET_LAYERS = [
    ("enc1a", (32, 1, 3, 3), "conv"), ("enc1b", (32, 32, 3, 3), "conv"),
    ("enc2a", (64, 32, 3, 3), "conv"), ("enc2b", (64, 64, 3, 3), "conv"),
    ("enc3a", (128, 64, 3, 3), "conv"), ("enc3b", (128, 128, 3, 3), "conv"),
    ("bota", (256, 128, 3, 3), "conv"), ("botb", (256, 256, 3, 3), "conv"),
    ("up3", (256, 128, 2, 2), "tconv"),
    ("dec3a", (128, 256, 3, 3), "conv"), ("dec3b", (128, 128, 3, 3), "conv"),
    ("up2", (128, 64, 2, 2), "tconv"),
    ("dec2a", (64, 128, 3, 3), "conv"), ("dec2b", (64, 64, 3, 3), "conv"),
    ("up1", (64, 32, 2, 2), "tconv"),
    ("dec1a", (32, 64, 3, 3), "conv"), ("dec1b", (32, 32, 3, 3), "conv"),
    ("out", (1, 32), "conv1x1"),
]


class UNet:
    """The warm-start network (device weights, Adam state and buffers)."""

    def __init__(self, H, W, max_batch=1):
        lib = load()
        self._lib = lib
        h = C.c_void_p()
        st = lib.slim_unet_create(H, W, max_batch, C.byref(h))
        if st != SLIM_OK:
            raise SlimError(st, "slim_unet_create failed")
        self.h = h
        self.H, self.W, self.max_batch = H, W, max_batch
        n = C.c_longlong()
        lib.slim_unet_param_count(C.byref(n))
        self.nparams = n.value

    def _chk(self, st, what):
        if st != SLIM_OK:
            raise SlimError(st, what + " failed")

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        self._chk(self._lib.slim_unet_set_params(self.h, a.ctypes.data_as(C.c_void_p), a.size),
                  "slim_unet_set_params")

    def get_params(self):
        a = np.empty(self.nparams, dtype=np.float32)
        self._chk(self._lib.slim_unet_get_params(self.h, a.ctypes.data_as(C.c_void_p), a.size),
                  "slim_unet_get_params")
        return a

    def get_grads(self):
        a = np.empty(self.nparams, dtype=np.float32)
        self._chk(self._lib.slim_unet_get_grads(self.h, a.ctypes.data_as(C.c_void_p), a.size),
                  "slim_unet_get_grads")
        return a

    def forward(self, x, y, stream_ptr=0):
        """x, y: float32 device tensors of n*H*W entries."""
        n = x.numel() // (self.H * self.W)
        self._chk(self._lib.slim_unet_forward(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                              n, C.c_void_p(stream_ptr)), "slim_unet_forward")

    def train_step(self, x, target, lr, stream_ptr=0):
        n = x.numel() // (self.H * self.W)
        loss = C.c_double()
        self._chk(self._lib.slim_unet_train_step(self.h, C.c_void_p(x.data_ptr()),
                                                 C.c_void_p(target.data_ptr()), n, C.c_float(lr),
                                                 C.byref(loss), C.c_void_p(stream_ptr)),
                  "slim_unet_train_step")
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.slim_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dptr(t):
    """Device pointer of a contiguous float32 CUDA tensor, or NULL for None."""
    if t is None:
        return C.c_void_p(0)
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _layer_call(name, *args):
    st = getattr(load(), name)(*args)
    if st != SLIM_OK:
        raise SlimError(st, f"{name} failed")


def unet_conv3x3(x, n, c_in, H, W, w, b, c_out, relu, y, stream_ptr=0):
    """y = max?(conv3x3(x, w) + b) on [channel][image][H][W] device arrays."""
    _layer_call("slim_unet_conv3x3", _dptr(x), n, c_in, H, W, _dptr(w), _dptr(b), c_out,
                int(bool(relu)), _dptr(y), C.c_void_p(stream_ptr))


def unet_conv3x3_grad(x, dy, n, c_in, H, W, w, c_out, dw, db, dx, stream_ptr=0):
    """dw += dL/dw, db += dL/db, dx = dL/dx for dy at the conv's output."""
    _layer_call("slim_unet_conv3x3_grad", _dptr(x), _dptr(dy), n, c_in, H, W, _dptr(w), c_out,
                _dptr(dw), _dptr(db), _dptr(dx), C.c_void_p(stream_ptr))


def unet_tconv2x2(x, n, c_in, H, W, w, b, c_out, y, stream_ptr=0):
    """y = tconv2x2(x, w) + b (stride 2) on [channel][image][H][W] device arrays."""
    _layer_call("slim_unet_tconv2x2", _dptr(x), n, c_in, H, W, _dptr(w), _dptr(b), c_out,
                _dptr(y), C.c_void_p(stream_ptr))


def unet_tconv2x2_grad(x, dy, n, c_in, H, W, w, c_out, dw, db, dx, stream_ptr=0):
    """dw += dL/dw, db += dL/db, dx = dL/dx for dy at the transposed conv's output."""
    _layer_call("slim_unet_tconv2x2_grad", _dptr(x), _dptr(dy), n, c_in, H, W, _dptr(w), c_out,
                _dptr(dw), _dptr(db), _dptr(dx), C.c_void_p(stream_ptr))


def flatten_params(params, layers=UNET_LAYERS):
    """{name: (w, b)} -> one float32 array in the layer order of the C ABI."""
    return np.concatenate([np.concatenate([np.asarray(params[name][0], np.float32).ravel(),
                                           np.asarray(params[name][1], np.float32).ravel()])
                           for name, _, _ in layers])


def unflatten_params(flat, layers=UNET_LAYERS):
    out, o = {}, 0
    for name, shape, kind in layers:
        nw = int(np.prod(shape))
        nb = shape[1] if kind == "tconv" else shape[0]
        out[name] = (flat[o:o + nw].reshape(shape), flat[o + nw:o + nw + nb])
        o += nw + nb
    return out
