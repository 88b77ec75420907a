"""ctypes binding of libtnite (include/tnite.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
memory (the context workspace, kernel-level operands) comes from PyTorch
tensors; host arrays are numpy float64.  The library must have been built
(paper_1411_0391_gb300.build); there is no fallback implementation.
"""
import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_PATH = os.path.join(_HERE, "libtnite.so")
_LIB = None

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ECUDA, TN_ENOCONV, TN_ENUMERIC, TN_ESTATE, TN_ESCRATCH, TN_ETIMEOUT, TN_EUNSTABLE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
TN_CELL_CHECKERBOARD, TN_CELL_SINGLE = 2, 1
TN_F64, TN_TF32X3, TN_BF16X3, TN_BF16S4, TN_F64S7 = 0, 1, 2, 3, 4
(TN_T_STATE, TN_T_CANON, TN_T_LAMBDA, TN_T_THETA, TN_T_PRE_P, TN_T_PRE_Q, TN_T_DOUBLE,
 TN_T_BOND_ENV, TN_T_FU_P, TN_T_FU_Q, TN_T_GAUGE_W, TN_T_GATE_K, TN_T_PEPO) = range(13)


class tn_config(ctypes.Structure):
    _fields_ = [("D", c_int), ("chi", c_int), ("cell", c_int), ("precision", c_int)]


class tn_ctm_report(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("converged", c_int), ("delta", c_double), ("svd_calls", c_int),
                ("svd_iterations", c_int)]


class tn_step_report(ctypes.Structure):
    _fields_ = [("canon_iters", c_int), ("ctm_iterations", c_int), ("ctm_delta", c_double),
                ("als_iters", c_int * 8), ("als_cost", c_double * 8)]


TN_RECYCLE_OFF, TN_RECYCLE_FIXED, TN_RECYCLE_THRESHOLD = 0, 1, 2


class tn_evolve_opts(ctypes.Structure):
    _fields_ = [("recycle", c_int), ("n_re", c_int), ("ctm_tol", c_double), ("ctm_max", c_int),
                ("recycle_eps", c_double), ("check_every", c_int), ("warmup_plain", c_int),
                ("als_tol", c_double), ("als_max", c_int), ("min_fidelity", c_double)]


class tn_evolve_report(ctypes.Structure):
    _fields_ = [("steps", c_int), ("env_computations", c_int), ("ctm_iterations", c_int),
                ("ctm_moves", c_int), ("nonconverged", c_int), ("last_fidelity", c_double),
                ("checks", c_int), ("last_change", c_double), ("fallbacks", c_int), ("final_n_re", c_int)]


class tn_observables(ctypes.Structure):
    _fields_ = [("e_site", c_double), ("e_link", c_double), ("mx", c_double * 2), ("mz", c_double * 2),
                ("zz", c_double * 4)]


_DP = POINTER(c_double)
_SIGS = {
    "tn_launch_count": (ctypes.c_ulonglong, []),
    "tn_workspace_bytes": (c_size_t, [POINTER(tn_config)]),
    "tn_create": (c_int, [POINTER(c_void_p), POINTER(tn_config), c_void_p, c_size_t, c_void_p]),
    "tn_destroy": (None, [c_void_p]),
    "tn_strerror": (ctypes.c_char_p, [c_int]),
    "tn_set_hamiltonian": (c_int, [c_void_p, c_double, c_double]),
    "tn_set_time_step": (c_int, [c_void_p, c_double]),
    "tn_set_state": (c_int, [c_void_p, _DP, c_size_t]),
    "tn_get_state": (c_int, [c_void_p, _DP, c_size_t]),
    "tn_build_double_layer": (c_int, [c_void_p]),
    "tn_set_network": (c_int, [c_void_p, _DP, c_int, _DP]),
    "tn_reset_env": (c_int, [c_void_p]),
    "tn_ctmrg": (c_int, [c_void_p, c_double, c_int, POINTER(tn_ctm_report)]),
    "tn_ctmrg_moves": (c_int, [c_void_p, c_int]),
    "tn_env_size": (c_size_t, [c_void_p]),
    "tn_get_env": (c_int, [c_void_p, _DP, c_size_t]),
    "tn_set_env": (c_int, [c_void_p, _DP, c_size_t]),
    "tn_corner_spectra": (c_int, [c_void_p, _DP, c_size_t]),
    "tn_site_scalars": (c_int, [c_void_p, c_int, _DP, _DP]),
    "tn_step_prepare": (c_int, [c_void_p, POINTER(tn_step_report)]),
    "tn_step_update": (c_int, [c_void_p, POINTER(tn_step_report)]),
    "tn_fu_step": (c_int, [c_void_p, c_double, c_int, POINTER(tn_step_report)]),
    "tn_su_step": (c_int, [c_void_p, POINTER(tn_step_report)]),
    "tn_recycle": (c_int, [c_void_p, c_int, _DP]),
    "tn_evolve": (c_int, [c_void_p, c_int, POINTER(tn_evolve_opts), POINTER(tn_evolve_report)]),
    "tn_measure": (c_int, [c_void_p, POINTER(tn_observables)]),
    "tn_evolve_batch": (c_int, [POINTER(c_void_p), c_int, c_int, POINTER(tn_evolve_opts), c_int, POINTER(c_int),
                                POINTER(tn_evolve_report)]),
    "tn_set_autotune": (c_int, [c_int]),
    "tn_imps_workspace_bytes": (c_size_t, [c_int]),
    "tn_imps_itebd": (c_int, [c_void_p, c_int, c_double, c_double, c_int, c_void_p, c_size_t, c_void_p]),
    "tn_imps_recycle": (c_int, [c_void_p, c_int, c_double, c_double, c_int, POINTER(c_double), c_void_p, c_size_t,
                                c_void_p]),
    "tn_imps_observables": (c_int, [c_void_p, c_int, c_double, POINTER(c_double), c_void_p, c_size_t, c_void_p]),
    "tn_get_tensor": (c_int, [c_void_p, c_int, c_int, _DP, c_size_t]),
    "tn_gemm_f64": (c_int, [c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_int, c_longlong,
                            c_void_p, c_int, c_longlong, c_double, c_void_p, c_int, c_longlong, c_int, c_void_p]),
    "tn_set_projector_cutoff": (c_int, [c_void_p, c_double]),
    "tn_gemm_split_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int]),
    "tn_gemm_split": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_int, c_void_p, c_int,
                              c_double, c_void_p, c_int, c_void_p, c_size_t, c_void_p]),
    "tn_selftest_wait_timeout": (c_int, [c_void_p]),
    "tn_fp64_rate_probe": (c_int, [c_int, POINTER(c_double), c_void_p]),
    "tn_permute_f64": (c_int, [c_void_p, c_void_p, c_int, POINTER(c_int), POINTER(c_int), c_void_p]),
    "tn_svd_small": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tn_eigh_small": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "tn_truncated_svd": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tn_truncated_svd_noalloc": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load libtnite.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_PATH):
            raise RuntimeError("libtnite.so is missing: build it with paper_1411_0391_gb300.build.build()")
        L = ctypes.CDLL(_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class TnError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().tn_strerror(status).decode()
        super().__init__("%s: %s (%d)" % (where, msg, status))
        self.status = status


def _check(status, where, allow_noconv=False):
    if status == TN_OK or (allow_noconv and status == TN_ENOCONV):
        return status
    raise TnError(status, where)


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_ptr(stream):
    return c_void_p(0 if stream is None else stream.cuda_stream)


def tn_launch_count():
    return int(lib().tn_launch_count())


# ---- kernel-level entry points (torch device tensors) ------------------------

def tn_gemm_f64(transA, transB, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC,
                batch, stream=None):
    _check(lib().tn_gemm_f64(int(transA), int(transB), m, n, k, alpha, c_void_p(A.data_ptr()), lda, strideA,
                             c_void_p(B.data_ptr()), ldb, strideB, beta, c_void_p(C.data_ptr()), ldc, strideC,
                             batch, _stream_ptr(stream)), "tn_gemm_f64")


def tn_gemm_split_workspace_bytes(precision, m, n, k):
    return int(lib().tn_gemm_split_workspace_bytes(precision, m, n, k))


def tn_gemm_split(precision, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, work, stream=None):
    """work: a device tensor of at least tn_gemm_split_workspace_bytes bytes (256-byte aligned)."""
    _check(lib().tn_gemm_split(precision, int(transA), int(transB), m, n, k, alpha, c_void_p(A.data_ptr()), lda,
                               c_void_p(B.data_ptr()), ldb, beta, c_void_p(C.data_ptr()), ldc,
                               c_void_p(work.data_ptr()), work.numel() * work.element_size(), _stream_ptr(stream)),
           "tn_gemm_split")


def tn_selftest_wait_timeout(stream=None):
    """Status of the bounded-wait self-test (TN_ETIMEOUT when the limit works)."""
    return int(lib().tn_selftest_wait_timeout(_stream_ptr(stream)))


def tn_fp64_rate_probe(iters, stream=None):
    """Launch the FP64 FMA probe (no sync); returns the FLOPs it performs."""
    f = c_double(0.0)
    _check(lib().tn_fp64_rate_probe(iters, byref(f), _stream_ptr(stream)), "tn_fp64_rate_probe")
    return f.value


def tn_permute_f64(inp, out, dims, perm, stream=None):
    r = len(dims)
    _check(lib().tn_permute_f64(c_void_p(inp.data_ptr()), c_void_p(out.data_ptr()), r, (c_int * r)(*dims),
                                (c_int * r)(*perm), _stream_ptr(stream)), "tn_permute_f64")


def tn_svd_small(A, m, n, batch, U, S, V, stream=None):
    _check(lib().tn_svd_small(c_void_p(A.data_ptr()), m, n, batch, c_void_p(U.data_ptr()), c_void_p(S.data_ptr()),
                              c_void_p(V.data_ptr()), _stream_ptr(stream)), "tn_svd_small")


def tn_eigh_small(A, n, batch, W, V, stream=None):
    _check(lib().tn_eigh_small(c_void_p(A.data_ptr()), n, batch, c_void_p(W.data_ptr()), c_void_p(V.data_ptr()),
                               _stream_ptr(stream)), "tn_eigh_small")


def tn_truncated_svd(ctx, M, m, k, U, S, V, warm=None):
    return _check(lib().tn_truncated_svd(ctx.handle, c_void_p(M.data_ptr()), m, k, c_void_p(U.data_ptr()),
                                         c_void_p(S.data_ptr()), c_void_p(V.data_ptr()),
                                         c_void_p(0 if warm is None else warm.data_ptr())),
                  "tn_truncated_svd", allow_noconv=True)


def tn_truncated_svd_noalloc(M, m, k, U, S, V, warm=None, stream=None):
    """Allocation-free truncated SVD: only the caller's buffers, fixed 8 MiB library scratch."""
    return _check(lib().tn_truncated_svd_noalloc(c_void_p(M.data_ptr()), m, k, c_void_p(U.data_ptr()),
                                                 c_void_p(S.data_ptr()), c_void_p(V.data_ptr()),
                                                 c_void_p(0 if warm is None else warm.data_ptr()),
                                                 _stream_ptr(stream)),
                  "tn_truncated_svd_noalloc", allow_noconv=True)


def tn_set_autotune(enable):
    """Turn the FP64 product tile autotuner on or off; returns the shapes tuned so far."""
    return int(lib().tn_set_autotune(1 if enable else 0))


def _evolve_opts(n_re, recycle, ctm_tol, ctm_max, recycle_eps, check_every, warmup_plain, als_tol, als_max,
                 min_fidelity):
    mode = TN_RECYCLE_THRESHOLD if recycle == "threshold" else (TN_RECYCLE_FIXED if recycle else TN_RECYCLE_OFF)
    eps = float("inf") if recycle_eps is None else recycle_eps
    return tn_evolve_opts(mode, n_re, ctm_tol, ctm_max, eps, check_every, warmup_plain, als_tol, als_max,
                          min_fidelity)


def _report(rep, s):
    return dict(steps=rep.steps, env_computations=rep.env_computations, ctm_iterations=rep.ctm_iterations,
                ctm_moves=rep.ctm_moves, nonconverged=rep.nonconverged, last_fidelity=rep.last_fidelity,
                checks=rep.checks, last_change=rep.last_change, fallbacks=rep.fallbacks,
                final_n_re=rep.final_n_re, status=s)


def tn_evolve_batch(contexts, n_steps, recycle=False, n_re=1, ctm_tol=1e-10, ctm_max=500, recycle_eps=None,
                    check_every=1, warmup_plain=0, als_tol=1e-12, als_max=50, min_fidelity=0.0, n_threads=0):
    """Evolve independent contexts (each on its own stream) concurrently; one report per context."""
    n = len(contexts)
    arr = (c_void_p * n)(*[c.handle for c in contexts])
    o = _evolve_opts(n_re, recycle, ctm_tol, ctm_max, recycle_eps, check_every, warmup_plain, als_tol, als_max,
                     min_fidelity)
    st = (c_int * n)()
    reps = (tn_evolve_report * n)()
    _check(lib().tn_evolve_batch(arr, n, n_steps, byref(o), n_threads, st, reps), "tn_evolve_batch")
    return [_report(reps[i], st[i]) for i in range(n)]


class IMPS:
    """A one-site iMPS on the GPU (1D chain, Sec. III and V): device tensor + workspace (torch)."""

    def __init__(self, A, device="cuda:0", stream=None):
        import torch
        A = np.ascontiguousarray(A, dtype=np.float64)
        self.chi = int(A.shape[1])
        nbytes = int(lib().tn_imps_workspace_bytes(self.chi))
        if nbytes == 0:
            raise TnError(TN_EINVAL, "tn_imps_workspace_bytes")
        self.A = torch.from_numpy(A).to(device)
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream

    def _w(self):
        return c_void_p(self.work.data_ptr()), self.work.numel()

    def tn_imps_itebd(self, h, tau, n_steps):
        w, nb = self._w()
        _check(lib().tn_imps_itebd(c_void_p(self.A.data_ptr()), self.chi, h, tau, n_steps, w, nb,
                                   _stream_ptr(self.stream)), "tn_imps_itebd")

    def tn_imps_recycle(self, h, tau, n_re):
        F = c_double(0.0)
        w, nb = self._w()
        _check(lib().tn_imps_recycle(c_void_p(self.A.data_ptr()), self.chi, h, tau, n_re, byref(F), w, nb,
                                     _stream_ptr(self.stream)), "tn_imps_recycle")
        return F.value

    def tn_imps_observables(self, h):
        out = (c_double * 3)()
        w, nb = self._w()
        _check(lib().tn_imps_observables(c_void_p(self.A.data_ptr()), self.chi, h, out, w, nb,
                                         _stream_ptr(self.stream)), "tn_imps_observables")
        return dict(zz=out[0], x=out[1], e=out[2])

    def state(self):
        return self.A.cpu().numpy()


# ---- context -----------------------------------------------------------------

class Context:
    """One tnite context: its device workspace is a torch uint8 tensor on `device`."""

    def __init__(self, D, chi, cell=TN_CELL_CHECKERBOARD, device="cuda:0", stream=None, precision=TN_F64):
        import torch
        self.cfg = tn_config(D, chi, cell, precision)
        nbytes = lib().tn_workspace_bytes(byref(self.cfg))
        if nbytes == 0:
            raise TnError(TN_EINVAL, "tn_workspace_bytes")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = c_void_p()
        _check(lib().tn_create(byref(h), byref(self.cfg), c_void_p(self.workspace.data_ptr()), nbytes,
                               c_void_p(self.stream.cuda_stream)), "tn_create")
        self.handle = h
        self.D, self.chi = D, chi
        self.n_tensors = 2 if cell == TN_CELL_CHECKERBOARD else 1
        self.n_links = 2 * self.n_tensors
        self.n_sites = 4 if cell == TN_CELL_CHECKERBOARD else 1

    def close(self):
        if getattr(self, "handle", None):
            lib().tn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # problem definition
    def tn_set_hamiltonian(self, J, h):
        _check(lib().tn_set_hamiltonian(self.handle, J, h), "tn_set_hamiltonian")

    def tn_set_time_step(self, tau):
        _check(lib().tn_set_time_step(self.handle, tau), "tn_set_time_step")

    def tn_set_state(self, tensors):
        buf = _f64(np.concatenate([np.ravel(t) for t in tensors]))
        _check(lib().tn_set_state(self.handle, _dp(buf), buf.size), "tn_set_state")

    def tn_get_state(self):
        per = 2 * self.D ** 4
        buf = np.empty(per * self.n_tensors)
        _check(lib().tn_get_state(self.handle, _dp(buf), buf.size), "tn_get_state")
        return [buf[i * per:(i + 1) * per].reshape(2, *(self.D,) * 4).copy() for i in range(self.n_tensors)]

    # environment
    def tn_build_double_layer(self):
        _check(lib().tn_build_double_layer(self.handle), "tn_build_double_layer")

    def tn_set_network(self, tensors, boundary=None):
        a = _f64(np.concatenate([np.ravel(t) for t in tensors]))
        leg = int(tensors[0].shape[0])
        b = None if boundary is None else _f64(boundary)
        _check(lib().tn_set_network(self.handle, _dp(a), leg, None if b is None else _dp(b)), "tn_set_network")
        self.leg = leg

    def tn_reset_env(self):
        _check(lib().tn_reset_env(self.handle), "tn_reset_env")

    def tn_ctmrg(self, tol, max_iter):
        rep = tn_ctm_report()
        s = _check(lib().tn_ctmrg(self.handle, tol, max_iter, byref(rep)), "tn_ctmrg", allow_noconv=True)
        return dict(iterations=rep.iterations, converged=bool(rep.converged), delta=rep.delta, status=s,
                    svd_calls=rep.svd_calls, svd_iterations=rep.svd_iterations)

    def tn_ctmrg_moves(self, n):
        _check(lib().tn_ctmrg_moves(self.handle, n), "tn_ctmrg_moves")

    def tn_get_env(self):
        n = lib().tn_env_size(self.handle)
        buf = np.empty(n)
        _check(lib().tn_get_env(self.handle, _dp(buf), n), "tn_get_env")
        return buf

    def tn_set_env(self, buf):
        buf = _f64(buf)
        _check(lib().tn_set_env(self.handle, _dp(buf), buf.size), "tn_set_env")

    def tn_corner_spectra(self):
        buf = np.empty(self.n_sites * 4 * self.chi)
        _check(lib().tn_corner_spectra(self.handle, _dp(buf), buf.size), "tn_corner_spectra")
        return buf.reshape(self.n_sites, 4, self.chi)

    def tn_site_scalars(self, site, a=None):
        out = np.empty(4)
        ap = None if a is None else _f64(a)
        _check(lib().tn_site_scalars(self.handle, site, None if ap is None else _dp(ap), _dp(out)), "tn_site_scalars")
        return out

    # imaginary-time step
    @staticmethod
    def _step(rep):
        return dict(canon_iters=rep.canon_iters, ctm_iterations=rep.ctm_iterations, ctm_delta=rep.ctm_delta,
                    als_iters=list(rep.als_iters), als_cost=list(rep.als_cost))

    def tn_step_prepare(self):
        rep = tn_step_report()
        _check(lib().tn_step_prepare(self.handle, byref(rep)), "tn_step_prepare")
        return self._step(rep)

    def tn_step_update(self):
        rep = tn_step_report()
        _check(lib().tn_step_update(self.handle, byref(rep)), "tn_step_update")
        return self._step(rep)

    def tn_fu_step(self, ctm_tol, ctm_max):
        rep = tn_step_report()
        _check(lib().tn_fu_step(self.handle, ctm_tol, ctm_max, byref(rep)), "tn_fu_step", allow_noconv=True)
        return self._step(rep)

    def tn_su_step(self):
        r = tn_step_report()
        _check(lib().tn_su_step(self.handle, byref(r)), "tn_su_step")
        return dict(canon_iters=r.canon_iters)

    def tn_recycle(self, n_re):
        F = c_double(0.0)
        _check(lib().tn_recycle(self.handle, n_re, byref(F)), "tn_recycle")
        return F.value

    def tn_evolve(self, n_steps, recycle=False, n_re=1, ctm_tol=1e-10, ctm_max=500, recycle_eps=None,
                  check_every=1, warmup_plain=0, als_tol=1e-12, als_max=50, min_fidelity=0.0):
        """recycle: False/True (fixed windows of n_re) or "threshold" (windows of at most n_re,
        ended when the bond environment drifts by more than recycle_eps).  The returned
        "status" is TN_OK or TN_EUNSTABLE (windows redone without recycling: "fallbacks")."""
        o = _evolve_opts(n_re, recycle, ctm_tol, ctm_max, recycle_eps, check_every, warmup_plain, als_tol, als_max,
                         min_fidelity)
        rep = tn_evolve_report()
        s = lib().tn_evolve(self.handle, n_steps, byref(o), byref(rep))
        if s != TN_EUNSTABLE:
            _check(s, "tn_evolve")
        return _report(rep, s)

    def tn_set_projector_cutoff(self, cut):
        _check(lib().tn_set_projector_cutoff(self.handle, cut), "tn_set_projector_cutoff")

    def tn_measure(self):
        o = tn_observables()
        _check(lib().tn_measure(self.handle, byref(o)), "tn_measure")
        nt, nl = self.n_tensors, self.n_links
        return dict(e_site=o.e_site, e_link=o.e_link, mx=list(o.mx)[:nt], mz=list(o.mz)[:nt], zz=list(o.zz)[:nl])

    def tn_get_tensor(self, which, index, shape):
        buf = np.empty(int(np.prod(shape)))
        _check(lib().tn_get_tensor(self.handle, which, index, _dp(buf), buf.size), "tn_get_tensor")
        return buf.reshape(shape)
