"""Python binding of the C ABI in include/gp.h (argument marshalling only).

Every computation runs in the CUDA library ``libgp_gb300.so``; this module only
moves pointers, sizes and streams across.  PyTorch supplies device memory (inputs,
outputs and the workspace) and the current CUDA stream.  If the library is
missing the import of this module fails: there is no fallback path.

Blocks of vectors are n x t matrices stored column-major on the C side.  Here
they are torch tensors of shape (n, t); they are passed as the column-major
storage of their transpose and returned the same way.
"""
import ctypes
import os
import re

import torch

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "gp.h")

RBF, MATERN32, MATERN52, RATQUAD = 0, 3, 5, 7
FP64, FP32, TF32, BF16 = 0, 1, 2, 3
FN_KERNEL_MVM, FN_KERNEL_GRAD_MVM, FN_PIVCHOL, FN_MBCG, FN_MLL_AND_GRAD = range(5)
STATUS = {0: "GP_OK", 1: "GP_WARN_NOT_CONVERGED", 2: "GP_WARN_RANK_DEFICIENT",
          -1: "GP_ERR_INVALID_ARG", -2: "GP_ERR_CUDA", -3: "GP_ERR_NOT_SPD",
          -4: "GP_ERR_WORKSPACE", -5: "GP_ERR_DEVICE_TIMEOUT", -6: "GP_ERR_NUMERIC"}

OUT_MLL, OUT_QUAD, OUT_LOGDETP, OUT_STOCH, OUT_LOGDET, OUT_HEAD = 0, 1, 2, 3, 4, 8
IOUT_STATUS, IOUT_RANK, IOUT_ITERS = 0, 1, 2


class GPError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} returned {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("ard", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("X", ctypes.c_void_p), ("theta", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("cg_tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("recompute_every", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("pivchol_tol", ctypes.c_double), ("check_every", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


_LIB = None


def library_path():
    return _build.LIB


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: run paper_2107_00243_gb300.build.build() "
                          "(the estimator has no CPU fallback)")
    lib = ctypes.CDLL(_build.LIB)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER(_Problem)
    O = ctypes.POINTER(_Opts)
    sig = {
        "gp_workspace_size": (sz, [i32, i64, i32, i32, i32, i32, i32]),
        "gp_kernel_mvm": (i32, [P, vp, i64, i32, vp, i64, vp, sz, vp]),
        "gp_kernel_grad_mvm": (i32, [P, vp, i64, i32, vp, i64, vp, sz, vp]),
        "gp_pivchol": (i32, [P, i32, ctypes.c_double, vp, vp, i64, vp, vp, vp, sz, vp]),
        "gp_mbcg": (i32, [P, vp, i64, i32, vp, i64, i32, vp, vp, i64, vp, vp, vp, vp, vp, vp,
                          O, vp, sz, vp]),
        "gp_mll_and_grad": (i32, [P, vp, i32, i32, vp, vp, vp, vp, vp, O, vp, sz, vp]),
        "gp_mll_and_grad_rff": (i32, [P, vp, i32, i32, vp, vp, vp, vp, vp, vp, O, vp, sz,
                                      vp]),
        "gp_mll_and_grad_qff": (i32, [P, vp, i32, i32, vp, vp, vp, vp, O, vp, sz, vp]),
        "gp_qff_rule": (i32, [i32, i32, vp, vp]),
        "gp_status_string": (ctypes.c_char_p, [i32]),
        "gp_last_error_message": (ctypes.c_char_p, []),
        "gp_rademacher": (i32, [ctypes.c_uint64, i32, i64, i32, vp, vp]),
        "gp_tc_exponent_tile": (i32, [P, vp, i64, i32, vp, i64, vp, vp, sz, vp]),
        "gp_kernel_mvm_noalloc": (i32, [P, vp, i64, i32, vp, i64, vp]),
        "gp_workspace_size_batched": (sz, [i32, P, i32, i32, i32]),
        "gp_autotune": (i32, [P, vp, i64, i32, vp, i64, vp, sz, vp, vp]),
        "gp_tc_config": (i32, [P, i32, vp]),
        "gp_mll_and_grad_batched": (i32, [i32, P, vp, i32, i32, vp, vp, O, vp, sz, vp]),
        "gp_launch_count": (i64, []),
        "gp_peaks_scratch_elems": (sz, []),
        "gp_measure_peaks": (i32, [vp, ctypes.POINTER(ctypes.c_double), vp]),
        "gp_mvm_timing": (None, [i32]),
        "gp_mvm_timing_read": (i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
        "gp_phase_timing_read": (i32, [i32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def declared_functions():
    """Names of the functions declared in include/gp.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gp_[a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


def _check(fn, status):
    if status < 0:
        msg = load().gp_last_error_message().decode()
        raise GPError(fn, status, msg)
    return status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def real_dtype(precision):
    return torch.float64 if precision == FP64 else torch.float32


def _colmajor(V, dtype, device):
    """(n, t) tensor -> contiguous (t, n) storage (column-major n x t)."""
    if V.dim() == 1:
        V = V[:, None]
    return V.to(device=device, dtype=dtype).t().contiguous()


class Problem:
    """A GP regression problem resident on the GPU: X (n x d), theta, kernel, precision."""

    def __init__(self, X, theta, kind=RBF, ard=True, precision=FP32, device="cuda"):
        self.precision = precision
        self.dtype = real_dtype(precision)
        self.X = torch.as_tensor(X).to(device=device, dtype=self.dtype).contiguous()
        self.theta = torch.as_tensor(theta).to(device=device, dtype=torch.float64).contiguous()
        self.kind = kind
        self.ard = bool(ard)
        self.n, self.d = self.X.shape
        self.D = self.d if self.ard else 1
        self.p = self.D + 2
        assert self.theta.numel() == self.p, (self.theta.numel(), self.p)
        self._c = _Problem(self.n, self.d, kind, int(self.ard), precision,
                           self.X.data_ptr(), self.theta.data_ptr())

    @property
    def device(self):
        return self.X.device

    def set_theta(self, theta):
        self.theta.copy_(torch.as_tensor(theta, dtype=torch.float64))

    def cref(self):
        self._c.X = self.X.data_ptr()
        self._c.theta = self.theta.data_ptr()
        return ctypes.byref(self._c)


OPT_SPLIT_P, OPT_AUTO_SPLIT, OPT_FAST_ONLY, OPT_SIMT_GRAD = 1, 2, 4, 8


def opts(cg_tol=1e-6, max_iter=200, recompute_every=0, seed=0, pivchol_tol=0.0, check_every=0,
         flags=0):
    return _Opts(float(cg_tol), int(max_iter), int(recompute_every), int(seed),
                 float(pivchol_tol), int(check_every), int(flags))


def status_string(code):
    """Name of a gp_status code."""
    return load().gp_status_string(int(code)).decode()


def opts_with(o, **changes):
    """A copy of the options struct `o` with the named fields replaced."""
    fields = {name: getattr(o, name) for name, _ in _Opts._fields_}
    for name, value in changes.items():
        if name not in fields:
            raise KeyError(f"gp_opts has no field {name!r}")
        fields[name] = value
    return opts(**fields)


def gp_workspace_size(fn, n, d, k, t, precision, max_iter=1):
    return int(load().gp_workspace_size(fn, n, d, k, t, precision, max_iter))


class Workspace:
    """Caches one device buffer and grows it on demand."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes, device):
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        return self.buf


_WS = Workspace()


def gp_kernel_mvm(prob, V, workspace=None):
    """W = (K + sigma^2 I) V for V of shape (n, t)."""
    lib = load()
    Vc = _colmajor(V, prob.dtype, prob.device)
    t = Vc.shape[0]
    W = torch.empty_like(Vc)
    ws = (workspace or _WS).get(gp_workspace_size(FN_KERNEL_MVM, prob.n, prob.d, 0, t,
                                                  prob.precision), prob.device)
    _check("gp_kernel_mvm", lib.gp_kernel_mvm(prob.cref(), _ptr(Vc), prob.n, t, _ptr(W), prob.n,
                                              _ptr(ws), ws.numel(), _stream()))
    return W.t()


def gp_kernel_mvm_noalloc(prob, V):
    """W = (K + sigma^2 I) V through the entry point that allocates nothing (its
    scratch is a static device array inside the library; FP32 / FP64 only)."""
    lib = load()
    Vc = _colmajor(V, prob.dtype, prob.device)
    t = Vc.shape[0]
    W = torch.empty_like(Vc)
    _check("gp_kernel_mvm_noalloc",
           lib.gp_kernel_mvm_noalloc(prob.cref(), _ptr(Vc), prob.n, t, _ptr(W), prob.n,
                                     _stream()))
    return W.t()


def gp_tc_exponent_tile(prob, V, workspace=None):
    """(W, S): the BF16 tensor-core product and its first 128 x 128 exponent tile."""
    lib = load()
    Vc = _colmajor(V, prob.dtype, prob.device)
    t = Vc.shape[0]
    W = torch.empty_like(Vc)
    S = torch.full((128, 128), float("nan"), dtype=torch.float32, device=prob.device)
    ws = (workspace or _WS).get(gp_workspace_size(FN_KERNEL_MVM, prob.n, prob.d, 0, t,
                                                  prob.precision), prob.device)
    _check("gp_tc_exponent_tile",
           lib.gp_tc_exponent_tile(prob.cref(), _ptr(Vc), prob.n, t, _ptr(W), prob.n, _ptr(S),
                                   _ptr(ws), ws.numel(), _stream()))
    return W.t(), S


def gp_kernel_grad_mvm(prob, V, workspace=None):
    """Stacked [dK_hat/dtheta_q V] of shape (p, n, t)."""
    lib = load()
    Vc = _colmajor(V, prob.dtype, prob.device)
    t = Vc.shape[0]
    dW = torch.empty((prob.p, t, prob.n), dtype=prob.dtype, device=prob.device)
    ws = (workspace or _WS).get(gp_workspace_size(FN_KERNEL_GRAD_MVM, prob.n, prob.d, 0, t,
                                                  prob.precision), prob.device)
    _check("gp_kernel_grad_mvm",
           lib.gp_kernel_grad_mvm(prob.cref(), _ptr(Vc), prob.n, t, _ptr(dW), prob.n, _ptr(ws),
                                  ws.numel(), _stream()))
    return dW.transpose(1, 2)


def _piv_override(piv_override, k, device):
    """k int32 pivots for the device: a shorter order is padded with -1 (an entry
    outside [0, n) stops the factor there); a longer one is an error."""
    po = torch.as_tensor(piv_override, dtype=torch.int32).reshape(-1)
    if po.numel() > max(k, 0):
        raise ValueError(f"piv_override has {po.numel()} entries, more than k = {k}")
    if po.numel() < k:
        po = torch.cat([po, torch.full((k - po.numel(),), -1, dtype=torch.int32)])
    return po.to(device).contiguous()


def gp_pivchol(prob, k, tol=0.0, piv_override=None, workspace=None):
    """Returns (L (n, k), piv (k,) int32, rank int tensor)."""
    lib = load()
    L = torch.empty((max(k, 1), prob.n), dtype=prob.dtype, device=prob.device)
    piv = torch.empty(max(k, 1), dtype=torch.int32, device=prob.device)
    rank = torch.empty(1, dtype=torch.int32, device=prob.device)
    po = None
    if piv_override is not None and k > 0:
        po = _piv_override(piv_override, k, prob.device)
    ws = (workspace or _WS).get(gp_workspace_size(FN_PIVCHOL, prob.n, prob.d, k, 1,
                                                  prob.precision), prob.device)
    _check("gp_pivchol", lib.gp_pivchol(prob.cref(), k, float(tol), _ptr(po), _ptr(L), prob.n,
                                        _ptr(piv), _ptr(rank), _ptr(ws), ws.numel(), _stream()))
    return L[:k].t(), piv[:k], rank


def gp_mbcg(prob, L, B, o, iters_override=None, workspace=None):
    """Preconditioned CG on B (n, t) with P = sigma^2 I + L L^T.  Synchronises."""
    lib = load()
    k = 0 if L is None else L.shape[1]
    Lc = _colmajor(L, prob.dtype, prob.device) if k > 0 else None
    Bc = _colmajor(B, prob.dtype, prob.device)
    t = Bc.shape[0]
    Xs = torch.empty_like(Bc)
    PinvB = torch.empty_like(Bc)
    Td = torch.empty((t, o.max_iter), dtype=torch.float64, device=prob.device)
    To = torch.empty_like(Td)
    rho0 = torch.empty(t, dtype=torch.float64, device=prob.device)
    iters = torch.empty(t, dtype=torch.int32, device=prob.device)
    status = torch.empty(1, dtype=torch.int32, device=prob.device)
    io = None
    if iters_override is not None:
        io = torch.as_tensor(iters_override, dtype=torch.int32).reshape(-1)
        if io.numel() != t:
            raise ValueError(f"iters_override has {io.numel()} entries, not t = {t}")
        io = io.to(prob.device).contiguous()
    ws = (workspace or _WS).get(gp_workspace_size(FN_MBCG, prob.n, prob.d, k, t, prob.precision,
                                                  o.max_iter), prob.device)
    st = _check("gp_mbcg", lib.gp_mbcg(prob.cref(), _ptr(Lc), prob.n, k, _ptr(Bc), prob.n, t,
                                       _ptr(io), _ptr(Xs), prob.n, _ptr(PinvB), _ptr(Td),
                                       _ptr(To), _ptr(rho0), _ptr(iters), _ptr(status),
                                       ctypes.byref(o), _ptr(ws), ws.numel(), _stream()))
    return {"X": Xs.t(), "PinvB": PinvB.t(), "T_diag": Td, "T_off": To, "rho0": rho0,
            "iters": iters, "status": st}


def out_len(p, n_probes):
    return OUT_HEAD + 4 * p + n_probes


def gp_mll_and_grad(prob, y, k, n_probes, o, eps_override=None, piv_override=None,
                    iters_override=None, workspace=None, out=None, iout=None):
    """The estimator (Alg. 1 + Alg. 2).  Returns (status, out, iout) device tensors."""
    lib = load()
    t = n_probes + 1
    yd = torch.as_tensor(y).to(device=prob.device, dtype=prob.dtype).contiguous()
    if out is None:
        out = torch.empty(out_len(prob.p, n_probes), dtype=torch.float64, device=prob.device)
    if iout is None:
        iout = torch.empty(2 + t + max(k, 1), dtype=torch.int32, device=prob.device)
    eo = po = io = None
    if eps_override is not None:
        eo = torch.as_tensor(eps_override)
        if tuple(eo.shape) != (k + prob.n, n_probes):
            raise ValueError(f"eps_override has shape {tuple(eo.shape)}, not "
                             f"(k + n, n_probes) = {(k + prob.n, n_probes)}")
        eo = eo.to(device=prob.device, dtype=torch.int8)
        eo = eo.t().contiguous()          # ((k + n), l) column-major
    if piv_override is not None and k > 0:
        po = _piv_override(piv_override, k, prob.device)
    if iters_override is not None:
        io = torch.as_tensor(iters_override, dtype=torch.int32).reshape(-1)
        if io.numel() != t:
            raise ValueError(f"iters_override has {io.numel()} entries, not t = {t}")
        io = io.to(prob.device).contiguous()
    ws = (workspace or _WS).get(gp_workspace_size(FN_MLL_AND_GRAD, prob.n, prob.d, k, t,
                                                  prob.precision, o.max_iter), prob.device)
    st = _check("gp_mll_and_grad",
                lib.gp_mll_and_grad(prob.cref(), _ptr(yd), k, n_probes, _ptr(eo), _ptr(po),
                                    _ptr(io), _ptr(out), _ptr(iout), ctypes.byref(o), _ptr(ws),
                                    ws.numel(), _stream()))
    return st, out, iout


def rff_gamma_shape(kind):
    """Shape nu of the Gamma(nu, 1) draws g that gp_mll_and_grad_rff expects for a kernel
    (None: the RBF needs none)."""
    return {RBF: None, MATERN32: 1.5, MATERN52: 2.5, RATQUAD: 1.0}[kind]


def gp_mll_and_grad_rff(prob, y, m, n_probes, o, eps, g=None, eps_override=None,
                        iters_override=None, workspace=None, out=None, iout=None):
    """The estimator with a random Fourier feature preconditioner of 2m features built
    from the draws eps (m, d) ~ N(0, 1) and g (m,) ~ Gamma(nu, 1) (Matern-nu), Gamma(1, 1)
    (rational quadratic) or None (RBF).  Returns (status, out, iout) device tensors,
    laid out as for gp_mll_and_grad with k = 2m."""
    lib = load()
    t = n_probes + 1
    k = 2 * m
    yd = torch.as_tensor(y).to(device=prob.device, dtype=prob.dtype).contiguous()
    ed = torch.as_tensor(eps, dtype=torch.float64).to(prob.device).contiguous()
    if tuple(ed.shape) != (m, prob.d):
        raise ValueError(f"eps has shape {tuple(ed.shape)}, not (m, d) = {(m, prob.d)}")
    gd = None
    if g is not None:
        gd = torch.as_tensor(g, dtype=torch.float64).to(prob.device).contiguous()
        if gd.numel() != m:
            raise ValueError(f"g has {gd.numel()} entries, not m = {m}")
    if out is None:
        out = torch.empty(out_len(prob.p, n_probes), dtype=torch.float64, device=prob.device)
    if iout is None:
        iout = torch.empty(2 + t + max(k, 1), dtype=torch.int32, device=prob.device)
    eo = io = None
    if eps_override is not None:
        eo = torch.as_tensor(eps_override)
        if tuple(eo.shape) != (k + prob.n, n_probes):
            raise ValueError(f"eps_override has shape {tuple(eo.shape)}, not "
                             f"(k + n, n_probes) = {(k + prob.n, n_probes)}")
        eo = eo.to(device=prob.device, dtype=torch.int8).t().contiguous()
    if iters_override is not None:
        io = torch.as_tensor(iters_override, dtype=torch.int32).reshape(-1)
        if io.numel() != t:
            raise ValueError(f"iters_override has {io.numel()} entries, not t = {t}")
        io = io.to(prob.device).contiguous()
    ws = (workspace or _WS).get(gp_workspace_size(FN_MLL_AND_GRAD, prob.n, prob.d, k, t,
                                                  prob.precision, o.max_iter), prob.device)
    st = _check("gp_mll_and_grad_rff",
                lib.gp_mll_and_grad_rff(prob.cref(), _ptr(yd), m, n_probes, _ptr(ed), _ptr(gd),
                                        _ptr(eo), _ptr(io), _ptr(out), _ptr(iout),
                                        ctypes.byref(o), _ptr(ws), ws.numel(), _stream()))
    return st, out, iout


def gp_qff_rule(mbar, d):
    """(U (m, d), W (m,)) numpy arrays: the quadrature rule of gp_mll_and_grad_qff."""
    import numpy as np
    lib = load()
    m = _check("gp_qff_rule", lib.gp_qff_rule(int(mbar), int(d), None, None))
    U = np.zeros((m, d))
    W = np.zeros(m)
    _check("gp_qff_rule", lib.gp_qff_rule(int(mbar), int(d), U.ctypes.data, W.ctypes.data))
    return U, W


def gp_mll_and_grad_qff(prob, y, mbar, n_probes, o, eps_override=None, iters_override=None,
                        workspace=None, out=None, iout=None):
    """The estimator with the quadrature Fourier feature preconditioner (RBF kernel,
    mbar Gauss-Hermite nodes per dimension, k = mbar^d features).  Synchronises.
    Returns (status, out, iout), laid out as for gp_mll_and_grad with k = mbar^d."""
    lib = load()
    t = n_probes + 1
    k = int(mbar) ** prob.d
    yd = torch.as_tensor(y).to(device=prob.device, dtype=prob.dtype).contiguous()
    if out is None:
        out = torch.empty(out_len(prob.p, n_probes), dtype=torch.float64, device=prob.device)
    if iout is None:
        iout = torch.empty(2 + t + max(k, 1), dtype=torch.int32, device=prob.device)
    eo = io = None
    if eps_override is not None:
        eo = torch.as_tensor(eps_override)
        if tuple(eo.shape) != (k + prob.n, n_probes):
            raise ValueError(f"eps_override has shape {tuple(eo.shape)}, not "
                             f"(k + n, n_probes) = {(k + prob.n, n_probes)}")
        eo = eo.to(device=prob.device, dtype=torch.int8).t().contiguous()
    if iters_override is not None:
        io = torch.as_tensor(iters_override, dtype=torch.int32).reshape(-1)
        if io.numel() != t:
            raise ValueError(f"iters_override has {io.numel()} entries, not t = {t}")
        io = io.to(prob.device).contiguous()
    # the library rejects k above its limit (min(n, 2048)) before touching the workspace
    ws = (workspace or _WS).get(gp_workspace_size(FN_MLL_AND_GRAD, prob.n, prob.d,
                                                  min(k, prob.n, 2048), t, prob.precision,
                                                  o.max_iter), prob.device)
    st = _check("gp_mll_and_grad_qff",
                lib.gp_mll_and_grad_qff(prob.cref(), _ptr(yd), int(mbar), n_probes, _ptr(eo),
                                        _ptr(io), _ptr(out), _ptr(iout), ctypes.byref(o),
                                        _ptr(ws), ws.numel(), _stream()))
    return st, out, iout


def gp_autotune(prob, V, workspace=None):
    """Tune the tensor-core product's launch configuration for this shape; returns
    (W, {chunks, b_ring, v_ring, candidates})."""
    lib = load()
    Vc = _colmajor(V, prob.dtype, prob.device)
    t = Vc.shape[0]
    W = torch.empty_like(Vc)
    ws = (workspace or _WS).get(gp_workspace_size(FN_KERNEL_MVM, prob.n, prob.d, 0, t,
                                                  prob.precision), prob.device)
    best = (ctypes.c_int32 * 4)()
    _check("gp_autotune", lib.gp_autotune(prob.cref(), _ptr(Vc), prob.n, t, _ptr(W), prob.n,
                                          _ptr(ws), ws.numel(), _stream(),
                                          ctypes.cast(best, ctypes.c_void_p)))
    return W.t(), {"chunks": best[0], "b_ring": best[1], "v_ring": best[2],
                   "candidates": best[3]}


def gp_tc_config(prob, t):
    c = (ctypes.c_int32 * 4)()
    _check("gp_tc_config", load().gp_tc_config(prob.cref(), t, ctypes.cast(c, ctypes.c_void_p)))
    return {"chunks": c[0], "b_ring": c[1], "v_ring": c[2], "tuned": bool(c[3])}


def _problem_array(probs):
    arr = (_Problem * len(probs))()
    for i, pr in enumerate(probs):
        pr.cref()                      # refresh the data pointers
        arr[i] = pr._c
    return arr


def gp_workspace_size_batched(probs, k, n_probes, max_iter):
    arr = _problem_array(probs)
    return int(load().gp_workspace_size_batched(len(probs), arr, k, n_probes, max_iter))


class Batch:
    """Device buffers of one batched evaluation (gp_mll_and_grad_batched): the
    problems, their targets, outputs and workspace, kept alive together so that the
    library's cached CUDA graph for these pointers stays valid across calls."""

    def __init__(self, probs, ys, k, n_probes, o):
        self.probs, self.k, self.n_probes, self.o = list(probs), k, n_probes, o
        t = n_probes + 1
        self.ys = [torch.as_tensor(y).to(device=pr.device, dtype=pr.dtype).contiguous()
                   for pr, y in zip(self.probs, ys)]
        self.outs = [torch.zeros(out_len(pr.p, n_probes), dtype=torch.float64, device=pr.device)
                     for pr in self.probs]
        self.iouts = [torch.zeros(2 + t + max(k, 1), dtype=torch.int32, device=pr.device)
                      for pr in self.probs]
        nbytes = gp_workspace_size_batched(self.probs, k, n_probes, o.max_iter)
        if nbytes == 0:
            raise GPError("gp_workspace_size_batched", -1, "invalid batch")
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.probs[0].device)
        vp = ctypes.c_void_p
        self._arr = _problem_array(self.probs)
        self._ys = (vp * len(self.probs))(*[y.data_ptr() for y in self.ys])
        self._outs = (vp * len(self.probs))(*[x.data_ptr() for x in self.outs])
        self._iouts = (vp * len(self.probs))(*[x.data_ptr() for x in self.iouts])

    def run(self):
        """Launch the batch on the current stream (asynchronous); returns the status."""
        return _check("gp_mll_and_grad_batched", load().gp_mll_and_grad_batched(
            len(self.probs), self._arr, self._ys, self.k, self.n_probes, self._outs,
            self._iouts, ctypes.byref(self.o), _ptr(self.ws), self.ws.numel(), _stream()))

    def results(self):
        """Host dicts (unpack) of every problem, after synchronising."""
        torch.cuda.synchronize()
        return [unpack(o, io, pr.p, self.n_probes, self.k)
                for pr, o, io in zip(self.probs, self.outs, self.iouts)]


def gp_mll_and_grad_batched(probs, ys, k, n_probes, o):
    """One call of the batched estimator; returns the Batch (outputs in .outs/.iouts)."""
    b = Batch(probs, ys, k, n_probes, o)
    b.run()
    return b


def unpack(out, iout, p, n_probes, k):
    """Host dict of the estimator outputs (layout of GP_OUT_* / GP_IOUT_* in gp.h)."""
    o = out.double().cpu().numpy()
    io = iout.cpu().numpy()
    t = n_probes + 1
    h = OUT_HEAD
    return {
        "mll": o[OUT_MLL], "quad": o[OUT_QUAD], "logdetP": o[OUT_LOGDETP],
        "stoch": o[OUT_STOCH], "logdet": o[OUT_LOGDET],
        "drift_quad": o[5], "drift_logdet": o[6],
        "grad": o[h:h + p].copy(), "gK": o[h + p:h + 2 * p].copy(),
        "probeP_p": o[h + 2 * p:h + 3 * p].copy(), "trP_p": o[h + 3 * p:h + 4 * p].copy(),
        "gamma": o[h + 4 * p:h + 4 * p + n_probes].copy(),
        "status": int(io[0]), "rank": int(io[1]), "iters": io[2:2 + t].copy(),
        "piv": io[2 + t:2 + t + k].copy(),
    }


def gp_rademacher(seed, stream_id, rows, cols, device="cuda"):
    """(rows, cols) int8 tensor of +-1 signs from the on-device generator."""
    lib = load()
    out = torch.empty((cols, rows), dtype=torch.int8, device=device)
    _check("gp_rademacher", lib.gp_rademacher(int(seed), int(stream_id), int(rows), int(cols),
                                              _ptr(out), _stream()))
    return out.t()


def launch_count():
    """Kernels launched by the library since it was loaded."""
    return int(load().gp_launch_count())


def mvm_timing(enable):
    load().gp_mvm_timing(1 if enable else 0)


def measure_peaks():
    """Measured throughputs of the units the path uses (gp_measure_peaks): FP32 FMA
    FLOP/s, ex2.approx.f32 results/s, ex2.approx.f16x2 results/s, FP64 FMA FLOP/s."""
    lib = load()
    scratch = torch.empty(int(lib.gp_peaks_scratch_elems()), dtype=torch.float32, device="cuda")
    out = (ctypes.c_double * 4)()
    _check("gp_measure_peaks", lib.gp_measure_peaks(_ptr(scratch), out, _stream()))
    return {"fp32_fma_flops": out[0], "ex2_f32_per_s": out[1], "ex2_f16x2_per_s": out[2],
            "fp64_fma_flops": out[3]}


def mvm_timing_read():
    """(total ms, number of kernel-matrix products) timed since the last read."""
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check("gp_mvm_timing_read", load().gp_mvm_timing_read(ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def phase_timing_read(phase):
    """(total ms, brackets) of a timed phase since the last read: 0 = kernel-matrix
    products, 1 = the gradient contraction (one bracket per evaluation), 2 = a CG
    iteration's work outside its products (two brackets per iteration, eager calls)."""
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check("gp_phase_timing_read",
           load().gp_phase_timing_read(int(phase), ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value
