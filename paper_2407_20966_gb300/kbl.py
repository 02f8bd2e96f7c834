"""ctypes binding of libkbl (include/kbl.h): argument marshalling only.

Every compute call goes straight to the CUDA library; there is no CPU path.
Device arrays are torch CUDA float64 tensors (contiguous), host arrays are
numpy.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkbl.so")

OK, EINVAL, ENONPHYSICAL, ECUDA, ENOMEM, ETIMEOUT, ESTATE = range(7)
FP64, FP32_MIXED = 0, 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENONPHYSICAL", 3: "ECUDA", 4: "ENOMEM", 5: "ETIMEOUT",
           6: "ESTATE"}

# FR operator ids of kbl_get_operator
OP_NODES, OP_WEIGHTS, OP_LMINUS, OP_LPLUS, OP_D, OP_GL, OP_GR = range(7)


class KblError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class KblConfig(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("nu", C.c_int * 2), ("gamma", C.c_double),
                ("k", C.c_double), ("r_fac", C.c_double), ("eps", C.c_double),
                ("rho_floor", C.c_double), ("p_floor", C.c_double), ("eps_rule", C.c_int),
                ("precision", C.c_int), ("uncoupled", C.c_int), ("flux", C.c_int),
                ("quadrature", C.c_int), ("stencil", C.c_int)]


class KblCounters(C.Structure):
    _fields_ = [("nonphysical", C.c_int32), ("timeout", C.c_int32),
                ("limited_elements", C.c_int64), ("pressure_relimits", C.c_int64),
                ("eps_rule_activations", C.c_int64), ("mean_outside_bounds", C.c_int64),
                ("alpha_hist", C.c_int64 * 10)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); mirrors include/kbl.h
_P = C.c_void_p
_SIGS = {
    "kbl_config_default": (C.c_int, [C.POINTER(KblConfig), C.c_int, C.c_int]),
    "kbl_create": (C.c_int, [C.POINTER(_P), C.POINTER(KblConfig), _P]),
    "kbl_destroy": (C.c_int, [_P]),
    "kbl_set_stream": (C.c_int, [_P, _P]),
    "kbl_last_error": (C.c_char_p, [_P]),
    "kbl_nv": (C.c_int, [_P]),
    "kbl_ns": (C.c_int, [_P]),
    "kbl_nfp": (C.c_int, [_P]),
    "kbl_nstencil": (C.c_int, [_P]),
    "kbl_mesh_upload": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "kbl_get_operator": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "kbl_bounds_stencil": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "kbl_limit_nodes": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P]),
    "kbl_velocity_weights": (C.c_int, [C.c_int, C.c_int, _P]),
    "kbl_residual_operator": (C.c_int, [C.c_int, _P, C.c_int]),
    "kbl_traces": (C.c_int, [_P, _P, _P]),
    "kbl_gather_stencil": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, _P]),
    "kbl_bounds": (C.c_int, [_P, _P, _P, _P]),
    "kbl_rhs": (C.c_int, [_P, _P, _P, _P]),
    "kbl_limit": (C.c_int, [_P, _P, _P, _P]),
    "kbl_stage": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "kbl_dt": (C.c_int, [_P, _P, C.c_double, _P]),
    "kbl_step": (C.c_int, [_P, _P, C.c_double]),
    "kbl_set_time": (C.c_int, [_P, C.c_double, C.c_double]),
    "kbl_time_sync": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "kbl_run_host": (C.c_int, [_P, _P, _P, C.c_int, C.c_double]),
    "kbl_run_host_ensemble": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.c_double]),
    "kbl_check": (C.c_int, [_P]),
    "kbl_read_counters": (C.c_int, [_P, C.POINTER(KblCounters)]),
    "kbl_launch_count": (C.c_int64, [_P]),
    "kbl_bounds_noalloc": (C.c_int, [C.POINTER(KblConfig), C.c_int, _P, C.c_int, _P, _P, _P, _P]),
    "kbl_batch_create": (C.c_int, [C.POINTER(_P), C.POINTER(KblConfig), C.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "kbl_batch_destroy": (C.c_int, [_P]),
    "kbl_batch_last_error": (C.c_char_p, [_P]),
    "kbl_batch_layout": (C.c_int, [_P, _P, _P]),
    "kbl_batch_nodes": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "kbl_batch_step": (C.c_int, [_P, _P, C.c_double]),
    "kbl_batch_dt": (C.c_int, [_P, _P]),
    "kbl_batch_bounds": (C.c_int, [_P, _P, _P]),
    "kbl_batch_set_form": (C.c_int, [_P, C.c_int]),
    "kbl_batch_stall_test": (C.c_int, [_P, C.c_int, C.c_int]),
    "kbl_batch_bounds_ms": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "kbl_batch_run_host": (C.c_int, [_P, _P, _P, C.c_int, C.c_double]),
    "kbl_batch_rhs": (C.c_int, [_P, _P, _P]),
    "kbl_batch_stage": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "kbl_batch_autotune": (C.c_int, [_P, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "kbl_batch_tuning": (C.c_int, [_P, _P]),
    "kbl_batch_check": (C.c_int, [_P]),
    "kbl_batch_launch_count": (C.c_int64, [_P]),
    "kbl_set_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "kbl_get_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "kbl_traces_vjp": (C.c_int, [_P, _P, _P, _P]),
    "kbl_rhs_vjp": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "kbl_bounds_vjp": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "kbl_stage_vjp": (C.c_int, [_P, C.c_int, C.c_double, _P, _P, _P, _P, _P, C.c_int, _P, _P, _P, _P]),
    "kbl_entropy": (C.c_int, [_P, _P, _P]),
    "kbl_entropy_vjp": (C.c_int, [_P, _P, C.c_double, _P]),
    "kbl_step_fixed": (C.c_int, [_P, _P, C.c_double]),
    "kbl_adjoint_step": (C.c_int, [_P, _P, C.c_double, _P]),
    "kbl_adjoint_segment": (C.c_int, [_P, _P, _P, C.c_int, _P, _P]),
    "kbl_forward_segment": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "kbl_tri_points": (C.c_int, [C.c_int, _P, _P]),
    "kbl_tri_create": (C.c_int, [C.POINTER(_P), C.POINTER(KblConfig), C.c_int, _P, _P, _P, C.c_int, _P, _P]),
    "kbl_tri_create_curved": (C.c_int, [C.POINTER(_P), C.POINTER(KblConfig), C.c_int, _P, _P, _P, C.c_int, _P,
                                        _P]),
    "kbl_tri_destroy": (C.c_int, [_P]),
    "kbl_tri_last_error": (C.c_char_p, [_P]),
    "kbl_tri_traces": (C.c_int, [_P, _P, _P]),
    "kbl_tri_gather_stencil": (C.c_int, [_P, _P, _P, _P]),
    "kbl_tri_residual": (C.c_int, [_P, _P, _P, _P]),
    "kbl_tri_bounds": (C.c_int, [_P, _P, _P, _P]),
    "kbl_tri_dt": (C.c_int, [_P, _P, C.c_double, C.POINTER(C.c_double)]),
    "kbl_tri_step": (C.c_int, [_P, _P, C.c_double]),
    "kbl_tri_check": (C.c_int, [_P]),
}

TUNE_BOUNDS_TILE = 0
TUNE_RHS_TC = 1
TUNE_RHS_OVERLAP = 2


def exported_symbols():
    return list(_SIGS)


def load(path: str | None = None):
    """Load libkbl.so (build it first with paper_2407_20966_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise KblError(ESTATE, f"{p} not found: build the CUDA library first "
                                       "(python -m paper_2407_20966_gb300.build)")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dev(t, name="array"):
    """Device pointer of a contiguous CUDA float64 tensor (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor")
    return C.c_void_p(t.data_ptr())


def _host(a, dtype, name="array"):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _current_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """One method configuration bound to one CUDA stream and (after mesh_upload) one mesh."""

    def __init__(self, dim=2, p=3, nu=None, precision=FP64, stream=None, **overrides):
        lib = load()
        cfg = KblConfig()
        self._check_static(lib.kbl_config_default(C.byref(cfg), dim, p), "config_default")
        if nu is not None:
            nu = list(nu) + [nu[0]] * (2 - len(nu))
            cfg.nu[0], cfg.nu[1] = nu[0], (nu[1] if dim == 2 else 1)
        cfg.precision = precision
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        h = C.c_void_p()
        s = stream if stream is not None else _current_stream()
        self._check_static(lib.kbl_create(C.byref(h), C.byref(cfg), s), "create")
        self._h = h
        self._lib = lib
        self.dim, self.p = dim, p
        self.nv = lib.kbl_nv(h)
        self.ns = lib.kbl_ns(h)
        self.nfp = lib.kbl_nfp(h)
        self.nstencil = lib.kbl_nstencil(h)
        self.E = 0

    @staticmethod
    def _check_static(st, what):
        if st != OK:
            raise KblError(st, what)

    def _check(self, st, what):
        if st != OK:
            msg = self._lib.kbl_last_error(self._h)
            raise KblError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kbl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up --------------------------------------------------------
    def set_stream(self, stream=None):
        self._check(self._lib.kbl_set_stream(self._h, stream if stream is not None else _current_stream()),
                    "set_stream")

    def mesh_upload(self, nbr, h, bc=None):
        nbr, pn = _host(nbr, np.int32)
        hh, ph = _host(h, np.float64)
        bc = np.zeros((0, self.nv)) if bc is None else bc
        bc, pb = _host(bc, np.float64)
        E = nbr.shape[0]
        self._check(self._lib.kbl_mesh_upload(self._h, E, pn, ph, bc.shape[0] if bc.size else 0, pb),
                    "mesh_upload")
        self.E = E

    def bounds_stencil(self, S, bnd):
        """Bounds of explicit stencils (kbl_bounds_stencil): S float64 [E][n_states][4] and
        bnd float64 [2][4][E], CUDA tensors."""
        E, n = int(S.shape[0]), int(S.shape[1])
        self._check(self._lib.kbl_bounds_stencil(self._h, E, n, _dev(S, "S"), _dev(bnd, "bnd")), "bounds_stencil")

    def limit_nodes(self, W, U, F, bnd, alpha=None):
        """Limit explicit node sets (kbl_limit_nodes): W host [ns] positive mean weights; U float64
        [E][ns][nv] (limited in place), F float64 [E][nf][nv], bnd [2][nv][E], alpha [2][E] or
        None: CUDA tensors."""
        E, ns, nf = int(U.shape[0]), int(U.shape[1]), int(F.shape[1])
        Wh, pW = _host(W, np.float64, "W")
        self._check(self._lib.kbl_limit_nodes(self._h, E, ns, nf, pW, _dev(U, "U"), _dev(F, "F") if nf else None,
                                              _dev(bnd, "bnd"), _dev(alpha, "alpha")), "limit_nodes")

    def operator(self, which):
        n = (self.p + 1) ** 2 if which == OP_D else self.p + 1
        out = np.zeros(n)
        self._check(self._lib.kbl_get_operator(self._h, which, out.ctypes.data_as(C.c_void_p), n),
                    "get_operator")
        return out.reshape(self.p + 1, self.p + 1) if which == OP_D else out

    # ---- compute (device tensors) -------------------------------------
    def traces(self, w, wf):
        self._check(self._lib.kbl_traces(self._h, _dev(w, "w"), _dev(wf, "wf")), "traces")

    def gather_stencil(self, w, wf, e0, n, S):
        self._check(self._lib.kbl_gather_stencil(self._h, _dev(w), _dev(wf), e0, n, _dev(S)), "gather")

    def bounds(self, w, wf, bnd):
        self._check(self._lib.kbl_bounds(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(bnd, "bnd")), "bounds")

    def rhs(self, w, wf, R):
        self._check(self._lib.kbl_rhs(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(R, "R")), "rhs")

    def limit(self, w, bnd, alpha=None):
        self._check(self._lib.kbl_limit(self._h, _dev(w, "w"), _dev(bnd, "bnd"), _dev(alpha)), "limit")

    def stage(self, s, wn, ws, R, bnd, dt_dev, wout, alpha=None):
        self._check(self._lib.kbl_stage(self._h, s, _dev(wn), _dev(ws), _dev(R), _dev(bnd), _dev(dt_dev),
                                        _dev(wout), _dev(alpha)), "stage")

    def dt(self, w, cfl, dt_dev):
        self._check(self._lib.kbl_dt(self._h, _dev(w), float(cfl), _dev(dt_dev)), "dt")

    def step(self, w, cfl):
        self._check(self._lib.kbl_step(self._h, _dev(w, "w"), float(cfl)), "step")

    def set_time(self, t, t_end=float("inf")):
        self._check(self._lib.kbl_set_time(self._h, float(t), float(t_end)), "set_time")

    def time(self):
        t = C.c_double()
        self._check(self._lib.kbl_time_sync(self._h, C.byref(t)), "time_sync")
        return t.value

    def run_host(self, w_in: np.ndarray, w_out: np.ndarray, n_steps, cfl):
        for a in (w_in, w_out):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("host arrays must be contiguous float64")
        self._check(self._lib.kbl_run_host(self._h, w_in.ctypes.data_as(C.c_void_p),
                                           w_out.ctypes.data_as(C.c_void_p), int(n_steps), float(cfl)),
                    "run_host")

    def run_host_ensemble(self, w_in: np.ndarray, w_out: np.ndarray, n_steps, cfl):
        """Independent states w_in[k] ([members][nv][E][Ns], host) stepped n_steps each, into
        w_out[k]; copies overlap the steps of neighbouring members (kbl_run_host_ensemble)."""
        for a in (w_in, w_out):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("host arrays must be contiguous float64")
        if w_in.shape != w_out.shape:
            raise TypeError("input and output shapes differ")
        self._check(self._lib.kbl_run_host_ensemble(self._h, int(w_in.shape[0]), w_in.ctypes.data_as(C.c_void_p),
                                                    w_out.ctypes.data_as(C.c_void_p), int(n_steps), float(cfl)),
                    "run_host_ensemble")

    def check(self):
        self._check(self._lib.kbl_check(self._h), "check")

    def counters(self):
        k = KblCounters()
        st = self._lib.kbl_read_counters(self._h, C.byref(k))
        out = {f: getattr(k, f) for f, _ in KblCounters._fields_}
        out["alpha_hist"] = list(k.alpha_hist)
        return st, out

    def launch_count(self):
        return int(self._lib.kbl_launch_count(self._h))

    def set_tuning(self, key, value):
        self._check(self._lib.kbl_set_tuning(self._h, int(key), int(value)), "set_tuning")

    def get_tuning(self, key):
        v = C.c_int()
        self._check(self._lib.kbl_get_tuning(self._h, int(key), C.byref(v)), "get_tuning")
        return v.value

    # ---- reverse mode (device tensors; *_vjp add into their outputs) -----
    def traces_vjp(self, wfb, wfb_ext, wb):
        self._check(self._lib.kbl_traces_vjp(self._h, _dev(wfb, "wfb"), _dev(wfb_ext), _dev(wb, "wb")),
                    "traces_vjp")

    def rhs_vjp(self, w, wf, Rb, wb, wfb, wfb_ext):
        self._check(self._lib.kbl_rhs_vjp(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(Rb, "Rb"), _dev(wb, "wb"),
                                          _dev(wfb, "wfb"), _dev(wfb_ext, "wfb_ext")), "rhs_vjp")

    def bounds_vjp(self, w, wf, bnd, bndb, wb, wfb, wfb_ext):
        self._check(self._lib.kbl_bounds_vjp(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(bnd, "bnd"),
                                             _dev(bndb, "bndb"), _dev(wb, "wb"), _dev(wfb, "wfb"),
                                             _dev(wfb_ext, "wfb_ext")), "bounds_vjp")

    def stage_vjp(self, s, dt, wn, ws, R, bnd, ob, wnb, wsb, Rb, bndb, accumulate_wn=False):
        self._check(self._lib.kbl_stage_vjp(self._h, int(s), float(dt), _dev(wn, "wn"), _dev(ws, "ws"), _dev(R, "R"),
                                            _dev(bnd, "bnd"), _dev(ob, "ob"), int(bool(accumulate_wn)),
                                            _dev(wnb, "wnb"), _dev(wsb, "wsb"), _dev(Rb, "Rb"), _dev(bndb, "bndb")),
                    "stage_vjp")

    def entropy(self, w, J_dev):
        self._check(self._lib.kbl_entropy(self._h, _dev(w, "w"), _dev(J_dev, "J")), "entropy")

    def entropy_vjp(self, w, Jb, wb):
        self._check(self._lib.kbl_entropy_vjp(self._h, _dev(w, "w"), float(Jb), _dev(wb, "wb")), "entropy_vjp")

    def step_fixed(self, w, dt):
        self._check(self._lib.kbl_step_fixed(self._h, _dev(w, "w"), float(dt)), "step_fixed")

    def adjoint_step(self, w, dt, wbar):
        self._check(self._lib.kbl_adjoint_step(self._h, _dev(w, "w"), float(dt), _dev(wbar, "wbar")),
                    "adjoint_step")

    def forward_segment(self, w, dts, bnd_out=None):
        d, dp = _host(dts, np.float64, "dts")
        self._check(self._lib.kbl_forward_segment(self._h, _dev(w, "w"), dp, len(d), _dev(bnd_out)),
                    "forward_segment")

    def adjoint_segment(self, w0, dts, wbar, bnd_in=None):
        d, dp = _host(dts, np.float64, "dts")
        self._check(self._lib.kbl_adjoint_segment(self._h, _dev(w0, "w0"), dp, len(d), _dev(bnd_in),
                                                  _dev(wbar, "wbar")), "adjoint_segment")


def _dev_any(t, dtype_name, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    if str(t.dtype) != dtype_name:
        raise TypeError(f"{name} must be {dtype_name}")
    return C.c_void_p(t.data_ptr())


def residual_operator(p):
    """The 2D FR residual as one matrix B[K][Ns] of order p (kbl_residual_operator; host only)."""
    N = int(p) + 1
    K, NS = 2 * N * N + 4 * N, N * N
    out = np.zeros(K * NS)
    st = load().kbl_residual_operator(int(p), out.ctypes.data_as(C.c_void_p), K * NS)
    if st != OK:
        raise KblError(st, "residual_operator")
    return out.reshape(K, NS)


def velocity_weights(nu, quadrature=0):
    """The library's velocity quadrature weights on an axis of nu points, in units of the grid
    spacing (kbl_velocity_weights; host only)."""
    out = np.zeros(int(nu))
    st = load().kbl_velocity_weights(int(nu), int(quadrature), out.ctypes.data_as(C.c_void_p))
    if st != OK:
        raise KblError(st, "velocity_weights")
    return out


def bounds_noalloc(cfg: KblConfig, nbr, bc, w, bnd, stream=None):
    """Element bounds with no device allocation (kbl_bounds_noalloc): nbr int32 [E][2d],
    bc float64 [n_bc][nv], w float64 [nv][E][Ns] and bnd float64 [2][nv][E], all CUDA tensors."""
    lib = load()
    E = int(nbr.shape[0])
    n_bc = int(bc.shape[0]) if bc is not None and bc.numel() else 0
    pb = _dev_any(bc, "torch.float64", "bc") if n_bc else None
    st = lib.kbl_bounds_noalloc(C.byref(cfg), E, _dev_any(nbr, "torch.int32", "nbr"), n_bc, pb,
                                _dev_any(w, "torch.float64", "w"), _dev_any(bnd, "torch.float64", "bnd"),
                                stream if stream is not None else _current_stream())
    if st != OK:
        raise KblError(st, "bounds_noalloc")


class Batch:
    """Many independent 2D problems advanced together (kbl_batch_*): FP32-mixed, orders 1..4,
    32 x 32 velocity grid.  meshes: list of (p, nbr[E][4], h[E][2], bc[n_bc][4])."""

    def __init__(self, meshes, stream=None, **overrides):
        lib = load()
        cfg = KblConfig()
        if lib.kbl_config_default(C.byref(cfg), 2, 1) != OK:
            raise KblError(EINVAL, "config_default")
        cfg.precision = FP32_MIXED
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.p = np.ascontiguousarray([m[0] for m in meshes], dtype=np.int32)
        self.n_elem = np.ascontiguousarray([len(m[1]) for m in meshes], dtype=np.int32)
        nbr = np.ascontiguousarray(np.concatenate([np.asarray(m[1], np.int32).reshape(-1, 4) for m in meshes]))
        h = np.ascontiguousarray(np.concatenate([np.asarray(m[2], np.float64).reshape(-1, 2) for m in meshes]))
        nbc = np.ascontiguousarray([len(m[3]) for m in meshes], dtype=np.int32)
        bcs = [np.asarray(m[3], np.float64).reshape(-1, 4) for m in meshes]
        bc = np.ascontiguousarray(np.concatenate(bcs) if sum(len(b) for b in bcs) else np.zeros((1, 4)))
        hnd = C.c_void_p()
        s = stream if stream is not None else _current_stream()
        st = lib.kbl_batch_create(C.byref(hnd), C.byref(cfg), len(meshes), self.p.ctypes.data_as(C.c_void_p),
                                  self.n_elem.ctypes.data_as(C.c_void_p), nbr.ctypes.data_as(C.c_void_p),
                                  h.ctypes.data_as(C.c_void_p), nbc.ctypes.data_as(C.c_void_p),
                                  bc.ctypes.data_as(C.c_void_p), s)
        if st != OK:
            raise KblError(st, "batch_create")
        self._h, self._lib, self.P = hnd, lib, len(meshes)
        so = np.zeros(self.P + 1, np.int64)
        eo = np.zeros(self.P + 1, np.int64)
        self._check(lib.kbl_batch_layout(hnd, so.ctypes.data_as(C.c_void_p), eo.ctypes.data_as(C.c_void_p)),
                    "layout")
        self.state_offsets, self.elem_offsets = so, eo

    def _check(self, st, what):
        if st != OK:
            msg = self._lib.kbl_batch_last_error(self._h)
            raise KblError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kbl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nodes(self, p):
        out = np.zeros(p + 1)
        self._check(self._lib.kbl_batch_nodes(self._h, p, out.ctypes.data_as(C.c_void_p), p + 1), "nodes")
        return out

    def state_view(self, w, i):
        """Problem i's block of the concatenated state as [4][E_i][(p_i+1)^2] (a view)."""
        a, b = int(self.state_offsets[i]), int(self.state_offsets[i + 1])
        return w[a:b].reshape(4, int(self.n_elem[i]), (int(self.p[i]) + 1) ** 2)

    def step(self, w, cfl):
        self._check(self._lib.kbl_batch_step(self._h, _dev(w, "w"), float(cfl)), "batch_step")

    def dt(self):
        out = np.zeros(self.P)
        self._check(self._lib.kbl_batch_dt(self._h, out.ctypes.data_as(C.c_void_p)), "batch_dt")
        return out

    def set_form(self, fused):
        """1: one persistent launch per step (default); 0: one launch per phase."""
        self._check(self._lib.kbl_batch_set_form(self._h, int(fused)), "batch_set_form")

    def stall_test(self, on, wait_polls=1 << 20):
        self._check(self._lib.kbl_batch_stall_test(self._h, int(on), int(wait_polls)), "batch_stall_test")

    def bounds_view(self, bnd, i):
        """Problem i's bounds [2][4][E_i] in a concatenated bounds array (a view)."""
        a, n = 8 * int(self.elem_offsets[i]), int(self.n_elem[i])
        return bnd[a:a + 8 * n].reshape(2, 4, n)

    def bounds(self, w, bnd):
        self._check(self._lib.kbl_batch_bounds(self._h, _dev(w, "w"), _dev(bnd, "bnd")), "batch_bounds")

    def bounds_ms(self):
        """Device time of the bounds launch of the last bounds() call (ms)."""
        ms = C.c_double()
        self._check(self._lib.kbl_batch_bounds_ms(self._h, C.byref(ms)), "batch_bounds_ms")
        return ms.value

    def run_host(self, w_in: np.ndarray, w_out: np.ndarray, n_steps, cfl):
        """End to end on host buffers (kbl_batch_run_host): copies overlap the steps by groups."""
        for a in (w_in, w_out):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != int(self.state_offsets[-1]):
                raise TypeError("host arrays must be contiguous float64 of the batch state's size")
        self._check(self._lib.kbl_batch_run_host(self._h, w_in.ctypes.data_as(C.c_void_p),
                                                 w_out.ctypes.data_as(C.c_void_p), int(n_steps), float(cfl)),
                    "batch_run_host")

    def rhs(self, w, R):
        self._check(self._lib.kbl_batch_rhs(self._h, _dev(w, "w"), _dev(R, "R")), "batch_rhs")

    def stage(self, s, wn, ws, R, bnd, dt_dev, wout):
        self._check(self._lib.kbl_batch_stage(self._h, int(s), _dev(wn, "wn"), _dev(ws, "ws"), _dev(R, "R"),
                                              _dev(bnd, "bnd"), _dev(dt_dev, "dt"), _dev(wout, "wout")),
                    "batch_stage")

    def autotune(self, w, with_cmp=False):
        ms, cmp = C.c_double(), C.c_double()
        self._check(self._lib.kbl_batch_autotune(self._h, _dev(w, "w"), C.byref(ms), C.byref(cmp)),
                    "batch_autotune")
        return (ms.value, cmp.value) if with_cmp else ms.value

    def tuning(self):
        out = np.zeros(4, np.int32)
        self._check(self._lib.kbl_batch_tuning(self._h, out.ctypes.data_as(C.c_void_p)), "batch_tuning")
        return {"tile": int(out[0]), "elements_per_item": int(out[1]), "blocks_per_sm": int(out[2]),
                "items": int(out[3])}   # tile: 0 = 4x4, 1 = 4x2, 2 = 2x4 velocity nodes per thread

    def check(self):
        self._check(self._lib.kbl_batch_check(self._h), "batch_check")

    def launch_count(self):
        return int(self._lib.kbl_batch_launch_count(self._h))


def tri_points(p):
    """Williams-Shunn solution points rs[ns][2] and weights w[ns] of order p (host only)."""
    ns = (int(p) + 1) * (int(p) + 2) // 2
    rs, w = np.zeros((ns, 2)), np.zeros(ns)
    st = load().kbl_tri_points(int(p), rs.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p))
    if st != OK:
        raise KblError(st, "tri_points")
    return rs, w


class TriMesh:
    """Affine triangles of order p in {1, 2} (kbl_tri_*): xy[E][3][2] counterclockwise,
    nbr[E][3] (neighbour or -(b+1)), nbr_edge[E][3], bc[n_bc][4] -- host arrays.  Solution
    arrays are CUDA float64 tensors w[E][ns][4]."""

    def __init__(self, p, xy, nbr, nbr_edge, bc, precision=FP64, stream=None, xy6=None, **overrides):
        lib = load()
        cfg = KblConfig()
        if lib.kbl_config_default(C.byref(cfg), 2, int(p)) != OK:
            raise KblError(EINVAL, "config_default")
        cfg.precision = precision
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        xy, px = _host(xy, np.float64, "xy")
        nb, pn = _host(nbr, np.int32, "nbr")
        ne, pe = _host(nbr_edge, np.int32, "nbr_edge")
        bc, pb = _host(bc, np.float64, "bc")
        self.E = int(xy.reshape(-1, 6).shape[0])
        n_bc = int(bc.reshape(-1, 4).shape[0]) if bc.size else 0
        h = C.c_void_p()
        s = stream if stream is not None else _current_stream()
        if xy6 is None:
            st = lib.kbl_tri_create(C.byref(h), C.byref(cfg), self.E, px, pn, pe, n_bc, pb if n_bc else None, s)
        else:   # curved elements: the corners and the edges' mid-parameter points
            x6, p6 = _host(xy6, np.float64, "xy6")
            st = lib.kbl_tri_create_curved(C.byref(h), C.byref(cfg), self.E, p6, pn, pe, n_bc,
                                           pb if n_bc else None, s)
        if st != OK:
            raise KblError(st, "tri_create")
        self._h, self._lib = h, lib
        self.p = int(p)
        self.ns = (self.p + 1) * (self.p + 2) // 2
        self.nfp = 3 * (self.p + 1)
        self.nstencil = self.ns + 2 * self.nfp

    def _check(self, st, what):
        if st != OK:
            msg = self._lib.kbl_tri_last_error(self._h)
            raise KblError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kbl_tri_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def traces(self, w, wf):
        self._check(self._lib.kbl_tri_traces(self._h, _dev(w, "w"), _dev(wf, "wf")), "tri_traces")

    def gather_stencil(self, w, wf, S):
        self._check(self._lib.kbl_tri_gather_stencil(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(S, "S")),
                    "tri_gather_stencil")

    def bounds(self, w, wf, bnd):
        """Bounds [2][4][E] of every stencil, gathered inside the kernel (kbl_tri_bounds)."""
        self._check(self._lib.kbl_tri_bounds(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(bnd, "bnd")), "tri_bounds")

    def residual(self, w, wf, R):
        self._check(self._lib.kbl_tri_residual(self._h, _dev(w, "w"), _dev(wf, "wf"), _dev(R, "R")),
                    "tri_residual")

    def dt(self, w, cfl):
        out = C.c_double()
        self._check(self._lib.kbl_tri_dt(self._h, _dev(w, "w"), float(cfl), C.byref(out)), "tri_dt")
        return out.value

    def step(self, w, dt):
        self._check(self._lib.kbl_tri_step(self._h, _dev(w, "w"), float(dt)), "tri_step")

    def check(self):
        self._check(self._lib.kbl_tri_check(self._h), "tri_check")
