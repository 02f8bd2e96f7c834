"""FP64 CPU oracle of the kinetic-bounds limiter (arXiv 2407.20966).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is a ctypes
wrapper around ``kbl_oracle.c`` (plain C, compiled here with gcc) and shares no
code with the CUDA library.

Array conventions follow ``kbl_oracle.h``: solution ``w[nv][E][Ns]``, traces
``wf[nv][E][Nfp]``, bounds ``bnd[2][nv][E]``, stencil ``S[|S|][nv]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbl_oracle.c")
_HDR = os.path.join(_HERE, "kbl_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("nu", C.c_int * 2), ("gamma", C.c_double),
                ("k", C.c_double), ("r_fac", C.c_double), ("eps", C.c_double),
                ("rho_floor", C.c_double), ("p_floor", C.c_double), ("eps_rule", C.c_int),
                ("uncoupled", C.c_int), ("flux", C.c_int), ("quadrature", C.c_int), ("stencil", C.c_int)]


class _Mesh(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("nbr", C.POINTER(C.c_int)), ("h", C.POINTER(C.c_double)),
                ("n_bc", C.c_int), ("bc", C.POINTER(C.c_double))]


class _TriMesh(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("xy", C.POINTER(C.c_double)), ("nbr", C.POINTER(C.c_int)),
                ("nbr_edge", C.POINTER(C.c_int)), ("n_bc", C.c_int), ("bc", C.POINTER(C.c_double)),
                ("xy6", C.POINTER(C.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d = C.POINTER(C.c_double)
            cfgp = C.POINTER(_Cfg)
            meshp = C.POINTER(_Mesh)
            trip = C.POINTER(_TriMesh)
            sig = {
                "orc_legendre": (None, [C.c_int, C.c_double, d, d]),
                "orc_gauss_legendre": (C.c_int, [C.c_int, d, d]),
                "orc_lagrange": (C.c_double, [C.c_int, d, C.c_int, C.c_double]),
                "orc_lagrange_deriv": (C.c_double, [C.c_int, d, C.c_int, C.c_double]),
                "orc_correction_deriv": (None, [C.c_int, C.c_double, d, d]),
                "orc_pressure": (C.c_double, [cfgp, d]),
                "orc_flux": (None, [cfgp, d, C.c_int, d]),
                "orc_rusanov": (None, [cfgp, d, d, C.c_int, d]),
                "orc_hllc": (None, [cfgp, d, d, C.c_int, d]),
                "orc_hll": (None, [cfgp, d, d, C.c_int, d]),
                "orc_romberg_weight": (C.c_double, [C.c_int, C.c_int]),
                "orc_bounds_stencil": (C.c_int, [cfgp, C.c_int, d, d, d]),
                "orc_state_moments": (C.c_int, [cfgp, C.c_int, d, C.c_int, d]),
                "orc_velocity_box": (C.c_int, [cfgp, C.c_int, d, d, d]),
                "orc_envelope_moments": (C.c_int, [cfgp, C.c_int, d, C.c_int, d]),
                "orc_traces": (None, [cfgp, meshp, d, d]),
                "orc_gather_stencil": (None, [cfgp, meshp, d, d, C.c_int, d]),
                "orc_bounds": (C.c_int, [cfgp, meshp, d, d, d]),
                "orc_rhs": (None, [cfgp, meshp, d, d, d]),
                "orc_limit_element": (None, [cfgp, d, d, d, d, d]),
                "orc_limit_nodes": (None, [cfgp, C.c_int, C.c_int, d, d, d, d, d, d]),
                "orc_limit": (None, [cfgp, meshp, d, d, d]),
                "orc_stage_combine": (None, [cfgp, meshp, C.c_int, d, d, d, C.c_double, d]),
                "orc_dt": (C.c_double, [cfgp, meshp, d, C.c_double]),
                "orc_ssprk3_step": (C.c_int, [cfgp, meshp, d, C.c_double, d]),
                "orc_tri_points": (C.c_int, [C.c_int, d, d]),
                "orc_tri_traces": (None, [cfgp, trip, d, d]),
                "orc_tri_gather_stencil": (None, [cfgp, trip, d, d, C.c_int, d]),
                "orc_tri_rhs": (None, [cfgp, trip, d, d, d]),
                "orc_tri_dt": (C.c_double, [cfgp, trip, d, C.c_double]),
                "orc_tri_ssprk3_step": (C.c_int, [cfgp, trip, d, C.c_double, d]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Config:
    """Method parameters (defaults: Sec. 3.4, 3.5, 3.7, 3.8 and Sec. 5, 2D values)."""
    dim: int = 2
    p: int = 3
    nu: tuple = (32, 32)
    gamma: float = 1.4
    k: float = 4.0
    r_fac: float = 1e-3
    eps: float = 1e-13
    rho_floor: float = 1e-12
    p_floor: float = 1e-12
    eps_rule: int = 0
    uncoupled: int = 0
    flux: int = 0
    quadrature: int = 0
    stencil: int = 0      # 1 (1D): own solution points and both face neighbours' solution points

    @property
    def nv(self):
        return self.dim + 2

    @property
    def ns(self):
        return (self.p + 1) ** self.dim

    @property
    def nfp(self):
        return 2 if self.dim == 1 else 4 * (self.p + 1)

    @property
    def nstencil(self):
        return 3 * self.ns if self.stencil == 1 else self.ns + 2 * self.nfp

    def _c(self):
        nu = list(self.nu) + [1] * (2 - len(self.nu))
        return _Cfg(self.dim, self.p, (C.c_int * 2)(*nu[:2]), self.gamma, self.k, self.r_fac,
                    self.eps, self.rho_floor, self.p_floor, self.eps_rule, self.uncoupled, self.flux,
                    self.quadrature, self.stencil)


class Mesh:
    """Cartesian mesh: nbr[E][2d] (>= 0 element, < 0 boundary id -(nbr+1)), h[E][d]."""

    def __init__(self, nbr, h, bc=None):
        self.nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        self.n_elem = self.nbr.shape[0]
        self.bc = np.ascontiguousarray(bc if bc is not None else np.zeros((1, 4)), dtype=np.float64)

    def _c(self):
        return _Mesh(self.n_elem, self.nbr.ctypes.data_as(C.POINTER(C.c_int)), _dp(self.h),
                     self.bc.shape[0], _dp(self.bc))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc == -1:
        raise OracleError(f"{what}: non-physical state (rho <= 0 or P <= 0)")
    if rc != 0:
        raise OracleError(f"{what}: bad argument (rc={rc})")


# ---- polynomial tools -------------------------------------------------
def legendre(n, x):
    P, dP = C.c_double(), C.c_double()
    _load().orc_legendre(n, float(x), C.byref(P), C.byref(dP))
    return P.value, dP.value


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(_load().orc_gauss_legendre(n, _dp(x), _dp(w)), "gauss_legendre")
    return x, w


def lagrange(nodes, j, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    return _load().orc_lagrange(len(nodes), _dp(nodes), j, float(x))


def lagrange_deriv(nodes, j, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    return _load().orc_lagrange_deriv(len(nodes), _dp(nodes), j, float(x))


def correction_deriv(p, x):
    a, b = C.c_double(), C.c_double()
    _load().orc_correction_deriv(p, float(x), C.byref(a), C.byref(b))
    return a.value, b.value


# ---- physics ----------------------------------------------------------
def pressure(cfg: Config, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    return _load().orc_pressure(C.byref(cfg._c()), _dp(w))


def flux(cfg: Config, w, direction):
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.zeros(cfg.nv)
    _load().orc_flux(C.byref(cfg._c()), _dp(w), direction, _dp(F))
    return F


def rusanov(cfg: Config, wl, wr, direction):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    F = np.zeros(cfg.nv)
    _load().orc_rusanov(C.byref(cfg._c()), _dp(wl), _dp(wr), direction, _dp(F))
    return F


def hllc(cfg: Config, wl, wr, direction):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    F = np.zeros(cfg.nv)
    _load().orc_hllc(C.byref(cfg._c()), _dp(wl), _dp(wr), direction, _dp(F))
    return F


def romberg_weights(n):
    """Romberg weights, in units of the grid spacing, of an axis of n equispaced nodes."""
    return np.array([_load().orc_romberg_weight(n, j) for j in range(n)])


def hll(cfg: Config, wl, wr, direction):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    F = np.zeros(cfg.nv)
    _load().orc_hll(C.byref(cfg._c()), _dp(wl), _dp(wr), direction, _dp(F))
    return F


# ---- bounds -----------------------------------------------------------
def bounds_stencil(cfg: Config, S):
    S = np.ascontiguousarray(S, dtype=np.float64)
    lo, hi = np.zeros(cfg.nv), np.zeros(cfg.nv)
    _check(_load().orc_bounds_stencil(C.byref(cfg._c()), S.shape[0], _dp(S), _dp(lo), _dp(hi)),
           "bounds_stencil")
    return lo, hi


def state_moments(cfg: Config, S, which):
    S = np.ascontiguousarray(S, dtype=np.float64)
    mom = np.zeros(cfg.nv)
    _check(_load().orc_state_moments(C.byref(cfg._c()), S.shape[0], _dp(S), which, _dp(mom)),
           "state_moments")
    return mom


def envelope_moments(cfg: Config, S, upper):
    S = np.ascontiguousarray(S, dtype=np.float64)
    mom = np.zeros(cfg.nv)
    _check(_load().orc_envelope_moments(C.byref(cfg._c()), S.shape[0], _dp(S), int(upper), _dp(mom)),
           "envelope_moments")
    return mom


def velocity_box(cfg: Config, S):
    S = np.ascontiguousarray(S, dtype=np.float64)
    lo, hi = np.zeros(2), np.zeros(2)
    _check(_load().orc_velocity_box(C.byref(cfg._c()), S.shape[0], _dp(S), _dp(lo), _dp(hi)),
           "velocity_box")
    return lo[:cfg.dim], hi[:cfg.dim]


# ---- mesh level ---------------------------------------------------------
def traces(cfg: Config, mesh: Mesh, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.zeros((cfg.nv, mesh.n_elem, cfg.nfp))
    _load().orc_traces(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), _dp(wf))
    return wf


def gather_stencil(cfg: Config, mesh: Mesh, w, wf, e):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.ascontiguousarray(wf, dtype=np.float64)
    S = np.zeros((cfg.nstencil, cfg.nv))
    _load().orc_gather_stencil(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), _dp(wf), e, _dp(S))
    return S


def bounds(cfg: Config, mesh: Mesh, w, wf):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.ascontiguousarray(wf, dtype=np.float64)
    bnd = np.zeros((2, cfg.nv, mesh.n_elem))
    _check(_load().orc_bounds(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), _dp(wf), _dp(bnd)),
           "bounds")
    return bnd


def rhs(cfg: Config, mesh: Mesh, w, wf):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.ascontiguousarray(wf, dtype=np.float64)
    R = np.zeros_like(w)
    _load().orc_rhs(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), _dp(wf), _dp(R))
    return R


def limit_element(cfg: Config, wel, wfel, wmin, wmax):
    wel = np.array(wel, dtype=np.float64, order="C")
    wfel = np.ascontiguousarray(wfel, dtype=np.float64)
    wmin = np.ascontiguousarray(wmin, dtype=np.float64)
    wmax = np.ascontiguousarray(wmax, dtype=np.float64)
    a = np.zeros(2)
    _load().orc_limit_element(C.byref(cfg._c()), _dp(wel), _dp(wfel), _dp(wmin), _dp(wmax), _dp(a))
    return wel, a


def limit_nodes(cfg: Config, Wq, wel, wfel, wmin, wmax):
    """Limit one element's node set: solution values wel[nv][ns] with mean weights Wq[ns], face
    values wfel[nv][nf]; returns the limited solution values and (alpha, alpha_P)."""
    Wq = np.ascontiguousarray(Wq, dtype=np.float64)
    wel = np.array(wel, dtype=np.float64, order="C")
    wfel = np.ascontiguousarray(wfel, dtype=np.float64)
    wmin = np.ascontiguousarray(wmin, dtype=np.float64)
    wmax = np.ascontiguousarray(wmax, dtype=np.float64)
    a = np.zeros(2)
    _load().orc_limit_nodes(C.byref(cfg._c()), wel.shape[1], wfel.shape[1], _dp(Wq), _dp(wel), _dp(wfel),
                            _dp(wmin), _dp(wmax), _dp(a))
    return wel, a


def limit(cfg: Config, mesh: Mesh, w, bnd):
    w = np.array(w, dtype=np.float64, order="C")
    bnd = np.ascontiguousarray(bnd, dtype=np.float64)
    alpha = np.zeros((2, mesh.n_elem))
    _load().orc_limit(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), _dp(bnd), _dp(alpha))
    return w, alpha


def stage_combine(cfg: Config, mesh: Mesh, s, wn, ws, R, dt):
    wn, ws, R = (np.ascontiguousarray(a, dtype=np.float64) for a in (wn, ws, R))
    wo = np.zeros_like(wn)
    _load().orc_stage_combine(C.byref(cfg._c()), C.byref(mesh._c()), s, _dp(wn), _dp(ws), _dp(R),
                              float(dt), _dp(wo))
    return wo


def dt(cfg: Config, mesh: Mesh, w, cfl):
    w = np.ascontiguousarray(w, dtype=np.float64)
    return _load().orc_dt(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), float(cfl))


def ssprk3_step(cfg: Config, mesh: Mesh, w, dt_):
    w = np.array(w, dtype=np.float64, order="C")
    alpha = np.zeros((2, mesh.n_elem))
    _check(_load().orc_ssprk3_step(C.byref(cfg._c()), C.byref(mesh._c()), _dp(w), float(dt_),
                                   _dp(alpha)), "ssprk3_step")
    return w, alpha


# ---- triangles (Sec. 5) ----------------------------------------------------
class TriMesh:
    """Affine triangles: xy[E][3][2] (counterclockwise), nbr[E][3] (element across edge f from vertex f
    to vertex f+1, < 0 boundary id -(nbr+1)), nbr_edge[E][3] (the neighbour's matched edge), bc."""

    def __init__(self, xy, nbr, nbr_edge, bc=None, xy6=None):
        """xy6: [E][6][2] curved (quadratic) elements, the corners then the mid-parameter points
        of edges 0, 1, 2 (xy then holds the corners); None for affine elements."""
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        self.nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        self.nbr_edge = np.ascontiguousarray(nbr_edge, dtype=np.int32)
        self.n_elem = self.nbr.shape[0]
        self.bc = np.ascontiguousarray(bc if bc is not None else np.zeros((1, 4)), dtype=np.float64)
        self.xy6 = None if xy6 is None else np.ascontiguousarray(xy6, dtype=np.float64)

    def _c(self):
        return _TriMesh(self.n_elem, _dp(self.xy), self.nbr.ctypes.data_as(C.POINTER(C.c_int)),
                        self.nbr_edge.ctypes.data_as(C.POINTER(C.c_int)), self.bc.shape[0], _dp(self.bc),
                        None if self.xy6 is None else _dp(self.xy6))


def tri_ns(p):
    return (p + 1) * (p + 2) // 2


def tri_points(p):
    """Williams-Shunn solution points rs[ns][2] and weights w[ns] on (0,0), (1,0), (0,1)."""
    ns = tri_ns(p)
    rs, w = np.zeros((ns, 2)), np.zeros(ns)
    _check(_load().orc_tri_points(int(p), _dp(rs), _dp(w)), "tri_points")
    return rs, w


def tri_traces(cfg: Config, m: TriMesh, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.zeros((m.n_elem, 3 * (cfg.p + 1), 4))
    _load().orc_tri_traces(C.byref(cfg._c()), C.byref(m._c()), _dp(w), _dp(wf))
    return wf


def tri_gather_stencil(cfg: Config, m: TriMesh, w, wf, e):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.ascontiguousarray(wf, dtype=np.float64)
    S = np.zeros((tri_ns(cfg.p) + 6 * (cfg.p + 1), 4))
    _load().orc_tri_gather_stencil(C.byref(cfg._c()), C.byref(m._c()), _dp(w), _dp(wf), int(e), _dp(S))
    return S


def tri_rhs(cfg: Config, m: TriMesh, w, wf):
    w = np.ascontiguousarray(w, dtype=np.float64)
    wf = np.ascontiguousarray(wf, dtype=np.float64)
    R = np.zeros_like(w)
    _load().orc_tri_rhs(C.byref(cfg._c()), C.byref(m._c()), _dp(w), _dp(wf), _dp(R))
    return R


def tri_dt(cfg: Config, m: TriMesh, w, cfl):
    w = np.ascontiguousarray(w, dtype=np.float64)
    return _load().orc_tri_dt(C.byref(cfg._c()), C.byref(m._c()), _dp(w), float(cfl))


def tri_ssprk3_step(cfg: Config, m: TriMesh, w, dt_):
    w = np.array(w, dtype=np.float64, order="C")
    alpha = np.zeros((2, m.n_elem))
    _check(_load().orc_tri_ssprk3_step(C.byref(cfg._c()), C.byref(m._c()), _dp(w), float(dt_), _dp(alpha)),
           "tri_ssprk3_step")
    return w, alpha
