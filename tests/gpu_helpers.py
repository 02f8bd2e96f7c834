"""Shared set-up for the GPU tests: one method configuration on both sides (the CUDA
library through the C-ABI, the CPU checker), seeded inputs, and the error measures."""
import numpy as np

from paper_2407_20966_gb300 import inputs

TOL_FP64 = 1e-12   # relative, bounds and limited states (FP64 path)
TOL_FP32 = 1e-5    # relative, bounds and limited states (FP32 path)


def both(orc, dim, p, nu, precision=0, **kw):
    from paper_2407_20966_gb300 import kbl
    ctx = kbl.Context(dim=dim, p=p, nu=nu, precision=precision, **kw)
    ocfg = orc.Config(dim=dim, p=p, nu=tuple(nu), **kw)
    return ctx, ocfg


def upload(ctx, orc, mesh):
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    return orc.Mesh(mesh.nbr, mesh.h, mesh.bc)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def zeros_dev(*shape):
    import torch
    return torch.zeros(shape, dtype=torch.float64, device="cuda")


def bounds_error(got, ref):
    """Scale-aware relative error of bounds [2][nv][E]: |x - x_ref| / max(|x_ref|, s) where s is
    the size of the sum behind the bound: rho_max for density, E_max for energy and
    sqrt(2 rho_max E_max) (a bound of sum M f_max |u|) for momentum."""
    nv = ref.shape[1]
    rho_hi, e_hi = ref[1, 0], ref[1, nv - 1]
    s = np.empty(ref.shape[1:])
    s[0] = rho_hi
    s[nv - 1] = e_hi
    for k in range(1, nv - 1):
        s[k] = np.sqrt(2 * rho_hi * e_hi)
    den = np.maximum(np.abs(ref), s[None])
    return np.abs(got - ref) / den


def state_error(got, ref):
    """Relative error of states [nv][E][Ns]: per component against the largest magnitude of that
    component in the element (and the element's energy scale for momentum)."""
    nv = ref.shape[0]
    sc = np.abs(ref).max(axis=2, keepdims=True)
    emax = np.abs(ref[nv - 1]).max(axis=1)[:, None]
    rmax = np.abs(ref[0]).max(axis=1)[:, None]
    for k in range(1, nv - 1):
        sc[k] = np.maximum(sc[k], np.sqrt(2 * rmax * emax))
    return np.abs(got - ref) / sc


def mesh_and_field(orc, dim, p, n, seed, kind="disc", periodic=False):
    rng = np.random.default_rng(seed)
    if dim == 1:
        mesh = inputs.mesh_1d(n, 0.0, 1.0, periodic=periodic, bc_left=0, bc_right=1)
        mesh.bc = inputs.random_states(rng, 2, 1)
    else:
        nx, ny = n if isinstance(n, tuple) else (n, n)
        mesh = inputs.mesh_2d(nx, ny, 0.0, 1.0, 0.0, 1.3, periodic=(periodic, periodic),
                              bc_of_face=lambda ix, iy, f: f % 2)
        mesh.bc = inputs.random_states(rng, 2, 2)
    xi, _ = orc.gauss_legendre(p + 1)
    gen = inputs.random_discontinuous_field if kind == "disc" else inputs.random_smooth_field
    w = gen(rng, mesh, xi)
    return mesh, w


def euler_flux_abs_max(q, gamma):
    """max over directions of |F_dir(q)| per component, for states q[nv][...] (Eq. 2)."""
    nv = q.shape[0]
    d = nv - 2
    rho, E = q[0], q[nv - 1]
    mm = sum(q[1 + k] ** 2 for k in range(d))
    P = (gamma - 1.0) * (E - 0.5 * mm / rho)
    out = np.zeros_like(q)
    for k in range(d):
        u = q[1 + k] / rho
        F = [q[1 + k]] + [q[1 + j] * u + (P if j == k else 0.0) for j in range(d)] + [(E + P) * u]
        for v in range(nv):
            out[v] = np.maximum(out[v], np.abs(F[v]))
    return out


def exterior_traces(wf, mesh):
    """Exterior value at every face point, wf_ext[nv][E][Nfp]: the neighbour's trace at the same
    point (face f^1), or the boundary state (the layout of include/kbl.h)."""
    nv, E, nfp = wf.shape
    nbr = np.asarray(mesh.nbr).reshape(E, -1)
    nf = nbr.shape[1]
    per = nfp // nf
    out = np.empty_like(wf)
    bc = np.asarray(mesh.bc, dtype=np.float64).reshape(-1, nv)
    for f in range(nf):
        nb = nbr[:, f]
        inner = nb >= 0
        for k in range(per):
            fp = f * per + k
            out[:, inner, fp] = wf[:, nb[inner], (f ^ 1) * per + k]
            if (~inner).any():
                out[:, ~inner, fp] = bc[-nb[~inner] - 1].T
    return out


def rhs_error(got, ref, w, wf, mesh, gamma=1.4):
    """Relative error of residuals R[nv][E][Ns], per element and component: |R - R_ref| divided by
    max(|R_ref|, s), s = (2 / h_min) (max |F_v| + lam max |q_v|) over the element's solution
    points, own face points and exterior face values, lam = the largest |u| + c there: the size
    of the terms the FR residual sums (D F, the lifted jumps of the common flux, whose Rusanov,
    HLL or HLLC dissipation is at most lam |q_R - q_L|; Sec. 2.3), so that a residual that is
    legitimately ~0 in a quiet region is still held to the precision of its terms."""
    nv = w.shape[0]
    wx = exterior_traces(wf, mesh)
    pts = np.concatenate([w, wf, wx], axis=2)          # [nv][E][points]
    F = euler_flux_abs_max(pts, gamma).max(axis=2)     # [nv][E]
    rho, E_ = pts[0], pts[nv - 1]
    mm = sum(pts[1 + k] ** 2 for k in range(nv - 2))
    with np.errstate(invalid="ignore", divide="ignore"):
        P = (gamma - 1.0) * (E_ - 0.5 * mm / rho)
        c = np.sqrt(np.maximum(gamma * P / rho, 0.0))
        speed = np.sqrt(mm) / np.abs(rho)
    lam = np.nan_to_num(speed + c, nan=0.0).max(axis=1)  # [E]
    Q = np.abs(pts).max(axis=2)                          # [nv][E]
    hmin = np.asarray(mesh.h).reshape(ref.shape[1], -1).min(axis=1)
    s = (2.0 / hmin)[None, :] * (F + lam[None, :] * Q)
    den = np.maximum(np.abs(ref), s[:, :, None])
    return np.abs(got - ref) / den


def step_sensitivity(orc, cfg, om, w, dt, ref, pert=1e-6, draws=3):
    """Per element, the largest change (state_error) of the checker's own SSP-RK3 step when, at
    every stage, its bounds and its residual are multiplied by (1 + pert U[-1, 1]) (a few seeded
    draws).  The FP32-mixed path differs from the checker by at most ~4e-7 in each stage's bounds
    and ~3e-6 of the term scale in each residual (the per-stage parity tests), so to first order
    its step differs by at most this sensitivity at pert = 1e-6; the full-step criterion
    max(1e-5, 10 x sensitivity) keeps a factor 10 for the draws and the nonlinearity.  Where the
    limiter is well conditioned the sensitivity is ~1e-7 and the criterion is the plain 1e-5;
    it grows where Eq. 37 or Eq. 47-49 amplify (an element driven towards vacuum, where
    P = (gamma-1)(E - |m|^2/2rho) cancels)."""
    out = np.zeros(w.shape[1])
    for d in range(draws):
        rng = np.random.default_rng(1000 + d)
        ws = w
        for s in range(3):
            wf = orc.traces(cfg, om, ws)
            bnd = orc.bounds(cfg, om, ws, wf)
            bnd = bnd * (1 + pert * rng.uniform(-1, 1, bnd.shape))
            R = orc.rhs(cfg, om, ws, wf)
            R = R * (1 + pert * rng.uniform(-1, 1, R.shape))
            comb = orc.stage_combine(cfg, om, s, w, ws, R, dt)
            ws, _ = orc.limit(cfg, om, comb, bnd)
        out = np.maximum(out, state_error(ws, ref).max(axis=(0, 2)))
    return out
