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
