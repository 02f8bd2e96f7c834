"""The FR residual as one matrix per order (kbl_residual_operator, the operator the tensor-core
residual multiplies by), checked on the CPU against the checker's own FR residual (Sec. 2.3 with
the g_DG correction of Sec. 5; an independent construction: Newton Gauss-Legendre nodes,
Lagrange derivatives, the interpolated discontinuous flux subtracted at the faces).

For every element, X = [(2/h_x) Fx at the solution points, (2/h_y) Fy, (2/h_x) F* at the x-face
points, (2/h_y) F* at the y-face points] with the checker's Rusanov common flux; X B must equal
the checker's residual to 1e-12 of the size of its terms.  A dropped lifting term, a transposed
derivative block or a sign slip fails it (the last part of the test plants each)."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import exterior_traces, rhs_error


def _euler_flux(q, d, gamma):
    rho, E = q[0], q[3]
    P = (gamma - 1.0) * (E - 0.5 * (q[1] ** 2 + q[2] ** 2) / rho)
    u = q[1 + d] / rho
    return np.stack([q[1 + d], q[1] * u + (P if d == 0 else 0.0), q[2] * u + (P if d == 1 else 0.0), (E + P) * u])


def _X(orc, cfg, mesh, w, wf):
    N = cfg.p + 1
    NS, NFP = N * N, 4 * N
    E = mesh.n_elem
    wx = exterior_traces(wf, mesh)
    sx = 2.0 / mesh.h[:, 0]
    sy = 2.0 / mesh.h[:, 1]
    X = np.zeros((4, E, 2 * NS + NFP))
    X[:, :, :NS] = _euler_flux(w, 0, cfg.gamma) * sx[None, :, None]
    X[:, :, NS:2 * NS] = _euler_flux(w, 1, cfg.gamma) * sy[None, :, None]
    for e in range(E):
        for fp in range(NFP):
            f = fp // N
            d, side = f >> 1, f & 1
            qi, qe = wf[:, e, fp], wx[:, e, fp]
            Fc = orc.rusanov(cfg, qe, qi, d) if side == 0 else orc.rusanov(cfg, qi, qe, d)
            X[:, e, 2 * NS + fp] = Fc * (sy[e] if d else sx[e])
    return X


@pytest.mark.parametrize("p,n", [(1, (4, 3)), (2, (5, 4)), (3, (4, 4)), (4, (3, 3)), (5, (2, 3))])
def test_residual_operator_reproduces_the_checkers_fr_residual(orc, p, n):
    from paper_2407_20966_gb300 import kbl
    from tests.gpu_helpers import mesh_and_field
    cfg = orc.Config(dim=2, p=p, nu=(16, 16))
    mesh, w = mesh_and_field(orc, 2, p, n, seed=400 + p, kind="disc")
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    wf = orc.traces(cfg, om, w)
    R_ref = orc.rhs(cfg, om, w, wf)
    B = kbl.residual_operator(p)
    X = _X(orc, cfg, mesh, w, wf)
    R = np.einsum("vek,kn->ven", X, B)
    err = rhs_error(R, R_ref, w, wf, mesh)
    assert err.max() < 1e-12, err.max()
    # planted mistakes: each must fail the same comparison
    N = p + 1
    NS = N * N
    bad = []
    B1 = B.copy(); B1[2 * NS:2 * NS + N] = 0.0                 # the -x lifting dropped
    bad.append(B1)
    B2 = B.copy(); B2[:NS], B2[NS:2 * NS] = B[NS:2 * NS].copy(), B[:NS].copy()   # x and y blocks swapped
    bad.append(B2)
    bad.append(-B)                                              # sign
    for Bb in bad:
        Rb = np.einsum("vek,kn->ven", X, Bb)
        assert rhs_error(Rb, R_ref, w, wf, mesh).max() > 1e-6


def test_residual_operator_rejects_bad_arguments():
    from paper_2407_20966_gb300 import kbl
    with pytest.raises(kbl.KblError):
        kbl.residual_operator(0)
    with pytest.raises(kbl.KblError):
        kbl.residual_operator(6)
