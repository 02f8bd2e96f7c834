"""The shock-vortex set-up (the adjoint workload): the two boundary states satisfy the
Rankine-Hugoniot conditions of a stationary normal shock at Mach 1.1, and the vortex is
isentropic with the upstream entropy."""
import math

import numpy as np

from paper_2407_20966_gb300 import inputs


def _prim(q, gamma=1.4):
    rho = q[0]
    u = q[1] / rho
    P = (gamma - 1) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / rho)
    return rho, u, P


def test_rankine_hugoniot_fluxes_match():
    mesh, ic = inputs.shock_vortex(8)
    (r1, u1, p1), (r2, u2, p2) = _prim(mesh.bc[0]), _prim(mesh.bc[1])
    assert abs(u1 / math.sqrt(1.4 * p1 / r1) - 1.1) < 1e-14
    # mass, momentum and energy fluxes across a stationary shock
    assert abs(r1 * u1 - r2 * u2) < 1e-14
    assert abs((r1 * u1 * u1 + p1) - (r2 * u2 * u2 + p2)) < 1e-13
    E1, E2 = mesh.bc[0][3], mesh.bc[1][3]
    assert abs((E1 + p1) * u1 - (E2 + p2) * u2) < 1e-13
    # compressive: subsonic downstream, entropy increases
    assert u2 / math.sqrt(1.4 * p2 / r2) < 1.0
    assert p2 / r2 ** 1.4 > p1 / r1 ** 1.4


def test_vortex_is_isentropic_and_mesh_layout():
    mesh, ic = inputs.shock_vortex(16)
    xi = np.array([-0.5, 0.5])
    w = inputs.nodal_field(mesh, xi, ic)
    x, y = inputs.node_coords(mesh, xi)
    up = x < 0.5
    rho, u, P = _prim(w)
    np.testing.assert_allclose((P / rho ** 1.4)[up], 1.0, rtol=1e-13)
    assert np.all(w[:, ~up] == mesh.bc[1][:, None])
    # the vortex is present: velocity deviates from the mean flow near its centre
    near = up & ((x - 0.25) ** 2 + (y - 0.5) ** 2 < 0.1 ** 2)
    assert near.any() and np.abs(w[2][near]).max() > 1e-2
    # domain [0, 2] x [0, 1]; x faces are Dirichlet (ids 0 upstream, 1 downstream), y is periodic
    assert np.allclose(mesh.h[0], [2 / 16, 1 / 16])
    assert (mesh.nbr[::16, 0] == -1).all() and (mesh.nbr[15::16, 1] == -2).all()
    assert (mesh.nbr >= 0)[:, 2:].all()
