"""Pins of the checker's triangle path (Sec. 5: Williams-Shunn solution points, Gauss-Legendre flux
points, FR with the DG correction on affine triangles), against what mathematics fixes:
* the solution-point rules integrate every monomial up to degree 2p exactly and fail at 2p + 1
  (the 6-point rule of P2 is the degree-4 rule of two symmetric orbits), with interior points
  and positive weights summing to the area;
* free stream: a constant state has zero residual on a jittered mesh;
* discrete conservation: the weighted residual sums to zero on a periodic mesh (every flux);
* exactness: where the physical flux is a polynomial of degree <= p (linear density for P1,
  quadratic for P2, constant velocity and pressure) the residual is the exact -div F at every
  solution point of an element whose neighbours share the polynomial;
* a limited step keeps the element means' totals (mass, energy) and positivity, and every
  value of V lies inside the element's kinetic bounds.
"""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs

G = 1.4


def _monos(deg):
    return [(i, d - i) for d in range(deg + 1) for i in range(d + 1)]


def _exact(i, j):
    from math import factorial
    return factorial(i) * factorial(j) / factorial(i + j + 2)


@pytest.mark.parametrize("p", [1, 2])
def test_williams_shunn_rules(orc, p):
    rs, w = orc.tri_points(p)
    assert np.all(w > 0) and abs(w.sum() - 0.5) < 1e-15
    lam = np.stack([1 - rs[:, 0] - rs[:, 1], rs[:, 0], rs[:, 1]])
    assert lam.min() > 0.05   # interior
    for i, j in _monos(2 * p):
        q = (w * rs[:, 0] ** i * rs[:, 1] ** j).sum()
        assert abs(q - _exact(i, j)) < 1e-15, (i, j)
    worst = max(abs((w * rs[:, 0] ** i * rs[:, 1] ** j).sum() - _exact(i, j)) for i, j in _monos(2 * p + 1))
    assert worst > 1e-6   # not exact one degree higher


def _cfg(orc, p, flux=0):
    return orc.Config(dim=2, p=p, nu=(16, 16), flux=flux)


def _state(x, y, rho, u=0.3, v=-0.2, P=1.0):
    rho = rho(x, y) + 0 * x
    E = P / (G - 1) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E + 0 * x])


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_free_stream_and_conservation(orc, p, flux):
    m = inputs.tri_mesh_2d(6, 5, 0.0, 1.0, 0.0, 0.8, jitter=0.25, seed=3)
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    cfg = _cfg(orc, p, flux)
    rs, wq = orc.tri_points(p)
    w = inputs.tri_nodal_field(m, rs, lambda x, y: _state(x, y, lambda a, b: 1.3))
    R = orc.tri_rhs(cfg, om, w, orc.tri_traces(cfg, om, w))
    assert np.abs(R).max() < 1e-12
    # a discontinuous periodic field: the weighted residual sums to zero
    rng = np.random.default_rng(p)
    w = w * (1 + 0.2 * rng.uniform(-1, 1, w.shape))
    R = orc.tri_rhs(cfg, om, w, orc.tri_traces(cfg, om, w))
    X0 = m.xy[:, 0]
    det = ((m.xy[:, 1, 0] - X0[:, 0]) * (m.xy[:, 2, 1] - X0[:, 1]) - (m.xy[:, 2, 0] - X0[:, 0]) * (m.xy[:, 1, 1] - X0[:, 1]))
    total = np.einsum("e,i,eiv->v", det, wq, R)
    scale = np.einsum("e,i,eiv->v", det, wq, np.abs(R))
    assert np.all(np.abs(total) < 1e-13 * scale), total / scale


@pytest.mark.parametrize("p,deg", [(1, 1), (2, 2)])
def test_residual_exact_for_polynomial_fluxes(orc, p, deg):
    m = inputs.tri_mesh_2d(5, 5, 0.0, 1.0, 0.0, 1.0, jitter=0.2, seed=7, periodic=(False, False))
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    cfg = _cfg(orc, p)
    rs, _ = orc.tri_points(p)
    u, v = 0.3, -0.2
    if deg == 1:
        rho, drx, dry = (lambda x, y: 1.0 + 0.4 * x - 0.3 * y), (lambda x, y: 0.4 + 0 * x), (lambda x, y: -0.3 + 0 * x)
    else:
        rho = lambda x, y: 1.0 + 0.4 * x - 0.3 * y + 0.5 * x * x - 0.2 * x * y + 0.3 * y * y
        drx = lambda x, y: 0.4 + x - 0.2 * y
        dry = lambda x, y: -0.3 - 0.2 * x + 0.6 * y
    w = inputs.tri_nodal_field(m, rs, lambda x, y: _state(x, y, rho, u, v))
    R = orc.tri_rhs(cfg, om, w, orc.tri_traces(cfg, om, w))
    X0 = m.xy[:, 0, :]
    x = X0[:, None, 0] + rs[None, :, 0] * (m.xy[:, 1, 0] - X0[:, 0])[:, None] + rs[None, :, 1] * (m.xy[:, 2, 0] - X0[:, 0])[:, None]
    y = X0[:, None, 1] + rs[None, :, 0] * (m.xy[:, 1, 1] - X0[:, 1])[:, None] + rs[None, :, 1] * (m.xy[:, 2, 1] - X0[:, 1])[:, None]
    adv = u * drx(x, y) + v * dry(x, y)          # u . grad rho
    exact = -np.stack([adv, u * adv, v * adv, 0.5 * (u * u + v * v) * adv], axis=-1)
    interior = np.all(m.nbr >= 0, axis=1) & np.all(m.nbr[m.nbr] >= 0, axis=(1, 2))
    err = np.abs(R - exact)[interior].max() / np.abs(exact).max()
    assert err < 1e-12, err
    # a wrong lifting sign or a wrong normal would break it: the residual without the face term
    # (-div F_h alone) differs where the fluxes jump, but agrees here; check that the face term is
    # active on a discontinuous field instead (its sum over an element is the net edge flux)
    wj = w.copy()
    wj[::2] *= 1.1
    Rj = orc.tri_rhs(cfg, om, wj, orc.tri_traces(cfg, om, wj))
    assert np.abs(Rj - R).max() > 1e-3


@pytest.mark.parametrize("p", [1, 2])
def test_limited_step_keeps_means_positivity_and_bounds(orc, p):
    m = inputs.tri_mesh_2d(8, 7, 0.0, 1.0, 0.0, 1.0, jitter=0.2, seed=11)
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    cfg = _cfg(orc, p, flux=1)
    rs, wq = orc.tri_points(p)

    def ic(x, y):   # a circular blast with a tanh front about a cell wide
        s = 0.5 * (1 - np.tanh((np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2) - 0.25) / 0.06))
        rho = 0.125 + 0.875 * s
        P = 0.1 + 0.9 * s
        return np.stack([rho, 0 * x, 0 * x, P / (G - 1)])
    w = inputs.tri_nodal_field(m, rs, ic)
    X0 = m.xy[:, 0]
    det = ((m.xy[:, 1, 0] - X0[:, 0]) * (m.xy[:, 2, 1] - X0[:, 1]) - (m.xy[:, 2, 0] - X0[:, 0]) * (m.xy[:, 1, 1] - X0[:, 1]))
    tot0 = np.einsum("e,i,eiv->v", det, wq, w)
    dt = orc.tri_dt(cfg, om, w, 0.1)
    w1, alpha = orc.tri_ssprk3_step(cfg, om, w, dt)
    assert (alpha[0] < 1).any()
    # after limiting, every value of V lies inside the element's bounds (Cor. 4.5.1): perturb the
    # state by a field of zero weighted mean per element (the mean, a convex combination of the
    # element's own stencil states, stays inside the bounds) and limit it against the bounds of
    # the unperturbed stencil
    wf = orc.tri_traces(cfg, om, w)
    ns = len(wq)
    d = np.sin(3.0 * np.arange(ns))
    d = d - (wq * d).sum() / wq.sum()
    amp = np.abs(w).max(axis=1, keepdims=True)                   # [E][1][4]
    wp = np.ascontiguousarray(w + 0.3 * amp * d[None, :, None])
    wfp = orc.tri_traces(cfg, om, wp)
    limited = 0
    for e in range(m.n_elem):
        lo, hi = orc.bounds_stencil(cfg, orc.tri_gather_stencil(cfg, om, w, wf, e))
        lim, a = orc.limit_nodes(cfg, wq, np.ascontiguousarray(wp[e].T), np.ascontiguousarray(wfp[e].T), lo, hi)
        limited += a[0] < 1
        tol = 1e-12 * np.maximum(np.abs(lo), np.abs(hi))
        assert np.all(lim.min(axis=1) >= lo - tol) and np.all(lim.max(axis=1) <= hi + tol), e
    assert limited > 0


# ---- curved (quadratic) elements --------------------------------------------------------------
def _jacobians(xy6, rs):
    """|J| of the quadratic map at reference points rs[n][2] of every element: [E][n]."""
    r, s = rs[None, :, 0], rs[None, :, 1]
    l1, l2, l3 = 1 - r - s, r, s
    dr = [-(4 * l1 - 1), 4 * l2 - 1, 0 * r, 4 * (l1 - l2), 4 * l3, -4 * l3]
    ds = [-(4 * l1 - 1), 0 * r, 4 * l3 - 1, -4 * l2, 4 * l2, 4 * (l1 - l3)]
    xr = sum(dr[k] * xy6[:, k, 0][:, None] for k in range(6))
    xs = sum(ds[k] * xy6[:, k, 0][:, None] for k in range(6))
    yr = sum(dr[k] * xy6[:, k, 1][:, None] for k in range(6))
    ys = sum(ds[k] * xy6[:, k, 1][:, None] for k in range(6))
    return xr * ys - xs * yr


@pytest.mark.parametrize("p", [1, 2])
def test_curved_with_straight_edges_is_the_affine_scheme(orc, p):
    """Mid-parameter points on the straight edges make the quadratic map affine: the curved
    residual and limited step equal the affine ones to rounding."""
    m = inputs.tri_mesh_2d(6, 5, 0.0, 1.0, 0.0, 0.8, jitter=0.25, seed=3, periodic=(False, False))
    xy6 = np.concatenate([m.xy, 0.5 * (m.xy + np.roll(m.xy, -1, axis=1))], axis=1)
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    oc = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc, xy6=xy6)
    cfg = _cfg(orc, p, flux=1)
    rs, _ = orc.tri_points(p)
    rng = np.random.default_rng(p)
    w = inputs.tri_nodal_field(m, rs, lambda x, y: _state(x, y, lambda a, b: 1.0 + 0.3 * a - 0.2 * b))
    w = np.ascontiguousarray(w * (1 + 0.1 * rng.uniform(-1, 1, w.shape)))
    wf = orc.tri_traces(cfg, om, w)
    Ra, Rc = orc.tri_rhs(cfg, om, w, wf), orc.tri_rhs(cfg, oc, w, wf)
    assert np.abs(Ra - Rc).max() < 1e-11 * np.abs(Ra).max()
    dt = orc.tri_dt(cfg, om, w, 0.1)
    wa, _ = orc.tri_ssprk3_step(cfg, om, w, dt)
    wc, _ = orc.tri_ssprk3_step(cfg, oc, w, dt)
    assert np.abs(wa - wc).max() < 1e-12 * np.abs(wa).max()


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_curved_free_stream_and_conservation(orc, p, flux):
    """On a periodic mesh of curved elements: a constant state has zero residual (the discrete
    metric identity of the transformed-flux form), and the residual of a discontinuous field
    weighted by the lumped mass w_i |J_i| sums to zero (the surface terms of the two sides of an
    edge cancel)."""
    m = inputs.tri_curved_mesh(6, 5, 0.0, 1.0, 0.0, 0.8, jitter=0.2, bump=0.15, seed=3)
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc, xy6=m.xy6)
    cfg = _cfg(orc, p, flux)
    rs, wq = orc.tri_points(p)
    J = _jacobians(m.xy6, rs)
    assert J.min() > 0
    w = inputs.tri_nodal_field(m, rs, lambda x, y: _state(x, y, lambda a, b: 1.3))
    R0 = orc.tri_rhs(cfg, om, w, orc.tri_traces(cfg, om, w))
    rng = np.random.default_rng(p)
    w = np.ascontiguousarray(w * (1 + 0.2 * rng.uniform(-1, 1, w.shape)))
    R = orc.tri_rhs(cfg, om, w, orc.tri_traces(cfg, om, w))
    # free stream to rounding of the terms the residual sums (their size: a discontinuous field's)
    assert np.abs(R0).max() < 1e-13 * np.abs(R).max(), np.abs(R0).max() / np.abs(R).max()
    total = np.einsum("en,n,env->v", J, wq, R)
    scale = np.einsum("en,n,env->v", J, wq, np.abs(R))
    assert np.all(np.abs(total) < 1e-13 * scale), total / scale
    # the curvature matters: the affine scheme on the corners gives a different residual
    oa = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    Ra = orc.tri_rhs(cfg, oa, w, orc.tri_traces(cfg, oa, w))
    assert np.abs(Ra - R).max() > 1e-3 * np.abs(R).max()


@pytest.mark.parametrize("p", [1, 2])
def test_curved_limited_step_keeps_totals_and_positivity(orc, p):
    m = inputs.tri_curved_mesh(8, 7, 0.0, 1.0, 0.0, 1.0, jitter=0.2, bump=0.15, seed=11)
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc, xy6=m.xy6)
    cfg = _cfg(orc, p, flux=1)
    rs, wq = orc.tri_points(p)
    J = _jacobians(m.xy6, rs)

    def ic(x, y):
        s = 0.5 * (1 - np.tanh((np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2) - 0.25) / 0.06))
        return np.stack([0.125 + 0.875 * s, 0 * x, 0 * x, (0.1 + 0.9 * s) / (G - 1)])
    w = inputs.tri_nodal_field(m, rs, ic)
    tot0 = np.einsum("en,n,env->v", J, wq, w)
    dt = orc.tri_dt(cfg, om, w, 0.1)
    w1, alpha = orc.tri_ssprk3_step(cfg, om, w, dt)
    assert (alpha[0] < 1).any()
    tot1 = np.einsum("en,n,env->v", J, wq, w1)
    assert abs(tot1[0] - tot0[0]) < 1e-13 * abs(tot0[0]) and abs(tot1[3] - tot0[3]) < 1e-13 * abs(tot0[3])
    P = (G - 1) * (w1[..., 3] - 0.5 * (w1[..., 1] ** 2 + w1[..., 2] ** 2) / w1[..., 0])
    assert w1[..., 0].min() > 0 and P.min() > 0
