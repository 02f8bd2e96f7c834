"""Pins of the oracle's polynomial tools, physics and time stepper (CPU only).

Each check compares the oracle with something other than itself: a library
routine, a closed form or a textbook identity.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_numpy(orc, n):
    x, w = orc.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 6))
def test_lagrange_interpolation_and_derivative_exact_on_polynomials(orc, p):
    x, _ = orc.gauss_legendre(p + 1)
    rng = np.random.default_rng(p)
    coef = rng.normal(size=p + 1)
    f = np.polynomial.Polynomial(coef)
    df = f.deriv()
    for t in np.concatenate([[-1.0, 1.0], rng.uniform(-1, 1, 5)]):
        val = sum(orc.lagrange(x, j, t) * f(x[j]) for j in range(p + 1))
        der = sum(orc.lagrange_deriv(x, j, t) * f(x[j]) for j in range(p + 1))
        assert abs(val - f(t)) < 1e-12
        assert abs(der - df(t)) < 1e-11


@pytest.mark.parametrize("p", range(1, 6))
def test_correction_functions_match_numpy_legendre(orc, p):
    """g_L = R_R,p+1 = (-1)^(p+1)/2 (P_{p+1} - P_p), g_R = (P_{p+1} + P_p)/2: endpoint values
    and derivatives, built here from numpy's Legendre series."""
    L = np.polynomial.legendre.Legendre
    gl = ((-1) ** (p + 1)) * 0.5 * (L.basis(p + 1) - L.basis(p))
    gr = 0.5 * (L.basis(p + 1) + L.basis(p))
    assert gl(-1) == pytest.approx(1) and abs(gl(1)) < 1e-14
    assert gr(1) == pytest.approx(1) and abs(gr(-1)) < 1e-14
    for t in np.linspace(-1, 1, 7):
        a, b = orc.correction_deriv(p, t)
        assert a == pytest.approx(gl.deriv()(t), abs=1e-12)
        assert b == pytest.approx(gr.deriv()(t), abs=1e-12)


@pytest.mark.parametrize("p", range(1, 6))
def test_dg_correction_equals_nodal_dg_lifting(orc, p):
    """With Gauss-Legendre solution points, FR with g_DG is nodal DG: the lifting of a
    face jump to node i is l_i(-1)/w_i (diagonal mass matrix), i.e. g_L'(x_i) = -l_i(-1)/w_i
    and g_R'(x_i) = l_i(1)/w_i."""
    x, w = orc.gauss_legendre(p + 1)
    for i in range(p + 1):
        a, b = orc.correction_deriv(p, x[i])
        assert a == pytest.approx(-orc.lagrange(x, i, -1.0) / w[i], rel=1e-12, abs=1e-12)
        assert b == pytest.approx(orc.lagrange(x, i, 1.0) / w[i], rel=1e-12, abs=1e-12)


def test_pressure_flux_and_rusanov_properties(orc):
    cfg = orc.Config(dim=2)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho, u, v, P = rng.uniform(0.2, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 2)
        w = np.array([rho, rho * u, rho * v, P / 0.4 + 0.5 * rho * (u * u + v * v)])
        assert orc.pressure(cfg, w) == pytest.approx(P, rel=1e-13)
        Fx = orc.flux(cfg, w, 0)
        np.testing.assert_allclose(Fx, [rho * u, rho * u * u + P, rho * u * v, (w[3] + P) * u], rtol=1e-13)
        Fy = orc.flux(cfg, w, 1)
        np.testing.assert_allclose(Fy, [rho * v, rho * u * v, rho * v * v + P, (w[3] + P) * v], rtol=1e-13)
        # consistency: the common flux of two equal states is the physical flux
        np.testing.assert_allclose(orc.rusanov(cfg, w, w, 0), Fx, rtol=1e-13, atol=1e-14)
        # mirror symmetry: reflecting x swaps sides and flips the normal component
        w2 = w * np.array([1.3, 0.7, 1.1, 1.5])
        mir = np.array([1, -1, 1, 1.0])
        F = orc.rusanov(cfg, w, w2, 0)
        Fm = orc.rusanov(cfg, w2 * mir, w * mir, 0)
        np.testing.assert_allclose(F, -(Fm * mir), rtol=1e-12, atol=1e-13)


def test_ssprk3_stage_combination_is_third_order_taylor(orc):
    """For R(w) = lam w the three stages must give (1 + z + z^2/2 + z^3/6) w, z = lam dt,
    the stability polynomial of every three-stage third-order Runge-Kutta method."""
    cfg = orc.Config(dim=1, p=1)
    mesh = orc.Mesh(np.array([[0, 0]]), np.array([[1.0]]))
    shape = (cfg.nv, 1, cfg.ns)
    w0 = np.random.default_rng(0).uniform(0.5, 1.5, shape)
    for lam, dt in ((-1.3, 0.1), (0.7, 0.05), (-4.0, 0.2)):
        ws = w0.copy()
        for s in range(3):
            ws = orc.stage_combine(cfg, mesh, s, w0, ws, lam * ws, dt)
        z = lam * dt
        np.testing.assert_allclose(ws, (1 + z + z * z / 2 + z ** 3 / 6) * w0, rtol=1e-14)


def test_dt_closed_form_constant_state(orc):
    cfg = orc.Config(dim=2, p=2)
    from paper_2407_20966_gb300 import inputs
    mesh = inputs.mesh_2d(4, 3, 0, 1, 0, 2, periodic=(True, True))
    om = orc.Mesh(mesh.nbr, mesh.h)
    rho, u, v, P = 1.2, 0.3, -0.8, 0.9
    w = np.zeros((4, mesh.n_elem, cfg.ns))
    w[:] = inputs.conservative(rho, [u, v], P)[:, None, None]
    c = math.sqrt(1.4 * P / rho)
    expect = 0.2 * min(0.25 / (abs(u) + c), (2 / 3) / (abs(v) + c))
    assert orc.dt(cfg, om, w, 0.2) == pytest.approx(expect, rel=1e-14)
