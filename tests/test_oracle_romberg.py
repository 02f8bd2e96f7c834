"""Pins of the checker's Romberg velocity quadrature (the alternative to the trapezoidal rule
that Sec. 5 names): the rule against textbook Newton-Cotes formulas, its polynomial degree,
positivity, and the bounds it gives against closed forms and the envelope invariants."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.test_oracle_bounds import maxwellian_box_moments


def test_first_level_is_simpson_and_second_is_boole(orc):
    """One extrapolation of the trapezoidal rule is Simpson's rule, two are Boole's rule
    (any numerical analysis text)."""
    np.testing.assert_allclose(orc.romberg_weights(3), np.array([1, 4, 1]) / 3, rtol=1e-15)
    # nu - 1 = 6 = 2 * 3: one level, composite Simpson
    np.testing.assert_allclose(orc.romberg_weights(7), np.array([1, 4, 2, 4, 2, 4, 1]) / 3, rtol=1e-15)
    np.testing.assert_allclose(orc.romberg_weights(5), 2 * np.array([7, 32, 12, 32, 7]) / 45, rtol=1e-14)
    # nu - 1 odd: no coarser grid, the trapezoidal rule itself
    np.testing.assert_allclose(orc.romberg_weights(4), [0.5, 1, 1, 0.5], rtol=0)


@pytest.mark.parametrize("n,levels", [(9, 3), (17, 4), (33, 5), (13, 2)])
def test_polynomial_degree(orc, n, levels):
    """L extrapolations integrate polynomials of degree 2L + 1 exactly and not degree 2L + 2
    (the Euler-Maclaurin expansion of the trapezoidal error has only even powers of h)."""
    q = orc.romberg_weights(n)
    x = np.linspace(0.0, 1.0, n)
    h = 1.0 / (n - 1)
    for deg in range(2 * levels + 2):
        assert (q * h * x ** deg).sum() == pytest.approx(1.0 / (deg + 1), rel=1e-12, abs=1e-13)
    deg = 2 * levels + 2
    assert abs((q * h * x ** deg).sum() - 1.0 / (deg + 1)) > 1e-12


@pytest.mark.parametrize("n", [3, 5, 17, 33, 65, 129, 257, 2049, 4097, 97])
def test_weights_positive_and_sum_to_the_interval(orc, n):
    """Romberg weights are positive, so the envelope arguments of Sec. 4 carry over; they add up
    to the interval length."""
    q = orc.romberg_weights(n)
    assert (q > 0).all()
    assert q.sum() == pytest.approx(n - 1, rel=1e-13)


@pytest.mark.parametrize("d,nu", [(1, (65,)), (2, (65, 65))])
def test_single_maxwellian_matches_the_box_erf_form_far_better_than_trapezoid(orc, d, nu):
    """k = 4: on one Maxwellian (smooth on the box) the extrapolation removes the h^2, h^4 ...
    terms of the trapezoidal error, so the moments meet the exact box moments written with
    erf about two orders of magnitude closer than the trapezoidal rule on the same grid.  The
    coarsest levels of the tableau have a few points across the box, outside the asymptotic
    range of the error expansion; below about 65 points per axis they take the gain away (at
    33 points both rules are off by about 1e-5)."""
    rng = np.random.default_rng(50 + d)
    w = inputs.random_states(rng, 1, d)[0]
    S = np.tile(w, (2, 1))
    errs = {}
    for quad in (0, 1):
        cfg = orc.Config(dim=d, p=3, nu=nu, k=4.0, r_fac=0.0, quadrature=quad)
        lo_b, hi_b = orc.velocity_box(cfg, S)
        exact = maxwellian_box_moments(w, d, lo_b, hi_b)
        lo, hi = orc.bounds_stencil(cfg, S)
        assert np.array_equal(lo, hi)
        errs[quad] = np.abs(lo - exact).max() / np.abs(exact).max()
    assert errs[1] < 1e-7, errs
    assert errs[1] < 2e-2 * errs[0], errs


@pytest.mark.parametrize("d,nu,r", [(1, (65,), 0.0), (1, (65,), 1e-3), (2, (17, 17), 0.0), (2, (17, 17), 1e-3)])
def test_every_stencil_state_lies_inside_its_romberg_bounds_exactly(orc, d, nu, r):
    """Each g_i lies between f_min and f_max pointwise (Eq. 32) and the weights are positive,
    so its quadrature moments lie inside the bounds with no tolerance."""
    rng = np.random.default_rng(60 + d)
    cfg = orc.Config(dim=d, p=3, nu=nu, k=4.0, r_fac=r, rho_floor=0.0, quadrature=1)
    for _ in range(5):
        S = inputs.random_states(rng, 9, d)
        lo, hi = orc.bounds_stencil(cfg, S)
        for i in range(len(S)):
            mom = orc.state_moments(cfg, S, i)
            assert np.all(lo <= mom) and np.all(mom <= hi), (i, lo, mom, hi)


def test_romberg_needs_an_even_number_of_intervals(orc):
    cfg = orc.Config(dim=1, p=3, nu=(64,), quadrature=1)
    S = inputs.random_states(np.random.default_rng(1), 3, 1)
    with pytest.raises(Exception):
        orc.bounds_stencil(cfg, S)


@pytest.mark.parametrize("n", [3, 5, 9, 17, 33, 63, 65, 97, 2049])
def test_library_weights_equal_the_checkers(orc, n):
    """The weights the kernels apply (library host code, kbl_velocity_weights) against the
    checker's independent construction: Romberg to rounding, the trapezoidal rule exactly.
    Host only, so this runs without a GPU."""
    from paper_2407_20966_gb300 import kbl
    np.testing.assert_allclose(kbl.velocity_weights(n, 1), orc.romberg_weights(n), rtol=1e-13, atol=1e-15)
    trap = np.ones(n)
    trap[0] = trap[-1] = 0.5
    np.testing.assert_array_equal(kbl.velocity_weights(n, 0), trap)


def test_library_weights_reject_bad_arguments():
    from paper_2407_20966_gb300 import kbl
    for nu, q in ((1, 0), (64, 1), (33, 2)):
        with pytest.raises(kbl.KblError):
            kbl.velocity_weights(nu, q)
