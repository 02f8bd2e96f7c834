"""The limiter's fast path certifies alpha = 1 (Eq. 37-39) and a passing pressure test (Eq. 47)
with an FP32 screen and skips the FP64 limiter for those elements; every other element takes the
exact FP64 path.  These cases sit on both sides of each decision, at relative distances from
1e-3 down to 1e-9: the device must take the same decision as the checker in every one of them
(a screen that wrongly passed an element would return alpha = 1 where the checker's is below 1)."""
import numpy as np
import pytest

from tests.gpu_helpers import TOL_FP64, both, mesh_and_field, state_error, to_dev, upload, zeros_dev

pytestmark = pytest.mark.gpu

GAPS = [-1e-3, -1e-6, -1e-7, -1e-8, -1e-9, 0.0, 1e-9, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _mean_and_V(orc, ocfg, om, w, dim, p):
    """Element means with the Gauss-Legendre weights of Eq. 13 and the values at V (solution
    and own face points)."""
    _, wq = orc.gauss_legendre(p + 1)
    W = np.asarray(wq) if dim == 1 else np.outer(wq, wq).ravel()
    mean = (w * W).sum(axis=2) / W.sum()
    V = np.concatenate([w, orc.traces(ocfg, om, w)], axis=2)
    return mean, V


def _limit_both(orc, ctx, ocfg, om, w, bnd):
    ref, a_ref = orc.limit(ocfg, om, w, bnd)
    wd = to_dev(w)
    alpha = zeros_dev(2, w.shape[1])
    ctx.limit(wd, to_dev(bnd), alpha)
    ctx.check()
    return wd.cpu().numpy(), alpha.cpu().numpy(), ref, a_ref


@pytest.mark.parametrize("dim,p,n", [(2, 3, (12, 8)), (2, 2, (8, 6)), (2, 4, (6, 7)), (1, 3, 96)])
@pytest.mark.parametrize("uncoupled", [0, 1])
def test_screen_at_the_bounds(orc, dim, p, n, uncoupled):
    """Bounds at the extremes of V times (1 + g), on the upper side, the lower side or both."""
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16), uncoupled=uncoupled)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=600 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    E = mesh.n_elem
    mean, V = _mean_and_V(orc, ocfg, om, w, dim, p)
    dmax, dmin = V.max(axis=2) - mean, V.min(axis=2) - mean
    g = np.array([GAPS[e % len(GAPS)] for e in range(E)])
    side = (np.arange(E) // len(GAPS)) % 3   # 0: the upper bound at the gap, 1: the lower, 2: both
    gu = np.where(side != 1, g, 1.0)         # the other side at twice the deviation
    gl = np.where(side != 0, g, 1.0)
    bnd = np.stack([mean + dmin * (1 + gl), mean + dmax * (1 + gu)])
    got, ga, ref, a_ref = _limit_both(orc, ctx, ocfg, om, w, bnd)
    assert state_error(got, ref).max() < TOL_FP64
    np.testing.assert_allclose(ga, a_ref, rtol=1e-10, atol=1e-12)
    decided = g != 0.0   # at g = 0 the last bit of the mean decides
    np.testing.assert_array_equal((ga[0] < 1)[decided], (a_ref[0] < 1)[decided])
    assert (a_ref[0][g > 0] == 1).all() and (a_ref[0][g < 0] < 1).all()


def test_screen_at_eps(orc):
    """Density constant up to deviations around eps = 1e-13 (the epsilon rule of Eq. 37)."""
    ctx, ocfg = both(orc, 2, 3, (16, 16))
    mesh, w = mesh_and_field(orc, 2, 3, (8, 6), seed=610, kind="smooth")
    om = upload(ctx, orc, mesh)
    rng = np.random.default_rng(611)
    deltas = [2e-14, 9e-14, 1.1e-13, 2e-13, 1e-12, 1e-9, 1e-7, 1e-6, 1e-4]
    for e in range(mesh.n_elem):
        w[0, e] = 1.0 + deltas[e % len(deltas)] * rng.uniform(-1.0, 1.0, w.shape[2])
    mean, V = _mean_and_V(orc, ocfg, om, w, 2, 3)
    span = V.max(axis=2) - V.min(axis=2)
    bnd = np.stack([mean - 2 * span - 1e-3 * np.abs(mean), mean + 2 * span + 1e-3 * np.abs(mean)])
    got, ga, ref, a_ref = _limit_both(orc, ctx, ocfg, om, w, bnd)
    assert state_error(got, ref).max() < TOL_FP64
    np.testing.assert_allclose(ga, a_ref, rtol=1e-10, atol=1e-12)
    assert (a_ref[0] == 0).any() and (a_ref[0] == 1).any()


@pytest.mark.parametrize("dim,p,n", [(2, 3, (8, 6)), (2, 2, (6, 6)), (1, 3, 48)])
def test_screen_at_the_pressure_floor(orc, dim, p, n):
    """Each element scaled so that its smallest pressure over V is p_floor (1 + g); the bounds are
    wide, so only Eq. 47-49 can act."""
    p_floor, gamma = 0.05, 1.4
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16), p_floor=p_floor)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=620 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    E = mesh.n_elem
    gp = np.array([[-1e-3, -1e-7, -1e-9, 1e-9, 1e-7, 1e-6, 1e-5, 1e-3, 0.1][e % 9] for e in range(E)])
    _, V = _mean_and_V(orc, ocfg, om, w, dim, p)
    mm = sum(V[1 + k] ** 2 for k in range(dim))
    pmin = ((gamma - 1.0) * (V[dim + 1] - 0.5 * mm / V[0])).min(axis=1)
    assert (pmin > 0).all()
    w = w * (p_floor * (1.0 + gp) / pmin)[None, :, None]   # pressure is homogeneous of degree 1
    mean, V = _mean_and_V(orc, ocfg, om, w, dim, p)
    span = V.max(axis=2) - V.min(axis=2)
    bnd = np.stack([mean - 2 * span - 0.5 * np.abs(mean), mean + 2 * span + 0.5 * np.abs(mean)])
    got, ga, ref, a_ref = _limit_both(orc, ctx, ocfg, om, w, bnd)
    assert (a_ref[0] == 1).all()
    assert state_error(got, ref).max() < TOL_FP64
    np.testing.assert_allclose(ga, a_ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(ga[1] < 1, a_ref[1] < 1)
    assert ((a_ref[1] < 1) == (gp < 0)).all()


@pytest.mark.parametrize("scale", [1e-30, 1e-8, 1e6, 1e25, 1e35, 1e100])
def test_screen_at_extreme_magnitudes(orc, scale):
    """States scaled into and beyond the FP32 range (eps = 0 and p_floor = 0, so that only the
    bound tests decide): where the screen cannot resolve the values it must leave the element
    to the exact path, and every result equals the checker's."""
    ctx, ocfg = both(orc, 2, 3, (16, 16), eps=0.0, p_floor=0.0)
    mesh, w = mesh_and_field(orc, 2, 3, (8, 6), seed=630, kind="smooth")
    om = upload(ctx, orc, mesh)
    w = w * scale
    mean, V = _mean_and_V(orc, ocfg, om, w, 2, 3)
    dmax, dmin = V.max(axis=2) - mean, V.min(axis=2) - mean
    g = np.array([[-1e-3, -1e-7, 1e-7, 1e-3, 0.5][e % 5] for e in range(mesh.n_elem)])
    bnd = np.stack([mean + dmin * (1 + g), mean + dmax * (1 + g)])
    got, ga, ref, a_ref = _limit_both(orc, ctx, ocfg, om, w, bnd)
    assert state_error(got, ref).max() < TOL_FP64
    np.testing.assert_allclose(ga, a_ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(ga[0] < 1, a_ref[0] < 1)
    assert ((a_ref[0] < 1) == (g < 0)).all()
