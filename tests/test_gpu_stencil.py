"""kbl_bounds_stencil: the kinetic bounds of stencils the caller assembles (any element family:
triangles with their own solution and face points, unstructured meshes), against the checker
element by element, and bit for bit against kbl_bounds when the stencils are the FR ones."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import TOL_FP32, TOL_FP64, both, bounds_error, mesh_and_field, to_dev, upload, zeros_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _random_stencils(seed, E, n, spread):
    """E stencils of n admissible 2D states around a per-element base state."""
    rng = np.random.default_rng(seed)
    base = inputs.random_states(rng, E, 2)
    S = np.repeat(base[:, None, :], n, axis=1)
    S = S * (1.0 + spread * rng.uniform(-1.0, 1.0, S.shape))
    # keep the internal energy positive: E >= |m|^2 / (2 rho) * 1.05
    ke = 0.5 * (S[..., 1] ** 2 + S[..., 2] ** 2) / S[..., 0]
    S[..., 3] = np.maximum(S[..., 3], 1.05 * ke + 1e-3)
    return S


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_FP32)])
@pytest.mark.parametrize("n,nu,quad", [(5, (32, 32), 0), (16, (32, 32), 0), (24, (32, 32), 0), (33, (16, 16), 0),
                                        (48, (32, 32), 0), (64, (32, 32), 0), (24, (17, 17), 1), (15, (24, 24), 0)])
def test_explicit_stencils_against_checker(orc, n, nu, quad, precision, tol):
    """Random stencils of n states (24 = a P2 triangle: 6 solution, 9 own and 9 exterior face
    points; 15 = P1), including padded and Romberg velocity grids."""
    from paper_2407_20966_gb300 import kbl
    E = 37
    S = _random_stencils(400 + n, E, n, spread=0.3)
    ctx = kbl.Context(dim=2, p=3, nu=nu, precision=precision, quadrature=quad)
    bnd = zeros_dev(2, 4, E)
    ctx.bounds_stencil(to_dev(S), bnd)
    ctx.check()
    cfg = orc.Config(dim=2, p=3, nu=nu, quadrature=quad)
    ref = np.zeros((2, 4, E))
    for e in range(E):
        ref[0, :, e], ref[1, :, e] = orc.bounds_stencil(cfg, S[e])
    err = bounds_error(bnd.cpu().numpy(), ref).max()
    assert err < tol, err


@pytest.mark.parametrize("precision", [0, 1])
def test_fr_stencils_give_the_fr_bounds_bit_for_bit(orc, precision):
    """Stencils gathered from an FR mesh through kbl_gather_stencil: the explicit-stencil entry
    runs the same bounds code, so its bounds equal kbl_bounds exactly."""
    ctx, ocfg = both(orc, 2, 3, (32, 32), precision=precision)
    mesh, w = mesh_and_field(orc, 2, 3, (9, 7), seed=410, kind="disc")
    om = upload(ctx, orc, mesh)
    wd = to_dev(w)
    wf = zeros_dev(4, mesh.n_elem, ocfg.nfp)
    ctx.traces(wd, wf)
    ref = zeros_dev(2, 4, mesh.n_elem)
    ctx.bounds(wd, wf, ref)
    S = zeros_dev(mesh.n_elem, ocfg.nstencil, 4)
    ctx.gather_stencil(wd, wf, 0, mesh.n_elem, S)
    got = zeros_dev(2, 4, mesh.n_elem)
    ctx.bounds_stencil(S, got)
    ctx.check()
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


@pytest.mark.parametrize("precision", [0, 1])
def test_nonphysical_state_gives_nan_for_its_element_only(orc, precision):
    from paper_2407_20966_gb300 import kbl
    E, n = 6, 20
    S = _random_stencils(420, E, n, spread=0.2)
    S[3, 7, 3] = 0.5 * (S[3, 7, 1] ** 2 + S[3, 7, 2] ** 2) / S[3, 7, 0] - 1e-3   # P < 0
    ctx = kbl.Context(dim=2, p=3, nu=(32, 32), precision=precision)
    bnd = zeros_dev(2, 4, E)
    ctx.bounds_stencil(to_dev(S), bnd)
    st, c = ctx.counters()
    assert st == kbl.ENONPHYSICAL and c["nonphysical"]
    b = bnd.cpu().numpy()
    assert np.isnan(b[:, :, 3]).all()
    assert np.isfinite(np.delete(b, 3, axis=2)).all()


def test_argument_checks():
    from paper_2407_20966_gb300 import kbl
    ctx = kbl.Context(dim=2, p=3, nu=(32, 32))
    for n in (0, 65):
        with pytest.raises(kbl.KblError):
            ctx.bounds_stencil(zeros_dev(3, max(n, 1), 4) if n else zeros_dev(3, 0, 4), zeros_dev(2, 4, 3))
    ctx1 = kbl.Context(dim=1, p=3, nu=(64,))
    with pytest.raises(kbl.KblError):
        ctx1.bounds_stencil(zeros_dev(3, 5, 4), zeros_dev(2, 4, 3))
    # no elements: nothing to do
    ctx.bounds_stencil(zeros_dev(0, 5, 4), zeros_dev(2, 4, 0))


def _node_sets(seed, E, ns, nf, d, spread):
    rng = np.random.default_rng(seed)
    nv = d + 2
    base = inputs.random_states(rng, E, d)
    U = base[:, None, :] * (1.0 + spread * rng.uniform(-1.0, 1.0, (E, ns, nv)))
    F = base[:, None, :] * (1.0 + spread * rng.uniform(-1.0, 1.0, (E, nf, nv)))
    for X in (U, F):
        ke = 0.5 * sum(X[..., 1 + k] ** 2 for k in range(d)) / X[..., 0]
        X[..., d + 1] = np.maximum(X[..., d + 1], 1.2 * ke + 1e-2)
    W = rng.uniform(0.2, 1.0, ns)
    m = np.einsum("n,enk->ek", W, U) / W.sum()
    lo = (m - 0.05 * np.abs(m) - 1e-3).T.copy()
    hi = (m + 0.05 * np.abs(m) + 1e-3).T.copy()
    return W, U, F, np.stack([lo, hi])


@pytest.mark.parametrize("d,ns,nf,p_floor", [(2, 6, 9, 1e-12), (2, 6, 9, 0.05), (2, 10, 12, 1e-12), (1, 5, 2, 0.05),
                                             (2, 1, 0, 1e-12)])
@pytest.mark.parametrize("uncoupled", [0, 1])
def test_limit_node_sets_against_checker(orc, d, ns, nf, p_floor, uncoupled):
    """Caller-assembled node sets (6 + 9: a P2 triangle's solution and face points) with any
    positive mean weights, limited on the device and by the checker's node-set limiter."""
    from paper_2407_20966_gb300 import kbl
    E = 53
    W, U, F, bnd = _node_sets(500 + ns + nf, E, ns, nf, d, 0.4)
    ctx = kbl.Context(dim=d, p=2, nu=(32,) * d if d == 2 else (64,), p_floor=p_floor, uncoupled=uncoupled)
    Ud = to_dev(U)
    alpha = zeros_dev(2, E)
    ctx.limit_nodes(W, Ud, to_dev(F) if nf else zeros_dev(E, 0, d + 2), to_dev(bnd), alpha)
    st, c = ctx.counters()
    assert st == kbl.OK and c["limited_elements"] > 0
    cfg = orc.Config(dim=d, p=2, nu=(16,) * d, p_floor=p_floor, uncoupled=uncoupled)
    got, ga = Ud.cpu().numpy(), alpha.cpu().numpy()
    for e in range(E):
        ref, a = orc.limit_nodes(cfg, W, U[e].T, F[e].T if nf else np.zeros((d + 2, 0)), bnd[0, :, e], bnd[1, :, e])
        scale = np.abs(U[e]).max()
        np.testing.assert_allclose(got[e], ref.T, rtol=1e-12, atol=1e-13 * scale)
        np.testing.assert_allclose(ga[:, e], a, rtol=1e-12, atol=1e-14)


def test_limit_node_sets_argument_checks():
    from paper_2407_20966_gb300 import kbl
    ctx = kbl.Context(dim=2, p=3, nu=(32, 32))
    U, F, bnd = zeros_dev(3, 6, 4), zeros_dev(3, 9, 4), zeros_dev(2, 4, 3)
    for W, UU, FF in ((np.ones(6) * -1.0, U, F), (np.ones(65), zeros_dev(3, 65, 4), F),
                      (np.ones(6), U, zeros_dev(3, 65, 4))):
        with pytest.raises(kbl.KblError):
            ctx.limit_nodes(W, UU, FF, bnd)
