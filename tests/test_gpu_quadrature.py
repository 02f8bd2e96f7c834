"""GPU parity of the velocity grid options: node counts that do not fill a 2D kernel tile
(padded with zero-weight nodes) and the Romberg quadrature that Sec. 5 names beside the
trapezoidal rule, against the checker, through the C ABI."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import (TOL_FP32, TOL_FP64, both, bounds_error, mesh_and_field, state_error, to_dev,
                               upload, zeros_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _bounds(orc, dim, p, nu, n, precision, seed, **kw):
    ctx, ocfg = both(orc, dim, p, nu, precision=precision, **kw)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=seed, kind="disc")
    om = upload(ctx, orc, mesh)
    wf = orc.traces(ocfg, om, w)
    ref = orc.bounds(ocfg, om, w, wf)
    bnd = zeros_dev(2, ocfg.nv, mesh.n_elem)
    ctx.bounds(to_dev(w), to_dev(wf), bnd)
    ctx.check()
    return bounds_error(bnd.cpu().numpy(), ref).max()


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_FP32)])
@pytest.mark.parametrize("p,nu,n", [(3, 24, (5, 4)), (2, 5, (6, 3)), (3, 40, (3, 3)), (1, 17, (4, 4)),
                                    (4, 63, (2, 3)), (2, 2, (3, 2))])
def test_padded_2d_grid_trapezoid(orc, p, nu, n, precision, tol):
    """Node counts between the tile sizes 8, 16, 32, 64: the extra tile nodes carry no weight."""
    assert _bounds(orc, 2, p, (nu, nu), n, precision, seed=300 + nu) < tol


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_FP32)])
@pytest.mark.parametrize("dim,p,nu,n", [(1, 3, (65,), 23), (1, 2, (2049,), 5), (1, 4, (97,), 9),
                                        (2, 3, (33, 33), (5, 4)), (2, 2, (17, 17), (6, 5)),
                                        (2, 1, (9, 9), (3, 3)), (2, 4, (63, 63), (2, 2))])
def test_bounds_romberg(orc, dim, p, nu, n, precision, tol):
    assert _bounds(orc, dim, p, nu, n, precision, seed=320 + p, quadrature=1) < tol


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_FP32)])
@pytest.mark.parametrize("dim,p,nu,n", [(1, 3, (65,), 40), (2, 3, (33, 33), (8, 6))])
def test_full_step_romberg(orc, dim, p, nu, n, precision, tol):
    ctx, ocfg = both(orc, dim, p, nu, precision=precision, quadrature=1)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=340 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    dt = orc.dt(ocfg, om, w, 0.05)
    ref, _ = orc.ssprk3_step(ocfg, om, w, dt)
    wd = to_dev(w)
    ctx.set_time(0.0)
    ctx.step(wd, 0.05)
    ctx.check()
    assert state_error(wd.cpu().numpy(), ref).max() < tol


def test_sod_romberg_equals_checker(orc):
    """Ten Sod steps (Sec. 6.1 set-up) with Romberg on 65 points: the same as the checker."""
    from paper_2407_20966_gb300 import kbl
    mesh, ic = inputs.sod(200)
    ctx = kbl.Context(dim=1, p=3, nu=(65,), precision=kbl.FP64, quadrature=1)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    xi = ctx.operator(kbl.OP_NODES)
    w0 = inputs.nodal_field(mesh, xi, ic)
    cfg = orc.Config(dim=1, p=3, nu=(65,), quadrature=1)
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    wd = to_dev(w0)
    ctx.set_time(0.0)
    ctx.counters()
    ref = w0.copy()
    for _ in range(10):
        ctx.step(wd, 0.1)
        ref, _ = orc.ssprk3_step(cfg, om, ref, orc.dt(cfg, om, ref, 0.1))
    st, c = ctx.counters()
    assert st == kbl.OK and c["limited_elements"] > 0
    assert state_error(wd.cpu().numpy(), ref).max() < TOL_FP64


def test_romberg_and_grid_argument_checks():
    from paper_2407_20966_gb300 import kbl
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=1, p=3, nu=(64,), quadrature=1)        # 63 intervals: no coarser grid
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=2, p=3, nu=(32, 32), quadrature=1)
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=2, p=3, nu=(65, 65))                   # above the largest tile
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=2, p=3, nu=(17, 33))                   # square grids only
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=1, p=3, nu=(65,), quadrature=2)
    m = inputs.mesh_2d(3, 3, 0.0, 1.0, 0.0, 1.0, periodic=(True, True))
    with pytest.raises(kbl.KblError):
        kbl.Batch([(2, m.nbr, m.h, np.zeros((0, 4)))], quadrature=1)


def test_adjoint_rejects_other_grids():
    from paper_2407_20966_gb300 import kbl
    m = inputs.mesh_2d(4, 4, 0.0, 1.0, 0.0, 1.0, periodic=(True, True))
    for kw in ({"nu": (17, 17), "quadrature": 1}, {"nu": (24, 24)}):
        ctx = kbl.Context(dim=2, p=2, precision=kbl.FP64, **kw)
        ctx.mesh_upload(m.nbr, m.h, m.bc)
        w = to_dev(np.zeros((4, m.n_elem, 9)))
        with pytest.raises(kbl.KblError):
            ctx.adjoint_segment(w, np.array([1e-3]), zeros_dev(4, m.n_elem, 9))
