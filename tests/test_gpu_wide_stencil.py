"""The wider 1D stencil (kbl_config.stencil = 1: own solution points and both face neighbours'
solution points, the stencil config 1 of the benchmark set names) on the GPU against the checker.

  gather    kbl_gather_stencil                    vs orc.gather_stencil      bit-exact
  bounds    kbl_bounds                            vs orc.bounds              1e-12 FP64 / 1e-5 FP32
  steps     kbl_step on the Sod tube (200 P3)     vs orc.ssprk3_step         1e-11 over 20 steps
  config    a 2D context with stencil = 1         KBL_EINVAL
"""
import numpy as np
import pytest

from tests.gpu_helpers import TOL_FP32, TOL_FP64, both, bounds_error, mesh_and_field, state_error, to_dev, \
    upload, zeros_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


@pytest.mark.parametrize("p,n,periodic", [(3, 37, False), (1, 130, True), (5, 9, False)])
def test_gather_and_bounds(orc, p, n, periodic):
    for precision in (0, 1):
        ctx, ocfg = both(orc, 1, p, (64,), precision=precision, stencil=1)
        mesh, w = mesh_and_field(orc, 1, p, n, seed=60 + p, periodic=periodic)
        om = upload(ctx, orc, mesh)
        assert ctx.nstencil == 3 * (p + 1) == ocfg.nstencil
        wf = orc.traces(ocfg, om, w)
        E = mesh.n_elem
        S = zeros_dev(E, ocfg.nstencil, ocfg.nv)
        ctx.gather_stencil(to_dev(w), to_dev(wf), 0, E, S)
        S = S.cpu().numpy()
        for e in range(E):
            np.testing.assert_array_equal(S[e], orc.gather_stencil(ocfg, om, w, wf, e))
        ref = orc.bounds(ocfg, om, w, wf)
        bnd = zeros_dev(2, ocfg.nv, E)
        ctx.bounds(to_dev(w), to_dev(wf), bnd)
        ctx.check()
        err = bounds_error(bnd.cpu().numpy(), ref)
        assert err.max() < (TOL_FP64 if precision == 0 else TOL_FP32), (precision, err.max())


def test_sod_steps(orc):
    from paper_2407_20966_gb300 import inputs
    mesh, ic = inputs.sod(200)
    ctx, ocfg = both(orc, 1, 3, (64,), stencil=1)
    om = upload(ctx, orc, mesh)
    xi, _ = orc.gauss_legendre(4)
    w = inputs.nodal_field(mesh, xi, ic)
    ref, limited = w.copy(), 0
    dts = []
    for _ in range(20):
        dt = orc.dt(ocfg, om, ref, 0.1)
        ref, alpha = orc.ssprk3_step(ocfg, om, ref, dt)
        limited += int((alpha[0] < 1).sum())
        dts.append(dt)
    assert limited > 0
    wd = to_dev(w)
    ctx.set_time(0.0)
    for _ in range(20):
        ctx.step(wd, 0.1)
    ctx.check()
    assert state_error(wd.cpu().numpy(), ref).max() < 1e-11


def test_wide_stencil_is_1d_only():
    from paper_2407_20966_gb300 import kbl
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=2, p=2, stencil=1)
    with pytest.raises(kbl.KblError):
        kbl.Context(dim=1, p=2, stencil=2)
