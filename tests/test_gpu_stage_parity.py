"""Per-stage parity on identical inputs: one SSP-RK3 stage (Sec. 5) split into its calls, each fed
exactly the inputs the checker uses, each output compared element by element.

For every stage s of a step, from the checker's stage input ws (and the step input wn):
  traces      kbl_traces(ws)                      vs orc.traces          FP64 in both modes: 1e-14
  bounds      kbl_bounds(ws, wf)                  vs orc.bounds          1e-12 FP64 / 1e-5 FP32-mixed
  residual    kbl_rhs(ws, wf)                     vs orc.rhs             1e-12 FP64 / 1e-5 FP32-mixed
  stage       kbl_stage(s, wn, ws, R, bnd, dt)    vs orc.stage_combine + orc.limit, with the checker's
              R and bounds: the limiter is FP64 in both modes, so 1e-12 in both, and alpha agrees
  composed    kbl_stage with the device's own R and bounds vs the checker's stage (its own R and
              bounds): 1e-12 FP64, 1e-5 FP32-mixed, element by element
Bounds use the scale-aware error of gpu_helpers.bounds_error, states state_error, residuals
rhs_error (per element and component).  The mesh spans many thread blocks with a ragged tail.
"""
import numpy as np
import pytest

from tests.gpu_helpers import (TOL_FP32, TOL_FP64, both, bounds_error, mesh_and_field, rhs_error,
                               state_error, to_dev, upload, zeros_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


CASES = [  # (dim, p, nu, mesh, precision, uncoupled, flux, kind)
    (2, 3, (32, 32), (13, 11), 1, 0, 0, "disc"),
    (2, 3, (32, 32), (13, 11), 1, 1, 0, "disc"),
    (2, 3, (32, 32), (13, 11), 0, 0, 0, "disc"),
    (2, 2, (16, 16), (17, 9), 1, 0, 1, "disc"),
    (2, 2, (16, 16), (17, 9), 0, 1, 2, "disc"),
    (2, 4, (32, 32), (7, 6), 1, 1, 2, "smooth"),
    (1, 3, (64,), 53, 1, 0, 0, "disc"),
    (1, 3, (64,), 53, 0, 1, 1, "disc"),
]


@pytest.mark.parametrize("dim,p,nu,n,precision,uncoupled,flux,kind", CASES)
def test_stage_parity_identical_inputs(orc, dim, p, nu, n, precision, uncoupled, flux, kind):
    import torch
    ctx, ocfg = both(orc, dim, p, nu, precision=precision, uncoupled=uncoupled, flux=flux)
    seed = 300 + 7 * p + 3 * uncoupled + flux + 50 * precision
    for sd in range(seed, seed + 40):   # the first field whose stage inputs stay physical
        mesh, w = mesh_and_field(orc, dim, p, n, seed=sd, kind=kind)
        om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
        try:
            dt = orc.dt(ocfg, om, w, 0.1)
            orc.ssprk3_step(ocfg, om, w, dt)
            break
        except orc.OracleError:
            continue
    om = upload(ctx, orc, mesh)
    tb = TOL_FP64 if precision == 0 else TOL_FP32
    wn, ws = w, w
    limited = 0
    for s in range(3):
        # traces
        wf_ref = orc.traces(ocfg, om, ws)
        wf = zeros_dev(*wf_ref.shape)
        ctx.traces(to_dev(ws), wf)
        np.testing.assert_allclose(wf.cpu().numpy(), wf_ref, rtol=1e-14, atol=1e-14 * np.abs(wf_ref).max())
        # bounds
        bnd_ref = orc.bounds(ocfg, om, ws, wf_ref)
        bnd = zeros_dev(2, ocfg.nv, mesh.n_elem)
        ctx.bounds(to_dev(ws), to_dev(wf_ref), bnd)
        ctx.check()
        eb = bounds_error(bnd.cpu().numpy(), bnd_ref)
        assert eb.max() < tb, ("bounds", s, eb.max())
        # residual
        R_ref = orc.rhs(ocfg, om, ws, wf_ref)
        R = zeros_dev(*w.shape)
        ctx.rhs(to_dev(ws), to_dev(wf_ref), R)
        er = rhs_error(R.cpu().numpy(), R_ref, ws, wf_ref, mesh)
        assert er.max() < tb, ("residual", s, er.max())
        # stage + limiter on the checker's residual and bounds
        comb = orc.stage_combine(ocfg, om, s, wn, ws, R_ref, dt)
        ref, a_ref = orc.limit(ocfg, om, comb, bnd_ref)
        limited += int((a_ref[0] < 1).sum())
        dtd = to_dev(np.array([dt]))
        out = zeros_dev(*w.shape)
        alpha = zeros_dev(2, mesh.n_elem)
        ctx.stage(s, to_dev(wn), to_dev(ws), to_dev(R_ref), to_dev(bnd_ref), dtd, out, alpha)
        es = state_error(out.cpu().numpy(), ref).max(axis=(0, 2))
        assert es.max() < TOL_FP64, ("stage", s, es.max())
        np.testing.assert_allclose(alpha.cpu().numpy(), a_ref, rtol=1e-10, atol=1e-12)
        # the composed stage: the device's own residual and bounds
        out2 = zeros_dev(*w.shape)
        ctx.stage(s, to_dev(wn), to_dev(ws), R, bnd, dtd, out2)
        ec = state_error(out2.cpu().numpy(), ref).max(axis=(0, 2))
        print(f"stage {s}: bounds {eb.max():.2e} residual {er.max():.2e} stage {es.max():.2e} "
              f"composed {ec.max():.2e} ({len(ec)} elements)")
        assert ec.max() < tb, ("composed", s, int(np.argmax(ec)), ec.max())
        ws = ref   # next stage from the checker's state
        torch.cuda.synchronize()
    print(f"dim {dim} p {p} precision {precision} uncoupled {uncoupled} flux {flux}: limited element-stages",
          limited)
