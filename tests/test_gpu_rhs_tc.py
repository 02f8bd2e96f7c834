"""The FP32-mixed 2D residual with its operator product on the tensor cores (tcgen05, TF32 split
pairs, FP32 accumulation in tensor memory; element tiles staged by TMA), orders 2 and 3: against
the checker (1e-5 of the size of the residual's terms, per element and component; the Sec. 2.3
residual), against the CUDA-core FP32 residual of the same context (knob KBL_TUNE_RHS_TC = 0),
on meshes of several 32-element tiles with a ragged tail, a single element, every flux, and
inside whole steps.  No bounded wait of the kernel may expire (the timeout flag stays clear)."""
import numpy as np
import pytest

from tests.gpu_helpers import (TOL_FP32, both, mesh_and_field, rhs_error, state_error, step_sensitivity, to_dev,
                               upload, zeros_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


@pytest.mark.parametrize("p,n,flux,kind", [
    (3, (13, 11), 0, "disc"), (3, (40, 33), 0, "smooth"), (2, (17, 9), 0, "disc"), (2, (64, 37), 2, "disc"),
    (3, (9, 7), 1, "disc"), (3, (1, 1), 0, "smooth"), (2, (3, 1), 1, "smooth")])
def test_rhs_tensor_cores_match_checker(orc, p, n, flux, kind):
    from paper_2407_20966_gb300 import kbl
    ctx, ocfg = both(orc, 2, p, (16, 16), precision=1, flux=flux)
    ctx.set_tuning(kbl.TUNE_RHS_TC, 1)
    assert ctx.get_tuning(kbl.TUNE_RHS_TC) == 1
    for seed in range(500, 540):   # a field whose face traces are physical (HLLC, HLL need it)
        mesh, w = mesh_and_field(orc, 2, p, n, seed=seed, kind=kind)
        om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
        wf = orc.traces(ocfg, om, w)
        mm = wf[1] ** 2 + wf[2] ** 2
        if wf[0].min() > 0 and (wf[3] - 0.5 * mm / wf[0]).min() > 0:
            break
    om = upload(ctx, orc, mesh)
    R_ref = orc.rhs(ocfg, om, w, wf)
    R = zeros_dev(*w.shape)
    ctx.rhs(to_dev(w), to_dev(wf), R)
    st, c = ctx.counters()
    assert st == 0 and c["timeout"] == 0
    got = R.cpu().numpy()
    err = rhs_error(got, R_ref, w, wf, mesh)
    print(f"P{p} {n} flux {flux}: tensor-core residual error {err.max():.2e}")
    assert err.max() < TOL_FP32, err.max()
    ctx.set_tuning(kbl.TUNE_RHS_TC, 0)
    R2 = zeros_dev(*w.shape)
    ctx.rhs(to_dev(w), to_dev(wf), R2)
    e2 = rhs_error(R2.cpu().numpy(), R_ref, w, wf, mesh)
    print(f"   CUDA-core FP32 residual error {e2.max():.2e}")
    assert rhs_error(got, R2.cpu().numpy(), w, wf, mesh).max() < 2 * TOL_FP32


@pytest.mark.parametrize("p", [3, 2])
def test_full_step_with_tensor_core_residual(orc, p):
    """A step with the tensor-core residual inside the step graph, against the checker with the
    device's time step (criterion of test_full_step_uncoupled)."""
    from paper_2407_20966_gb300 import kbl
    ctx, ocfg = both(orc, 2, p, (32, 32), precision=1)
    ctx.set_tuning(kbl.TUNE_RHS_TC, 1)
    mesh, w = mesh_and_field(orc, 2, p, (11, 9), seed=77 + p, kind="disc")
    om = upload(ctx, orc, mesh)
    wd = to_dev(w)
    ctx.set_time(0.0)
    ctx.step(wd, 0.1)
    dt = ctx.time()
    ref, _ = orc.ssprk3_step(ocfg, om, w, dt)
    st, c = ctx.counters()
    assert st == 0 and c["timeout"] == 0
    err = state_error(wd.cpu().numpy(), ref).max(axis=(0, 2))
    allowed = np.maximum(TOL_FP32, 10 * step_sensitivity(orc, ocfg, om, w, dt, ref))
    print(f"P{p}: step with the tensor-core residual, max error {err.max():.2e}")
    assert np.all(err <= allowed), (int(np.argmax(err / allowed)), err.max())
