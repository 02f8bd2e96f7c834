"""GPU tests of the batched form (kbl_batch_*): many independent four-quadrant problems with
uneven sizes and orders in persistent launches.  Each problem's step must equal the
single-mesh FP32-mixed path on the same problem (same device code), and match the FP64
checker within the FP32 tolerance."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import TOL_FP32, TOL_FP64, bounds_error, rhs_error, state_error, step_sensitivity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _batch(seed=3, n_problems=11, n_range=(2, 9)):
    from paper_2407_20966_gb300 import kbl
    probs = inputs.four_quadrant_batch(seed, n_problems, n_range=n_range)
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs])
    w0 = inputs.batch_state(probs, b.nodes, b.state_offsets)
    return b, probs, w0


def test_batch_layout_and_orders():
    b, probs, w0 = _batch()
    assert b.P == len(probs)
    assert sorted(set(b.p.tolist())) == [1, 2, 3, 4]
    for i, (p, m, _) in enumerate(probs):
        assert b.state_offsets[i + 1] - b.state_offsets[i] == 4 * m.n_elem * (p + 1) ** 2


def test_batch_step_equals_single_mesh_path(orc):
    import torch
    from paper_2407_20966_gb300 import kbl
    b, probs, w0 = _batch()
    wd = torch.from_numpy(w0).cuda()
    b.step(wd, 0.2)
    b.check()
    got = wd.cpu().numpy()
    dts = b.dt()
    for i, (p, m, ic) in enumerate(probs):
        ctx = kbl.Context(dim=2, p=p, nu=(32, 32), precision=kbl.FP32_MIXED)
        ctx.set_tuning(kbl.TUNE_RHS_TC, 0)   # the batch runs the CUDA-core residual
        ctx.set_tuning(kbl.TUNE_BOUNDS_TILE, b.tuning()["tile"])   # and its bounds thread tile
        ctx.mesh_upload(m.nbr, m.h, m.bc)
        wi = torch.from_numpy(np.ascontiguousarray(b.state_view(w0, i))).cuda()
        ctx.set_time(0.0)
        ctx.step(wi, 0.2)
        assert ctx.time() == dts[i]
        np.testing.assert_array_equal(b.state_view(got, i), wi.cpu().numpy())


def _oracle_step(orc, cfg, om, w, dt):
    """One SSP-RK3 step of the checker, limited after every stage (Sec. 5)."""
    ws = w
    for s in range(3):
        wf = orc.traces(cfg, om, ws)
        bnd = orc.bounds(cfg, om, ws, wf)
        comb = orc.stage_combine(cfg, om, s, w, ws, orc.rhs(cfg, om, ws, wf), dt)
        ws, _ = orc.limit(cfg, om, comb, bnd)
    return ws


def test_batch_matches_fp64_checker(orc):
    """Full steps of discontinuous problems against the FP64 checker, the checker taking each
    problem's device time step (FP32 arithmetic in the batch), element by element against
    max(1e-5, 10 x the checker's own sensitivity to 1e-6 bound and residual errors)
    (gpu_helpers.step_sensitivity).  Per-stage parity on identical inputs, at a flat 1e-5:
    test_batch_stage_parity_identical_inputs."""
    import torch
    b, probs, w0 = _batch(seed=5, n_problems=6, n_range=(2, 6))
    wd = torch.from_numpy(w0).cuda()
    b.step(wd, 0.2)
    got = wd.cpu().numpy()
    dts = b.dt()
    for i, (p, m, ic) in enumerate(probs):
        cfg = orc.Config(dim=2, p=p, nu=(32, 32))
        om = orc.Mesh(m.nbr, m.h, m.bc)
        wi = np.ascontiguousarray(b.state_view(w0, i))
        xi, _ = orc.gauss_legendre(p + 1)
        np.testing.assert_allclose(b.nodes(p), xi, atol=2e-15)
        assert dts[i] == pytest.approx(orc.dt(cfg, om, wi, 0.2), rel=1e-6)
        ref = _oracle_step(orc, cfg, om, wi, dts[i])
        err = state_error(b.state_view(got, i), ref).max(axis=(0, 2))
        allowed = np.maximum(TOL_FP32, 10 * step_sensitivity(orc, cfg, om, wi, dts[i], ref))
        print(f"problem {i} (P{p}, {m.n_elem} elements): max error {err.max():.2e}, "
              f"elements above 1e-5: {int((err > TOL_FP32).sum())}")
        assert np.all(err <= allowed), (i, int(np.argmax(err / allowed)), err.max())


@pytest.mark.parametrize("flux,uncoupled", [(0, 0), (1, 1), (2, 0)])
def test_batch_stage_parity_identical_inputs(orc, flux, uncoupled):
    """Every problem of a batch, every stage of a step, on identical inputs (paper Sec. 3.3-3.8
    bounds, Sec. 2.3 residual, Sec. 5 SSP-RK3 stage with Eq. 37-39 and Eq. 47-49): the batched
    phase calls (the step graph's persistent kernels) against the checker's bounds (1e-5), residual
    (1e-5 per element and component) and stage + limiter on the checker's residual and bounds
    (1e-12: the limiter is FP64); the composed stage (the batch's own residual and bounds) to 1e-5
    element by element."""
    import torch
    from paper_2407_20966_gb300 import kbl
    probs = inputs.four_quadrant_batch(21 + flux, 7, n_range=(2, 9))
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs], flux=flux, uncoupled=uncoupled)
    w0 = inputs.batch_state(probs, b.nodes, b.state_offsets)
    cfgs = [orc.Config(dim=2, p=p, nu=(32, 32), flux=flux, uncoupled=uncoupled) for p, _, _ in probs]
    oms = [orc.Mesh(m.nbr, m.h, m.bc) for _, m, _ in probs]
    wn = [np.ascontiguousarray(b.state_view(w0, i)) for i in range(b.P)]
    dts = np.array([orc.dt(cfgs[i], oms[i], wn[i], 0.1) for i in range(b.P)])
    dtd = torch.from_numpy(dts).cuda()
    E = int(b.elem_offsets[-1])
    ws = list(wn)
    limited = 0
    for s in range(3):
        cat = np.zeros_like(w0)
        for i in range(b.P):
            b.state_view(cat, i)[...] = ws[i]
        wsd = torch.from_numpy(cat).cuda()
        wnd = torch.from_numpy(w0).cuda()
        bnd = torch.zeros(8 * E, dtype=torch.float64, device="cuda")
        R = torch.zeros_like(wsd)
        b.bounds(wsd, bnd)
        b.rhs(wsd, R)
        b.check()
        bg, Rg = bnd.cpu().numpy(), R.cpu().numpy()
        refs, combs, bnd_refs, R_refs = [], [], [], []
        for i in range(b.P):
            cfg, om = cfgs[i], oms[i]
            wf = orc.traces(cfg, om, ws[i])
            bnd_ref = orc.bounds(cfg, om, ws[i], wf)
            eb = bounds_error(b.bounds_view(bg, i), bnd_ref)
            assert eb.max() < TOL_FP32, ("bounds", s, i, eb.max())
            R_ref = orc.rhs(cfg, om, ws[i], wf)
            er = rhs_error(b.state_view(Rg, i), R_ref, ws[i], wf, oms[i])
            assert er.max() < TOL_FP32, ("residual", s, i, er.max())
            comb = orc.stage_combine(cfg, om, s, wn[i], ws[i], R_ref, dts[i])
            ref, a = orc.limit(cfg, om, comb, bnd_ref)
            limited += int((a[0] < 1).sum())
            refs.append(ref), combs.append(comb), bnd_refs.append(bnd_ref), R_refs.append(R_ref)
        # stage + limiter on the checker's residual and bounds
        Rc = np.zeros_like(w0)
        bc = np.zeros(8 * E)
        for i in range(b.P):
            b.state_view(Rc, i)[...] = R_refs[i]
            b.bounds_view(bc, i)[...] = bnd_refs[i]
        out = torch.zeros_like(wsd)
        b.stage(s, wnd, wsd, torch.from_numpy(Rc).cuda(), torch.from_numpy(bc).cuda(), dtd, out)
        out2 = torch.zeros_like(wsd)
        b.stage(s, wnd, wsd, R, bnd, dtd, out2)
        b.check()
        got, got2 = out.cpu().numpy(), out2.cpu().numpy()
        for i in range(b.P):
            es = state_error(b.state_view(got, i), refs[i]).max(axis=(0, 2))
            assert es.max() < TOL_FP64, ("stage", s, i, es.max())
            ec = state_error(b.state_view(got2, i), refs[i]).max(axis=(0, 2))
            assert ec.max() < TOL_FP32, ("composed", s, i, int(np.argmax(ec)), ec.max())
        ws = refs
    print(f"batch flux {flux} uncoupled {uncoupled}: {b.P} problems, limited element-stages {limited}")


def test_batch_autotune_keeps_results(orc):
    """The autotuner changes the launch shape only (the FP32 summation order of the bounds), so the
    tuned step meets the criterion of test_batch_matches_fp64_checker against the FP64 checker.
    Among these problems a P4 element driven towards vacuum (density bound at the floor, a
    pressure re-limit) changes by 1.9e-5 in the checker itself under a 1e-8 input perturbation."""
    import torch
    b, probs, w0 = _batch(seed=7, n_problems=9, n_range=(4, 12))
    ms, cmp = b.autotune(torch.from_numpy(w0).cuda(), with_cmp=True)
    assert cmp > 0
    t = b.tuning()
    assert ms > 0 and t["tile"] in (0, 1, 2) and t["elements_per_item"] in (4, 16, 64) and t["blocks_per_sm"] >= 1
    wd2 = torch.from_numpy(w0).cuda()
    b.step(wd2, 0.2)
    b.check()
    got = wd2.cpu().numpy()
    dts = b.dt()
    for i, (p, m, ic) in enumerate(probs):
        cfg = orc.Config(dim=2, p=p, nu=(32, 32))
        om = orc.Mesh(m.nbr, m.h, m.bc)
        wi = np.ascontiguousarray(b.state_view(w0, i))
        ref = _oracle_step(orc, cfg, om, wi, dts[i])
        err = state_error(b.state_view(got, i), ref).max(axis=(0, 2))
        allowed = np.maximum(TOL_FP32, 10 * step_sensitivity(orc, cfg, om, wi, dts[i], ref))
        assert np.all(err <= allowed), (i, int(np.argmax(err / allowed)), err.max())
    assert b.launch_count() > 0


def test_batch_rejects_bad_input():
    from paper_2407_20966_gb300 import kbl
    m = inputs.mesh_2d(2, 2, 0, 1, 0, 1, periodic=(True, True))
    with pytest.raises(kbl.KblError):
        kbl.Batch([(5, m.nbr, m.h, np.zeros((0, 4)))])          # order out of range
    bad = m.nbr.copy()
    bad[0, 0] = 7
    with pytest.raises(kbl.KblError):
        kbl.Batch([(2, bad, m.h, np.zeros((0, 4)))])             # neighbour out of range


@pytest.mark.parametrize("flux", [1, 2])
def test_batch_hllc_equals_single_mesh_path(flux):
    """With the HLLC (flux = 1) or HLL (flux = 2) flux each problem's batched step equals the
    single-mesh step."""
    import torch
    from paper_2407_20966_gb300 import kbl
    probs = inputs.four_quadrant_batch(9, 5, n_range=(2, 6))
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs], flux=flux)
    w0 = inputs.batch_state(probs, b.nodes, b.state_offsets)
    wd = torch.from_numpy(w0).cuda()
    b.step(wd, 0.05)
    b.check()
    got = wd.cpu().numpy()
    for i, (p, m, ic) in enumerate(probs):
        ctx = kbl.Context(dim=2, p=p, nu=(32, 32), precision=kbl.FP32_MIXED, flux=flux)
        ctx.set_tuning(kbl.TUNE_RHS_TC, 0)   # the batch runs the CUDA-core residual
        ctx.set_tuning(kbl.TUNE_BOUNDS_TILE, b.tuning()["tile"])   # and its bounds thread tile
        ctx.mesh_upload(m.nbr, m.h, m.bc)
        wi = torch.from_numpy(np.ascontiguousarray(b.state_view(w0, i))).cuda()
        ctx.set_time(0.0)
        ctx.step(wi, 0.05)
        np.testing.assert_array_equal(b.state_view(got, i), wi.cpu().numpy())


def test_batch_run_host_matches_device_steps():
    """kbl_batch_run_host (host buffers; the problems in groups whose copies overlap the steps of
    other groups) gives exactly the state of kbl_batch_step on device data: every element is
    computed by the same device code whichever work item or group holds it."""
    import torch
    b, probs, w0 = _batch(seed=13, n_problems=19, n_range=(2, 10))
    wd = torch.from_numpy(w0).cuda()
    for _ in range(2):
        b.step(wd, 0.1)
    b.check()
    ref = wd.cpu().numpy()
    w_in = torch.from_numpy(w0).pin_memory()
    w_out = torch.empty_like(w_in).pin_memory()
    b.run_host(w_in.numpy(), w_out.numpy(), 2, 0.1)
    b.check()
    np.testing.assert_array_equal(w_out.numpy(), ref)
    w_inout = w0.copy()   # the output may alias the input
    b.run_host(w_inout, w_inout, 2, 0.1)
    np.testing.assert_array_equal(w_inout, ref)


@pytest.mark.parametrize("flux", [0, 1])
def test_batch_one_launch_equals_per_phase_launches(flux):
    """The fused form (the whole step as one persistent launch, per-problem dataflow between the
    13 phases) gives bit for bit the state and time steps of one persistent launch per phase:
    every element runs the same device code whichever block takes its work item."""
    import torch
    from paper_2407_20966_gb300 import kbl
    probs = inputs.four_quadrant_batch(31 + flux, 23, n_range=(2, 14))
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs], flux=flux)
    w0 = inputs.batch_state(probs, b.nodes, b.state_offsets)
    out = []
    for form in (1, 0):
        b.set_form(form)
        wd = torch.from_numpy(w0).cuda()
        for _ in range(2):
            b.step(wd, 0.1)
        b.check()
        out.append((wd.cpu().numpy(), b.dt()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert b.launch_count() > 0


def test_batch_one_launch_wait_timeout_is_reported():
    """Failure detection without a fault: a wait of the fused step is made to run out (it waits
    for a completion count no item reaches); the step ends with KBL_ETIMEOUT instead of hanging,
    and the batch then steps correctly again."""
    import time
    import torch
    from paper_2407_20966_gb300 import kbl
    probs = inputs.four_quadrant_batch(41, 9, n_range=(2, 8))
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs])
    b.set_form(1)
    w0 = inputs.batch_state(probs, b.nodes, b.state_offsets)
    wref = torch.from_numpy(w0).cuda()
    b.step(wref, 0.1)
    b.check()
    b.stall_test(1, wait_polls=200000)      # about 0.2 s
    wd = torch.from_numpy(w0).cuda()
    t0 = time.perf_counter()
    b.step(wd, 0.1)
    with pytest.raises(kbl.KblError) as ei:
        b.check()
    assert ei.value.status == kbl.ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    b.stall_test(0)
    wd = torch.from_numpy(w0).cuda()
    b.step(wd, 0.1)
    b.check()
    np.testing.assert_array_equal(wd.cpu().numpy(), wref.cpu().numpy())
