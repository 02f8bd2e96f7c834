"""GPU tests of the batched form (kbl_batch_*): many independent four-quadrant problems with
uneven sizes and orders in persistent launches.  Each problem's step must equal the
single-mesh FP32-mixed path on the same problem (same device code), and match the FP64
checker within the FP32 tolerance."""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import TOL_FP32, state_error

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
        ctx.mesh_upload(m.nbr, m.h, m.bc)
        wi = torch.from_numpy(np.ascontiguousarray(b.state_view(w0, i))).cuda()
        ctx.set_time(0.0)
        ctx.step(wi, 0.2)
        assert ctx.time() == dts[i]
        np.testing.assert_array_equal(b.state_view(got, i), wi.cpu().numpy())


def _oracle_step(orc, cfg, om, w, dt, pert=0.0, seed=0):
    """One SSP-RK3 step of the checker; with pert > 0 its bounds are multiplied by
    (1 + pert U[-1, 1]) at every stage, which measures how strongly the limiter's
    factor (Eq. 37) amplifies a bound error of that size on this input."""
    rng = np.random.default_rng(seed)
    ws = w
    for s in range(3):
        wf = orc.traces(cfg, om, ws)
        bnd = orc.bounds(cfg, om, ws, wf)
        if pert:
            bnd = bnd * (1 + pert * rng.uniform(-1, 1, bnd.shape))
        comb = orc.stage_combine(cfg, om, s, w, ws, orc.rhs(cfg, om, ws, wf), dt)
        ws, _ = orc.limit(cfg, om, comb, bnd)
    return ws


def test_batch_matches_fp64_checker(orc):
    """Full steps of discontinuous problems: heavily limited elements amplify any bound error by
    |b| / |b - mean| (the conditioning of alpha in Eq. 37), so the criterion is per element:
    error <= max(1e-5, 10 x the checker's own change under a 1e-6 bound perturbation, the size of
    the FP32 bound error).  Per-stage parity on identical inputs is tested in test_gpu_parity."""
    import torch
    b, probs, w0 = _batch(seed=5, n_problems=6, n_range=(2, 6))
    wd = torch.from_numpy(w0).cuda()
    b.step(wd, 0.2)
    got = wd.cpu().numpy()
    for i, (p, m, ic) in enumerate(probs):
        cfg = orc.Config(dim=2, p=p, nu=(32, 32))
        om = orc.Mesh(m.nbr, m.h, m.bc)
        wi = np.ascontiguousarray(b.state_view(w0, i))
        xi, _ = orc.gauss_legendre(p + 1)
        np.testing.assert_allclose(b.nodes(p), xi, atol=2e-15)
        dt = orc.dt(cfg, om, wi, 0.2)
        ref = _oracle_step(orc, cfg, om, wi, dt)
        sens = state_error(_oracle_step(orc, cfg, om, wi, dt, pert=1e-6, seed=i), ref).max(axis=(0, 2))
        err = state_error(b.state_view(got, i), ref).max(axis=(0, 2))
        assert np.all(err <= np.maximum(TOL_FP32, 10 * sens)), (i, err.max(), sens[np.argmax(err)])


def test_batch_autotune_keeps_results(orc):
    """The autotuner changes the launch shape only: the state after a step differs by the FP32
    summation order of the bounds, which the limiter amplifies where it cuts deep (Eq. 37), so
    the criterion per element is that of test_batch_matches_fp64_checker."""
    import torch
    b, probs, w0 = _batch(seed=7, n_problems=9, n_range=(4, 12))
    wd = torch.from_numpy(w0).cuda()
    b.step(wd, 0.2)
    first = wd.cpu().numpy()
    ms, cmp = b.autotune(torch.from_numpy(w0).cuda(), with_cmp=True)
    assert cmp > 0
    t = b.tuning()
    assert ms > 0 and t["tile"] in (0, 1) and t["elements_per_item"] in (4, 16, 64) and t["blocks_per_sm"] >= 1
    wd2 = torch.from_numpy(w0).cuda()
    b.step(wd2, 0.2)
    b.check()
    # a different thread tile only changes the FP32 summation order of the bounds
    got = wd2.cpu().numpy()
    dts = b.dt()
    for i, (p, m, ic) in enumerate(probs):
        cfg = orc.Config(dim=2, p=p, nu=(32, 32))
        om = orc.Mesh(m.nbr, m.h, m.bc)
        wi = np.ascontiguousarray(b.state_view(w0, i))
        ref = _oracle_step(orc, cfg, om, wi, dts[i])
        sens = state_error(_oracle_step(orc, cfg, om, wi, dts[i], pert=1e-6, seed=i), ref).max(axis=(0, 2))
        err = state_error(b.state_view(got, i), b.state_view(first, i)).max(axis=(0, 2))
        assert np.all(err <= np.maximum(TOL_FP32, 10 * sens)), (i, err.max(), sens[np.argmax(err)])
    launches = b.launch_count()
    assert launches > 0


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
        ctx.mesh_upload(m.nbr, m.h, m.bc)
        wi = torch.from_numpy(np.ascontiguousarray(b.state_view(w0, i))).cuda()
        ctx.set_time(0.0)
        ctx.step(wi, 0.05)
        np.testing.assert_array_equal(b.state_view(got, i), wi.cpu().numpy())
