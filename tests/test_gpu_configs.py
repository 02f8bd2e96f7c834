"""GPU checks at the benchmark workloads' full sizes, in the launch configuration bench.py times.

The checker computes sampled elements one by one (gathering each stencil from its own traces).
* vortex, 128^2 P3, 32^2 grid: FP32 bound error per moment; no clipping of the smooth flow
* Sedov-type blast, 512^2 P2: sampled FP64 / FP32 bounds; positivity and conservation under
  many limited steps (the extreme-ratio stress)
* Sod, 200 P3, 64 points: the full run to t = 0.2 (Sec. 6.1) against the checker and the exact
  Riemann solution
"""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import TOL_FP32, TOL_FP64, bounds_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _sampled_bounds(orc, ctx, cfg, mesh, w, n_sample=160, seed=0):
    import torch
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    wf = orc.traces(cfg, om, w)
    bnd = torch.zeros((2, cfg.nv, mesh.n_elem), dtype=torch.float64, device="cuda")
    ctx.bounds(torch.from_numpy(w).cuda(), torch.from_numpy(wf).cuda(), bnd)
    ctx.check()
    got = bnd.cpu().numpy()
    idx = np.random.default_rng(seed).choice(mesh.n_elem, n_sample, replace=False)
    ref = np.zeros((2, cfg.nv, n_sample))
    for k, e in enumerate(idx):
        lo, hi = orc.bounds_stencil(cfg, orc.gather_stencil(cfg, om, w, wf, int(e)))
        ref[0, :, k], ref[1, :, k] = lo, hi
    return bounds_error(got[:, :, idx], ref)


def test_vortex_fp32_bound_error_per_moment(orc):
    from paper_2407_20966_gb300 import kbl
    mesh, ic = inputs.isentropic_vortex(128)
    ctx = kbl.Context(dim=2, p=3, nu=(32, 32), precision=kbl.FP32_MIXED)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    w = inputs.nodal_field(mesh, ctx.operator(kbl.OP_NODES), ic)
    cfg = orc.Config(dim=2, p=3, nu=(32, 32))
    err = _sampled_bounds(orc, ctx, cfg, mesh, w)
    per_moment = {name: float(err[:, k].max()) for k, name in enumerate(("rho", "m_x", "m_y", "E"))}
    print("vortex FP32 bound error per moment (max over lower/upper, 160 sampled elements):", per_moment)
    assert max(per_moment.values()) < TOL_FP32


def test_vortex_smooth_flow_is_not_clipped(orc):
    """Sec. 6.2's claim in 2D: in a smooth flow the kinetic bounds leave the solution alone."""
    import torch
    from paper_2407_20966_gb300 import kbl
    mesh, ic = inputs.isentropic_vortex(128)
    ctx = kbl.Context(dim=2, p=3, nu=(32, 32), precision=kbl.FP32_MIXED)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    wd = torch.from_numpy(inputs.nodal_field(mesh, ctx.operator(kbl.OP_NODES), ic)).cuda()
    ctx.set_time(0.0)
    ctx.counters()
    for _ in range(5):
        ctx.step(wd, 0.05)
    st, c = ctx.counters()
    print("vortex, 5 steps at CFL 0.05: limited element-stages", c["limited_elements"], "of", 15 * mesh.n_elem)
    assert st == kbl.OK
    assert c["limited_elements"] == 0


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_FP32)])
def test_sedov_sampled_bounds(orc, precision, tol):
    from paper_2407_20966_gb300 import kbl
    mesh, ic = inputs.sedov(512)
    ctx = kbl.Context(dim=2, p=2, nu=(32, 32), precision=precision)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    xi = ctx.operator(kbl.OP_NODES)
    w = inputs.nodal_field(mesh, xi, ic)
    # sample around the blast as well as in the ambient gas
    cfg = orc.Config(dim=2, p=2, nu=(32, 32))
    err = _sampled_bounds(orc, ctx, cfg, mesh, w, n_sample=96, seed=precision)
    assert err.max() < tol
    centre = [255 * 512 + 255, 256 * 512 + 256, 255 * 512 + 257, 254 * 512 + 256]
    import torch
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    wf = orc.traces(cfg, om, w)
    bnd = torch.zeros((2, 4, mesh.n_elem), dtype=torch.float64, device="cuda")
    ctx.bounds(torch.from_numpy(w).cuda(), torch.from_numpy(wf).cuda(), bnd)
    got = bnd.cpu().numpy()[:, :, centre]
    ref = np.zeros_like(got)
    for k, e in enumerate(centre):
        ref[0, :, k], ref[1, :, k] = orc.bounds_stencil(cfg, orc.gather_stencil(cfg, om, w, wf, e))
    assert bounds_error(got, ref).max() < tol


@pytest.mark.parametrize("flux", [0, 2])
@pytest.mark.parametrize("precision,cons_tol", [(1, 1e-7), (0, 1e-12)])
def test_sedov_positivity_and_conservation_under_limiting(precision, cons_tol, flux):
    """Extreme pressure ratio (4.5e3 / 1e-6): 40 steps stay physical, the pressure stays above the
    floor at every solution point, and mass and energy are conserved (the blast has not reached
    the boundary).  The limiter keeps element means exactly; the FP32-mixed residual conserves to
    FP32 rounding of its volume terms, the FP64 path to FP64 rounding.  Rusanov, and HLL, the
    flux of the paper's own Sedov run (Sec. 6.6)."""
    import torch
    from paper_2407_20966_gb300 import kbl
    mesh, ic = inputs.sedov(512)
    ctx = kbl.Context(dim=2, p=2, nu=(32, 32), precision=precision, flux=flux)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    xi = ctx.operator(kbl.OP_NODES)
    wq = ctx.operator(kbl.OP_WEIGHTS)
    w = inputs.nodal_field(mesh, xi, ic)
    W = np.outer(wq, wq).ravel() * (mesh.h[0, 0] * mesh.h[0, 1] / 4)
    mass0, energy0 = (w[0] * W).sum(), (w[3] * W).sum()
    wd = torch.from_numpy(w).cuda()
    ctx.set_time(0.0)
    ctx.counters()
    for _ in range(40):
        ctx.step(wd, 0.05)
    st, c = ctx.counters()
    assert st == kbl.OK and c["nonphysical"] == 0
    assert c["limited_elements"] > 0
    w1 = wd.cpu().numpy()
    P = 0.4 * (w1[3] - 0.5 * (w1[1] ** 2 + w1[2] ** 2) / w1[0])
    assert w1[0].min() > 0 and P.min() >= 1e-12 * (1 - 1e-9)
    assert (w1[0] * W).sum() == pytest.approx(mass0, rel=cons_tol)
    assert (w1[3] * W).sum() == pytest.approx(energy0, rel=cons_tol)
    print(f"Sedov 512^2 P2, 40 steps, precision {precision}, flux {flux}: limited element-stages",
          c["limited_elements"],
          "pressure re-limits", c["pressure_relimits"], "min P", P.min(),
          "mass drift", (w1[0] * W).sum() / mass0 - 1, "energy drift", (w1[3] * W).sum() / energy0 - 1)


def test_sod_full_run_matches_checker(orc):
    """The whole Sod run (Sec. 6.1 set-up, t = 0.2) on the device against the checker: the same
    number of steps, the same end state to 1e-9, and the same L1 error against the exact
    solution."""
    import torch
    from paper_2407_20966_gb300 import kbl
    from tests import riemann_exact
    mesh, ic = inputs.sod(200)
    ctx = kbl.Context(dim=1, p=3, nu=(64,), precision=kbl.FP64)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    cfg = orc.Config(dim=1, p=3, nu=(64,))
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    xi, _ = orc.gauss_legendre(4)
    w = inputs.nodal_field(mesh, xi, ic)
    ref, t, n = w.copy(), 0.0, 0
    while t < 0.2 - 1e-14:
        dt = min(orc.dt(cfg, om, ref, 0.1), 0.2 - t)
        ref, _ = orc.ssprk3_step(cfg, om, ref, dt)
        t += dt
        n += 1
    wd = torch.from_numpy(w).cuda()
    ctx.set_time(0.0, 0.2)
    for _ in range(n):
        ctx.step(wd, 0.1)
    assert ctx.time() == pytest.approx(0.2, rel=1e-12)
    got = wd.cpu().numpy()
    x = inputs.node_coords(mesh, xi)[0].ravel()
    exact = riemann_exact.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), x, 0.2)
    l1_gpu = np.abs(got[0].ravel() - exact[0]).mean()
    l1_ref = np.abs(ref[0].ravel() - exact[0]).mean()
    print(f"Sod, {n} steps: L1(rho) device {l1_gpu:.6e}, checker {l1_ref:.6e}, paper 1.181e-3 (HLLC, 2048 pts)")
    assert l1_gpu == pytest.approx(l1_ref, rel=1e-8)
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()


def _fullsize_sample(E, n_side, n_sample, seed, extra=()):
    """>= n_sample distinct elements: random ones, the first and last thread blocks of the
    FR and stage kernels (8 elements each), and the given extra elements."""
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(E, n_sample, replace=False).tolist())
    idx.update(range(0, 8))
    idx.update(range(E - 8, E))
    idx.update(int(e) for e in extra)
    return np.array(sorted(idx))


@pytest.mark.parametrize("workload", ["vortex", "sedov"])
def test_fullsize_stage_parity_identical_inputs(orc, workload):
    """The benchmark workloads at full size, in bench.py's launch configuration (FP32-mixed, one
    launch over the whole mesh per call): the three stages of a step, each on identical inputs.
    Device traces, bounds, residual and stage + limiter of the whole mesh; the checker computes
    2000+ sampled elements one by one (the first and last blocks and, for Sedov, the blast cells
    and their neighbours among them): bounds to 1e-5, residual to 1e-5 per element and component,
    the limited state to 1e-12 when both sides limit against the same bounds, and the composed
    FP32 stage (the device's own residual and bounds) to 1e-5."""
    import torch
    from paper_2407_20966_gb300 import kbl
    from tests.gpu_helpers import rhs_error, state_error
    if workload == "vortex":
        mesh, ic = inputs.isentropic_vortex(128)
        p, flux, nside = 3, 0, 128
        extra = ()
    else:
        mesh, ic = inputs.sedov(512)
        p, flux, nside = 2, 2, 512
        c = 256
        extra = [(c + dy) * nside + c + dx for dy in range(-4, 4) for dx in range(-4, 4)]
    ctx = kbl.Context(dim=2, p=p, nu=(32, 32), precision=kbl.FP32_MIXED, flux=flux)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    cfg = orc.Config(dim=2, p=p, nu=(32, 32), flux=flux)
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    w = inputs.nodal_field(mesh, ctx.operator(kbl.OP_NODES), ic)
    E = mesh.n_elem
    idx = _fullsize_sample(E, nside, 2000, seed=17, extra=extra)
    dt = orc.dt(cfg, om, w, 0.05)
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    wn, ws = w, w
    limited = 0
    for s in range(3):
        wsd = torch.from_numpy(ws).cuda()
        wf_ref = orc.traces(cfg, om, ws)
        wf = torch.zeros(wf_ref.shape, dtype=torch.float64, device="cuda")
        ctx.traces(wsd, wf)
        np.testing.assert_allclose(wf.cpu().numpy(), wf_ref, rtol=1e-14, atol=1e-14 * np.abs(wf_ref).max())
        wfd = torch.from_numpy(wf_ref).cuda()
        bnd = torch.zeros((2, 4, E), dtype=torch.float64, device="cuda")
        ctx.bounds(wsd, wfd, bnd)
        R = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
        ctx.rhs(wsd, wfd, R)
        ctx.check()
        bg, Rg = bnd.cpu().numpy(), R.cpu().numpy()
        bref = np.zeros((2, 4, len(idx)))
        for k, e in enumerate(idx):
            bref[0, :, k], bref[1, :, k] = orc.bounds_stencil(cfg, orc.gather_stencil(cfg, om, ws, wf_ref, int(e)))
        eb = bounds_error(bg[:, :, idx], bref)
        assert eb.max() < TOL_FP32, ("bounds", s, eb.max())
        R_ref = orc.rhs(cfg, om, ws, wf_ref)
        er = rhs_error(Rg, R_ref, ws, wf_ref, mesh)
        assert er.max() < TOL_FP32, ("residual", s, er.max())
        # stage + limiter: both sides limit against the device's bounds (identical inputs)
        out = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
        ctx.stage(s, torch.from_numpy(wn).cuda(), wsd, torch.from_numpy(R_ref).cuda(), bnd, dtd, out)
        # the composed FP32 stage: the device's own residual and bounds
        out2 = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
        ctx.stage(s, torch.from_numpy(wn).cuda(), wsd, R, bnd, dtd, out2)
        got, got2 = out.cpu().numpy(), out2.cpu().numpy()
        comb = orc.stage_combine(cfg, om, s, wn, ws, R_ref, dt)
        wfc = orc.traces(cfg, om, comb)
        ref = np.zeros((4, len(idx), w.shape[2]))
        ref2 = np.zeros_like(ref)
        for k, e in enumerate(idx):
            ref[:, k], a = orc.limit_element(cfg, comb[:, e], wfc[:, e], bg[0, :, e], bg[1, :, e])
            ref2[:, k], _ = orc.limit_element(cfg, comb[:, e], wfc[:, e], bref[0, :, k], bref[1, :, k])
            limited += int(a[0] < 1)
        es = state_error(got[:, idx], ref).max(axis=(0, 2))
        assert es.max() < TOL_FP64, ("stage", s, es.max())
        ec = state_error(got2[:, idx], ref2).max(axis=(0, 2))
        assert ec.max() < TOL_FP32, ("composed", s, ec.max())
        print(f"{workload} stage {s}: bounds {eb.max():.2e} residual {er.max():.2e} stage {es.max():.2e} "
              f"composed {ec.max():.2e} on {len(idx)} elements")
        ws = got
    print(f"{workload}: limited element-stages in the sample", limited)


def test_fullsize_batch_phase_parity_identical_inputs(orc):
    """The 4096-problem batch at full size (25.8 M elements, orders P1..P4), in the launch shape
    the autotuner picks and bench.py times, after two steps of the batch itself: one stage's
    bounds, residual and stage + limiter, each on identical inputs, against the checker on 16
    sampled problems of every order: bounds of 48 sampled elements per problem to 1e-5, the
    residual of the whole problem to 1e-5 per element and component, and the limited state of
    the whole problem to 1e-12 when both sides limit against the device's bounds."""
    import torch
    from paper_2407_20966_gb300 import kbl
    from tests.gpu_helpers import rhs_error, state_error
    probs = inputs.four_quadrant_batch(0x5EED, 4096)
    b = kbl.Batch([(p, m.nbr, m.h, m.bc) for p, m, _ in probs])
    E = int(b.elem_offsets[-1])
    assert E > 25_000_000
    wd = torch.from_numpy(inputs.batch_state(probs, b.nodes, b.state_offsets)).cuda()
    b.autotune(wd)
    for _ in range(2):
        b.step(wd, 0.05)
    b.check()
    dts = np.asarray(b.dt(), dtype=np.float64)
    rng = np.random.default_rng(5)
    sample = []
    for p in (1, 2, 3, 4):
        cand = np.flatnonzero(np.asarray(b.p) == p)
        sample += list(rng.choice(cand, 4, replace=False))
    bnd = torch.zeros(8 * E, dtype=torch.float64, device="cuda")
    R = torch.zeros_like(wd)
    b.bounds(wd, bnd)
    b.rhs(wd, R)
    out = torch.zeros_like(wd)
    b.stage(0, wd, wd, R, bnd, torch.from_numpy(dts).cuda(), out)
    b.check()
    limited = 0
    for i in sample:
        p, mesh, _ = probs[i]
        cfg = orc.Config(dim=2, p=p, nu=(32, 32))
        om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
        ws = np.ascontiguousarray(b.state_view(wd, i).cpu().numpy())
        wf = orc.traces(cfg, om, ws)
        bg = b.bounds_view(bnd, i).cpu().numpy()
        idx = rng.choice(mesh.n_elem, min(48, mesh.n_elem), replace=False)
        bref = np.zeros((2, 4, len(idx)))
        for k, e in enumerate(idx):
            bref[0, :, k], bref[1, :, k] = orc.bounds_stencil(cfg, orc.gather_stencil(cfg, om, ws, wf, int(e)))
        eb = bounds_error(bg[:, :, idx], bref)
        assert eb.max() < TOL_FP32, ("bounds", i, p, eb.max())
        Rg = np.ascontiguousarray(b.state_view(R, i).cpu().numpy())
        R_ref = orc.rhs(cfg, om, ws, wf)
        er = rhs_error(Rg, R_ref, ws, wf, om)
        assert er.max() < TOL_FP32, ("residual", i, p, er.max())
        comb = orc.stage_combine(cfg, om, 0, ws, ws, Rg, dts[i])
        ref, a = orc.limit(cfg, om, comb, bg)
        limited += int((a[0] < 1).sum())
        got = b.state_view(out, i).cpu().numpy()
        es = state_error(got, ref).max()
        assert es < TOL_FP64, ("stage", i, p, es)
    assert limited > 0
    print(f"batch: {len(sample)} sampled problems, limited elements {limited}")
