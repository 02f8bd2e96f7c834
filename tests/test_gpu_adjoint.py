"""GPU tests of the hand-written reverse mode (kbl_*_vjp, kbl_adjoint_step,
kbl_adjoint_segment and the torch.autograd wrappers).

Each vector-Jacobian product is checked against central finite differences of the
matching FP64 forward kernel in random directions: <ybar, (f(x + h v) - f(x - h v)) / 2h>
must equal <J^T ybar, v>.  The full gradient of the integrated entropy through limited
SSP-RK3 steps of the shock-vortex problem (16 x 16 P3 cut-down) is checked the same way
against the device forward pass, and against the FP64 CPU checker's forward pass (the
FP64 reference gradient, evaluated in random directions).
"""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import to_dev, zeros_dev

pytestmark = pytest.mark.gpu

FD_TOL = 1e-6      # |fd - ad| / sum |ad terms| for one smooth VJP
FD_TOL_STEP = 1e-5 # through whole limited steps


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _ctx(mesh, p, nu=16, **kw):
    from paper_2407_20966_gb300 import kbl
    ctx = kbl.Context(dim=2, p=p, nu=(nu, nu), precision=kbl.FP64, **kw)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    return ctx


def _field(orc, p, n=(5, 4), seed=0, kind="smooth", periodic=True):
    rng = np.random.default_rng(seed)
    mesh = inputs.mesh_2d(*n, 0.0, 1.0, 0.0, 1.3, periodic=(periodic, periodic),
                          bc_of_face=lambda ix, iy, f: f % 2)
    mesh.bc = inputs.random_states(rng, 2, 2)
    xi, _ = orc.gauss_legendre(p + 1)
    gen = inputs.random_smooth_field if kind == "smooth" else inputs.random_discontinuous_field
    return mesh, gen(rng, mesh, xi), rng


def _dir(rng, x, rel=1.0):
    """Random direction scaled per component by the component's magnitude."""
    scale = np.abs(x).reshape(x.shape[0], -1).max(axis=1)
    return rel * rng.standard_normal(x.shape) * scale.reshape((-1,) + (1,) * (x.ndim - 1))


def _check(fd, ad_terms, tol):
    ad = sum(float(t.sum()) for t in ad_terms)
    mag = sum(float(np.abs(t).sum()) for t in ad_terms)
    assert abs(fd - ad) <= tol * mag, (fd, ad, mag)
    return abs(fd - ad) / mag


def test_traces_vjp_is_the_transpose(orc):
    for periodic in (True, False):
        mesh, w, rng = _field(orc, 3, periodic=periodic)
        ctx = _ctx(mesh, 3)
        wf = zeros_dev(4, mesh.n_elem, ctx.nfp)
        ctx.traces(to_dev(w), wf)
        a, b = rng.standard_normal(wf.shape), rng.standard_normal(wf.shape)
        wb = zeros_dev(*w.shape)
        ctx.traces_vjp(to_dev(a), to_dev(b), wb)
        lhs = float(((a + b) * wf.cpu().numpy()).sum())
        rhs = float((wb.cpu().numpy() * w).sum())
        assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("p,periodic", [(3, True), (2, False), (4, True)])
def test_rhs_vjp_matches_fd(orc, p, periodic):
    mesh, w, rng = _field(orc, p, seed=p, periodic=periodic)
    ctx = _ctx(mesh, p)
    E, ns, nfp = mesh.n_elem, ctx.ns, ctx.nfp
    wd = to_dev(w)
    wf = zeros_dev(4, E, nfp)
    ctx.traces(wd, wf)
    wf0 = wf.cpu().numpy()
    Rb = rng.standard_normal(w.shape)
    wb, wfb, wfbx = zeros_dev(*w.shape), zeros_dev(4, E, nfp), zeros_dev(4, E, nfp)
    ctx.rhs_vjp(wd, wf, to_dev(Rb), wb, wfb, wfbx)
    vw, vf = _dir(rng, w), _dir(rng, wf0)
    h = 1e-6

    def R(x, xf):
        out = zeros_dev(4, E, ns)
        ctx.rhs(to_dev(x), to_dev(xf), out)
        return out.cpu().numpy()
    fd = float((Rb * (R(w + h * vw, wf0 + h * vf) - R(w - h * vw, wf0 - h * vf))).sum()) / (2 * h)
    _check(fd, [wb.cpu().numpy() * vw, (wfb.cpu().numpy() + wfbx.cpu().numpy()) * vf], FD_TOL)


@pytest.mark.parametrize("p,nu,kind", [(3, 16, "smooth"), (2, 32, "disc"), (1, 8, "disc"), (3, 64, "smooth")])
def test_bounds_vjp_matches_fd(orc, p, nu, kind):
    mesh, w, rng = _field(orc, p, seed=10 + p, kind=kind)
    ctx = _ctx(mesh, p, nu=nu)
    E, nfp = mesh.n_elem, ctx.nfp
    wd = to_dev(w)
    wf = zeros_dev(4, E, nfp)
    ctx.traces(wd, wf)
    wf0 = wf.cpu().numpy()
    bnd = zeros_dev(2, 4, E)
    ctx.bounds(wd, wf, bnd)
    bb = rng.standard_normal((2, 4, E))
    wb, wfb, wfbx = zeros_dev(*w.shape), zeros_dev(4, E, nfp), zeros_dev(4, E, nfp)
    ctx.bounds_vjp(wd, wf, bnd, to_dev(bb), wb, wfb, wfbx)
    ctx.check()
    vw, vf = _dir(rng, w), _dir(rng, wf0)
    h = 1e-7

    def B(x, xf):
        out = zeros_dev(2, 4, E)
        ctx.bounds(to_dev(x), to_dev(xf), out)
        return out.cpu().numpy()
    fd = float((bb * (B(w + h * vw, wf0 + h * vf) - B(w - h * vw, wf0 - h * vf))).sum()) / (2 * h)
    err = _check(fd, [wb.cpu().numpy() * vw, (wfb.cpu().numpy() + wfbx.cpu().numpy()) * vf], FD_TOL)
    print(f"bounds VJP p={p} nu={nu} {kind}: relative FD mismatch {err:.2e}")


def test_bounds_vjp_single_state_stencil(orc):
    """One state everywhere: the bounds are that state times (1 -+ r) up to quadrature error, so
    d(rho_hi)/d(rho) through the winning node must be close to 1 + r in total."""
    mesh = inputs.mesh_2d(3, 3, 0.0, 1.0, 0.0, 1.0, periodic=(True, True))
    q = inputs.conservative(1.3, [0.2, -0.1], 0.9)
    p = 2
    ctx = _ctx(mesh, p, nu=32)
    w = np.broadcast_to(q[:, None, None], (4, mesh.n_elem, ctx.ns)).copy()
    wd = to_dev(w)
    wf = zeros_dev(4, mesh.n_elem, ctx.nfp)
    ctx.traces(wd, wf)
    bnd = zeros_dev(2, 4, mesh.n_elem)
    ctx.bounds(wd, wf, bnd)
    bb = np.zeros((2, 4, mesh.n_elem))
    bb[1, 0, 4] = 1.0                       # d(rho_max of element 4)
    wb, wfb, wfbx = zeros_dev(*w.shape), zeros_dev(4, mesh.n_elem, ctx.nfp), zeros_dev(4, mesh.n_elem, ctx.nfp)
    ctx.bounds_vjp(wd, wf, bnd, to_dev(bb), wb, wfb, wfbx)
    tot = wb.cpu().numpy().sum(axis=(1, 2)) + wfb.cpu().numpy().sum(axis=(1, 2)) + wfbx.cpu().numpy().sum(axis=(1, 2))
    # moving every stencil state together by d rho moves rho_max by (1 + r) d rho (to quadrature error)
    assert tot[0] == pytest.approx(1.0 + 1e-3, rel=2e-3)


@pytest.mark.parametrize("stage", [0, 1, 2])
@pytest.mark.parametrize("case", ["tight", "pressure", "uncoupled"])
def test_stage_vjp_matches_fd(orc, stage, case):
    """Stage + limiter.  'tight': the kinetic bounds narrowed by a quarter of their width on both
    sides, so that Eq. 37 limits most elements; 'pressure': the bounds as computed and a
    pressure floor of 0.5, so that Eq. 48-49 re-limit elements; 'uncoupled': as 'tight' with each
    component limited by its own factor."""
    from paper_2407_20966_gb300 import kbl
    p = 3
    p_floor = 0.5 if case == "pressure" else 1e-12
    mesh, w, rng = _field(orc, p, n=(6, 5), seed=20 + stage, kind="disc")
    ctx = _ctx(mesh, p, nu=16, eps_rule=1, p_floor=p_floor, uncoupled=int(case == "uncoupled"))
    E, ns, nfp = mesh.n_elem, ctx.ns, ctx.nfp
    wd = to_dev(w)
    wf = zeros_dev(4, E, nfp)
    ctx.traces(wd, wf)
    bnd = zeros_dev(2, 4, E)
    ctx.bounds(wd, wf, bnd)
    R = zeros_dev(4, E, ns)
    ctx.rhs(wd, wf, R)
    bnd0, R0 = bnd.cpu().numpy(), R.cpu().numpy()
    if case in ("tight", "uncoupled"):
        width = bnd0[1] - bnd0[0]
        bnd0 = np.stack([bnd0[0] + 0.25 * width, bnd0[1] - 0.25 * width])
    bnd = to_dev(bnd0)
    wn = w * (1 + 0.01 * rng.standard_normal(w.shape))
    dt = 2e-3
    dtd = torch_scalar(dt)
    out = zeros_dev(4, E, ns)
    ctx.counters()
    ctx.stage(stage, to_dev(wn), wd, R, bnd, dtd, out)
    st, c = ctx.counters()
    assert st == kbl.OK
    assert (c["pressure_relimits"] if case == "pressure" else c["limited_elements"]) > 0
    ob = rng.standard_normal(w.shape)
    wnb, wsb, Rb, bndb = zeros_dev(*w.shape), zeros_dev(*w.shape), zeros_dev(*w.shape), zeros_dev(2, 4, E)
    ctx.stage_vjp(stage, dt, to_dev(wn), wd, R, bnd, to_dev(ob), wnb, wsb, Rb, bndb)
    vn, vs, vR, vb = _dir(rng, wn), _dir(rng, w), _dir(rng, R0), _dir(rng, bnd0.reshape(8, E)).reshape(2, 4, E)
    h = 1e-7

    def F(sgn):
        o = zeros_dev(4, E, ns)
        ctx.stage(stage, to_dev(wn + sgn * h * vn), to_dev(w + sgn * h * vs), to_dev(R0 + sgn * h * vR),
                  to_dev(bnd0 + sgn * h * vb), dtd, o)
        return o.cpu().numpy()
    fd = float((ob * (F(1) - F(-1))).sum()) / (2 * h)
    terms = [wnb.cpu().numpy() * vn, wsb.cpu().numpy() * vs, Rb.cpu().numpy() * vR, bndb.cpu().numpy() * vb]
    err = _check(fd, terms, FD_TOL)
    print(f"stage VJP s={stage} {case}: limited {c['limited_elements']} relimits "
          f"{c['pressure_relimits']} relative FD mismatch {err:.2e}")
    # the stage-0 combination does not use wn
    if stage == 0:
        assert not wnb.cpu().numpy().any()


def torch_scalar(v):
    import torch
    return torch.tensor([v], dtype=torch.float64, device="cuda")


def test_entropy_vjp_matches_fd(orc):
    mesh, w, rng = _field(orc, 3, seed=3)
    ctx = _ctx(mesh, 3)
    J = zeros_dev(1)

    def f(x):
        ctx.entropy(to_dev(x), J)
        return float(J.item())
    wb = zeros_dev(*w.shape)
    ctx.entropy_vjp(to_dev(w), 0.7, wb)
    v = _dir(rng, w)
    h = 1e-6
    fd = 0.7 * (f(w + h * v) - f(w - h * v)) / (2 * h)
    _check(fd, [wb.cpu().numpy() * v], 1e-8)
    # the value itself: sum |J_e| W rho ln(P rho^-gamma) written out on the host
    xi, wq = orc.gauss_legendre(4)
    W = np.outer(wq, wq).ravel()
    P = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
    ref = float((0.25 * mesh.h[:, 0:1] * mesh.h[:, 1:2] * W[None] * w[0] * np.log(P * w[0] ** -1.4)).sum())
    assert f(w) == pytest.approx(ref, rel=1e-13)


# ---------------------------------------------------------------------------
# whole steps: the shock-vortex problem, 16 x 16 P3 cut-down
#
# The uniform regions of the set-up hold exactly equal states, where every min / max
# of the method is a tie: there the adjoint returns the subgradient of its tie rule while
# central differences average the one-sided derivatives.  The checks therefore start
# from the set-up times (1 + 1e-4 N(0, 1)) per node (seeded), a point where the method
# is differentiable.  CFL 0.05: with the per-axis time-step rule and the 2:1 elements of
# this domain, SSP-RK3 with P3 FR is linearly stable there; near CFL 0.1 it is not, which
# the limiter hides in the state but the tangent and adjoint show as growth of about 2x
# per step.
# ---------------------------------------------------------------------------
CFL_2D = 0.05


def _shock_vortex(n=16, p=3, nu=32, noise=1e-4):
    from paper_2407_20966_gb300 import kbl
    mesh, ic = inputs.shock_vortex(n)
    ctx = kbl.Context(dim=2, p=p, nu=(nu, nu), precision=kbl.FP64, eps_rule=1)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
    w0 = inputs.nodal_field(mesh, ctx.operator(kbl.OP_NODES), ic)
    if noise:
        w0 = w0 * (1 + noise * np.random.default_rng(0).standard_normal(w0.shape))
    return ctx, mesh, w0


def _J_device(ctx, w0, dts):
    w = to_dev(w0)
    for dt in dts:
        ctx.step_fixed(w, dt)
    J = zeros_dev(1)
    ctx.entropy(w, J)
    return float(J.item())


def _grad_device(ctx, w0, dts, every, keep_bounds=True):
    from paper_2407_20966_gb300 import adjoint
    x = to_dev(w0).requires_grad_(True)
    J = adjoint.entropy(adjoint.trajectory(x, ctx, dts, checkpoint_every=every, keep_bounds=keep_bounds), ctx)
    J.backward()
    ctx.check()
    return float(J.detach().item()), x.grad.cpu().numpy()


def _fd_check(ctx, w0, dts, g, seed, h, tol, label):
    rng = np.random.default_rng(seed)
    v = _dir(rng, w0)
    fd = (_J_device(ctx, w0 + h * v, dts) - _J_device(ctx, w0 - h * v, dts)) / (2 * h)
    err = _check(fd, [g * v], tol)
    print(f"{label}: relative FD mismatch {err:.2e}")


def test_adjoint_step_matches_fd_shock_vortex(orc):
    from paper_2407_20966_gb300 import adjoint
    ctx, mesh, w0 = _shock_vortex()
    dts = adjoint.cfl_time_steps(ctx, to_dev(w0), 1, CFL_2D)
    wd = to_dev(w0)
    w1 = wd.clone()
    ctx.step_fixed(w1, dts[0])
    g = zeros_dev(*w0.shape)
    ctx.entropy_vjp(w1, 1.0, g)
    ctx.adjoint_step(wd, dts[0], g)
    for k in range(3):
        _fd_check(ctx, w0, dts, g.cpu().numpy(), k, 1e-7, FD_TOL, f"one step, direction {k}")


def test_trajectory_gradient_checkpointing_and_fd(orc):
    """20 limited steps: checkpoints every 5 steps give bit for bit the gradient of one
    20-step segment, and so does recomputing the stage bounds instead of keeping them;
    central differences of the device forward pass agree."""
    from paper_2407_20966_gb300 import adjoint
    ctx, mesh, w0 = _shock_vortex()
    dts = adjoint.cfl_time_steps(ctx, to_dev(w0), 20, CFL_2D)
    ctx.counters()
    J, g5 = _grad_device(ctx, w0, dts, 5)
    _, g20 = _grad_device(ctx, w0, dts, 20)
    _, g5r = _grad_device(ctx, w0, dts, 5, keep_bounds=False)
    np.testing.assert_array_equal(g5, g20)
    np.testing.assert_array_equal(g5, g5r)
    assert J == _J_device(ctx, w0, dts)
    for k in range(2):
        _fd_check(ctx, w0, dts, g5, 10 + k, 1e-8, FD_TOL, f"20 steps, direction {k}")


def test_gradient_100_steps_checkpointed_vs_fd(orc):
    """The adjoint workload's shape on the cut-down mesh: the entropy at t_end through 100
    SSP-RK3 steps with the limiter active, checkpoints every 10 steps, against central
    differences of the device forward pass."""
    from paper_2407_20966_gb300 import adjoint
    ctx, mesh, w0 = _shock_vortex()
    dts = adjoint.cfl_time_steps(ctx, to_dev(w0), 100, CFL_2D)
    ctx.counters()
    _J_device(ctx, w0, dts)
    st, c = ctx.counters()
    assert c["limited_elements"] > 0
    J, g = _grad_device(ctx, w0, dts, 10)
    _fd_check(ctx, w0, dts, g, 20, 1e-8, FD_TOL, f"100 steps ({c['limited_elements']} limited element-stages)")


def test_gradient_vs_fp64_checker_forward(orc):
    """FP64 reference gradient: central differences of the CPU checker's forward pass (its own
    SSP-RK3 steps with the same time steps and its own entropy sum) in random directions."""
    from paper_2407_20966_gb300 import adjoint
    ctx, mesh, w0 = _shock_vortex()
    n_steps = 4
    dts = adjoint.cfl_time_steps(ctx, to_dev(w0), n_steps, CFL_2D)
    _, g = _grad_device(ctx, w0, dts, 2)
    cfg = orc.Config(dim=2, p=3, nu=(32, 32), eps_rule=1)
    om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
    xi, wq = orc.gauss_legendre(4)
    W = np.outer(wq, wq).ravel()[None] * (0.25 * mesh.h[:, 0:1] * mesh.h[:, 1:2])

    def J_ref(x):
        for dt in dts:
            x, _ = orc.ssprk3_step(cfg, om, x, dt)
        P = 0.4 * (x[3] - 0.5 * (x[1] ** 2 + x[2] ** 2) / x[0])
        return float((W * x[0] * np.log(P * x[0] ** -1.4)).sum())
    rng = np.random.default_rng(4)
    for k in range(2):
        v = _dir(rng, w0)
        h = 1e-7
        fd = (J_ref(w0 + h * v) - J_ref(w0 - h * v)) / (2 * h)
        err = _check(fd, [g * v], FD_TOL)
        print(f"{n_steps} steps vs checker forward, direction {k}: relative FD mismatch {err:.2e}")


def test_exact_ties_take_the_documented_subgradient(orc):
    """From the set-up itself (exact ties in the uniform regions) the gradient is the tie rule's
    subgradient: close to, but not equal to, the central difference (which averages the one-sided
    derivatives).  Recorded, with a loose bound."""
    from paper_2407_20966_gb300 import adjoint
    ctx, mesh, w0 = _shock_vortex(noise=0.0)
    dts = adjoint.cfl_time_steps(ctx, to_dev(w0), 20, CFL_2D)
    _, g = _grad_device(ctx, w0, dts, 10)
    _fd_check(ctx, w0, dts, g, 30, 1e-7, 1e-3, "20 steps from the exact set-up (ties)")


def test_adjoint_rejects_bad_input():
    from paper_2407_20966_gb300 import kbl
    mesh = inputs.mesh_1d(4, 0.0, 1.0, periodic=True)
    ctx = kbl.Context(dim=1, p=2)
    ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc[:, :3])
    w = zeros_dev(3, 4, 3)
    with pytest.raises(kbl.KblError):
        ctx.adjoint_step(w, 0.1, zeros_dev(3, 4, 3))      # the adjoint is 2D only
    ctx64, m2, w0 = _shock_vortex(n=4, p=2, nu=8)
    ctx32 = kbl.Context(dim=2, p=2, nu=(8, 8), precision=kbl.FP32_MIXED)
    ctx32.mesh_upload(m2.nbr, m2.h, m2.bc)
    with pytest.raises(kbl.KblError):
        ctx32.adjoint_step(to_dev(w0), 0.1, to_dev(w0))   # FP64 only
    with pytest.raises(kbl.KblError):
        ctx64.adjoint_segment(to_dev(w0), [0.1, -1.0], to_dev(w0))
    ctxh = kbl.Context(dim=2, p=2, nu=(8, 8), precision=kbl.FP64, flux=1)
    ctxh.mesh_upload(m2.nbr, m2.h, m2.bc)
    with pytest.raises(kbl.KblError):
        ctxh.adjoint_step(to_dev(w0), 0.1, to_dev(w0))   # the residual adjoint covers Rusanov
