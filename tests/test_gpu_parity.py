"""GPU parity: every entry point of the C-ABI against the CPU checker on the same seeded inputs.

Bar: bit-exact for the stencil gather (plain index work); 1e-12 relative for FP64 bounds,
residuals and limited states; 1e-5 relative for the FP32 bounds.  Sizes span several
thread blocks with a ragged tail; edge cases: an empty mesh, a one-element periodic mesh,
a non-physical state.
"""
import numpy as np
import pytest

from tests.gpu_helpers import (TOL_FP32, TOL_FP64, both, bounds_error, mesh_and_field, rhs_error,
                               state_error, step_sensitivity, to_dev, upload, zeros_dev)

pytestmark = pytest.mark.gpu

CASES_2D = [  # (p, nu, elements per side)
    (3, 32, (13, 11)),
    (2, 32, (9, 7)),
    (1, 16, (5, 17)),
    (4, 8, (6, 5)),
    (3, 64, (3, 4)),
    (4, 32, (4, 3)),
    (5, 16, (3, 3)),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


@pytest.mark.parametrize("dim,p", [(1, 3), (2, 3), (2, 2), (2, 4)])
def test_operators_match_checker(orc, dim, p):
    from paper_2407_20966_gb300 import kbl
    ctx, _ = both(orc, dim, p, (64,) if dim == 1 else (32, 32))
    x, wq = orc.gauss_legendre(p + 1)
    np.testing.assert_allclose(ctx.operator(kbl.OP_NODES), x, rtol=0, atol=2e-15)
    np.testing.assert_allclose(ctx.operator(kbl.OP_WEIGHTS), wq, rtol=0, atol=2e-15)
    lm = [orc.lagrange(x, j, -1.0) for j in range(p + 1)]
    np.testing.assert_allclose(ctx.operator(kbl.OP_LMINUS), lm, rtol=0, atol=1e-13)
    D = [[orc.lagrange_deriv(x, m, x[i]) for m in range(p + 1)] for i in range(p + 1)]
    np.testing.assert_allclose(ctx.operator(kbl.OP_D), D, rtol=0, atol=1e-12)
    gl = [orc.correction_deriv(p, xi)[0] for xi in x]
    np.testing.assert_allclose(ctx.operator(kbl.OP_GL), gl, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim,p,n", [(1, 3, 37), (2, 3, (7, 5)), (2, 1, (3, 9))])
def test_traces_and_gather(orc, dim, p, n):
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16))
    mesh, w = mesh_and_field(orc, dim, p, n, seed=1)
    om = upload(ctx, orc, mesh)
    wf_ref = orc.traces(ocfg, om, w)
    wd = to_dev(w)
    wf = zeros_dev(*wf_ref.shape)
    ctx.traces(wd, wf)
    np.testing.assert_allclose(wf.cpu().numpy(), wf_ref, rtol=1e-14, atol=1e-14)
    # gather is a copy: bit-exact given the same traces
    E = mesh.n_elem
    S = zeros_dev(E, ocfg.nstencil, ocfg.nv)
    ctx.gather_stencil(wd, to_dev(wf_ref), 0, E, S)
    S = S.cpu().numpy()
    for e in range(E):
        np.testing.assert_array_equal(S[e], orc.gather_stencil(ocfg, om, w, wf_ref, e))


def _bounds_case(orc, dim, p, nu, n, precision, seed, kind="disc", **kw):
    ctx, ocfg = both(orc, dim, p, nu, precision=precision, **kw)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=seed, kind=kind)
    om = upload(ctx, orc, mesh)
    wf = orc.traces(ocfg, om, w)
    ref = orc.bounds(ocfg, om, w, wf)
    bnd = zeros_dev(2, ocfg.nv, mesh.n_elem)
    ctx.bounds(to_dev(w), to_dev(wf), bnd)
    ctx.check()
    return bounds_error(bnd.cpu().numpy(), ref), ref


@pytest.mark.parametrize("p,nu,n", CASES_2D)
def test_bounds_fp64_2d(orc, p, nu, n):
    err, _ = _bounds_case(orc, 2, p, (nu, nu), n, 0, seed=p)
    assert err.max() < TOL_FP64, err.max()


@pytest.mark.parametrize("p,nu,n", [(3, 64, 41), (2, 200, 9), (5, 33, 4), (1, 2048, 3)])
def test_bounds_fp64_1d(orc, p, nu, n):
    err, _ = _bounds_case(orc, 1, p, (nu,), n, 0, seed=10 + p)
    assert err.max() < TOL_FP64, err.max()


@pytest.mark.parametrize("p,nu,n", CASES_2D)
def test_bounds_fp32_2d(orc, p, nu, n):
    err, _ = _bounds_case(orc, 2, p, (nu, nu), n, 1, seed=20 + p)
    assert err.max() < TOL_FP32, err.max()


@pytest.mark.parametrize("p,nu,n", [(3, 32, (13, 11)), (4, 32, (4, 3)), (2, 64, (3, 3))])
def test_bounds_fp32_2d_tile_4x2(orc, p, nu, n):
    """The 4 x 2 thread tile (a launch-shape knob) gives the same bounds."""
    from paper_2407_20966_gb300 import kbl
    ctx, ocfg = both(orc, 2, p, (nu, nu), precision=1)
    ctx.set_tuning(kbl.TUNE_BOUNDS_TILE, 1)
    mesh, w = mesh_and_field(orc, 2, p, n, seed=25 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    wf = orc.traces(ocfg, om, w)
    ref = orc.bounds(ocfg, om, w, wf)
    bnd = zeros_dev(2, ocfg.nv, mesh.n_elem)
    ctx.bounds(to_dev(w), to_dev(wf), bnd)
    assert bounds_error(bnd.cpu().numpy(), ref).max() < TOL_FP32


@pytest.mark.parametrize("p,n,kind", [(3, (13, 11), "disc"), (1, (1, 1), "smooth"), (2, (7, 5), "disc"),
                                      (4, (4, 3), "smooth"), (5, (3, 2), "disc"), (3, (40, 33), "smooth")])
def test_bounds_fp32_2d_tile_variants(orc, p, n, kind):
    """Launch-shape knobs of the FP32 bounds (32 x 32 grid): the 4 x 2 and 2 x 4 tiles against the
    checker, on ragged meshes and with boundary faces; an unknown tile is refused."""
    from paper_2407_20966_gb300 import kbl
    ctx, ocfg = both(orc, 2, p, (32, 32), precision=1)
    mesh, w = mesh_and_field(orc, 2, p, n, seed=60 + p, kind=kind)
    om = upload(ctx, orc, mesh)
    wf = orc.traces(ocfg, om, w)
    ref = orc.bounds(ocfg, om, w, wf)
    for tile in (1, 2):
        ctx.set_tuning(kbl.TUNE_BOUNDS_TILE, tile)
        bnd = zeros_dev(2, ocfg.nv, mesh.n_elem)
        ctx.bounds(to_dev(w), to_dev(wf), bnd)
        ctx.check()
        assert bounds_error(bnd.cpu().numpy(), ref).max() < TOL_FP32, tile
    with pytest.raises(kbl.KblError):
        ctx.set_tuning(kbl.TUNE_BOUNDS_TILE, 3)


@pytest.mark.parametrize("p,nu,n", [(3, 64, 41), (2, 200, 9), (1, 2048, 3)])
def test_bounds_fp32_1d(orc, p, nu, n):
    err, _ = _bounds_case(orc, 1, p, (nu,), n, 1, seed=30 + p)
    assert err.max() < TOL_FP32, err.max()


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_FP32)])
def test_bounds_strict_mode_and_eps_rule(orc, precision, tol):
    """Strict bounds (r_fac = 0, k = 8; Sec. 3.5, Sec. 5) and the skip reading of the epsilon rule."""
    err, _ = _bounds_case(orc, 2, 3, (32, 32), (5, 4), precision, seed=41, r_fac=0.0, k=8.0, eps_rule=1)
    assert err.max() < tol, err.max()


@pytest.mark.parametrize("dim,p,n", [(1, 3, 37), (2, 3, (9, 7)), (2, 2, (4, 13)), (2, 5, (3, 3))])
def test_rhs(orc, dim, p, n):
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16))
    mesh, w = mesh_and_field(orc, dim, p, n, seed=50 + p)
    om = upload(ctx, orc, mesh)
    wf = orc.traces(ocfg, om, w)
    ref = orc.rhs(ocfg, om, w, wf)
    R = zeros_dev(*w.shape)
    ctx.rhs(to_dev(w), to_dev(wf), R)
    err = rhs_error(R.cpu().numpy(), ref, w, wf, mesh)   # per element and component
    assert err.max() < TOL_FP64, err.max()


@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_non_finite_input_stays_local(orc, precision):
    """A NaN in one element's energy reaches the residual of that element as a non-finite value
    (the FP32 path truncates it to an infinity and widens the non-finite results back to FP64
    with integer operations), and the residual of every element that shares no face with it is
    bit for bit the one of the clean field: the FR residual reads only the element's own nodes and
    the traces across its faces (Sec. 2.3)."""
    ctx, ocfg = both(orc, 2, 3, (16, 16), precision=precision)
    mesh, w = mesh_and_field(orc, 2, 3, (7, 6), seed=61, kind="smooth")
    upload(ctx, orc, mesh)
    e_bad = 17

    def residual(field):
        wd = to_dev(field)
        wf = zeros_dev(field.shape[0], field.shape[1], 4 * 4)
        ctx.traces(wd, wf)
        R = zeros_dev(*field.shape)
        ctx.rhs(wd, wf, R)
        return R.cpu().numpy()

    clean = residual(w)
    w_bad = w.copy()
    w_bad[3, e_bad, 5] = np.nan
    got = residual(w_bad)
    assert not np.isfinite(got[:, e_bad]).all()
    touched = {e_bad} | {int(nb) for nb in np.asarray(mesh.nbr).reshape(-1, 4)[e_bad] if nb >= 0}
    rest = [e for e in range(w.shape[1]) if e not in touched]
    np.testing.assert_array_equal(got[:, rest], clean[:, rest])
    assert np.isfinite(clean).all()


@pytest.mark.parametrize("dim,p,n", [(1, 3, 37), (2, 3, (9, 7)), (2, 2, (4, 13))])
def test_fp32_mixed_traces_rhs_dt(orc, dim, p, n):
    """FP32-mixed contexts run the residual and the time step in FP32 arithmetic (FP64 storage)."""
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16), precision=1)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=55 + p)
    om = upload(ctx, orc, mesh)
    wf_ref = orc.traces(ocfg, om, w)
    wd = to_dev(w)
    wf = zeros_dev(*wf_ref.shape)
    ctx.traces(wd, wf)
    np.testing.assert_allclose(wf.cpu().numpy(), wf_ref, rtol=1e-14, atol=1e-14)   # FP64 in both modes
    R_ref = orc.rhs(ocfg, om, w, wf_ref)
    R = zeros_dev(*w.shape)
    ctx.rhs(wd, to_dev(wf_ref), R)
    err = rhs_error(R.cpu().numpy(), R_ref, w, wf_ref, mesh)   # per element and component
    assert err.max() < TOL_FP32, err.max()
    d = zeros_dev(1)
    ctx.dt(wd, 0.3, d)
    assert d.item() == pytest.approx(orc.dt(ocfg, om, w, 0.3), rel=1e-6)


@pytest.mark.parametrize("dim,p,n", [(1, 3, 37), (2, 3, (9, 7)), (2, 2, (4, 13))])
def test_limit(orc, dim, p, n):
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16))
    mesh, w = mesh_and_field(orc, dim, p, n, seed=60 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    bnd = orc.bounds(ocfg, om, w, orc.traces(ocfg, om, w))
    rng = np.random.default_rng(3)
    w2 = w * (1 + 0.3 * rng.uniform(-1, 1, w.shape))   # rough data against smooth bounds
    ref, a_ref = orc.limit(ocfg, om, w2, bnd)
    wd = to_dev(w2)
    alpha = zeros_dev(2, mesh.n_elem)
    ctx.limit(wd, to_dev(bnd), alpha)
    assert state_error(wd.cpu().numpy(), ref).max() < TOL_FP64
    np.testing.assert_allclose(alpha.cpu().numpy(), a_ref, rtol=1e-10, atol=1e-12)
    assert (a_ref[0] < 1).any()


@pytest.mark.parametrize("dim,p,n", [(1, 3, 37), (2, 3, (9, 7)), (2, 2, (4, 13))])
def test_limit_uncoupled(orc, dim, p, n):
    """The independent limiting stated after Eq. 39 (uncoupled = 1): each component by its own
    alpha_i, on both sides; it differs from the coupled result where the factors differ."""
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16), uncoupled=1)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=160 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    bnd = orc.bounds(ocfg, om, w, orc.traces(ocfg, om, w))
    rng = np.random.default_rng(13)
    w2 = w * (1 + 0.3 * rng.uniform(-1, 1, w.shape))
    ref, a_ref = orc.limit(ocfg, om, w2, bnd)
    wd = to_dev(w2)
    alpha = zeros_dev(2, mesh.n_elem)
    ctx.limit(wd, to_dev(bnd), alpha)
    got = wd.cpu().numpy()
    assert state_error(got, ref).max() < TOL_FP64
    np.testing.assert_allclose(alpha.cpu().numpy(), a_ref, rtol=1e-10, atol=1e-12)
    ocfg.uncoupled = 0
    coupled, _ = orc.limit(ocfg, om, w2, bnd)
    assert state_error(got, coupled).max() > 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_full_step_uncoupled(orc, precision):
    """A whole SSP-RK3 step with uncoupled limiting against the checker, element by element: 1e-12
    FP64; FP32-mixed against max(1e-5, 10 x the checker's own sensitivity to 1e-6 bound and
    residual errors) (gpu_helpers.step_sensitivity).  The checker takes the device's time step
    (FP32 arithmetic in the mixed mode)."""
    ctx, ocfg = both(orc, 2, 3, (16, 16), precision=precision, uncoupled=1)
    mesh, w = mesh_and_field(orc, 2, 3, (7, 6), seed=170, kind="disc")
    om = upload(ctx, orc, mesh)
    wd = to_dev(w)
    ctx.set_time(0.0)
    ctx.counters()
    ctx.step(wd, 0.05)
    st, c = ctx.counters()
    assert st == 0 and c["limited_elements"] > 0
    dt = ctx.time()
    assert dt == pytest.approx(orc.dt(ocfg, om, w, 0.05), rel=1e-14 if precision == 0 else 1e-6)
    ref, _ = orc.ssprk3_step(ocfg, om, w, dt)
    err = state_error(wd.cpu().numpy(), ref).max(axis=(0, 2))
    print("uncoupled step, precision", precision, ": max error", err.max())
    if precision == 0:
        assert err.max() < TOL_FP64, (int(np.argmax(err)), err.max())
    else:
        allowed = np.maximum(TOL_FP32, 10 * step_sensitivity(orc, ocfg, om, w, dt, ref))
        assert np.all(err <= allowed), (int(np.argmax(err / allowed)), err.max())


def test_pressure_relimit_path(orc):
    """Elements with negative pressure at some nodes exercise Eq. 47-49 on both sides."""
    ctx, ocfg = both(orc, 2, 2, (16, 16))
    mesh, w = mesh_and_field(orc, 2, 2, (6, 5), seed=70, kind="smooth")
    om = upload(ctx, orc, mesh)
    bnd = orc.bounds(ocfg, om, w, orc.traces(ocfg, om, w))
    bnd[0] -= 10.0   # wide bounds: only the pressure step acts
    bnd[1] += 10.0
    w2 = w.copy()
    w2[1, ::3, 0] *= 6.0   # kinetic energy above total energy at one node
    ref, a_ref = orc.limit(ocfg, om, w2, bnd)
    assert (a_ref[1] < 1).any()
    wd = to_dev(w2)
    alpha = zeros_dev(2, mesh.n_elem)
    ctx.limit(wd, to_dev(bnd), alpha)
    assert state_error(wd.cpu().numpy(), ref).max() < TOL_FP64
    np.testing.assert_allclose(alpha.cpu().numpy(), a_ref, rtol=1e-10, atol=1e-12)
    st, c = ctx.counters()
    assert c["pressure_relimits"] == int((a_ref[1] < 1).sum())


@pytest.mark.parametrize("s", [0, 1, 2])
def test_stage(orc, s):
    ctx, ocfg = both(orc, 2, 3, (16, 16))
    mesh, w = mesh_and_field(orc, 2, 3, (7, 6), seed=80 + s, kind="smooth")
    om = upload(ctx, orc, mesh)
    wf = orc.traces(ocfg, om, w)
    bnd = orc.bounds(ocfg, om, w, wf)
    R = orc.rhs(ocfg, om, w, wf)
    wn = w * 1.01
    dt = 0.2 * orc.dt(ocfg, om, w, 0.1)
    ref = orc.stage_combine(ocfg, om, s, wn, w, R, dt)
    ref, _ = orc.limit(ocfg, om, ref, bnd)
    out = zeros_dev(*w.shape)
    ctx.stage(s, to_dev(wn), to_dev(w), to_dev(R), to_dev(bnd), to_dev(np.array([dt])), out)
    assert state_error(out.cpu().numpy(), ref).max() < TOL_FP64


@pytest.mark.parametrize("flux", [1, 2])
@pytest.mark.parametrize("dim,p,n,precision", [(1, 3, 37, 0), (2, 3, (9, 7), 0), (2, 2, (4, 13), 0),
                                               (2, 3, (9, 7), 1), (1, 4, 21, 1)])
def test_rhs_hllc(orc, dim, p, n, precision, flux):
    """The residual with the HLLC flux of Sec. 5 (flux = 1) or the HLL flux of Sec. 6.6 (flux = 2)
    on both sides, on discontinuous data (every branch of the flux is taken)."""
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16), precision=precision, flux=flux)
    for seed in range(180, 200):   # the first discontinuous field whose face traces are physical
        mesh, w = mesh_and_field(orc, dim, p, n, seed=seed, kind="disc")
        om = orc.Mesh(mesh.nbr, mesh.h, mesh.bc)
        wf = orc.traces(ocfg, om, w)
        mm = sum(wf[1 + k] ** 2 for k in range(dim))
        if wf[0].min() > 0 and ((wf[dim + 1] - 0.5 * mm / wf[0]).min() > 0):
            break
    om = upload(ctx, orc, mesh)
    R_ref = orc.rhs(ocfg, om, w, wf)
    R = zeros_dev(*w.shape)
    ctx.rhs(to_dev(w), to_dev(wf), R)
    err = rhs_error(R.cpu().numpy(), R_ref, w, wf, mesh).max()   # per element and component
    assert err < (TOL_FP64 if precision == 0 else TOL_FP32), err
    ocfg.flux = 0
    assert np.abs(orc.rhs(ocfg, om, w, wf) - R_ref).max() > 1e-3 * np.abs(R_ref).max()


@pytest.mark.parametrize("flux", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_full_step_hllc(orc, precision, flux):
    ctx, ocfg = both(orc, 2, 3, (16, 16), precision=precision, flux=flux)
    mesh, w = mesh_and_field(orc, 2, 3, (7, 6), seed=190, kind="smooth")
    om = upload(ctx, orc, mesh)
    dt = orc.dt(ocfg, om, w, 0.05)
    ref, _ = orc.ssprk3_step(ocfg, om, w, dt)
    wd = to_dev(w)
    ctx.set_time(0.0)
    ctx.step(wd, 0.05)
    ctx.check()
    assert state_error(wd.cpu().numpy(), ref).max() < (TOL_FP64 if precision == 0 else TOL_FP32)


@pytest.mark.parametrize("dim,p,n", [(1, 3, 37), (2, 3, (9, 7))])
def test_dt(orc, dim, p, n):
    ctx, ocfg = both(orc, dim, p, (64,) if dim == 1 else (16, 16))
    mesh, w = mesh_and_field(orc, dim, p, n, seed=90)
    om = upload(ctx, orc, mesh)
    d = zeros_dev(1)
    ctx.dt(to_dev(w), 0.3, d)
    assert d.item() == pytest.approx(orc.dt(ocfg, om, w, 0.3), rel=1e-14)


@pytest.mark.parametrize("dim,p,n,nu,precision", [
    (1, 3, 40, (64,), 0), (2, 3, (8, 6), (32, 32), 0), (2, 2, (6, 9), (16, 16), 0),
    (1, 3, 40, (64,), 1), (2, 3, (8, 6), (32, 32), 1)])
def test_full_step(orc, dim, p, n, nu, precision):
    """One SSP-RK3 step with bounds and limiting after each stage (Sec. 3.9), from the same
    state; the device time step is compared too."""
    ctx, ocfg = both(orc, dim, p, nu, precision=precision)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=100 + p, kind="smooth")
    om = upload(ctx, orc, mesh)
    dt = orc.dt(ocfg, om, w, 0.1)
    ref, _ = orc.ssprk3_step(ocfg, om, w, dt)
    wd = to_dev(w)
    ctx.set_time(0.0)
    ctx.step(wd, 0.1)
    # FP32-mixed contexts compute the time step in FP32
    assert ctx.time() == pytest.approx(dt, rel=1e-14 if precision == 0 else 1e-6)
    tol = TOL_FP64 if precision == 0 else TOL_FP32
    assert state_error(wd.cpu().numpy(), ref).max() < tol
    ctx.check()


def test_sod_steps_and_end_time(orc):
    """Config of the 1D shock tube (Sec. 6.1 set-up, 200 P3 elements, 64 velocity points): the
    steps to a short end time against the checker, the last one clipped to the end time."""
    from paper_2407_20966_gb300 import inputs
    mesh, ic = inputs.sod(200)
    ctx, ocfg = both(orc, 1, 3, (64,))
    om = upload(ctx, orc, mesh)
    xi, _ = orc.gauss_legendre(4)
    w = inputs.nodal_field(mesh, xi, ic)
    t_end = 9.5 * orc.dt(ocfg, om, w, 0.1)
    ref, t, nsteps = w.copy(), 0.0, 0
    while t < t_end - 1e-15:
        dt = min(orc.dt(ocfg, om, ref, 0.1), t_end - t)
        ref, _ = orc.ssprk3_step(ocfg, om, ref, dt)
        t += dt
        nsteps += 1
    wd = to_dev(w)
    ctx.set_time(0.0, t_end)
    for _ in range(nsteps):
        ctx.step(wd, 0.1)
    assert ctx.time() == pytest.approx(t_end, rel=1e-13)
    assert state_error(wd.cpu().numpy(), ref).max() < 1e-11


def test_run_host_matches_device_steps(orc):
    ctx, ocfg = both(orc, 2, 2, (16, 16), precision=1)
    mesh, w = mesh_and_field(orc, 2, 2, (5, 6), seed=5, kind="smooth")
    upload(ctx, orc, mesh)
    out = np.zeros_like(w)
    ctx.set_time(0.0)
    ctx.run_host(w, out, 3, 0.1)
    wd = to_dev(w)
    ctx.set_time(0.0)
    for _ in range(3):
        ctx.step(wd, 0.1)
    np.testing.assert_array_equal(out, wd.cpu().numpy())


def test_empty_mesh_and_single_periodic_element(orc):
    ctx, ocfg = both(orc, 2, 3, (16, 16))
    ctx.mesh_upload(np.zeros((0, 4), np.int32), np.zeros((0, 2)), None)
    e = zeros_dev(0)
    ctx.traces(e, e)
    ctx.bounds(e, e, e)
    ctx.step(e, 0.1)
    ctx.check()
    from paper_2407_20966_gb300 import inputs
    mesh = inputs.mesh_2d(1, 1, 0, 1, 0, 1, periodic=(True, True))
    om = upload(ctx, orc, mesh)
    xi, _ = orc.gauss_legendre(4)
    rng = np.random.default_rng(0)
    base = inputs.random_states(rng, 1, 2)[0]
    w = np.ascontiguousarray(base[:, None, None] * (1 + 0.05 * rng.uniform(-1, 1, (4, 1, 16))))
    wf = orc.traces(ocfg, om, w)
    ref = orc.bounds(ocfg, om, w, wf)
    bnd = zeros_dev(2, 4, 1)
    ctx.bounds(to_dev(w), to_dev(wf), bnd)
    assert bounds_error(bnd.cpu().numpy(), ref).max() < TOL_FP64


def test_nonphysical_state_is_reported(orc):
    from paper_2407_20966_gb300 import kbl
    ctx, ocfg = both(orc, 2, 2, (16, 16))
    mesh, w = mesh_and_field(orc, 2, 2, (4, 4), seed=7, kind="smooth")
    upload(ctx, orc, mesh)
    w[3, 5, 2] = -1.0      # negative energy -> negative pressure at one node of element 5
    wd = to_dev(w)
    wf = zeros_dev(4, mesh.n_elem, 12)
    ctx.traces(wd, wf)
    bnd = zeros_dev(2, 4, mesh.n_elem)
    ctx.bounds(wd, wf, bnd)
    with pytest.raises(kbl.KblError) as ei:
        ctx.check()
    assert ei.value.status == kbl.ENONPHYSICAL
    b = bnd.cpu().numpy()
    assert np.isnan(b[:, :, 5]).all()
    ctx.check()   # flags were cleared


def test_bad_arguments_rejected(orc):
    from paper_2407_20966_gb300 import kbl
    ctx, _ = both(orc, 2, 3, (16, 16))
    with pytest.raises(kbl.KblError):
        ctx.traces(zeros_dev(1), zeros_dev(1))          # no mesh yet
    with pytest.raises(kbl.KblError):
        ctx.mesh_upload(np.array([[5, 0, 0, 0]]), np.ones((1, 2)), None)   # neighbour out of range
    with pytest.raises(kbl.KblError):
        ctx.mesh_upload(np.array([[-3, 0, 0, 0]]), np.ones((1, 2)), np.ones((1, 4)))  # bad bc id


def test_limiter_counters(orc):
    """The limiter's counters: the alpha histogram matches the factors the checker computes, the
    epsilon rule of Eq. 37 fires on exactly the (element, component) pairs whose extreme over V
    lies within eps of the mean, and the mean-outside-bounds count matches the pairs whose mean
    lies outside [w_min, w_max]."""
    ctx, ocfg = both(orc, 2, 2, (16, 16))
    mesh, w = mesh_and_field(orc, 2, 2, (9, 8), seed=77, kind="smooth")
    om = upload(ctx, orc, mesh)
    E = mesh.n_elem
    bnd = orc.bounds(ocfg, om, w, orc.traces(ocfg, om, w))
    rng = np.random.default_rng(8)
    w2 = w * (1 + 0.3 * rng.uniform(-1, 1, w.shape))
    w2[2, 3:9] = w2[2, 3:9, :1]          # m_y constant in six elements: the epsilon rule fires
    x, wq = orc.gauss_legendre(3)
    W = np.outer(wq, wq).ravel()
    mean = (w2 * W).sum(axis=2) / W.sum()
    bnd[0, 0, 20:25] = mean[0, 20:25] + 0.05   # the density mean below its lower bound
    bnd[1, 3, 30:33] = mean[3, 30:33] - 0.05   # the energy mean above its upper bound
    ref, a_ref = orc.limit(ocfg, om, w2, bnd)
    wf = orc.traces(ocfg, om, w2)
    vmax = np.maximum(w2.max(axis=2), wf.max(axis=2))
    vmin = np.minimum(w2.min(axis=2), wf.min(axis=2))
    n_eps = int(((np.abs(vmin - mean) < ocfg.eps) | (np.abs(vmax - mean) < ocfg.eps)).sum())
    n_out = int(((mean < bnd[0]) | (mean > bnd[1])).sum())
    a = a_ref[0][a_ref[0] < 1]
    hist = np.bincount(np.minimum((a * 10).astype(int), 9), minlength=10)
    ctx.counters()
    wd = to_dev(w2)
    ctx.limit(wd, to_dev(bnd))
    st, c = ctx.counters()
    assert state_error(wd.cpu().numpy(), ref).max() < TOL_FP64
    print("counters:", c)
    assert n_eps == 6 and n_out >= 8
    assert c["eps_rule_activations"] == n_eps
    assert c["mean_outside_bounds"] == n_out
    assert c["alpha_hist"] == hist.tolist()
    assert sum(c["alpha_hist"]) == c["limited_elements"] == int((a_ref[0] < 1).sum())


def test_run_host_ensemble_matches_device_steps(orc):
    """kbl_run_host_ensemble: independent states on one mesh, two alternating device copies with
    the copies of neighbouring members overlapping each member's steps; every member's result
    equals kbl_step on device data from the same start time, bit for bit, and aliasing the
    output with the input gives the same."""
    import torch
    ctx, ocfg = both(orc, 2, 3, (16, 16), precision=1)
    mesh, w = mesh_and_field(orc, 2, 3, (6, 5), seed=31, kind="smooth")
    upload(ctx, orc, mesh)
    rng = np.random.default_rng(4)
    members = np.ascontiguousarray(np.stack([w * (1 + 0.01 * rng.uniform(-1, 1, w.shape)) for _ in range(5)]))
    ref = []
    for k in range(5):
        wd = to_dev(members[k])
        ctx.set_time(0.25)
        for _ in range(2):
            ctx.step(wd, 0.1)
        ref.append(wd.cpu().numpy())
    ref = np.stack(ref)
    w_in = torch.from_numpy(members).pin_memory()
    w_out = torch.zeros_like(w_in).pin_memory()
    ctx.set_time(0.25)
    ctx.run_host_ensemble(w_in.numpy(), w_out.numpy(), 2, 0.1)
    np.testing.assert_array_equal(w_out.numpy(), ref)
    inout = members.copy()
    ctx.set_time(0.25)
    ctx.run_host_ensemble(inout, inout, 2, 0.1)
    np.testing.assert_array_equal(inout, ref)
    ctx.check()


@pytest.mark.parametrize("strict", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dim,p,n", [(2, 3, (13, 11)), (2, 1, (9, 7)), (2, 2, (12, 10)), (2, 4, (11, 9)),
                                     (1, 3, 45)])
def test_step_residual_branch_is_bitwise_serial(orc, precision, dim, p, n, strict):
    """The step graph with branches (the default: each stage's residual beside its bounds, the time
    step beside the traces) gives the serial graph's state and limiter counters bit for bit: the
    same arithmetic and the same decisions.  Discontinuous fields, so that the screen leaves elements
    to the exact limiter; element counts that end in a partial block; with the strict bounds
    (r = 0, k = 8) the limiter cuts elements."""
    from paper_2407_20966_gb300 import kbl
    nu = (64,) if dim == 1 else (16, 16)
    kw = dict(r_fac=0.0, k=8.0) if strict else {}
    ctx, _ = both(orc, dim, p, nu, precision=precision, **kw)
    mesh, w = mesh_and_field(orc, dim, p, n, seed=21, kind="disc", periodic=True)
    if strict:   # blasts in every seventh element: shocks the limiter has to cut
        w = w.copy()
        w[-1, ::7] *= 1e3
    upload(ctx, orc, mesh)
    out, cnt = [], []
    for ov in (1, 0):
        ctx.set_tuning(kbl.TUNE_RHS_OVERLAP, ov)
        assert ctx.get_tuning(kbl.TUNE_RHS_OVERLAP) == ov
        wd = to_dev(w)
        ctx.set_time(0.0)
        ctx.counters()   # reading the counters clears them
        for _ in range(3):
            ctx.step(wd, 0.05)
        st, c1 = ctx.counters()
        assert st == 0, st
        out.append(wd.cpu().numpy())
        cnt.append({k: np.asarray(c1[k]) for k in c1})
        assert ctx.time() > 0.0
    np.testing.assert_array_equal(out[0], out[1])
    if strict:
        assert cnt[0]["limited_elements"] > 0 and cnt[0]["pressure_relimits"] > 0   # the exact limiter cut
    for k in cnt[0]:
        np.testing.assert_array_equal(cnt[0][k], cnt[1][k], err_msg=k)
