"""Triangle path (Sec. 5) on the GPU against the checker, element by element.

  points     kbl_tri_points                 vs orc.tri_points        5e-15 (two Newton solves)
  traces     kbl_tri_traces(w)              vs orc.tri_traces        1e-14 of the element's scale
  stencils   kbl_tri_gather_stencil(w, wf)  vs orc.tri_gather_stencil, same inputs: bit-exact
  residual   kbl_tri_residual(w, wf)        vs orc.tri_rhs, same inputs: 1e-12 of the term scale
             (FP64), 1e-5 (FP32-mixed: FP32 arithmetic on FP64 storage)
  dt         kbl_tri_dt                     vs orc.tri_dt            1e-14
  bounds     kbl_bounds_stencil of the device's stencils vs orc.bounds_stencil: 1e-12 / 1e-5
  step       kbl_tri_step                   vs orc.tri_ssprk3_step   1e-12 FP64; FP32-mixed (bounds
             and residual): 1e-5 where the step is well conditioned (a blast, density >= 0.125)
  curved     kbl_tri_create_curved meshes (quadratic edges): residual 1e-12 / 1e-5 and steps
             1e-12 / 1e-5 against the checker's curved scheme; straight midpoints reproduce the
             affine path to 1e-12; a folded element is KBL_EINVAL
Meshes of 2 x nx x ny jittered triangles span several thread blocks with a ragged tail, periodic
and with boundary states, for every common flux.
"""
import numpy as np
import pytest

from paper_2407_20966_gb300 import inputs
from tests.gpu_helpers import TOL_FP32, TOL_FP64, bounds_error

pytestmark = pytest.mark.gpu
G = 1.4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _blast(x, y):
    s = 0.5 * (1 - np.tanh((np.sqrt((x - 0.5) ** 2 + (y - 0.45) ** 2) - 0.25) / 0.05))
    rho = 0.125 + 0.875 * s
    P = 0.1 + 0.9 * s
    u = 0.2 * np.sin(2 * np.pi * y)
    v = -0.1 * np.cos(2 * np.pi * x)
    return np.stack([rho, rho * u, rho * v, P / (G - 1) + 0.5 * rho * (u * u + v * v)])


def _smooth(x, y):
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    u, v, P = 0.3 + 0 * x, -0.2 + 0 * x, 1.0 + 0.1 * np.cos(2 * np.pi * x)
    return np.stack([rho, rho * u, rho * v, P / (G - 1) + 0.5 * rho * (u * u + v * v)])


def _setup(orc, p, nx, ny, periodic, flux=0, precision=0, seed=5, ic=None):
    from paper_2407_20966_gb300 import kbl
    m = inputs.tri_mesh_2d(nx, ny, 0.0, 1.0, 0.0, 0.9, jitter=0.2, seed=seed, periodic=(periodic, periodic))
    rng = np.random.default_rng(seed)
    m.bc = np.stack([_blast(np.array(0.0), np.array(0.0)), _blast(np.array(1.0), np.array(0.5))])
    m.bc = m.bc * (1 + 0.05 * rng.uniform(-1, 1, m.bc.shape))
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    cfg = orc.Config(dim=2, p=p, nu=(16, 16), flux=flux)
    tm = kbl.TriMesh(p, m.xy, m.nbr, m.nbr_edge, m.bc, precision=precision, flux=flux, nu=(16, 16))
    rs, _ = orc.tri_points(p)
    w = inputs.tri_nodal_field(m, rs, ic if ic is not None else _blast)
    w = w * (1 + 0.02 * rng.uniform(-1, 1, w.shape))   # discontinuous across elements
    return m, om, cfg, tm, np.ascontiguousarray(w)


def _elem_scale(a):
    """[E][n][4] -> per element and component the largest magnitude, momentum held to the
    energy scale sqrt(2 rho_max E_max)."""
    sc = np.abs(a).max(axis=1)                           # [E][4]
    mom = np.sqrt(2 * sc[:, 0] * sc[:, 3])
    sc[:, 1] = np.maximum(sc[:, 1], mom)
    sc[:, 2] = np.maximum(sc[:, 2], mom)
    return sc[:, None, :]


def _geometry(m):
    X = m.xy
    J1, J2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    det = J1[:, 0] * J2[:, 1] - J2[:, 0] * J1[:, 1]
    edges = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 1], X[:, 0] - X[:, 2]], axis=1)
    lmax = np.sqrt((edges ** 2).sum(axis=2)).max(axis=1)
    return det, det / lmax


def _residual_scale(m, w, S):
    """Size of the terms the triangle residual sums, per element and component: (2 / h) (max |F| +
    lam max |q|) over the element's stencil (solution, flux and exterior points), lam the
    largest |u| + c there."""
    q = S                                                # [E][n][4]
    rho, E_ = q[..., 0], q[..., 3]
    mm = q[..., 1] ** 2 + q[..., 2] ** 2
    P = (G - 1) * (E_ - 0.5 * mm / rho)
    F = np.zeros_like(q)
    for k in range(2):
        u = q[..., 1 + k] / rho
        comp = [q[..., 1 + k], q[..., 1] * u + (P if k == 0 else 0), q[..., 2] * u + (P if k == 1 else 0),
                (E_ + P) * u]
        for v in range(4):
            F[..., v] = np.maximum(F[..., v], np.abs(comp[v]))
    lam = (np.sqrt(mm) / rho + np.sqrt(G * P / rho)).max(axis=1)   # [E]
    _, h = _geometry(m)
    s = (2.0 / h)[:, None] * (F.max(axis=1) + lam[:, None] * np.abs(q).max(axis=1))
    return s[:, None, :]


@pytest.mark.parametrize("p", [1, 2])
def test_points_match(orc, p):
    from paper_2407_20966_gb300 import kbl
    rs, w = kbl.tri_points(p)
    rso, wo = orc.tri_points(p)
    # two different Newton solves of the same moment equations (the checker's with a
    # finite-difference Jacobian stops a few ulps short): agreement to a few ulps
    assert np.abs(rs - rso).max() < 5e-15 and np.abs(w - wo).max() < 5e-15


@pytest.mark.parametrize("p,nx,ny,periodic,flux", [
    (1, 13, 11, True, 0), (2, 13, 11, True, 1), (1, 9, 14, False, 2), (2, 17, 7, False, 0), (2, 9, 14, True, 2)])
def test_traces_stencils_residual_dt(orc, p, nx, ny, periodic, flux):
    import torch
    m, om, cfg, tm, w = _setup(orc, p, nx, ny, periodic, flux)
    E = m.n_elem
    assert E % 128 != 0 and E > 128
    wd = _dev(w)
    wf_d = torch.zeros(E, tm.nfp, 4, dtype=torch.float64, device="cuda")
    tm.traces(wd, wf_d)
    wf_ref = orc.tri_traces(cfg, om, w)
    err = np.abs(wf_d.cpu().numpy() - wf_ref) / _elem_scale(wf_ref)
    assert err.max() < 1e-14, err.max()
    # stencils and residual from the checker's traces (identical inputs)
    wf_in = _dev(wf_ref)
    S_d = torch.zeros(E, tm.nstencil, 4, dtype=torch.float64, device="cuda")
    tm.gather_stencil(wd, wf_in, S_d)
    S = S_d.cpu().numpy()
    for e in range(E):
        np.testing.assert_array_equal(S[e], orc.tri_gather_stencil(cfg, om, w, wf_ref, e))
    R_d = torch.zeros_like(wd)
    tm.residual(wd, wf_in, R_d)
    R_ref = orc.tri_rhs(cfg, om, w, wf_ref)
    err = np.abs(R_d.cpu().numpy() - R_ref) / np.maximum(np.abs(R_ref), _residual_scale(m, w, S))
    assert err.max() < TOL_FP64, err.max()
    dt = tm.dt(wd, 0.3)
    dt_ref = orc.tri_dt(cfg, om, w, 0.3)
    assert abs(dt - dt_ref) <= 1e-14 * dt_ref


@pytest.mark.parametrize("p,flux,periodic", [(1, 0, True), (2, 1, False), (2, 2, True), (1, 1, False)])
def test_residual_fp32(orc, p, flux, periodic):
    """FP32-mixed: the residual in FP32 arithmetic on FP64 storage, against the checker's FP64
    residual on the same inputs, to 1e-5 of the size of the terms it sums."""
    import torch
    m, om, cfg, tm, w = _setup(orc, p, 13, 11, periodic, flux, precision=1)
    E = m.n_elem
    wf_ref = orc.tri_traces(cfg, om, w)
    wd, wf_in = _dev(w), _dev(wf_ref)
    S_d = torch.zeros(E, tm.nstencil, 4, dtype=torch.float64, device="cuda")
    tm.gather_stencil(wd, wf_in, S_d)
    R_d = torch.zeros_like(wd)
    tm.residual(wd, wf_in, R_d)
    R_ref = orc.tri_rhs(cfg, om, w, wf_ref)
    err = np.abs(R_d.cpu().numpy() - R_ref) / np.maximum(np.abs(R_ref), _residual_scale(m, w, S_d.cpu().numpy()))
    assert err.max() < TOL_FP32, err.max()
    assert err.max() > 1e-12   # FP32 arithmetic is in use


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p", [1, 2])
def test_stencil_bounds(orc, p, precision):
    import torch
    from paper_2407_20966_gb300 import kbl
    m, om, cfg, tm, w = _setup(orc, p, 11, 9, False, precision=precision)
    E = m.n_elem
    wf_ref = orc.tri_traces(cfg, om, w)
    S_d = torch.zeros(E, tm.nstencil, 4, dtype=torch.float64, device="cuda")
    tm.gather_stencil(_dev(w), _dev(wf_ref), S_d)
    ctx = kbl.Context(dim=2, p=p, nu=(16, 16), precision=precision)
    bnd = torch.zeros(2, 4, E, dtype=torch.float64, device="cuda")
    ctx.bounds_stencil(S_d, bnd)
    ctx.check()
    ref = np.zeros((2, 4, E))
    for e in range(E):
        ref[0, :, e], ref[1, :, e] = orc.bounds_stencil(cfg, orc.tri_gather_stencil(cfg, om, w, wf_ref, e))
    err = bounds_error(bnd.cpu().numpy(), ref)
    assert err.max() < (TOL_FP64 if precision == 0 else TOL_FP32), err.max()


@pytest.mark.parametrize("p,flux,periodic", [(1, 0, True), (2, 1, False), (2, 2, True), (1, 1, False)])
def test_step_fp64(orc, p, flux, periodic):
    m, om, cfg, tm, w = _setup(orc, p, 12, 11, periodic, flux)
    wd = _dev(w)
    dt = orc.tri_dt(cfg, om, w, 0.2)
    for _ in range(2):
        tm.step(wd, dt)
    tm.check()
    ref, alpha = w, None
    for _ in range(2):
        ref, alpha = orc.tri_ssprk3_step(cfg, om, ref, dt)
    assert (alpha[0] < 1).any()   # the limiter is active
    err = np.abs(wd.cpu().numpy() - ref) / _elem_scale(ref)
    assert err.max() < TOL_FP64, err.max()


@pytest.mark.parametrize("p", [1, 2])
def test_step_fp32_mixed(orc, p):
    m, om, cfg, tm, w = _setup(orc, p, 12, 11, True, flux=1, precision=1)
    wd = _dev(w)
    dt = orc.tri_dt(cfg, om, w, 0.2)
    tm.step(wd, dt)
    tm.check()
    ref, _ = orc.tri_ssprk3_step(cfg, om, w, dt)
    err = np.abs(wd.cpu().numpy() - ref) / _elem_scale(ref)
    assert err.max() < TOL_FP32, err.max()


def test_empty_and_invalid_meshes(orc):
    import torch
    from paper_2407_20966_gb300 import kbl
    tm = kbl.TriMesh(1, np.zeros((0, 3, 2)), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32),
                     np.zeros((1, 4)))
    w = torch.zeros(0, 3, 4, dtype=torch.float64, device="cuda")
    tm.step(w, 0.1)
    assert tm.dt(w, 0.5) == 0.0
    tm.check()
    m = inputs.tri_mesh_2d(3, 3, 0.0, 1.0, 0.0, 1.0)
    with pytest.raises(kbl.KblError):   # p outside {1, 2}
        kbl.TriMesh(3, m.xy, m.nbr, m.nbr_edge, m.bc)
    bad = m.xy.copy()
    bad[0] = bad[0][::-1]               # clockwise
    with pytest.raises(kbl.KblError):
        kbl.TriMesh(1, bad, m.nbr, m.nbr_edge, m.bc)
    nb = m.nbr.copy()
    nb[0, 0] = m.n_elem                 # out of range
    with pytest.raises(kbl.KblError):
        kbl.TriMesh(1, m.xy, nb, m.nbr_edge, m.bc)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p,periodic", [(1, False), (2, True), (2, False)])
def test_fused_bounds_equal_gathered_stencil_bounds(orc, p, periodic, precision):
    """kbl_tri_bounds (stencils gathered inside the bounds kernel, the step's bounds) equals
    kbl_tri_gather_stencil + kbl_bounds_stencil bit for bit."""
    import torch
    from paper_2407_20966_gb300 import kbl
    m, om, cfg, tm, w = _setup(orc, p, 11, 13, periodic, precision=precision)
    E = m.n_elem
    wd = _dev(w)
    wf = torch.zeros(E, tm.nfp, 4, dtype=torch.float64, device="cuda")
    tm.traces(wd, wf)
    fused = torch.zeros(2, 4, E, dtype=torch.float64, device="cuda")
    tm.bounds(wd, wf, fused)
    S = torch.zeros(E, tm.nstencil, 4, dtype=torch.float64, device="cuda")
    tm.gather_stencil(wd, wf, S)
    ctx = kbl.Context(dim=2, p=p, nu=(16, 16), precision=precision)
    ref = torch.zeros_like(fused)
    ctx.bounds_stencil(S, ref)
    tm.check()
    ctx.check()
    assert torch.equal(fused, ref)


def test_full_size_workload_per_call(orc):
    """The benchmark's triangle workload at full size (2 x 256^2 jittered periodic P2 triangles,
    32 x 32 grid, FP32-mixed, HLLC), each call of a stage on the checker's inputs: traces of the
    whole mesh (1e-14), residual of the whole mesh (1e-5 of the term scale), bounds of 192
    sampled elements (1e-5) and the node-set limiter of the whole mesh with the device's bounds
    against the checker's limiter on 192 sampled elements (1e-12: FP64)."""
    import torch
    from paper_2407_20966_gb300 import kbl
    m = inputs.tri_mesh_2d(256, 256, 0.0, 1.0, 0.0, 1.0, jitter=0.2, seed=17)
    E = m.n_elem
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc)
    cfg = orc.Config(dim=2, p=2, nu=(32, 32), flux=1)
    tm = kbl.TriMesh(2, m.xy, m.nbr, m.nbr_edge, m.bc, precision=kbl.FP32_MIXED, flux=1, nu=(32, 32))
    rs, wq = orc.tri_points(2)
    w = inputs.tri_nodal_field(m, rs, inputs.tri_blast)
    wd = _dev(w)
    wf_d = torch.zeros(E, tm.nfp, 4, dtype=torch.float64, device="cuda")
    tm.traces(wd, wf_d)
    wf_ref = orc.tri_traces(cfg, om, w)
    assert (np.abs(wf_d.cpu().numpy() - wf_ref) / _elem_scale(wf_ref)).max() < 1e-14
    wf_in = _dev(wf_ref)
    R_d = torch.zeros_like(wd)
    tm.residual(wd, wf_in, R_d)
    S_d = torch.zeros(E, tm.nstencil, 4, dtype=torch.float64, device="cuda")
    tm.gather_stencil(wd, wf_in, S_d)
    S = S_d.cpu().numpy()
    R_ref = orc.tri_rhs(cfg, om, w, wf_ref)
    err = np.abs(R_d.cpu().numpy() - R_ref) / np.maximum(np.abs(R_ref), _residual_scale(m, w, S))
    assert err.max() < TOL_FP32, err.max()
    bnd = torch.zeros(2, 4, E, dtype=torch.float64, device="cuda")
    tm.bounds(wd, wf_in, bnd)
    tm.check()
    bnd_h = bnd.cpu().numpy()
    sample = np.random.default_rng(3).choice(E, 192, replace=False)
    ref = np.zeros((2, 4, len(sample)))
    for k, e in enumerate(sample):
        ref[0, :, k], ref[1, :, k] = orc.bounds_stencil(cfg, S[e])
    assert bounds_error(bnd_h[:, :, sample], ref).max() < TOL_FP32
    # limiter of a perturbed state (zero weighted mean per element) against the device's bounds
    d = np.sin(3.0 * np.arange(len(wq)))
    d = d - (wq * d).sum() / wq.sum()
    amp = np.abs(w).max(axis=1, keepdims=True)
    wp = np.ascontiguousarray(w + 0.05 * amp * d[None, :, None])
    wfp = orc.tri_traces(cfg, om, wp)
    ctx = kbl.Context(dim=2, p=2, nu=(32, 32), precision=kbl.FP32_MIXED)
    U = _dev(wp)
    alpha = torch.zeros(2, E, dtype=torch.float64, device="cuda")
    ctx.limit_nodes(wq, U, _dev(wfp), bnd, alpha)
    ctx.check()
    U_h, a_h = U.cpu().numpy(), alpha.cpu().numpy()
    limited = 0
    for e in sample:
        lim, a = orc.limit_nodes(cfg, wq, np.ascontiguousarray(wp[e].T), np.ascontiguousarray(wfp[e].T),
                                 bnd_h[0, :, e], bnd_h[1, :, e])
        limited += a[0] < 1
        err = np.abs(U_h[e].T - lim) / _elem_scale(lim.T[None])[0].T
        assert err.max() < TOL_FP64, (e, err.max())
        assert abs(a_h[0, e] - a[0]) < 1e-12 and abs(a_h[1, e] - a[1]) < 1e-12
    assert limited > 0


@pytest.mark.parametrize("p,nx,ny,periodic", [(1, 1, 1, True), (2, 1, 1, True), (2, 2, 1, False), (1, 3, 2, False)])
def test_tiny_meshes_step(orc, p, nx, ny, periodic):
    """Meshes of 2 to 12 triangles (one partial block everywhere; on the 1 x 1 periodic mesh both
    elements are each other's neighbours across all three edges), a smooth field perturbed per
    node: two FP64 steps against the checker."""
    m, om, cfg, tm, w = _setup(orc, p, nx, ny, periodic, flux=1, seed=9, ic=_smooth)
    wd = _dev(w)
    dt = orc.tri_dt(cfg, om, w, 0.2)
    ref = w
    for _ in range(2):
        tm.step(wd, dt)
        ref, _ = orc.tri_ssprk3_step(cfg, om, ref, dt)
    tm.check()
    err = np.abs(wd.cpu().numpy() - ref) / _elem_scale(ref)
    assert err.max() < TOL_FP64, err.max()


# ---- curved (quadratic) elements --------------------------------------------------------------
def _setup_curved(orc, p, nx, ny, periodic, flux=0, precision=0, seed=5, bump=0.15, straight=False):
    from paper_2407_20966_gb300 import kbl
    m = inputs.tri_curved_mesh(nx, ny, 0.0, 1.0, 0.0, 0.9, jitter=0.2, bump=bump, seed=seed,
                               periodic=(periodic, periodic))
    if straight:
        m.xy6 = np.concatenate([m.xy, 0.5 * (m.xy + np.roll(m.xy, -1, axis=1))], axis=1)
    rng = np.random.default_rng(seed)
    m.bc = np.stack([_blast(np.array(0.0), np.array(0.0)), _blast(np.array(1.0), np.array(0.5))])
    om = orc.TriMesh(m.xy, m.nbr, m.nbr_edge, m.bc, xy6=m.xy6)
    cfg = orc.Config(dim=2, p=p, nu=(16, 16), flux=flux)
    tm = kbl.TriMesh(p, m.xy, m.nbr, m.nbr_edge, m.bc, precision=precision, flux=flux, nu=(16, 16), xy6=m.xy6)
    rs, _ = orc.tri_points(p)
    w = inputs.tri_nodal_field(m, rs, _blast)
    w = w * (1 + 0.02 * rng.uniform(-1, 1, w.shape))
    return m, om, cfg, tm, np.ascontiguousarray(w)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p,flux,periodic", [(1, 0, True), (2, 1, False), (2, 2, True)])
def test_curved_residual(orc, p, flux, periodic, precision):
    import torch
    m, om, cfg, tm, w = _setup_curved(orc, p, 13, 11, periodic, flux, precision)
    E = m.n_elem
    wf_ref = orc.tri_traces(cfg, om, w)
    wd, wf_in = _dev(w), _dev(wf_ref)
    S_d = torch.zeros(E, tm.nstencil, 4, dtype=torch.float64, device="cuda")
    tm.gather_stencil(wd, wf_in, S_d)
    R_d = torch.zeros_like(wd)
    tm.residual(wd, wf_in, R_d)
    R_ref = orc.tri_rhs(cfg, om, w, wf_ref)
    err = np.abs(R_d.cpu().numpy() - R_ref) / np.maximum(np.abs(R_ref), _residual_scale(m, w, S_d.cpu().numpy()))
    assert err.max() < (TOL_FP64 if precision == 0 else TOL_FP32), err.max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p,flux,periodic", [(1, 1, True), (2, 1, False), (2, 0, True)])
def test_curved_step(orc, p, flux, periodic, precision):
    m, om, cfg, tm, w = _setup_curved(orc, p, 12, 11, periodic, flux, precision)
    wd = _dev(w)
    dt = orc.tri_dt(cfg, om, w, 0.2)
    ref, alpha = w, None
    for _ in range(2 if precision == 0 else 1):   # FP32-mixed: one step, as on affine meshes
        tm.step(wd, dt)
        ref, alpha = orc.tri_ssprk3_step(cfg, om, ref, dt)
    tm.check()
    assert (alpha[0] < 1).any()
    err = np.abs(wd.cpu().numpy() - ref) / _elem_scale(ref)
    assert err.max() < (TOL_FP64 if precision == 0 else TOL_FP32), err.max()


def test_curved_with_straight_edges_equals_affine_on_the_device(orc):
    """The quadratic map of straight edges is the affine one: the curved path's step equals the
    affine path's to rounding."""
    from paper_2407_20966_gb300 import kbl
    m, om, cfg, tc, w = _setup_curved(orc, 2, 9, 8, True, flux=1, straight=True)
    ta = kbl.TriMesh(2, m.xy, m.nbr, m.nbr_edge, m.bc, flux=1, nu=(16, 16))
    wc, wa = _dev(w), _dev(w)
    dt = orc.tri_dt(cfg, om, w, 0.2)
    for _ in range(2):
        tc.step(wc, dt)
        ta.step(wa, dt)
    tc.check()
    ta.check()
    a = wa.cpu().numpy()
    err = np.abs(wc.cpu().numpy() - a) / _elem_scale(a)
    assert err.max() < 1e-12, err.max()


def test_curved_rejects_a_folded_element(orc):
    from paper_2407_20966_gb300 import kbl
    m = inputs.tri_curved_mesh(3, 3, 0.0, 1.0, 0.0, 1.0, bump=0.15)
    xy6 = m.xy6.copy()
    xy6[0, 3] = xy6[0, 2] + 2.0 * (xy6[0, 2] - 0.5 * (xy6[0, 0] + xy6[0, 1]))   # edge 0 pulled past the opposite corner
    with pytest.raises(kbl.KblError):
        kbl.TriMesh(1, m.xy, m.nbr, m.nbr_edge, m.bc, xy6=xy6)
