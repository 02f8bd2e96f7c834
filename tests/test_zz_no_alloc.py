"""kbl_bounds_noalloc: the bounds for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (they hand all device memory to their own pool at
start-up, or cannot afford cudaMalloc's implicit synchronisation), so this entry point
takes every array from the caller and keeps its scratch (the face traces) in a fixed
static device array.  Checked through the C-ABI against kbl_traces + kbl_bounds of a
context, on two calls in a row (the second must not see the first call's scratch).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests.gpu_helpers import bounds_error, mesh_and_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


@pytest.mark.parametrize("dim,p,nu,n,precision", [
    (2, 3, (32, 32), (13, 11), 0),
    (2, 3, (32, 32), (13, 11), 1),
    (2, 2, (24, 24), (9, 7), 1),      # 24 points per axis run on the padded 32-point tile
    (1, 3, (64,), 37, 0),
    (1, 4, (200,), 23, 1),
])
def test_noalloc_matches_context_path_twice(orc, dim, p, nu, n, precision):
    """The same kernels run on the same inputs with the same launch shape, so the bounds must be
    bitwise equal to the context path's, on both calls in a row: the second call must see none
    of the first call's scratch (its traces are rewritten, its flag word cleared)."""
    import torch
    from paper_2407_20966_gb300 import kbl
    ctx = kbl.Context(dim=dim, p=p, nu=nu, precision=precision)
    for call, seed in enumerate((11, 12)):
        mesh, w = mesh_and_field(orc, dim, p, n if call == 0 else _smaller(n), seed=seed)
        ctx.mesh_upload(mesh.nbr, mesh.h, mesh.bc)
        wd = torch.from_numpy(w).cuda()
        wf = torch.zeros((ctx.nv, mesh.n_elem, ctx.nfp), dtype=torch.float64, device="cuda")
        ref = torch.zeros((2, ctx.nv, mesh.n_elem), dtype=torch.float64, device="cuda")
        ctx.traces(wd, wf)
        ctx.bounds(wd, wf, ref)
        got = torch.full_like(ref, float("nan"))
        nbr = torch.from_numpy(np.ascontiguousarray(mesh.nbr, dtype=np.int32)).cuda()
        bc = torch.from_numpy(np.ascontiguousarray(mesh.bc)).cuda()
        kbl.bounds_noalloc(ctx.cfg, nbr, bc, wd, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (call, bounds_error(got.cpu().numpy(), ref.cpu().numpy()).max())


def _smaller(n):
    """A smaller mesh for the second call, so that stale traces of the first call would be read
    if the second call did not rewrite them."""
    return (n[0] - 2, n[1] - 1) if isinstance(n, tuple) else n - 5


def test_noalloc_rejects_what_kbl_create_rejects(orc):
    """Both entry points accept the same configurations (plus: the trapezoidal rule only)."""
    import torch
    from paper_2407_20966_gb300 import kbl
    nbr = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    bc = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    w = torch.ones((4, 1, 16), dtype=torch.float64, device="cuda")
    bnd = torch.zeros((2, 4, 1), dtype=torch.float64, device="cuda")
    for field, val in (("uncoupled", 2), ("flux", 3), ("eps_rule", 5), ("precision", 7), ("quadrature", 1),
                       ("gamma", 1.0)):
        cfg = kbl.KblConfig()
        kbl.load().kbl_config_default(kbl.C.byref(cfg), 2, 3)
        setattr(cfg, field, val)
        with pytest.raises(kbl.KblError) as ei:
            kbl.bounds_noalloc(cfg, nbr, bc, w, bnd)
        assert ei.value.status == kbl.EINVAL, field


def test_noalloc_rejects_sizes_beyond_its_scratch(orc):
    import torch
    from paper_2407_20966_gb300 import kbl
    cfg = kbl.KblConfig()
    kbl.load().kbl_config_default(kbl.C.byref(cfg), 2, 3)
    E = (1 << 20) // (4 * 16) + 1          # one element more than the static scratch holds
    nbr = torch.zeros((E, 4), dtype=torch.int32, device="cuda")
    bc = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    w = torch.zeros((4, E, 16), dtype=torch.float64, device="cuda")
    bnd = torch.zeros((2, 4, E), dtype=torch.float64, device="cuda")
    with pytest.raises(kbl.KblError) as ei:
        kbl.bounds_noalloc(cfg, nbr, bc, w, bnd)
    assert ei.value.status == kbl.EINVAL
