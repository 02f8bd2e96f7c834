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

from tests.gpu_helpers import TOL_FP32, TOL_FP64, bounds_error, mesh_and_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20966_gb300 import build
    build.build()


@pytest.mark.parametrize("dim,p,nu,n,precision,tol", [
    (2, 3, (32, 32), (13, 11), 0, TOL_FP64),
    (2, 3, (32, 32), (13, 11), 1, TOL_FP32),
    (1, 3, (64,), 37, 0, TOL_FP64),
])
def test_noalloc_matches_context_path_twice(orc, dim, p, nu, n, precision, tol):
    import torch
    from paper_2407_20966_gb300 import kbl
    ctx = kbl.Context(dim=dim, p=p, nu=nu, precision=precision)
    for call, seed in enumerate((11, 12)):
        mesh, w = mesh_and_field(orc, dim, p, n, seed=seed)
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
        err = bounds_error(got.cpu().numpy(), ref.cpu().numpy())
        assert err.max() < tol, (call, err.max())


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
