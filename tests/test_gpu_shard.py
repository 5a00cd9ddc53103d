"""The z-slab decomposition through the C ABI (fdtd_step on each slab,
fdtd_planes_get / fdtd_planes_set for the ghost planes) on one GPU: the
ranks' slabs are stepped one after the other in this process and the host
copies the boundary planes between the launches (no kernel waits on another),
against the one-grid fdtd_step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import shard  # noqa: E402
from tests.helpers import drive, ragged_grid  # noqa: E402


@pytest.mark.parametrize("world,prec,tol", [(2, "f64", 1e-12), (3, "f64", 1e-12), (3, "f32", 1e-5)])
def test_slabs_on_gpu_match_one_grid(world, prec, tol):
    g = ragged_grid(41, 19, 23, seed=101)
    full = F.Grid(g, prec)
    dt = 0.95 * full.cfl_dt()
    dtype = torch.float64 if prec == "f64" else torch.float32
    u = torch.tensor(drive(g, dt, 80), dtype=dtype, device="cuda")
    yref = full.step(dt, u, reset=True)
    fref = full.fields()
    slabs = [shard.local_slab(g, world, r) for r in range(world)]
    loc = [shard.GridSlab(sl.spec, prec, dt) for sl in slabs]
    y = torch.zeros_like(yref)
    for n in range(u.shape[0]):
        for r in range(world):
            y[n] += loc[r].step(u[n:n + 1])[0]
        # exchange: each rank's first / last owned plane into its neighbours' ghosts
        sends = []
        for r, sl in enumerate(slabs):
            nzl = sl.spec.nz
            if sl.lo:
                sends.append((r - 1, loc[r - 1].grid.spec.nz - 1, loc[r].planes(sl.lo, 1)))
            if sl.hi:
                sends.append((r + 1, 0, loc[r].planes(nzl - 1 - sl.hi, 1)))
        for r, k, f in sends:
            loc[r].set_planes(k, f)
    scale = float(yref.abs().max())
    assert float((y - yref).abs().max()) <= tol * scale
    for r, sl in enumerate(slabs):
        own = loc[r].planes(sl.lo, sl.k1 - sl.k0)
        ref = fref[:, sl.k0:sl.k1]
        assert float((own - ref).abs().max()) <= tol * float(fref.abs().max()), r
