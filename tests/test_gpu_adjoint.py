"""The discrete adjoint on the GPU (fdtd_adjoint, through the C ABI) against
the FP64 oracle adjoint, against central differences of the GPU forward run,
across checkpoint counts and leap-frog kernel forms, and through the
torch.autograd binding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as oadj  # noqa: E402
from oracle import yee  # noqa: E402
from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import workloads as W  # noqa: E402
from tests.helpers import drive, ragged_grid  # noqa: E402


def _loss_grad_gpu(grid, prec, dt, u, kernel="auto", ncheck=0):
    g = F.Grid(grid, prec)
    g.set_kernel(kernel)
    ut = torch.tensor(u, dtype=g.dtype, device="cuda")
    y = g.step(dt, ut, reset=True)
    L = float((y.double() ** 2).sum()) * dt
    gy = (2.0 * dt) * y
    gc, gm = g.adjoint(dt, ut, gy, ncheckpoints=ncheck)
    torch.cuda.synchronize()
    return g, L, gc.cpu().numpy().ravel(), gm.cpu().numpy()


def _oracle_grad(grid, dt, u):
    s = yee.assemble(grid)
    y, _, _ = yee.Stepper(s, dt).run(u)
    L, dLdy = oadj.probe_energy_loss(y, dt)
    return L, oadj.grad_eps_cells(s, dt, u, dLdy)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("kernel", ["split", "persist", "fused", "march"])
def test_adjoint_f64_matches_oracle(kernel):
    grid = ragged_grid(nx=13, ny=11, nz=9, seed=31)
    dt = 0.95 * yee.cfl_dt(grid)
    u = drive(grid, dt, 150)
    Lo, go = _oracle_grad(grid, dt, u)
    _, L, gc, gm = _loss_grad_gpu(grid, "f64", dt, u, kernel)
    assert abs(L - Lo) <= 1e-10 * abs(Lo)
    assert np.max(np.abs(gc - go)) <= 1e-8 * np.abs(go).max()
    # per material = sum over its cells
    ids = grid.mat_id.ravel().astype(np.int64)
    gm_ref = np.bincount(ids, weights=gc, minlength=grid.nmat)
    assert np.allclose(gm, gm_ref, rtol=1e-10, atol=1e-14 * np.abs(gm_ref).max())


def test_adjoint_f32_matches_oracle():
    grid = ragged_grid(nx=24, ny=13, nz=11, seed=32)
    dt = 0.95 * yee.cfl_dt(grid)
    u = drive(grid, dt, 200)
    _, go = _oracle_grad(grid, dt, u)
    _, _, gc, _ = _loss_grad_gpu(grid, "f32", dt, u)
    assert _rel(gc, go) <= 2e-3


def test_checkpoint_count_does_not_change_the_gradient():
    grid = ragged_grid(nx=12, ny=10, nz=8, seed=33)
    dt = 0.9 * yee.cfl_dt(grid)
    u = drive(grid, dt, 97)
    ref = None
    for K in (1, 4, 0, 97):
        _, _, gc, _ = _loss_grad_gpu(grid, "f64", dt, u, ncheck=K)
        if ref is None:
            ref = gc
        else:
            assert np.max(np.abs(gc - ref)) <= 1e-12 * np.abs(ref).max(), K


def test_adjoint_matches_central_differences_of_gpu_forward():
    grid = ragged_grid(nx=14, ny=9, nz=10, seed=34)
    dt = 0.9 * yee.cfl_dt(grid)
    u = drive(grid, dt, 120)
    g, _, _, gm = _loss_grad_gpu(grid, "f64", dt, u)
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    ids = np.unique(grid.mat_id)
    live = [m for m in ids if not grid.pec[m]]
    rng = np.random.default_rng(3)
    for m in rng.choice(live, min(4, len(live)), replace=False):
        h = 1e-6 * grid.eps_r[m]
        Ls = []
        for sgn in (1, -1):
            e = grid.eps_r.copy()
            e[m] += sgn * h
            g.set_materials(e)
            y = g.step(dt, ut, reset=True)
            Ls.append(float((y ** 2).sum()) * dt)
        fd = (Ls[0] - Ls[1]) / (2 * h)
        assert abs(fd - gm[m]) <= 1e-5 * max(abs(gm).max(), 1e-300), (m, fd, gm[m])
    g.set_materials(grid.eps_r)


def test_autograd_binding():
    grid = ragged_grid(nx=12, ny=9, nz=8, seed=35)
    dt = 0.9 * yee.cfl_dt(grid)
    u = drive(grid, dt, 80)
    g = F.Grid(grid, "f64")
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    eps = torch.tensor(grid.eps_r, dtype=torch.float64, requires_grad=True)
    y = F.probe_response(g, eps, dt, ut)
    loss = (y ** 2).sum() * dt
    loss.backward()
    _, _, _, gm = _loss_grad_gpu(grid, "f64", dt, u)
    assert np.allclose(eps.grad.numpy(), gm, rtol=1e-10, atol=1e-14 * np.abs(gm).max())


def test_metascreen_downscale_gradient_against_oracle():
    """The 48x48x16 metascreen (8x8 design pixels of 6x6x2 cells) with a
    short broadband pulse: per-pixel FP32 GPU gradient against the FP64
    oracle gradient summed over each pixel's cells."""
    wl = W.metascreen_workload(downscale=True)
    grid = wl.grid
    dt = wl.s_ref * yee.cfl_dt(grid)
    u = W.excitation(grid, 30e9, 60e9, dt, 400)
    _, go = _oracle_grad(grid, dt, u)
    _, _, _, gm = _loss_grad_gpu(grid, "f32", dt, u)
    ids = grid.mat_id.ravel().astype(np.int64)
    gm_ref = np.bincount(ids, weights=go, minlength=grid.nmat)
    pix = np.arange(2, grid.nmat)
    assert _rel(gm[pix], gm_ref[pix]) <= 2e-3


def test_metascreen_full_size_central_differences():
    """384x384x64 metascreen, 2048 FP32 steps with the default sqrt(T)
    checkpoints: adjoint per-pixel gradient against central differences
    (relative step 1e-2) of the FP32 forward loss on 16 seeded pixels."""
    wl = W.metascreen_workload()
    grid = wl.grid
    g = F.Grid(grid, "f32")
    dt = wl.s_ref * g.cfl_dt()
    n = wl.nsteps_ref
    ut = torch.tensor(W.excitation(grid, wl.f0, wl.bw, dt, n), dtype=torch.float32, device="cuda")
    y = g.step(dt, ut, reset=True)
    gy = (2.0 * dt) * y
    _, gm = g.adjoint(dt, ut, gy, per_cell=False)
    gm = gm.cpu().numpy()
    rng = np.random.default_rng(20140630)
    pix = rng.choice(np.arange(2, grid.nmat), 16, replace=False)
    fd = []
    for m in pix:
        h = 1e-2 * grid.eps_r[m]
        Ls = []
        for sgn in (1, -1):
            e = grid.eps_r.copy()
            e[m] += sgn * h
            g.set_materials(e)
            yy = g.step(dt, ut, reset=True)
            Ls.append(float((yy.double() ** 2).sum()) * dt)
        fd.append((Ls[0] - Ls[1]) / (2 * h))
    fd = np.array(fd)
    assert _rel(gm[pix], fd) <= 5e-2, (gm[pix], fd)


def _oracle_basis_from_gpu(sys, basis, spec):
    """The GPU basis columns in the oracle's unknown order (live E / H edges)."""
    nz, ny, nx = spec.nz, spec.ny, spec.nx
    zero = np.zeros((nz, ny, nx))
    out = []
    for which, keys in ((1, ("Ex", "Ey", "Ez")), (2, ("Hx", "Hy", "Hz"))):
        V = basis.V(which).double().cpu().numpy().reshape(-1, 3, nz, ny, nx)
        cols = []
        for col in V:
            d = {k: zero for k in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")}
            d.update({keys[c]: col[c] for c in range(3)})
            x = sys.from_arrays(d)
            cols.append(x[:sys.Ne] if which == 1 else x[sys.Ne:])
        out.append(np.stack(cols, axis=1))
    return out


@pytest.mark.parametrize("prec,tol", [("f64", 1e-8), ("f32", 2e-3)])
def test_reduced_model_gradient_matches_oracle(prec, tol):
    """mor_gradient (basis frozen) against the oracle's reduced-model adjoint
    on the same basis: dL/dD~eps and the per-cell gradient."""
    from oracle import mor
    g = ragged_grid(nx=14, ny=10, nz=9, seed=36)
    grid = F.Grid(g, prec)
    dt0 = 0.99 * grid.cfl_dt()
    basis = F.Basis(grid, 12, dt0, L=1, M=1.1, fmax=40e9, tol=1e-10 if prec == "f64" else 1e-6, defl_tol=1e-6)
    model = F.Model(grid, basis)
    assert model.perturb(dt0) == 0
    T = 150
    u = drive(g, dt0, T)
    ut = torch.tensor(u, dtype=grid.dtype, device="cuda")
    y = model.run(ut)
    gy = (2.0 * dt0) * y
    gc, gm, gD = model.gradient(basis, ut, gy)
    sys = yee.assemble(g)
    V1, V2 = _oracle_basis_from_gpu(sys, basis, g)
    red = mor.project(sys, V1, V2)
    yo = mor.reduced_run(red, dt0, u)
    Go = oadj.reduced_grad_De(red, dt0, u, 2.0 * dt0 * yo)
    gco = oadj.reduced_grad_eps_cells(sys, V1, Go)
    assert _rel(gD, Go) <= tol
    assert np.max(np.abs(gc.cpu().numpy().ravel() - gco)) <= tol * np.abs(gco).max()
    ids = g.mat_id.ravel().astype(np.int64)
    gm_ref = np.bincount(ids, weights=gc.cpu().numpy().ravel(), minlength=g.nmat)
    assert np.allclose(gm.cpu().numpy(), gm_ref, rtol=1e-9, atol=1e-12 * np.abs(gm_ref).max())
