"""Batched stepping (fdtd_step_batched) and the tile autotuner, through the
C ABI: every grid of a batch advances exactly as it does alone, and a tuned
grid still matches the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import yee  # noqa: E402
from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import workloads as W  # noqa: E402
from tests.helpers import drive, oracle_state_to_arrays, ragged_grid  # noqa: E402


def _specs():
    """Uneven grids: ragged widths (1, 2, 4 cells per thread), uint8 and
    uint16 ids, uniform and non-uniform mu, a grid without sources."""
    out = [ragged_grid(nx=41, ny=19, nz=23, seed=51),
           ragged_grid(nx=64, ny=12, nz=10, seed=52, many_materials=True),
           ragged_grid(nx=128, ny=10, nz=10, seed=53, magnetic=False),
           ragged_grid(nx=30, ny=9, nz=10, seed=54)]
    out[3].ports = []
    return out


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("nsteps", [7, 70])
def test_batched_equals_separate_runs(prec, nsteps):
    specs = _specs()
    dts = [0.93 * yee.cfl_dt(s) for s in specs]
    us_np = [drive(s, dt, nsteps) if s.ports else None for s, dt in zip(specs, dts)]
    gb = [F.Grid(s, prec) for s in specs]
    us = [torch.tensor(u, dtype=gb[0].dtype, device="cuda") if u is not None else None for u in us_np]
    ys = F.step_batched(gb, dts, us)
    fb = [g.fields() for g in gb]
    for q, s in enumerate(specs):
        g = F.Grid(s, prec)
        g.set_kernel("split")
        y = g.step(dts[q], us[q] if us[q] is not None else torch.zeros((nsteps, 0), device="cuda"),
                   nsteps=nsteps, reset=True)
        f = g.fields()
        torch.cuda.synchronize()
        tol = 1e-5 if prec == "f32" else 1e-12
        scale = float(f.abs().max()) or 1.0
        assert float((fb[q] - f).abs().max()) <= tol * scale, q
        if y is not None:
            ysc = float(y.abs().max()) or 1.0
            assert float((ys[q] - y).abs().max()) <= tol * ysc, q


def test_batched_f64_matches_oracle_and_continues():
    specs = _specs()[:2]
    dts = [0.9 * yee.cfl_dt(s) for s in specs]
    n = 90
    us_np = [drive(s, dt, n) for s, dt in zip(specs, dts)]
    gb = [F.Grid(s, "f64") for s in specs]
    us = [torch.tensor(u, dtype=torch.float64, device="cuda") for u in us_np]
    ya = F.step_batched(gb, dts, [u[:40] for u in us])
    yb = F.step_batched(gb, dts, [u[40:] for u in us], reset=False)
    for q, s in enumerate(specs):
        sys = yee.assemble(s)
        yo, xo, _ = yee.Stepper(sys, dts[q]).run(us_np[q])
        fo = oracle_state_to_arrays(sys, xo)
        fg = gb[q].fields().cpu().numpy()
        yg = torch.cat([ya[q], yb[q]]).cpu().numpy()
        assert np.max(np.abs(fg - fo)) <= 1e-9 * np.abs(fo).max()
        assert np.max(np.abs(yg - yo)) <= 1e-9 * np.abs(yo).max()


def test_cavity_batch_workload_runs():
    """The 32 uneven cavities (24^3 .. 96^3) and the iris waveguide in one batch."""
    specs = W.cavity_batch() + [W.waveguide_iris()]
    gb = [F.Grid(s, "f32") for s in specs]
    dts = [0.99 * g.cfl_dt() for g in gb]
    n = 40
    us = [torch.tensor(W.excitation(s, 10e9, 10e9, dt, n), dtype=torch.float32, device="cuda")
          for s, dt in zip(specs, dts)]
    ys = F.step_batched(gb, dts, us)
    # spot-check two members against separate runs
    for q in (0, len(specs) - 1):
        g = F.Grid(specs[q], "f32")
        g.set_kernel("split")
        y = g.step(dts[q], us[q], reset=True)
        torch.cuda.synchronize()
        assert torch.allclose(ys[q], y, rtol=1e-5, atol=1e-5 * float(y.abs().max()))


def test_invalid_batches_are_rejected():
    s = ragged_grid(seed=55)
    g = F.Grid(s, "f32")
    u = torch.zeros((5, g.m), device="cuda")
    with pytest.raises(F.FdtdError):
        F.step_batched([g, g], [1e-13, 1e-13], [u, u])
    with pytest.raises(F.FdtdError):
        F.step_batched([g], [-1.0], [u])


def test_autotune_keeps_results_and_state():
    s = ragged_grid(nx=64, ny=16, nz=12, seed=56)
    dt = 0.9 * yee.cfl_dt(s)
    u = drive(s, dt, 100)
    g = F.Grid(s, "f64")
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    g.step(dt, ut[:30], reset=True)
    f0 = g.fields()
    vw, lz = g.autotune(dt, 20)
    assert vw in (1, 2) and 64 % vw == 0 and lz in (1, 2, 4, 8)
    assert torch.equal(g.fields(), f0)
    y = g.step(dt, ut, reset=True)
    sys = yee.assemble(s)
    yo, _, _ = yee.Stepper(sys, dt).run(u)
    assert np.max(np.abs(y.cpu().numpy() - yo)) <= 1e-9 * np.abs(yo).max()


def _reduce_specs():
    """Uneven grids for the batched reduction: ragged spacing, lossy and
    magnetic blocks, one grid of three ports."""
    out = [ragged_grid(nx=22, ny=15, nz=12, seed=61),
           ragged_grid(nx=14, ny=18, nz=10, seed=62),
           ragged_grid(nx=30, ny=11, nz=9, seed=63)]
    out[1].ports.append(W.Port.point(W.COMP_EZ, 5, 6, 4))
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_bases_equal_separate_builds(prec):
    """mor_build_basis_batched: every basis of the batch is the one its grid
    builds alone (the builds only run side by side), to rounding, and its
    projected model the same; the launches of every worker are counted."""
    specs = _reduce_specs()
    grids = [F.Grid(s, prec) for s in specs]
    tol = 1e-10 if prec == "f64" else 1e-5
    opts = [dict(q=12, dt0=0.99 * g.cfl_dt(), L=1, M=1.1, fmax=60e9, tol=tol) for g in grids]
    torch.cuda.synchronize()
    F.launch_count(reset=True)
    bs = F.build_bases(grids, opts)
    torch.cuda.synchronize()
    n_batched = F.launch_count(reset=True)
    n_alone = 0
    for g, o, b in zip(grids, opts, bs):
        a = F.Basis(g, **o)
        n_alone += F.launch_count(reset=True)
        assert b.status == a.status == F.FDTD_OK
        ib, ia = b.info(), a.info()
        assert (ib["q1"], ib["q2"]) == (ia["q1"], ia["q2"])
        assert abs(ib["max_resid"] - ia["max_resid"]) <= 0.1 * ia["max_resid"]
        for which in (1, 2):
            vb, va = b.V(which), a.V(which)
            assert float((vb - va).abs().max()) <= (1e-12 if prec == "f64" else 1e-5), which
        mb, ma = F.Model(g, b), F.Model(g, a)
        for name in ("De", "Dm", "K", "BE", "CE"):
            x, y = mb.get(name), ma.get(name)
            assert np.max(np.abs(x - y)) <= (1e-10 if prec == "f64" else 1e-4) * np.abs(y).max(), name
    assert n_batched > 0 and abs(n_batched - n_alone) <= 0.1 * n_alone, (n_batched, n_alone)


def test_batched_f64_bases_match_the_oracle():
    """Two small members of a batch, FP64: the batched bases span the oracle's
    SPRIM bases (sparse-LU chains, CGS2), principal cosines to 1e-8."""
    from oracle import mor
    specs = _reduce_specs()[:2]
    grids = [F.Grid(s, "f64") for s in specs]
    opts = [dict(q=12, dt0=0.99 * yee.cfl_dt(s), L=1, M=1.1, fmax=60e9, tol=1e-12, defl_tol=1e-6) for s in specs]
    bs = F.build_bases(grids, opts)
    for s, o, b in zip(specs, opts, bs):
        sys = yee.assemble(s)
        ob = mor.sprim_basis(sys, o["dt0"], o["q"], o["L"], o["M"], o["fmax"], defl_tol=1e-6)
        for which, comps, Vo in ((1, "E", ob.V1), (2, "H", ob.V2)):
            V = b.V(which).cpu().numpy()
            q = V.shape[0]
            nz, ny, nx = sys.shape
            A = V.reshape(q, 3, nz, ny, nx)
            masks = sys.e_mask if comps == "E" else sys.h_mask
            Vg = np.concatenate([A[:, c][:, masks[c]] for c in range(3)], axis=1).T
            assert Vg.shape[1] == Vo.shape[1]
            cosines = np.linalg.svd(Vg.T @ Vo, compute_uv=False)
            assert cosines.min() > 1 - 1e-8, (which, cosines.min())


def test_batched_bases_report_the_failing_member():
    specs = _reduce_specs()
    grids = [F.Grid(s, "f32") for s in specs]
    good = dict(q=8, dt0=0.99 * grids[0].cfl_dt(), L=1, M=1.1, fmax=60e9, tol=1e-4)
    bad = dict(good, dt0=-1.0)
    with pytest.raises(F.FdtdError, match="grid 1"):
        F.build_bases(grids, [good, bad, dict(good, dt0=0.99 * grids[2].cfl_dt())])
    with pytest.raises(F.FdtdError, match="twice"):
        F.build_bases([grids[0], grids[0]], [good, good])
    assert F.build_bases([], []) == []
