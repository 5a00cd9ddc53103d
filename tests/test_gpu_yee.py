"""Parity of the CUDA Yee leap-frog (fdtd_step, through the C ABI) with the
FP64 oracle: whole fields and probes on small ragged grids, the FP64 10^3
cavity in full, and light-cone samples of the full-size graded cavity and
metascreen grids in the launch configuration the benchmark uses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import yee  # noqa: E402
from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import workloads as W  # noqa: E402
from tests.helpers import drive, oracle_state_to_arrays, ragged_grid, subgrid  # noqa: E402

# FP32 tolerance of the full-order path: 2e-4 relative L2 on probe waveforms.
TOL_F32_PROBE = 2e-4
TOL_F64 = 1e-9


def _run_gpu(grid, prec, dt, u, reset=True, kernel="auto"):
    g = F.Grid(grid, prec)
    g.set_kernel(kernel)
    ut = torch.tensor(u, dtype=g.dtype, device="cuda")
    y = g.step(dt, ut, reset=reset)
    f = g.fields()
    torch.cuda.synchronize()
    return g, (y.cpu().numpy() if y is not None else None), f.cpu().numpy()


def _run_oracle(grid, dt, u):
    s = yee.assemble(grid)
    y, x, _ = yee.Stepper(s, dt).run(u)
    return s, y, oracle_state_to_arrays(s, x)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_cfl_matches_oracle():
    for grid in (W.cavity10_workload().grid, W.graded_cavity_workload().grid, ragged_grid()):
        g = F.Grid(grid, "f32")
        assert abs(g.cfl_dt() - yee.cfl_dt(grid)) <= 1e-15 * yee.cfl_dt(grid)


KERNEL_CASES = [("persist", 41), ("split", 41), ("fused", 41), ("march", 41), ("persist", 48), ("split", 48),
                ("tma", 48), ("march", 48)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("many", [False, True])
@pytest.mark.parametrize("kernel,nx", KERNEL_CASES)
def test_ragged_graded_lossy_parity(prec, many, kernel, nx):
    """Every kernel form on a ragged graded lossy grid.  nx = 41: x rows not
    a multiple of the 32-wide tiles; nx = 48: rows 16-byte aligned, as the
    TMA form needs (uint8 ids with few materials, uint16 with many)."""
    grid = ragged_grid(nx=nx, many_materials=many)
    dt = 0.95 * yee.cfl_dt(grid)
    u = drive(grid, dt, 160)
    g, yg, fg = _run_gpu(grid, prec, dt, u, kernel=kernel)
    g.check()
    s, yo, fo = _run_oracle(grid, dt, u)
    if prec == "f64":
        assert np.max(np.abs(fg - fo)) <= TOL_F64 * np.abs(fo).max()
        assert np.max(np.abs(yg - yo)) <= TOL_F64 * np.abs(yo).max()
    else:
        for c in range(6):
            assert _rel(fg[c], fo[c]) <= 1e-4, c
        assert _rel(yg, yo) <= TOL_F32_PROBE
    # removed unknowns (PEC / walls) are exactly zero on the GPU
    for c in range(3):
        assert np.all(fg[c][~s.e_mask[c]] == 0)
        assert np.all(fg[3 + c][~s.h_mask[c]] == 0)


def test_cavity10_f64_full_run():
    wl = W.cavity10_workload()
    dt = wl.s_ref * yee.cfl_dt(wl.grid)
    u = W.excitation(wl.grid, wl.f0, wl.bw, dt, wl.nsteps_ref)
    _, yg, fg = _run_gpu(wl.grid, "f64", dt, u)
    _, yo, fo = _run_oracle(wl.grid, dt, u)
    assert np.max(np.abs(yg - yo)) <= TOL_F64 * np.abs(yo).max()
    assert np.max(np.abs(fg - fo)) <= TOL_F64 * np.abs(fo).max()


@pytest.mark.parametrize("kernel", ["persist", "split", "fused", "march"])
def test_state_continues_across_calls_and_host_variant(kernel):
    grid = ragged_grid(seed=7)
    dt = 0.9 * yee.cfl_dt(grid)
    u = drive(grid, dt, 90)
    g = F.Grid(grid, "f32")
    g.set_kernel(kernel)
    ut = torch.tensor(u, dtype=torch.float32, device="cuda")
    y1 = g.step(dt, ut[:40], reset=True)
    y2 = g.step(dt, ut[40:], reset=False)
    f_split = g.fields().cpu().numpy()
    yall = g.step(dt, ut, reset=True)
    f_once = g.fields().cpu().numpy()
    torch.cuda.synchronize()
    # multi-edge probes are summed with atomics: equal up to summation order
    yref = yall.cpu().numpy()
    assert np.allclose(torch.cat([y1, y2]).cpu().numpy(), yref, rtol=1e-6, atol=1e-7 * np.abs(yref).max())
    assert np.array_equal(f_split, f_once)
    uh = torch.tensor(u, dtype=torch.float32).pin_memory()
    yh = torch.empty((90, g.p), dtype=torch.float32).pin_memory()
    g.step_host(dt, uh, yh, reset=True)
    assert np.allclose(yh.numpy(), yref, rtol=1e-6, atol=1e-7 * np.abs(yref).max())
    g.check()


def test_kernel_forms_agree_and_persistent_chunks():
    """8200 steps cross the persistent form's 8192-step launch boundary; the
    FP64 result must equal the oracle's and the other forms' results."""
    grid = ragged_grid(nx=12, ny=10, nz=9, seed=11)
    dt = 0.97 * yee.cfl_dt(grid)
    u = drive(grid, dt, 8200)
    _, yo, fo = _run_oracle(grid, dt, u)
    for kernel in ("persist", "split", "fused", "march"):
        g, yg, fg = _run_gpu(grid, "f64", dt, u, kernel=kernel)
        g.check()
        assert np.max(np.abs(fg - fo)) <= 1e-8 * np.abs(fo).max(), kernel
        assert np.max(np.abs(yg - yo)) <= 1e-8 * np.abs(yo).max(), kernel


@pytest.mark.parametrize("kernel", ["split", "fused", "march"])
def test_graph_replays_follow_parity_and_dt(kernel):
    """Runs long enough to be replayed from captured graphs: an odd-length
    call first (the next replays start from the other buffer), then a new dt
    (the captured coefficients must not be reused); results equal a fresh
    grid's run of the same steps."""
    grid = ragged_grid(nx=48, seed=13)
    dt1, dt2 = 0.9 * yee.cfl_dt(grid), 0.7 * yee.cfl_dt(grid)
    u = drive(grid, dt2, 150)
    ut = torch.tensor(u, dtype=torch.float32, device="cuda")
    g = F.Grid(grid, "f32")
    g.set_kernel(kernel)
    g.step(dt1, ut[:77], reset=True)
    g.step(dt1, ut, reset=True)
    y = g.step(dt2, ut, reset=True)
    f = g.fields()
    h = F.Grid(grid, "f32")
    h.set_kernel(kernel)
    y_ref = h.step(dt2, ut, reset=True)
    f_ref = h.fields()
    torch.cuda.synchronize()
    assert torch.equal(f, f_ref)
    assert torch.allclose(y, y_ref, rtol=1e-6, atol=1e-7 * float(y_ref.abs().max()))


def test_set_kernel_rejects_bad_values():
    g = F.Grid(ragged_grid(nx=41), "f32")
    with pytest.raises(F.FdtdError):
        g.set_kernel("tma")              # 41 is not a multiple of 16
    with pytest.raises(F.FdtdError):
        F.check(F.lib().fdtd_grid_set_kernel(g.h, 9))


def test_degenerate_grids_and_empty_ports():
    for (nx, ny, nz) in [(1, 1, 1), (1, 5, 3), (33, 1, 2), (2, 9, 1)]:
        eps, mu, se, sm, pec = W.vacuum_table()
        grid = W.GridSpec(nx, ny, nz, np.full(nx, 1e-3), np.full(ny, 1e-3), np.full(nz, 1e-3),
                          eps, mu, se, sm, pec, np.zeros((nz, ny, nx), np.uint16))
        g = F.Grid(grid, "f32")
        y = g.step(1e-13, torch.zeros((5, 0), device="cuda"), nsteps=5)
        assert y is None
        f = g.fields()
        torch.cuda.synchronize()
        assert torch.count_nonzero(f).item() == 0
    grid = ragged_grid(seed=9)
    g = F.Grid(grid, "f32")
    y = g.step(0.5 * g.cfl_dt(), torch.zeros((0, g.m), device="cuda"), nsteps=0)
    assert y.shape == (0, g.p)


def test_invalid_arguments_are_rejected():
    grid = ragged_grid(seed=3)
    g = F.Grid(grid, "f32")
    with pytest.raises(F.FdtdError) as e:
        g.step(-1.0, torch.zeros((3, g.m), device="cuda"))
    assert e.value.status == F.FDTD_EINVAL
    bad = ragged_grid(seed=3)
    bad.mat_id = bad.mat_id.copy()
    bad.mat_id[0, 0, 0] = bad.nmat
    with pytest.raises(F.FdtdError):
        F.Grid(bad, "f32")


def _light_cone_check(grid, prec, dt, nsteps, centres, half):
    """GPU run on the full grid vs the oracle on a sub-grid around each centre:
    after n steps a field value depends only on data within n+1 cells, so the
    sub-grid's own PEC walls (n+2 cells away) cannot reach the sampled block."""
    u = drive(grid, dt, nsteps, f0=10e9, bw=10e9)
    _, yg, fg = _run_gpu(grid, prec, dt, u)
    r = nsteps + 2
    for (ci, cj, ck) in centres:
        lo = (max(0, ci - half - r), max(0, cj - half - r), max(0, ck - half - r))
        hi = (min(grid.nx, ci + half + r + 1), min(grid.ny, cj + half + r + 1), min(grid.nz, ck + half + r + 1))
        sg = subgrid(grid, lo, hi)
        us = u[:, :len(sg.ports)] if sg.ports else np.zeros((nsteps, 0))
        s = yee.assemble(sg)
        _, xs, _ = yee.Stepper(s, dt).run(us if sg.ports else np.zeros((nsteps, 0)))
        fo = oracle_state_to_arrays(s, xs)
        sl = (slice(None), slice(ck - half - lo[2], ck + half + 1 - lo[2]),
              slice(cj - half - lo[1], cj + half + 1 - lo[1]), slice(ci - half - lo[0], ci + half + 1 - lo[0]))
        gsl = (slice(None), slice(ck - half, ck + half + 1), slice(cj - half, cj + half + 1),
               slice(ci - half, ci + half + 1))
        a, b = fg[gsl], fo[sl]
        scale = max(np.abs(fo).max(), 1e-30)
        assert np.max(np.abs(a - b)) <= (1e-4 if prec == "f32" else 1e-10) * scale


def test_full_size_graded_cavity_light_cone():
    wl = W.graded_cavity_workload()
    grid = wl.grid
    dt = wl.s_ref * yee.cfl_dt(grid)
    p = grid.ports[0]
    centres = [(int(p.i[0]), int(p.j[0]), int(p.k[0])), (32, 32, 32), (60, 3, 40)]
    _light_cone_check(grid, "f32", dt, 12, centres, 3)


def test_full_size_metascreen_light_cone():
    wl = W.metascreen_workload()
    grid = wl.grid
    dt = wl.s_ref * yee.cfl_dt(grid)
    centres = [(192, 192, 9), (70, 300, 31), (383 - 5, 5, 8)]
    _light_cone_check(grid, "f32", dt, 10, centres, 3)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 2e-4)])
def test_absorbing_microstrip_parity(prec, tol):
    """The 100x50x24 microstrip with the matched absorber on five faces
    (graded sigma_e and sigma_m, uint8 ids): whole fields and probes against
    the oracle."""
    wl = W.microstrip_workload(downscale=True, absorbing=True)
    grid = wl.grid
    dt = wl.s_ref * yee.cfl_dt(grid)
    u = W.excitation(grid, wl.f0, wl.bw, dt, 300)
    _, yg, fg = _run_gpu(grid, prec, dt, u)
    _, yo, fo = _run_oracle(grid, dt, u)
    if prec == "f64":
        assert np.max(np.abs(fg - fo)) <= tol * np.abs(fo).max()
        assert np.max(np.abs(yg - yo)) <= tol * np.abs(yo).max()
    else:
        assert _rel(yg, yo) <= tol
        for c in range(6):
            assert _rel(fg[c], fo[c]) <= 10 * tol, c


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_edge_coefficient_map_is_bit_exact(monkeypatch, prec):
    """The split form's E launch with the per-edge coefficient map (the small
    grid default) and with the per-cell material lookups give the same fields,
    also after the materials change (the map follows the table): bit-exact in
    FP64; in FP32 the compiler may contract the coefficient arithmetic
    differently in the two contexts, so within a few FP32 roundings."""
    grid = ragged_grid(nx=26, ny=15, nz=12, seed=71)
    dt = 0.95 * yee.cfl_dt(grid)
    u = drive(grid, dt, 90)
    out = {}
    for pre in ("0", "1"):
        monkeypatch.setenv("FDTDMOR_PRECOEF", pre)
        g = F.Grid(grid, prec)
        g.set_kernel("split")
        ut = torch.tensor(u, dtype=g.dtype, device="cuda")
        y1 = g.step(dt, ut, reset=True)
        eps = grid.eps_r.copy()
        eps[1:] *= 1.3
        g.set_materials(eps)
        y2 = g.step(dt, ut, reset=True)
        out[pre] = (y1.cpu().numpy(), y2.cpu().numpy(), g.fields().cpu().numpy())
    for a, b in zip(out["0"], out["1"]):
        if prec == "f64":
            assert np.array_equal(a, b)
        else:
            assert np.max(np.abs(a - b)) <= 1e-5 * np.abs(b).max()
    assert np.max(np.abs(out["1"][0] - out["1"][1])) > 1e-3 * np.abs(out["1"][0]).max()


@pytest.mark.parametrize("staged", ["1", "0"])
@pytest.mark.parametrize("many", [False, True])
@pytest.mark.parametrize("nx", [48, 272])
def test_march_four_cells_per_thread(monkeypatch, staged, many, nx):
    """The fused one-pass form with 4 FP32 cells per thread, its plane inputs
    staged through shared memory by TMA or loaded per thread: parity with the
    oracle on one tile (nx = 48) and on three tiles with a ragged last one
    (nx = 272: +x halo columns between tiles), uint8 and uint16 ids."""
    monkeypatch.setenv("FDTDMOR_MARCH_VW", "4")
    monkeypatch.setenv("FDTDMOR_MARCH_TMA", staged)
    grid = ragged_grid(nx=nx, ny=13, nz=9, many_materials=many)
    dt = 0.95 * yee.cfl_dt(grid)
    u = drive(grid, dt, 120)
    g, yg, fg = _run_gpu(grid, "f32", dt, u, kernel="march")
    g.check()
    s, yo, fo = _run_oracle(grid, dt, u)
    for c in range(6):
        assert _rel(fg[c], fo[c]) <= 1e-4, c
    assert _rel(yg, yo) <= TOL_F32_PROBE
    for c in range(3):
        assert np.all(fg[c][~s.e_mask[c]] == 0)
        assert np.all(fg[3 + c][~s.h_mask[c]] == 0)


@pytest.mark.parametrize("kernel", ["march", "tma"])
def test_tensor_maps_follow_a_new_grid_at_reused_addresses(monkeypatch, kernel):
    """The TMA-fed forms cache their tensor maps per grid; a second grid with
    the same cell count (so the allocator hands back the same device blocks)
    but other row lengths must get maps of its own shape."""
    monkeypatch.setenv("FDTDMOR_MARCH_VW", "4")
    monkeypatch.setenv("FDTDMOR_MARCH_TMA", "1")
    first = ragged_grid(nx=48, ny=26, nz=9, seed=81)
    dt1 = 0.95 * yee.cfl_dt(first)
    g1, _, _ = _run_gpu(first, "f32", dt1, drive(first, dt1, 40), kernel=kernel)
    g1.check()
    g1.close()
    del g1
    second = ragged_grid(nx=96, ny=13, nz=9, seed=82)
    dt = 0.95 * yee.cfl_dt(second)
    u = drive(second, dt, 100)
    g, yg, fg = _run_gpu(second, "f32", dt, u, kernel=kernel)
    g.check()
    _, yo, fo = _run_oracle(second, dt, u)
    for c in range(6):
        assert _rel(fg[c], fo[c]) <= 1e-4, c
    assert _rel(yg, yo) <= TOL_F32_PROBE


@pytest.mark.parametrize("case", ["gathered", "probe_on_source", "two_ports_one_edge"])
def test_march_source_terms_against_oracle(case):
    """The fused z-march form applies sources and probes after its pass from
    terms gathered per field value: in one launch (case "gathered"), with the
    probes in a second launch when a probe edge carries a source term, and
    with the atomic source kernel when two ports drive one edge.  FP64 fields
    and probes against the oracle."""
    g = ragged_grid(nx=24, ny=14, nz=10, seed=77)
    p0 = g.ports[0]
    if case == "probe_on_source":
        g.probes.append(W.Port.point(p0.comp, int(p0.i[0]), int(p0.j[0]), int(p0.k[0]), 0.7))
    elif case == "two_ports_one_edge":
        g.ports.append(W.Port.point(p0.comp, int(p0.i[0]), int(p0.j[0]), int(p0.k[0]), -0.4))
    dt = 0.95 * yee.cfl_dt(g)
    u = drive(g, dt, 120)
    _, yg, fg = _run_gpu(g, "f64", dt, u, kernel="march")
    _, yo, fo = _run_oracle(g, dt, u)
    assert np.max(np.abs(fg - fo)) <= TOL_F64 * np.abs(fo).max()
    assert np.max(np.abs(yg - yo)) <= TOL_F64 * np.abs(yo).max()
