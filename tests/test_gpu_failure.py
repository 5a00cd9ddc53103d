"""Failure detection on the GPU in forms that fault, trap or hang nothing:
the field watchdog of fdtd_step on a leap-frog run beyond its stability limit
(Eq. (singular_limit)), a bounded completion-counter wait of the dataflow form
made to run out, and a device allocator that refuses every request."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import yee  # noqa: E402
from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import workloads as W  # noqa: E402
from tests.helpers import oracle_state_to_arrays, ragged_grid  # noqa: E402


def _source_free_box():
    """A 12 x 10 x 8 vacuum PEC box without sources, one probe, and a seeded
    initial state on the live edges only."""
    eps, mu, se, sm, pec = W.vacuum_table()
    g = W.GridSpec(12, 10, 8, np.full(12, 1e-3), np.full(10, 1e-3), np.full(8, 1e-3), eps, mu, se, sm, pec,
                   np.zeros((8, 10, 12), np.uint16))
    g.probes.append(W.Port.point(W.COMP_EZ, 5, 4, 3))
    s = yee.assemble(g)
    x0 = np.random.default_rng(11).standard_normal(s.N)
    x0[s.Ne:] /= np.sqrt(yee.MU0 / yee.EPS0)  # H in proportion to E (impedance of free space)
    return g, s, oracle_state_to_arrays(s, x0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_watchdog_flags_run_beyond_stability_limit(prec):
    g, s, f0 = _source_free_box()
    dt_max = yee.exact_dt_limit(s)
    grid = F.Grid(g, prec)
    dtype = torch.float64 if prec == "f64" else torch.float32
    ft = torch.tensor(f0, dtype=dtype, device="cuda")
    # stable: 0.99 of the CFL step, source-free energy checked (growth 10x)
    grid.set_watchdog(True, growth=10.0, sync=True)
    grid.set_fields(ft)
    grid.step(0.99 * grid.cfl_dt(), None, nsteps=2000)
    grid.check()
    # beyond the exact limit: the energy grows without sources -> FDTD_EUNSTABLE from step
    grid.set_fields(ft)
    with pytest.raises(F.FdtdError) as e:
        grid.step(1.2 * dt_max, None, nsteps=200)
    assert e.value.status == F.FDTD_EUNSTABLE
    grid.check()  # the flag was cleared by the failing call
    # default mode (asynchronous, NaN/Inf only): the run overflows, step returns,
    # fdtd_check reports it
    grid.set_watchdog(True)
    grid.set_fields(ft)
    grid.step(1.5 * dt_max, None, nsteps=6000)
    with pytest.raises(F.FdtdError) as e:
        grid.check()
    assert e.value.status == F.FDTD_EUNSTABLE
    # the handle stays usable: a stable run afterwards is clean
    grid.set_fields(ft)
    grid.step(0.99 * grid.cfl_dt(), None, nsteps=100)
    grid.check()
    assert torch.isfinite(grid.fields()).all()


def test_dataflow_wait_limit_reports_etimeout():
    """A wait limit of zero polls makes the first completion-counter wait that
    is not already satisfied give up: the kernel sets the flag and returns,
    fdtd_check reports FDTD_ETIMEOUT, and with the default limit restored the
    same grid steps like the split form."""
    g = ragged_grid(48, 40, 36, seed=21)
    dt = 0.9 * yee.cfl_dt(g)
    u = torch.tensor(W.excitation(g, 40e9, 60e9, dt, 400) * np.ones((1, len(g.ports))), dtype=torch.float32,
                     device="cuda")
    ref = F.Grid(g, "f32")
    ref.set_kernel("split")
    yref = ref.step(dt, u, reset=True)
    grid = F.Grid(g, "f32")
    grid.set_kernel("persist")
    grid.set_wait_limit(0)
    timed_out = False
    for _ in range(3):
        grid.step(dt, u, reset=True)
        try:
            grid.check()
        except F.FdtdError as e:
            assert e.status == F.FDTD_ETIMEOUT
            timed_out = True
            break
    assert timed_out
    grid.set_wait_limit(-1)
    y = grid.step(dt, u, reset=True)
    grid.check()
    assert torch.allclose(y, yref, rtol=0, atol=2e-4 * float(yref.abs().max()))


def test_refusing_allocator_reports_enomem_and_handle_survives():
    """Every device allocation refused (the hook returns NULL): a basis build
    that needs new buffers fails with FDTD_ENOMEM; with the PyTorch allocator
    back, the same grid steps and builds a basis."""
    g = ragged_grid(29, 17, 13, seed=31)
    grid = F.Grid(g, "f32")
    dt = 0.99 * grid.cfl_dt()
    u = torch.tensor(W.excitation(g, 40e9, 60e9, dt, 50) * np.ones((1, len(g.ports))), dtype=torch.float32,
                     device="cuda")
    grid.step(dt, u, reset=True)
    L = F.lib()

    def refuse(nbytes, stream):
        return None

    def release(ptr, stream):  # everything alive came from PyTorch's allocator
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    cbs = (F.ALLOC_FN(refuse), F.FREE_FN(release))
    assert L.fdtd_set_allocator(*cbs) == F.FDTD_OK
    try:
        with pytest.raises(F.FdtdError) as e:
            F.Basis(grid, 8, dt, 1, 1.1, 60e9)
        assert e.value.status == F.FDTD_ENOMEM
    finally:
        F._install_torch_allocator()
    y = grid.step(dt, u, reset=True)
    grid.check()
    assert torch.isfinite(y).all()
    b = F.Basis(grid, 8, dt, 1, 1.1, 60e9, tol=1e-5)
    assert b.info()["q1"] > 0
