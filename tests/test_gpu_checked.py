"""The checked build (paper_1406_7042_gb300.build with checked=True, loaded
with FDTDMOR_CHECKED=1) runs the hot path with a device synchronisation after
every launch, no CUDA graphs and the port-list index checks, and gives the
same results: a leap-frog run against the FP64 oracle, the fused z-march form
with a plane of sources, and a reduction with its reduced run, each followed
by a clean fdtd_check.  Run in a child process, since one process loads one
library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
from oracle import yee, mor
from paper_1406_7042_gb300 import fdtdmor as F
from paper_1406_7042_gb300 import workloads as W
from tests.helpers import drive, ragged_grid
assert F.LIB_PATH.endswith("libfdtdmor_checked.so")
g = ragged_grid(nx=40, ny=13, nz=11, seed=71)
dt = 0.95 * yee.cfl_dt(g)
u = drive(g, dt, 300)
grid = F.Grid(g, "f64")
y = grid.step(dt, torch.tensor(u, device="cuda"), reset=True).cpu().numpy()
grid.check()
yo = yee.Stepper(yee.assemble(g), dt).run(u)[0]
assert mor.rel_l2(y, yo) < 1e-10, mor.rel_l2(y, yo)
wl = W.metascreen_workload(downscale=True)
gm = F.Grid(wl.grid, "f32")
gs = F.Grid(wl.grid, "f32")
gm.set_kernel("march"); gs.set_kernel("split")
dtm = 0.99 * gm.cfl_dt()
um = torch.tensor(W.excitation(wl.grid, wl.f0, wl.bw, dtm, 200), dtype=torch.float32, device="cuda")
ym, ys = gm.step(dtm, um, reset=True), gs.step(dtm, um, reset=True)
gm.check(); gs.check()
assert float((ym - ys).abs().max()) <= 1e-5 * float(ys.abs().max())
g32 = F.Grid(g, "f32")
b = F.Basis(g32, 12, dt, 1, 1.1, 60e9, tol=1e-5)
m = F.Model(g32, b)
m.perturb(3 * dt)
yr = m.run(torch.tensor(drive(g, 3 * dt, 100), dtype=torch.float32, device="cuda"))
assert torch.isfinite(yr).all()
g32.check()
print("checked build ok")
'''


def test_checked_build_runs_the_hot_path():
    from paper_1406_7042_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, FDTDMOR_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
