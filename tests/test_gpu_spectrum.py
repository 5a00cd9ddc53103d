"""fdtd_dft and fdtd_resonances through the C ABI against the spectrum
oracle, and on the GPU FDTD of the paper's demo cavity (Sec. III-B) against
the printed resonances."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import spectrum, yee  # noqa: E402
from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import workloads as W  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-11)])
@pytest.mark.parametrize("hann", [False, True])
def test_dft_matches_oracle(dtype, tol, hann):
    rng = np.random.default_rng(5)
    N, p, dt = 5000, 3, 1.3e-12
    y = rng.standard_normal((N, p)).astype(np.float64 if dtype == torch.float64 else np.float32)
    f = np.linspace(1e9, 60e9, 257)
    got = F.dft(torch.tensor(y, device="cuda"), dt, f, hann)
    ref = spectrum.dft(y.astype(np.float64), dt, f, hann)
    assert np.max(np.abs(got - ref)) <= tol * np.abs(ref).max()


def test_demo_cavity_resonances_on_gpu():
    d = GOLD["demo_cavity"]
    n = d["cells_per_side"]
    g = W.cavity_uniform(n, 1.0 / n, seed=7)
    g.ports = [W.Port.point(W.COMP_EZ, 2, 3, 2), W.Port.point(W.COMP_EX, 5, 2, 3)]
    g.probes = [W.Port.point(W.COMP_EZ, 6, 2, 5), W.Port.point(W.COMP_EX, 3, 5, 6)]
    grid = F.Grid(g, "f64")
    dt = d["s_below"] * grid.cfl_dt()
    T = 8000
    u = torch.tensor(W.excitation(g, 0.15e9, 0.3e9, dt, T), device="cuda")
    y = grid.step(dt, u, reset=True)
    pk = F.resonances(y, dt, 0.15e9, 0.30e9, nf=3000, rel_floor=0.05)
    pko = spectrum.resonances(y.cpu().numpy(), dt, 0.15e9, 0.30e9, nf=3000, rel_floor=0.05)
    assert pk.size == 2 and np.allclose(pk, pko, rtol=1e-9)
    assert np.all(np.abs(pk / 1e9 - d["resonances_ghz"]) / d["resonances_ghz"] < 0.01)
