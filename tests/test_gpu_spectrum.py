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


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 1e-6)])
def test_sparams_match_oracle_and_closed_form(dtype, tol):
    """fdtd_sparams against the oracle on random waveforms, and on a delayed,
    scaled reflection and transmission of a pulse against r exp(-j 2 pi f d)
    and a exp(-j 2 pi f e)."""
    npd = np.float64 if dtype == torch.float64 else np.float32
    rng = np.random.default_rng(9)
    N, p, dt = 3000, 3, 1e-12
    y = rng.standard_normal((N, p)).astype(npd)
    yi = rng.standard_normal((N, p)).astype(npd)
    f = np.linspace(2e9, 40e9, 65)
    got = F.sparams(torch.tensor(y, device="cuda"), torch.tensor(yi, device="cuda"), dt, f, port_in=1)
    ref = spectrum.sparams(y.astype(np.float64), yi.astype(np.float64), dt, f, port_in=1)
    # same input values on both sides (FP64 sums): agreement to rounding
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.abs(ref).max()
    t = (np.arange(N) + 1) * dt
    x = np.exp(-((t - 0.4e-9) * np.pi * 8e9) ** 2) * np.sin(2 * np.pi * 12e9 * (t - 0.4e-9))
    d, e, r, a = 500, 300, -0.4, 0.75
    yinc = np.zeros((N, 2)); yinc[:, 0] = x
    ys = yinc.copy(); ys[d:, 0] += r * x[:N - d]; ys[e:, 1] = a * x[:N - e]
    f = np.linspace(6e9, 18e9, 25)
    S = F.sparams(torch.tensor(ys.astype(npd), device="cuda"), torch.tensor(yinc.astype(npd), device="cuda"), dt, f)
    # closed forms up to the rounding of r x, a x in the waveform type
    assert np.max(np.abs(S[0] - r * np.exp(-2j * np.pi * f * d * dt))) <= tol
    assert np.max(np.abs(S[1] - a * np.exp(-2j * np.pi * f * e * dt))) <= tol
    with pytest.raises(F.FdtdError):
        F.sparams(torch.tensor(ys, device="cuda"), torch.zeros((N, 2), dtype=torch.float64, device="cuda"), dt, f)
