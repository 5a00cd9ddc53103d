"""Pins of the spectrum oracle: the plain DFT sum equals numpy's FFT on the
FFT frequency grid (phase shift of t_n = (n + 1) dt included), and the
resonance finder applied to the oracle FDTD of the paper's demo cavity
(Sec. III-B) returns the printed resonances."""
import json
import math
import os

import numpy as np

from oracle import spectrum, yee
from paper_1406_7042_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_dft_equals_fft_on_its_grid():
    rng = np.random.default_rng(4)
    N, dt = 256, 1e-12
    y = rng.standard_normal((N, 3))
    f = np.fft.rfftfreq(N, dt)
    ref = np.fft.rfft(y, axis=0).T * dt * np.exp(-2j * np.pi * f * dt)[None, :]
    got = spectrum.dft(y, dt, f)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # Hann window = weights applied before the transform
    w = np.sin(np.pi * (np.arange(N) + 0.5) / N) ** 2
    refh = np.fft.rfft(y * w[:, None], axis=0).T * dt * np.exp(-2j * np.pi * f * dt)[None, :]
    assert np.allclose(spectrum.dft(y, dt, f, hann=True), refh, rtol=1e-12, atol=1e-12 * np.abs(refh).max())


def test_resonances_of_demo_cavity_match_printed_values():
    d = GOLD["demo_cavity"]
    n = d["cells_per_side"]
    g = W.cavity_uniform(n, 1.0 / n, seed=7)
    g.ports = [W.Port.point(W.COMP_EZ, 2, 3, 2), W.Port.point(W.COMP_EX, 5, 2, 3)]
    g.probes = [W.Port.point(W.COMP_EZ, 6, 2, 5), W.Port.point(W.COMP_EX, 3, 5, 6)]
    dt = d["s_below"] * yee.cfl_dt(g)
    T = 8000
    u = W.excitation(g, 0.15e9, 0.3e9, dt, T)
    y, _, _ = yee.Stepper(yee.assemble(g), dt).run(u)
    pk = spectrum.resonances(y, dt, 0.15e9, 0.30e9, nf=3000, rel_floor=0.05)
    assert pk.size == 2
    assert np.all(np.abs(pk / 1e9 - d["resonances_ghz"]) / d["resonances_ghz"] < 0.01)
