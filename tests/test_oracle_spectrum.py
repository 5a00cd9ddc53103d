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


def _pulse(n, dt, f0, bw, t0):
    t = (np.arange(n) + 1) * dt
    tau = 1.0 / (np.pi * bw)
    return np.exp(-((t - t0) / tau) ** 2) * np.sin(2 * np.pi * f0 * (t - t0))


def test_sparams_of_delayed_scaled_waves_are_closed_forms():
    """A reflected copy r x(t - d) at the driven port and a transmitted copy
    a x(t - e) at the second port, every pulse inside the window: S11 =
    r exp(-j 2 pi f d) and S21 = a exp(-j 2 pi f e) exactly (shift theorem of
    the finite sum), whatever the pulse."""
    n, dt = 4000, 1e-12
    x = _pulse(n, dt, 12e9, 8e9, 0.4e-9)
    d, e = 700, 450                       # samples
    r, a = -0.37, 0.81
    y_inc = np.zeros((n, 2))
    y_inc[:, 0] = x
    y = np.zeros((n, 2))
    y[:, 0] = x
    y[d:, 0] += r * x[:n - d]
    y[e:, 1] = a * x[:n - e]
    f = np.linspace(4e9, 20e9, 33)
    S = spectrum.sparams(y, y_inc, dt, f, port_in=0)
    assert np.allclose(S[0], r * np.exp(-2j * np.pi * f * d * dt), rtol=0, atol=1e-9)
    assert np.allclose(S[1], a * np.exp(-2j * np.pi * f * e * dt), rtol=0, atol=1e-9)


def test_sparams_of_a_matched_through_are_unit_transmission():
    """The reference run itself: no reflection at the driven port; a port that
    sees the same wave transmits with S = 1; and a lossless two-path split
    conserves |S11|^2 + |S21|^2 = 1."""
    n, dt = 3000, 2e-12
    x = _pulse(n, dt, 10e9, 6e9, 0.5e-9)
    y_inc = np.stack([x, x], axis=1)
    f = np.linspace(5e9, 15e9, 21)
    S = spectrum.sparams(y_inc, y_inc, dt, f, port_in=0)
    assert np.allclose(S[0], 0, atol=1e-12)
    assert np.allclose(S[1], 1, atol=1e-12)
    c, s_ = 0.6, 0.8
    y = np.zeros((n, 2))
    y[:, 0] = x
    y[300:, 0] += c * x[:n - 300]
    y[200:, 1] = s_ * x[:n - 200]
    S = spectrum.sparams(y, y_inc[:, :1], dt, f, port_in=0)
    assert np.allclose(np.abs(S[0]) ** 2 + np.abs(S[1]) ** 2, 1.0, atol=1e-9)
