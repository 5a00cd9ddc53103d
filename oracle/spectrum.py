"""FP64 oracle of the frequency-domain post-processing of probe waveforms.
Test infrastructure only.  Y_q(f) = sum_n w_n y^n_q exp(-j 2 pi f t_n) dt,
t_n = (n + 1) dt, w_n = sin^2(pi (n + 1/2) / N) (Hann) or 1, evaluated as the
plain sum; resonances are the largest local maxima of sum_q |Y_q| on a
uniform frequency grid, each moved to the vertex of the parabola through its
three samples; S-parameters are the ratios of port spectra to the incident
spectrum of a reference run (Sec. V-D reads S11 and S21 off the time-domain
port waveforms this way)."""
from __future__ import annotations

import numpy as np


def dft(y: np.ndarray, dt: float, freqs, hann: bool = False) -> np.ndarray:
    """(p, nf) complex spectra of y (nsteps, p)."""
    y = np.asarray(y, np.float64).reshape(len(y), -1)
    N = len(y)
    n = np.arange(N)
    w = np.sin(np.pi * (n + 0.5) / N) ** 2 if hann else np.ones(N)
    t = (n + 1) * dt
    f = np.asarray(freqs, np.float64)
    E = np.exp(-2j * np.pi * np.outer(f, t))          # (nf, N)
    return (E @ (w[:, None] * y)).T * dt


def resonances(y: np.ndarray, dt: float, fmin: float, fmax: float, nf: int = 4000, hann: bool = True,
               rel_floor: float = 0.05, npk: int = 16) -> np.ndarray:
    f = fmin + (fmax - fmin) * np.arange(nf) / (nf - 1)
    mag = np.abs(dft(y, dt, f, hann)).sum(axis=0)
    top = mag.max()
    pk = []
    for i in range(1, nf - 1):
        if mag[i] > mag[i - 1] and mag[i] >= mag[i + 1] and mag[i] >= rel_floor * top:
            a, b, c = mag[i - 1], mag[i], mag[i + 1]
            den = a - 2 * b + c
            off = 0.5 * (a - c) / den if den != 0 else 0.0
            pk.append((b, f[i] + off * (f[1] - f[0])))
    pk.sort(key=lambda t: -t[0])
    return np.sort(np.array([q[1] for q in pk[:npk]]))


def sparams(y: np.ndarray, y_inc: np.ndarray, dt: float, freqs, port_in: int, hann: bool = False) -> np.ndarray:
    """(p, nf) complex S_{q, port_in}(f) = (Y_q - [q = port_in] Yinc_q) / Yinc_port_in.

    y: probe waveforms (nsteps, p) of the structure excited at port port_in;
    y_inc: the same probes in a reference run that carries only the incident
    wave (the structure replaced by a matched line).  At the driven port the
    reflected wave is the total minus the incident one; at the other ports the
    whole wave is transmitted."""
    Y = dft(y, dt, freqs, hann)
    Yi = dft(y_inc, dt, freqs, hann)
    num = Y.copy()
    num[port_in] -= Yi[port_in]
    return num / Yi[port_in][None, :]
