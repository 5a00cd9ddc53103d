"""Textbook closed forms used to pin the oracle (not the oracle's own code).

Yee dispersion in a uniform PEC box (Taflove & Hagness, "Computational
Electrodynamics", ch. 4): a discrete mode with indices m_i in [0, N_i - 1]
(at most one zero) has phase w dt with
    sin^2(w dt / 2) = (c dt)^2 sum_i sin^2(m_i pi / (2 N_i)) / Delta_i^2,
and two polarisations when all m_i > 0.  The continuum resonances of an
a x b x d PEC box are c/2 sqrt((m/a)^2 + (n/b)^2 + (p/d)^2).
"""
import math

import numpy as np

C0 = 299792458.0


def box_mode_phases(nx, ny, nz, dxs, dys, dzs, dt, c=C0):
    out = []
    for m1 in range(nx):
        for m2 in range(ny):
            for m3 in range(nz):
                zeros = (m1 == 0) + (m2 == 0) + (m3 == 0)
                if zeros > 1:
                    continue
                s2 = (c * dt) ** 2 * ((math.sin(m1 * math.pi / (2 * nx)) / dxs) ** 2 +
                                      (math.sin(m2 * math.pi / (2 * ny)) / dys) ** 2 +
                                      (math.sin(m3 * math.pi / (2 * nz)) / dzs) ** 2)
                ph = 2.0 * math.asin(math.sqrt(s2)) if s2 <= 1.0 else float("nan")
                out.extend([ph] * (2 if zeros == 0 else 1))
    return np.sort(np.array(out))


def box_resonances_continuum(a, b, d, count, c=C0):
    out = []
    r = 12
    for m in range(r):
        for n in range(r):
            for p in range(r):
                zeros = (m == 0) + (n == 0) + (p == 0)
                if zeros > 1:
                    continue
                f = 0.5 * c * math.sqrt((m / a) ** 2 + (n / b) ** 2 + (p / d) ** 2)
                out.extend([f] * (2 if zeros == 0 else 1))
    return np.sort(np.array(out))[:count]


def max_stable_dt_uniform_box(nx, ny, nz, dxs, dys, dzs, c=C0):
    """Largest stable dt of the uniform box: the highest mode m_i = N_i - 1
    reaches sin^2(w dt/2) = 1."""
    s = ((math.sin((nx - 1) * math.pi / (2 * nx)) / dxs) ** 2 +
         (math.sin((ny - 1) * math.pi / (2 * ny)) / dys) ** 2 +
         (math.sin((nz - 1) * math.pi / (2 * nz)) / dzs) ** 2)
    return 1.0 / (c * math.sqrt(s))
