"""Seeded synthetic inputs shaped like the test structures of Sec. V.

This module is the only code shared by the CUDA path and the FP64 oracle. It
builds plain data (grid spacings, a material table, a per-cell material id,
source and probe edge lists, excitation samples) and holds none of the
method's arithmetic: no curl operator, no material averaging, no time step.

Storage convention shared by both sides (six components per cell, the
"N = 6 x cells" accounting of Table I and Secs. V-C/V-D):

* cells are indexed (k, j, i) with i fastest; cell (i, j, k) spans
  [x_i, x_{i+1}] x [y_j, y_{j+1}] x [z_k, z_{k+1}];
* Ex[k, j, i] sits at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2);
* Hx[k, j, i] sits at (i, j+1/2, k+1/2), Hy at (i+1/2, j, k+1/2),
  Hz at (i+1/2, j+1/2, k);
* the outer boundary is a perfect electric conductor (PEC) box.

A source or probe ("port") is a weighted list of E edges: a source is one
column of B driven by u(t) (a current density, Sec. II-A), a probe is one row
of C.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 20140625  # submission date of the paper, plus the config index

COMP_EX, COMP_EY, COMP_EZ = 0, 1, 2


@dataclass
class Port:
    """Weighted set of E edges of one component (one B column or one C row)."""
    comp: int
    k: np.ndarray
    j: np.ndarray
    i: np.ndarray
    w: np.ndarray

    @staticmethod
    def point(comp: int, i: int, j: int, k: int, w: float = 1.0) -> "Port":
        return Port(comp, np.array([k], np.int64), np.array([j], np.int64),
                    np.array([i], np.int64), np.array([w], np.float64))

    @property
    def n(self) -> int:
        return int(self.w.size)


@dataclass
class GridSpec:
    """A rectilinear Yee grid in a PEC box with a per-cell material id."""
    nx: int
    ny: int
    nz: int
    dx: np.ndarray          # (nx,) cell sizes in metres
    dy: np.ndarray          # (ny,)
    dz: np.ndarray          # (nz,)
    eps_r: np.ndarray       # (nmat,) relative permittivity
    mu_r: np.ndarray        # (nmat,) relative permeability
    sig_e: np.ndarray       # (nmat,) electric conductivity, S/m
    sig_m: np.ndarray       # (nmat,) magnetic conductivity, ohm/m
    pec: np.ndarray         # (nmat,) uint8, 1 = perfect electric conductor
    mat_id: np.ndarray      # (nz, ny, nx) uint16 material index per cell
    ports: List[Port] = field(default_factory=list)
    probes: List[Port] = field(default_factory=list)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nmat(self) -> int:
        return int(self.eps_r.size)


@dataclass
class Workload:
    """One synthetic case: grid, excitation and the reduction settings."""
    name: str
    grid: GridSpec
    s_ref: float            # CFL factor of the full-order reference run
    nsteps_ref: int
    f0: float               # pulse centre frequency, Hz
    bw: float               # pulse bandwidth, Hz
    q: int = 0              # reduced order (columns of V1 and of V2)
    L: int = 2              # expansion points l = -L..L
    M: float = 1.1          # radius of the expansion-point arc
    fmax: float = 0.0
    include_center: bool = True
    s_red: List[float] = field(default_factory=list)
    nsteps_red: List[int] = field(default_factory=list)
    precision: str = "f32"


def _uniform(n: int, d: float) -> np.ndarray:
    return np.full(n, float(d), np.float64)


def vacuum_table(extra: Optional[List[tuple]] = None):
    """Material table: id 0 vacuum, id 1 PEC, then (eps_r, sigma) extras."""
    eps, mu, se, sm, pec = [1.0, 1.0], [1.0, 1.0], [0.0, 0.0], [0.0, 0.0], [0, 1]
    for (e, s) in (extra or []):
        eps.append(float(e)); mu.append(1.0); se.append(float(s)); sm.append(0.0); pec.append(0)
    return (np.array(eps), np.array(mu), np.array(se), np.array(sm),
            np.array(pec, np.uint8))


EPS0 = 8.8541878128e-12
MU0 = 4e-7 * math.pi


def add_absorber(g: GridSpec, sides: str = "xXyYzZ", n: int = 5, order: int = 4,
                 R0: float = 1e-6) -> GridSpec:
    """Graded matched absorber of n cells (the paper's 4th-order, 5-cell layer
    of Secs. V-B to V-D) on the faces named in `sides` (x / X: low / high x,
    likewise y, z).  A cell at layer depth d (1 = innermost, n = at the wall;
    where layers overlap the deepest counts) gets the electric conductivity
    sigma_max ((d - 1/2) / n)^order added to its material and the matched
    magnetic conductivity sigma_m = sigma_e mu / eps, so that the layer's
    impedance equals the medium's.  sigma_max gives a normal-incidence
    round-trip reflection R0 through the layer: sigma_max = -(order + 1)
    ln(R0) / (2 eta n delta), eta the medium's impedance and delta the cell
    size normal to the face.  Returns a new GridSpec (new materials appended;
    PEC cells stay PEC)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    depth = np.zeros((nz, ny, nx), np.int64)
    normal = np.full((nz, ny, nx), -1, np.int64)   # axis of the deepest layer
    idx = [np.arange(nx), np.arange(ny), np.arange(nz)]
    for axis, (lo, hi) in enumerate((("x", "X"), ("y", "Y"), ("z", "Z"))):
        size = (nx, ny, nz)[axis]
        d1 = np.zeros(size, np.int64)
        if lo in sides:
            d1 = np.maximum(d1, np.where(idx[axis] < n, n - idx[axis], 0))
        if hi in sides:
            d1 = np.maximum(d1, np.where(idx[axis] >= size - n, idx[axis] - (size - n) + 1, 0))
        shape = [1, 1, 1]
        shape[2 - axis] = size
        d3 = np.broadcast_to(d1.reshape(shape), (nz, ny, nx))
        upd = d3 > depth
        depth = np.where(upd, d3, depth)
        normal = np.where(upd, axis, normal)
    spacing = (g.dx, g.dy, g.dz)
    eps, mu = list(g.eps_r), list(g.mu_r)
    se, sm, pec = list(g.sig_e), list(g.sig_m), list(g.pec)
    mat = g.mat_id.astype(np.int64).copy()
    new_id = {}
    ks, js, is_ = np.nonzero(depth)
    for k, j, i in zip(ks, js, is_):
        m0 = int(mat[k, j, i])
        if g.pec[m0]:
            continue
        d, ax = int(depth[k, j, i]), int(normal[k, j, i])
        pos = (i, j, k)[ax]
        key = (m0, d, ax, float(spacing[ax][pos]))
        if key not in new_id:
            eta = math.sqrt(MU0 * g.mu_r[m0] / (EPS0 * g.eps_r[m0]))
            smax = -(order + 1) * math.log(R0) / (2.0 * eta * n * spacing[ax][pos])
            dse = smax * ((d - 0.5) / n) ** order
            eps.append(g.eps_r[m0]); mu.append(g.mu_r[m0]); pec.append(0)
            se.append(g.sig_e[m0] + dse)
            sm.append(g.sig_m[m0] + dse * MU0 * g.mu_r[m0] / (EPS0 * g.eps_r[m0]))
            new_id[key] = len(eps) - 1
        mat[k, j, i] = new_id[key]
    if len(eps) > 65535:
        raise ValueError("too many materials after adding the absorber")
    out = GridSpec(nx, ny, nz, g.dx, g.dy, g.dz, np.array(eps), np.array(mu), np.array(se), np.array(sm),
                   np.array(pec, np.uint8), mat.astype(np.uint16))
    out.ports, out.probes = list(g.ports), list(g.probes)
    return out


def gaussian_pulse(f0: float, bw: float, dt: float, nsteps: int) -> np.ndarray:
    """Gaussian-modulated sine sampled at t = (n + 1/2) dt, n = 0..nsteps-1.

    u(t) = sin(2 pi f0 (t - t0)) exp(-((t - t0)/tau)^2) with
    tau = 2 sqrt(ln 10) / (pi bw) (spectrum 20 dB down at f0 +- bw/2) and
    t0 = 4 tau.  Row n is the source value u^{n+1} of Eq. (matrix), taken at
    the half step where the electric current J^{n+1/2} of Eq. (FDTD1) lives.
    """
    tau = 2.0 * math.sqrt(math.log(10.0)) / (math.pi * bw)
    t0 = 4.0 * tau
    t = (np.arange(nsteps, dtype=np.float64) + 0.5) * dt - t0
    return np.sin(2.0 * math.pi * f0 * t) * np.exp(-(t / tau) ** 2)


def excitation(grid: GridSpec, f0: float, bw: float, dt: float, nsteps: int) -> np.ndarray:
    """(nsteps, m) samples: every port driven by the same pulse."""
    u = gaussian_pulse(f0, bw, dt, nsteps)
    return np.repeat(u[:, None], max(1, len(grid.ports)), axis=1)


def _interior_cell(rng, n: int, margin: int = 2) -> int:
    if n < 2 * margin + 3:
        return int(rng.integers(1, max(2, n)))
    return int(rng.integers(margin, n - margin))


def _distinct_cell(rng, used: set, dims, margin: int = 2):
    """A seeded cell not in ``used`` (repeats allowed once the grid is too small)."""
    c = None
    for _ in range(1000):
        c = tuple(_interior_cell(rng, n, margin) for n in dims)
        if c not in used:
            break
    used.add(c)
    return c


# ---------------------------------------------------------------- 10^3 PEC cavity
def cavity_uniform(n: int = 10, d: float = 1e-3, seed: int = SEED_BASE + 1,
                   nports: int = 1, nprobes: int = 1) -> GridSpec:
    """Lossless vacuum PEC cube of n^3 cells of size d, Ez point ports/probes."""
    rng = np.random.default_rng(seed)
    eps, mu, se, sm, pec = vacuum_table()
    g = GridSpec(n, n, n, _uniform(n, d), _uniform(n, d), _uniform(n, d),
                 eps, mu, se, sm, pec, np.zeros((n, n, n), np.uint16))
    used = set()
    for lst, cnt in ((g.ports, nports), (g.probes, nprobes)):
        for _ in range(cnt):
            i, j, k = _distinct_cell(rng, used, (n, n, n))
            lst.append(Port.point(COMP_EZ, i, j, k))
    return g


def cavity10_workload(seed: int = SEED_BASE + 1) -> Workload:
    g = cavity_uniform(10, 1e-3, seed)
    return Workload("cavity10_f64", g, 0.99, 4000, 10e9, 10e9, q=40, L=2, M=1.1,
                    fmax=15e9, s_red=[0.99, 4.95, 9.9], nsteps_red=[4000, 800, 400],
                    precision="f64")


# ---------------------------------------------------------------- graded cavity
def graded_z(n_total: int = 64, coarse: float = 0.5e-3, fine: float = 0.05e-3,
             n_grade: int = 8, n_slab: int = 2) -> np.ndarray:
    """z spacings: coarse cells, a geometric grading over n_grade cells down to
    a slab of n_slab fine cells, and the mirror image above it."""
    r = (coarse / fine) ** (1.0 / (n_grade + 1))
    grade_up = fine * r ** np.arange(1, n_grade + 1)
    n_coarse = n_total - n_slab - 2 * n_grade
    lo = n_coarse // 2
    hi = n_coarse - lo
    return np.concatenate([np.full(lo, coarse), grade_up[::-1], np.full(n_slab, fine),
                           grade_up, np.full(hi, coarse)])


def cavity_graded(n: int = 64, seed: int = SEED_BASE + 2, nblocks: int = 16,
                  nprobes: int = 4) -> GridSpec:
    rng = np.random.default_rng(seed)
    dz = graded_z(n)
    extra = [(4.0, 0.01)]  # slab
    for _ in range(nblocks):
        extra.append((float(rng.uniform(1.0, 6.0)), float(rng.uniform(0.0, 0.05))))
    eps, mu, se, sm, pec = vacuum_table(extra)
    mat = np.zeros((n, n, n), np.uint16)
    n_coarse = n - 2 - 16
    zs = n_coarse // 2 + 8
    mat[zs:zs + 2, :, :] = 2
    for b in range(nblocks):
        sx, sy, sz = (int(rng.integers(4, 13)) for _ in range(3))
        x0 = int(rng.integers(1, n - sx)); y0 = int(rng.integers(1, n - sy)); z0 = int(rng.integers(1, n - sz))
        mat[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = 3 + b
    g = GridSpec(n, n, n, _uniform(n, 0.5e-3), _uniform(n, 0.5e-3), dz, eps, mu, se, sm, pec, mat)
    used = set()
    for lst, cnt in ((g.ports, 1), (g.probes, nprobes)):
        for _ in range(cnt):
            i, j, k = _distinct_cell(rng, used, (n, n, n), 4)
            lst.append(Port.point(COMP_EZ, i, j, k))
    return g


def graded_cavity_workload(seed: int = SEED_BASE + 2, n: int = 64) -> Workload:
    """64^3 graded cavity.  Its 0.163 ps step puts the whole 5-15 GHz band on an
    arc of 2 pi fmax dt0 = 0.0154 rad of the unit circle, so the expansion
    radius is taken as 1 + pi fmax dt0 = 1.0077 (half that arc away from the
    circle) instead of 1.1, which would sit 13 arcs away."""
    g = cavity_graded(n, seed)
    return Workload(f"graded_cavity{n}_f32", g, 0.99, 400000, 10e9, 10e9, q=200, L=2,
                    M=1.0077, fmax=15e9, s_red=[19.8], nsteps_red=[20000], precision="f32")


# ---------------------------------------------------------------- waveguide and cavity batch
def waveguide_iris(seed: int = SEED_BASE + 3, nx: int = 256, ny: int = 64, nz: int = 32,
                   d: float = 0.1e-3) -> GridSpec:
    """PEC rectangular guide (broad wall along y) with one seeded iris and two
    TE10-profile Ez current sheets / line probes near the ends."""
    rng = np.random.default_rng(seed)
    eps, mu, se, sm, pec = vacuum_table()
    mat = np.zeros((nz, ny, nx), np.uint16)
    xi = int(rng.integers(int(nx * 0.375), int(nx * 0.625) + 1))
    ay = int(rng.integers(ny // 4, ny // 2 + 1)); az = int(rng.integers(nz // 4, nz // 2 + 1))
    y0 = int(rng.integers(1, ny - ay)); z0 = int(rng.integers(1, nz - az))
    mat[:, :, xi] = 1
    mat[z0:z0 + az, y0:y0 + ay, xi] = 0
    g = GridSpec(nx, ny, nz, _uniform(nx, d), _uniform(ny, d), _uniform(nz, d),
                 eps, mu, se, sm, pec, mat)
    jj, kk = np.meshgrid(np.arange(1, ny), np.arange(0, nz), indexing="xy")
    prof = np.sin(np.pi * jj.astype(np.float64) / ny)
    for x in (min(8, nx // 4), max(nx - 9, 3 * nx // 4)):
        sheet = Port(COMP_EZ, kk.ravel().astype(np.int64), jj.ravel().astype(np.int64),
                     np.full(jj.size, x, np.int64), prof.ravel().copy())
        g.ports.append(sheet)
        g.probes.append(Port(sheet.comp, sheet.k.copy(), sheet.j.copy(), sheet.i.copy(),
                             sheet.w / sheet.w.size))
    return g


def cavity_batch(seed: int = SEED_BASE + 30, count: int = 32, lo: int = 24, hi: int = 96,
                 d: float = 1e-3) -> List[GridSpec]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny, nz = (int(rng.integers(lo, hi + 1)) for _ in range(3))
        eps, mu, se, sm, pec = vacuum_table()
        g = GridSpec(nx, ny, nz, _uniform(nx, d), _uniform(ny, d), _uniform(nz, d),
                     eps, mu, se, sm, pec, np.zeros((nz, ny, nx), np.uint16))
        m = int(rng.integers(1, 5))
        used = set()
        for lst in (g.ports, g.probes):
            for _ in range(m):
                lst.append(Port.point(COMP_EZ, *_distinct_cell(rng, used, (nx, ny, nz))))
        out.append(g)
    return out


def waveguide_workload(seed: int = SEED_BASE + 3, absorbing: bool = False) -> Workload:
    g = waveguide_iris(seed)
    if absorbing:   # the paper's guide ends on matched absorbers (Sec. V-B)
        g = add_absorber(g, "xX")
    return Workload("waveguide_iris" + ("_abs" if absorbing else "") + "_f32", g, 0.99, 20000, 35e9, 20e9, q=200, L=2, M=1.1,
                    fmax=45e9, s_red=[0.99], nsteps_red=[20000], precision="f32")


# ---------------------------------------------------------------- the paper's cavities and 2-D guide
def plates2d(nx: int, ny: int, d: float, eps_r: float = 1.0) -> GridSpec:
    """A 2-D TM problem (Ez, Hx, Hy) as one layer of cells between two PEC
    plates: with nz = 1 the tangential Ex, Ey and the normal Hz vanish on the
    plates, leaving (nx-1)(ny-1) Ez, (nx-1) ny Hx and nx (ny-1) Hy unknowns."""
    eps, mu, se, sm, pec = vacuum_table([(eps_r, 0.0)] if eps_r != 1.0 else None)
    mat = np.full((1, ny, nx), 2 if eps_r != 1.0 else 0, np.uint16)
    return GridSpec(nx, ny, 1, _uniform(nx, d), _uniform(ny, d), _uniform(1, d), eps, mu, se, sm, pec, mat)


def cavity2d_workload(seed: int = SEED_BASE + 6) -> Workload:
    """The 2-D PEC cavity of Sec. V-A (Table I): 101 x 101 cells of 1 cm, a
    single source and probe (Ez, seeded interior nodes), a pulse of bandwidth
    0.5 GHz centred at 0.35 GHz (its -20 dB band holds the first six TM
    resonances but for the sixth at 0.61 GHz), 10,000 steps; q = 80 with five
    expansion points, M = 1.1, fmax = 0.6 GHz; reduced at s = 0.99 and 4.95."""
    rng = np.random.default_rng(seed)
    g = plates2d(101, 101, 1e-2)
    used = set()
    for lst in (g.ports, g.probes):
        i, j, _ = _distinct_cell(rng, used, (101, 101, 1), 5)
        lst.append(Port.point(COMP_EZ, i, j, 0))
    return Workload("cavity2d_f32", g, 0.99, 10000, 0.35e9, 0.5e9, q=80, L=2, M=1.1, fmax=0.6e9,
                    s_red=[0.99, 4.95], nsteps_red=[10000, 2000], precision="f32")


def cavity3d_workload(seed: int = SEED_BASE + 7) -> Workload:
    """The 3-D PEC cavity of Sec. V-A (Table I): 51^3 cells of 2 cm, a single
    Ez source and probe at seeded interior cells, the same pulse (the first
    six resonances, 0.21-0.44 GHz, inside its band), 10,000 steps; q = 80,
    five expansion points, M = 1.1, fmax = 0.5 GHz; reduced at s = 0.99,
    1.98, 2.97."""
    g = cavity_uniform(51, 2e-2, seed)
    return Workload("cavity3d_f32", g, 0.99, 10000, 0.35e9, 0.5e9, q=80, L=2, M=1.1, fmax=0.5e9,
                    s_red=[0.99, 1.98, 2.97], nsteps_red=[10000, 5000, 3333], precision="f32")


def cavity_resonances(a: float, b: float, c: float = None, count: int = 6) -> np.ndarray:
    """Lowest distinct resonance frequencies (Hz) of an empty PEC box of sides
    a, b (and c; 2-D TM when None): f = c0/2 sqrt((m/a)^2 + (n/b)^2 + (p/c)^2),
    m, n >= 1 in 2-D; in 3-D at most one index zero (TE and TM together)."""
    c0 = 299792458.0
    fs = set()
    rng = range(0, 12)
    for m in rng:
        for n in rng:
            if c is None:
                if m >= 1 and n >= 1:
                    fs.add(round(c0 / 2 * np.sqrt((m / a) ** 2 + (n / b) ** 2), 3))
                continue
            for p_ in rng:
                if (m == 0) + (n == 0) + (p_ == 0) <= 1:
                    fs.add(round(c0 / 2 * np.sqrt((m / a) ** 2 + (n / b) ** 2 + (p_ / c) ** 2), 3))
    return np.array(sorted(fs)[:count])


def waveguide2d(irises: bool = True, d: float = 1.25e-3) -> GridSpec:
    """The 2-D waveguide filter of Sec. V-B as a TM problem between plates:
    5 cm x 50 cm (41 x 401 cells of 1.25 mm) filled with eps_r = 2.5, five
    thin PEC irises across the guide (one cell thick, an aperture of 8 cells =
    1 cm at the centre, 40 cells = 5 cm apart, centred on the guide; the
    layout figure is not available and "length 1.25 cm" is read as the
    cross-section of each iris wall), 5-cell 4th-order matched absorbers at
    both ends, an Ez current line across the guide at y = 8 (TM1 profile),
    line probes at y = 12 (port 1) and y = 392 (port 2).  Without irises it
    is the matched reference line of the S-parameters."""
    nx, ny = 41, 401
    g = plates2d(nx, ny, d, 2.5)   # material 2: the filling; 1: PEC
    if irises:
        x0 = (nx - 8) // 2
        for t in range(5):
            y0 = ny // 2 + (t - 2) * 40
            g.mat_id[0, y0, :] = 1
            g.mat_id[0, y0, x0:x0 + 8] = 2
    g = add_absorber(g, "yY")
    xs = np.arange(1, nx, dtype=np.int64)
    prof = np.sin(np.pi * xs / nx)

    def line(y, w):
        return Port(COMP_EZ, np.zeros(xs.size, np.int64), np.full(xs.size, y, np.int64), xs, w)
    g.ports.append(line(8, prof))
    g.probes.append(line(12, prof / xs.size))
    g.probes.append(line(ny - 9, prof / xs.size))
    return g


def waveguide2d_workload(irises: bool = True) -> Workload:
    """Sec. V-B: pulse of bandwidth 3 GHz (f0 = 2.5 GHz), 20,000 steps; q = 200,
    five expansion points, M = 1.1, fmax = 3 GHz; reduced at s = 0.99, 4.95,
    8.91."""
    return Workload("waveguide2d" + ("" if irises else "_line") + "_f32", waveguide2d(irises), 0.99, 20000,
                    2.5e9, 3e9, q=200, L=2, M=1.1, fmax=3e9, s_red=[0.99, 4.95, 8.91],
                    nsteps_red=[20000, 4040, 2244], precision="f32")


# ---------------------------------------------------------------- microstrip filter
def microstrip(seed: int = SEED_BASE + 4, nx: int = 400, ny: int = 200, nz: int = 24,
               dxy: float = 0.4e-3, dz: float = 0.2e-3, n_sub: int = 6) -> GridSpec:
    """Substrate of n_sub layers (eps_r 9.8) on the PEC ground (z = 0), a
    one-cell PEC strip layer from a seeded mask of three coupled-line
    resonators plus two feed lines, and two z-directed ports under the feeds."""
    rng = np.random.default_rng(seed)
    eps, mu, se, sm, pec = vacuum_table([(9.8, 0.0)])
    mat = np.zeros((nz, ny, nx), np.uint16)
    mat[:n_sub] = 2
    mask = np.zeros((ny, nx), bool)
    sx = nx / 400.0; sy = ny / 200.0
    w = 3
    yc = ny // 2
    x = int(round(40 * sx))
    feed_len = max(4, int(round(30 * sx)))
    mask[yc - 1:yc + 2, x - feed_len:x] = True          # input feed
    ports_at = [(x - feed_len + 1, yc)]
    y = yc
    for r in range(3):
        length = max(6, int(round(rng.integers(60, 101) * sx)))
        gap = int(rng.integers(2, 5))
        y_new = y + (w + gap) * (1 if r % 2 == 0 else -1)
        y_new = int(np.clip(y_new, 2, ny - 3 - w))
        mask[y_new - 1:y_new + 2, x - length // 2:x + length // 2] = True
        x = x + length // 2
        y = y_new
    mask[y - 1:y + 2, x:x + feed_len] = True              # output feed
    ports_at.append((x + feed_len - 2, y))
    mask[:, 0] = mask[:, -1] = False
    mask[0, :] = mask[-1, :] = False
    mat[n_sub][mask] = 1
    g = GridSpec(nx, ny, nz, _uniform(nx, dxy), _uniform(ny, dxy), _uniform(nz, dz),
                 eps, mu, se, sm, pec, mat)
    for (pi, pj) in ports_at:
        pi = int(np.clip(pi, 2, nx - 3)); pj = int(np.clip(pj, 2, ny - 3))
        ks = np.arange(0, n_sub, dtype=np.int64)
        p = Port(COMP_EZ, ks, np.full(n_sub, pj, np.int64), np.full(n_sub, pi, np.int64),
                 np.ones(n_sub))
        g.ports.append(p)
        g.probes.append(Port(p.comp, p.k.copy(), p.j.copy(), p.i.copy(), np.full(n_sub, dz)))
    return g


def microstrip_workload(seed: int = SEED_BASE + 4, downscale: bool = False, absorbing: bool = False) -> Workload:
    if downscale:
        g = microstrip(seed, 100, 50, 24)
    else:
        g = microstrip(seed)
    if absorbing:   # five absorbing faces, PEC ground at z = 0 (Sec. V-D)
        g = add_absorber(g, "xXyYZ")
    return Workload("microstrip" + ("_down" if downscale else "") + ("_abs" if absorbing else "") + "_f32", g, 0.99, 8000,
                    10e9, 20e9, q=400 if not downscale else 100, L=2, M=1.1, fmax=20e9,
                    s_red=[0.99, 2.97, 4.95], nsteps_red=[8000, 2667, 1600], precision="f32")


# ---------------------------------------------------------------- focusing metascreen
def metascreen(seed: int = SEED_BASE + 5, nxy: int = 384, nz: int = 64, d: float = 0.25e-3,
               npix: int = 64, pix_xy: int = 6, pix_z: int = 2) -> GridSpec:
    """Dielectric screen of npix x npix design pixels (pix_xy^2 x pix_z cells
    each, eps_r ~ U[1, 12]) at mid height, a plane of uniform Ex currents
    below it and one focal Ex probe above it."""
    rng = np.random.default_rng(seed)
    eps_pix = rng.uniform(1.0, 12.0, size=npix * npix)
    eps, mu, se, sm, pec = vacuum_table([(e, 0.0) for e in eps_pix])
    mat = np.zeros((nz, nxy, nxy), np.uint16)
    z0 = nz // 2
    ids = (2 + np.arange(npix * npix)).reshape(npix, npix).astype(np.uint16)
    span = npix * pix_xy
    off = (nxy - span) // 2
    blk = np.kron(ids, np.ones((pix_xy, pix_xy), np.uint16))
    for dzc in range(pix_z):
        mat[z0 + dzc, off:off + span, off:off + span] = blk
    g = GridSpec(nxy, nxy, nz, _uniform(nxy, d), _uniform(nxy, d), _uniform(nz, d),
                 eps, mu, se, sm, pec, mat)
    zs = nz // 8
    jj, ii = np.meshgrid(np.arange(1, nxy), np.arange(0, nxy), indexing="ij")
    g.ports.append(Port(COMP_EX, np.full(jj.size, zs, np.int64), jj.ravel().astype(np.int64),
                        ii.ravel().astype(np.int64), np.ones(jj.size)))
    g.probes.append(Port.point(COMP_EX, nxy // 2, nxy // 2, (7 * nz) // 8))
    return g


def metascreen_workload(seed: int = SEED_BASE + 5, downscale: bool = False, absorbing: bool = False) -> Workload:
    if downscale:
        g = metascreen(seed, 48, 16, 0.25e-3, 8, 6, 2)
    else:
        g = metascreen(seed)
    if absorbing:   # all six faces absorbing (Sec. V-C)
        g = add_absorber(g, "xXyYzZ")
    return Workload("metascreen" + ("_down" if downscale else "") + ("_abs" if absorbing else "") + "_f32", g, 0.99, 2048,
                    10e9, 5e9, q=40, L=1, M=1.1, fmax=10e9, include_center=False,
                    s_red=[0.99], nsteps_red=[2048], precision="f32")


def pixel_map(grid: GridSpec, first_pixel_id: int = 2) -> np.ndarray:
    """Cell -> design-pixel index (or -1) for metascreen grids."""
    pm = grid.mat_id.astype(np.int64) - first_pixel_id
    pm[grid.mat_id < first_pixel_id] = -1
    return pm
