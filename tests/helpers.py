"""Test-side glue: seeded grids for parity cases and conversions between the
oracle's unknown vectors and the six storage arrays of the CUDA library."""
import numpy as np

from paper_1406_7042_gb300 import workloads as W


def oracle_state_to_arrays(sys, x):
    """(6, nz, ny, nx) array from an oracle state vector (zeros where removed)."""
    a = sys.to_arrays(x)
    return np.stack([a[k] for k in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")])


def ragged_grid(nx=41, ny=19, nz=23, seed=101, many_materials=False, magnetic=True):
    """Graded spacing on every axis, lossy dielectric and magnetic blocks, PEC
    blocks, multi-edge sources crossing tile borders and several probes."""
    rng = np.random.default_rng(seed)
    extra = []
    nblk = 300 if many_materials else 6
    for _ in range(nblk):
        extra.append((float(rng.uniform(1, 8)), float(rng.uniform(0, 0.5))))
    eps, mu, se, sm, pec = W.vacuum_table(extra)
    if magnetic:
        mu = mu.copy(); sm = sm.copy()
        mu[2::3] = rng.uniform(1, 3, size=mu[2::3].size)
        sm[3::4] = rng.uniform(0, 200, size=sm[3::4].size)
    mat = np.zeros((nz, ny, nx), np.uint16)
    for b in range(nblk):
        sx, sy, sz = (int(rng.integers(2, 7)) for _ in range(3))
        x0 = int(rng.integers(0, nx - sx)); y0 = int(rng.integers(0, ny - sy)); z0 = int(rng.integers(0, nz - sz))
        mat[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = 2 + b
    for _ in range(3):
        x0 = int(rng.integers(2, nx - 4)); y0 = int(rng.integers(2, ny - 4)); z0 = int(rng.integers(2, nz - 4))
        mat[z0:z0 + 2, y0:y0 + 2, x0:x0 + 3] = 1
    dx = 1e-3 * rng.uniform(0.6, 1.4, nx)
    dy = 1e-3 * rng.uniform(0.6, 1.4, ny)
    dz = 1e-3 * rng.uniform(0.3, 1.4, nz)
    g = W.GridSpec(nx, ny, nz, dx, dy, dz, eps, mu, se, sm, pec, mat)
    # a line source in x crossing the tile border at i = 32, a y-line crossing
    # j = 8 / 16 (positions clipped into smaller grids)
    def ci(v, n):
        return int(min(max(v, 1), n - 2))
    is_ = np.arange(ci(26, nx), ci(38, nx) + 1)
    ks = np.full(is_.size, nz // 2); js = np.full(is_.size, ci(8, ny))
    g.ports.append(W.Port(W.COMP_EZ, ks.astype(np.int64), js.astype(np.int64), is_.astype(np.int64),
                          rng.uniform(0.5, 1.5, is_.size)))
    js2 = np.arange(ci(4, ny), ci(18, ny) + 1)
    g.ports.append(W.Port(W.COMP_EX, np.full(js2.size, ci(5, nz), np.int64), js2.astype(np.int64),
                          np.full(js2.size, ci(32, nx), np.int64), np.ones(js2.size)))
    g.ports.append(W.Port.point(W.COMP_EY, ci(32, nx), ci(16, ny), ci(11, nz), 2.0))
    for c, (i, j, k) in enumerate([(31, 7, 12), (32, 8, 12), (5, 17, 20), (40, 18, 1)]):
        g.probes.append(W.Port.point(c % 3, ci(i, nx), ci(j, ny), ci(k, nz)))
    js3 = np.arange(ci(5, ny), ci(10, ny))
    g.probes.append(W.Port(W.COMP_EZ, np.full(js3.size, ci(9, nz), np.int64), js3.astype(np.int64),
                           np.full(js3.size, ci(20, nx), np.int64), np.full(js3.size, 0.2)))
    return g


def drive(grid, dt, nsteps, f0=40e9, bw=60e9):
    u = W.gaussian_pulse(f0, bw, dt, nsteps)
    m = max(1, len(grid.ports))
    return np.stack([u * (1.0 + 0.25 * c) for c in range(m)], axis=1)


def subgrid(grid, lo, hi):
    """Sub-grid of cells [lo, hi) per axis (i, j, k order) with PEC walls,
    carrying the sources that fall inside it (for light-cone checks)."""
    (i0, j0, k0), (i1, j1, k1) = lo, hi
    g = W.GridSpec(i1 - i0, j1 - j0, k1 - k0, grid.dx[i0:i1], grid.dy[j0:j1], grid.dz[k0:k1],
                   grid.eps_r, grid.mu_r, grid.sig_e, grid.sig_m, grid.pec,
                   np.ascontiguousarray(grid.mat_id[k0:k1, j0:j1, i0:i1]))
    for p in grid.ports:
        sel = (p.i >= i0) & (p.i < i1) & (p.j >= j0) & (p.j < j1) & (p.k >= k0) & (p.k < k1)
        g.ports.append(W.Port(p.comp, p.k[sel] - k0, p.j[sel] - j0, p.i[sel] - i0, p.w[sel]))
    return g
