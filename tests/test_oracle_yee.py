"""Pins of the FP64 Yee oracle against closed forms, invariants, the paper's
printed values and brute force (no GPU)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import yee
from paper_1406_7042_gb300 import workloads as W
from tests.closed_forms import (box_mode_phases, box_resonances_continuum,
                                max_stable_dt_uniform_box)

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _box(nx, ny, nz, dxs, dys, dzs, eps=1.0, sig=0.0):
    eps_t, mu, se, sm, pec = W.vacuum_table([(eps, sig)])
    return W.GridSpec(nx, ny, nz, np.full(nx, dxs), np.full(ny, dys), np.full(nz, dzs),
                      eps_t, mu, se, sm, pec, np.full((nz, ny, nx), 2, np.uint16))


def _nonstatic_phases(Phi):
    ev = np.linalg.eigvals(Phi)
    ph = np.sort(np.angle(ev))
    return ev, ph[ph > 1e-9]


@pytest.mark.parametrize("dims", [(2, 2, 2, 1e-3, 1e-3, 1e-3), (3, 3, 3, 1e-3, 1e-3, 1e-3),
                                  (2, 3, 4, 1e-3, 1.5e-3, 0.7e-3), (4, 3, 2, 2e-3, 1e-3, 1e-3)])
def test_dispersion_relation_uniform_box(dims):
    """P-a: eigenvalues of Phi = (R+F)^{-1}(R-F) are 1 (static) and exp(+-j w dt)
    with w from the Yee dispersion relation."""
    nx, ny, nz, a, b, c = dims
    g = _box(nx, ny, nz, a, b, c)
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    ev, ph = _nonstatic_phases(yee.amplification_matrix(s, dt))
    ref = box_mode_phases(nx, ny, nz, a, b, c, dt)
    assert np.allclose(np.abs(ev), 1.0, atol=1e-12)
    assert ph.size == ref.size
    assert np.max(np.abs(ph - ref)) < 1e-12
    # static eigenvalues: dim null(K^T) + dim null(K)
    n_static = np.sum(np.abs(ev - 1.0) < 1e-9)
    assert n_static == s.N - 2 * ref.size
    if (nx, ny, nz) == (2, 2, 2):
        assert ref.size == 5  # five mode pairs in the 2^3 box


def test_dispersion_dielectric_fill_halves_frequencies():
    """A box filled with eps_r = 4 has the dispersion relation of c0/2."""
    g = _box(3, 2, 3, 1e-3, 1e-3, 1e-3, eps=4.0)
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    _, ph = _nonstatic_phases(yee.amplification_matrix(s, dt))
    ref = box_mode_phases(3, 2, 3, 1e-3, 1e-3, 1e-3, dt, c=yee.C0 / 2)
    assert np.max(np.abs(ph - ref)) < 1e-12


def test_uniform_loss_decay_rate():
    """Uniform sigma_e: each oscillating mode's 2x2 recursion has product of
    roots ca = (eps/dt - sigma/2)/(eps/dt + sigma/2), so |lambda| = sqrt(ca); the
    static (gradient) E modes decay by ca per step."""
    g = _box(3, 3, 2, 1e-3, 1e-3, 1e-3, eps=2.0, sig=3.0)
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    ev = np.linalg.eigvals(yee.amplification_matrix(s, dt))
    e = 2.0 * yee.EPS0
    ca = (e / dt - 1.5) / (e / dt + 1.5)
    osc = ev[np.abs(ev.imag) > 1e-9]
    assert np.allclose(np.abs(osc), math.sqrt(ca), atol=1e-12)
    real = ev[np.abs(ev.imag) <= 1e-9]
    assert np.all(np.isclose(real, 1.0, atol=1e-10) | np.isclose(real, ca, atol=1e-10) |
                  (np.abs(real) < math.sqrt(ca) + 1e-9))


def test_golden_demo_resonances():
    """Sec. III-B: 1 m PEC cube, cell 1/9 m, resonances printed as 0.21199 and
    0.25963 GHz.  The analytic continuum values equal them to the printed
    digits; the oracle FDTD's probe spectrum peaks at the discrete dispersion
    values, which lie within 1 % of the printed ones."""
    d = GOLD["demo_cavity"]
    fa = box_resonances_continuum(1.0, 1.0, 1.0, 6)
    lowest = sorted(set(np.round(fa, 1)))[:2]
    assert np.allclose(np.array(lowest) / 1e9, d["resonances_ghz"], atol=5e-6)
    n = d["cells_per_side"]
    g = W.cavity_uniform(n, 1.0 / n, seed=7)
    g.ports = [W.Port.point(W.COMP_EZ, 2, 3, 2)]
    g.probes = [W.Port.point(W.COMP_EZ, 6, 2, 5), W.Port.point(W.COMP_EX, 3, 5, 6)]
    g.ports.append(W.Port.point(W.COMP_EX, 5, 2, 3))
    s = yee.assemble(g)
    dt = d["s_below"] * yee.cfl_dt(g)
    T = 8000
    u = W.excitation(g, 0.15e9, 0.3e9, dt, T)
    y, _, _ = yee.Stepper(s, dt).run(u)
    spec = np.abs(np.fft.rfft(y * np.hanning(T)[:, None], n=8 * T, axis=0)).sum(axis=1)
    f = np.fft.rfftfreq(8 * T, dt)
    band = (f > 0.15e9) & (f < 0.30e9)
    fb, sb = f[band], spec[band]
    peaks = [fb[i] for i in range(1, fb.size - 1) if sb[i] > sb[i - 1] and sb[i] > sb[i + 1]
             and sb[i] > 0.05 * sb.max()]
    disc = np.unique(np.round(box_mode_phases(n, n, n, 1 / n, 1 / n, 1 / n, dt) / (2 * math.pi * dt), -3))
    disc = disc[(disc > 0.15e9) & (disc < 0.30e9)]
    assert len(peaks) == 2 and disc.size == 2
    res = 1.0 / (8 * T * dt)
    assert np.all(np.abs(np.array(peaks) - disc) < 2 * res)
    assert np.all(np.abs(np.array(peaks) / 1e9 - d["resonances_ghz"]) / d["resonances_ghz"] < 0.01)


def test_energy_conserved_lossless_nonuniform():
    """P-c: W = x^T R x is conserved to rounding after the source stops."""
    g = W.cavity_uniform(6, 1e-3, seed=3)
    g.dx = np.linspace(0.8e-3, 1.3e-3, 6)
    g.dz = np.array([1e-3, 0.5e-3, 0.25e-3, 0.25e-3, 0.5e-3, 1e-3])
    g.eps_r = np.array([1.0, 1.0, 3.0]); g.mu_r = np.array([1.0, 1.0, 2.0])
    g.sig_e = np.zeros(3); g.sig_m = np.zeros(3); g.pec = np.array([0, 1, 0], np.uint8)
    g.mat_id[2:4, 1:4, 2:5] = 2
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    st = yee.Stepper(s, dt)
    u = W.excitation(g, 30e9, 40e9, dt, 400)
    _, x, _ = st.run(u)
    w0 = yee.energy(s, dt, x)
    _, x2, _ = st.run(np.zeros((10000, 1)), x0=x)
    assert abs(yee.energy(s, dt, x2) - w0) / w0 < 1e-12


def test_energy_nonincreasing_lossy():
    g = W.cavity_uniform(5, 1e-3, seed=4)
    g.sig_e = np.array([0.5, 0.0]); g.sig_m = np.array([100.0, 0.0])
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    st = yee.Stepper(s, dt)
    _, x, _ = st.run(W.excitation(g, 30e9, 40e9, dt, 300))
    w = [yee.energy(s, dt, x)]
    for _ in range(20):
        _, x, _ = st.run(np.zeros((50, 1)), x0=x)
        w.append(yee.energy(s, dt, x))
    assert np.all(np.diff(w) <= 1e-15 * w[0])
    assert w[-1] < 0.9 * w[0]


def test_block_substitution_is_matrix_form():
    """The leap-frog equals the literal solve of Eq. (MNAform)."""
    g = W.cavity_uniform(4, 1e-3, seed=5)
    g.sig_e = np.array([0.2, 0.0]); g.sig_m = np.array([30.0, 0.0])
    g.dy = np.array([1e-3, 2e-3, 0.5e-3, 1e-3])
    s = yee.assemble(g)
    dt = 0.9 * yee.cfl_dt(g)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(s.N)
    e, h = yee.Stepper(s, dt).step(x[:s.Ne], x[s.Ne:], np.array([0.7]))
    x1 = yee.step_matrix_form(s, dt, x, np.array([0.7]))
    assert np.max(np.abs(np.concatenate([e, h]) - x1)) < 1e-12 * np.max(np.abs(x1))


def test_source_and_first_step_follow_eq_fdtd1():
    """From rest, one step with u = J at a source edge gives E = -J dt/(eps0 eps_r)
    there (Eq. (FDTD1)) and, by Faraday, H^{3/2} = -dt/(mu0) curl E around it."""
    g = W.cavity_uniform(5, 1e-3, seed=6)
    g.eps_r = np.array([2.5, 1.0])
    g.ports = [W.Port.point(W.COMP_EZ, 2, 2, 2)]
    g.probes = [W.Port.point(W.COMP_EZ, 2, 2, 2)]
    s = yee.assemble(g)
    dt = 0.5 * yee.cfl_dt(g)
    J = 3.0
    y, x, _ = yee.Stepper(s, dt).run(np.array([[J]]))
    arr = s.to_arrays(x)
    ez = -J * dt / (yee.EPS0 * 2.5)
    assert np.isclose(y[0, 0], ez, rtol=1e-14)
    assert np.isclose(arr["Ez"][2, 2, 2], ez, rtol=1e-14)
    assert np.count_nonzero(arr["Ex"]) == 0 and np.count_nonzero(arr["Ey"]) == 0
    # mu dHx/dt = -(dEz/dy): Hx[k,j,i] at (i, j+1/2, k+1/2) sees Ez[k, j+1, i] - Ez[k, j, i]
    mu = yee.MU0
    assert np.isclose(arr["Hx"][2, 2, 2], -dt / mu * (0 - ez) / 1e-3, rtol=1e-13)
    assert np.isclose(arr["Hx"][2, 1, 2], -dt / mu * (ez - 0) / 1e-3, rtol=1e-13)
    # mu dHy/dt = +dEz/dx: Hy[k,j,i] at (i+1/2, j, k+1/2) sees Ez[k, j, i+1] - Ez[k, j, i]
    assert np.isclose(arr["Hy"][2, 2, 2], dt / mu * (0 - ez) / 1e-3, rtol=1e-13)
    assert np.isclose(arr["Hy"][2, 2, 1], dt / mu * (ez - 0) / 1e-3, rtol=1e-13)
    assert np.count_nonzero(arr["Hz"]) == 0


def test_edge_material_average_brute_force():
    """Area-weighted edge permittivity on a graded grid, by hand."""
    g = W.cavity_uniform(3, 1e-3, seed=8)
    g.dz = np.array([1e-3, 3e-3, 1e-3])
    g.eps_r = np.array([1.0, 1.0, 5.0]); g.mu_r = np.ones(3); g.sig_e = np.zeros(3)
    g.sig_m = np.zeros(3); g.pec = np.array([0, 1, 0], np.uint8)
    g.mat_id[0] = 2                       # bottom layer eps 5
    s = yee.assemble(g)
    # Ex[k=1, j=1, i=0]: cells (0, 0|1, 0|1): bottom two have eps 5, weights dz/(dz0+dz1)
    idx = s.e_index[0][1, 1, 0]
    assert np.isclose(s.eps_edge[idx], (5.0 * 1e-3 + 1.0 * 3e-3) / 4e-3)
    # Ez[k=0, j=1, i=1]: four cells in layer 0 -> eps 5
    assert np.isclose(s.eps_edge[s.e_index[2][0, 1, 1]], 5.0)
    # PEC cell removes its 12 edges
    g.mat_id[1, 1, 1] = 1
    s2 = yee.assemble(g)
    assert s2.e_index[0][1, 1, 1] == -1 and s2.e_index[2][1, 2, 2] == -1
    assert s2.e_index[1][2, 1, 2] == -1 and s2.Ne < s.Ne


def test_unknown_counts_pec_box_and_paper_sizes():
    """P-j: N = 6 x cells for the paper's grids (storage layout, Table I,
    Secs. V-C, V-D); live unknowns of a PEC box: Ne = 3n(n-1)^2, Nh = 3n^2(n-1)."""
    for nx, ny, nz, N in GOLD["system_sizes"]["cases"]:
        assert 6 * nx * ny * nz == N
    for n in (2, 3, 5):
        s = yee.assemble(W.cavity_uniform(n, 1e-3, seed=9))
        assert s.Ne == 3 * n * (n - 1) ** 2 and s.Nh == 3 * n * n * (n - 1)


def test_stability_conditions_and_cfl():
    """C6/P-d: F + F^T >= 0 and R > 0 below the exact limit 2/sigma_max, R not
    positive definite above it; Eq. (CFL) <= exact limit; on a uniform box the
    exact limit equals the closed form of the highest mode."""
    g = _box(4, 3, 5, 1e-3, 0.8e-3, 1.2e-3)
    s = yee.assemble(g)
    dte = yee.exact_dt_limit(s)
    assert yee.cfl_dt(g) <= dte
    assert np.isclose(dte, max_stable_dt_uniform_box(4, 3, 5, 1e-3, 0.8e-3, 1.2e-3), rtol=1e-10)
    np.linalg.cholesky(s.R(0.999 * dte).toarray())
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(s.R(1.001 * dte).toarray())
    g.sig_e = np.array([0.0, 0.0, 0.3]); g.sig_m = np.array([0.0, 0.0, 50.0])
    s = yee.assemble(g)
    F = s.F().toarray()
    assert np.min(np.linalg.eigvalsh(F + F.T)) > -1e-12 * np.abs(F).max()


def test_graded_grid_resonance_converges():
    """Non-uniform spacing: the lowest resonance of a 1 m cube with a strongly
    graded z axis stays within 0.5 % of the analytic c/sqrt(2) / 2."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n = 14
    r = np.linspace(0.4, 1.6, n); dz = r / r.sum()
    g = _box(n, n, n, 1.0 / n, 1.0 / n, 1.0)
    g.dz = dz
    s = yee.assemble(g)
    Sm = sp.diags(1.0 / s.Dm)
    A = (s.K @ Sm @ s.K.T).tocsc()
    w2 = sla.eigsh(A, k=12, M=sp.diags(s.De).tocsc(), sigma=(2 * np.pi * 0.2e9) ** 2,
                   return_eigenvectors=False)
    f = np.sort(np.sqrt(np.abs(w2))) / (2 * np.pi)
    f = f[f > 1e6]
    fa = box_resonances_continuum(1.0, 1.0, 1.0, 3)
    assert abs(f[0] - fa[0]) / fa[0] < 5e-3


def test_matched_absorber_reduces_reflection():
    """The graded matched absorber (the paper's 4th-order 5-cell layer): a
    TE10 pulse in a PEC guide ending on absorbers at both x ends matches the
    unbounded guide (a much longer one, ends far outside the time window)
    several times better than the same guide with PEC ends; the added
    materials keep the matched condition sigma_m / mu = sigma_e / eps."""
    def guide(nx, xs, xp, ny=16, nz=8, d=1e-3):
        eps, mu, se, sm, pec = W.vacuum_table()
        g = W.GridSpec(nx, ny, nz, np.full(nx, d), np.full(ny, d), np.full(nz, d), eps, mu, se, sm, pec,
                       np.zeros((nz, ny, nx), np.uint16))
        jj, kk = np.meshgrid(np.arange(1, ny), np.arange(0, nz), indexing="xy")
        prof = np.sin(np.pi * jj.astype(float) / ny)
        for x, lst in ((xs, g.ports), (xp, g.probes)):
            lst.append(W.Port(W.COMP_EZ, kk.ravel().astype(np.int64), jj.ravel().astype(np.int64),
                              np.full(jj.size, x, np.int64), prof.ravel().copy()))
        return g

    T = 1400
    long_ = guide(800, 400, 420)
    dt = 0.99 * yee.cfl_dt(long_)
    u = W.excitation(long_, 15e9, 8e9, dt, T)
    run = lambda g: yee.Stepper(yee.assemble(g), dt).run(u)[0][:, 0]
    yl = run(long_)
    short = guide(160, 70, 90)
    absorbed = W.add_absorber(short, "xX")
    r_pec = np.linalg.norm(run(short) - yl) / np.linalg.norm(yl)
    r_abs = np.linalg.norm(run(absorbed) - yl) / np.linalg.norm(yl)
    assert r_abs < 0.2 * r_pec, (r_abs, r_pec)
    new = np.arange(short.nmat, absorbed.nmat)
    assert new.size > 0
    ratio_m = absorbed.sig_m[new] / (W.MU0 * absorbed.mu_r[new])
    ratio_e = absorbed.sig_e[new] / (W.EPS0 * absorbed.eps_r[new])
    assert np.allclose(ratio_m, ratio_e, rtol=1e-12)


def _exact_dt_uniform(N, d, c):
    """Largest stable dt of the leap-frog on a uniform box from the discrete
    dispersion relation sin^2(w dt/2)/(c dt)^2 = sum_i sin^2(m_i pi/(2 N_i))/d_i^2
    at its highest mode m_i = N_i - 1 (the right side times (c dt)^2 <= 1)."""
    s = sum(np.sin((n - 1) * np.pi / (2 * n)) ** 2 / di ** 2 for n, di in zip(N, d))
    return 1.0 / (c * np.sqrt(s))


def test_cfl_dt_pinned_to_dispersion_limit():
    """Eq. (CFL) against the exact limit of the discrete dispersion relation:
    on uniform anisotropic boxes the exact limit from the highest mode equals
    the oracle's power-iteration limit (small box, 1e-9) and approaches
    Eq. (CFL) from above as the box grows (within (pi/2N)^2 / 2 at N = 60);
    a uniform eps_r = 4 fill scales both by exactly 2."""
    from paper_1406_7042_gb300 import workloads as W
    c0 = yee.C0

    def box(N, d, eps_r=1.0):
        eps, mu, se, sm, pec = W.vacuum_table([(eps_r, 0.0)])
        nx, ny, nz = N
        return W.GridSpec(nx, ny, nz, np.full(nx, d[0]), np.full(ny, d[1]), np.full(nz, d[2]), eps, mu, se, sm, pec,
                          np.full((nz, ny, nx), 2 if eps_r != 1.0 else 0, np.uint16))

    N, d = (6, 5, 4), (1e-3, 0.7e-3, 1.3e-3)
    ex = _exact_dt_uniform(N, d, c0)
    assert abs(yee.exact_dt_limit(yee.assemble(box(N, d))) / ex - 1) < 1e-9
    assert yee.cfl_dt(box(N, d)) <= ex
    N = (60, 70, 80)
    ex = _exact_dt_uniform(N, d, c0)
    cfl = yee.cfl_dt(box(N, d))
    assert cfl <= ex and ex / cfl - 1 < 0.5 * (np.pi / (2 * 60)) ** 2
    assert abs(yee.cfl_dt(box(N, d, 4.0)) / cfl - 2.0) < 1e-14
    assert abs(_exact_dt_uniform(N, d, c0 / 2) / ex - 2.0) < 1e-14


@pytest.mark.parametrize("dims", [(4, 3, 1, 1e-3, 1.5e-3, 1e-3), (5, 5, 1, 1e-2, 1e-2, 1e-2)])
def test_single_layer_is_the_2d_tm_problem(dims):
    """A single layer of cells between the z plates (Sec. V-A/V-B 2-D cases):
    the live unknowns are Ez, Hx, Hy only, the eigenvalues of the step matrix
    follow the 2-D Yee dispersion relation (the closed form with m_z = 0), and
    Eq. (CFL) loses its z term: the exact limit equals the closed form of the
    highest 2-D mode, above Eq. (CFL) as in 3-D."""
    nx, ny, nz, a, b, c = dims
    g = _box(nx, ny, nz, a, b, c)
    s = yee.assemble(g)
    assert s.Ne == (nx - 1) * (ny - 1) and s.Nh == (nx - 1) * ny + nx * (ny - 1)
    assert int(s.e_mask[0].sum()) == 0 and int(s.e_mask[1].sum()) == 0 and int(s.h_mask[2].sum()) == 0
    dt = 0.99 * yee.cfl_dt(g)
    ev, ph = _nonstatic_phases(yee.amplification_matrix(s, dt))
    ref = box_mode_phases(nx, ny, nz, a, b, c, dt)
    assert np.allclose(np.abs(ev), 1.0, atol=1e-12)
    assert ph.size == ref.size == (nx - 1) * (ny - 1)
    assert np.max(np.abs(ph - ref)) < 1e-12
    exact = max_stable_dt_uniform_box(nx, ny, nz, a, b, c)
    assert abs(yee.exact_dt_limit(s) / exact - 1) < 1e-9
    assert yee.cfl_dt(g) <= exact and exact / yee.cfl_dt(g) < 1.25


def test_paper_2d_system_sizes():
    """Table I: N = 30,200 for the 101 x 101 2-D cavity; Sec. V-B: N = 48,440
    for the 41 x 401 guide (counted without its iris conductors) -- the live
    Ez, Hx, Hy unknowns of one layer between plates."""
    for wl, n in ((W.cavity2d_workload(), GOLD["system_sizes_2d"]["cavity"]),
                  (W.waveguide2d_workload(irises=False), GOLD["system_sizes_2d"]["waveguide"])):
        assert yee.assemble(wl.grid).N == n
