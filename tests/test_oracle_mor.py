"""Pins of the FP64 reduction oracle (Secs. II-C, II-D, III, IV): transfer
function of the recursion, moment matching, orthonormality, stability by
congruence below CFL, perturbation above it, convergence in q (no GPU)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import mor, yee
from paper_1406_7042_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def cav10():
    wl = W.cavity10_workload()
    s = yee.assemble(wl.grid)
    dt0 = wl.s_ref * yee.cfl_dt(wl.grid)
    b = mor.sprim_basis(s, dt0, wl.q, wl.L, wl.M, wl.fmax)
    red = mor.project(s, b.V1, b.V2)
    return wl, s, dt0, b, red


def _lossy_small():
    g = W.cavity_uniform(5, 1e-3, seed=11, nports=2, nprobes=2)
    g.eps_r = np.array([1.0, 1.0, 3.0]); g.mu_r = np.ones(3)
    g.sig_e = np.array([0.0, 0.0, 0.8]); g.sig_m = np.zeros(3)
    g.pec = np.array([0, 1, 0], np.uint8)
    g.mat_id[1:3, 1:4, 1:3] = 2
    g.dz = np.array([1e-3, 0.6e-3, 0.6e-3, 1e-3, 1.2e-3])
    return g


def test_expansion_points_eq_distrib():
    M = GOLD["expansion_points"]["M"]
    pts = mor.expansion_points(M, 2, 15e9, 1e-12)
    assert len(pts) == 3 and pts[0] == complex(M, 0)
    for l, z in enumerate(pts):
        assert math.isclose(abs(z), M, rel_tol=1e-15)
        assert math.isclose(np.angle(z), 2 * math.pi * (l / 2) * 15e9 * 1e-12, rel_tol=1e-12, abs_tol=1e-15)
    pair = mor.expansion_points(M, 1, 10e9, 2e-12, include_center=False)
    assert len(pair) == 1 and math.isclose(np.angle(pair[0]), 2 * math.pi * 10e9 * 2e-12)


def test_shifted_system_is_transfer_function_of_the_recursion():
    """Reading of Eq. (linear_system_solution): sum_n y^n z^{-n} of the FDTD
    impulse response equals C [z(R+F) - (R-F)]^{-1} z B (|z| = 1.1 > 1)."""
    g = _lossy_small()
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    T = 600
    z = 1.1 * np.exp(0.3j)
    H = mor.transfer_full(s, dt, z)
    for col in range(s.m):
        u = np.zeros((T, s.m)); u[0, col] = 1.0
        y, _, _ = yee.Stepper(s, dt).run(u)
        zs = z ** (-np.arange(T, dtype=np.float64))
        Hz = (y * zs[:, None]).sum(axis=0)
        assert np.allclose(Hz, H[:, col], rtol=1e-9, atol=1e-12 * np.abs(H).max())
    # the printed sign (R-F) + z(R+F) does not reproduce it
    A_printed = ((s.R(dt) - s.F()) + z * (s.R(dt) + s.F())).tocsc()
    import scipy.sparse.linalg as sla
    Hp = s.C() @ sla.spsolve(A_printed.astype(complex), s.B().toarray()[:, 0] * z)
    assert not np.allclose(Hp, H[:, 0], rtol=1e-3)


def test_schur_solve_equals_direct_solve():
    """Eqs. (reduced_linear_system_solution1/2) give the solution of A(z) x = b;
    at z = 0, A = -(R - F) is block upper triangular (Sec. IV-B)."""
    g = _lossy_small()
    s = yee.assemble(g)
    dt = 0.99 * yee.cfl_dt(g)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(s.N) + 1j * rng.standard_normal(s.N)
    import scipy.sparse.linalg as sla
    for z in (1.1 * np.exp(0.2j), 1.1, 0.0):
        x1, x2 = mor.schur_solve(s, dt, z, b[:s.Ne], b[s.Ne:])
        xd = sla.spsolve(mor.shifted_matrix(s, dt, z), b)
        assert np.allclose(np.concatenate([x1, x2]), xd, rtol=1e-10, atol=1e-12 * np.abs(xd).max())
    A0 = mor.shifted_matrix(s, dt, 0.0).toarray()
    assert np.allclose(np.tril(A0[:s.Ne, :s.Ne], -1), 0) and np.allclose(A0[s.Ne:, :s.Ne], 0)


def test_orthonormal_and_block_structure(cav10):
    """P-f: V1^T V1 = I, V2^T V2 = I."""
    _, s, _, b, _ = cav10
    for V in (b.V1, b.V2):
        assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) < 1e-13
    assert b.V1.shape[0] == s.Ne and b.V2.shape[0] == s.Nh


def test_moment_matching(cav10):
    """P-e: reduced and full moments about every expansion point agree for the
    first k block moments (1e-8 relative)."""
    _, s, dt0, b, red = cav10
    for z in b.points:
        mf = mor.moments_full(s, dt0, z, b.k)
        mr = mor.moments_reduced(red, dt0, z, b.k)
        for a, c in zip(mf, mr):
            assert np.max(np.abs(a - c)) <= 1e-8 * np.max(np.abs(a))
        zc = np.conj(z)
        assert np.allclose(mor.transfer_reduced(red, dt0, zc), mor.transfer_full(s, dt0, zc),
                           rtol=1e-8)


def test_moment_matching_lossy_multiport():
    g = _lossy_small()
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    b = mor.sprim_basis(s, dt0, 20, 2, 1.1, 60e9)
    red = mor.project(s, b.V1, b.V2)
    assert b.k == 2
    for z in b.points:
        for a, c in zip(mor.moments_full(s, dt0, z, b.k), mor.moments_reduced(red, dt0, z, b.k)):
            assert np.max(np.abs(a - c)) <= 1e-8 * np.max(np.abs(a))


def test_stable_by_congruence_below_cfl():
    """P-g / Sec. II-D: for s < 1, F~ + F~^T >= 0, R~ > 0, nothing is clipped and
    every eigenvalue of the reduced recursion is inside the unit circle."""
    g = _lossy_small()
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    b = mor.sprim_basis(s, dt0, 20, 2, 1.1, 60e9)
    red = mor.project(s, b.V1, b.V2)
    Ft = red.F()
    assert np.min(np.linalg.eigvalsh(Ft + Ft.T)) > -1e-12 * np.abs(Ft).max()
    np.linalg.cholesky(red.R(dt0))
    _, ncl, sv = mor.perturb(red, dt0, GOLD["perturbation"]["gamma"])
    assert ncl == 0 and sv.max() < 2 / dt0
    lam = np.abs(np.linalg.eigvals(mor.reduced_amplification(red, dt0)))
    assert lam.max() <= 1 + 1e-12


def test_lossless_reduced_energy_conserved(cav10):
    _, s, dt0, b, red = cav10
    Phi = mor.reduced_amplification(red, dt0)
    lam = np.abs(np.linalg.eigvals(Phi))
    assert np.allclose(lam, 1.0, atol=1e-10)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(red.q1 + red.q2)
    R = red.R(dt0)
    w0 = x @ R @ x
    for _ in range(5000):
        x = Phi @ x
    assert abs(x @ R @ x - w0) / w0 < 1e-11


def test_singular_value_criterion_eq_singular_limit(cav10):
    """C11: R~ > 0 iff sigma_max(D~e^{-1/2} K~ D~m^{-1/2}) < 2/dt."""
    _, _, _, _, red = cav10
    smax = mor.singular_values(red).max()
    np.linalg.cholesky(red.R(0.999 * 2 / smax))
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(red.R(1.001 * 2 / smax))


def test_perturbation_above_cfl(cav10):
    """P-h: at s = 4.95 some sigma_i exceed gamma 2/dt; after the procedure of
    Sec. III-A all sigma' <= gamma 2/dt and |lambda| <= 1; a Cholesky factor
    gives the same K~' as the symmetric square root."""
    wl, s, dt0, b, red = cav10
    gamma = GOLD["perturbation"]["gamma"]
    dt = 5 * dt0
    lam0 = np.abs(np.linalg.eigvals(mor.reduced_amplification(red, dt)))
    assert lam0.max() > 1 + 1e-6
    pr, ncl, sv = mor.perturb(red, dt, gamma)
    assert ncl == int(np.sum(sv >= gamma * 2 / dt)) and ncl > 0
    s2 = mor.singular_values(pr)
    assert s2.max() <= gamma * 2 / dt * (1 + 1e-12)
    lam = np.abs(np.linalg.eigvals(mor.reduced_amplification(pr, dt)))
    assert lam.max() <= 1 + 1e-12
    # Cholesky route (independent of the oracle's eigh square root)
    Le = np.linalg.cholesky(red.De); Lm = np.linalg.cholesky(red.Dm)
    Mc = sl.solve_triangular(Le, red.K, lower=True)
    Mc = sl.solve_triangular(Lm, Mc.T, lower=True).T
    U, sg, Wt = np.linalg.svd(Mc, full_matrices=False)
    sg = np.minimum(sg, gamma * 2 / dt)
    Kc = Le @ (U * sg) @ Wt @ Lm.T
    assert np.max(np.abs(Kc - pr.K)) <= 1e-12 * np.abs(pr.K).max()
    # no-op when nothing exceeds the limit
    same, n0, _ = mor.perturb(red, 0.5 * dt0, gamma)
    assert n0 == 0 and np.max(np.abs(same.K - red.K)) <= 1e-12 * np.abs(red.K).max()


def test_demo_perturbation_of_full_system():
    """Sec. III-B on the full system (small cube): s = 1.98 has eigenvalues
    outside the unit circle; after perturbing K they are all on it."""
    n = 5
    g = W.cavity_uniform(n, 1.0 / n, seed=12)
    s = yee.assemble(g)
    dt = GOLD["demo_cavity"]["s_above"] * yee.cfl_dt(g)
    lam = np.abs(np.linalg.eigvals(yee.amplification_matrix(s, dt)))
    assert lam.max() > 1.0 + 1e-3
    Kp, ncl, _ = mor.perturb_full(s, dt, GOLD["perturbation"]["gamma"])
    red = mor.Reduced(np.diag(s.De), np.diag(s.Dse), np.diag(s.Dm), np.diag(s.Dsm), Kp,
                      s.BE.toarray(), np.zeros((s.Nh, s.m)), s.CE.toarray())
    lam2 = np.abs(np.linalg.eigvals(mor.reduced_amplification(red, dt)))
    assert ncl > 0 and np.allclose(lam2, 1.0, atol=1e-9)


def test_reduced_run_matches_fdtd_and_converges_in_q():
    """P-i: the probe error at s = 0.99 falls with q; with V spanning the whole
    space the reduced model reproduces FDTD to rounding."""
    g = W.cavity_uniform(4, 1e-3, seed=13)
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    u = W.excitation(g, 40e9, 60e9, dt0, 600)
    yref, _, _ = yee.Stepper(s, dt0).run(u)
    errs = []
    for q in (5, 10, 20):
        b = mor.sprim_basis(s, dt0, q, 2, 1.1, 70e9)
        red = mor.project(s, b.V1, b.V2)
        errs.append(mor.rel_l2(mor.reduced_run(red, dt0, u), yref))
    assert errs[1] < errs[0] and errs[2] < errs[1]
    V1 = np.eye(s.Ne); V2 = np.eye(s.Nh)
    full = mor.project(s, V1, V2)
    assert mor.rel_l2(mor.reduced_run(full, dt0, u), yref) < 1e-10


def test_cavity10_reduced_error_small(cav10):
    wl, s, dt0, b, red = cav10
    u = W.excitation(wl.grid, wl.f0, wl.bw, dt0, wl.nsteps_ref)
    yref, _, _ = yee.Stepper(s, dt0).run(u)
    y = mor.reduced_run(red, dt0, u)
    assert mor.rel_l2(y, yref) < 1e-5


def test_moments_pinned_to_transfer_function_derivatives():
    """moments_full about z_l against the Taylor coefficients of the transfer
    function itself: with G(z) = H(z)/z = C A(z)^{-1} B and dA/dz = R + F,
    M_j = (-1)^j G^(j)(z_l)/j!, taken from transfer_full on a circle around
    z_l by the Cauchy integral (trapezoid rule, spectrally accurate) -- a
    wrong chain operator or sign fails it."""
    from tests.helpers import ragged_grid
    g = ragged_grid(12, 10, 9, seed=13)
    s = yee.assemble(g)
    dt = 0.9 * yee.cfl_dt(g)
    for z in (1.1 + 0j, 1.1 * np.exp(0.3j)):
        rho, npts, count = 0.03, 24, 4
        th = 2 * np.pi * np.arange(npts) / npts
        Gs = [mor.transfer_full(s, dt, z + rho * np.exp(1j * t)) / (z + rho * np.exp(1j * t)) for t in th]
        mom = mor.moments_full(s, dt, z, count)
        for j in range(count):
            taylor = sum(G * np.exp(-1j * j * t) for G, t in zip(Gs, th)) / npts / rho ** j
            ref = (-1) ** j * taylor
            assert np.max(np.abs(mom[j] - ref)) <= 1e-6 * np.max(np.abs(ref)), (z, j)
