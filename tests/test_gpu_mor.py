"""Parity of the CUDA reduction path (mor_build_basis, mor_project,
mor_perturb, mor_run, mor_compare through the C ABI) with the FP64 oracle.

Each stage is checked on its own against the oracle applied to the GPU's
inputs of that stage (so a mismatch points at one kernel), and the pipeline
end to end against the oracle pipeline."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mor, yee  # noqa: E402
from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402
from paper_1406_7042_gb300 import workloads as W  # noqa: E402
from tests.helpers import drive, ragged_grid  # noqa: E402

GAMMA = 0.9999
TOL_RED_F32 = 1e-3   # reduced-model probe error against the FP64 oracle (FP32 path)


def _vectors_to_oracle(sys, V, comps):
    """(q, 3nc) storage-layout basis -> oracle unknown ordering (live edges only)."""
    q = V.shape[0]
    nz, ny, nx = sys.shape
    A = V.reshape(q, 3, nz, ny, nx)
    masks = sys.e_mask if comps == "E" else sys.h_mask
    return np.concatenate([A[:, c][:, masks[c]] for c in range(3)], axis=1).T


def _gpu_reduced(model):
    return mor.Reduced(model.get("De"), model.get("Dse"), model.get("Dm"), model.get("Dsm"), model.get("K"),
                       model.get("BE"), np.zeros((model.get("Dm").shape[0], model.get("BE").shape[1])),
                       model.get("CE"))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_edge_props_match_oracle(prec):
    """A1: per-edge eps, sigma (area-weighted over the cells around an E edge)
    and mu, sigma_m (length-weighted over the two cells of an H edge's dual
    edge) used by the reduction kernels, with dead edges marked by zero."""
    g = ragged_grid(29, 17, 13, seed=31, magnetic=True)
    s = yee.assemble(g)
    grid = F.Grid(g, prec)
    ep = grid.edge_props().cpu().numpy().astype(np.float64)
    tol = 1e-13 if prec == "f64" else 1e-6
    eps_o = s.De / s.vol_e
    sig_o = s.Dse / s.vol_e
    mu_o = s.Dm / s.vol_h
    sgm_o = s.Dsm / s.vol_h
    off = 0
    for c in range(3):
        n = int(s.e_mask[c].sum())
        assert np.all(ep[0, c][~s.e_mask[c]] == 0)
        assert np.allclose(ep[0, c][s.e_mask[c]], eps_o[off:off + n], rtol=tol, atol=0)
        assert np.allclose(ep[1, c][s.e_mask[c]], sig_o[off:off + n], rtol=tol, atol=tol * sig_o.max())
        off += n
    off = 0
    for c in range(3):
        n = int(s.h_mask[c].sum())
        assert np.all(ep[2, c][~s.h_mask[c]] == 0)
        assert np.allclose(ep[2, c][s.h_mask[c]], mu_o[off:off + n], rtol=tol, atol=0)
        assert np.allclose(ep[3, c][s.h_mask[c]], sgm_o[off:off + n], rtol=tol, atol=tol * sgm_o.max())
        off += n


@pytest.fixture(scope="module")
def cav10():
    wl = W.cavity10_workload()
    g = wl.grid
    s = yee.assemble(g)
    dt0 = wl.s_ref * yee.cfl_dt(g)
    ob = mor.sprim_basis(s, dt0, wl.q, wl.L, wl.M, wl.fmax)
    grid = F.Grid(g, "f64")
    gb = F.Basis(grid, wl.q, dt0, wl.L, wl.M, wl.fmax, tol=1e-13)
    return wl, s, dt0, ob, grid, gb


@pytest.mark.parametrize("q,L,center", [(6, 0, True), (8, 1, False)])
def test_basis_matches_oracle_f64(cav10, q, L, center):
    """Columns of V1, V2 against the oracle for short chains (a real point with
    six moments; the complex pair with two).  Each chain vector is the small
    remainder of A^{-1}(R+F) q after orthogonalisation, so solve error grows by
    the inverse of that remainder at every moment: exact column parity is only
    well posed for short chains; the long multi-point chains of the default
    settings are checked through their invariants (moments, waveforms)."""
    wl, s, dt0, _, grid, _ = cav10
    ob = mor.sprim_basis(s, dt0, q, L, wl.M, wl.fmax, include_center=center, defl_tol=1e-6)
    gb = F.Basis(grid, q, dt0, L, wl.M, wl.fmax, include_center=center, tol=1e-13, defl_tol=1e-6)
    inf = gb.info()
    assert inf["max_resid"] <= 2e-13
    V1 = _vectors_to_oracle(s, gb.V(1).cpu().numpy(), "E")
    V2 = _vectors_to_oracle(s, gb.V(2).cpu().numpy(), "H")
    full1 = gb.V(1).cpu().numpy().reshape(inf["q1"], 3, *s.shape)
    for c in range(3):
        assert np.all(full1[:, c][:, ~s.e_mask[c]] == 0)   # dead edges carry exactly zero
    assert np.max(np.abs(V1.T @ V1 - np.eye(V1.shape[1]))) < 1e-12
    assert np.max(np.abs(V2.T @ V2 - np.eye(V2.shape[1]))) < 1e-12
    for Vg, Vo in ((V1, ob.V1), (V2, ob.V2)):
        cosines = np.linalg.svd(Vg.T @ Vo, compute_uv=False)
        msg = f"q gpu {Vg.shape[1]} oracle {Vo.shape[1]}, cosines {np.round(cosines, 9)}"
        assert Vg.shape[1] == Vo.shape[1], msg
        assert cosines.min() > 1 - 1e-8, msg
        assert np.max(np.abs(Vg - Vo)) < 1e-5, msg   # same pool order and CGS2


def test_projection_kernel_matches_oracle_on_gpu_basis(cav10):
    wl, s, dt0, ob, grid, gb = cav10
    V1 = _vectors_to_oracle(s, gb.V(1).cpu().numpy(), "E")
    V2 = _vectors_to_oracle(s, gb.V(2).cpu().numpy(), "H")
    ref = mor.project(s, V1, V2)
    model = F.Model(grid, gb)
    for name, R in (("De", ref.De), ("Dse", ref.Dse), ("Dm", ref.Dm), ("Dsm", ref.Dsm), ("K", ref.K),
                    ("BE", ref.BE), ("CE", ref.CE)):
        G = model.get(name)
        scale = max(np.abs(R).max(), 1e-300)
        assert G.shape == R.shape, name
        assert np.max(np.abs(G - R)) <= 1e-11 * scale, name


@pytest.mark.parametrize("k", [1, 5, 10])
def test_perturbation_and_run_match_oracle(cav10, k):
    wl, s, dt0, ob, grid, gb = cav10
    model = F.Model(grid, gb)
    red = _gpu_reduced(model)
    dt = k * dt0 if k > 1 else dt0
    ncl = model.perturb(dt, GAMMA)
    pr, ncl_o, sv = mor.perturb(red, dt, GAMMA)
    assert ncl == ncl_o
    if k > 1:
        assert ncl > 0
    sg = np.sort(model.get("sigma").ravel())[::-1][:sv.size]
    assert np.allclose(sg, np.sort(sv)[::-1], rtol=1e-10, atol=1e-12 * sv.max())
    Kp = model.get("Kp")
    assert np.max(np.abs(Kp - pr.K)) <= 1e-9 * np.abs(pr.K).max()
    n = 400
    u = W.excitation(wl.grid, wl.f0, wl.bw, dt, n)
    y = model.run(torch.tensor(u, device="cuda")).cpu().numpy()
    yo = mor.reduced_run(pr, dt, u)
    assert np.max(np.abs(y - yo)) <= 1e-9 * np.abs(yo).max()
    lam = np.abs(np.linalg.eigvals(mor.reduced_amplification(pr, dt)))
    assert lam.max() <= 1 + 1e-9


def test_pipeline_end_to_end_f64(cav10):
    wl, s, dt0, ob, grid, gb = cav10
    red_o = mor.project(s, ob.V1, ob.V2)
    model = F.Model(grid, gb)
    u = W.excitation(wl.grid, wl.f0, wl.bw, dt0, wl.nsteps_ref)
    yref = grid.step(dt0, torch.tensor(u, device="cuda"), reset=True)
    for sf, ns in zip(wl.s_red, wl.nsteps_red):
        k = int(round(sf / 0.99))
        dt = k * dt0
        model.perturb(dt, GAMMA)
        pr_o, _, _ = mor.perturb(red_o, dt, GAMMA)
        uu = W.excitation(wl.grid, wl.f0, wl.bw, dt, ns)
        yg = model.run(torch.tensor(uu, device="cuda"))
        yo = mor.reduced_run(pr_o, dt, uu)
        # different (equally valid) deflation choices: both models must be
        # accurate; at large steps their own time-discretisation error dominates
        e = F.compare(yg, yref, stride=k, offset=k - 1)
        eo = mor.rel_l2(yo, yref.cpu().numpy()[k - 1::k][:ns])
        e_host = mor.rel_l2(yg.cpu().numpy(), yref.cpu().numpy()[k - 1::k][:ns])
        assert abs(e - e_host) <= 1e-9 * max(e_host, 1e-12) + 1e-12   # mor_compare itself
        if k == 1:
            assert e < 1e-5 and eo < 1e-5
        else:
            assert abs(e - eo) <= 0.05 * eo, (k, e, eo)


def test_moments_of_gpu_model_match_full_system(cav10):
    """P-e on the GPU's reduced model: moments about every expansion point."""
    wl, s, dt0, ob, grid, gb = cav10
    model = F.Model(grid, gb)
    red = _gpu_reduced(model)
    for z in ob.points:
        for a, c in zip(mor.moments_full(s, dt0, z, ob.k), mor.moments_reduced(red, dt0, z, ob.k)):
            assert np.max(np.abs(a - c)) <= 1e-7 * np.max(np.abs(a))


def _lossy_ragged():
    g = ragged_grid(29, 17, 13, seed=31, magnetic=False)
    g.ports = g.ports[:2]
    return g


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("center", [True, False])
def test_shifted_solve_parity_lossy_multiport(prec, center):
    """One block moment per port (k = 1): V1, V2 are the orthonormalised E and
    H parts of A(z)^{-1} B (real point z = M, or Re/Im at the complex pair),
    so this checks the Schur-complement CGS solve itself against sparse LU."""
    g = _lossy_ragged()
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    L, q = (0, 2) if center else (1, 4)
    ob = mor.sprim_basis(s, dt0, q, L, 1.1, 60e9, include_center=center, defl_tol=1e-6)
    grid = F.Grid(g, prec)
    gb = F.Basis(grid, q, dt0, L, 1.1, 60e9, include_center=center,
                 tol=1e-12 if prec == "f64" else 1e-6, defl_tol=1e-6)
    for which, comps, Vo in ((1, "E", ob.V1), (2, "H", ob.V2)):
        Vg = _vectors_to_oracle(s, gb.V(which).cpu().numpy().astype(np.float64), comps)
        cosines = np.linalg.svd(Vg.T @ Vo, compute_uv=False)
        assert Vg.shape[1] == Vo.shape[1]
        assert cosines.min() > 1 - (1e-10 if prec == "f64" else 1e-6), cosines


@pytest.mark.parametrize("center", [True, False])
def test_cocg_f64_matches_oracle(center):
    """The COCG path (volume-weighted unconjugated products, gradient-corrected
    preconditioner) in FP64 solves the same shifted systems as the oracle's
    sparse LU: one block moment per port, principal cosines to 1e-10."""
    g = _lossy_ragged()
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    L, q = (0, 2) if center else (1, 4)
    ob = mor.sprim_basis(s, dt0, q, L, 1.1, 60e9, include_center=center, defl_tol=1e-6)
    grid = F.Grid(g, "f64")
    gb = F.Basis(grid, q, dt0, L, 1.1, 60e9, include_center=center, tol=1e-12, defl_tol=1e-6, solver="cocg")
    assert gb.status == F.FDTD_OK
    for which, comps, Vo in ((1, "E", ob.V1), (2, "H", ob.V2)):
        Vg = _vectors_to_oracle(s, gb.V(which).cpu().numpy(), comps)
        cosines = np.linalg.svd(Vg.T @ Vo, compute_uv=False)
        assert Vg.shape[1] == Vo.shape[1]
        assert cosines.min() > 1 - 1e-10, cosines


def _graded20():
    """The bench cavity's construction (0.5 mm cells, z graded to a 2-cell
    0.05 mm slab of eps_r 4, lossy seeded blocks) at 20^3, small enough for
    the oracle's sparse LU to factorise three shifted systems in a minute."""
    g = W.cavity_graded(20)
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    fmax = 15e9
    return g, s, dt0, fmax, 1.0 + np.pi * fmax * dt0


def test_cocg_refined_solves_reach_paper_tolerance():
    """FP32 fields on the finely graded cavity: inside the basis build the FP64
    refinement takes every shifted solve to a true residual <= 1e-4
    (Sec. IV-B), which FP32 arithmetic alone cannot reach there."""
    g, s, dt0, fmax, M = _graded20()
    grid = F.Grid(g, "f32")
    gb = F.Basis(grid, 20, dt0, 2, M, fmax, tol=1e-4, defl_tol=1e-5)
    inf = gb.info()
    assert gb.status == F.FDTD_OK
    assert 0 < inf["max_resid"] <= 1e-4, inf
    assert inf["max_iters"] < 1000, inf


def _storage_to_live(s, x):
    """(nb, 3, nz, ny, nx) storage-layout E blocks -> (nb, Ne) live unknowns."""
    return np.stack([np.concatenate([x[b, c][s.e_mask[c]] for c in range(3)]) for b in range(x.shape[0])])


def _live_to_storage(s, v):
    nz, ny, nx = s.shape
    out = np.zeros((v.shape[0], 3, nz, ny, nx), v.dtype)
    for b in range(v.shape[0]):
        off = 0
        for c in range(3):
            n = int(s.e_mask[c].sum())
            out[b, c][s.e_mask[c]] = v[b, off:off + n]
            off += n
    return out


@pytest.mark.parametrize("case,prec,solver,tol,fwd_tol", [
    ("ragged", "f64", "cgs", 1e-10, 1e-7),
    ("ragged", "f64", "bicgstab", 1e-10, 1e-7),
    ("ragged", "f64", "cocg", 1e-10, 1e-7),
    ("ragged", "f32", "cocg", 1e-4, 2e-3),
    ("graded", "f32", "cocg", 1e-4, 2e-3),
])
def test_shifted_solve_matches_lu(case, prec, solver, tol, fwd_tol):
    """A4 through mor_shifted_solve: S(z) x = b for seeded complex b at points
    of the arc of Eq. (distrib), against the oracle's sparse LU of the Schur
    complement (Eqs. (reduced_linear_system_solution1/2)), element by
    element.  The GPU works in per-volume rows, S_gpu = V_e^{-1} S."""
    if case == "ragged":
        g = _lossy_ragged()
        s = yee.assemble(g)
        dt0 = 0.99 * yee.cfl_dt(g)
        zs = [1.1 + 0j, 1.1 * np.exp(1j * 2 * np.pi * 60e9 * dt0)]
    else:
        g, s, dt0, fmax, M = _graded20()
        zs = [M + 0j, M * np.exp(1j * 2 * np.pi * fmax * dt0)]
    rng = np.random.default_rng(7)
    bl = rng.standard_normal((len(zs), s.Ne)) + 1j * rng.standard_normal((len(zs), s.Ne))
    grid = F.Grid(g, prec)
    cdt = torch.complex128 if prec == "f64" else torch.complex64
    bt = torch.tensor(_live_to_storage(s, bl), dtype=cdt, device="cuda")
    x, iters, resid = F.shifted_solve(grid, dt0, zs, bt, tol=tol, solver=solver)
    xl = _storage_to_live(s, x.cpu().numpy().astype(np.complex128))
    for b, z in enumerate(zs):
        a11, a22 = mor.schur_blocks(s, dt0, z)
        K = s.K.astype(np.complex128)
        S = (sp.diags(a11) + z * K @ sp.diags(1.0 / a22) @ K.T).tocsc()
        xo = sla.splu(S).solve(s.vol_e * bl[b])
        assert resid[b] <= tol, (b, resid, iters)
        assert np.linalg.norm(xl[b] - xo) <= fwd_tol * np.linalg.norm(xo), (b, np.linalg.norm(xl[b] - xo) / np.linalg.norm(xo))


def test_reduced_model_matches_oracle_at_bench_settings():
    """Separates the GPU path's error from the method's on a config-2-shaped
    grid: FP32 fields, COCG with FP64 refinement, L = 2, M = 1 + pi fmax dt0,
    q = 60.  Near z = 1 the later chain vectors are dependent to below the
    solves' error, so the GPU basis keeps other columns than the exact one;
    what must agree is the model.  Sec. IV-B picks the residual limit at which
    the iterative solver matches the direct one (1e-4 on the paper's cases,
    M = 1.1); on this arc the shifted systems are closer to singular and the
    same criterion takes 1e-6 (at 1e-4 the model differs from the direct-solver
    model by about 5e-3).  With it, the GPU model's probe error against the
    oracle's full-order run at s = 0.99 is at most the oracle reduction's own
    (sparse-LU chains, CGS2, projection, reduced leap-frog) plus 1e-3."""
    g, s, dt0, fmax, M = _graded20()
    q, L, nref = 60, 2, 4000
    ob = mor.sprim_basis(s, dt0, q, L, M, fmax, defl_tol=1e-5)
    red = mor.project(s, ob.V1, ob.V2)
    uref = W.excitation(g, 10e9, 10e9, dt0, nref)
    yref = yee.Stepper(s, dt0).run(uref)[0]
    g32 = F.Grid(g, "f32")
    b32 = F.Basis(g32, q, dt0, L, M, fmax, tol=1e-6, defl_tol=1e-5)
    assert b32.status == F.FDTD_OK and b32.info()["max_resid"] <= 1e-6
    m32 = F.Model(g32, b32)
    u = W.excitation(g, 10e9, 10e9, dt0, nref)
    pr, _, _ = mor.perturb(red, dt0, GAMMA)
    yo = mor.reduced_run(pr, dt0, u)
    m32.perturb(dt0, GAMMA)
    y32 = m32.run(torch.tensor(u, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    e_or, e_32 = mor.rel_l2(yo, yref), mor.rel_l2(y32, yref)
    assert e_or < 1e-4, e_or  # the exact reduction is converged at this order
    assert e_32 <= e_or + TOL_RED_F32, (e_32, e_or)


@pytest.mark.parametrize("prec,q,tol,tol_cta", [("f64", 120, 1e-9, 1e-11), ("f32", 200, 5e-3, 1e-5)])
def test_cluster_reduced_run_matches_oracle(prec, q, tol, tol_cta, monkeypatch):
    """A8, the thread-block-cluster form (row slices of the step matrices
    resident per CTA, state exchanged through distributed shared memory; the
    default at every order where a cluster can be scheduled, forced here):
    steps the GPU-projected model like the one-CTA form in the same precision
    (only the summation order differs) and, in FP64, like the oracle's reduced
    leap-frog on the same matrices, below and above CFL (FP32 stepping of this
    ill-conditioned q = 200 model stays within 5e-3 of the FP64 recursion)."""
    g, s, dt0, fmax, M = _graded20()
    grid = F.Grid(g, prec)
    gb = F.Basis(grid, q, dt0, 2, M, fmax, tol=1e-8 if prec == "f64" else 1e-5, defl_tol=1e-6, solver="cocg")
    model = F.Model(grid, gb)
    red = _gpu_reduced(model)
    monkeypatch.setenv("FDTDMOR_RUN", "cluster")
    dtype = torch.float64 if prec == "f64" else torch.float32
    for kk in (1, 5):
        dt = kk * dt0
        model.perturb(dt, GAMMA)
        pr, _, _ = mor.perturb(red, dt, GAMMA)
        u = W.excitation(g, 10e9, 10e9, dt, 600)
        yo = mor.reduced_run(pr, dt, u)
        ut = torch.tensor(u, dtype=dtype, device="cuda")
        yg = model.run(ut).cpu().numpy().astype(np.float64)
        assert mor.rel_l2(yg, yo) < tol, (kk, mor.rel_l2(yg, yo))
        monkeypatch.setenv("FDTDMOR_RUN", "cta")
        yc = model.run(ut).cpu().numpy().astype(np.float64)
        monkeypatch.setenv("FDTDMOR_RUN", "cluster")
        assert mor.rel_l2(yg, yc) < tol_cta, (kk, mor.rel_l2(yg, yc))


@pytest.mark.parametrize("orth,mat_tol", [("tf32", 5e-5), ("bf16", 5e-4)])
def test_tensor_core_projection_matches_oracle(orth, mat_tol):
    """A6 / A10: with a TF32 or BF16 basis build the five Gram products of the
    projection run on the tensor cores in split precision; on the GPU basis
    they match the oracle's FP64 projection of the same columns, and the
    reduced model's probe waveforms match the oracle's reduced leap-frog on
    that projection to 1e-3 below and above CFL (the 100x50x24 microstrip with
    matched absorbers on five faces, q = 100)."""
    wl = W.microstrip_workload(downscale=True, absorbing=True)
    g = wl.grid
    s = yee.assemble(g)
    dt0 = wl.s_ref * yee.cfl_dt(g)
    grid = F.Grid(g, "f32")
    gb = F.Basis(grid, 100, dt0, wl.L, 1.0 + np.pi * wl.fmax * dt0, wl.fmax, tol=1e-5, defl_tol=1e-5, orth=orth)
    model = F.Model(grid, gb)
    V1 = _vectors_to_oracle(s, gb.V(1).cpu().numpy().astype(np.float64), "E")
    V2 = _vectors_to_oracle(s, gb.V(2).cpu().numpy().astype(np.float64), "H")
    ref = mor.project(s, V1, V2)
    for name in ("De", "Dse", "Dm", "Dsm", "K"):
        G, R = model.get(name), getattr(ref, name)
        assert np.max(np.abs(G - R)) <= mat_tol * np.abs(R).max(), (name, np.max(np.abs(G - R)) / np.abs(R).max())
    for kk in (1, 5):
        dt = kk * dt0
        model.perturb(dt, GAMMA)
        pr, _, _ = mor.perturb(ref, dt, GAMMA)
        u = W.excitation(g, wl.f0, wl.bw, dt, 4000 // kk)
        yo = mor.reduced_run(pr, dt, u)
        yg = model.run(torch.tensor(u, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
        assert mor.rel_l2(yg, yo) <= TOL_RED_F32, (kk, mor.rel_l2(yg, yo))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_model_save_load_reuses_one_reduction(prec, tmp_path):
    """mor_model_save / mor_model_load: the reloaded model carries the same
    projected matrices bit for bit, and perturbed and stepped at several s it
    gives the same probe waveforms as the model it was saved from."""
    g = _lossy_ragged()
    grid = F.Grid(g, prec)
    dt0 = 0.99 * grid.cfl_dt()
    gb = F.Basis(grid, 12, dt0, 1, 1.1, 60e9, tol=1e-10 if prec == "f64" else 1e-5)
    model = F.Model(grid, gb)
    path = str(tmp_path / "model.bin")
    model.save(path)
    back = F.Model.load(path, grid)
    for name in ("De", "Dse", "Dm", "Dsm", "K", "BE", "CE"):
        assert np.array_equal(back.get(name), model.get(name)), name
    dtype = torch.float64 if prec == "f64" else torch.float32
    for k in (1, 3, 6):
        dt = k * dt0
        u = torch.tensor(drive(g, dt, 200), dtype=dtype, device="cuda")
        assert model.perturb(dt, GAMMA) == back.perturb(dt, GAMMA)
        assert torch.equal(model.run(u), back.run(u)), k
    with open(path, "r+b") as f:
        f.write(b"NOTAMODL")
    with pytest.raises(F.FdtdError):
        F.Model.load(path, grid)


def test_lossy_multiport_moments_and_stages_f64():
    """Two ports (block Arnoldi across ports), loss, PEC blocks, graded cells:
    the GPU model matches the full system's moments at every point, and
    projection / perturbation / run agree with the oracle on the GPU basis
    (Pe != I here because of the loss)."""
    g = _lossy_ragged()
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    q, L, fmax = 24, 1, 60e9
    grid = F.Grid(g, "f64")
    gb = F.Basis(grid, q, dt0, L, 1.1, fmax, tol=1e-12)
    model = F.Model(grid, gb)
    red = _gpu_reduced(model)
    pts = mor.expansion_points(1.1, L, fmax, dt0)
    k = q // (3 * 2)
    for z in pts:
        for a, c in zip(mor.moments_full(s, dt0, z, k), mor.moments_reduced(red, dt0, z, k)):
            assert np.max(np.abs(a - c)) <= 1e-6 * np.max(np.abs(a))
    V1 = _vectors_to_oracle(s, gb.V(1).cpu().numpy(), "E")
    V2 = _vectors_to_oracle(s, gb.V(2).cpu().numpy(), "H")
    ref = mor.project(s, V1, V2)
    for name in ("De", "Dse", "Dm", "Dsm", "K", "BE", "CE"):
        G, R = model.get(name), getattr(ref, name)
        assert np.max(np.abs(G - R)) <= 1e-11 * max(np.abs(R).max(), 1e-300), name
    for kk in (1, 3):
        dt = kk * dt0
        model.perturb(dt, GAMMA)
        pr, _, _ = mor.perturb(red, dt, GAMMA)
        uu = drive(g, dt, 300)
        yg = model.run(torch.tensor(uu, device="cuda")).cpu().numpy()
        yo = mor.reduced_run(pr, dt, uu)
        assert mor.rel_l2(yg, yo) < 1e-9


def test_invalid_reduction_arguments():
    g = ragged_grid(seed=5)
    grid = F.Grid(g, "f32")
    with pytest.raises(F.FdtdError):
        F.Basis(grid, 0, 1e-13)
    with pytest.raises(F.FdtdError):
        F.Basis(grid, 10, -1.0)
    g2 = ragged_grid(seed=5)
    g2.ports = []
    grid2 = F.Grid(g2, "f32")
    with pytest.raises(F.FdtdError):
        F.Basis(grid2, 10, 0.5 * grid2.cfl_dt())


def test_solver_iteration_cap_reports_noconv():
    g = ragged_grid(21, 11, 9, seed=6)
    grid = F.Grid(g, "f32")
    b = F.Basis(grid, 8, 0.9 * grid.cfl_dt(), 1, 1.1, 50e9, tol=1e-12, maxit=3, allow_noconv=True)
    assert b.status == F.FDTD_ENOCONV
    assert b.info()["max_iters"] == 3


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_schur_apply_matches_oracle(prec, tol):
    """mor_schur_apply against the oracle's A11 - A12 A22^-1 A21 (rows scaled
    by the edge volumes), several complex shifts at once."""
    from oracle import mor
    g = ragged_grid(nx=20, ny=11, nz=9, seed=41)
    sys = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    zs = [1.05 * np.exp(0.3j), 0.97 * np.exp(-0.1j), 1.2 + 0j]
    rng = np.random.default_rng(7)
    Ne, Nh = sys.Ne, sys.Nh
    K = sys.K.astype(np.complex128)

    def arrays(v):
        a = sys.to_arrays(np.concatenate([v, np.zeros(Nh)]))
        return np.stack([a["Ex"], a["Ey"], a["Ez"]])

    vol = arrays(sys.vol_e)
    xs, ys = [], []
    for z in zs:
        xe = rng.standard_normal(Ne) + 1j * rng.standard_normal(Ne)
        a11, a22 = mor.schur_blocks(sys, dt0, z)
        y = a11 * xe - K @ ((-z * (K.T @ xe)) / a22)
        xs.append(arrays(xe.real) + 1j * arrays(xe.imag))
        ys.append(arrays(y.real) + 1j * arrays(y.imag))
    ctype = torch.complex128 if prec == "f64" else torch.complex64
    grid = F.Grid(g, prec)
    x = torch.tensor(np.stack(xs), dtype=ctype, device="cuda")
    yg = F.schur_apply(grid, dt0, zs, x).cpu().numpy() * vol[None]
    yo = np.stack(ys)
    assert np.max(np.abs(yg - yo)) <= tol * np.abs(yo).max()


@pytest.mark.parametrize("orth,ortho_tol,span_tol", [("tf32", 2e-5, 2e-3), ("bf16", 2e-5, 2e-2)])
def test_tensor_core_gram_schmidt_basis(orth, ortho_tol, span_tol):
    """Basis with the first CGS2 pass on the tcgen05 tensor cores (TF32 / BF16
    inputs) and the second in FP32: orthonormality at FP32 level, the spanned
    space matches the FP32 basis, and the projected model (tensor-core Gram
    products too) matches the FP32 one."""
    g = ragged_grid(nx=24, ny=13, nz=11, seed=61)
    grid = F.Grid(g, "f32")
    dt0 = 0.99 * grid.cfl_dt()
    kw = dict(L=1, M=1.1, fmax=40e9, tol=1e-6, defl_tol=1e-5)
    bn = F.Basis(grid, 24, dt0, orth="native", **kw)
    bt = F.Basis(grid, 24, dt0, orth=orth, **kw)
    for which in (1, 2):
        Vn = bn.V(which).double()
        Vt = bt.V(which).double()
        assert Vt.shape == Vn.shape
        eye = torch.eye(Vt.shape[0], dtype=torch.float64, device="cuda")
        assert float((Vt @ Vt.T - eye).abs().max()) <= ortho_tol
        resid = Vn - (Vn @ Vt.T) @ Vt          # native columns outside span(Vt)
        assert float(resid.norm() / Vn.norm()) <= span_tol
    mn, mt = F.Model(grid, bn), F.Model(grid, bt)
    for name in ("De", "Dm", "K"):
        a, b = mn.get(name), mt.get(name)
        # same subspaces, possibly different bases: compare invariants
        sa, sb = np.linalg.svd(a, compute_uv=False), np.linalg.svd(b, compute_uv=False)
        assert np.max(np.abs(sa - sb)) <= 10 * span_tol * sa.max(), name


def test_full_size_bench_workload_properties():
    """The 64^3 graded cavity at full size in the bench's launch configuration
    (FP32, BiCGSTAB, M = 1.0077), with a small order: orthonormal basis,
    symmetric positive definite D~eps and D~mu, and after the perturbation at
    20x CFL a reduced step matrix with no eigenvalue outside the unit circle
    (Sec. III-A), checked in FP64 on the host from the projected matrices."""
    from oracle import mor
    wl = W.graded_cavity_workload()
    grid = F.Grid(wl.grid, "f32")
    dt0 = wl.s_ref * grid.cfl_dt()
    b = F.Basis(grid, 20, dt0, wl.L, wl.M, wl.fmax, tol=1e-4, defl_tol=1e-5, allow_noconv=True)
    for which in (1, 2):
        V = b.V(which).double()
        eye = torch.eye(V.shape[0], dtype=torch.float64, device="cuda")
        assert float((V @ V.T - eye).abs().max()) <= 1e-4
    m = F.Model(grid, b)
    De, Dm = m.get("De"), m.get("Dm")
    for D in (De, Dm):
        assert np.allclose(D, D.T, rtol=1e-6, atol=1e-9 * np.abs(D).max())
        assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0
    dt = wl.s_red[0] / wl.s_ref * dt0
    m.perturb(dt)
    red = mor.Reduced(De, m.get("Dse"), Dm, m.get("Dsm"), m.get("Kp"), m.get("BE"),
                      np.zeros((Dm.shape[0], m.get("BE").shape[1])), m.get("CE"))
    lam = np.abs(np.linalg.eigvals(mor.reduced_amplification(red, dt)))
    assert lam.max() <= 1.0 + 1e-6


@pytest.mark.parametrize("orth", ["tf32", "bf16"])
def test_tensor_core_gram_schmidt_many_blocks(orth):
    """The 100x50x24 microstrip with order 100 (seven blocks of 16 pool
    vectors, nearly dependent H parts): both halves of the tensor-core CGS2
    basis orthonormal to FP32 level, and D~eps, D~mu positive definite (the
    perturbation factorises them)."""
    wl = W.microstrip_workload(downscale=True)
    grid = F.Grid(wl.grid, "f32")
    dt0 = wl.s_ref * grid.cfl_dt()
    b = F.Basis(grid, 100, dt0, wl.L, wl.M, wl.fmax, tol=1e-5, defl_tol=1e-5, orth=orth, allow_noconv=True)
    for which in (1, 2):
        V = b.V(which).double()
        eye = torch.eye(V.shape[0], dtype=torch.float64, device="cuda")
        assert float((V @ V.T - eye).abs().max()) <= 1e-4, which
    m = F.Model(grid, b)
    m.perturb(dt0)
    for name in ("De", "Dm"):
        D = m.get(name)
        assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0, name
