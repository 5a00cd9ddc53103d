"""P-k: the oracle's discrete adjoint gradient against central finite
differences of the oracle forward run (FP64, no GPU)."""
import numpy as np

from oracle import adjoint, yee
from paper_1406_7042_gb300 import workloads as W


def _grid_with_cell_eps(eps_cells, base):
    """Every cell its own material so that eps_r can be perturbed per cell."""
    g = W.cavity_uniform(base[0], 1e-3, seed=21)
    nx = ny = nz = base[0]
    nc = nx * ny * nz
    g.eps_r = np.concatenate([[1.0, 1.0], eps_cells])
    g.mu_r = np.ones(nc + 2); g.sig_e = np.concatenate([[0.0, 0.0], np.full(nc, 0.05)])
    g.sig_m = np.zeros(nc + 2); g.pec = np.zeros(nc + 2, np.uint8); g.pec[1] = 1
    g.mat_id = (2 + np.arange(nc)).reshape(nz, ny, nx).astype(np.uint16)
    g.ports = [W.Port.point(W.COMP_EX, 1, 2, 2), W.Port.point(W.COMP_EZ, 2, 1, 3)]
    g.probes = [W.Port.point(W.COMP_EX, 3, 3, 3)]
    g.dz = np.array([1e-3, 0.7e-3, 0.7e-3, 1e-3, 1.3e-3])
    return g


def test_adjoint_matches_central_differences():
    n = 5
    rng = np.random.default_rng(5)
    eps = rng.uniform(1.0, 4.0, n ** 3)
    g = _grid_with_cell_eps(eps, (n,))
    dt = 0.9 * yee.cfl_dt(g)
    T = 120
    u = W.excitation(g, 60e9, 60e9, dt, T)
    s = yee.assemble(g)
    y, _, _ = yee.Stepper(s, dt).run(u)
    L, dLdy = adjoint.probe_energy_loss(y, dt)
    grad = adjoint.grad_eps_cells(s, dt, u, dLdy)
    cells = rng.choice(n ** 3, 8, replace=False)
    for c in cells:
        h = 1e-6 * eps[c]
        ep = eps.copy(); ep[c] += h
        em = eps.copy(); em[c] -= h
        Lp = adjoint.loss_of_eps(lambda e: _grid_with_cell_eps(e, (n,)), ep, dt, u)
        Lm = adjoint.loss_of_eps(lambda e: _grid_with_cell_eps(e, (n,)), em, dt, u)
        fd = (Lp - Lm) / (2 * h)
        assert abs(grad[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max())


def test_reduced_model_gradient_matches_central_differences():
    """Gradient of a probe loss of the reduced model with the projection V
    frozen (D~eps = V1^T D_eps V1 rebuilt from the perturbed grid, same V1)
    against central differences of that reduced run."""
    from oracle import mor
    n = 5
    rng = np.random.default_rng(8)
    eps = rng.uniform(1.0, 4.0, n ** 3)
    g = _grid_with_cell_eps(eps, (n,))
    s = yee.assemble(g)
    dt0 = 0.99 * yee.cfl_dt(g)
    basis = mor.sprim_basis(s, dt0, 12, 1, 1.1, 40e9)
    red = mor.project(s, basis.V1, basis.V2)
    T = 150
    u = W.excitation(g, 60e9, 60e9, dt0, T)
    y = mor.reduced_run(red, dt0, u)
    L, dLdy = adjoint.probe_energy_loss(y, dt0)
    G = adjoint.reduced_grad_De(red, dt0, u, dLdy)
    grad = adjoint.reduced_grad_eps_cells(s, basis.V1, G)

    def loss(e_cells):
        s2 = yee.assemble(_grid_with_cell_eps(e_cells, (n,)))
        red2 = mor.project(s2, basis.V1, basis.V2)
        return adjoint.probe_energy_loss(mor.reduced_run(red2, dt0, u), dt0)[0]

    for c in rng.choice(n ** 3, 6, replace=False):
        h = 1e-6 * eps[c]
        ep = eps.copy(); ep[c] += h
        em = eps.copy(); em[c] -= h
        fd = (loss(ep) - loss(em)) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-5 * np.abs(grad).max(), (c, fd, grad[c])
