"""FP64 oracle of the discrete adjoint of the full FDTD recursion.
Test infrastructure only.  (Not in the paper: the gradient pattern added
beside the method.)

Forward constraints g_n = (R+F) x^{n+1} - (R-F) x^n - B u^{n+1} = 0, n = 0..T-1,
x^0 = 0, probe y^n = C x^{n+1}, loss L(y).  With multipliers lambda_n:

    (R+F)^T lambda_n = C^T dL/dy^n + (R-F)^T lambda_{n+1},   lambda_T = 0,
    dL/dp = - sum_n lambda_n^T [d(R+F)/dp x^{n+1} - d(R-F)/dp x^n].

(R+F)^T is block upper triangular, so each backward step solves the H block
first and then the E block (a transposed Yee step).  For p = eps_r of a cell,
d(R+-F)/dp = d D_eps/dp / dt, with d D_eps,e / d eps_cell = eps0 A~_e L_e w_{e,cell}
and w the area weights of the edge average.
"""
from __future__ import annotations

import numpy as np

from .yee import EPS0, Stepper, YeeSystem


def probe_energy_loss(y: np.ndarray, dt: float):
    """L = sum_n (y^n)^2 dt over all probes, and dL/dy."""
    return float(np.sum(y * y) * dt), 2.0 * y * dt


def grad_eps_cells(sys: YeeSystem, dt: float, u: np.ndarray, dL_dy: np.ndarray) -> np.ndarray:
    """dL/d eps_r for every cell (nz*ny*nx,), by the adjoint recursion."""
    st = Stepper(sys, dt)
    _, _, states = st.run(u, record_states=True)
    T = len(u)
    Ne = sys.Ne
    K = sys.K.tocsr()
    KT = sys.K.T.tocsr()
    CE_T = sys.CE.T.tocsr()
    lam_e_next = np.zeros(Ne)
    lam_h_next = np.zeros(sys.Nh)
    g_edge = np.zeros(Ne)
    for n in range(T - 1, -1, -1):
        # rhs = C^T dL/dy^n + (R-F)^T lambda_{n+1}, with
        # R-F = [[be, -K], [0, bh]]  =>  (R-F)^T = [[be, 0], [-K^T, bh]].
        rhs_e = st.be * lam_e_next + CE_T @ dL_dy[n]
        rhs_h = st.bh * lam_h_next - KT @ lam_e_next
        # (R+F)^T = [[ae, -K], [0, ah]]: H block first, then E block.
        lam_h = rhs_h / st.ah
        lam_e = (rhs_e + K @ lam_h) / st.ae
        x1 = states[n + 1][:Ne]
        x0 = states[n][:Ne]
        g_edge += -lam_e * (x1 - x0) / dt
        lam_e_next, lam_h_next = lam_e, lam_h
    # d D_eps,e / d eps_edge = eps0 vol_e ; chain rule to cells.
    g_edge = g_edge * EPS0 * sys.vol_e
    return np.asarray(sys.cell_weights.T @ g_edge).ravel()


def loss_of_eps(grid_factory, eps_cells: np.ndarray, dt: float, u: np.ndarray):
    """Forward loss for a grid whose cells carry their own eps_r (used for
    central differences): grid_factory(eps_cells) returns a GridSpec."""
    from .yee import assemble
    g = grid_factory(eps_cells)
    sys = assemble(g)
    y, _, _ = Stepper(sys, dt).run(u)
    return probe_energy_loss(y, dt)[0]
