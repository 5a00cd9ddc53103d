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


def reduced_grad_De(red, dt: float, u: np.ndarray, dL_dy: np.ndarray) -> np.ndarray:
    """dL/dD~eps (q1 x q1) of a probe loss of the reduced leap-frog (the block
    form of Eq. (R_and_Freduced)) with the projection V and K~ held fixed, by
    the adjoint of that recursion:

        A_e e' = B_e e - K~ h + B~_E u,   A_h h' = B_h h + K~^T e' + B~_H u,
        A_e = D~e/dt + D~se/2, B_e = D~e/dt - D~se/2 (likewise A_h, B_h), y = C~ e'.

    Backwards, with adjoint carries (eb, hb) of (e^{n+1}, h^{n+1}):
    g_h = A_h^{-1} hb, ebar = eb + C~^T dL/dy^n + K~ g_h, g_e = A_e^{-1} ebar,
    dL/dD~e += g_e (e^n - e^{n+1})^T / dt, eb <- B_e g_e, hb <- B_h g_h - K~^T g_e."""
    import scipy.linalg as sl
    u = np.asarray(u, np.float64).reshape(len(u), -1)
    q1, q2 = red.q1, red.q2
    Ae = red.De / dt + 0.5 * red.Dse
    Be = red.De / dt - 0.5 * red.Dse
    Ah = red.Dm / dt + 0.5 * red.Dsm
    Bh = red.Dm / dt - 0.5 * red.Dsm
    ce, ch = sl.cho_factor(Ae), sl.cho_factor(Ah)
    T = len(u)
    es = np.zeros((T + 1, q1))
    e, h = np.zeros(q1), np.zeros(q2)
    for n in range(T):
        e = sl.cho_solve(ce, Be @ e - red.K @ h + red.BE @ u[n])
        h = sl.cho_solve(ch, Bh @ h + red.K.T @ e + red.BH @ u[n])
        es[n + 1] = e
    eb, hb = np.zeros(q1), np.zeros(q2)
    G = np.zeros((q1, q1))
    for n in range(T - 1, -1, -1):
        gh = sl.cho_solve(ch, hb)
        ebar = eb + red.CE.T @ dL_dy[n] + red.K @ gh
        ge = sl.cho_solve(ce, ebar)
        G += np.outer(ge, es[n] - es[n + 1]) / dt
        eb = Be @ ge
        hb = Bh @ gh - red.K.T @ ge
    return G


def reduced_grad_eps_cells(sys: YeeSystem, V1: np.ndarray, G: np.ndarray) -> np.ndarray:
    """dL/d eps_r per cell through D~eps = V1^T D_eps V1 with V1 frozen
    (V1: Ne x q1 in the oracle's unknown order): per E edge v_e^T G v_e times
    d D_eps,e / d eps_cell = eps0 vol_e w_{e,cell}."""
    ge = np.einsum("ea,ab,eb->e", V1, G, V1)
    return np.asarray(sys.cell_weights.T @ (ge * EPS0 * sys.vol_e)).ravel()
