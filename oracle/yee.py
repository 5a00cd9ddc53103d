"""FP64 oracle of the Yee FDTD system in matrix form (Sec. II-A, Eqs. (matrix),
(MNAform), (R_and_F), (CFL)).  Test infrastructure only.

Unknowns.  E is kept on every edge that is neither tangential to the PEC box
nor touching a PEC cell; those edges are removed (their field is zero).  H
is kept on every edge except the ones normal to a box wall (identically zero).
Unknowns are ordered component-major (Ex, Ey, Ez | Hx, Hy, Hz), each in
(k, j, i) C order over the storage positions of ``workloads``.

Non-uniform grid (the paper states the form holds, Sec. II-A, without
giving it; reading): with L_e the primal edge length, A~_e the area of the
dual face pierced by edge e, A_h the primal face pierced by H edge h and L~_h
its dual length,

    D_eps = diag(eps0 eps_e A~_e L_e),   D_sigma_e = diag(sigma_e A~_e L_e),
    D_mu  = diag(mu0 mu_h A_h L~_h),     D_sigma_m = diag(sigma_m,h A_h L~_h),
    K[e, h] = -c[e, h] L_e L~_h,

where c[e, h] = +-1 is the sign with which H edge h enters the circulation
around the dual face of e (the discrete curl of Ampere's law).  On a uniform
grid these are Delta^3 times the paper's D = eps and K = +-1/Delta.  eps_e and
sigma_e are the area-weighted means over the (up to) four cells sharing edge
e; mu_h and sigma_m,h the length-weighted means over the two cells the dual
edge crosses.  An E edge touching a PEC cell is PEC.

Sign.  The matrix form (E row: ... - K H, H row: - K^T E on the left) is the
authoritative one; it gives a skew-symmetric off-diagonal part of F and the
energy identity.  The printed one-dimensional H update has the opposite sign.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

C0 = 299792458.0
MU0 = 4.0e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)

E_COMPS = ("Ex", "Ey", "Ez")
H_COMPS = ("Hx", "Hy", "Hz")


def dual_spacing(d: np.ndarray) -> np.ndarray:
    """Dual (node-centred) spacing: (d[i-1] + d[i]) / 2, and d[0]/2 at i = 0."""
    out = np.empty_like(d)
    out[0] = d[0] / 2.0
    out[1:] = 0.5 * (d[:-1] + d[1:])
    return out


@dataclass
class YeeSystem:
    """Assembled sparse matrices of Eq. (matrix) for one grid."""
    grid: object
    shape: Tuple[int, int, int]          # (nz, ny, nx)
    e_mask: List[np.ndarray]             # live E unknowns per component (storage shape)
    h_mask: List[np.ndarray]
    e_index: List[np.ndarray]            # storage -> unknown index (or -1)
    h_index: List[np.ndarray]
    Ne: int
    Nh: int
    De: np.ndarray                       # diagonals
    Dse: np.ndarray
    Dm: np.ndarray
    Dsm: np.ndarray
    K: sp.csr_matrix                     # Ne x Nh
    BE: sp.csr_matrix                    # Ne x m
    CE: sp.csr_matrix                    # p x Ne
    eps_edge: np.ndarray                 # (Ne,) relative permittivity per E unknown
    vol_e: np.ndarray                    # (Ne,) A~_e L_e
    vol_h: np.ndarray                    # (Nh,) A_h L~_h
    cell_weights: sp.csr_matrix          # Ne x ncells: d eps_e / d eps_cell

    @property
    def N(self) -> int:
        return self.Ne + self.Nh

    @property
    def m(self) -> int:
        return self.BE.shape[1]

    @property
    def p(self) -> int:
        return self.CE.shape[0]

    # -- Eq. (R_and_F) ------------------------------------------------------
    def R(self, dt: float) -> sp.csr_matrix:
        return sp.bmat([[sp.diags(self.De / dt), -0.5 * self.K],
                        [-0.5 * self.K.T, sp.diags(self.Dm / dt)]], format="csr")

    def F(self) -> sp.csr_matrix:
        return sp.bmat([[sp.diags(0.5 * self.Dse), 0.5 * self.K],
                        [-0.5 * self.K.T, sp.diags(0.5 * self.Dsm)]], format="csr")

    def B(self) -> sp.csr_matrix:
        return sp.vstack([self.BE, sp.csr_matrix((self.Nh, self.m))], format="csr")

    def C(self) -> sp.csr_matrix:
        return sp.hstack([self.CE, sp.csr_matrix((self.p, self.Nh))], format="csr")

    # -- conversions between unknown vectors and storage arrays ------------
    def to_arrays(self, x: np.ndarray) -> Dict[str, np.ndarray]:
        out = {}
        off = 0
        for c in range(3):
            a = np.zeros(self.shape, x.dtype)
            n = int(self.e_mask[c].sum())
            a[self.e_mask[c]] = x[off:off + n]
            out[E_COMPS[c]] = a
            off += n
        for c in range(3):
            a = np.zeros(self.shape, x.dtype)
            n = int(self.h_mask[c].sum())
            a[self.h_mask[c]] = x[off:off + n]
            out[H_COMPS[c]] = a
            off += n
        return out

    def from_arrays(self, arrs: Dict[str, np.ndarray]) -> np.ndarray:
        parts = [np.asarray(arrs[E_COMPS[c]])[self.e_mask[c]] for c in range(3)]
        parts += [np.asarray(arrs[H_COMPS[c]])[self.h_mask[c]] for c in range(3)]
        return np.concatenate(parts).astype(np.float64)


def _cell_lookup(mat_id: np.ndarray, prop: np.ndarray) -> np.ndarray:
    return prop[mat_id.astype(np.int64)]


def assemble(grid) -> YeeSystem:
    """Build D_eps, D_mu, D_sigma_e, D_sigma_m, K, B and C (Sec. II-A)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    dx, dy, dz = (np.asarray(a, np.float64) for a in (grid.dx, grid.dy, grid.dz))
    xd, yd, zd = dual_spacing(dx), dual_spacing(dy), dual_spacing(dz)
    shape = (nz, ny, nx)
    K3, J3, I3 = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mat = grid.mat_id.astype(np.int64)
    pec_cell = np.asarray(grid.pec, bool)[mat]
    eps_c = _cell_lookup(mat, np.asarray(grid.eps_r, np.float64))
    sig_c = _cell_lookup(mat, np.asarray(grid.sig_e, np.float64))
    mu_c = _cell_lookup(mat, np.asarray(grid.mu_r, np.float64))
    sgm_c = _cell_lookup(mat, np.asarray(grid.sig_m, np.float64))
    cell_flat = np.arange(nx * ny * nz).reshape(shape)

    # ---- E edges: the four cells around each edge and their area weights.
    # Ex(i+1/2, j, k): cells (i, j-1|j, k-1|k); dual face ydual_j x zdual_k.
    # Ey(i, j+1/2, k): cells (i-1|i, j, k-1|k); dual face xdual_i x zdual_k.
    # Ez(i, j, k+1/2): cells (i-1|i, j-1|j, k); dual face xdual_i x ydual_j.
    def e_neighbours(c):
        out = []  # list of (kk, jj, ii, weight) arrays, weight = quarter area / dual area
        for a in (-1, 0):
            for b in (-1, 0):
                if c == 0:
                    kk, jj, ii = K3 + a, J3 + b, I3
                    w = (np.take(dy, np.clip(jj, 0, ny - 1)) / 2) * (np.take(dz, np.clip(kk, 0, nz - 1)) / 2) / (yd[J3] * zd[K3])
                elif c == 1:
                    kk, jj, ii = K3 + a, J3, I3 + b
                    w = (np.take(dx, np.clip(ii, 0, nx - 1)) / 2) * (np.take(dz, np.clip(kk, 0, nz - 1)) / 2) / (xd[I3] * zd[K3])
                else:
                    kk, jj, ii = K3, J3 + a, I3 + b
                    w = (np.take(dx, np.clip(ii, 0, nx - 1)) / 2) * (np.take(dy, np.clip(jj, 0, ny - 1)) / 2) / (xd[I3] * yd[J3])
                out.append((kk, jj, ii, w))
        return out

    e_wall = [(J3 == 0) | (K3 == 0), (I3 == 0) | (K3 == 0), (I3 == 0) | (J3 == 0)]
    e_mask, e_eps, e_sig, e_vol, e_cells = [], [], [], [], []
    for c in range(3):
        nb = e_neighbours(c)
        touches_pec = np.zeros(shape, bool)
        eps_e = np.zeros(shape)
        sig_e = np.zeros(shape)
        for (kk, jj, ii, w) in nb:
            valid = (kk >= 0) & (jj >= 0) & (ii >= 0)
            kc, jc, ic = np.clip(kk, 0, None), np.clip(jj, 0, None), np.clip(ii, 0, None)
            touches_pec |= valid & pec_cell[kc, jc, ic]
            eps_e += np.where(valid, w * eps_c[kc, jc, ic], 0.0)
            sig_e += np.where(valid, w * sig_c[kc, jc, ic], 0.0)
        live = ~e_wall[c] & ~touches_pec
        if c == 0:
            vol = dx[I3] * yd[J3] * zd[K3]
        elif c == 1:
            vol = dy[J3] * xd[I3] * zd[K3]
        else:
            vol = dz[K3] * xd[I3] * yd[J3]
        e_mask.append(live)
        e_eps.append(eps_e[live]); e_sig.append(sig_e[live]); e_vol.append(vol[live])
        rows = []
        for (kk, jj, ii, w) in nb:
            rows.append((cell_flat[np.clip(kk, 0, None), np.clip(jj, 0, None), np.clip(ii, 0, None)][live],
                         w[live]))
        e_cells.append(rows)

    # ---- H edges: two cells along the dual edge, length weights.
    h_wall = [I3 == 0, J3 == 0, K3 == 0]
    h_mask, h_mu, h_sgm, h_vol = [], [], [], []
    for c in range(3):
        live = ~h_wall[c]
        mu_h = np.zeros(shape); sg_h = np.zeros(shape)
        for a in (-1, 0):
            if c == 0:
                kk, jj, ii = K3, J3, I3 + a
                w = np.take(dx, np.clip(ii, 0, nx - 1)) / 2 / xd[I3]
            elif c == 1:
                kk, jj, ii = K3, J3 + a, I3
                w = np.take(dy, np.clip(jj, 0, ny - 1)) / 2 / yd[J3]
            else:
                kk, jj, ii = K3 + a, J3, I3
                w = np.take(dz, np.clip(kk, 0, nz - 1)) / 2 / zd[K3]
            valid = (kk >= 0) & (jj >= 0) & (ii >= 0)
            kc, jc, ic = np.clip(kk, 0, None), np.clip(jj, 0, None), np.clip(ii, 0, None)
            mu_h += np.where(valid, w * mu_c[kc, jc, ic], 0.0)
            sg_h += np.where(valid, w * sgm_c[kc, jc, ic], 0.0)
        if c == 0:
            vol = dy[J3] * dz[K3] * xd[I3]
        elif c == 1:
            vol = dx[I3] * dz[K3] * yd[J3]
        else:
            vol = dx[I3] * dy[J3] * zd[K3]
        h_mask.append(live)
        h_mu.append(mu_h[live]); h_sgm.append(sg_h[live]); h_vol.append(vol[live])

    def index_maps(masks):
        idx, off = [], 0
        for mk in masks:
            a = -np.ones(shape, np.int64)
            n = int(mk.sum())
            a[mk] = off + np.arange(n)
            idx.append(a)
            off += n
        return idx, off

    e_index, Ne = index_maps(e_mask)
    h_index, Nh = index_maps(h_mask)

    # ---- K: K[e, h] = -c[e, h] L_e Ldual_h (circulation sign c of Ampere's law).
    # (dE, dH component offsets, sign c, primal length of e, dual length of h)
    rows, cols, vals = [], [], []

    def add(ecomp, hcomp, dk, dj, di, sign, Le, Lh):
        live = e_mask[ecomp]
        kk, jj, ii = K3 + dk, J3 + dj, I3 + di
        inside = (kk >= 0) & (jj >= 0) & (ii >= 0) & (kk < nz) & (jj < ny) & (ii < nx)
        sel = live & inside
        hi = h_index[hcomp][kk[sel], jj[sel], ii[sel]]
        ok = hi >= 0
        rows.append(e_index[ecomp][sel][ok])
        cols.append(hi[ok])
        vals.append((-sign * Le[sel] * Lh[sel])[ok])

    # (curl H)_x = dHz/dy - dHy/dz at Ex[k,j,i]
    add(0, 2, 0, 0, 0, +1, dx[I3], zd[K3]); add(0, 2, 0, -1, 0, -1, dx[I3], zd[K3])
    add(0, 1, 0, 0, 0, -1, dx[I3], yd[J3]); add(0, 1, -1, 0, 0, +1, dx[I3], yd[J3])
    # (curl H)_y = dHx/dz - dHz/dx at Ey[k,j,i]
    add(1, 0, 0, 0, 0, +1, dy[J3], xd[I3]); add(1, 0, -1, 0, 0, -1, dy[J3], xd[I3])
    add(1, 2, 0, 0, 0, -1, dy[J3], zd[K3]); add(1, 2, 0, 0, -1, +1, dy[J3], zd[K3])
    # (curl H)_z = dHy/dx - dHx/dy at Ez[k,j,i]
    add(2, 1, 0, 0, 0, +1, dz[K3], yd[J3]); add(2, 1, 0, 0, -1, -1, dz[K3], yd[J3])
    add(2, 0, 0, 0, 0, -1, dz[K3], xd[I3]); add(2, 0, 0, -1, 0, +1, dz[K3], xd[I3])
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(Ne, Nh))

    eps_edge = np.concatenate(e_eps)
    vol_e = np.concatenate(e_vol)
    vol_h = np.concatenate(h_vol)
    De = EPS0 * eps_edge * vol_e
    Dse = np.concatenate(e_sig) * vol_e
    Dm = MU0 * np.concatenate(h_mu) * vol_h
    Dsm = np.concatenate(h_sgm) * vol_h

    # d eps_e / d eps_cell (area weights), used by the adjoint.
    wr, wc, wv = [], [], []
    off = 0
    for c in range(3):
        n = int(e_mask[c].sum())
        for (cells, w) in e_cells[c]:
            wr.append(off + np.arange(n)); wc.append(cells); wv.append(w)
        off += n
    cell_weights = sp.csr_matrix((np.concatenate(wv), (np.concatenate(wr), np.concatenate(wc))),
                                 shape=(Ne, nx * ny * nz))

    def port_matrix(ports, scale_by_volume):
        r, cidx, v = [], [], []
        for pi, p in enumerate(ports):
            ei = e_index[p.comp][p.k, p.j, p.i]
            ok = ei >= 0
            w = np.asarray(p.w, np.float64)[ok]
            if scale_by_volume:
                w = -w * vol_e[ei[ok]]
            r.append(ei[ok]); cidx.append(np.full(int(ok.sum()), pi)); v.append(w)
        if not ports:
            return None
        return (np.concatenate(r), np.concatenate(cidx), np.concatenate(v))

    bp = port_matrix(grid.ports, True)
    BE = (sp.csr_matrix((bp[2], (bp[0], bp[1])), shape=(Ne, len(grid.ports)))
          if bp else sp.csr_matrix((Ne, 0)))
    cp = port_matrix(grid.probes, False)
    CE = (sp.csr_matrix((cp[2], (cp[1], cp[0])), shape=(len(grid.probes), Ne))
          if cp else sp.csr_matrix((0, Ne)))

    return YeeSystem(grid, shape, e_mask, h_mask, e_index, h_index, Ne, Nh, De, Dse, Dm, Dsm,
                     K, BE, CE, eps_edge, vol_e, vol_h, cell_weights)


# ------------------------------------------------------------------ Eq. (CFL)
def cfl_dt(grid) -> float:
    """Eq. (CFL) with the fastest wave speed c0 / sqrt(min eps_r mu_r) and the
    smallest cell on each axis (conservative reading for graded grids).  A
    single layer of cells between the z plates (nz = 1) is the 2-D TM problem
    of Sec. V-A/V-B: no update differences along z, so Eq. (CFL) has only the
    x and y terms."""
    er = np.asarray(grid.eps_r, np.float64)
    mr = np.asarray(grid.mu_r, np.float64)
    used = np.unique(grid.mat_id)
    nonpec = [int(u) for u in used if not grid.pec[int(u)]]
    emin = min(er[u] * mr[u] for u in nonpec) if nonpec else 1.0
    c = C0 / math.sqrt(emin)
    dxm, dym, dzm = float(np.min(grid.dx)), float(np.min(grid.dy)), float(np.min(grid.dz))
    zterm = 0.0 if grid.nz == 1 else 1.0 / dzm ** 2
    return 1.0 / (c * math.sqrt(1.0 / dxm ** 2 + 1.0 / dym ** 2 + zterm))


def exact_dt_limit(sys: YeeSystem) -> float:
    """Largest dt with R > 0 (Eq. (Dstability2)): R > 0 iff the singular values
    of D_eps^{-1/2} K D_mu^{-1/2} are below 2/dt (Schur complement)."""
    import scipy.sparse.linalg as sla
    Se = sp.diags(1.0 / np.sqrt(sys.De))
    Sm = sp.diags(1.0 / np.sqrt(sys.Dm))
    A = (Se @ sys.K @ Sm).tocsr()
    if min(A.shape) <= 64:
        smax = float(np.linalg.svd(A.toarray(), compute_uv=False)[0])
    else:
        smax = float(sla.svds(A, k=1, return_singular_vectors=False, tol=1e-12)[0])
    return 2.0 / smax


# ------------------------------------------------------------------ stepping
class Stepper:
    """Leap-frog of Eq. (MNAform) by block substitution: R + F is block lower
    triangular with diagonal blocks D_eps/dt + D_se/2 and D_mu/dt + D_sm/2."""

    def __init__(self, sys: YeeSystem, dt: float):
        self.sys = sys
        self.dt = dt
        self.ae = sys.De / dt + 0.5 * sys.Dse   # diagonal of the (1,1) block of R+F
        self.be = sys.De / dt - 0.5 * sys.Dse   # diagonal of the (1,1) block of R-F
        self.ah = sys.Dm / dt + 0.5 * sys.Dsm
        self.bh = sys.Dm / dt - 0.5 * sys.Dsm
        self.K = sys.K.tocsr()
        self.KT = sys.K.T.tocsr()
        self.BE = sys.BE.tocsr()
        self.CE = sys.CE.tocsr()

    def step(self, e: np.ndarray, h: np.ndarray, u_np1: np.ndarray):
        """One step: (E^n, H^{n+1/2}) -> (E^{n+1}, H^{n+3/2})."""
        rhs_e = self.be * e - self.K @ h
        if self.BE.shape[1]:
            rhs_e = rhs_e + self.BE @ u_np1
        e1 = rhs_e / self.ae
        h1 = (self.bh * h + self.KT @ e1) / self.ah
        return e1, h1

    def run(self, u: np.ndarray, x0: np.ndarray = None, record_states: bool = False):
        """Run len(u) steps from x0 (zero by default).  Row n of the returned
        probe matrix is C x^{n+1}; with record_states the list of all states
        x^0 .. x^T is returned too."""
        sys = self.sys
        u = np.asarray(u, np.float64).reshape(len(u), -1)
        if x0 is None:
            e = np.zeros(sys.Ne); h = np.zeros(sys.Nh)
        else:
            e = np.array(x0[:sys.Ne], np.float64); h = np.array(x0[sys.Ne:], np.float64)
        y = np.zeros((len(u), sys.p))
        states = [np.concatenate([e, h])] if record_states else None
        for n in range(len(u)):
            e, h = self.step(e, h, u[n])
            if sys.p:
                y[n] = self.CE @ e
            if record_states:
                states.append(np.concatenate([e, h]))
        return y, np.concatenate([e, h]), states


def step_matrix_form(sys: YeeSystem, dt: float, x: np.ndarray, u_np1: np.ndarray) -> np.ndarray:
    """Literal Eq. (MNAform): solve (R + F) x^{n+1} = (R - F) x^n + B u^{n+1}
    with a general sparse solver (no use of the block structure)."""
    import scipy.sparse.linalg as sla
    R, F = sys.R(dt), sys.F()
    rhs = (R - F) @ x
    if sys.m:
        rhs = rhs + sys.B() @ np.asarray(u_np1, np.float64)
    return sla.spsolve((R + F).tocsc(), rhs)


def energy(sys: YeeSystem, dt: float, x: np.ndarray) -> float:
    """Discrete energy W = x^T R x; conserved when F is skew (lossless) and
    there is no source, since (x'+x)^T R (x'-x) = -(x'+x)^T F (x'+x)."""
    return float(x @ (sys.R(dt) @ x))


def amplification_matrix(sys: YeeSystem, dt: float) -> np.ndarray:
    """Dense Phi = (R+F)^{-1}(R-F) for tiny grids (eigenvalue pins)."""
    R, F = sys.R(dt).toarray(), sys.F().toarray()
    return np.linalg.solve(R + F, R - F)
