"""FP64 oracle of the structure-preserving reduction (Secs. II-C, II-D, III-A,
IV-A, IV-B).  Test infrastructure only.

Readings of points the paper leaves open (each restated in the design notes):

* Shifted system.  The printed system (R - F) + z (R + F) does not match the
  transfer function of Eq. (MNAform), H(z) = C [z(R+F) - (R-F)]^{-1} z B, nor
  the remark that z = 1 means static conditions.  We use
  A(z) = z (R + F) - (R - F); its blocks are A11 = (z-1) D_eps/dt +
  (z+1) D_se/2, A12 = K, A21 = -z K^T, A22 = (z-1) D_mu/dt + (z+1) D_sm/2.
* Krylov chain at z_l: v_0 = A_l^{-1} B, v_j = A_l^{-1} (R+F) v_{j-1}
  (moments of A(z)^{-1} about z_l), orthonormalised within the chain (block
  Arnoldi, "robust Arnoldi" of Sec. II-C).
* Real basis from complex points: the chain at conj(z) is the conjugate of
  the chain at z, so only l = 0..L are built and Re, Im of every complex
  vector enter the pool.
* Column budget: k = q / ((2L+1) m) block moments per point (l = 0 gives k m
  real vectors, a conjugate pair gives 2 k m).
* SPRIM split: the E parts of all real vectors form pool 1, the H parts pool
  2; each pool is orthonormalised by classical Gram-Schmidt with a second
  pass (CGS2) in the Euclidean inner product, in pool order, dropping a vector
  whose norm after both passes is below defl_tol times its norm before.
* The basis is built once at dt0 and reused for every dt.
* x^n ~ V x~^n and u^{n+1} in the reduced recursion (the printed indices in
  Eqs. (projection) and (reducedMNAform1) are read this way).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from .yee import YeeSystem


# ------------------------------------------------------------ Eq. (distrib)
def expansion_points(M: float, L: int, fmax: float, dt0: float,
                     include_center: bool = True) -> List[complex]:
    """z_l = M exp(j 2 pi (l/L) fmax dt0) for l = 0..L (l < 0 are conjugates).

    With include_center False only l = L is returned: the pair
    z = M exp(+-j 2 pi fmax dt) of Sec. V-C."""
    if not include_center:
        return [M * np.exp(1j * 2 * math.pi * fmax * dt0)]
    pts = []
    for l in range(0, L + 1):
        ang = 2 * math.pi * (l / L if L else 0.0) * fmax * dt0
        pts.append(complex(M * math.cos(ang), M * math.sin(ang)) if l else complex(M, 0.0))
    return pts


def shifted_matrix(sys: YeeSystem, dt: float, z: complex) -> sp.csc_matrix:
    """A(z) = z (R + F) - (R - F)."""
    R, F = sys.R(dt), sys.F()
    return (z * (R + F) - (R - F)).tocsc().astype(np.complex128)


def schur_blocks(sys: YeeSystem, dt: float, z: complex):
    """Diagonals of A11 and A22 of Eq. (linear_system_solution) (reading above)."""
    a11 = (z - 1) * sys.De / dt + (z + 1) * sys.Dse / 2
    a22 = (z - 1) * sys.Dm / dt + (z + 1) * sys.Dsm / 2
    return a11, a22


def schur_solve(sys: YeeSystem, dt: float, z: complex, b1: np.ndarray, b2: np.ndarray):
    """Solve A(z) x = b by Eqs. (reduced_linear_system_solution1/2):
    (A11 - A12 A22^{-1} A21) x1 = b1 - A12 A22^{-1} b2, x2 = A22^{-1}(b2 - A21 x1),
    with the Schur complement factorised by sparse LU."""
    a11, a22 = schur_blocks(sys, dt, z)
    K = sys.K.astype(np.complex128)
    A12 = K
    A21 = -z * K.T
    A22inv = sp.diags(1.0 / a22)
    S = (sp.diags(a11) - A12 @ A22inv @ A21).tocsc()
    x1 = sla.spsolve(S, b1 - A12 @ (b2 / a22))
    x2 = (b2 - A21 @ x1) / a22
    return x1, x2


def _orth_against(Q: List[np.ndarray], w: np.ndarray, passes: int = 2) -> np.ndarray:
    """Classical Gram-Schmidt of w against the orthonormal list Q, twice."""
    if not Q:
        return w
    Qm = np.stack(Q, axis=1)
    for _ in range(passes):
        w = w - Qm @ (Qm.conj().T @ w)
    return w


def krylov_chain(sys: YeeSystem, dt0: float, z: complex, k: int,
                 lu=None) -> List[np.ndarray]:
    """Block Arnoldi chain of k block moments at z: columns of A^{-1} B, then
    A^{-1} (R+F) applied to the previous orthonormal block, each new column
    orthogonalised (CGS2) against the whole chain and normalised."""
    A = shifted_matrix(sys, dt0, z)
    if lu is None:
        lu = sla.splu(A)
    RpF = (sys.R(dt0) + sys.F()).astype(np.complex128)
    B = sys.B().toarray().astype(np.complex128)
    Q: List[np.ndarray] = []
    block = [lu.solve(B[:, c]) for c in range(B.shape[1])]
    for j in range(k):
        new = []
        for w in block:
            w = _orth_against(Q, w)
            nrm = np.linalg.norm(w)
            if nrm == 0:
                continue
            q = w / nrm
            Q.append(q)
            new.append(q)
        if j + 1 < k:
            block = [lu.solve(RpF @ q) for q in new]
    return Q


def cgs2_deflate(pool: List[np.ndarray], defl_tol: float) -> np.ndarray:
    """Orthonormalise pool vectors in order (CGS2), dropping a vector whose
    norm after two passes is below defl_tol times its norm before."""
    V: List[np.ndarray] = []
    for p in pool:
        n0 = np.linalg.norm(p)
        if n0 == 0:
            continue
        w = _orth_against(V, p.astype(np.float64))
        n1 = np.linalg.norm(w)
        if n1 < defl_tol * n0:
            continue
        V.append(w / n1)
    return np.stack(V, axis=1) if V else np.zeros((pool[0].size, 0))


@dataclass
class Basis:
    V1: np.ndarray
    V2: np.ndarray
    points: List[complex]
    k: int
    pool_e: List[np.ndarray] = field(default_factory=list)
    pool_h: List[np.ndarray] = field(default_factory=list)


def sprim_basis(sys: YeeSystem, dt0: float, q: int, L: int, M: float, fmax: float,
                include_center: bool = True, defl_tol: float = 1e-8,
                keep_pool: bool = False) -> Basis:
    """SPRIM projection matrices V1 (Ne x q1), V2 (Nh x q2) (Eq. (V))."""
    pts = expansion_points(M, L, fmax, dt0, include_center)
    m = sys.m
    nreal = (1 if include_center else 0) + 2 * (len(pts) - (1 if include_center else 0))
    k = max(1, q // (nreal * m))
    pool_e, pool_h = [], []
    for z in pts:
        chain = krylov_chain(sys, dt0, z, k)
        for v in chain:
            parts = [v.real] if (abs(z.imag) == 0.0) else [v.real, v.imag]
            for r in parts:
                pool_e.append(r[:sys.Ne].copy())
                pool_h.append(r[sys.Ne:].copy())
    V1 = cgs2_deflate(pool_e, defl_tol)
    V2 = cgs2_deflate(pool_h, defl_tol)
    return Basis(V1, V2, pts, k, pool_e if keep_pool else [], pool_h if keep_pool else [])


# ------------------------------------------------------ Eq. (R_and_Freduced)
@dataclass
class Reduced:
    De: np.ndarray     # V1^T D_eps V1
    Dse: np.ndarray    # V1^T D_sigma_e V1
    Dm: np.ndarray     # V2^T D_mu V2
    Dsm: np.ndarray    # V2^T D_sigma_m V2
    K: np.ndarray      # V1^T K V2
    BE: np.ndarray     # V1^T B_E   (q1 x m)
    BH: np.ndarray     # V2^T B_H   (q2 x m), zero for electric sources
    CE: np.ndarray     # C_E V1     (p x q1)

    @property
    def q1(self) -> int:
        return self.De.shape[0]

    @property
    def q2(self) -> int:
        return self.Dm.shape[0]

    def R(self, dt: float) -> np.ndarray:
        return np.block([[self.De / dt, -0.5 * self.K], [-0.5 * self.K.T, self.Dm / dt]])

    def F(self) -> np.ndarray:
        return np.block([[0.5 * self.Dse, 0.5 * self.K], [-0.5 * self.K.T, 0.5 * self.Dsm]])

    def B(self) -> np.ndarray:
        return np.vstack([self.BE, self.BH])

    def C(self) -> np.ndarray:
        return np.hstack([self.CE, np.zeros((self.CE.shape[0], self.q2))])

    def with_K(self, Knew: np.ndarray) -> "Reduced":
        return Reduced(self.De, self.Dse, self.Dm, self.Dsm, Knew, self.BE, self.BH, self.CE)


def project(sys: YeeSystem, V1: np.ndarray, V2: np.ndarray) -> Reduced:
    """D~ = V_i^T D V_i, K~ = V1^T K V2, B~ = V^T B, C~ = C V."""
    De = V1.T @ (sys.De[:, None] * V1)
    Dse = V1.T @ (sys.Dse[:, None] * V1)
    Dm = V2.T @ (sys.Dm[:, None] * V2)
    Dsm = V2.T @ (sys.Dsm[:, None] * V2)
    K = V1.T @ (sys.K @ V2)
    BE = V1.T @ sys.BE.toarray()
    BH = np.zeros((V2.shape[1], sys.m))
    CE = sys.CE.toarray() @ V1
    return Reduced(De, Dse, Dm, Dsm, K, BE, BH, CE)


# --------------------------------------------------------------- Sec. III-A
def _sym_sqrt(A: np.ndarray) -> np.ndarray:
    w, Q = np.linalg.eigh(0.5 * (A + A.T))
    return (Q * np.sqrt(w)) @ Q.T


def singular_values(red: Reduced) -> np.ndarray:
    """sigma_i of D~eps^{-1/2} K~ D~mu^{-1/2} (Eq. (singular_limit))."""
    Se, Sm = _sym_sqrt(red.De), _sym_sqrt(red.Dm)
    M = np.linalg.solve(Se, red.K) @ np.linalg.inv(Sm)
    return np.linalg.svd(M, compute_uv=False)


def perturb(red: Reduced, dt: float, gamma: float = 0.9999):
    """Steps 1-3 of Sec. III-A: SVD of D~eps^{-1/2} K~ D~mu^{-1/2} = U S W^T,
    sigma'_i = sigma_i if sigma_i < gamma 2/dt else gamma 2/dt,
    K~' = D~eps^{1/2} U S' W^T D~mu^{1/2}.  Returns (reduced model with K~',
    number of clipped singular values, sigma before clipping)."""
    Se, Sm = _sym_sqrt(red.De), _sym_sqrt(red.Dm)
    M = np.linalg.solve(Se, red.K) @ np.linalg.inv(Sm)
    U, s, Wt = np.linalg.svd(M, full_matrices=False)
    lim = gamma * 2.0 / dt
    s_new = np.where(s < lim, s, lim)
    n_clip = int(np.sum(~(s < lim)))
    Knew = Se @ (U * s_new) @ Wt @ Sm
    return red.with_K(Knew), n_clip, s


def perturb_full(sys: YeeSystem, dt: float, gamma: float = 0.9999) -> np.ndarray:
    """The same procedure applied to the full system (the demonstration of
    Sec. III-B, tiny grids only): returns the perturbed dense K."""
    red = Reduced(np.diag(sys.De), np.diag(sys.Dse), np.diag(sys.Dm), np.diag(sys.Dsm),
                  sys.K.toarray(), sys.BE.toarray(), np.zeros((sys.Nh, sys.m)),
                  sys.CE.toarray())
    pr, n, s = perturb(red, dt, gamma)
    return pr.K, n, s


# ------------------------------------------------------ Eq. (reducedMNAform)
def reduced_amplification(red: Reduced, dt: float) -> np.ndarray:
    R, F = red.R(dt), red.F()
    return np.linalg.solve(R + F, R - F)


def reduced_run(red: Reduced, dt: float, u: np.ndarray, x0: Optional[np.ndarray] = None,
                return_state: bool = False):
    """Leap-frog of the reduced model in the block form of Eq. (R_and_Freduced):
    (D~e/dt + D~se/2) e' = (D~e/dt - D~se/2) e - K~ h + B~_E u,
    (D~m/dt + D~sm/2) h' = (D~m/dt - D~sm/2) h + K~^T e' + B~_H u,  y = C~ x'."""
    u = np.asarray(u, np.float64).reshape(len(u), -1)
    Ae = red.De / dt + 0.5 * red.Dse
    Be = red.De / dt - 0.5 * red.Dse
    Ah = red.Dm / dt + 0.5 * red.Dsm
    Bh = red.Dm / dt - 0.5 * red.Dsm
    import scipy.linalg as sl
    ce = sl.cho_factor(Ae)
    ch = sl.cho_factor(Ah)
    e = np.zeros(red.q1) if x0 is None else np.array(x0[:red.q1])
    h = np.zeros(red.q2) if x0 is None else np.array(x0[red.q1:])
    y = np.zeros((len(u), red.CE.shape[0]))
    for n in range(len(u)):
        e = sl.cho_solve(ce, Be @ e - red.K @ h + red.BE @ u[n])
        h = sl.cho_solve(ch, Bh @ h + red.K.T @ e + red.BH @ u[n])
        y[n] = red.CE @ e
    if return_state:
        return y, np.concatenate([e, h])
    return y


# ------------------------------------------------ transfer functions/moments
def transfer_full(sys: YeeSystem, dt: float, z: complex) -> np.ndarray:
    """H(z) = C [z(R+F) - (R-F)]^{-1} z B (p x m)."""
    A = shifted_matrix(sys, dt, z)
    X = sla.spsolve(A, sys.B().toarray().astype(np.complex128) * z)
    X = X.reshape(sys.N, -1)
    return sys.C() @ X


def transfer_reduced(red: Reduced, dt: float, z: complex) -> np.ndarray:
    R, F = red.R(dt), red.F()
    X = np.linalg.solve(z * (R + F) - (R - F), red.B() * z)
    return red.C() @ X


def moments_full(sys: YeeSystem, dt: float, z: complex, count: int) -> List[np.ndarray]:
    """C (A^{-1}(R+F))^j A^{-1} B, j = 0..count-1, about z."""
    A = shifted_matrix(sys, dt, z)
    lu = sla.splu(A)
    RpF = (sys.R(dt) + sys.F()).astype(np.complex128)
    X = np.column_stack([lu.solve(c) for c in sys.B().toarray().astype(np.complex128).T])
    C = sys.C()
    out = []
    for _ in range(count):
        out.append(C @ X)
        X = np.column_stack([lu.solve(RpF @ X[:, c]) for c in range(X.shape[1])])
    return out


def moments_reduced(red: Reduced, dt: float, z: complex, count: int) -> List[np.ndarray]:
    R, F = red.R(dt), red.F()
    A = z * (R + F) - (R - F)
    X = np.linalg.solve(A, red.B().astype(np.complex128))
    out = []
    for _ in range(count):
        out.append(red.C() @ X)
        X = np.linalg.solve(A, (R + F) @ X)
    return out


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """Relative L2 error ||a - b|| / ||b|| over the common samples."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))
