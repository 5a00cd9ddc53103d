"""Partitioning of the hot path over several GPUs, one process per GPU
(torch.distributed: NCCL on GPUs, gloo for host tensors).

z-slab decomposition of the full-order leap-frog (Eq. (MNAform) stepped as the
explicit Yee update of Sec. II-A).  Rank r of W owns the planes [k0, k1) of
slab_range(nz, W, r) and keeps one ghost plane on each side that has a
neighbour, so its local grid spans [k0 - lo, k1 + hi), with PEC walls at the
local ends.  One global step is one local step followed by an exchange of the
six field components of the boundary planes: rank r sends its first and last
owned planes to r - 1 and r + 1 and overwrites its ghost planes with theirs.
The local walls corrupt only ghost values within one step -- E on the low
ghost plane (tangential E forced to zero there), H on the high ghost plane
(it reads the zero E beyond the local wall) -- and the exchange replaces them
before any owned value reads them, so the owned planes follow the one-grid
run exactly:
  E(k) reads H(k), H(k - 1);  H(k) reads E(k), E(k + 1);
  owned E(k0) reads the low ghost H, refreshed by the last exchange;
  owned H(k1 - 1) reads the high ghost E of the current step, computed from
  ghost H(k1) (refreshed) and owned H(k1 - 1).
Sources with entries in a rank's local planes (owned or ghost) are applied
there, so ghost E carries them; probe entries are read on the owning rank
only, and the probe outputs are the sum over ranks (one all-reduce per run).

Row-partitioned Gram and projection sums (Sec. II-C, Eq. (R_and_Freduced)):
a rank holding the rows of its slab forms its part of G = A^T diag(w) B
(mor_gram or mor_project on the local rows) and allreduce_sum adds the parts;
cgs2_deflate_rows orthonormalises row-partitioned pools the same way, one
all-reduce per Gram-Schmidt pass and per norm, and cocg_rows solves a
row-partitioned shifted system with one all-reduce per inner product.

The local stepping is delegated to an object with step(u_rows) -> y_rows,
planes(k0, nk) and set_planes(k0, f) over (6, nk, ny, nx) arrays: GridSlab
runs it through the C ABI on this process's GPU.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Tuple

import numpy as np

from . import workloads as W


def slab_range(nz: int, world: int, rank: int) -> Tuple[int, int]:
    """Owned planes [k0, k1) of rank `rank`: nz split into `world` contiguous
    slabs whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if nz < world:
        raise ValueError(f"{nz} planes cannot be split over {world} ranks")
    base, extra = divmod(nz, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def row_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [r0, r1) of a row-partitioned n-row matrix on rank `rank`."""
    base, extra = divmod(n, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def _restrict(port: W.Port, k_lo: int, k_hi: int, shift: int) -> W.Port:
    """Entries of `port` on planes [k_lo, k_hi), moved down by `shift` planes;
    a port with none keeps one zero-weight entry so every rank has the same
    columns of B and rows of C."""
    sel = (port.k >= k_lo) & (port.k < k_hi)
    if not sel.any():
        return W.Port(port.comp, np.array([k_lo - shift], np.int64), np.array([port.j[0]], np.int64),
                      np.array([port.i[0]], np.int64), np.zeros(1))
    return W.Port(port.comp, port.k[sel] - shift, port.j[sel], port.i[sel], port.w[sel])


@dataclass
class Slab:
    """This rank's part of a z-slab decomposition."""
    spec: W.GridSpec   # local grid: planes [k0 - lo, k1 + hi) of the global one
    k0: int            # first owned global plane
    k1: int            # one past the last owned global plane
    lo: int            # ghost planes below (0 or 1)
    hi: int            # ghost planes above (0 or 1)


def local_slab(spec: W.GridSpec, world: int, rank: int) -> Slab:
    """The local grid of rank `rank`: owned planes plus one ghost plane towards
    each neighbour; sources restricted to the local planes, probes to the owned
    ones."""
    k0, k1 = slab_range(spec.nz, world, rank)
    lo = 1 if rank > 0 else 0
    hi = 1 if rank < world - 1 else 0
    a, b = k0 - lo, k1 + hi
    g = W.GridSpec(spec.nx, spec.ny, b - a, spec.dx, spec.dy, np.asarray(spec.dz)[a:b], spec.eps_r, spec.mu_r,
                   spec.sig_e, spec.sig_m, spec.pec, np.ascontiguousarray(spec.mat_id[a:b]))
    g.ports = [_restrict(p, a, b, a) for p in spec.ports]
    g.probes = [_restrict(p, k0, k1, a) for p in spec.probes]
    return Slab(g, k0, k1, lo, hi)


class SlabStepper:
    """Leap-frog of a grid split in z over the ranks of `group`.

    `make_local(slab_spec)` builds the local stepper.  run(u) steps len(u)
    steps with the global excitation u (nsteps, m) and returns the global
    probe outputs (nsteps, p) on every rank (torch tensors on the local
    stepper's device)."""

    def __init__(self, spec: W.GridSpec, make_local: Callable, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.slab = local_slab(spec, self.world, self.rank)
        self.local = make_local(self.slab.spec)
        self.nzl = self.slab.spec.nz

    def _peer(self, r: int) -> int:
        """Global rank of group rank r."""
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def exchange(self):
        """Owned boundary planes to the neighbours, their planes into the ghosts."""
        dist, s = self.dist, self.slab
        ops, recv = [], []
        if s.lo:
            ops.append(dist.P2POp(dist.isend, self.local.planes(s.lo, 1).contiguous(), self._peer(self.rank - 1),
                                  self.group))
            buf = self.local.planes(0, 1).clone()
            ops.append(dist.P2POp(dist.irecv, buf, self._peer(self.rank - 1), self.group))
            recv.append((0, buf))
        if s.hi:
            ops.append(dist.P2POp(dist.isend, self.local.planes(self.nzl - 1 - s.hi, 1).contiguous(),
                                  self._peer(self.rank + 1), self.group))
            buf = self.local.planes(self.nzl - 1, 1).clone()
            ops.append(dist.P2POp(dist.irecv, buf, self._peer(self.rank + 1), self.group))
            recv.append((self.nzl - 1, buf))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for k, buf in recv:
            self.local.set_planes(k, buf)

    def run(self, u):
        import torch
        ys: List = []
        for n in range(u.shape[0]):
            ys.append(self.local.step(u[n:n + 1]))
            self.exchange()
        y = torch.cat(ys, 0) if ys else u.new_zeros((0, len(self.slab.spec.probes)))
        return allreduce_sum(y, self.group)

    def owned_fields(self):
        """(6, k1 - k0, ny, nx) owned planes of the local fields."""
        s = self.slab
        return self.local.planes(s.lo, s.k1 - s.k0)


def allreduce_sum(t, group=None):
    """Sum of a tensor over the ranks of `group` (in place, returned): the
    partial Gram products A_r^T diag(w_r) B_r of row-partitioned operands, the
    partial projections V_r^T D_r V_r of Eq. (R_and_Freduced), or partial
    probe sums."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def cgs2_deflate_rows(pool_rows, defl_tol: float, gram: Callable = None, group=None):
    """CGS2 with deflation (Sec. II-C: the orthonormalisation of the SPRIM
    pools) over row-partitioned vectors.  This rank holds the same rows of
    every pool vector (pool_rows: list of 1-D tensors) and of the basis it
    builds.  Each of the two passes against the basis forms the rank's part of
    the coefficients V_r^T w_r and adds the parts over the ranks with one
    all-reduce, then updates w_r -= V_r h locally; each norm is a local sum of
    squares added by one all-reduce.  All ranks see the same reduced sums and
    so keep or drop the same vectors: a vector whose norm after the passes is
    below defl_tol times its norm before is dropped.  gram(V_r, w_r) returns
    V_r^T w_r (a matmul on the tensors' device by default; mor_gram for rows
    held on a GPU).  Returns the rank's rows of the basis (n_r x q tensor)."""
    import torch
    gram = gram or (lambda V, w: V.transpose(0, 1) @ w)

    def norm(w):
        return float(allreduce_sum((w * w).sum().reshape(1), group)[0]) ** 0.5

    cols = []
    for p in pool_rows:
        w = p.clone()
        n0 = norm(w)
        if n0 == 0:
            continue
        if cols:
            V = torch.stack(cols, dim=1)
            for _ in range(2):
                h = allreduce_sum(gram(V, w), group)
                w = w - V @ h
        n1 = norm(w)
        if n1 < defl_tol * n0:
            continue
        cols.append(w / n1)
    if not cols:
        return torch.zeros((pool_rows[0].shape[0], 0), dtype=pool_rows[0].dtype, device=pool_rows[0].device)
    return torch.stack(cols, dim=1)


def cocg_rows(apply_rows: Callable, b_rows, pinv_rows, tol: float, maxit: int, group=None):
    """Preconditioned COCG on a row-partitioned complex symmetric system
    (the shifted Schur-complement solves of Sec. IV-B): this rank holds rows
    of b, of the diagonal preconditioner pinv and of every iterate;
    apply_rows(p_rows) returns this rank's rows of S p (it exchanges what the
    operator needs from other ranks).  The unconjugated products (p, S p) and
    (r, P r) and the residual norm are local sums added by one all-reduce
    each; the vector updates are local.  Stops at ||r|| <= tol ||b|| or
    maxit.  Returns (x_rows, iterations, relative residual)."""
    import torch

    def reduce(*vals):
        t = torch.tensor([float(v) for v in vals], dtype=torch.float64)
        return allreduce_sum(t, group).tolist()

    def udot(a, b):  # sum a_i b_i, unconjugated
        v = (a * b).sum()
        return complex(*reduce(v.real, v.imag))

    x = torch.zeros_like(b_rows)
    r = b_rows.clone()
    bn = reduce((b_rows.abs() ** 2).sum())[0] ** 0.5
    if bn == 0:
        return x, 0, 0.0
    z = pinv_rows * r
    p = z.clone()
    rho = udot(r, z)
    rel = 1.0
    it = 0
    while it < maxit:
        q = apply_rows(p)
        alpha = rho / udot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        z = pinv_rows * r
        v = (r * z).sum()
        re, im, rn2 = reduce(v.real, v.imag, (r.abs() ** 2).sum())
        rel = rn2 ** 0.5 / bn
        if rel <= tol:
            break
        rho_new = complex(re, im)
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, it, rel


class GridSlab:
    """Local stepper of a slab on this process's GPU through the C ABI."""

    def __init__(self, spec: W.GridSpec, prec: str, dt: float):
        from . import fdtdmor as F
        self.grid = F.Grid(spec, prec)
        self.dt = dt
        self.first = True

    def step(self, u_rows):
        y = self.grid.step(self.dt, u_rows, reset=self.first)
        self.first = False
        return y

    def planes(self, k0: int, nk: int):
        return self.grid.planes(k0, nk)

    def set_planes(self, k0: int, f):
        self.grid.set_planes(k0, f)
