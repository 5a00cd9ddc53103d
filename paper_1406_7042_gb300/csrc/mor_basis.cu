// A3-A5: Krylov basis of the SPRIM reduction (Sec. II-C) with complex frequency
// hopping (Sec. IV-A, Eq. (distrib)) and the shifted solves of Sec. IV-B.
//
// All operators act on the per-volume form of Eq. (matrix) (each E row divided
// by its edge volume, each H row by its dual volume), in which -K/V_e is the
// discrete curl of Ampere's law and -K^T/V_h the curl of Faraday's law:
//   (R+F) v:  r1 = (eps/dt + sig/2) v1,  r2 = curlE(v1) + (mu/dt + sgm/2) v2
//   A(z) = z(R+F) - (R-F):  a11 = (z-1) eps/dt + (z+1) sig/2,
//                           a22 = (z-1) mu/dt + (z+1) sgm/2,
//   Schur complement  S x1 = a11 x1 + z curlH(curlE(x1)/a22),
//   right-hand side   b^  = r1 + curlH(r2/a22),    x2 = (r2 - z curlE(x1))/a22.
// Row scaling leaves the Krylov subspaces of A^{-1}(R+F) unchanged.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <complex>
#include <cstdlib>
#include <string>
#include <vector>

#include "grid_internal.cuh"
#include "mor_common.cuh"
#include "mor_internal.cuh"

namespace fdtdmor {

constexpr int MB = 256;  // threads per block of the elementwise / stencil kernels

// ------------------------------------------------------------------ edge props
template <typename T, typename ID>
__global__ void edge_props_kernel(Geo<T> g, const ID *__restrict__ mat, const T *__restrict__ mtab,
                                  int nmat, T *__restrict__ out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nc) return;
  const int nx = g.nx, ny = g.ny;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / ((int64_t)nx * ny));
  const T *eps = mtab, *sig = mtab + nmat, *mu = mtab + 2 * nmat, *sgm = mtab + 3 * nmat, *pec = mtab + 4 * nmat;
  const int nt = g.ntot();
  auto W = [&](int axis, int idx, bool hi) { return __ldg(g.ax + (hi ? AX_WHI : AX_WLO) * nt + g.off(axis) + idx); };
  auto M = [&](int ii, int jj, int kk) { return (int)mat[g.id(ii, jj, kk)]; };
  const int64_t nc = g.nc;
  // E edges: area-weighted mean over the four cells around the edge
  for (int c = 0; c < 3; ++c) {
    int a0, a1, i0, i1;  // transverse axes and indices
    bool wall;
    if (c == 0) { a0 = 1; a1 = 2; i0 = j; i1 = k; wall = (j == 0 || k == 0); }
    else if (c == 1) { a0 = 0; a1 = 2; i0 = i; i1 = k; wall = (i == 0 || k == 0); }
    else { a0 = 0; a1 = 1; i0 = i; i1 = j; wall = (i == 0 || j == 0); }
    T e = 0, s = 0;
    if (!wall) {
      bool anypec = false;
      for (int b1 = 0; b1 < 2; ++b1)
        for (int b0 = 0; b0 < 2; ++b0) {
          int ii = i, jj = j, kk = k;
          int d0 = b0 - 1, d1 = b1 - 1;
          if (a0 == 0) ii += d0; else jj += d0;
          if (a1 == 1) jj += d1; else kk += d1;
          const int m = M(ii, jj, kk);
          const T w = W(a0, i0, b0) * W(a1, i1, b1);
          anypec |= __ldg(pec + m) != T(0);
          e += w * __ldg(eps + m);
          s += w * __ldg(sig + m);
        }
      if (anypec) { e = 0; s = 0; }
    }
    out[EP_EPS * 3 * nc + c * nc + n] = e;
    out[EP_SIG * 3 * nc + c * nc + n] = s;
  }
  // H edges: length-weighted mean over the two cells the dual edge crosses
  for (int c = 0; c < 3; ++c) {
    const int idx = c == 0 ? i : (c == 1 ? j : k);
    T m_ = 0, s = 0;
    if (idx > 0) {
      const int m0 = c == 0 ? M(i - 1, j, k) : (c == 1 ? M(i, j - 1, k) : M(i, j, k - 1));
      const int m1 = M(i, j, k);
      const T w0 = W(c, idx, false), w1 = W(c, idx, true);
      m_ = w0 * __ldg(mu + m0) + w1 * __ldg(mu + m1);
      s = w0 * __ldg(sgm + m0) + w1 * __ldg(sgm + m1);
    }
    out[EP_MU * 3 * nc + c * nc + n] = m_;
    out[EP_SGM * 3 * nc + c * nc + n] = s;
  }
}

fdtd_status ensure_edge_props(fdtd_grid *g, cudaStream_t s) {
  if (g->eprops_ready) return FDTD_OK;
  FDTD_CHECK(g->eprops.alloc((size_t)12 * g->nc * g->elem, s));
  const int bl = (int)((g->nc + MB - 1) / MB);
  if (g->prec == FDTD_F64) {
    if (g->id_bytes == 1)
      edge_props_kernel<double, uint8_t><<<bl, MB, 0, s>>>(make_geo<double>(g), g->mat.as<uint8_t>(), g->mtab.as<double>(), g->nmat, g->eprops.as<double>());
    else
      edge_props_kernel<double, uint16_t><<<bl, MB, 0, s>>>(make_geo<double>(g), g->mat.as<uint16_t>(), g->mtab.as<double>(), g->nmat, g->eprops.as<double>());
  } else {
    if (g->id_bytes == 1)
      edge_props_kernel<float, uint8_t><<<bl, MB, 0, s>>>(make_geo<float>(g), g->mat.as<uint8_t>(), g->mtab.as<float>(), g->nmat, g->eprops.as<float>());
    else
      edge_props_kernel<float, uint16_t><<<bl, MB, 0, s>>>(make_geo<float>(g), g->mat.as<uint16_t>(), g->mtab.as<float>(), g->nmat, g->eprops.as<float>());
  }
  FDTD_CHECK(after_launch("edge_props_kernel"));
  g->eprops_ready = true;
  return FDTD_OK;
}

// ------------------------------------------------------------------ operators
template <typename T>
struct OpArgs {
  Geo<T> g;
  const T *eps, *sig, *mu, *sgm;   // per-edge properties (3 x nc each)
  T inv_dt;
  T vscale;                        // 1 / (volume of cell 0): edge volumes in units of it
  cplx<T> z[kMaxRhs];              // expansion point of each right-hand side
  cplx<T> cz[kMaxRhs];             // coefficient of the curl term
};

// Volume of E edge c at cell (i, j, k) -- primal length times dual area --
// in units of the volume of cell 0; 0 on wall edges (dual length 0).
template <typename T>
__device__ __forceinline__ T edge_volume(const OpArgs<T> &a, int c, int i, int j, int k) {
  const Geo<T> &g = a.g;
  T d;
  if (c == 0) d = g.rd(0, i) * g.rdd(1, j) * g.rdd(2, k);
  else if (c == 1) d = g.rd(1, j) * g.rdd(0, i) * g.rdd(2, k);
  else d = g.rd(2, k) * g.rdd(0, i) * g.rdd(1, j);
  return d != T(0) ? a.vscale / d : T(0);
}

// r1 = (eps/dt + sig/2) v1, r2 = curlE(v1) + (mu/dt + sgm/2) v2   [(R+F) v]
template <typename T>
__global__ void rpf_kernel(OpArgs<T> a, const cplx<T> *__restrict__ v, int64_t vstride,
                           cplx<T> *__restrict__ r, int64_t rstride) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  const cplx<T> *vb = v + b * vstride;
  cplx<T> *rb = r + b * rstride;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, a.g.nc, i, j, k);
  auto ld = [&](int64_t idx) { return vb[idx]; };
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const T ep = a.eps[e];
    rb[e] = ep == T(0) ? cplx<T>() : (ep * a.inv_dt + T(0.5) * a.sig[e]) * vb[e];
    const T mu = a.mu[e];
    cplx<T> h;
    if (mu != T(0)) h = curl_e_at<T, cplx<T>>(a.g, ld, c, i, j, k) + (mu * a.inv_dt + T(0.5) * a.sgm[e]) * vb[3 * nc + e];
    rb[3 * nc + e] = h;
  }
}

// t = (r2 + cz curlE(P x)) / a22(z); r2 and x optional; P optional diagonal.
template <typename T>
__global__ void h_from_e_kernel(OpArgs<T> a, const cplx<T> *__restrict__ x, int64_t xstride,
                                const cplx<T> *__restrict__ P, int64_t pstride,
                                const cplx<T> *__restrict__ r2, int64_t r2stride,
                                cplx<T> *__restrict__ t, int64_t tstride, const int *__restrict__ active,
                                int astride = 1) {
  const int b = blockIdx.y;
  if (active && !active[b * astride]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, a.g.nc, i, j, k);
  const cplx<T> *xb = x ? x + b * xstride : nullptr;
  const cplx<T> *pb = P ? P + b * pstride : nullptr;
  auto ld = [&](int64_t idx) { return pb ? pb[idx] * xb[idx] : xb[idx]; };
  const cplx<T> z = a.z[b], zm1(z.re - T(1), z.im), zp1(z.re + T(1), z.im);
  cplx<T> ce[3];
  if (xb) curl_e3<T, cplx<T>>(a.g, ld, i, j, k, n, ce);
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const T mu = a.mu[e];
    cplx<T> out;
    if (mu != T(0)) {
      cplx<T> num;
      if (r2) num = r2[b * r2stride + e];
      if (xb) num = num + a.cz[b] * ce[c];
      const cplx<T> a22 = (mu * a.inv_dt) * zm1 + (T(0.5) * a.sgm[e]) * zp1;
      out = cdiv(num, a22);
    }
    t[b * tstride + e] = out;
  }
}

// Per right-hand-side scalars of the Krylov solvers (device resident).
// itol / imaxit: per right-hand-side tolerance and iteration cap, used when
// the scalar kernel is launched with tol <= 0 (the COCG inner solves of the
// refinement loop, whose captured graph is replayed with changing limits).
struct CgsScal {
  double rho_re, rho_im, alpha_re, alpha_im, beta_re, beta_im, omega_re, omega_im, rn2, bn2;
  double itol;
  int active, iters, status, restarts, imaxit, pad;
};

enum EMode { EM_RHS = 0, EM_APPLY = 1, EM_APPLY_DOT = 2, EM_APPLY_RUPDATE = 3, EM_RESID = 4, EM_APPLY_VDOT = 5 };
enum ScalMode { SM_INIT = 0, SM_ALPHA = 1, SM_CGS_RHO = 2, SM_OMEGA = 3, SM_BICG_RHO = 4, SM_VERIFY = 5, SM_NORM = 6 };

// Sums nv (<= 3) doubles over the block (blockDim.x a multiple of 32, <= 1024);
// the totals are valid in vals[] of thread 0.  sh holds >= 3*32 doubles.
__device__ __forceinline__ void block_sum(double *vals, int nv, double *sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < nv; ++q) {
    double v = vals[q];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[q * 32 + w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < nv; ++q) {
      double acc = 0;
      for (int ww = 0; ww < nw; ++ww) acc += sh[q * 32 + ww];
      vals[q] = acc;
    }
  }
}

// Update of one right-hand side's scalars from its summed partials acc.
__device__ void scal_update(CgsScal &s, const double *acc, int mode, double tol, int maxit, int max_restarts) {
  if (tol <= 0) { tol = s.itol; maxit = s.imaxit; }
  const cplx<double> rho(s.rho_re, s.rho_im), d(acc[0], acc[1]);
  auto breakdown = [&]() { s.status = 2; s.active = 0; };
  if (mode == SM_NORM) {
    s.rn2 = acc[2];
  } else if (mode == SM_INIT) {
    s.rho_re = acc[0]; s.rho_im = acc[1]; s.rn2 = acc[2]; s.bn2 = acc[2];
    s.beta_re = s.beta_im = 0; s.omega_re = 1; s.omega_im = 0;
    s.iters = 0; s.status = 0; s.restarts = 0;
    s.active = acc[2] > 0 ? 1 : 0;   // zero right-hand side: x = 0
  } else if (mode == SM_ALPHA) {
    const double ad = sqrt(norm2(d));
    if (ad == 0 || !isfinite(ad)) breakdown();
    else { const cplx<double> al = cdiv(rho, d); s.alpha_re = al.re; s.alpha_im = al.im; }
  } else if (mode == SM_OMEGA) {
    if (!(acc[2] > 0) || !isfinite(acc[2])) breakdown();
    else { s.omega_re = acc[0] / acc[2]; s.omega_im = -acc[1] / acc[2]; }
    if (s.omega_re == 0 && s.omega_im == 0) breakdown();
  } else if (mode == SM_CGS_RHO || mode == SM_BICG_RHO) {
    s.rn2 = acc[2];
    s.iters += 1;
    if (!isfinite(acc[2]) || acc[2] > 1e16 * s.bn2) breakdown();   // diverged
    else if (sqrt(acc[2]) <= tol * sqrt(s.bn2)) s.active = 0;
    else if (s.iters >= maxit) { s.status = 1; s.active = 0; }
    else if (norm2(rho) == 0) breakdown();
    else {
      cplx<double> be = cdiv(d, rho);
      if (mode == SM_BICG_RHO) be = be * cdiv(cplx<double>(s.alpha_re, s.alpha_im), cplx<double>(s.omega_re, s.omega_im));
      s.beta_re = be.re; s.beta_im = be.im;
      s.rho_re = d.re; s.rho_im = d.im;
    }
  } else {  // SM_VERIFY: acc[2] = |b - S x|^2
    s.rn2 = acc[2];
    const bool ok = isfinite(acc[2]) && sqrt(acc[2]) <= 2.0 * tol * sqrt(s.bn2);
    if (!ok && s.restarts < max_restarts && s.iters < maxit) {
      s.restarts += 1; s.active = 1; s.status = 0;
      s.rho_re = acc[2]; s.rho_im = 0; s.beta_re = s.beta_im = 0; s.omega_re = 1; s.omega_im = 0;
    } else if (!ok && s.status == 0) {
      s.status = 3;  // true residual above tolerance after the last restart
    }
  }
}

__global__ void solver_scalars_kernel(int nb, int nblk, const double *__restrict__ partials, CgsScal *sc,
                                      int mode, double tol, int maxit, int max_restarts) {
  const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (b >= nb) return;
  if (mode != SM_VERIFY && mode != SM_INIT && mode != SM_NORM && !sc[b].active) return;  // uniform across the warp
  if (mode == SM_VERIFY && sc[b].status == 1) return;                  // iteration cap reached
  double acc[3] = {0, 0, 0};
#pragma unroll 8
  for (int blk = lane; blk < nblk; blk += 32) {  // unrolled: the loads go out together
    const double *p = partials + ((size_t)b * nblk + blk) * 3;
    acc[0] += p[0]; acc[1] += p[1]; acc[2] += p[2];
  }
  for (int o = 16; o; o >>= 1) {
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
    acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
    acc[2] += __shfl_xor_sync(0xffffffffu, acc[2], o);
  }
  if (lane == 0) scal_update(sc[b], acc, mode, tol, maxit, max_restarts);
}

// Scalar update fused into a producing kernel: each CTA has stored its
// partial triple for right-hand side b; the CTA that takes the last ticket
// sums all gridDim.x triples of b (fixed order: thread-strided, then the
// block tree), applies `mode` with the per-RHS limits and returns the ticket
// counter to 0 for the next launch.  No CTA waits for another.
__device__ void last_block_scalars(int b, const double *partials, unsigned *tickets, CgsScal *sc, int mode,
                                   double *sh, int nparts = -1) {
  __shared__ int last;
  if (nparts < 0) nparts = (int)gridDim.x;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&tickets[b], 1u) == (unsigned)nparts - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[3] = {0, 0, 0};
  const double *pb = partials + (size_t)b * nparts * 3;
  for (int blk = threadIdx.x; blk < nparts; blk += blockDim.x) {
    acc[0] += __ldcg(pb + 3 * blk);
    acc[1] += __ldcg(pb + 3 * blk + 1);
    acc[2] += __ldcg(pb + 3 * blk + 2);
  }
  block_sum(acc, 3, sh);
  if (threadIdx.x == 0) {
    scal_update(sc[b], acc, mode, -1.0, 0, 0);
    tickets[b] = 0;
  }
}

// y = A + cz curlH(t), A = r1 (EM_RHS) or a11(z) P x (apply modes); dead E edges 0.
// EM_APPLY_DOT: partials of rt^H y and |y|^2.  EM_APPLY_VDOT: partials of the
// unconjugated volume-weighted product sum_e V_e x_e y_e (COCG's (p, S p)_V).
// EM_APPLY_RUPDATE: r -= alpha y,
// partials of rt^H r and |r|^2 (y not stored).  EM_RESID: true residual
// y = bhat - S x (bhat passed in rt), partials of |y|^2.
template <typename T, int MODE>
__global__ void __launch_bounds__(MB) e_from_h_kernel(OpArgs<T> a, const cplx<T> *__restrict__ t, int64_t tstride,
                                const cplx<T> *__restrict__ x, int64_t xstride,
                                const cplx<T> *__restrict__ P, int64_t pstride,
                                cplx<T> *__restrict__ y, int64_t ystride,
                                const cplx<T> *__restrict__ rt, cplx<T> *__restrict__ r, int64_t rstride,
                                const CgsScal *__restrict__ sc, double *__restrict__ partials,
                                unsigned *__restrict__ tickets = nullptr) {
  __shared__ double sh[3 * 32];
  const int b = blockIdx.y;
  if (sc && MODE != EM_RESID && !sc[b].active) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  double acc[3] = {0, 0, 0};
  if (n < nc) {
    int i, j, k;
    cell_ijk(n, a.g.nx, a.g.ny, a.g.nc, i, j, k);
    const cplx<T> *tb = t + b * tstride;
    auto ld = [&](int64_t idx) { return tb[idx]; };
    const cplx<T> z = a.z[b], zm1(z.re - T(1), z.im), zp1(z.re + T(1), z.im);
    cplx<T> alpha;
    if (MODE == EM_APPLY_RUPDATE) alpha = cplx<T>((T)sc[b].alpha_re, (T)sc[b].alpha_im);
    cplx<T> ch[3];
    curl_h3<T, cplx<T>>(a.g, ld, i, j, k, n, ch);
    // this cell's three terms of each dot product, summed in the field type
    T s0 = 0, s1 = 0, s2 = 0;
    for (int c = 0; c < 3; ++c) {
      const int64_t e = c * nc + n;
      const T ep = a.eps[e];
      cplx<T> out;
      if (ep != T(0)) {
        cplx<T> A;
        if (MODE == EM_RHS) {
          A = x[b * xstride + e];
        } else {
          const cplx<T> a11 = (ep * a.inv_dt) * zm1 + (T(0.5) * a.sig[e]) * zp1;
          const cplx<T> px = P ? P[b * pstride + e] * x[b * xstride + e] : x[b * xstride + e];
          A = a11 * px;
        }
        out = A + a.cz[b] * ch[c];
      }
      if (MODE == EM_APPLY_VDOT) {
        if (ep != T(0)) {
          const cplx<T> w = edge_volume(a, c, i, j, k) * (x[b * xstride + e] * out);
          s0 += w.re;
          s1 += w.im;
        }
        s2 += norm2(out);
        y[b * ystride + e] = out;
      } else if (MODE == EM_APPLY_DOT) {
        const cplx<T> w = conj(rt[b * rstride + e]) * out;
        s0 += w.re;
        s1 += w.im;
        s2 += norm2(out);
        y[b * ystride + e] = out;
      } else if (MODE == EM_RESID) {
        cplx<T> rv = rt[b * rstride + e] - out;
        if (ep == T(0)) rv = cplx<T>();
        y[b * ystride + e] = rv;
        s0 += norm2(rv);
        s2 += norm2(rv);
      } else if (MODE == EM_APPLY_RUPDATE) {
        cplx<T> rv = r[b * rstride + e] - alpha * out;
        if (ep == T(0)) rv = cplx<T>();
        r[b * rstride + e] = rv;
        const cplx<T> w = conj(rt[b * rstride + e]) * rv;
        s0 += w.re;
        s1 += w.im;
        s2 += norm2(rv);
      } else {
        y[b * ystride + e] = out;
      }
    }
    acc[0] = (double)s0;
    acc[1] = (double)s1;
    acc[2] = (double)s2;
  }
  if (MODE == EM_APPLY_DOT || MODE == EM_APPLY_VDOT || MODE == EM_APPLY_RUPDATE || MODE == EM_RESID) {
    block_sum(acc, 3, sh);
    if (threadIdx.x == 0) {
      double *pb = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
      pb[0] = acc[0]; pb[1] = acc[1]; pb[2] = acc[2];
    }
    // COCG: alpha = rho / (p, S p)_V by the last CTA of this right-hand side
    if (MODE == EM_APPLY_VDOT && tickets) last_block_scalars(b, partials, tickets, const_cast<CgsScal *>(sc), SM_ALPHA, sh);
  }
}

// ------------------------------------------- fused one-pass Schur apply
// q = a11 p + z curlH(curlE(p) / a22) in one pass over memory: the H-part
// intermediate t lives in shared memory only.  A CTA owns a tile of
// kSX x kSY cells in x, y, a group of NB right-hand sides, and marches a
// chunk of z planes upwards.  Per plane k: warps 0..kSY compute t(k) =
// curlE(p)/a22 on rows j0-1 .. j0+kSY-1 of the tile's 32 columns and warp
// kSY+1 on the -x halo column (i0-1), into the plane-parity slot of the shared
// tile; after one barrier warps 1..kSY form q at their own cells from t(k)
// (own, -x, -y neighbours) and t(k-1) (own position, kept in registers).  Two
// parity slots make one barrier per plane enough.  Every thread issues the
// loads of all NB right-hand sides of a plane (and the material properties of
// both phases) before using them: the march is latency-bound, and NB
// independent load streams per warp keep more of them in flight.  H edges
// outside the grid contribute zero, as in curl_h3.
// VDOT: partials of (p, q)_V and, with tickets, alpha = rho / (p, q)_V by
// the last CTA of each right-hand side.  Grid: (RHS groups, tiles, z chunks).
// The COCG form (FP32, dot terms, one RHS per thread) is held to 64
// registers for three CTAs per SM, without spills: more warps in flight,
// 2.84 against 2.99 s for the q = 200 basis of the 64^3 cavity (four CTAs
// spill: 2.85 s).
constexpr int kSX = 32, kSY = 8;
constexpr int kSThreads = 32 * (kSY + 2);

template <typename T, bool VDOT, int NB>
__global__ void __launch_bounds__(kSThreads, (VDOT && NB == 1 && sizeof(T) == 4) ? 3 : 2) schur_fused_kernel(OpArgs<T> a, int nb, const cplx<T> *__restrict__ p,
                                                                   cplx<T> *__restrict__ q, int64_t stride, int ntx,
                                                                   int zchunk, CgsScal *__restrict__ sc,
                                                                   double *__restrict__ partials,
                                                                   unsigned *__restrict__ tickets) {
  extern __shared__ __align__(16) unsigned char ts_raw[];
  cplx<T> *ts = reinterpret_cast<cplx<T> *>(ts_raw);  // [parity][r][c][row][col]
  auto TS = [&](int par, int r, int c, int row, int col) -> cplx<T> & {
    return ts[((((par * NB + r) * 3 + c) * (kSY + 1) + row) * (kSX + 1)) + col];
  };
  __shared__ double sh[3 * 32];
  const int b0 = blockIdx.x * NB;
  bool act[NB];
  bool any = false;
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    act[r] = b0 + r < nb && (!VDOT || !sc || sc[b0 + r].active);
    any |= act[r];
  }
  if (!any) return;
  const Geo<T> &g = a.g;
  const int64_t nc = g.nc, sy = g.nx, sz = (int64_t)g.nx * g.ny;
  const int tile = blockIdx.y, i0 = (tile % ntx) * kSX, j0 = (tile / ntx) * kSY;
  const int k0 = blockIdx.z * zchunk, k1 = min(g.nz, k0 + zchunk);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pi, pj, prow, pcol;  // phase-1 position of this thread and its shared slot
  if (warp <= kSY) { pi = i0 + lane; pj = j0 - 1 + warp; prow = warp; pcol = lane + 1; }
  else { pi = i0 - 1; pj = j0 - 1 + lane; prow = lane; pcol = 0; }
  const bool writer = warp <= kSY || lane <= kSY;
  const bool p1 = writer && pi >= 0 && pi < g.nx && pj >= 0 && pj < g.ny;
  const bool own = warp >= 1 && warp <= kSY && pi < g.nx && pj < g.ny;  // phase-2 owner of (pi, pj)
  const bool ip = pi + 1 < g.nx, jp = pj + 1 < g.ny;
  cplx<T> zm1[NB], zp1[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    const cplx<T> z = a.z[min(b0 + r, nb - 1)];
    zm1[r] = cplx<T>(z.re - T(1), z.im);
    zp1[r] = cplx<T>(z.re + T(1), z.im);
  }
  const T rx = p1 ? g.rd(0, pi) : T(0), ry = p1 ? g.rd(1, pj) : T(0);
  const T rdx = own ? g.rdd(0, pi) : T(0), rdy = own ? g.rdd(1, pj) : T(0);
  const int64_t n00 = p1 ? g.id(pi, pj, 0) : 0;
  // own Ex, Ey of the position at the current plane, carried up the march
  cplx<T> cex[NB], cey[NB], tpx[NB], tpy[NB];
  auto load_carry = [&](int kk) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const cplx<T> *pb = p + (int64_t)(b0 + (act[r] ? r : 0)) * stride;
      const int64_t n = n00 + kk * sz;
      cex[r] = act[r] ? pb[n] : cplx<T>();
      cey[r] = act[r] ? pb[nc + n] : cplx<T>();
    }
  };
  // t at the position at plane kk from the carried own ex, ey and the seven
  // other E values of curlE (all NB right-hand sides loaded first); own ez
  // and the plane kk+1 ex, ey are returned for the caller.
  auto tplane = [&](int kk, cplx<T> (*tk)[3], cplx<T> *oez, cplx<T> *nex, cplx<T> *ney, const T *mu,
                    const T *sgm) {
    const int64_t n = n00 + kk * sz;
    const bool kp = kk + 1 < g.nz;
    const T rz = g.rd(2, kk);
    cplx<T> ez[NB], eyi[NB], ezi[NB], exj[NB], ezj[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const cplx<T> *pb = p + (int64_t)(b0 + (act[r] ? r : 0)) * stride;
      const bool ok = act[r];
      ez[r] = ok ? pb[2 * nc + n] : cplx<T>();
      eyi[r] = ok && ip ? pb[nc + n + 1] : cplx<T>();
      ezi[r] = ok && ip ? pb[2 * nc + n + 1] : cplx<T>();
      exj[r] = ok && jp ? pb[n + sy] : cplx<T>();
      ezj[r] = ok && jp ? pb[2 * nc + n + sy] : cplx<T>();
      nex[r] = ok && kp ? pb[n + sz] : cplx<T>();
      ney[r] = ok && kp ? pb[nc + n + sz] : cplx<T>();
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      cplx<T> ce[3];
      ce[0] = ry * (ezj[r] - ez[r]) - rz * (ney[r] - cey[r]);
      ce[1] = rz * (nex[r] - cex[r]) - rx * (ezi[r] - ez[r]);
      ce[2] = rx * (eyi[r] - cey[r]) - ry * (exj[r] - cex[r]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cplx<T> o;
        if (mu[c] != T(0)) o = cdiv(ce[c], (mu[c] * a.inv_dt) * zm1[r] + (T(0.5) * sgm[c]) * zp1[r]);
        tk[r][c] = o;
      }
      oez[r] = ez[r];
    }
  };
#pragma unroll
  for (int r = 0; r < NB; ++r) { tpx[r] = cplx<T>(); tpy[r] = cplx<T>(); cex[r] = cplx<T>(); cey[r] = cplx<T>(); }
  if (p1) load_carry(k0 > 0 ? k0 - 1 : k0);
  if (p1 && k0 > 0) {
    // t(k0-1) at the position (owners keep its x, y components); the carry
    // moves to plane k0
    const int64_t e = n00 + (int64_t)(k0 - 1) * sz;
    T mu[3], sgm[3];
    for (int c = 0; c < 3; ++c) { mu[c] = a.mu[c * nc + e]; sgm[c] = a.sgm[c * nc + e]; }
    cplx<T> tk[NB][3], oez[NB], nex[NB], ney[NB];
    tplane(k0 - 1, tk, oez, nex, ney, mu, sgm);
#pragma unroll
    for (int r = 0; r < NB; ++r) { tpx[r] = tk[r][0]; tpy[r] = tk[r][1]; cex[r] = nex[r]; cey[r] = ney[r]; }
  }
  T s0[NB], s1[NB], s2[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) s0[r] = s1[r] = s2[r] = T(0);
  for (int kk = k0; kk < k1; ++kk) {
    const int par = kk & 1;
    const int64_t e = n00 + (int64_t)kk * sz;
    // material properties of both phases first
    T mu[3] = {0, 0, 0}, sgm[3] = {0, 0, 0}, ep[3] = {0, 0, 0}, sg[3] = {0, 0, 0};
    if (p1)
      for (int c = 0; c < 3; ++c) { mu[c] = a.mu[c * nc + e]; sgm[c] = a.sgm[c * nc + e]; }
    if (own)
      for (int c = 0; c < 3; ++c) { ep[c] = a.eps[c * nc + e]; sg[c] = a.sig[c * nc + e]; }
    cplx<T> tk[NB][3], pe[NB][3];
    if (p1) {
      cplx<T> oez[NB], nex[NB], ney[NB];
      tplane(kk, tk, oez, nex, ney, mu, sgm);
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        pe[r][0] = cex[r]; pe[r][1] = cey[r]; pe[r][2] = oez[r];
        cex[r] = nex[r]; cey[r] = ney[r];
      }
    } else {
#pragma unroll
      for (int r = 0; r < NB; ++r) tk[r][0] = tk[r][1] = tk[r][2] = pe[r][0] = pe[r][1] = pe[r][2] = cplx<T>();
    }
    if (writer)
#pragma unroll
      for (int r = 0; r < NB; ++r)
        for (int c = 0; c < 3; ++c) TS(par, r, c, prow, pcol) = tk[r][c];
    __syncthreads();
    if (own) {
      const T rz = g.rdd(2, kk);
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        if (!act[r]) continue;
        const cplx<T> hx = tk[r][0], hy = tk[r][1], hz = tk[r][2];
        const cplx<T> hz_jm = TS(par, r, 2, prow - 1, pcol), hx_jm = TS(par, r, 0, prow - 1, pcol);
        const cplx<T> hz_im = TS(par, r, 2, prow, pcol - 1), hy_im = TS(par, r, 1, prow, pcol - 1);
        const cplx<T> hy_km = kk > 0 ? tpy[r] : cplx<T>(), hx_km = kk > 0 ? tpx[r] : cplx<T>();
        cplx<T> ch[3];
        ch[0] = rdy * (hz - hz_jm) - rz * (hy - hy_km);
        ch[1] = rz * (hx - hx_km) - rdx * (hz - hz_im);
        ch[2] = rdx * (hy - hy_im) - rdy * (hx - hx_jm);
        const cplx<T> czb = a.cz[b0 + r];
        for (int c = 0; c < 3; ++c) {
          cplx<T> out;
          if (ep[c] != T(0)) {
            const cplx<T> a11 = (ep[c] * a.inv_dt) * zm1[r] + (T(0.5) * sg[c]) * zp1[r];
            out = a11 * pe[r][c] + czb * ch[c];
            if (VDOT) {
              const cplx<T> w = edge_volume(a, c, pi, pj, kk) * (pe[r][c] * out);
              s0[r] += w.re;
              s1[r] += w.im;
            }
            s2[r] += norm2(out);
          }
          q[(int64_t)(b0 + r) * stride + c * nc + e] = out;
        }
        tpx[r] = hx; tpy[r] = hy;
      }
    }
  }
  if (VDOT) {
    const int nparts = gridDim.y * gridDim.z;
    const int part = blockIdx.y + gridDim.y * blockIdx.z;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      if (!act[r]) continue;  // uniform across the CTA
      double acc[3] = {(double)s0[r], (double)s1[r], (double)s2[r]};
      block_sum(acc, 3, sh);
      if (threadIdx.x == 0) {
        double *pp = partials + ((size_t)(b0 + r) * nparts + part) * 3;
        pp[0] = acc[0]; pp[1] = acc[1]; pp[2] = acc[2];
      }
      if (tickets) last_block_scalars(b0 + r, partials, tickets, sc, SM_ALPHA, sh, nparts);
      __syncthreads();
    }
  }
}

// Launch of schur_fused_kernel: tiles of kSX x kSY, right-hand sides in
// groups of NB (3 for FP32: one per expansion point of L = 2; 1 for FP64),
// z chunks sized for about four CTAs per SM.
template <typename T, bool VDOT>
fdtd_status launch_schur_fused(const fdtd_grid *g, const OpArgs<T> &a, int nb, const cplx<T> *p, cplx<T> *q,
                               int64_t stride, CgsScal *sc, double *partials, unsigned *tickets, cudaStream_t s) {
  // NB = 3 for the plain apply (0.80 against 1.00 ms on 384x384x64 with three
  // right-hand sides); the COCG form keeps NB = 1, whose registers fit without
  // spilling beside the dot-product terms
  const char *env = getenv("FDTDMOR_SCHUR_NB");
  int NB = (sizeof(T) == 8 || VDOT) ? 1 : std::min(nb, 3);
  if (env && sizeof(T) == 4) NB = std::max(1, std::min(3, atoi(env)));
  const int ntx = (g->nx + kSX - 1) / kSX, nty = (g->ny + kSY - 1) / kSY;
  const int ngrp = (nb + NB - 1) / NB;
  const int64_t per = (int64_t)ntx * nty * ngrp;
  int want = (int)std::max<int64_t>(1, (152 * 4 + per - 1) / per);
  want = std::min(want, std::max(1, g->nz / 4));
  const int zchunk = (g->nz + want - 1) / want;
  const int nchunk = (g->nz + zchunk - 1) / zchunk;
  const dim3 grid(ngrp, ntx * nty, nchunk);
  const size_t smem = sizeof(cplx<T>) * 2 * NB * 3 * (kSY + 1) * (kSX + 1);
  auto go = [&](auto kern) -> fdtd_status {
    if (smem > 48 * 1024)
      FDTD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kSThreads, smem, s>>>(a, nb, p, q, stride, ntx, zchunk, sc, partials, tickets);
    return after_launch("schur_fused_kernel");
  };
  if (NB == 1) return go(schur_fused_kernel<T, VDOT, 1>);
  if (NB == 2) return go(schur_fused_kernel<T, VDOT, 2>);
  return go(schur_fused_kernel<T, VDOT, 3>);
}

// Jacobi preconditioner: P = 1 / diag(S(z)) on live E edges, 0 on dead ones.
template <typename T>
__global__ void jacobi_kernel(OpArgs<T> a, cplx<T> *__restrict__ P, int64_t pstride) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  const int nx = a.g.nx, ny = a.g.ny;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / ((int64_t)nx * ny));
  const cplx<T> z = a.z[b], zm1(z.re - T(1), z.im), zp1(z.re + T(1), z.im);
  auto inv_a22 = [&](int c, int ii, int jj, int kk) {
    const int64_t e = c * nc + a.g.id(ii, jj, kk);
    const cplx<T> a22 = (a.mu[e] * a.inv_dt) * zm1 + (T(0.5) * a.sgm[e]) * zp1;
    return cdiv(cplx<T>(T(1)), a22);
  };
  const int idx[3] = {i, j, k};
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const T ep = a.eps[e];
    cplx<T> out;
    if (ep != T(0)) {
      // transverse axes and the H component paired with each in curl H
      const int ta[2] = {(c + 1) % 3, (c + 2) % 3};
      const int hc[2] = {(c + 2) % 3, (c + 1) % 3};
      cplx<T> sum;
      for (int q = 0; q < 2; ++q) {
        const int ax = ta[q], h = hc[q], ia = idx[ax];
        int lo[3] = {i, j, k};
        lo[ax] -= 1;
        const cplx<T> t0 = inv_a22(h, i, j, k);
        const cplx<T> t1 = inv_a22(h, lo[0], lo[1], lo[2]);
        sum = sum + a.g.rdd(ax, ia) * (a.g.rd(ax, ia) * t0 + a.g.rd(ax, ia - 1) * t1);
      }
      const cplx<T> a11 = (ep * a.inv_dt) * zm1 + (T(0.5) * a.sig[e]) * zp1;
      out = cdiv(cplx<T>(T(1)), a11 + a.z[b] * sum);
    }
    P[b * pstride + e] = out;
  }
}

// ------------------------------------------------- COCG with a gradient-space
// correction of the Jacobi preconditioner.  The Schur complement
// S = A11 - A12 A22^{-1} A21 of A(z) = z(R+F) - (R-F) is complex symmetric
// (A11, A22 diagonal, A21 = -z A12^T); in the per-volume rows used here it is
// self-adjoint in the unconjugated form (u, w)_V = sum_e V_e u_e w_e, so the
// conjugate-orthogonal CG applies with that product.  Gradient fields G phi
// (G the discrete gradient from grid nodes to E edges, curlE G = 0) are
// annihilated by the curl-curl part, so S G phi = a11 G phi: near z = 1 these
// are the near-null directions a diagonal preconditioner leaves to the Krylov
// method.  The preconditioner adds one damped Jacobi step on the nodal
// operator N = G^T diag(V a11) G:
//   P w = w / diag(S) + G (omega (G^T V w) / diag(N)),
// with phi = 0 on wall nodes and on nodes touching a dead (PEC) edge.  P is
// symmetric in the same product, as COCG requires.
constexpr double kNodalOmega = 0.8;

// diag(N) per node and right-hand side; 0 marks nodes held at phi = 0.
// Node (i, j, k) is the lower corner of cell (i, j, k); its six E edges are
// Ex(i-1|i, j, k), Ey(i, j-1|j, k), Ez(i, j, k-1|k).  For both x edges of a
// node rd_e V_e equals the dual area 1/(rdd_y rdd_z), likewise for y and z.
template <typename T>
__global__ void cocg_dn_kernel(OpArgs<T> a, cplx<T> *__restrict__ dN) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
  const Geo<T> &g = a.g;
  cplx<T> out;
  if (i >= 1 && j >= 1 && k >= 1) {  // i < nx etc. by construction; the far walls are not stored
    const int64_t sx = 1, sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const int64_t lo[3] = {n - sx, n - sy, n - sz};
    const int idx[3] = {i, j, k};
    const cplx<T> z = a.z[b], zm1(z.re - T(1), z.im), zp1(z.re + T(1), z.im);
    bool live = true;
    cplx<T> acc;
    for (int c = 0; c < 3 && live; ++c) {
      const T area = c == 0 ? T(1) / (g.rdd(1, j) * g.rdd(2, k))
                   : (c == 1 ? T(1) / (g.rdd(0, i) * g.rdd(2, k)) : T(1) / (g.rdd(0, i) * g.rdd(1, j)));
      for (int h = 0; h < 2; ++h) {
        const int64_t e = c * nc + (h ? n : lo[c]);
        const T ep = a.eps[e];
        if (ep == T(0)) { live = false; break; }
        const cplx<T> a11 = (ep * a.inv_dt) * zm1 + (T(0.5) * a.sig[e]) * zp1;
        acc = acc + (a.vscale * area * g.rd(c, idx[c] - 1 + h)) * a11;
      }
    }
    if (live) out = acc;
  }
  dN[b * nc + n] = out;
}

// phi = omega (G^T V (r - alpha q)) / diag(N) per node (INIT: alpha = 0, q unused).
template <typename T, bool INIT>
__global__ void __launch_bounds__(MB) cocg_node_kernel(OpArgs<T> a, const cplx<T> *__restrict__ r,
                                                       const cplx<T> *__restrict__ q, int64_t stride,
                                                       const cplx<T> *__restrict__ dN, cplx<T> *__restrict__ phi,
                                                       const CgsScal *__restrict__ sc) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  const cplx<T> dn = dN[b * nc + n];
  cplx<T> out;
  if (dn.re != T(0) || dn.im != T(0)) {  // live node: interior, all six edges live
    int i, j, k;
    cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
    const Geo<T> &g = a.g;
    cplx<T> alpha;
    if (!INIT) alpha = cplx<T>((T)sc[b].alpha_re, (T)sc[b].alpha_im);
    const cplx<T> *rb = r + b * stride;
    const cplx<T> *qb = INIT ? nullptr : q + b * stride;
    auto w = [&](int64_t e) { return INIT ? rb[e] : rb[e] - alpha * qb[e]; };
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const cplx<T> fx = w(n - 1) - w(n), fy = w(nc + n - sy) - w(nc + n), fz = w(2 * nc + n - sz) - w(2 * nc + n);
    const T ax = T(1) / (g.rdd(1, j) * g.rdd(2, k)), ay = T(1) / (g.rdd(0, i) * g.rdd(2, k)),
            az = T(1) / (g.rdd(0, i) * g.rdd(1, j));
    const cplx<T> f = (a.vscale * ax) * fx + (a.vscale * ay) * fy + (a.vscale * az) * fz;
    out = (T)kNodalOmega * cdiv(f, dn);
  }
  phi[b * nc + n] = out;
}

// Edge pass of a COCG iteration: r' = r - alpha q, x += alpha p,
// zv = P r' = r' / diag(S) + G phi; partials (r', zv)_V and |r'|^2.
// INIT: r' = r, x untouched, partials written for every right-hand side
// (zero for inactive ones, which SM_INIT then leaves inactive).
template <typename T, bool INIT>
__global__ void __launch_bounds__(MB) cocg_edge_kernel(OpArgs<T> a, cplx<T> *__restrict__ r,
                                                       const cplx<T> *__restrict__ q, cplx<T> *__restrict__ x,
                                                       const cplx<T> *__restrict__ p, const cplx<T> *__restrict__ phi,
                                                       const cplx<T> *__restrict__ Jinv, cplx<T> *__restrict__ zv,
                                                       int64_t stride, CgsScal *__restrict__ sc,
                                                       double *__restrict__ partials, unsigned *__restrict__ tickets) {
  __shared__ double sh[3 * 32];
  const int b = blockIdx.y;
  const bool active = sc[b].active != 0;
  if (!active && !INIT) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  double acc[3] = {0, 0, 0};
  if (active && n < nc) {
    int i, j, k;
    cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
    const Geo<T> &g = a.g;
    cplx<T> alpha;
    if (!INIT) alpha = cplx<T>((T)sc[b].alpha_re, (T)sc[b].alpha_im);
    const cplx<T> *phb = phi + b * nc;
    const cplx<T> ph0 = phb[n];
    const int idx[3] = {i, j, k}, nax[3] = {g.nx, g.ny, g.nz};
    const int64_t st[3] = {1, g.nx, (int64_t)g.nx * g.ny};
    T s0 = 0, s1 = 0, s2 = 0;
    for (int c = 0; c < 3; ++c) {
      const int64_t e = c * nc + n, o = b * stride + e;
      if (a.eps[e] == T(0)) {
        if (!INIT) r[o] = cplx<T>();
        zv[o] = cplx<T>();
        continue;
      }
      cplx<T> rv = r[o];
      if (!INIT) {
        rv = rv - alpha * q[o];
        r[o] = rv;
        x[o] = x[o] + alpha * p[o];
      }
      const cplx<T> ph1 = idx[c] + 1 < nax[c] ? phb[n + st[c]] : cplx<T>();
      const cplx<T> zz = Jinv[o] * rv + g.rd(c, idx[c]) * (ph1 - ph0);
      zv[o] = zz;
      const cplx<T> wv = edge_volume(a, c, i, j, k) * (rv * zz);
      s0 += wv.re;
      s1 += wv.im;
      s2 += norm2(rv);
    }
    acc[0] = (double)s0;
    acc[1] = (double)s1;
    acc[2] = (double)s2;
  }
  block_sum(acc, 3, sh);
  if (threadIdx.x == 0) {
    double *pb = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
    pb[0] = acc[0]; pb[1] = acc[1]; pb[2] = acc[2];
  }
  // convergence test and beta = rho'/rho by the last CTA of this right-hand side
  if (!INIT && tickets) last_block_scalars(b, partials, tickets, sc, SM_CGS_RHO, sh);
}

// COCG: p = zv + beta p
template <typename T>
__global__ void cocg_update_p_kernel(int64_t len, const CgsScal *__restrict__ sc, const cplx<T> *__restrict__ zv,
                                     cplx<T> *__restrict__ p, int64_t stride) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const cplx<T> beta((T)sc[b].beta_re, (T)sc[b].beta_im);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    p[o] = zv[o] + beta * p[o];
  }
}

// Refinement loop, FP64 residual r = bhat - S x of the FP64 solution x (the
// FP32 iterates lose the near-static gradient part of x to rounding: S
// amplifies a relative error eps of x by the ratio of its curl-curl and
// diagonal parts, about 1e4 on finely graded cells).  Material properties and
// axis tables are those of the grid, converted to double.
template <typename T>
__global__ void __launch_bounds__(MB) resid64_h_kernel(OpArgs<T> a, const cplx<double> *__restrict__ x,
                                                       cplx<double> *__restrict__ t, int64_t stride) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
  const cplx<double> *xb = x + b * stride;
  auto ld = [&](int64_t idx) { return xb[idx]; };
  const cplx<double> z((double)a.z[b].re, (double)a.z[b].im), zm1(z.re - 1.0, z.im), zp1(z.re + 1.0, z.im);
  cplx<double> ce[3];
  curl_e3<T, cplx<double>>(a.g, ld, i, j, k, n, ce);
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const double mu = (double)a.mu[e];
    cplx<double> out;
    if (mu != 0.0) {
      const cplx<double> a22 = (mu * (double)a.inv_dt) * zm1 + (0.5 * (double)a.sgm[e]) * zp1;
      out = cdiv(ce[c], a22);
    }
    t[b * stride + e] = out;
  }
}

template <typename T>
__global__ void __launch_bounds__(MB) resid64_e_kernel(OpArgs<T> a, const cplx<double> *__restrict__ t,
                                                       const cplx<double> *__restrict__ x, int64_t stride,
                                                       const cplx<double> *__restrict__ bhat, cplx<T> *__restrict__ rout,
                                                       double *__restrict__ partials) {
  __shared__ double sh[3 * 32];
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  double acc[3] = {0, 0, 0};
  if (n < nc) {
    int i, j, k;
    cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
    const cplx<double> *tb = t + b * stride;
    auto ld = [&](int64_t idx) { return tb[idx]; };
    const cplx<double> z((double)a.z[b].re, (double)a.z[b].im), zm1(z.re - 1.0, z.im), zp1(z.re + 1.0, z.im);
    cplx<double> ch[3];
    curl_h3<T, cplx<double>>(a.g, ld, i, j, k, n, ch);
    for (int c = 0; c < 3; ++c) {
      const int64_t e = c * nc + n, o = b * stride + e;
      const double ep = (double)a.eps[e];
      cplx<double> rv;
      if (ep != 0.0) {
        const cplx<double> a11 = (ep * (double)a.inv_dt) * zm1 + (0.5 * (double)a.sig[e]) * zp1;
        rv = bhat[o] - (a11 * x[o] + z * ch[c]);
      }
      rout[o] = cplx<T>((T)rv.re, (T)rv.im);
      acc[2] += norm2(rv);
    }
  }
  block_sum(acc, 3, sh);
  if (threadIdx.x == 0) {
    double *pb = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
    pb[0] = 0; pb[1] = 0; pb[2] = acc[2];
  }
}

// Right-hand side of the Schur system in FP64 from a chain vector v of the
// field type (or from B in r_in when v is null): r = (R+F) v, then
// bhat = r1 + curlH(r2 / a22).  The curls of v and of r2 / a22 difference
// neighbouring values of vectors whose near-static gradient part dominates;
// in FP32 that cancellation leaves errors far above the solve tolerance in
// the chain, so these steps run in FP64 like the residual.
template <typename T>
__global__ void __launch_bounds__(MB) rhs64_h_kernel(OpArgs<T> a, const cplx<T> *__restrict__ v, int64_t vstride,
                                                     cplx<double> *__restrict__ r2, cplx<double> *__restrict__ t,
                                                     int64_t stride) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
  const cplx<double> z((double)a.z[b].re, (double)a.z[b].im), zm1(z.re - 1.0, z.im), zp1(z.re + 1.0, z.im);
  cplx<double> ce[3];
  const cplx<T> *vb = v ? v + b * vstride : nullptr;
  if (vb) {
    auto ld = [&](int64_t idx) { const cplx<T> x = vb[idx]; return cplx<double>((double)x.re, (double)x.im); };
    curl_e3<T, cplx<double>>(a.g, ld, i, j, k, n, ce);
  }
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const double mu = (double)a.mu[e];
    cplx<double> rv, tv;
    if (mu != 0.0 && vb) {
      const cplx<T> h = vb[3 * nc + e];
      rv = ce[c] + (mu * (double)a.inv_dt + 0.5 * (double)a.sgm[e]) * cplx<double>((double)h.re, (double)h.im);
      tv = cdiv(rv, (mu * (double)a.inv_dt) * zm1 + (0.5 * (double)a.sgm[e]) * zp1);
    }
    r2[b * stride + e] = rv;
    t[b * stride + e] = tv;
  }
}

template <typename T>
__global__ void __launch_bounds__(MB) rhs64_e_kernel(OpArgs<T> a, const cplx<T> *__restrict__ v, int64_t vstride,
                                                     const cplx<double> *__restrict__ t,
                                                     cplx<double> *__restrict__ bhat, int64_t stride) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
  const cplx<double> *tb = t + b * stride;
  auto ld = [&](int64_t idx) { return tb[idx]; };
  cplx<double> ch[3];
  curl_h3<T, cplx<double>>(a.g, ld, i, j, k, n, ch);
  const cplx<T> *vb = v + b * vstride;
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const double ep = (double)a.eps[e];
    cplx<double> out;
    if (ep != 0.0) {
      const cplx<T> x = vb[e];
      out = (ep * (double)a.inv_dt + 0.5 * (double)a.sig[e]) * cplx<double>((double)x.re, (double)x.im) + ch[c];
    }
    bhat[b * stride + e] = out;
  }
}

// bhat (FP64) = B in r_in's E part (the chain's first right-hand side)
template <typename T>
__global__ void rhs64_b_kernel(OpArgs<T> a, const cplx<T> *__restrict__ rin, int64_t rstride,
                               cplx<double> *__restrict__ bhat, cplx<double> *__restrict__ r2, int64_t stride) {
  const int b = blockIdx.y;
  const int64_t n3 = 3 * a.g.nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
    const cplx<T> x = rin[b * rstride + e];
    bhat[b * stride + e] = a.eps[e] != T(0) ? cplx<double>((double)x.re, (double)x.im) : cplx<double>();
    r2[b * stride + e] = cplx<double>();
  }
}

// out = [x1; x2] from the FP64 solution: x1 = x, x2 = (r2 - z curlE(x1)) / a22
// in FP64, both rounded to the field type
template <typename T>
__global__ void __launch_bounds__(MB) recover64_kernel(OpArgs<T> a, const cplx<double> *__restrict__ x,
                                                       const cplx<double> *__restrict__ r2, int64_t stride,
                                                       cplx<T> *__restrict__ out, int64_t ostride) {
  const int b = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = a.g.nc;
  if (n >= nc) return;
  int i, j, k;
  cell_ijk(n, a.g.nx, a.g.ny, nc, i, j, k);
  const cplx<double> *xb = x + b * stride;
  auto ld = [&](int64_t idx) { return xb[idx]; };
  const cplx<double> z((double)a.z[b].re, (double)a.z[b].im), zm1(z.re - 1.0, z.im), zp1(z.re + 1.0, z.im);
  cplx<double> ce[3];
  curl_e3<T, cplx<double>>(a.g, ld, i, j, k, n, ce);
  cplx<T> *ob = out + b * ostride;
  for (int c = 0; c < 3; ++c) {
    const int64_t e = c * nc + n;
    const cplx<double> x1 = xb[e];
    ob[e] = cplx<T>((T)x1.re, (T)x1.im);
    const double mu = (double)a.mu[e];
    cplx<double> x2;
    if (mu != 0.0) x2 = cdiv(r2[b * stride + e] - z * ce[c], (mu * (double)a.inv_dt) * zm1 + (0.5 * (double)a.sgm[e]) * zp1);
    ob[3 * nc + e] = cplx<T>((T)x2.re, (T)x2.im);
  }
}

// FP64 copy of an E block of the field type
template <typename T>
__global__ void to64_kernel(int64_t len, const cplx<T> *__restrict__ x, cplx<double> *__restrict__ y, int64_t stride) {
  const int b = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const cplx<T> v = x[b * stride + e];
    y[b * stride + e] = cplx<double>((double)v.re, (double)v.im);
  }
}

// x64 += d for the right-hand sides of the last inner solve (flag per RHS)
template <typename T>
__global__ void acc64_kernel(int64_t len, const int *__restrict__ upd, const cplx<T> *__restrict__ d,
                             cplx<double> *__restrict__ x, int64_t stride) {
  const int b = blockIdx.y;
  if (!upd[b]) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    const cplx<T> v = d[o];
    x[o] = x[o] + cplx<double>((double)v.re, (double)v.im);
  }
}

// out[b] (stride ostride) = x64[b] in the field type
template <typename T>
__global__ void from64_kernel(int64_t len, const cplx<double> *__restrict__ x, int64_t stride,
                              cplx<T> *__restrict__ out, int64_t ostride) {
  const int b = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const cplx<double> v = x[b * stride + e];
    out[b * ostride + e] = cplx<T>((T)v.re, (T)v.im);
  }
}

// CGS vector update 1: u = r + beta q; p = u + beta (q + beta p)
template <typename T>
__global__ void cgs_update1_kernel(int64_t len, const CgsScal *__restrict__ sc, const cplx<T> *__restrict__ r,
                                   cplx<T> *__restrict__ q, cplx<T> *__restrict__ p, cplx<T> *__restrict__ u,
                                   int64_t stride) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const cplx<T> beta((T)sc[b].beta_re, (T)sc[b].beta_im);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    const cplx<T> qq = q[o];
    const cplx<T> uu = r[o] + beta * qq;
    u[o] = uu;
    p[o] = uu + beta * (qq + beta * p[o]);
  }
}

// CGS vector update 2: q = u - alpha v; w = u + q; x += alpha P w  (w stored in v)
template <typename T>
__global__ void cgs_update2_kernel(int64_t len, const CgsScal *__restrict__ sc, const cplx<T> *__restrict__ u,
                                   cplx<T> *__restrict__ v, cplx<T> *__restrict__ q, cplx<T> *__restrict__ x,
                                   const cplx<T> *__restrict__ P, int64_t stride) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const cplx<T> alpha((T)sc[b].alpha_re, (T)sc[b].alpha_im);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    const cplx<T> uu = u[o];
    const cplx<T> qq = uu - alpha * v[o];
    q[o] = qq;
    const cplx<T> w = uu + qq;
    v[o] = w;
    x[o] = x[o] + alpha * (P[o] * w);
  }
}

// Solver scalars from block partials (acc[0] + j acc[1] and acc[2] per RHS).
//   SM_INIT:     rho = rt^H r = |r|^2, |b|^2 = |r|^2, beta = 0
//   SM_ALPHA:    alpha = rho / (rt^H v)
//   SM_CGS_RHO:  rho' = rt^H r, |r|^2 -> convergence; beta = rho'/rho      (CGS)
//   SM_OMEGA:    omega = (t^H s)/(t^H t) from s^H t and |t|^2              (BiCGSTAB)
//   SM_BICG_RHO: rho' = rt^H r, |r|^2 -> convergence; beta = (rho'/rho)(alpha/omega)
//   SM_VERIFY:   true residual |b - S x|^2: restart (rt = r) when above tolerance
//   SM_NORM:     |r|^2 into rn2 only (every right-hand side)
// COCG reuses SM_INIT (rho = (r, P r)_V), SM_ALPHA (alpha = rho / (p, S p)_V)
// and SM_CGS_RHO (rho' = (r, P r)_V, beta = rho'/rho).
// One warp per right-hand side (launch with 32 * nb threads): the warp sums
// that right-hand side's nblk partial triples in a fixed order (lane-strided,
// then a shuffle tree), and lane 0 updates its scalars.

// Restart of the active right-hand sides: shadow residual rt = r, search
// directions zero.
template <typename T>
__global__ void solver_restart_kernel(int64_t len, const CgsScal *__restrict__ sc, const cplx<T> *__restrict__ r,
                                      cplx<T> *__restrict__ rt, cplx<T> *__restrict__ p, cplx<T> *__restrict__ q,
                                      int64_t stride) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    rt[o] = r[o];
    p[o] = cplx<T>();
    q[o] = cplx<T>();
  }
}

// BiCGSTAB: p = r + beta (p - omega v)
template <typename T>
__global__ void bicg_update_p_kernel(int64_t len, const CgsScal *__restrict__ sc, const cplx<T> *__restrict__ r,
                                     const cplx<T> *__restrict__ v, cplx<T> *__restrict__ p, int64_t stride) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const cplx<T> beta((T)sc[b].beta_re, (T)sc[b].beta_im), om((T)sc[b].omega_re, (T)sc[b].omega_im);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    p[o] = r[o] + beta * (p[o] - om * v[o]);
  }
}

// BiCGSTAB: s = r - alpha v
template <typename T>
__global__ void bicg_update_s_kernel(int64_t len, const CgsScal *__restrict__ sc, const cplx<T> *__restrict__ r,
                                     const cplx<T> *__restrict__ v, cplx<T> *__restrict__ sv, int64_t stride) {
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const cplx<T> al((T)sc[b].alpha_re, (T)sc[b].alpha_im);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    sv[o] = r[o] - al * v[o];
  }
}

// BiCGSTAB: x += alpha P p + omega P s; r = s - omega t; partials rt^H r, |r|^2
template <typename T>
__global__ void __launch_bounds__(MB) bicg_update_xr_kernel(int64_t len, const CgsScal *__restrict__ sc,
                                      const cplx<T> *__restrict__ P, const cplx<T> *__restrict__ p,
                                      const cplx<T> *__restrict__ sv, const cplx<T> *__restrict__ tv,
                                      const cplx<T> *__restrict__ rt, cplx<T> *__restrict__ x, cplx<T> *__restrict__ r,
                                      int64_t stride, double *__restrict__ partials) {
  __shared__ double sh[3 * 32];
  const int b = blockIdx.y;
  if (!sc[b].active) return;
  const cplx<T> al((T)sc[b].alpha_re, (T)sc[b].alpha_im), om((T)sc[b].omega_re, (T)sc[b].omega_im);
  T s0 = 0, s1 = 0, s2 = 0;  // this thread's few terms in the field type, then FP64
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    const cplx<T> pw = P[o];
    x[o] = x[o] + pw * (al * p[o] + om * sv[o]);
    const cplx<T> rv = sv[o] - om * tv[o];
    r[o] = rv;
    const cplx<T> w = conj(rt[o]) * rv;
    s0 += w.re; s1 += w.im; s2 += norm2(rv);
  }
  double acc[3] = {(double)s0, (double)s1, (double)s2};
  block_sum(acc, 3, sh);
  if (threadIdx.x == 0) {
    double *pb = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
    pb[0] = acc[0]; pb[1] = acc[1]; pb[2] = acc[2];
  }
}

// partials for the init: rt = r (copy), rho = r^H r, |r|^2
template <typename T>
__global__ void __launch_bounds__(MB) cgs_init_kernel(int64_t len, const cplx<T> *__restrict__ bhat, cplx<T> *__restrict__ r,
                                cplx<T> *__restrict__ rt, cplx<T> *__restrict__ x, cplx<T> *__restrict__ p,
                                cplx<T> *__restrict__ q, int64_t stride, double *__restrict__ partials) {
  __shared__ double sh[3 * 32];
  const int b = blockIdx.y;
  double acc[3] = {0, 0, 0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b * stride + e;
    const cplx<T> v = bhat[o];
    r[o] = v; rt[o] = v; x[o] = cplx<T>(); p[o] = cplx<T>(); q[o] = cplx<T>();
    const double n2 = (double)norm2(v);
    acc[0] += n2; acc[2] += n2;
  }
  block_sum(acc, 3, sh);
  if (threadIdx.x == 0) {
    double *pb = partials + ((size_t)b * gridDim.x + blockIdx.x) * 3;
    pb[0] = acc[0]; pb[1] = 0; pb[2] = acc[2];
  }
}

// ------------------------------------------------------- Gram-Schmidt pieces
// partial dots h[c] = sum_i conj(Q[c][i]) x[i], c < nq (V: T or cplx<T>)
template <typename T, typename V>
__global__ void __launch_bounds__(256) multidot_kernel(int64_t len, const V *__restrict__ Q, int64_t qstride, int nq,
                                                       const V *__restrict__ x, double *__restrict__ partials) {
  constexpr int CH = 8;  // elements per thread
  __shared__ __align__(16) unsigned char xs_raw[256 * CH * sizeof(V)];
  V *xs = reinterpret_cast<V *>(xs_raw);
  __shared__ double wsum[kMaxDots * 2 * 8];
  const int64_t base = (int64_t)blockIdx.x * 256 * CH;
  for (int t = 0; t < CH; ++t) {
    const int64_t e = base + t * 256 + threadIdx.x;
    xs[t * 256 + threadIdx.x] = e < len ? x[e] : V(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < nq; ++c) {
    double re = 0, im = 0;
    const V *qc = Q + c * qstride;
    for (int t = 0; t < CH; ++t) {
      const int64_t e = base + t * 256 + threadIdx.x;
      if (e < len) {
        const V qv = qc[e], xv = xs[t * 256 + threadIdx.x];
        if constexpr (sizeof(V) == 2 * sizeof(T)) {
          const cplx<T> pr = conj(*(const cplx<T> *)&qv) * *(const cplx<T> *)&xv;
          re += (double)pr.re; im += (double)pr.im;
        } else {
          re += (double)(*(const T *)&qv) * (double)(*(const T *)&xv);
        }
      }
    }
    for (int o = 16; o; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) { wsum[(c * 2) * 8 + w] = re; wsum[(c * 2 + 1) * 8 + w] = im; }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * nq; q += 256) {
    double a = 0;
    for (int ww = 0; ww < 8; ++ww) a += wsum[q * 8 + ww];
    partials[(size_t)q * gridDim.x + blockIdx.x] = a;
  }
}

// h[q] = sum over blocks of partials (2*nq values, complex as re/im pairs)
__global__ void reduce_partials_kernel(int nvals, int nblk, const double *__restrict__ partials,
                                       double *__restrict__ out) {
  const int q = blockIdx.x;
  if (q >= nvals) return;
  double a = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += partials[(size_t)q * nblk + b];
  for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    out[q] = t;
  }
}

// x -= sum_c Q[c] h[c]
template <typename T, typename V>
__global__ void multiaxpy_kernel(int64_t len, const V *__restrict__ Q, int64_t qstride, int nq,
                                 const double *__restrict__ h, V *__restrict__ x) {
  __shared__ double hs[kMaxDots * 2];
  for (int q = threadIdx.x; q < 2 * nq; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(V) == 2 * sizeof(T)) {
      cplx<T> acc = *(const cplx<T> *)&x[e];
      for (int c = 0; c < nq; ++c) {
        const cplx<T> qv = *(const cplx<T> *)&Q[c * qstride + e];
        acc = acc - cplx<T>((T)hs[2 * c], (T)hs[2 * c + 1]) * qv;
      }
      *(cplx<T> *)&x[e] = acc;
    } else {
      T acc = *(const T *)&x[e];
      for (int c = 0; c < nq; ++c) acc -= (T)hs[2 * c] * *(const T *)&Q[c * qstride + e];
      *(T *)&x[e] = acc;
    }
  }
}

// out = x * s (s = 1/norm from device), or plain copy when s == nullptr
template <typename V, typename T>
__global__ void scale_copy_kernel(int64_t len, const V *__restrict__ x, V *__restrict__ out, T s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(V) == 2 * sizeof(T)) {
      const cplx<T> v = *(const cplx<T> *)&x[e];
      *(cplx<T> *)&out[e] = s * v;
    } else {
      *(T *)&out[e] = s * *(const T *)&x[e];
    }
  }
}

// real part (part = 0) or imaginary part (part = 1) of a complex vector
template <typename T>
__global__ void take_part_kernel(int64_t len, const cplx<T> *__restrict__ x, int part, T *__restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = part ? x[e].im : x[e].re;
}

// ------------------------------------------------------------------ host side
template <typename T>
struct Work {
  int nb = 0;
  int64_t nc = 0;
  DevBuf v;        // nb x 6nc complex: current chain vector (input to (R+F))
  DevBuf r;        // nb x 6nc complex: (R+F) v
  DevBuf bhat;     // nb x 3nc
  DevBuf P;        // nb x 3nc preconditioner
  DevBuf x, rr, rt, u, p, q, vv;   // nb x 3nc CGS vectors
  DevBuf t;        // nb x 3nc H-part temporary
  DevBuf partials; // nb x nblk x 3 doubles
  DevBuf sc;       // nb CgsScal
  DevBuf dots;     // kMaxDots*2 doubles
  DevBuf dpart;    // 2*kMaxDots x nblk_dot doubles
  DevBuf x64, t64; // nb x 3nc complex FP64: refined solution and H-part temporary (COCG)
  DevBuf phi, dN;  // nb x nc nodal potential and nodal diagonal (COCG)
  DevBuf upd;      // nb ints: right-hand sides the last inner solve updated
  DevBuf tickets;  // 2 x kMaxRhs CTA tickets of the fused scalar updates (COCG)
  DevBuf bhat64, r2_64;  // nb x 3nc complex FP64: right-hand side and H part of (R+F) v (COCG)
};

template <typename T>
static OpArgs<T> make_op(fdtd_grid *g, double dt0, const std::vector<std::complex<double>> &zs,
                         const std::vector<std::complex<double>> &czs) {
  OpArgs<T> a;
  a.g = make_geo<T>(g);
  const T *ep = g->eprops.as<T>();
  a.eps = ep + EP_EPS * 3 * g->nc;
  a.sig = ep + EP_SIG * 3 * g->nc;
  a.mu = ep + EP_MU * 3 * g->nc;
  a.sgm = ep + EP_SGM * 3 * g->nc;
  a.inv_dt = (T)(1.0 / dt0);
  a.vscale = (T)(1.0 / (g->dx[0] * g->dy[0] * g->dz[0]));
  for (size_t b = 0; b < zs.size(); ++b) {
    a.z[b] = cplx<T>((T)zs[b].real(), (T)zs[b].imag());
    a.cz[b] = cplx<T>((T)czs[b].real(), (T)czs[b].imag());
  }
  return a;
}

// W[c][r] -= sum_k V[k][r] H[k][c] for r < len, c < nb (H: qc x nb FP64,
// row-major); V columns of stride ldv, W columns of stride ldw.  H is staged
// in shared memory as FP32 (kBlkMax columns at most).
constexpr int kBlkMax = 16;
template <typename T>
__global__ void __launch_bounds__(256) block_axpy_kernel(int64_t len, const T *__restrict__ V, int64_t ldv, int qc,
                                                         const double *__restrict__ H, int nb, T *__restrict__ W,
                                                         int64_t ldw) {
  extern __shared__ float hs[];  // [qc][kBlkMax]
  for (int t = threadIdx.x; t < qc * kBlkMax; t += blockDim.x) {
    const int k = t / kBlkMax, c = t % kBlkMax;
    hs[t] = c < nb ? (float)H[(size_t)k * nb + c] : 0.0f;
  }
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < len; r += (int64_t)gridDim.x * blockDim.x) {
    float acc[kBlkMax];
#pragma unroll
    for (int c = 0; c < kBlkMax; ++c) acc[c] = 0.0f;
    for (int k = 0; k < qc; ++k) {
      const float v = (float)V[(size_t)k * ldv + r];
#pragma unroll
      for (int c = 0; c < kBlkMax; ++c) acc[c] += v * hs[k * kBlkMax + c];
    }
    for (int c = 0; c < nb; ++c) W[(size_t)c * ldw + r] -= (T)acc[c];
  }
}

template <typename T>
struct BasisBuilder {
  fdtd_grid *g;
  const mor_opts o;
  cudaStream_t s;
  int64_t nc;
  int nblk;
  int max_iters = 0;
  double max_resid = 0;
  bool noconv = false;
  bool last_failed = false;
  int fallbacks = 0;
  std::vector<int> rhs_failed;  // per right-hand side, of the last solve
  std::vector<int> rhs_iters;   // per right-hand side, of the last solve
  std::vector<double> rhs_resid;
  cudaStream_t cap = nullptr;   // private stream the solver iterations are captured on
  cudaGraphExec_t cocg_graph = nullptr;  // 16 captured COCG iterations (the buffers and points
  int64_t cocg_graph_launches = 0;       // are fixed for a whole build)
  int outer_max = 0;            // most refinement steps one shifted solve took (COCG)

  BasisBuilder(fdtd_grid *g_, const mor_opts &o_, cudaStream_t s_) : g(g_), o(o_), s(s_) {
    nc = g->nc;
    nblk = (int)((nc + MB - 1) / MB);
  }
  ~BasisBuilder() {
    if (cocg_graph) cudaGraphExecDestroy(cocg_graph);
    if (cap) cudaStreamDestroy(cap);
  }
  BasisBuilder(const BasisBuilder &) = delete;
  BasisBuilder &operator=(const BasisBuilder &) = delete;

  // Solve A(z_b) x = (R+F) v for every active right-hand side b (x = [x1; x2]
  // written to out, nb x 6nc).  v: nb x 6nc (B itself when from_b).
  fdtd_status solve(Work<T> &w, const std::vector<std::complex<double>> &zs, bool from_b,
                    const cplx<T> *vin, cplx<T> *out) {
    if (uses_cocg()) {
      FDTD_CHECK(make_rhs64(w, zs, from_b, vin));
      FDTD_CHECK(schur_cocg(w, zs));
      return recover64(w, zs, out);
    }
    FDTD_CHECK(make_rhs(w, zs, from_b, vin));
    FDTD_CHECK(schur_solve(w, zs));
    return recover(w, zs, out);
  }

  bool uses_cocg() const {
    return o.solver == MOR_SOLVER_COCG || (o.solver == MOR_SOLVER_AUTO && g->prec != FDTD_F64);
  }

  fdtd_status alloc64(Work<T> &w, int nb) {
    const size_t n = sizeof(cplx<double>) * nb * 3 * nc;
    FDTD_CHECK(w.bhat64.alloc(n, s));
    FDTD_CHECK(w.r2_64.alloc(n, s));
    FDTD_CHECK(w.x64.alloc(n, s));
    return w.t64.alloc(n, s);
  }

  // FP64 bhat (and r2 for the recovery) from the chain vector or from B
  fdtd_status make_rhs64(Work<T> &w, const std::vector<std::complex<double>> &zs, bool from_b, const cplx<T> *vin) {
    const int nb = (int)zs.size();
    const int64_t n3 = 3 * nc, n6 = 6 * nc;
    std::vector<std::complex<double>> one(nb, 1.0);
    FDTD_CHECK(alloc64(w, nb));
    OpArgs<T> a = make_op<T>(g, o.dt0, zs, one);
    cplx<double> *bh = w.bhat64.template as<cplx<double>>(), *r2 = w.r2_64.template as<cplx<double>>();
    cplx<double> *t = w.t64.template as<cplx<double>>();
    if (from_b) {
      rhs64_b_kernel<T><<<dim3(std::min(nblk, 152 * 8), nb), MB, 0, s>>>(a, w.r.template as<cplx<T>>(), n6, bh, r2, n3);
      return after_launch("rhs64_b_kernel");
    }
    rhs64_h_kernel<T><<<dim3(nblk, nb), MB, 0, s>>>(a, vin, n6, r2, t, n3);
    FDTD_CHECK(after_launch("rhs64_h_kernel"));
    rhs64_e_kernel<T><<<dim3(nblk, nb), MB, 0, s>>>(a, vin, n6, t, bh, n3);
    return after_launch("rhs64_e_kernel");
  }

  fdtd_status recover64(Work<T> &w, const std::vector<std::complex<double>> &zs, cplx<T> *out) {
    const int nb = (int)zs.size();
    OpArgs<T> a = make_op<T>(g, o.dt0, zs, zs);
    recover64_kernel<T><<<dim3(nblk, nb), MB, 0, s>>>(a, w.x64.template as<cplx<double>>(),
                                                      w.r2_64.template as<cplx<double>>(), 3 * nc, out, 6 * nc);
    return after_launch("recover64_kernel");
  }

  // bhat = r1 + curlH(r2 / a22) of r = (R+F) v (or of r = B already in w.r)
  fdtd_status make_rhs(Work<T> &w, const std::vector<std::complex<double>> &zs, bool from_b, const cplx<T> *vin) {
    const int nb = (int)zs.size();
    const int64_t n3 = 3 * nc, n6 = 6 * nc;
    std::vector<std::complex<double>> one(nb, 1.0);
    dim3 grid2(nblk, nb);
    cplx<T> *r = w.r.template as<cplx<T>>(), *t = w.t.template as<cplx<T>>();
    OpArgs<T> a = make_op<T>(g, o.dt0, zs, one);
    if (!from_b) {
      rpf_kernel<T><<<grid2, MB, 0, s>>>(a, vin, n6, r, n6);
      FDTD_CHECK(after_launch("rpf_kernel"));
    }
    h_from_e_kernel<T><<<grid2, MB, 0, s>>>(a, nullptr, 0, nullptr, 0, r + n3, n6, t, n3, nullptr);
    FDTD_CHECK(after_launch("h_from_e_kernel"));
    e_from_h_kernel<T, EM_RHS><<<grid2, MB, 0, s>>>(a, t, n3, r, n6, nullptr, 0, w.bhat.template as<cplx<T>>(), n3,
                                                    nullptr, nullptr, 0, nullptr, nullptr);
    return after_launch("e_from_h_kernel");
  }

  // out = [x1; x2] with x1 = w.x and x2 = (r2 - z curlE(x1)) / a22
  fdtd_status recover(Work<T> &w, const std::vector<std::complex<double>> &zs, cplx<T> *out) {
    const int nb = (int)zs.size();
    const int64_t n3 = 3 * nc, n6 = 6 * nc;
    std::vector<std::complex<double>> negz(nb);
    for (int b = 0; b < nb; ++b) negz[b] = -zs[b];
    cplx<T> *x = w.x.template as<cplx<T>>(), *r = w.r.template as<cplx<T>>();
    for (int b = 0; b < nb; ++b)
      FDTD_CHECK_CUDA(cudaMemcpyAsync(out + b * n6, x + b * n3, sizeof(cplx<T>) * n3, cudaMemcpyDeviceToDevice, s));
    OpArgs<T> ah = make_op<T>(g, o.dt0, zs, negz);
    // h_from_e writes its output with stride tstride; point it at the H half of out
    h_from_e_kernel<T><<<dim3(nblk, nb), MB, 0, s>>>(ah, x, n3, nullptr, 0, r + n3, n6, out + n3, n6, nullptr);
    return after_launch("h_from_e_kernel");
  }

  // S(z_b) x1 = bhat_b (w.bhat) -> w.x.  COCG (MOR_SOLVER_COCG, AUTO on FP32
  // grids); the paper's CGS (AUTO on FP64 grids, falling back to BiCGSTAB for
  // the whole block when a right-hand side fails); or BiCGSTAB.
  fdtd_status schur_solve(Work<T> &w, const std::vector<std::complex<double>> &zs) {
    if (uses_cocg()) {
      // bhat of the field type (mor_shifted_solve) -> FP64
      const int nb = (int)zs.size();
      FDTD_CHECK(alloc64(w, nb));
      to64_kernel<T><<<dim3(std::min(nblk, 152 * 8), nb), MB, 0, s>>>(3 * nc, w.bhat.template as<cplx<T>>(),
                                                                       w.bhat64.template as<cplx<double>>(), 3 * nc);
      FDTD_CHECK(after_launch("to64_kernel"));
      return schur_cocg(w, zs);
    }
    if (o.solver != MOR_SOLVER_AUTO) return schur_krylov(w, zs, o.solver);
    const bool nc0 = noconv;
    const int it0 = max_iters;
    const double r0 = max_resid;
    FDTD_CHECK(schur_krylov(w, zs, MOR_SOLVER_CGS));
    if (!last_failed) return FDTD_OK;
    noconv = nc0; max_iters = it0; max_resid = r0;
    fallbacks += 1;
    return schur_krylov(w, zs, MOR_SOLVER_BICGSTAB);
  }

  // COCG with the gradient-corrected preconditioner inside a refinement loop:
  // x (FP64) starts at 0; each outer step forms the true residual
  // r = bhat - S x in FP64, stops when |r| <= tol |bhat| (Sec. IV-B's
  // criterion, on the FP64 residual), else solves S d = r with COCG in the
  // field type to a relative kInnerTol (FDTD_F32) and adds d to x.  With
  // FDTD_F64 fields the inner solve goes straight to the requested tolerance.
  // o.maxit caps the inner iterations of one shifted solve (all outer steps).
  static constexpr double kInnerTol = 1e-2;
  static constexpr int kMaxOuter = 8;
  static double inner_tol() {  // FDTDMOR_INNER_TOL overrides kInnerTol
    static const double t = [] {
      const char *e = getenv("FDTDMOR_INNER_TOL");
      const double v = e ? atof(e) : 0.0;
      return v > 0 && v < 1 ? v : kInnerTol;
    }();
    return t;
  }

  fdtd_status schur_cocg(Work<T> &w, const std::vector<std::complex<double>> &zs) {
    const int nb = (int)zs.size();
    const int64_t n3 = 3 * nc;
    std::vector<std::complex<double>> one(nb, 1.0), zz(zs);
    dim3 grid2(nblk, nb);
    OpArgs<T> ap = make_op<T>(g, o.dt0, zs, zz);    // e_from_h half: cz = z
    OpArgs<T> ah1 = make_op<T>(g, o.dt0, zs, one);  // h_from_e half: cz = 1
    cplx<T> *t = w.t.template as<cplx<T>>();
    const cplx<double> *bh = w.bhat64.template as<cplx<double>>();
    FDTD_CHECK(w.phi.alloc(sizeof(cplx<T>) * nb * nc, s));
    FDTD_CHECK(w.dN.alloc(sizeof(cplx<T>) * nb * nc, s));
    FDTD_CHECK(w.upd.alloc(sizeof(int) * kMaxRhs, s));
    if (!w.tickets.ptr) {
      FDTD_CHECK(w.tickets.alloc(sizeof(unsigned) * 2 * kMaxRhs, s));
      FDTD_CHECK_CUDA(cudaMemsetAsync(w.tickets.ptr, 0, sizeof(unsigned) * 2 * kMaxRhs, s));
    }
    unsigned *tk = w.tickets.template as<unsigned>();
    cplx<double> *x64 = w.x64.template as<cplx<double>>(), *t64 = w.t64.template as<cplx<double>>();
    cplx<T> *phi = w.phi.template as<cplx<T>>(), *dN = w.dN.template as<cplx<T>>();
    cplx<T> *P = w.P.template as<cplx<T>>(), *x = w.x.template as<cplx<T>>(), *rr = w.rr.template as<cplx<T>>();
    cplx<T> *zv = w.u.template as<cplx<T>>(), *p = w.p.template as<cplx<T>>(), *q = w.q.template as<cplx<T>>();
    CgsScal *sc = w.sc.template as<CgsScal>();
    double *part = w.partials.template as<double>();
    int *upd = w.upd.template as<int>();
    const int eblk = std::min(nblk, 152 * 8);
    dim3 gridE(eblk, nb);
    jacobi_kernel<T><<<grid2, MB, 0, s>>>(ap, P, n3);
    FDTD_CHECK(after_launch("jacobi_kernel"));
    cocg_dn_kernel<T><<<grid2, MB, 0, s>>>(ap, dN);
    FDTD_CHECK(after_launch("cocg_dn_kernel"));
    FDTD_CHECK_CUDA(cudaMemsetAsync(x64, 0, sizeof(cplx<double>) * nb * n3, s));
    const bool trace = getenv("FDTDMOR_TRACE") != nullptr;
    auto scal_on = [&](cudaStream_t st, int mode) -> fdtd_status {
      solver_scalars_kernel<<<1, 32 * nb, 0, st>>>(nb, nblk, part, sc, mode, -1.0, 0, 0);
      return after_launch("solver_scalars_kernel");
    };
    const int astride = (int)(sizeof(CgsScal) / sizeof(int));
    // one-pass Schur apply (FDTDMOR_SCHUR=pair selects the two-kernel form)
    const char *sch = getenv("FDTDMOR_SCHUR");
    const bool fused = !(sch && std::string(sch) == "pair");
    const int *act = reinterpret_cast<const int *>(reinterpret_cast<const char *>(sc) + offsetof(CgsScal, active));
    auto iteration = [&](cudaStream_t st) -> fdtd_status {
      cocg_update_p_kernel<T><<<gridE, MB, 0, st>>>(n3, sc, zv, p, n3);
      FDTD_CHECK(after_launch("cocg_update_p_kernel"));
      if (fused) {
        FDTD_CHECK((launch_schur_fused<T, true>(g, ap, nb, p, q, n3, sc, part, tk, st)));
      } else {
        h_from_e_kernel<T><<<grid2, MB, 0, st>>>(ah1, p, n3, nullptr, 0, nullptr, 0, t, n3, act, astride);
        FDTD_CHECK(after_launch("h_from_e_kernel"));
        e_from_h_kernel<T, EM_APPLY_VDOT><<<grid2, MB, 0, st>>>(ap, t, n3, p, n3, nullptr, 0, q, n3, nullptr, nullptr,
                                                                n3, sc, part, tk);
        FDTD_CHECK(after_launch("e_from_h_kernel"));
      }
      cocg_node_kernel<T, false><<<grid2, MB, 0, st>>>(ap, rr, q, n3, dN, phi, sc);
      FDTD_CHECK(after_launch("cocg_node_kernel"));
      cocg_edge_kernel<T, false><<<grid2, MB, 0, st>>>(ap, rr, q, x, p, phi, P, zv, n3, sc, part, tk + kMaxRhs);
      return after_launch("cocg_edge_kernel");
    };
    const int poll = 16;
    if (!cocg_graph && !graphs_off()) {
      if (!cap) FDTD_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      const int64_t before = fdtd_launch_count(0);
      FDTD_CHECK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      fdtd_status st = FDTD_OK;
      for (int k = 0; k < poll && st == FDTD_OK; ++k) st = iteration(cap);
      cocg_graph_launches = fdtd_launch_count(0) - before;
      add_launches(-cocg_graph_launches);  // captured, not launched
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cap, &graph);
      if (st != FDTD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(e, "COCG graph capture");
      const cudaError_t e2 = cudaGraphInstantiate(&cocg_graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e2 != cudaSuccess) { cocg_graph = nullptr; return cuda_fail(e2, "COCG graph instantiate"); }
    }
    std::vector<CgsScal> hsc(nb);
    std::vector<double> bn(nb, 0.0), rn(nb, 0.0);
    std::vector<int> used(nb, 0), capped(nb, 0), need(nb, 0);
    const bool f64 = sizeof(T) == 8;
    int outer = 0;
    for (;; ++outer) {
      // true residual in FP64 (x64 = 0 on the first pass: r = bhat)
      resid64_h_kernel<T><<<grid2, MB, 0, s>>>(ah1, x64, t64, n3);
      FDTD_CHECK(after_launch("resid64_h_kernel"));
      resid64_e_kernel<T><<<grid2, MB, 0, s>>>(ap, t64, x64, n3, bh, rr, part);
      FDTD_CHECK(after_launch("resid64_e_kernel"));
      solver_scalars_kernel<<<1, 32 * nb, 0, s>>>(nb, nblk, part, sc, SM_NORM, 1.0, 1, 0);
      FDTD_CHECK(after_launch("solver_scalars_kernel"));
      FDTD_CHECK_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(CgsScal) * nb, cudaMemcpyDeviceToHost, s));
      FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
      bool any = false;
      for (int b = 0; b < nb; ++b) {
        rn[b] = std::sqrt(std::max(hsc[b].rn2, 0.0));
        if (outer == 0) bn[b] = rn[b];
        need[b] = bn[b] > 0 && std::isfinite(rn[b]) && rn[b] > o.tol * bn[b] && !capped[b] && used[b] < o.maxit;
        any |= need[b] != 0;
      }
      if (trace) {
        fprintf(stderr, "[cocg] outer %d true residual", outer);
        for (int b = 0; b < nb; ++b) fprintf(stderr, " %.3e", bn[b] > 0 ? rn[b] / bn[b] : 0.0);
        fprintf(stderr, "\n");
      }
      if (!any || outer >= kMaxOuter) break;
      // inner solve S d = r for the right-hand sides still above tolerance
      for (int b = 0; b < nb; ++b) {
        CgsScal &c = hsc[b];
        c = CgsScal{};
        c.active = need[b];
        c.itol = f64 ? std::min(0.5, 0.5 * o.tol * bn[b] / std::max(rn[b], 1e-300))
                     : std::max(inner_tol(), std::min(0.5, 0.5 * o.tol * bn[b] / std::max(rn[b], 1e-300)));
        c.imaxit = std::max(1, o.maxit - used[b]);
      }
      FDTD_CHECK_CUDA(cudaMemcpyAsync(sc, hsc.data(), sizeof(CgsScal) * nb, cudaMemcpyHostToDevice, s));
      FDTD_CHECK_CUDA(cudaMemcpyAsync(upd, need.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
      FDTD_CHECK_CUDA(cudaMemsetAsync(x, 0, sizeof(cplx<T>) * nb * n3, s));
      FDTD_CHECK_CUDA(cudaMemsetAsync(p, 0, sizeof(cplx<T>) * nb * n3, s));
      cocg_node_kernel<T, true><<<grid2, MB, 0, s>>>(ap, rr, nullptr, n3, dN, phi, sc);
      FDTD_CHECK(after_launch("cocg_node_kernel"));
      cocg_edge_kernel<T, true><<<grid2, MB, 0, s>>>(ap, rr, nullptr, nullptr, nullptr, phi, P, zv, n3, sc, part,
                                                     nullptr);
      FDTD_CHECK(after_launch("cocg_edge_kernel"));
      FDTD_CHECK(scal_on(s, SM_INIT));
      for (int it = 0; it < o.maxit + poll; it += poll) {
        if (cocg_graph) {
          FDTD_CHECK_CUDA(cudaGraphLaunch(cocg_graph, s));
          add_launches(cocg_graph_launches);
        } else {
          for (int k = 0; k < poll; ++k) FDTD_CHECK(iteration(s));
        }
        FDTD_CHECK_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(CgsScal) * nb, cudaMemcpyDeviceToHost, s));
        FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
        bool act_any = false;
        for (auto &c : hsc) act_any |= c.active != 0;
        if (trace) {
          fprintf(stderr, "[cocg] it %d", it + poll);
          for (auto &c : hsc) fprintf(stderr, " %.3e%s", c.bn2 > 0 ? std::sqrt(c.rn2 / c.bn2) : 0.0, c.active ? "" : "*");
          fprintf(stderr, "\n");
        }
        if (!act_any) break;
      }
      for (int b = 0; b < nb; ++b) {
        if (!need[b]) continue;
        used[b] += hsc[b].iters;
        if (hsc[b].status != 0) capped[b] = 1;  // iteration cap or breakdown: keep x, stop refining
      }
      const int eblk2 = std::min(nblk, 152 * 8);
      acc64_kernel<T><<<dim3(eblk2, nb), MB, 0, s>>>(n3, upd, x, x64, n3);
      FDTD_CHECK(after_launch("acc64_kernel"));
    }
    outer_max = std::max(outer_max, outer);
    last_failed = false;
    rhs_failed.assign(nb, 0);
    rhs_iters = used;
    rhs_resid.assign(nb, 0.0);
    for (int b = 0; b < nb; ++b) {
      max_iters = std::max(max_iters, used[b]);
      if (bn[b] > 0) rhs_resid[b] = rn[b] / bn[b];
      if (bn[b] > 0) max_resid = std::max(max_resid, rn[b] / bn[b]);
      if (bn[b] > 0 && !(rn[b] <= o.tol * bn[b])) { noconv = true; last_failed = true; rhs_failed[b] = 1; }
    }
    from64_kernel<T><<<dim3(eblk, nb), MB, 0, s>>>(n3, x64, n3, x, n3);
    return after_launch("from64_kernel");
  }

  fdtd_status schur_krylov(Work<T> &w, const std::vector<std::complex<double>> &zs, int solver) {
    const int nb = (int)zs.size();
    const int64_t n3 = 3 * nc;
    std::vector<std::complex<double>> one(nb, 1.0), zz(zs);
    dim3 grid2(nblk, nb);
    cplx<T> *t = w.t.template as<cplx<T>>();
    // S x = a11 x + z curlH(curlE(x)/a22): the curlE half carries no factor,
    // the curlH half carries z.
    OpArgs<T> ap = make_op<T>(g, o.dt0, zs, zz);       // e_from_h half: cz = z
    OpArgs<T> ah1 = make_op<T>(g, o.dt0, zs, one);     // h_from_e half: cz = 1
    CgsScal *sc = w.sc.template as<CgsScal>();
    std::vector<CgsScal> hsc(nb);
    for (auto &x : hsc) { x = CgsScal{}; x.active = 1; }
    const bool trace = getenv("FDTDMOR_TRACE") != nullptr;
    FDTD_CHECK_CUDA(cudaMemcpyAsync(sc, hsc.data(), sizeof(CgsScal) * nb, cudaMemcpyHostToDevice, s));
    cplx<T> *P = w.P.template as<cplx<T>>(), *x = w.x.template as<cplx<T>>(), *rr = w.rr.template as<cplx<T>>();
    cplx<T> *rt = w.rt.template as<cplx<T>>(), *u = w.u.template as<cplx<T>>(), *p = w.p.template as<cplx<T>>();
    cplx<T> *q = w.q.template as<cplx<T>>(), *vv = w.vv.template as<cplx<T>>();
    double *part = w.partials.template as<double>();
    jacobi_kernel<T><<<grid2, MB, 0, s>>>(ap, P, n3);
    FDTD_CHECK(after_launch("jacobi_kernel"));
    const int eblk = std::min(nblk, 152 * 8);
    dim3 gridE(eblk, nb);
    cgs_init_kernel<T><<<gridE, MB, 0, s>>>(n3, w.bhat.template as<cplx<T>>(), rr, rt, x, p, q, n3, part);
    FDTD_CHECK(after_launch("cgs_init_kernel"));
    FDTD_CHECK_CUDA(cudaMemsetAsync(vv, 0, sizeof(cplx<T>) * nb * n3, s));
    solver_scalars_kernel<<<1, 32 * nb, 0, s>>>(nb, eblk, part, sc, SM_INIT, o.tol, o.maxit, kMaxRestarts);
    FDTD_CHECK(after_launch("solver_scalars_kernel"));
    auto scal_on = [&](cudaStream_t st, int mode, int nbk) -> fdtd_status {
      solver_scalars_kernel<<<1, 32 * nb, 0, st>>>(nb, nbk, part, sc, mode, o.tol, o.maxit, kMaxRestarts);
      return after_launch("solver_scalars_kernel");
    };
    auto scal = [&](int mode, int nbk) { return scal_on(s, mode, nbk); };
    const bool bicg = solver == MOR_SOLVER_BICGSTAB;
    cplx<T> *bh_ = w.bhat.template as<cplx<T>>();
    // One iteration; converged right-hand sides are frozen by the device-side
    // scalars, so the iterations need no host decision and are issued in
    // blocks of `poll` as replays of one captured graph.
    auto iteration = [&](cudaStream_t st) -> fdtd_status {
      if (!bicg) {
        // conjugate gradient squared (right-preconditioned, P = Jacobi)
        // u = r + beta q; p = u + beta (q + beta p)
        cgs_update1_kernel<T><<<gridE, MB, 0, st>>>(n3, sc, rr, q, p, u, n3);
        FDTD_CHECK(after_launch("cgs_update1_kernel"));
        // v = S P p, sigma = rt^H v
        h_from_e_kernel<T><<<grid2, MB, 0, st>>>(ah1, p, n3, P, n3, nullptr, 0, t, n3, nullptr);
        FDTD_CHECK(after_launch("h_from_e_kernel"));
        e_from_h_kernel<T, EM_APPLY_DOT><<<grid2, MB, 0, st>>>(ap, t, n3, p, n3, P, n3, vv, n3, rt, nullptr, n3, sc, part);
        FDTD_CHECK(after_launch("e_from_h_kernel"));
        FDTD_CHECK(scal_on(st, SM_ALPHA, nblk));
        // q = u - alpha v; w = u + q (into vv); x += alpha P w
        cgs_update2_kernel<T><<<gridE, MB, 0, st>>>(n3, sc, u, vv, q, x, P, n3);
        FDTD_CHECK(after_launch("cgs_update2_kernel"));
        // r -= alpha S P w; rho = rt^H r; |r|^2
        h_from_e_kernel<T><<<grid2, MB, 0, st>>>(ah1, vv, n3, P, n3, nullptr, 0, t, n3, nullptr);
        FDTD_CHECK(after_launch("h_from_e_kernel"));
        e_from_h_kernel<T, EM_APPLY_RUPDATE><<<grid2, MB, 0, st>>>(ap, t, n3, vv, n3, P, n3, nullptr, 0, rt, rr, n3, sc, part);
        FDTD_CHECK(after_launch("e_from_h_kernel"));
        return scal_on(st, SM_CGS_RHO, nblk);
      }
      // BiCGSTAB (right-preconditioned, P = Jacobi); p in p, v in vv, s in u, t in q
      bicg_update_p_kernel<T><<<gridE, MB, 0, st>>>(n3, sc, rr, vv, p, n3);
      FDTD_CHECK(after_launch("bicg_update_p_kernel"));
      h_from_e_kernel<T><<<grid2, MB, 0, st>>>(ah1, p, n3, P, n3, nullptr, 0, t, n3, nullptr);
      FDTD_CHECK(after_launch("h_from_e_kernel"));
      e_from_h_kernel<T, EM_APPLY_DOT><<<grid2, MB, 0, st>>>(ap, t, n3, p, n3, P, n3, vv, n3, rt, nullptr, n3, sc, part);
      FDTD_CHECK(after_launch("e_from_h_kernel"));
      FDTD_CHECK(scal_on(st, SM_ALPHA, nblk));
      bicg_update_s_kernel<T><<<gridE, MB, 0, st>>>(n3, sc, rr, vv, u, n3);
      FDTD_CHECK(after_launch("bicg_update_s_kernel"));
      h_from_e_kernel<T><<<grid2, MB, 0, st>>>(ah1, u, n3, P, n3, nullptr, 0, t, n3, nullptr);
      FDTD_CHECK(after_launch("h_from_e_kernel"));
      // t = S P s with partials s^H t and |t|^2
      e_from_h_kernel<T, EM_APPLY_DOT><<<grid2, MB, 0, st>>>(ap, t, n3, u, n3, P, n3, q, n3, u, nullptr, n3, sc, part);
      FDTD_CHECK(after_launch("e_from_h_kernel"));
      FDTD_CHECK(scal_on(st, SM_OMEGA, nblk));
      bicg_update_xr_kernel<T><<<gridE, MB, 0, st>>>(n3, sc, P, p, u, q, rt, x, rr, n3, part);
      FDTD_CHECK(after_launch("bicg_update_xr_kernel"));
      return scal_on(st, SM_BICG_RHO, eblk);
    };
    const int poll = 16;
    cudaGraphExec_t block = nullptr;
    int64_t block_launches = 0;
    if (!graphs_off()) {
      if (!cap) FDTD_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      const int64_t before = fdtd_launch_count(0);
      FDTD_CHECK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      fdtd_status st = FDTD_OK;
      for (int k = 0; k < poll && st == FDTD_OK; ++k) st = iteration(cap);
      block_launches = fdtd_launch_count(0) - before;
      add_launches(-block_launches);  // captured, not launched
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cap, &graph);
      if (st != FDTD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(e, "solver graph capture");
      const cudaError_t e2 = cudaGraphInstantiate(&block, graph, 0);
      cudaGraphDestroy(graph);
      if (e2 != cudaSuccess) return cuda_fail(e2, "solver graph instantiate");
    }
    struct GraphGuard {
      cudaGraphExec_t &g;
      ~GraphGuard() { if (g) cudaGraphExecDestroy(g); }
    } guard{block};
    int it = 0;
    for (int round = 0; round <= kMaxRestarts; ++round) {
      for (; it < o.maxit + poll; it += poll) {
        if (block) {
          FDTD_CHECK_CUDA(cudaGraphLaunch(block, s));
          add_launches(block_launches);
        } else {
          for (int k = 0; k < poll; ++k) FDTD_CHECK(iteration(s));
        }
        FDTD_CHECK_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(CgsScal) * nb, cudaMemcpyDeviceToHost, s));
        FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
        bool any = false;
        for (auto &x2 : hsc) any |= x2.active != 0;
        if (trace) {
          fprintf(stderr, "[%s] it %d", bicg ? "bicgstab" : "cgs", it + poll);
          for (auto &x2 : hsc) fprintf(stderr, " %.3e%s", x2.bn2 > 0 ? std::sqrt(x2.rn2 / x2.bn2) : 0.0, x2.active ? "" : "*");
          fprintf(stderr, "\n");
        }
        if (!any) { it += poll; break; }
      }
      // verify with the true residual b - S x; restart the ones above tolerance
      h_from_e_kernel<T><<<grid2, MB, 0, s>>>(ah1, x, n3, nullptr, 0, nullptr, 0, t, n3, nullptr);
      FDTD_CHECK(after_launch("h_from_e_kernel"));
      e_from_h_kernel<T, EM_RESID><<<grid2, MB, 0, s>>>(ap, t, n3, x, n3, nullptr, 0, rr, n3, bh_, nullptr, n3, sc, part);
      FDTD_CHECK(after_launch("e_from_h_kernel"));
      FDTD_CHECK(scal(SM_VERIFY, nblk));
      FDTD_CHECK_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(CgsScal) * nb, cudaMemcpyDeviceToHost, s));
      FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
      bool any = false;
      for (auto &x2 : hsc) any |= x2.active != 0;
      if (trace) {
        fprintf(stderr, "[verify] round %d true residual", round);
        for (auto &x2 : hsc) fprintf(stderr, " %.3e%s", x2.bn2 > 0 ? std::sqrt(x2.rn2 / x2.bn2) : 0.0, x2.active ? " (restart)" : "");
        fprintf(stderr, "\n");
      }
      if (!any) break;
      solver_restart_kernel<T><<<gridE, MB, 0, s>>>(n3, sc, rr, rt, p, q, n3);
      FDTD_CHECK(after_launch("solver_restart_kernel"));
      if (bicg) FDTD_CHECK_CUDA(cudaMemsetAsync(vv, 0, sizeof(cplx<T>) * nb * n3, s));
    }
    FDTD_CHECK_CUDA(cudaMemcpyAsync(hsc.data(), sc, sizeof(CgsScal) * nb, cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    last_failed = false;
    rhs_failed.assign(nb, 0);
    rhs_iters.assign(nb, 0);
    rhs_resid.assign(nb, 0.0);
    for (int b = 0; b < nb; ++b) {
      const CgsScal &x2 = hsc[b];
      rhs_iters[b] = x2.iters;
      if (x2.bn2 > 0) rhs_resid[b] = std::sqrt(x2.rn2 / x2.bn2);
      max_iters = std::max(max_iters, x2.iters);
      if (x2.bn2 > 0) max_resid = std::max(max_resid, std::sqrt(x2.rn2 / x2.bn2));
      if (x2.status != 0 || x2.active) { noconv = true; last_failed = true; rhs_failed[b] = 1; }
    }
    return FDTD_OK;
  }

  // Euclidean norm of vec (FP64 partial sums; synchronises).
  template <typename V>
  fdtd_status norm(Work<T> &w, const V *vec, int64_t len, double &out) {
    const int dblk = (int)((len + 256 * 8 - 1) / (256 * 8));
    FDTD_CHECK(w.dpart.alloc(sizeof(double) * 2 * (kMaxDots + 1) * dblk, s));
    double *dp = w.dpart.template as<double>();
    double *h = w.dots.template as<double>();
    multidot_kernel<T, V><<<dblk, 256, 0, s>>>(len, vec, 0, 1, vec, dp);
    FDTD_CHECK(after_launch("multidot_kernel"));
    reduce_partials_kernel<<<2, 256, 0, s>>>(2, dblk, dp, h);
    FDTD_CHECK(after_launch("reduce_partials_kernel"));
    double hh[2];
    FDTD_CHECK_CUDA(cudaMemcpyAsync(hh, h, sizeof(hh), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    out = std::sqrt(std::max(hh[0], 0.0));
    return FDTD_OK;
  }

  // Gram-Schmidt of vec (len) against Q[0..nq) (stride qstride), two passes,
  // returns the norm before (n0) and after (n1) via host sync.
  template <typename V>
  fdtd_status cgs2(Work<T> &w, const V *Q, int64_t qstride, int nq, V *vec, int64_t len, double &n0,
                   double &n1, int passes = 2) {
    const int dblk = (int)((len + 256 * 8 - 1) / (256 * 8));
    FDTD_CHECK(w.dpart.alloc(sizeof(double) * 2 * (kMaxDots + 1) * dblk, s));
    double *dp = w.dpart.template as<double>();
    double *h = w.dots.template as<double>();
    auto norm = [&](double &out) -> fdtd_status {
      multidot_kernel<T, V><<<dblk, 256, 0, s>>>(len, vec, 0, 1, vec, dp);
      FDTD_CHECK(after_launch("multidot_kernel"));
      reduce_partials_kernel<<<2, 256, 0, s>>>(2, dblk, dp, h);
      FDTD_CHECK(after_launch("reduce_partials_kernel"));
      double hh[2];
      FDTD_CHECK_CUDA(cudaMemcpyAsync(hh, h, sizeof(hh), cudaMemcpyDeviceToHost, s));
      FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
      out = std::sqrt(std::max(hh[0], 0.0));
      return FDTD_OK;
    };
    FDTD_CHECK(norm(n0));
    for (int pass = 0; pass < passes && nq > 0; ++pass) {
      for (int c0 = 0; c0 < nq; c0 += kMaxDots) {
        const int cn = std::min(kMaxDots, nq - c0);
        multidot_kernel<T, V><<<dblk, 256, 0, s>>>(len, Q + c0 * qstride, qstride, cn, vec, dp);
        FDTD_CHECK(after_launch("multidot_kernel"));
        reduce_partials_kernel<<<2 * cn, 256, 0, s>>>(2 * cn, dblk, dp, h);
        FDTD_CHECK(after_launch("reduce_partials_kernel"));
        multiaxpy_kernel<T, V><<<std::min<int64_t>((len + 255) / 256, 152 * 16), 256, 0, s>>>(len, Q + c0 * qstride, qstride, cn, h, vec);
        FDTD_CHECK(after_launch("multiaxpy_kernel"));
      }
    }
    FDTD_CHECK(norm(n1));
    return FDTD_OK;
  }
};


// A4 on its own: S(z_b) x_b = b_b for nb given right-hand sides (b, x: device
// [nb][3 nc] complex in the grid's type).
template <typename T>
static fdtd_status shifted_solve_t(fdtd_grid *g, const mor_opts &o, const std::vector<std::complex<double>> &zs,
                                   const void *b, void *x, int *iters, double *resid, cudaStream_t s) {
  FDTD_CHECK(ensure_edge_props(g, s));
  const int nb = (int)zs.size();
  const int64_t n3 = 3 * g->nc;
  BasisBuilder<T> bb(g, o, s);
  Work<T> w;
  w.nb = nb;
  const size_t cb = sizeof(cplx<T>);
  struct Rel {
    Work<T> &w;
    cudaStream_t s;
    ~Rel() {
      cudaStreamSynchronize(s);
      for (DevBuf *d : {&w.bhat, &w.P, &w.x, &w.rr, &w.rt, &w.u, &w.p, &w.q, &w.vv, &w.t, &w.partials, &w.sc,
                        &w.x64, &w.t64, &w.phi, &w.dN, &w.upd, &w.tickets, &w.bhat64, &w.r2_64})
        d->release(s);
    }
  } rel{w, s};
  for (DevBuf *d : {&w.bhat, &w.P, &w.x, &w.rr, &w.rt, &w.u, &w.p, &w.q, &w.vv, &w.t}) FDTD_CHECK(d->alloc(cb * nb * n3, s));
  FDTD_CHECK(w.partials.alloc(sizeof(double) * 3 * nb * (size_t)std::max(bb.nblk, 152 * 16), s));
  FDTD_CHECK(w.sc.alloc(sizeof(CgsScal) * nb, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(w.bhat.ptr, b, cb * nb * n3, cudaMemcpyDefault, s));
  FDTD_CHECK(bb.schur_solve(w, zs));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(x, w.x.ptr, cb * nb * n3, cudaMemcpyDefault, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < nb; ++i) {
    if (iters) iters[i] = i < (int)bb.rhs_iters.size() ? bb.rhs_iters[i] : 0;
    if (resid) resid[i] = i < (int)bb.rhs_resid.size() ? bb.rhs_resid[i] : 0.0;
  }
  return bb.noconv ? FDTD_ENOCONV : FDTD_OK;
}

template <typename T>
static fdtd_status build_basis_t(fdtd_grid *g, const mor_opts &o, cudaStream_t s, mor_basis *B) {
  FDTD_CHECK(ensure_edge_props(g, s));
  const int m = (int)g->ports.size();
  FDTD_REQUIRE(m >= 1, "mor_build_basis: the grid has no sources (B has no columns)");
  // expansion points, l = 0..L (conjugates implied)
  std::vector<std::complex<double>> pts;
  if (o.include_center) {
    for (int l = 0; l <= o.L; ++l) {
      const double ang = 2 * kPi * (o.L ? (double)l / o.L : 0.0) * o.fmax * o.dt0;
      pts.push_back(l == 0 ? std::complex<double>(o.M, 0) : std::polar(o.M, ang));
    }
  } else {
    pts.push_back(std::polar(o.M, 2 * kPi * o.fmax * o.dt0));
  }
  int nreal = 0;
  for (auto &z : pts) nreal += (z.imag() == 0.0) ? 1 : 2;
  const int k = std::max(1, o.q / (nreal * m));
  const int np = (int)pts.size();
  const int nb = np * m;
  FDTD_REQUIRE(nb <= kMaxRhs, "too many expansion points x ports (max %d)", kMaxRhs);
  FDTD_REQUIRE(k * m <= kMaxDots * 64, "chain too long");
  const int64_t nc = g->nc, n3 = 3 * nc, n6 = 6 * nc;
  BasisBuilder<T> bb(g, o, s);
  Work<T> w;
  w.nb = nb;
  const size_t cb = sizeof(cplx<T>);
  FDTD_CHECK(w.v.alloc(cb * nb * n6, s));
  FDTD_CHECK(w.r.alloc(cb * nb * n6, s));
  for (DevBuf *d : {&w.bhat, &w.P, &w.x, &w.rr, &w.rt, &w.u, &w.p, &w.q, &w.vv, &w.t}) FDTD_CHECK(d->alloc(cb * nb * n3, s));
  // one partial triple per CTA of the widest reducing kernel (operator: one
  // CTA per MB cells; vector updates: up to 16 CTAs per SM)
  FDTD_CHECK(w.partials.alloc(sizeof(double) * 3 * nb * (size_t)std::max(bb.nblk, 152 * 16), s));
  FDTD_CHECK(w.sc.alloc(sizeof(CgsScal) * nb, s));
  FDTD_CHECK(w.dots.alloc(sizeof(double) * 2 * (kMaxDots + 1), s));
  // chains: per point, k*m complex vectors of 6nc
  const int clen = k * m;
  DevBuf chains;
  FDTD_CHECK(chains.alloc(cb * (size_t)np * clen * n6, s));
  cplx<T> *Qc = chains.as<cplx<T>>();
  std::vector<int> ccount(np, 0);
  DevBuf xs;
  FDTD_CHECK(xs.alloc(cb * nb * n6, s));
  cplx<T> *X = xs.as<cplx<T>>();
  std::vector<std::complex<double>> zs(nb);
  for (int pidx = 0; pidx < np; ++pidx)
    for (int c = 0; c < m; ++c) zs[pidx * m + c] = pts[pidx];
  // v_0 = A^{-1} B: right-hand side (R+F)-free, r = [B_E column / V_e; 0]
  {
    // B column in the per-volume form: -w at the source edges
    std::vector<cplx<T>> host((size_t)nb * n6);
    for (int b = 0; b < nb; ++b) {
      const HostPort &hp = g->ports[b % m];
      for (size_t e = 0; e < hp.cell.size(); ++e) {
        cplx<T> &dst = host[(size_t)b * n6 + (size_t)hp.comp * nc + hp.cell[e]];
        dst = dst + cplx<T>((T)(-hp.w[e]));
      }
    }
    FDTD_CHECK_CUDA(cudaMemcpyAsync(w.r.ptr, host.data(), cb * host.size(), cudaMemcpyHostToDevice, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  // dead source edges (PEC) must carry no right-hand side: r1 is masked by
  // e_from_h (A = r1 only on live edges), so nothing else to do here.
  // a chain whose shifted solve failed ends there: its vector does not enter
  // the pool, and its later right-hand sides are zero (skipped by the solver)
  std::vector<int> dead(nb, 0);
  for (int j = 0; j < k; ++j) {
    for (int b = 0; b < nb; ++b)
      if (dead[b]) {
        cplx<T> *src = j == 0 ? w.r.template as<cplx<T>>() : w.v.template as<cplx<T>>();
        FDTD_CHECK_CUDA(cudaMemsetAsync(src + (size_t)b * n6, 0, cb * n6, s));
      }
    FDTD_CHECK(bb.solve(w, zs, j == 0, w.v.template as<cplx<T>>(), X));
    for (int b = 0; b < nb; ++b) dead[b] |= bb.rhs_failed.empty() ? 0 : bb.rhs_failed[b];
    // block Arnoldi per point: each new column against the whole chain
    for (int c = 0; c < m; ++c) {
      for (int pidx = 0; pidx < np; ++pidx) {
        const int b = pidx * m + c;
        if (dead[b]) continue;
        cplx<T> *vec = X + (size_t)b * n6;
        cplx<T> *chain = Qc + (size_t)pidx * clen * n6;
        double n0, n1;
        FDTD_CHECK(bb.cgs2(w, chain, n6, ccount[pidx], vec, n6, n0, n1));
        cplx<T> *dst = chain + (size_t)ccount[pidx] * n6;
        if (n1 > 0 && std::isfinite(n1)) {
          scale_copy_kernel<cplx<T>, T><<<std::min<int64_t>((n6 + 255) / 256, 152 * 16), 256, 0, s>>>(n6, vec, dst, (T)(1.0 / n1));
          FDTD_CHECK(after_launch("scale_copy_kernel"));
          // next moment starts from the orthonormal vector
          FDTD_CHECK_CUDA(cudaMemcpyAsync(w.v.template as<cplx<T>>() + (size_t)b * n6, dst, cb * n6, cudaMemcpyDeviceToDevice, s));
          ccount[pidx] += 1;
        } else {
          FDTD_CHECK_CUDA(cudaMemcpyAsync(w.v.template as<cplx<T>>() + (size_t)b * n6, vec, cb * n6, cudaMemcpyDeviceToDevice, s));
        }
      }
    }
  }
  // SPRIM split + CGS2 with deflation, pool order: point, chain order, Re then Im
  std::vector<std::pair<int, int>> pool;  // (point, chain index)
  int qmax = 0;
  for (int pidx = 0; pidx < np; ++pidx) {
    const int parts = pts[pidx].imag() == 0.0 ? 1 : 2;
    qmax += parts * ccount[pidx];
  }
  FDTD_CHECK(B->V1.alloc(sizeof(T) * std::max(1, qmax) * n3, s));
  FDTD_CHECK(B->V2.alloc(sizeof(T) * std::max(1, qmax) * n3, s));
  DevBuf tmp;
  FDTD_CHECK(tmp.alloc(sizeof(T) * n3, s));
  T *wv = tmp.as<T>();
  B->orth = sizeof(T) == 4 ? o.orth : MOR_ORTH_NATIVE;
  if (B->orth != MOR_ORTH_NATIVE) {
    // Block CGS2 with a tensor-core first pass: pool vectors in blocks of
    // kBlkMax; the first pass's coefficients H = V^T W come from tcgen05 Gram
    // products (TF32 or BF16 inputs, FP32 accumulation, FP64 chunk sums)
    // against a K-major copy of V in the operand type and W -= V H runs on the
    // CUDA cores; the second pass is the FP32 one; the block's vectors are
    // then orthonormalised among themselves by CGS2 with the usual deflation
    // test against their norm before the block projection.
    const bool bf16 = B->orth == MOR_ORTH_BF16;
    const int es = bf16 ? 2 : 4;
    const int64_t n_pad = std::max<int64_t>(64, (n3 + 63) / 64 * 64);
    DevBuf Vp, Wb, Wp, Hd, part;
    struct Rel {
      std::vector<DevBuf *> b;
      cudaStream_t s;
      ~Rel() { for (auto *x : b) x->release(s); }
    } rel{{&Vp, &Wb, &Wp, &Hd, &part}, s};
    FDTD_CHECK(Vp.alloc((size_t)std::max(1, qmax) * n_pad * es, s));
    FDTD_CHECK(Wb.alloc((size_t)kBlkMax * n_pad * sizeof(T), s));
    if (bf16) FDTD_CHECK(Wp.alloc((size_t)kBlkMax * n_pad * es, s));
    FDTD_CHECK(Hd.alloc((size_t)std::max(1, qmax) * kBlkMax * sizeof(double), s));
    DevBuf tflag;  // set by a tensor-core pipeline wait that gave up
    rel.b.push_back(&tflag);
    FDTD_CHECK(tflag.alloc(sizeof(unsigned), s));
    FDTD_CHECK_CUDA(cudaMemsetAsync(tflag.ptr, 0, sizeof(unsigned), s));
    unsigned *err = tflag.as<unsigned>();
    for (int half = 0; half < 2; ++half) {
      T *V = (half == 0 ? B->V1 : B->V2).as<T>();
      std::vector<std::pair<const cplx<T> *, int>> items;
      for (int pidx = 0; pidx < np; ++pidx) {
        const int parts = pts[pidx].imag() == 0.0 ? 1 : 2;
        for (int c = 0; c < ccount[pidx]; ++c)
          for (int part_ = 0; part_ < parts; ++part_)
            items.push_back({Qc + ((size_t)pidx * clen + c) * n6 + (half ? n3 : 0), part_});
      }
      int qc = 0;
      for (size_t p0 = 0; p0 < items.size(); p0 += kBlkMax) {
        const int nbk = (int)std::min<size_t>(kBlkMax, items.size() - p0);
        T *W = Wb.as<T>();
        FDTD_CHECK_CUDA(cudaMemsetAsync(W, 0, (size_t)kBlkMax * n_pad * sizeof(T), s));
        std::vector<double> n0(nbk);
        for (int c = 0; c < nbk; ++c) {
          take_part_kernel<T><<<std::min<int64_t>((n3 + 255) / 256, 152 * 16), 256, 0, s>>>(
              n3, items[p0 + c].first, items[p0 + c].second, W + (size_t)c * n_pad);
          FDTD_CHECK(after_launch("take_part_kernel"));
          FDTD_CHECK(bb.norm(w, W + (size_t)c * n_pad, n3, n0[c]));
        }
        if (qc > 0) {
          // first pass: coefficients on the tensor cores
          const void *Bop = W;
          if (bf16) {
            FDTD_CHECK(gram_pack(s, true, n3, n_pad, reinterpret_cast<const float *>(W), n_pad, nbk, nullptr, Wp.ptr));
            Bop = Wp.ptr;
          }
          FDTD_CHECK(gram_tensor_kmajor(s, bf16, n_pad, Vp.ptr, n_pad, qc, Bop, n_pad, nbk, Hd.as<double>(), err, part));
          const int ablk = (int)std::min<int64_t>((n3 + 255) / 256, 152 * 8);
          const size_t hsm = sizeof(float) * qc * kBlkMax;
          FDTD_REQUIRE(hsm <= 227 * 1024, "mor_build_basis: too many basis columns for the block update");
          if (hsm > 48 * 1024)
            FDTD_CHECK_CUDA(cudaFuncSetAttribute(block_axpy_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)hsm));
          block_axpy_kernel<T><<<ablk, 256, hsm, s>>>(n3, V, n3, qc, Hd.as<double>(), nbk, W, n_pad);
          FDTD_CHECK(after_launch("block_axpy_kernel"));
        }
        const int qb0 = qc;
        for (int c = 0; c < nbk; ++c) {
          T *wc = W + (size_t)c * n_pad;
          // FP32 passes with FP64 dot sums against the columns before the
          // block restore orthogonality to the field precision (the
          // cancellation of nearly dependent Krylov vectors magnifies the
          // first pass's TF32 / BF16 coefficient error); a pass that cancels
          // more than half the norm is repeated (the "twice is enough" test)
          for (int rep = 0; rep < 3 && qb0 > 0; ++rep) {
            double a0, a1;
            FDTD_CHECK(bb.cgs2(w, V, n3, qb0, wc, n3, a0, a1, 1));
            if (a1 >= 0.5 * a0) break;
          }
          double m0, n1;
          FDTD_CHECK(bb.cgs2(w, V + (size_t)qb0 * n3, n3, qc - qb0, wc, n3, m0, n1));
          // a strong cancellation against the block's own columns re-exposes
          // their small error along the earlier columns: one more FP32 pass
          // against all columns
          for (int rep = 0; rep < 2 && n1 < 0.5 * m0 && qc > 0; ++rep) {
            double a0;
            FDTD_CHECK(bb.cgs2(w, V, n3, qc, wc, n3, a0, n1, 1));
            m0 = a0;
          }
          if (n0[c] > 0 && n1 >= o.defl_tol * n0[c]) {
            scale_copy_kernel<T, T><<<std::min<int64_t>((n3 + 255) / 256, 152 * 16), 256, 0, s>>>(
                n3, wc, V + (size_t)qc * n3, (T)(1.0 / n1));
            FDTD_CHECK(after_launch("scale_copy_kernel"));
            FDTD_CHECK(gram_pack(s, bf16, n3, n_pad, reinterpret_cast<const float *>(V + (size_t)qc * n3), n3, 1, nullptr,
                                 static_cast<char *>(Vp.ptr) + (size_t)qc * n_pad * es));
            ++qc;
          }
        }
      }
      (half == 0 ? B->q1 : B->q2) = qc;
    }
    unsigned hflag = 0;
    FDTD_CHECK_CUDA(cudaMemcpyAsync(&hflag, err, sizeof(hflag), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    FDTD_REQUIRE_STATUS(hflag == 0, FDTD_ETIMEOUT, "mor_build_basis: a bounded tensor-core wait gave up");
  }
  for (int half = 0; half < 2 && B->orth == MOR_ORTH_NATIVE; ++half) {
    T *V = (half == 0 ? B->V1 : B->V2).as<T>();
    int qc = 0;
    for (int pidx = 0; pidx < np; ++pidx) {
      const int parts = pts[pidx].imag() == 0.0 ? 1 : 2;
      for (int c = 0; c < ccount[pidx]; ++c) {
        for (int part = 0; part < parts; ++part) {
          const cplx<T> *src = Qc + ((size_t)pidx * clen + c) * n6 + (half ? n3 : 0);
          take_part_kernel<T><<<std::min<int64_t>((n3 + 255) / 256, 152 * 16), 256, 0, s>>>(n3, src, part, wv);
          FDTD_CHECK(after_launch("take_part_kernel"));
          double n0, n1;
          FDTD_CHECK(bb.cgs2(w, V, n3, qc, wv, n3, n0, n1));
          if (n0 > 0 && n1 >= o.defl_tol * n0) {
            scale_copy_kernel<T, T><<<std::min<int64_t>((n3 + 255) / 256, 152 * 16), 256, 0, s>>>(n3, wv, V + (size_t)qc * n3, (T)(1.0 / n1));
            FDTD_CHECK(after_launch("scale_copy_kernel"));
            ++qc;
          }
        }
      }
    }
    (half == 0 ? B->q1 : B->q2) = qc;
  }
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  for (DevBuf *d : {&w.v, &w.r, &w.bhat, &w.P, &w.x, &w.rr, &w.rt, &w.u, &w.p, &w.q, &w.vv, &w.t, &w.partials, &w.sc,
                    &w.dots, &w.dpart, &w.x64, &w.t64, &w.phi, &w.dN, &w.upd, &w.tickets, &w.bhat64, &w.r2_64,
                    &chains, &xs, &tmp})
    d->release(s);
  B->max_iters = bb.max_iters;
  B->max_resid = bb.max_resid;
  return bb.noconv ? FDTD_ENOCONV : FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status mor_opts_default(mor_opts *o) {
  FDTD_REQUIRE(o, "mor_opts_default: NULL");
  o->q = 0; o->L = 2; o->M = 1.1; o->fmax = 0; o->dt0 = 0; o->include_center = 1;
  o->tol = 1e-4; o->maxit = 20000; o->defl_tol = 1e-8; o->orth = MOR_ORTH_TF32;
  o->solver = MOR_SOLVER_AUTO;
  return FDTD_OK;
}

fdtd_status mor_build_basis(fdtd_grid *g, const mor_opts *o, fdtd_stream_t stream, mor_basis **out) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && o && out, "mor_build_basis: NULL argument");
  *out = nullptr;
  FDTD_REQUIRE(o->q >= 1 && o->L >= 0 && o->M > 0 && o->dt0 > 0 && o->tol > 0 && o->maxit >= 1,
               "mor_build_basis: need q >= 1, L >= 0, M > 0, dt0 > 0, tol > 0, maxit >= 1");
  FDTD_REQUIRE(o->defl_tol >= 0 && o->defl_tol < 1, "defl_tol must be in [0, 1)");
  FDTD_REQUIRE(o->include_center || o->fmax > 0, "the pair of points needs fmax > 0");
  cudaStream_t s = (cudaStream_t)stream;
  mor_basis *B = new mor_basis();
  B->n3 = 3 * g->nc;
  B->elem = g->elem;
  B->prec = g->prec;
  B->stream = s;
  fdtd_status st = g->prec == FDTD_F64 ? build_basis_t<double>(g, *o, s, B) : build_basis_t<float>(g, *o, s, B);
  if (st != FDTD_OK && st != FDTD_ENOCONV) {
    mor_basis_destroy(B);
    return st;
  }
  *out = B;
  if (st == FDTD_ENOCONV) set_error("a shifted solve reached maxit (worst relative residual %.3e)", B->max_resid);
  return st;
}

fdtd_status mor_shifted_solve(fdtd_grid *g, const mor_opts *o, int nb, const double *z, const void *b, void *x,
                              int *iters, double *resid, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && o && z && b && x, "mor_shifted_solve: NULL argument");
  FDTD_REQUIRE(nb >= 1 && nb <= kMaxRhs, "mor_shifted_solve: nb must be 1..%d", kMaxRhs);
  FDTD_REQUIRE(o->dt0 > 0 && o->tol > 0 && o->maxit >= 1, "mor_shifted_solve: need dt0 > 0, tol > 0, maxit >= 1");
  std::vector<std::complex<double>> zs(nb);
  for (int i = 0; i < nb; ++i) zs[i] = std::complex<double>(z[2 * i], z[2 * i + 1]);
  cudaStream_t s = (cudaStream_t)stream;
  const fdtd_status st = g->prec == FDTD_F64 ? shifted_solve_t<double>(g, *o, zs, b, x, iters, resid, s)
                                             : shifted_solve_t<float>(g, *o, zs, b, x, iters, resid, s);
  if (st == FDTD_ENOCONV) set_error("mor_shifted_solve: a right-hand side missed tol");
  return st;
}

fdtd_status mor_basis_info(const mor_basis *b, int *q1, int *q2, int *max_iters, double *max_resid) {
  FDTD_REQUIRE(b, "mor_basis_info: NULL basis");
  if (q1) *q1 = b->q1;
  if (q2) *q2 = b->q2;
  if (max_iters) *max_iters = b->max_iters;
  if (max_resid) *max_resid = b->max_resid;
  return FDTD_OK;
}

fdtd_status mor_basis_get(const mor_basis *b, int which, void *dst, fdtd_stream_t stream) {
  FDTD_REQUIRE(b && dst && (which == 1 || which == 2), "mor_basis_get: bad argument");
  const int q = which == 1 ? b->q1 : b->q2;
  const DevBuf &src = which == 1 ? b->V1 : b->V2;
  FDTD_CHECK_CUDA(cudaMemcpyAsync(dst, src.ptr, (size_t)q * b->n3 * b->elem, cudaMemcpyDefault, (cudaStream_t)stream));
  return FDTD_OK;
}

fdtd_status fdtd_edge_props_get(fdtd_grid *g, void *dst, fdtd_stream_t stream) {
  FDTD_REQUIRE(g && dst, "fdtd_edge_props_get: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  FDTD_CHECK(ensure_edge_props(g, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(dst, g->eprops.ptr, (size_t)12 * g->nc * g->elem, cudaMemcpyDefault, s));
  return FDTD_OK;
}

fdtd_status mor_schur_apply(fdtd_grid *g, double dt0, int nb, const double *z, const void *x, void *y,
                            fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(g && z && x && y, "mor_schur_apply: NULL argument");
  FDTD_REQUIRE(dt0 > 0, "mor_schur_apply: dt0 must be > 0");
  FDTD_REQUIRE(nb >= 1 && nb <= kMaxRhs, "mor_schur_apply: nb must be 1..%d", kMaxRhs);
  cudaStream_t s = (cudaStream_t)stream;
  FDTD_CHECK(ensure_edge_props(g, s));
  std::vector<std::complex<double>> zs(nb), one(nb, 1.0);
  for (int b = 0; b < nb; ++b) zs[b] = std::complex<double>(z[2 * b], z[2 * b + 1]);
  const int64_t n3 = 3 * g->nc;
  const int nblk = (int)((g->nc + MB - 1) / MB);
  const dim3 grid2(nblk, nb);
  const char *sch = getenv("FDTDMOR_SCHUR");
  const bool pair = sch && std::string(sch) == "pair";
  auto run = [&](auto tag) -> fdtd_status {
    using T = decltype(tag);
    const OpArgs<T> ah1 = make_op<T>(g, dt0, zs, one), ap = make_op<T>(g, dt0, zs, zs);
    const cplx<T> *xv = static_cast<const cplx<T> *>(x);
    if (!pair)
      return launch_schur_fused<T, false>(g, ap, nb, xv, static_cast<cplx<T> *>(y), n3, nullptr, nullptr, nullptr, s);
    DevBuf t;
    FDTD_CHECK(t.alloc((size_t)nb * n3 * sizeof(cplx<T>), s));
    h_from_e_kernel<T><<<grid2, MB, 0, s>>>(ah1, xv, n3, nullptr, 0, nullptr, 0, t.as<cplx<T>>(), n3, nullptr);
    fdtd_status st = after_launch("h_from_e_kernel");
    if (st == FDTD_OK) {
      e_from_h_kernel<T, EM_APPLY><<<grid2, MB, 0, s>>>(ap, t.as<cplx<T>>(), n3, xv, n3, nullptr, 0,
                                                        static_cast<cplx<T> *>(y), n3, nullptr, nullptr, 0, nullptr,
                                                        nullptr);
      st = after_launch("e_from_h_kernel");
    }
    t.release(s);
    return st;
  };
  return g->prec == FDTD_F64 ? run(double()) : run(float());
}

fdtd_status mor_basis_destroy(mor_basis *b) {
  if (!b) return FDTD_OK;
  cudaStreamSynchronize(b->stream);
  b->V1.release(b->stream);
  b->V2.release(b->stream);
  cudaStreamSynchronize(b->stream);
  delete b;
  return FDTD_OK;
}

}  // extern "C"
