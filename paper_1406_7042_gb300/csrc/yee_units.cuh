// Per-cell leap-frog units shared by the split, dataflow and batched forms of
// the Yee update (yee_split.cu, yee_batch.cu): loads, the E and H half-step
// units of one tile, and launch helpers.
#pragma once
#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "grid_internal.cuh"
#include "yee_internal.cuh"

namespace fdtdmor {

constexpr int LTX = 32, LTY = 8;

// Field loads: read-only path inside one split launch (no field is written
// and read in the same launch), L2 (coherent across CTAs) in the dataflow
// form, where the values were written by other CTAs earlier in the launch.
template <bool COH, typename T>
__device__ __forceinline__ T ldf(const T *p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
// Per cell: the material shared by the 8 cells around its E edges' dual faces
// (i-1..i, j-1..j, k-1..k, inside the grid), or the sentinel ~0 when they differ.
template <typename ID>
__global__ void emat_kernel(const ID *__restrict__ mat, int nx, int ny, int nz, ID *__restrict__ out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)nx * ny;
  if (n >= plane * nz) return;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / plane);
  const ID m = mat[n];
  bool uni = true;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        if (i + di < 0 || j + dj < 0 || k + dk < 0) continue;
        uni &= mat[n + dk * plane + dj * nx + di] == m;
      }
  out[n] = uni ? m : (ID)~(ID)0;
}

// VW consecutive values starting at p (p aligned to VW values): one 4-, 8- or
// 16-byte load.
template <int VW, bool COH, typename T>
__device__ __forceinline__ void ldv(T (&r)[VW], const T *p) {
  if constexpr (VW == 1) {
    r[0] = ldf<COH>(p);
  } else if constexpr (sizeof(T) == 4 && VW == 4) {
    const float4 v = COH ? __ldcg(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  } else if constexpr (sizeof(T) == 4 && VW == 2) {
    const float2 v = COH ? __ldcg(reinterpret_cast<const float2 *>(p)) : __ldg(reinterpret_cast<const float2 *>(p));
    r[0] = v.x; r[1] = v.y;
  } else {
    static_assert(sizeof(T) == 8 && VW == 2, "unsupported vector width");
    const double2 v = COH ? __ldcg(reinterpret_cast<const double2 *>(p)) : __ldg(reinterpret_cast<const double2 *>(p));
    r[0] = v.x; r[1] = v.y;
  }
}

template <int VW, typename T>
__device__ __forceinline__ void stv(T *p, const T (&r)[VW]) {
  if constexpr (VW == 1) {
    p[0] = r[0];
  } else if constexpr (sizeof(T) == 4 && VW == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
  } else if constexpr (sizeof(T) == 4 && VW == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
  } else {
    *reinterpret_cast<double2 *>(p) = make_double2(r[0], r[1]);
  }
}

// VW material ids starting at p (aligned), in one load.
template <int VW, typename ID>
__device__ __forceinline__ void ldids(ID (&r)[VW], const ID *p) {
  constexpr int B = VW * (int)sizeof(ID);
  if constexpr (B == 1 || B == 2 && sizeof(ID) == 2) {
    r[0] = __ldg(p);
  } else if constexpr (B == 2) {
    const unsigned short v = __ldg(reinterpret_cast<const unsigned short *>(p));
    r[0] = (ID)(v & 0xff); r[1] = (ID)(v >> 8);
  } else if constexpr (B == 4) {
    const unsigned v = __ldg(reinterpret_cast<const unsigned *>(p));
    if constexpr (sizeof(ID) == 1) { r[0] = (ID)(v & 0xff); r[1] = (ID)((v >> 8) & 0xff); r[2] = (ID)((v >> 16) & 0xff); r[3] = (ID)(v >> 24); }
    else { r[0] = (ID)(v & 0xffff); r[1] = (ID)(v >> 16); }
  } else {
    static_assert(B == 8, "unsupported id width");
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    r[0] = (ID)(v.x & 0xffff); r[1] = (ID)(v.x >> 16); r[2] = (ID)(v.y & 0xffff); r[3] = (ID)(v.y >> 16);
  }
}

// (Ca, Cb) of the three E edges of cell c = (i, j, k): from the material
// table where the cell's uniform-neighbourhood id mu is set, else the area
// weighted edge average; zero on the walls (tangential E of the PEC box).
template <typename T, typename ID>
__device__ __forceinline__ void cell_e_coefs(const YeeArgs<T, ID> &a, ID mu, int64_t c, int i, int j, int k, T wyl,
                                             T wyh, T (&ca)[3], T (&cb)[3]) {
  const int nx = a.nx, ny = a.ny, ntot = nx + ny + a.nz;
  const int64_t plane = (int64_t)nx * ny;
  const ID none = (ID)~(ID)0;
  if (mu != none) {
    ca[0] = ca[1] = ca[2] = __ldg(a.ctab + mu);
    cb[0] = cb[1] = cb[2] = __ldg(a.ctab + a.nmat + mu);
  } else {
    const ID *M = a.mat;
    const T wxl = __ldg(a.ax + AX_WLO * ntot + i), wxh = __ldg(a.ax + AX_WHI * ntot + i);
    const T wzl = __ldg(a.ax + AX_WLO * ntot + nx + ny + k), wzh = __ldg(a.ax + AX_WHI * ntot + nx + ny + k);
    const ID m = M[c];
    const ID m_i = i > 0 ? M[c - 1] : m, m_j = j > 0 ? M[c - nx] : m, m_k = k > 0 ? M[c - plane] : m;
    const ID m_ij = (i > 0 && j > 0) ? M[c - 1 - nx] : m, m_ik = (i > 0 && k > 0) ? M[c - 1 - plane] : m;
    const ID m_jk = (j > 0 && k > 0) ? M[c - nx - plane] : m;
    e_coef(a, m_jk, m_k, m_j, m, wyl, wyh, wzl, wzh, ca[0], cb[0]);
    e_coef(a, m_ik, m_k, m_i, m, wxl, wxh, wzl, wzh, ca[1], cb[1]);
    e_coef(a, m_ij, m_j, m_i, m, wxl, wxh, wyl, wyh, ca[2], cb[2]);
  }
  if (j == 0 || k == 0) ca[0] = cb[0] = T(0);
  if (i == 0 || k == 0) ca[1] = cb[1] = T(0);
  if (i == 0 || j == 0) ca[2] = cb[2] = T(0);
}

// The per-edge coefficient map of a grid: what e_unit computes per cell,
// stored once (Ca of x, y, z edges, then Cb of x, y, z, each nc long).
template <typename T, typename ID>
__global__ void ecoef_kernel(YeeArgs<T, ID> a, const ID *__restrict__ emat, T *__restrict__ out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)a.nx * a.ny;
  if (n >= a.nc) return;
  const int i = (int)(n % a.nx), j = (int)((n / a.nx) % a.ny), k = (int)(n / plane);
  const int ntot = a.nx + a.ny + a.nz;
  const T wyl = __ldg(a.ax + AX_WLO * ntot + a.nx + j), wyh = __ldg(a.ax + AX_WHI * ntot + a.nx + j);
  T ca[3], cb[3];
  cell_e_coefs(a, emat[n], n, i, j, k, wyl, wyh, ca, cb);
  for (int c = 0; c < 3; ++c) {
    out[c * a.nc + n] = ca[c];
    out[(3 + c) * a.nc + n] = cb[c];
  }
}

// E^{n+1} on planes [k0, k1) of tile (bx, by), which spans LTX * VW cells in
// x: thread (tx, ty) owns cells i0 .. i0 + VW - 1 of row j and marches in z.
// The x neighbour i0 - 1 comes from the lane to the left (a shuffle) or, for
// lane 0, from one extra load.  All lanes of a warp run the loop, so lanes
// past the end of a row (whose loads read as zero) still feed the shuffles.
// In place when a.Eout == a.Ein: the only E value read is the one written by
// the same thread, and the store depends on it.
//
// With PRE the coefficients come from the per-edge map a.ecoef (six more
// vector loads, no material lookups): the form for small, L2-resident grids,
// where the averaging at material interfaces would set the pace.
template <typename T, typename ID, bool COH, int VW, bool PRE = false>
__device__ __forceinline__ void e_unit(const YeeArgs<T, ID> &a, const ID *__restrict__ emat, int bx, int by,
                                       int k0, int k1) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * LTX + tx;
  const int i0 = (bx * LTX + tx) * VW, j = by * LTY + ty;
  const int nx = a.nx, ny = a.ny, ntot = nx + ny + a.nz;
  const int64_t nc = a.nc, plane = (int64_t)nx * ny;
  auto ax = [&](int table, int idx) { return __ldg(a.ax + table * ntot + idx); };
  if (j < ny) {  // warp-uniform
    const bool live = i0 < nx;
    const T ryd = ax(AX_RDD, nx + j), wyl = ax(AX_WLO, nx + j), wyh = ax(AX_WHI, nx + j);
    T rxd[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) rxd[e] = live ? ax(AX_RDD, i0 + e) : T(0);
    const T *Hx = a.Hin, *Hy = a.Hin + nc, *Hz = a.Hin + 2 * nc;
    int64_t n = k0 * plane + (int64_t)j * nx + i0;
    T hx_km[VW], hy_km[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) hx_km[e] = hy_km[e] = T(0);
    if (live && k0 > 0) {
      ldv<VW, COH>(hx_km, Hx + n - plane);
      ldv<VW, COH>(hy_km, Hy + n - plane);
    }
    for (int k = k0; k < k1; ++k, n += plane) {
      T hx[VW], hy[VW], hz[VW], hx_jm[VW], hz_jm[VW], ex[VW], ey[VW], ez[VW];
      ID mu[VW];
      T pca[3][VW], pcb[3][VW];  // per-edge coefficients (PRE)
#pragma unroll
      for (int e = 0; e < VW; ++e) hx[e] = hy[e] = hz[e] = hx_jm[e] = hz_jm[e] = ex[e] = ey[e] = ez[e] = T(0);
      T hy_l = T(0), hz_l = T(0);  // Hy, Hz at i0 - 1 for lane 0
      if (live) {
        if constexpr (PRE) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            ldv<VW, COH>(pca[c], a.ecoef + c * nc + n);
            ldv<VW, COH>(pcb[c], a.ecoef + (3 + c) * nc + n);
          }
        }
        ldv<VW, COH>(hx, Hx + n);
        ldv<VW, COH>(hy, Hy + n);
        ldv<VW, COH>(hz, Hz + n);
        if (j > 0) {
          ldv<VW, COH>(hx_jm, Hx + n - nx);
          ldv<VW, COH>(hz_jm, Hz + n - nx);
        }
        ldv<VW, COH>(ex, a.Ein + n);
        ldv<VW, COH>(ey, a.Ein + nc + n);
        ldv<VW, COH>(ez, a.Ein + 2 * nc + n);
        if constexpr (!PRE) ldids<VW>(mu, emat + n);
        if (tx == 0 && i0 > 0) {
          hy_l = ldf<COH>(Hy + n - 1);
          hz_l = ldf<COH>(Hz + n - 1);
        }
      }
      const T hy_s = __shfl_up_sync(0xffffffffu, hy[VW - 1], 1), hz_s = __shfl_up_sync(0xffffffffu, hz[VW - 1], 1);
      if (tx > 0) { hy_l = hy_s; hz_l = hz_s; }
      if (live) {
        const T rzd = ax(AX_RDD, nx + ny + k);
        T ox[VW], oy[VW], oz[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const int i = i0 + e;
          const T hy_im = e == 0 ? hy_l : hy[e - 1], hz_im = e == 0 ? hz_l : hz[e - 1];
          T cax, cbx, cay, cby, caz, cbz;
          if constexpr (PRE) {
            cax = pca[0][e]; cay = pca[1][e]; caz = pca[2][e];
            cbx = pcb[0][e]; cby = pcb[1][e]; cbz = pcb[2][e];
          } else {
            T ca[3], cb[3];
            cell_e_coefs(a, mu[e], n + e, i, j, k, wyl, wyh, ca, cb);
            cax = ca[0]; cay = ca[1]; caz = ca[2];
            cbx = cb[0]; cby = cb[1]; cbz = cb[2];
          }
          ox[e] = cax * ex[e] + cbx * ((hz[e] - hz_jm[e]) * ryd - (hy[e] - hy_km[e]) * rzd);
          oy[e] = cay * ey[e] + cby * ((hx[e] - hx_km[e]) * rzd - (hz[e] - hz_im) * rxd[e]);
          oz[e] = caz * ez[e] + cbz * ((hy[e] - hy_im) * rxd[e] - (hx[e] - hx_jm[e]) * ryd);
        }
        stv<VW>(a.Eout + n, ox);
        stv<VW>(a.Eout + nc + n, oy);
        stv<VW>(a.Eout + 2 * nc + n, oz);
      }
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        hx_km[e] = hx[e];
        hy_km[e] = hy[e];
      }
    }
  }
  // sources of this tile on these planes: E -= Cb w u
  const int tile = by * a.ntx + bx;
  const int s0 = a.src_ptr[tile], s1 = a.src_ptr[tile + 1];
  if (s1 > s0) {
    __syncthreads();
    for (int q = s0 + tid; q < s1; q += LTX * LTY) {
      const PortEntry pe = a.src[q];
      if (pe.k < k0 || pe.k >= k1 || pe.lx >= LTX * VW || pe.ly >= LTY) continue;
      if (!dcheck(a.err, pe.comp >= 0 && pe.comp < 3 && pe.lx >= 0 && pe.ly >= 0 && pe.port >= 0)) continue;
      const int si = bx * LTX * VW + pe.lx, sj = by * LTY + pe.ly, k = pe.k;
      if (si >= nx || sj >= ny) continue;
      const int64_t n = k * plane + (int64_t)sj * nx + si;
      const ID *M = a.mat;
      T ca, cb = 0;
      const T wzl = ax(AX_WLO, nx + ny + k), wzh = ax(AX_WHI, nx + ny + k);
      if (pe.comp == 0 && sj > 0 && k > 0)
        e_coef(a, M[n - nx - plane], M[n - plane], M[n - nx], M[n], ax(AX_WLO, nx + sj), ax(AX_WHI, nx + sj), wzl, wzh, ca, cb);
      else if (pe.comp == 1 && si > 0 && k > 0)
        e_coef(a, M[n - 1 - plane], M[n - plane], M[n - 1], M[n], ax(AX_WLO, si), ax(AX_WHI, si), wzl, wzh, ca, cb);
      else if (pe.comp == 2 && si > 0 && sj > 0)
        e_coef(a, M[n - 1 - nx], M[n - nx], M[n - 1], M[n], ax(AX_WLO, si), ax(AX_WHI, si), ax(AX_WLO, nx + sj),
               ax(AX_WHI, nx + sj), ca, cb);
      atomicAdd(&a.Eout[pe.comp * nc + n], -cb * (T)pe.w * a.u[pe.port]);
    }
  }
}

// H^{n+3/2} on planes [k0, k1) of tile (bx, by), from E^{n+1} in a.Eout; the
// x neighbour i0 + VW comes from the lane to the right or, for lane 31, from
// one extra load.  In place when a.Hout == a.Hin (as in e_unit).
template <typename T, typename ID, bool HOMOG_H, bool COH, int VW>
__device__ __forceinline__ void h_unit(const YeeArgs<T, ID> &a, int bx, int by, int k0, int k1) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * LTX + tx;
  const int i0 = (bx * LTX + tx) * VW, j = by * LTY + ty;
  const int nx = a.nx, ny = a.ny, nz = a.nz, ntot = nx + ny + nz;
  const int64_t nc = a.nc, plane = (int64_t)nx * ny;
  auto ax = [&](int table, int idx) { return __ldg(a.ax + table * ntot + idx); };
  const T *Ex = a.Eout, *Ey = a.Eout + nc, *Ez = a.Eout + 2 * nc;  // E^{n+1}
  if (j < ny) {  // warp-uniform
    const bool live = i0 < nx;
    const T rdy = ax(AX_RD, nx + j);
    T rdx[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) rdx[e] = live ? ax(AX_RD, i0 + e) : T(0);
    const T da0 = __ldg(a.ctab + 2 * a.nmat), db0 = __ldg(a.ctab + 3 * a.nmat);
    int64_t n = k0 * plane + (int64_t)j * nx + i0;
    T ex[VW], ey[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) ex[e] = ey[e] = T(0);
    if (live) {
      ldv<VW, COH>(ex, Ex + n);
      ldv<VW, COH>(ey, Ey + n);
    }
    for (int k = k0; k < k1; ++k, n += plane) {
      T ez[VW], ex_kp[VW], ey_kp[VW], ex_jp[VW], ez_jp[VW], h0[VW], h1[VW], h2[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) ez[e] = ex_kp[e] = ey_kp[e] = ex_jp[e] = ez_jp[e] = h0[e] = h1[e] = h2[e] = T(0);
      T ey_r = T(0), ez_r = T(0);  // Ey, Ez at i0 + VW for lane 31
      if (live) {
        ldv<VW, COH>(ez, Ez + n);
        if (k + 1 < nz) {
          ldv<VW, COH>(ex_kp, Ex + n + plane);
          ldv<VW, COH>(ey_kp, Ey + n + plane);
        }
        if (j + 1 < ny) {
          ldv<VW, COH>(ex_jp, Ex + n + nx);
          ldv<VW, COH>(ez_jp, Ez + n + nx);
        }
        ldv<VW, COH>(h0, a.Hin + n);
        ldv<VW, COH>(h1, a.Hin + nc + n);
        ldv<VW, COH>(h2, a.Hin + 2 * nc + n);
        if (tx == LTX - 1 && i0 + VW < nx) {
          ey_r = ldf<COH>(Ey + n + VW);
          ez_r = ldf<COH>(Ez + n + VW);
        }
      }
      const T ey_s = __shfl_down_sync(0xffffffffu, ey[0], 1), ez_s = __shfl_down_sync(0xffffffffu, ez[0], 1);
      if (tx < LTX - 1) { ey_r = ey_s; ez_r = ez_s; }
      if (live) {
        const T rdz = ax(AX_RD, nx + ny + k);
        T ox[VW], oy[VW], oz[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          const int i = i0 + e;
          const T ey_ip = e == VW - 1 ? ey_r : ey[e + 1], ez_ip = e == VW - 1 ? ez_r : ez[e + 1];
          T da[3] = {da0, da0, da0}, db[3] = {db0, db0, db0};
          if (!HOMOG_H) {
            const ID *M = a.mat;
            const int64_t c = n + e;
            const ID m = M[c];
            if (i > 0) h_coef(a, M[c - 1], m, ax(AX_WLO, i), ax(AX_WHI, i), da[0], db[0]);
            if (j > 0) h_coef(a, M[c - nx], m, ax(AX_WLO, nx + j), ax(AX_WHI, nx + j), da[1], db[1]);
            if (k > 0) h_coef(a, M[c - plane], m, ax(AX_WLO, nx + ny + k), ax(AX_WHI, nx + ny + k), da[2], db[2]);
          }
          const T hx = da[0] * h0[e] - db[0] * ((ez_jp[e] - ez[e]) * rdy - (ey_kp[e] - ey[e]) * rdz);
          const T hy = da[1] * h1[e] - db[1] * ((ex_kp[e] - ex[e]) * rdz - (ez_ip - ez[e]) * rdx[e]);
          const T hz = da[2] * h2[e] - db[2] * ((ey_ip - ey[e]) * rdx[e] - (ex_jp[e] - ex[e]) * rdy);
          ox[e] = i == 0 ? T(0) : hx;
          oy[e] = j == 0 ? T(0) : hy;
          oz[e] = k == 0 ? T(0) : hz;
        }
        stv<VW>(a.Hout + n, ox);
        stv<VW>(a.Hout + nc + n, oy);
        stv<VW>(a.Hout + 2 * nc + n, oz);
      }
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        ex[e] = ex_kp[e];
        ey[e] = ey_kp[e];
      }
    }
  }
  // probes of this tile on these planes read the final E^{n+1}
  const int tile = by * a.ntx + bx;
  const int p0 = a.prb_ptr[tile], p1 = a.prb_ptr[tile + 1];
  for (int q = p0 + tid; q < p1; q += LTX * LTY) {
    const PortEntry pe = a.prb[q];
    if (pe.k < k0 || pe.k >= k1) continue;
    if (!dcheck(a.err, pe.comp >= 0 && pe.comp < 3 && pe.lx >= 0 && pe.ly >= 0 && pe.port >= 0)) continue;
    const int si = bx * LTX * VW + pe.lx, sj = by * LTY + pe.ly;
    if (si >= nx || sj >= ny) continue;
    atomicAdd(&a.y[pe.port], (T)pe.w * ldf<COH>(a.Eout + pe.comp * nc + pe.k * plane + (int64_t)sj * nx + si));
  }
}

// The split kernels are launched as programmatic dependents of the kernel
// before them: a CTA waits for that grid to complete (and its writes to be
// visible) before touching memory, and lets the next launch begin once its own
// work is done, so consecutive launches overlap their launch latency.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialisation (see wait_prior_grid).
template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                         Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = getenv("FDTDMOR_NO_PDL") ? 0 : 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  return launch_dependent_smem(kern, grid, block, 0, s, args...);
}

template <typename T, typename ID>
inline YeeArgs<T, ID> split_args(fdtd_grid *g) {
  YeeArgs<T, ID> a;
  a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.kchunk = 0; a.nc = g->nc;
  a.ntx = g->lists.ntx; a.nty = g->lists.nty;
  const T *in = g->fields[g->cur].as<T>();
  T *out = g->fields[g->cur ^ 1].as<T>();
  a.Ein = in; a.Hin = in + 3 * g->nc;
  a.Eout = out; a.Hout = out + 3 * g->nc;
  a.mat = g->mat.as<ID>();
  a.ax = g->axis.as<T>();
  a.mtab = g->mtab.as<T>();
  a.ctab = g->ctab.as<T>();
  a.ecoef = nullptr;
  a.nmat = g->nmat;
  a.inv_dt = (T)(1.0 / g->ctab_dt);
  a.src_ptr = g->lists.src_ptr.as<int32_t>();
  a.src = g->lists.src.as<PortEntry>();
  a.u = nullptr;
  a.prb_ptr = g->lists.prb_ptr.as<int32_t>();
  a.prb = g->lists.prb.as<PortEntry>();
  a.y = nullptr;
  a.err = g->errflag.as<unsigned>();
  return a;
}

template <typename ID>
inline fdtd_status ensure_emat(fdtd_grid *g, cudaStream_t s) {
  if (g->emat_ready) return FDTD_OK;
  FDTD_CHECK(g->emat.alloc((size_t)g->nc * sizeof(ID), s));
  emat_kernel<ID><<<(int)((g->nc + 255) / 256), 256, 0, s>>>(g->mat.as<ID>(), g->nx, g->ny, g->nz, g->emat.as<ID>());
  FDTD_CHECK(after_launch("emat_kernel"));
  g->emat_ready = true;
  return FDTD_OK;
}

// The per-edge coefficient map for the current coefficient table.
template <typename T, typename ID>
inline fdtd_status ensure_ecoef(fdtd_grid *g, const YeeArgs<T, ID> &a, cudaStream_t s) {
  if (g->ecoef_version == g->ctab_version && g->ecoef.ptr) return FDTD_OK;
  FDTD_CHECK(ensure_emat<ID>(g, s));
  FDTD_CHECK(g->ecoef.alloc((size_t)6 * g->nc * sizeof(T), s));
  ecoef_kernel<T, ID><<<(int)((g->nc + 255) / 256), 256, 0, s>>>(a, g->emat.as<ID>(), g->ecoef.as<T>());
  FDTD_CHECK(after_launch("ecoef_kernel"));
  g->ecoef_version = g->ctab_version;
  return FDTD_OK;
}

inline int env_int(const char *name, int dflt) {
  const char *e = getenv(name);
  return e ? std::max(1, atoi(e)) : dflt;
}

inline int device_sms() {
  static const int sms = [] {  // thread-safe one-time query
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

}  // namespace fdtdmor
