// A2 (large grids): the Yee leap-frog of Eq. (matrix) fused into one pass over
// memory per step.
//
// A CTA of 8 warps (one per row) owns 7 rows of a 32 VW-cell-wide tile and
// marches up a chunk of z planes; thread (tx, ty) owns VW consecutive x cells
// of row ty.  At plane k every warp computes E^{n+1}(k) for its cells (warp 7
// for the first row of the next tile, which the last owned row's H needs) and
// publishes Ex, Ez in shared memory; the first lanes of warp 7 also compute
// Ey, Ez of the +x halo column.  The owned rows then update H^{n+3/2} one
// plane behind, at k - 1, from E^{n+1} at k - 1 (own cells, the next lane's by
// a shuffle, the row above and the halo column from shared memory) and at k
// (own cells).  One barrier per plane; the shared slots alternate with the
// plane parity.  A chunk's top plane is computed once more by the chunk above.
// The new state goes to the other buffer (ping-pong), so neighbours always
// read the old one.
//
// In FP32 with 4 cells per thread the plane inputs (H with the row below and
// the columns either side, E and the material map with the +x column) are
// staged in shared memory by TMA, three planes ahead of the plane in work.
//
// DRAM sees each field value read once and written once per step (the 48 B
// per cell of the fused form, plus the material map); the halo row's and
// chunk tops' reads come mostly from L2.  Sources and probes are applied
// afterwards by one small kernel: the step is linear, so a source's effect on
// this step's H is -Db curlE(dE) on the four H edges around the source edge;
// these terms are gathered once per dt into one term per field value and port
// (ensure_fix), and the probes share the launch when no probe edge carries a
// term (else an atomic source kernel and a probe kernel follow).
#include <algorithm>
#include <cstring>
#include <vector>

#include "tma_util.cuh"
#include "yee_units.cuh"

namespace fdtdmor {

// One E^{n+1} component (without sources) at any cell, zero outside the box:
// Ca E^n + Cb (curl H^{n+1/2})_c, coefficients from the uniform-neighbourhood
// map or the edge average.
template <typename T, typename ID>
__device__ __forceinline__ T e_comp_at(const YeeArgs<T, ID> &a, const ID *__restrict__ emat, int c, int i, int j,
                                       int k) {
  const int nx = a.nx, ny = a.ny, nz = a.nz, ntot = nx + ny + nz;
  if (i >= nx || j >= ny || k >= nz) return T(0);
  if ((c == 0 && (j == 0 || k == 0)) || (c == 1 && (i == 0 || k == 0)) || (c == 2 && (i == 0 || j == 0))) return T(0);
  const int64_t nc = a.nc, plane = (int64_t)nx * ny, n = k * plane + (int64_t)j * nx + i;
  auto ax = [&](int table, int idx) { return __ldg(a.ax + table * ntot + idx); };
  const T *Hx = a.Hin, *Hy = a.Hin + nc, *Hz = a.Hin + 2 * nc;
  const ID none = (ID)~(ID)0, mu = __ldg(emat + n);
  T ca, cb, curl;
  const ID *M = a.mat;
  if (c == 0) {
    curl = (__ldg(Hz + n) - __ldg(Hz + n - nx)) * ax(AX_RDD, nx + j) -
           (__ldg(Hy + n) - __ldg(Hy + n - plane)) * ax(AX_RDD, nx + ny + k);
    if (mu != none) { ca = __ldg(a.ctab + mu); cb = __ldg(a.ctab + a.nmat + mu); }
    else e_coef(a, M[n - nx - plane], M[n - plane], M[n - nx], M[n], ax(AX_WLO, nx + j), ax(AX_WHI, nx + j),
                ax(AX_WLO, nx + ny + k), ax(AX_WHI, nx + ny + k), ca, cb);
  } else if (c == 1) {
    curl = (__ldg(Hx + n) - __ldg(Hx + n - plane)) * ax(AX_RDD, nx + ny + k) -
           (__ldg(Hz + n) - __ldg(Hz + n - 1)) * ax(AX_RDD, i);
    if (mu != none) { ca = __ldg(a.ctab + mu); cb = __ldg(a.ctab + a.nmat + mu); }
    else e_coef(a, M[n - 1 - plane], M[n - plane], M[n - 1], M[n], ax(AX_WLO, i), ax(AX_WHI, i),
                ax(AX_WLO, nx + ny + k), ax(AX_WHI, nx + ny + k), ca, cb);
  } else {
    curl = (__ldg(Hy + n) - __ldg(Hy + n - 1)) * ax(AX_RDD, i) - (__ldg(Hx + n) - __ldg(Hx + n - nx)) * ax(AX_RDD, nx + j);
    if (mu != none) { ca = __ldg(a.ctab + mu); cb = __ldg(a.ctab + a.nmat + mu); }
    else e_coef(a, M[n - 1 - nx], M[n - nx], M[n - 1], M[n], ax(AX_WLO, i), ax(AX_WHI, i), ax(AX_WLO, nx + j),
                ax(AX_WHI, nx + j), ca, cb);
  }
  return ca * __ldg(a.Ein + c * nc + n) + cb * curl;
}

// TMA staging of the 4-cell FP32 form: per plane, boxes of the tile with its
// halos, x from i0 - 4 (H: the -x neighbour column and the +x halo column at
// i0 + 128) or i0 (E, material map: the +x halo column), y from j0 - 1 (H: the
// row below the tile) or j0, S planes in flight, one mbarrier per slot.
struct MarchMaps {
  CUtensorMap H[3], E[3], M;
};
template <typename ID>
struct MarchStage {
  static constexpr int HX = 136, HY = 9, EX = 132, EY = 8, MX = 144, MY = 8;
  static constexpr int rup(int b) { return (b + 127) / 128 * 128; }
  static constexpr int HB = rup(HX * HY * 4), EB = rup(EX * EY * 4), MB = rup(MX * MY * (int)sizeof(ID));
  static constexpr int BYTES = 3 * HB + 3 * EB + MB;
  static constexpr uint32_t TX = 3u * HX * HY * 4 + 3u * EX * EY * 4 + MX * MY * sizeof(ID);
  static constexpr int S = 3;
  static constexpr size_t SMEM = (size_t)S * BYTES + S * sizeof(uint64_t);
};

// CTAs per SM the register budget is sized for (MTY rows of 32 threads;
// measured on 384 x 384 x 64: 8 rows beat 16, whose barrier spans twice the warps).
template <typename T, int VW, int MTY>
constexpr int march_min_blocks() {
  return MTY > 8 ? 1 : (sizeof(T) == 8 ? 3 - VW : (VW == 4 ? 2 : 3));
}

//
// STAGED (FP32, 4 cells per thread, 8 warps): the plane inputs arrive in
// shared memory by TMA, S planes ahead, instead of per-thread loads; waits are
// bounded and a wait that gives up sets *err and ends the CTA after its copies
// in flight have landed.
template <typename T, typename ID, bool HOMOG_H, int VW, int MTY, bool STAGED>
__global__ void __launch_bounds__(LTX *MTY, march_min_blocks<T, VW, MTY>()) yee_march_kernel(YeeArgs<T, ID> a, const ID *__restrict__ emat, int lz,
                                                                                            const __grid_constant__ MarchMaps maps,
                                                                                            unsigned *err) {
  constexpr int OWN = MTY - 1;  // rows a CTA owns; the last warp computes E of the next tile's first row
  constexpr int W = LTX * VW;   // cells per tile row
  static_assert(!STAGED || (sizeof(T) == 4 && VW == 4 && MTY == 8), "staged form: FP32, 4 cells, 8 warps");
  using St = MarchStage<ID>;
  __shared__ T sx[2][MTY][W], sz[2][MTY][W];  // Ex, Ez of E^{n+1} by row, planes k & 1
  __shared__ T sh[2][2][OWN];                 // Ey, Ez of E^{n+1} on the +x halo column
  extern __shared__ __align__(128) unsigned char stg[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(stg + (STAGED ? St::S * St::BYTES : 0));
  wait_prior_grid();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool halo = ty == OWN;  // warp-uniform
  const int nx = a.nx, ny = a.ny, nz = a.nz, ntot = nx + ny + nz;
  const int64_t nc = a.nc, plane = (int64_t)nx * ny;
  auto ax = [&](int table, int idx) { return __ldg(a.ax + table * ntot + idx); };
  // this CTA: chunk blockIdx.z of tile (blockIdx.x, blockIdx.y)
  {
  const int k0 = blockIdx.z * lz, k1 = min(nz, k0 + lz);
  const int bx = blockIdx.x, by = blockIdx.y;
  const int i0 = (bx * LTX + tx) * VW, j0 = by * OWN, j = j0 + ty;
  const bool live = i0 < nx && j < ny;
  const int jc = min(j, ny - 1);
  const T *Hx = a.Hin, *Hy = a.Hin + nc, *Hz = a.Hin + 2 * nc;
  const ID *M = a.mat;
  const ID none = (ID)~(ID)0;
  const T ryd = ax(AX_RDD, nx + jc), wyl = ax(AX_WLO, nx + jc), wyh = ax(AX_WHI, nx + jc);
  const T rdy = ax(AX_RD, nx + jc);
  T rxd[VW], rdx[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) {
    rxd[e] = live ? ax(AX_RDD, i0 + e) : T(0);
    rdx[e] = live ? ax(AX_RD, i0 + e) : T(0);
  }
  const T da0 = __ldg(a.ctab + 2 * a.nmat), db0 = __ldg(a.ctab + 3 * a.nmat);
  // the halo warp's first lanes compute Ey, Ez of the +x halo column ih (the
  // next tile's first column) for the owned rows, carrying its old Hx
  const int ih = (bx + 1) * W, jh = j0 + tx;
  const bool xl = halo && tx < OWN && ih < nx && jh < ny;
  const int64_t nhrow = (int64_t)min(jh, ny - 1) * nx + min(ih, nx - 1);
  const T rxdh = xl ? ax(AX_RDD, ih) : T(0), rydh = xl ? ax(AX_RDD, nx + jh) : T(0);
  // carried from plane k - 1: old H and new E of the own cells (and the halo cell)
  T hx_p[VW], hy_p[VW], hz_p[VW], ex_p[VW], ey_p[VW], ez_p[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) hx_p[e] = hy_p[e] = hz_p[e] = ex_p[e] = ey_p[e] = ez_p[e] = T(0);
  T hxh_p = T(0);
  int64_t n = k0 * plane + (int64_t)jc * nx + i0;
  if (live && k0 > 0) {
    ldv<VW, false>(hx_p, Hx + n - plane);
    ldv<VW, false>(hy_p, Hy + n - plane);
  }
  if (xl && k0 > 0) hxh_p = __ldg(Hx + k0 * plane + nhrow - plane);
  // staged: planes k0 .. kmax are loaded, plane k0 + r into slot r % S
  const int kmax = min(k1, nz - 1), nload = kmax - k0 + 1;
  const int i0t = bx * W;
  const int tid = ty * LTX + tx;
  bool ok = true;
  int waited = -1, issued = -1;
  auto issue = [&](int r) {
    unsigned char *st = stg + (r % St::S) * St::BYTES;
    uint64_t *bar = &bars[r % St::S];
    const int kk = k0 + r;
    mbar_expect_tx(bar, St::TX);
    for (int c = 0; c < 3; ++c) tma_load_3d(st + c * St::HB, &maps.H[c], i0t - 4, j0 - 1, kk, bar);
    for (int c = 0; c < 3; ++c) tma_load_3d(st + 3 * St::HB + c * St::EB, &maps.E[c], i0t, j0, kk, bar);
    tma_load_3d(st + 3 * St::HB + 3 * St::EB, &maps.M, i0t, j0, kk, bar);
    issued = r;
  };
  if constexpr (STAGED) {
    if (tid == 0) {
      for (int q = 0; q < St::S; ++q) mbar_init(&bars[q], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (int r = 0; r < min(St::S, nload); ++r) issue(r);
    }
    __syncthreads();
  }
  for (int k = k0; k <= k1; ++k, n += plane) {
    const bool top = k == k1;  // plane of the chunk above: E for H(k-1) only
    const bool inbox = k < nz;
    const int b = k & 1;
    const int r = k - k0;
    const unsigned char *st = stg + (r % St::S) * St::BYTES;
    if constexpr (STAGED) {
      if (k <= kmax) {
        if (mbar_wait(&bars[r % St::S], (r / St::S) & 1)) waited = r;
        else ok = false;
      }
    }
    // staged reads: component c of H (rows j0 - 1 .. j0 + 7, x from i0t - 4),
    // of E and of the material map (rows j0 .. j0 + 7, x from i0t)
    auto hs = [&](int c, int row, int x) -> const float * {
      return reinterpret_cast<const float *>(st + c * St::HB) + row * St::HX + x;
    };
    auto es = [&](int c, int row, int x) -> const float * {
      return reinterpret_cast<const float *>(st + 3 * St::HB + c * St::EB) + row * St::EX + x;
    };
    auto ms = [&](int row, int x) -> const ID * {
      return reinterpret_cast<const ID *>(st + 3 * St::HB + 3 * St::EB) + row * St::MX + x;
    };
    T hx[VW], hy[VW], hz[VW], hx_jm[VW], hz_jm[VW], ex[VW], ey[VW], ez[VW];
    ID mu[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) hx[e] = hy[e] = hz[e] = hx_jm[e] = hz_jm[e] = ex[e] = ey[e] = ez[e] = T(0);
    T hy_l = T(0), hz_l = T(0);
    if (live && inbox) {
      if constexpr (STAGED) {
        const int xo = 4 + tx * VW;
        auto ld4 = [](T (&r4)[VW], const float *p) {
          const float4 v = *reinterpret_cast<const float4 *>(p);
          r4[0] = v.x; r4[1] = v.y; r4[2] = v.z; r4[3] = v.w;
        };
        if constexpr (VW == 4) {
          ld4(hx, hs(0, ty + 1, xo));
          ld4(hy, hs(1, ty + 1, xo));
          ld4(hz, hs(2, ty + 1, xo));
          ld4(hx_jm, hs(0, ty, xo));   // zero-filled below the grid
          ld4(hz_jm, hs(2, ty, xo));
          ld4(ex, es(0, ty, tx * VW));
          ld4(ey, es(1, ty, tx * VW));
          ld4(ez, es(2, ty, tx * VW));
          const ID *mp = ms(ty, tx * VW);
#pragma unroll
          for (int e = 0; e < VW; ++e) mu[e] = mp[e];
          hy_l = *hs(1, ty + 1, 3);    // x = i0 - 1 (zero-filled left of the grid)
          hz_l = *hs(2, ty + 1, 3);
        }
      } else {
        ldv<VW, false>(hx, Hx + n);
        ldv<VW, false>(hy, Hy + n);
        ldv<VW, false>(hz, Hz + n);
        if (j > 0) {
          ldv<VW, false>(hx_jm, Hx + n - nx);
          ldv<VW, false>(hz_jm, Hz + n - nx);
        }
        ldv<VW, false>(ex, a.Ein + n);
        ldv<VW, false>(ey, a.Ein + nc + n);
        ldv<VW, false>(ez, a.Ein + 2 * nc + n);
        ldids<VW>(mu, emat + n);
        if (tx == 0 && i0 > 0) {
          hy_l = __ldg(Hy + n - 1);
          hz_l = __ldg(Hz + n - 1);
        }
      }
    }
    T hxh = T(0), hxh_jm = T(0), hyh = T(0), hyh_m = T(0), hzh = T(0), hzh_m = T(0), eyh_o = T(0), ezh_o = T(0);
    ID muh = none;
    const int64_t nhc = k * plane + nhrow;
    if (xl && inbox) {
      if constexpr (STAGED) {
        // halo cell (i0t + 128, j0 + tx): staged x 132 (H) / 128 (E, map)
        hxh = *hs(0, tx + 1, 4 + W);
        hxh_jm = *hs(0, tx, 4 + W);
        hyh = *hs(1, tx + 1, 4 + W);
        hyh_m = *hs(1, tx + 1, 3 + W);
        hzh = *hs(2, tx + 1, 4 + W);
        hzh_m = *hs(2, tx + 1, 3 + W);
        eyh_o = *es(1, tx, W);
        ezh_o = *es(2, tx, W);
        muh = *ms(tx, W);
      } else {
        hxh = __ldg(Hx + nhc);
        if (jh > 0) hxh_jm = __ldg(Hx + nhc - nx);
        hyh = __ldg(Hy + nhc);
        hyh_m = __ldg(Hy + nhc - 1);
        hzh = __ldg(Hz + nhc);
        hzh_m = __ldg(Hz + nhc - 1);
        eyh_o = __ldg(a.Ein + nc + nhc);
        ezh_o = __ldg(a.Ein + 2 * nc + nhc);
        muh = __ldg(emat + nhc);
      }
    }
    const T hy_s = __shfl_up_sync(0xffffffffu, hy[VW - 1], 1), hz_s = __shfl_up_sync(0xffffffffu, hz[VW - 1], 1);
    if (tx > 0) { hy_l = hy_s; hz_l = hz_s; }
    // E^{n+1}(k) on the own cells
    T ox[VW], oy[VW], oz[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) ox[e] = oy[e] = oz[e] = T(0);
    if (live && inbox) {
      const T rzd = ax(AX_RDD, nx + ny + k);
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int i = i0 + e;
        const T hy_im = e == 0 ? hy_l : hy[e - 1], hz_im = e == 0 ? hz_l : hz[e - 1];
        T cax, cbx, cay, cby, caz, cbz;
        if (mu[e] != none) {
          cax = cay = caz = __ldg(a.ctab + mu[e]);
          cbx = cby = cbz = __ldg(a.ctab + a.nmat + mu[e]);
        } else {
          const int64_t c = n + e;
          const T wxl = ax(AX_WLO, i), wxh = ax(AX_WHI, i);
          const T wzl = ax(AX_WLO, nx + ny + k), wzh = ax(AX_WHI, nx + ny + k);
          const ID m = M[c];
          const ID m_i = i > 0 ? M[c - 1] : m, m_j = j > 0 ? M[c - nx] : m, m_k = k > 0 ? M[c - plane] : m;
          const ID m_ij = (i > 0 && j > 0) ? M[c - 1 - nx] : m, m_ik = (i > 0 && k > 0) ? M[c - 1 - plane] : m;
          const ID m_jk = (j > 0 && k > 0) ? M[c - nx - plane] : m;
          e_coef(a, m_jk, m_k, m_j, m, wyl, wyh, wzl, wzh, cax, cbx);
          e_coef(a, m_ik, m_k, m_i, m, wxl, wxh, wzl, wzh, cay, cby);
          e_coef(a, m_ij, m_j, m_i, m, wxl, wxh, wyl, wyh, caz, cbz);
        }
        if (j == 0 || k == 0) cax = cbx = T(0);
        if (i == 0 || k == 0) cay = cby = T(0);
        if (i == 0 || j == 0) caz = cbz = T(0);
        ox[e] = cax * ex[e] + cbx * ((hz[e] - hz_jm[e]) * ryd - (hy[e] - hy_p[e]) * rzd);
        oy[e] = cay * ey[e] + cby * ((hx[e] - hx_p[e]) * rzd - (hz[e] - hz_im) * rxd[e]);
        oz[e] = caz * ez[e] + cbz * ((hy[e] - hy_im) * rxd[e] - (hx[e] - hx_jm[e]) * ryd);
      }
      if (!top && !halo && ok) {
        stv<VW>(a.Eout + n, ox);
        stv<VW>(a.Eout + nc + n, oy);
        stv<VW>(a.Eout + 2 * nc + n, oz);
      }
    }
    if (halo && tx < OWN) {
      T eyh = T(0), ezh = T(0);
      if (xl && inbox) {
        T ca1, cb1, ca2, cb2;
        if (muh != none) {
          ca1 = ca2 = __ldg(a.ctab + muh);
          cb1 = cb2 = __ldg(a.ctab + a.nmat + muh);
        } else {
          const int64_t c = nhc;
          const T wzl = ax(AX_WLO, nx + ny + k), wzh = ax(AX_WHI, nx + ny + k);
          const T wxlh = ax(AX_WLO, ih), wxhh = ax(AX_WHI, ih);
          const T wylh = ax(AX_WLO, nx + jh), wyhh = ax(AX_WHI, nx + jh);
          const ID m = M[c], m_i = M[c - 1], m_j = jh > 0 ? M[c - nx] : m, m_k = k > 0 ? M[c - plane] : m;
          const ID m_ij = jh > 0 ? M[c - 1 - nx] : m, m_ik = k > 0 ? M[c - 1 - plane] : m;
          e_coef(a, m_ik, m_k, m_i, m, wxlh, wxhh, wzl, wzh, ca1, cb1);
          e_coef(a, m_ij, m_j, m_i, m, wxlh, wxhh, wylh, wyhh, ca2, cb2);
        }
        if (k == 0) ca1 = cb1 = T(0);
        if (jh == 0) ca2 = cb2 = T(0);
        const T rzd = ax(AX_RDD, nx + ny + k);
        eyh = ca1 * eyh_o + cb1 * ((hxh - hxh_p) * rzd - (hzh - hzh_m) * rxdh);
        ezh = ca2 * ezh_o + cb2 * ((hyh - hyh_m) * rxdh - (hxh - hxh_jm) * rydh);
        hxh_p = hxh;
      }
      sh[b][0][tx] = eyh;
      sh[b][1][tx] = ezh;
    }
    // publish the y neighbours of the row below
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      sx[b][ty][tx * VW + e] = ox[e];
      sz[b][ty][tx * VW + e] = oz[e];
    }
    // H^{n+3/2}(k - 1) from E^{n+1}(k - 1) (own, the next lane's, and the row
    // above's and the halo column's shared at k - 1 & 1, complete since the last
    // barrier) and E^{n+1}(k) (own)
    const int bp = b ^ 1;
    T eyx = __shfl_down_sync(0xffffffffu, ey_p[0], 1), ezx = __shfl_down_sync(0xffffffffu, ez_p[0], 1);
    if (tx == LTX - 1 && !halo) {
      eyx = sh[bp][0][ty];
      ezx = sh[bp][1][ty];
    }
    if (k > k0 && !halo && live && ok) {
      const int kh = k - 1;
      const int64_t nh = n - plane;
      const T rdz = ax(AX_RD, nx + ny + kh);
      T nhx[VW], nhy[VW], nhz[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int i = i0 + e;
        T da[3] = {da0, da0, da0}, db[3] = {db0, db0, db0};
        if (!HOMOG_H) {
          const int64_t c = nh + e;
          const ID m = M[c];
          if (i > 0) h_coef(a, M[c - 1], m, ax(AX_WLO, i), ax(AX_WHI, i), da[0], db[0]);
          if (j > 0) h_coef(a, M[c - nx], m, ax(AX_WLO, nx + j), ax(AX_WHI, nx + j), da[1], db[1]);
          if (kh > 0) h_coef(a, M[c - plane], m, ax(AX_WLO, nx + ny + kh), ax(AX_WHI, nx + ny + kh), da[2], db[2]);
        }
        const T ey_ip = e == VW - 1 ? eyx : ey_p[e + 1], ez_ip = e == VW - 1 ? ezx : ez_p[e + 1];
        const T exy = sx[bp][ty + 1][tx * VW + e], ezy = sz[bp][ty + 1][tx * VW + e];
        const T hxv = da[0] * hx_p[e] - db[0] * ((ezy - ez_p[e]) * rdy - (oy[e] - ey_p[e]) * rdz);
        const T hyv = da[1] * hy_p[e] - db[1] * ((ox[e] - ex_p[e]) * rdz - (ez_ip - ez_p[e]) * rdx[e]);
        const T hzv = da[2] * hz_p[e] - db[2] * ((ey_ip - ey_p[e]) * rdx[e] - (exy - ex_p[e]) * rdy);
        nhx[e] = i == 0 ? T(0) : hxv;
        nhy[e] = j == 0 ? T(0) : hyv;
        nhz[e] = kh == 0 ? T(0) : hzv;
      }
      stv<VW>(a.Hout + nh, nhx);
      stv<VW>(a.Hout + nc + nh, nhy);
      stv<VW>(a.Hout + 2 * nc + nh, nhz);
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      hx_p[e] = hx[e];
      hy_p[e] = hy[e];
      hz_p[e] = hz[e];
      ex_p[e] = ox[e];
      ey_p[e] = oy[e];
      ez_p[e] = oz[e];
    }
    // plane k's shared values are complete, and plane k - 1's are no longer
    // read, before the next plane overwrites that slot
    if constexpr (STAGED) {
      if (__syncthreads_or(!ok)) break;
      // every thread is done with slot r % S: refill it with plane r + S
      if (tid == 0 && r + St::S < nload) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(r + St::S);
      }
    } else {
      __syncthreads();
    }
  }
  if constexpr (STAGED) {
    if (!ok) {
      // a wait gave up: record it, then let the copies in flight land
      // (bounded) before the CTA's shared memory is released
      if (tid == 0) {
        atomicExch(err, 1u);
        for (int rr = waited + 1; rr <= issued; ++rr) mbar_wait(&bars[rr % St::S], (rr / St::S) & 1);
      }
      __syncthreads();
    }
  }
  }
  allow_next_grid();
}

// Sources after the fused pass: E^{n+1}_e += dE = -Cb w u on each source edge
// and H^{n+3/2} -= Db (curlE dE) on the four H edges whose curl contains it.
struct FlatPort {
  int64_t cell;
  int comp, port;
  double w;
};

// The terms of source entry f, per unit of its port's u: dE = -Cb w on its E
// edge, then -Db (curlE dE) on each H edge whose curl contains that edge.
// emit(offset from the E base of the field buffer, factor).
template <typename T, typename ID, bool HOMOG_H, typename Emit>
__device__ __forceinline__ void src_terms(const YeeArgs<T, ID> &a, const FlatPort &f, Emit emit) {
  const int nx = a.nx, ny = a.ny, ntot = nx + ny + a.nz;
  const int64_t nc = a.nc, plane = (int64_t)nx * ny, n = f.cell;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / plane);
  auto ax = [&](int table, int idx) { return __ldg(a.ax + table * ntot + idx); };
  const ID *M = a.mat;
  T ca, cb = 0;
  const int c = f.comp;
  if (c == 0 && j > 0 && k > 0)
    e_coef(a, M[n - nx - plane], M[n - plane], M[n - nx], M[n], ax(AX_WLO, nx + j), ax(AX_WHI, nx + j),
           ax(AX_WLO, nx + ny + k), ax(AX_WHI, nx + ny + k), ca, cb);
  else if (c == 1 && i > 0 && k > 0)
    e_coef(a, M[n - 1 - plane], M[n - plane], M[n - 1], M[n], ax(AX_WLO, i), ax(AX_WHI, i),
           ax(AX_WLO, nx + ny + k), ax(AX_WHI, nx + ny + k), ca, cb);
  else if (c == 2 && i > 0 && j > 0)
    e_coef(a, M[n - 1 - nx], M[n - nx], M[n - 1], M[n], ax(AX_WLO, i), ax(AX_WHI, i), ax(AX_WLO, nx + j),
           ax(AX_WHI, nx + j), ca, cb);
  const T dE = -cb * (T)f.w;
  if (dE == T(0)) return;
  emit(c * nc + n, dE);
  // Db of H component hc at cell (ii, jj, kk), 0 where the update forces H to 0
  auto dbh = [&](int hc, int ii, int jj, int kk) -> T {
    if (ii < 0 || jj < 0 || kk < 0) return T(0);
    if ((hc == 0 && ii == 0) || (hc == 1 && jj == 0) || (hc == 2 && kk == 0)) return T(0);
    T da = __ldg(a.ctab + 2 * a.nmat), db = __ldg(a.ctab + 3 * a.nmat);
    if (!HOMOG_H) {
      const int64_t cc = kk * plane + (int64_t)jj * nx + ii;
      const int idx = hc == 0 ? ii : (hc == 1 ? nx + jj : nx + ny + kk);
      const int64_t lo = hc == 0 ? cc - 1 : (hc == 1 ? cc - nx : cc - plane);
      h_coef(a, M[lo], M[cc], ax(AX_WLO, idx), ax(AX_WHI, idx), da, db);
    }
    return db;
  };
  auto addh = [&](int hc, int ii, int jj, int kk, T coef) {
    const T db = dbh(hc, ii, jj, kk);
    if (db != T(0)) emit(3 * nc + hc * nc + kk * plane + (int64_t)jj * nx + ii, -db * coef * dE);
  };
  // (curl E)_hc at an H edge = sum of +-(1/d) E over its face; the terms of this E edge:
  if (c == 0) {         // Ex(i,j,k): Hy(i,j,k) -1/dz_k, Hy(i,j,k-1) +1/dz_{k-1}, Hz(i,j,k) +1/dy_j, Hz(i,j-1,k) -1/dy_{j-1}
    addh(1, i, j, k, -ax(AX_RD, nx + ny + k));
    if (k > 0) addh(1, i, j, k - 1, ax(AX_RD, nx + ny + k - 1));
    addh(2, i, j, k, ax(AX_RD, nx + j));
    if (j > 0) addh(2, i, j - 1, k, -ax(AX_RD, nx + j - 1));
  } else if (c == 1) {  // Ey(i,j,k): Hz(i,j,k) -1/dx_i, Hz(i-1,j,k) +1/dx_{i-1}, Hx(i,j,k) +1/dz_k, Hx(i,j,k-1) -1/dz_{k-1}
    addh(2, i, j, k, -ax(AX_RD, i));
    if (i > 0) addh(2, i - 1, j, k, ax(AX_RD, i - 1));
    addh(0, i, j, k, ax(AX_RD, nx + ny + k));
    if (k > 0) addh(0, i, j, k - 1, -ax(AX_RD, nx + ny + k - 1));
  } else {              // Ez(i,j,k): Hx(i,j,k) -1/dy_j, Hx(i,j-1,k) +1/dy_{j-1}, Hy(i,j,k) +1/dx_i, Hy(i-1,j,k) -1/dx_{i-1}
    addh(0, i, j, k, -ax(AX_RD, nx + j));
    if (j > 0) addh(0, i, j - 1, k, ax(AX_RD, nx + j - 1));
    addh(1, i, j, k, ax(AX_RD, i));
    if (i > 0) addh(1, i - 1, j, k, -ax(AX_RD, i - 1));
  }
}

template <typename T, typename ID, bool HOMOG_H>
__global__ void yee_march_src_kernel(YeeArgs<T, ID> a, const FlatPort *__restrict__ src, int nsrc) {
  wait_prior_grid();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nsrc && dcheck(a.err, src[q].cell >= 0 && src[q].cell < a.nc && src[q].comp >= 0 && src[q].comp < 3)) {
    const FlatPort f = src[q];
    const T u = a.u[f.port];
    src_terms<T, ID, HOMOG_H>(a, f, [&](int64_t off, T fac) { atomicAdd(a.Eout + off, fac * u); });
  }
  allow_next_grid();
}

// Source terms of every entry for the current coefficients (at most five per
// entry; unused slots get offset -1), gathered on the host into one term per
// (field value, port).
template <typename T, typename ID, bool HOMOG_H>
__global__ void yee_march_src_terms_kernel(YeeArgs<T, ID> a, const FlatPort *__restrict__ src, int nsrc,
                                           int64_t *__restrict__ off, T *__restrict__ fac) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsrc) return;
  int used = 0;
  src_terms<T, ID, HOMOG_H>(a, src[q], [&](int64_t o, T v) {
    if (used < 5) { off[5 * (int64_t)q + used] = o; fac[5 * (int64_t)q + used] = v; ++used; }
  });
  for (; used < 5; ++used) off[5 * (int64_t)q + used] = -1;
}

// Sources and probes of one step in one launch, after the fused pass: thread
// t < nterm adds its term (one per field value and port, so no two threads
// write the same value) times u; the others read a probe entry's E^{n+1}
// (no probe edge carries a source term, checked when the terms were built).
template <typename T, typename ID>
__global__ void yee_march_fix_kernel(YeeArgs<T, ID> a, const uint32_t *__restrict__ off, const T *__restrict__ fac,
                                     const int32_t *__restrict__ port, int nterm, const FlatPort *__restrict__ prb,
                                     int nprb) {
  wait_prior_grid();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nterm) {
    if (!dcheck(a.err, off[t] < 6 * a.nc)) return;
    T *f = a.Eout + off[t];
    *f += fac[t] * a.u[port ? port[t] : 0];
  } else if (t - nterm < nprb) {
    const FlatPort pe = prb[t - nterm];
    if (!dcheck(a.err, pe.cell >= 0 && pe.cell < a.nc && pe.comp >= 0 && pe.comp < 3)) return;
    atomicAdd(&a.y[pe.port], (T)pe.w * a.Eout[pe.comp * a.nc + pe.cell]);
  }
  allow_next_grid();
}

// Probes of the final E^{n+1}.
template <typename T, typename ID>
__global__ void yee_march_prb_kernel(YeeArgs<T, ID> a, const FlatPort *__restrict__ prb, int nprb) {
  wait_prior_grid();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nprb && dcheck(a.err, prb[q].cell >= 0 && prb[q].cell < a.nc && prb[q].comp >= 0 && prb[q].comp < 3)) {
    const FlatPort f = prb[q];
    atomicAdd(&a.y[f.port], (T)f.w * a.Eout[f.comp * a.nc + f.cell]);
  }
  allow_next_grid();
}

static fdtd_status ensure_flat(fdtd_grid *g, cudaStream_t s) {
  if (g->flat_ready) return FDTD_OK;
  auto build = [&](const std::vector<HostPort> &ports, DevBuf &buf, int &count) -> fdtd_status {
    std::vector<FlatPort> v;
    for (size_t p = 0; p < ports.size(); ++p)
      for (size_t e = 0; e < ports[p].cell.size(); ++e)
        v.push_back(FlatPort{ports[p].cell[e], ports[p].comp, (int)p, ports[p].w[e]});
    count = (int)v.size();
    FDTD_CHECK(buf.alloc(std::max<size_t>(1, v.size()) * sizeof(FlatPort), s));
    if (!v.empty())
      FDTD_CHECK_CUDA(cudaMemcpyAsync(buf.ptr, v.data(), v.size() * sizeof(FlatPort), cudaMemcpyHostToDevice, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    return FDTD_OK;
  };
  FDTD_CHECK(build(g->ports, g->flat_src, g->nflat_src));
  FDTD_CHECK(build(g->probes, g->flat_prb, g->nflat_prb));
  g->flat_ready = true;
  return FDTD_OK;
}

// Gathers the sources' terms for the current coefficients (outside any graph
// capture: the first step of a run is launched directly): one term per field
// value and port, so the per-step kernel needs no atomics, and a check that no
// probe edge carries a term, so probes can share its launch.
template <typename T, typename ID, bool HH>
static fdtd_status ensure_fix(fdtd_grid *g, const YeeArgs<T, ID> &a, cudaStream_t s) {
  if (g->fix_version == g->ctab_version) return FDTD_OK;
  g->fix_one = false;
  g->nfix = 0;
  if (g->nflat_src) {
    const int n = g->nflat_src;
    DevBuf doff, dfac;
    struct Rel {
      DevBuf *a, *b;
      cudaStream_t s;
      ~Rel() { a->release(s); b->release(s); }
    } rel{&doff, &dfac, s};
    FDTD_CHECK(doff.alloc((size_t)5 * n * sizeof(int64_t), s));
    FDTD_CHECK(dfac.alloc((size_t)5 * n * sizeof(T), s));
    yee_march_src_terms_kernel<T, ID, HH><<<(n + 127) / 128, 128, 0, s>>>(a, g->flat_src.as<const FlatPort>(), n,
                                                                       doff.as<int64_t>(), dfac.as<T>());
    FDTD_CHECK(after_launch("yee_march_src_terms_kernel"));
    std::vector<int64_t> off((size_t)5 * n);
    std::vector<T> fac((size_t)5 * n);
    std::vector<FlatPort> src(n);
    FDTD_CHECK_CUDA(cudaMemcpyAsync(off.data(), doff.ptr, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaMemcpyAsync(fac.data(), dfac.ptr, fac.size() * sizeof(T), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaMemcpyAsync(src.data(), g->flat_src.ptr, n * sizeof(FlatPort), cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
    struct Term {
      int64_t off;
      int port;
      T fac;
    };
    std::vector<Term> t;
    t.reserve(off.size());
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < 5; ++r)
        if (off[5 * (size_t)q + r] >= 0) t.push_back(Term{off[5 * (size_t)q + r], src[q].port, fac[5 * (size_t)q + r]});
    std::sort(t.begin(), t.end(), [](const Term &x, const Term &y) { return x.off != y.off ? x.off < y.off : x.port < y.port; });
    std::vector<int64_t> uo;
    std::vector<T> uf;
    std::vector<int32_t> up;
    for (size_t q = 0; q < t.size(); ++q) {
      if (!uo.empty() && uo.back() == t[q].off && up.back() == t[q].port) uf.back() += t[q].fac;
      else { uo.push_back(t[q].off); uf.push_back(t[q].fac); up.push_back(t[q].port); }
    }
    // one writer per field value: the same value under two ports would race
    bool unique = true;
    for (size_t q = 1; q < uo.size(); ++q) unique &= uo[q] != uo[q - 1];
    bool disjoint = true;
    if (g->nflat_prb) {
      std::vector<FlatPort> prb(g->nflat_prb);
      FDTD_CHECK_CUDA(cudaMemcpyAsync(prb.data(), g->flat_prb.ptr, prb.size() * sizeof(FlatPort),
                                      cudaMemcpyDeviceToHost, s));
      FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
      for (const FlatPort &pe : prb)
        disjoint &= !std::binary_search(uo.begin(), uo.end(), pe.comp * g->nc + pe.cell);
    }
    if (unique && !uo.empty() && 6 * g->nc <= (int64_t)UINT32_MAX) {
      g->nfix = (int)uo.size();
      // 32-bit offsets (the grid is checked below 2^32 field values) and no
      // port array on single-port grids: 8 bytes of term data per value
      const std::vector<uint32_t> u32(uo.begin(), uo.end());
      FDTD_CHECK(g->fix_off.alloc(u32.size() * sizeof(uint32_t), s));
      FDTD_CHECK(g->fix_fac.alloc(uf.size() * sizeof(T), s));
      FDTD_CHECK_CUDA(cudaMemcpyAsync(g->fix_off.ptr, u32.data(), u32.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      FDTD_CHECK_CUDA(cudaMemcpyAsync(g->fix_fac.ptr, uf.data(), uf.size() * sizeof(T), cudaMemcpyHostToDevice, s));
      g->fix_port.release(s);
      if (g->ports.size() > 1) {
        FDTD_CHECK(g->fix_port.alloc(up.size() * sizeof(int32_t), s));
        FDTD_CHECK_CUDA(cudaMemcpyAsync(g->fix_port.ptr, up.data(), up.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      }
      FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
      g->fix_one = disjoint;
    }
  }
  g->fix_version = g->ctab_version;
  return FDTD_OK;
}

// Tensor maps of the staged form for both state buffers of the last grid
// used, keyed on everything they encode (a later grid may reuse the same
// device addresses with other sizes or id width).
struct MarchMapCache {
  MarchMaps maps[2];
  const void *f0 = nullptr, *f1 = nullptr, *emat = nullptr;
  int nx = 0, ny = 0, nz = 0, id_bytes = 0;
  bool same(const fdtd_grid *g) const {
    return f0 == g->fields[0].ptr && f1 == g->fields[1].ptr && emat == g->emat.ptr && nx == g->nx && ny == g->ny &&
           nz == g->nz && id_bytes == g->id_bytes;
  }
};

// The staged form needs 16-byte rows of the fields and of the material map.
static bool march_staged_ok(const fdtd_grid *g) {
  if (const char *e = getenv("FDTDMOR_MARCH_TMA")) return atoi(e) != 0 && encode_fn() != nullptr;
  return g->prec == FDTD_F32 && g->nx % 4 == 0 && (g->nx * g->id_bytes) % 16 == 0 && encode_fn() != nullptr;
}

template <typename ID>
static fdtd_status march_maps(fdtd_grid *g, const MarchMaps **out) {
  static thread_local MarchMapCache cache;
  if (!cache.same(g)) {
    using St = MarchStage<ID>;
    for (int b = 0; b < 2; ++b) {
      char *base = static_cast<char *>(g->fields[b].ptr);
      for (int c = 0; c < 3; ++c) {
        FDTD_CHECK(make_map(&cache.maps[b].E[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base + (size_t)c * g->nc * 4, g,
                            St::EX, St::EY));
        FDTD_CHECK(make_map(&cache.maps[b].H[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base + (size_t)(3 + c) * g->nc * 4,
                            g, St::HX, St::HY));
      }
      FDTD_CHECK(make_map(&cache.maps[b].M, sizeof(ID) == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                          (int)sizeof(ID), g->emat.ptr, g, St::MX, St::MY));
    }
    cache.f0 = g->fields[0].ptr; cache.f1 = g->fields[1].ptr; cache.emat = g->emat.ptr;
    cache.nx = g->nx; cache.ny = g->ny; cache.nz = g->nz; cache.id_bytes = g->id_bytes;
  }
  *out = &cache.maps[g->cur];
  return FDTD_OK;
}

template <typename T, typename ID, bool HH, int VW, int MTY, bool STAGED>
static fdtd_status launch_march_main(fdtd_grid *g, const YeeArgs<T, ID> &a, cudaStream_t s) {
  auto kern = yee_march_kernel<T, ID, HH, VW, MTY, STAGED>;
  const size_t smem = STAGED ? MarchStage<ID>::SMEM : 0;
  static int per_sm = 0;
  if (!per_sm) {
    if (STAGED) FDTD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FDTD_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LTX * MTY, smem));
    per_sm = std::max(1, per_sm);
  }
  const int ntx = (g->nx + LTX * VW - 1) / (LTX * VW), nty = (g->ny + MTY - 2) / (MTY - 1);
  const char *lz_env = getenv("FDTDMOR_LZ");
  const int lz = std::min(g->nz, lz_env ? env_int("FDTDMOR_LZ", 16) : choose_kchunk(g, ntx * nty, per_sm));
  const dim3 grid(ntx, nty, (g->nz + lz - 1) / lz);
  MarchMaps none_maps;
  memset(&none_maps, 0, sizeof(none_maps));
  const MarchMaps *mp = &none_maps;
  if (STAGED) FDTD_CHECK(march_maps<ID>(g, &mp));
  FDTD_CHECK_CUDA(launch_dependent_smem(kern, grid, dim3(LTX, MTY), smem, s, a, g->emat.as<ID>(), lz, *mp,
                                        g->errflag.as<unsigned>()));
  return FDTD_OK;
}

template <typename T, typename ID, bool HH, int VW, int MTY>
static fdtd_status launch_march_v(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s) {
  FDTD_CHECK(ensure_emat<ID>(g, s));
  FDTD_CHECK(ensure_flat(g, s));
  YeeArgs<T, ID> a = split_args<T, ID>(g);
  FDTD_CHECK((ensure_fix<T, ID, HH>(g, a, s)));
  a.u = static_cast<const T *>(u_row);
  a.y = static_cast<T *>(y_row);
  if constexpr (sizeof(T) == 4 && VW == 4 && MTY == 8) {
    if (march_staged_ok(g)) FDTD_CHECK((launch_march_main<T, ID, HH, VW, MTY, true>(g, a, s)));
    else FDTD_CHECK((launch_march_main<T, ID, HH, VW, MTY, false>(g, a, s)));
  } else {
    FDTD_CHECK((launch_march_main<T, ID, HH, VW, MTY, false>(g, a, s)));
  }
  FDTD_CHECK(after_launch("yee_march_kernel"));
  if (g->nfix && g->fix_one) {  // gathered source terms and the probes in one launch
    const int nt = g->nfix + g->nflat_prb;
    FDTD_CHECK_CUDA(launch_dependent(yee_march_fix_kernel<T, ID>, dim3((nt + 255) / 256), dim3(256), s, a,
                                     g->fix_off.as<const uint32_t>(), g->fix_fac.as<const T>(),
                                     g->fix_port.as<const int32_t>(), g->nfix, g->flat_prb.as<const FlatPort>(),
                                     g->nflat_prb));
    FDTD_CHECK(after_launch("yee_march_fix_kernel"));
    return FDTD_OK;
  }
  if (g->nfix) {
    FDTD_CHECK_CUDA(launch_dependent(yee_march_fix_kernel<T, ID>, dim3((g->nfix + 255) / 256), dim3(256), s, a,
                                     g->fix_off.as<const uint32_t>(), g->fix_fac.as<const T>(),
                                     g->fix_port.as<const int32_t>(), g->nfix, g->flat_prb.as<const FlatPort>(), 0));
    FDTD_CHECK(after_launch("yee_march_fix_kernel"));
  } else if (g->nflat_src) {
    FDTD_CHECK_CUDA(launch_dependent(yee_march_src_kernel<T, ID, HH>, dim3((g->nflat_src + 127) / 128), dim3(128), s, a,
                                     g->flat_src.as<const FlatPort>(), g->nflat_src));
    FDTD_CHECK(after_launch("yee_march_src_kernel"));
  }
  if (g->nflat_prb) {
    FDTD_CHECK_CUDA(launch_dependent(yee_march_prb_kernel<T, ID>, dim3((g->nflat_prb + 127) / 128), dim3(128), s, a,
                                     g->flat_prb.as<const FlatPort>(), g->nflat_prb));
    FDTD_CHECK(after_launch("yee_march_prb_kernel"));
  }
  return FDTD_OK;
}

// Cells per thread: 16-byte rows (4 FP32 values) on grids wide enough to fill
// the 128-cell tiles, else the split form's width.
int yee_march_vw(const fdtd_grid *g) {
  if (const char *e = getenv("FDTDMOR_MARCH_VW")) {
    const int v = atoi(e);
    if ((v == 1 || v == 2 || (v == 4 && g->elem == 4)) && g->nx % v == 0) return v;
  }
  if (g->elem == 4 && g->nx % 4 == 0 && g->nx >= 256) return 4;
  return yee_split_vw(g);
}

template <typename T, typename ID, bool HH>
static fdtd_status launch_march_t(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s) {
  const int vw = yee_march_vw(g);
  if constexpr (sizeof(T) == 4)
    if (vw == 4) return launch_march_v<T, ID, HH, 4, 8>(g, u_row, y_row, s);
  if (vw == 2) return launch_march_v<T, ID, HH, 2, 8>(g, u_row, y_row, s);
  return launch_march_v<T, ID, HH, 1, 8>(g, u_row, y_row, s);
}

fdtd_status launch_yee_march(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s) {
  if (g->prec == FDTD_F64) {
    if (g->id_bytes == 1)
      return g->homog_h ? launch_march_t<double, uint8_t, true>(g, u_row, y_row, s)
                        : launch_march_t<double, uint8_t, false>(g, u_row, y_row, s);
    return g->homog_h ? launch_march_t<double, uint16_t, true>(g, u_row, y_row, s)
                      : launch_march_t<double, uint16_t, false>(g, u_row, y_row, s);
  }
  if (g->id_bytes == 1)
    return g->homog_h ? launch_march_t<float, uint8_t, true>(g, u_row, y_row, s)
                      : launch_march_t<float, uint8_t, false>(g, u_row, y_row, s);
  return g->homog_h ? launch_march_t<float, uint16_t, true>(g, u_row, y_row, s)
                    : launch_march_t<float, uint16_t, false>(g, u_row, y_row, s);
}

}  // namespace fdtdmor
