// Shared pieces of the Yee leap-frog kernels (yee.cu, yee_tma.cu, yee_split.cu): kernel
// arguments and the per-edge update coefficients of Eq. (matrix).
#pragma once
#include "common.cuh"

namespace fdtdmor {

template <typename T, typename ID>
struct YeeArgs {
  int nx, ny, nz, kchunk;
  int ntx, nty;                // xy-tile counts of the source/probe lists
  int64_t nc;
  const T *__restrict__ Ein;   // 3 components, stride nc
  const T *__restrict__ Hin;
  T *__restrict__ Eout;
  T *__restrict__ Hout;
  const ID *__restrict__ mat;
  const T *__restrict__ ax;    // axis tables (AX_COUNT x (nx+ny+nz))
  const T *__restrict__ mtab;  // eps, sig, mu, sigm, pec (5 x nmat)
  const T *__restrict__ ctab;  // ca, cb, da, db (4 x nmat)
  const T *__restrict__ ecoef; // per-edge Ca (3 x nc) then Cb (3 x nc), or null
  int nmat;
  T inv_dt;
  const int32_t *__restrict__ src_ptr;
  const PortEntry *__restrict__ src;
  const T *__restrict__ u;     // row of this step: u[port]
  const int32_t *__restrict__ prb_ptr;
  const PortEntry *__restrict__ prb;
  T *__restrict__ y;           // row of this step: y[probe]
  unsigned *err = nullptr;     // the grid's error flag (index checks of the checked build)
};

template <typename T>
__device__ __forceinline__ T axv(const T *ax, int ntot, int table, int idx) {
  return __ldg(ax + table * ntot + idx);
}

// (Ca, Cb) of an E edge from the four cells around it (c00: lo/lo, c10: hi/lo,
// c01: lo/hi, c11: hi/hi along the two transverse axes) and their weights.
template <typename T, typename ID>
__device__ __forceinline__ void e_coef(const YeeArgs<T, ID> &a, ID c00, ID c10, ID c01, ID c11,
                                       T wa_lo, T wa_hi, T wb_lo, T wb_hi, T &ca, T &cb) {
  if (c00 == c10 && c00 == c01 && c00 == c11) {
    ca = __ldg(a.ctab + c00);
    cb = __ldg(a.ctab + a.nmat + c00);
    return;
  }
  const T *pec = a.mtab + 4 * a.nmat;
  if (__ldg(pec + c00) != T(0) || __ldg(pec + c10) != T(0) || __ldg(pec + c01) != T(0) ||
      __ldg(pec + c11) != T(0)) {
    ca = T(0);
    cb = T(0);
    return;
  }
  const T *eps = a.mtab, *sig = a.mtab + a.nmat;
  T w00 = wa_lo * wb_lo, w10 = wa_hi * wb_lo, w01 = wa_lo * wb_hi, w11 = wa_hi * wb_hi;
  T e = w00 * __ldg(eps + c00) + w10 * __ldg(eps + c10) + w01 * __ldg(eps + c01) + w11 * __ldg(eps + c11);
  T s = w00 * __ldg(sig + c00) + w10 * __ldg(sig + c10) + w01 * __ldg(sig + c01) + w11 * __ldg(sig + c11);
  T ae = e * a.inv_dt;
  cb = T(1) / (ae + T(0.5) * s);
  ca = (ae - T(0.5) * s) * cb;
}

// (Da, Db) of an H edge from the two cells its dual edge crosses.
template <typename T, typename ID>
__device__ __forceinline__ void h_coef(const YeeArgs<T, ID> &a, ID c0, ID c1, T w0, T w1, T &da,
                                       T &db) {
  if (c0 == c1) {
    da = __ldg(a.ctab + 2 * a.nmat + c0);
    db = __ldg(a.ctab + 3 * a.nmat + c0);
    return;
  }
  const T *mu = a.mtab + 2 * a.nmat, *sgm = a.mtab + 3 * a.nmat;
  T m = w0 * __ldg(mu + c0) + w1 * __ldg(mu + c1);
  T s = w0 * __ldg(sgm + c0) + w1 * __ldg(sgm + c1);
  T am = m * a.inv_dt;
  db = T(1) / (am + T(0.5) * s);
  da = (am - T(0.5) * s) * db;
}


bool yee_tma_eligible(const fdtd_grid *g);
void yee_tma_tile(int *tx, int *ty);
int yee_split_vw(const fdtd_grid *g);
int yee_split_lz(const fdtd_grid *g);
fdtd_status launch_yee_march(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s);
int choose_kchunk(const fdtd_grid *g, int ntiles, int ctas_per_sm);
int yee_march_vw(const fdtd_grid *g);
bool yee_split_precoef(const fdtd_grid *g);
fdtd_status launch_yee_split(fdtd_grid *g, const void *u_row, void *y_row, cudaStream_t s);
fdtd_status run_yee_stream(fdtd_grid *g, int64_t nsteps, const void *u, void *y, cudaStream_t s);
fdtd_status launch_yee_tma(fdtd_grid *g, const void *u_row, void *y_row, int kchunk, cudaStream_t s);

}  // namespace fdtdmor
