// Device helpers shared by the reduction kernels: complex arithmetic, the two
// discrete curls of Eq. (matrix) in the per-volume form, per-edge material
// properties and the reduction handles.
#pragma once

#include "common.cuh"

namespace fdtdmor {

template <typename T>
struct cplx {
  T re, im;
  __host__ __device__ cplx() : re(0), im(0) {}
  __host__ __device__ cplx(T r, T i = T(0)) : re(r), im(i) {}
};
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T> __host__ __device__ __forceinline__ T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cdiv(cplx<T> a, cplx<T> b) {
  T d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
template <typename T, typename U> __host__ __device__ __forceinline__ cplx<T> ccast(cplx<U> a) { return {(T)a.re, (T)a.im}; }
// FP32 coefficient times an FP64 complex value (the FP64 residual of the
// refinement loop reads the FP32 axis tables and material properties).
__host__ __device__ __forceinline__ cplx<double> operator*(float s, cplx<double> a) {
  return {(double)s * a.re, (double)s * a.im};
}

// Geometry view for stencils over the storage layout.
template <typename T>
struct Geo {
  int nx, ny, nz;
  int64_t nc;
  const T *ax;  // axis tables
  __device__ __forceinline__ int ntot() const { return nx + ny + nz; }
  __device__ __forceinline__ T rd(int axis, int i) const { return __ldg(ax + AX_RD * ntot() + off(axis) + i); }
  __device__ __forceinline__ T rdd(int axis, int i) const { return __ldg(ax + AX_RDD * ntot() + off(axis) + i); }
  __device__ __forceinline__ int off(int axis) const { return axis == 0 ? 0 : (axis == 1 ? nx : nx + ny); }
  __device__ __forceinline__ int64_t id(int i, int j, int k) const { return ((int64_t)k * ny + j) * nx + i; }
};

// (i, j, k) of linear cell index n (x fastest), with 32-bit divisions when the
// grid has fewer than 2^32 cells.
__device__ __forceinline__ void cell_ijk(int64_t n, int nx, int ny, int64_t nc, int &i, int &j, int &k) {
  if (nc <= 0xffffffffll) {
    const unsigned u = (unsigned)n, q = u / (unsigned)nx;
    i = (int)(u - q * (unsigned)nx);
    j = (int)(q % (unsigned)ny);
    k = (int)(q / (unsigned)ny);
  } else {
    i = (int)(n % nx);
    j = (int)((n / nx) % ny);
    k = (int)(n / ((int64_t)nx * ny));
  }
}

// (curl E)_c at H edge (i, j, k) of a 3-component vector field x (stride nc),
// values outside the box are zero (tangential E on the PEC walls).
template <typename T, typename V, typename LD>
__device__ __forceinline__ V curl_e_at(const Geo<T> &g, LD ld, int c, int i, int j, int k) {
  const int64_t n = g.id(i, j, k), nc = g.nc;
  V z(0);
  if (c == 0) {
    V ezp = (j + 1 < g.ny) ? ld(2 * nc + g.id(i, j + 1, k)) : z;
    V eyp = (k + 1 < g.nz) ? ld(1 * nc + g.id(i, j, k + 1)) : z;
    return g.rd(1, j) * (ezp - ld(2 * nc + n)) - g.rd(2, k) * (eyp - ld(1 * nc + n));
  } else if (c == 1) {
    V exp_ = (k + 1 < g.nz) ? ld(0 * nc + g.id(i, j, k + 1)) : z;
    V ezp = (i + 1 < g.nx) ? ld(2 * nc + g.id(i + 1, j, k)) : z;
    return g.rd(2, k) * (exp_ - ld(0 * nc + n)) - g.rd(0, i) * (ezp - ld(2 * nc + n));
  } else {
    V eyp = (i + 1 < g.nx) ? ld(1 * nc + g.id(i + 1, j, k)) : z;
    V exp_ = (j + 1 < g.ny) ? ld(0 * nc + g.id(i, j + 1, k)) : z;
    return g.rd(0, i) * (eyp - ld(1 * nc + n)) - g.rd(1, j) * (exp_ - ld(0 * nc + n));
  }
}

// (curl H)_c at E edge (i, j, k) of a 3-component vector field t.
template <typename T, typename V, typename LD>
__device__ __forceinline__ V curl_h_at(const Geo<T> &g, LD ld, int c, int i, int j, int k) {
  const int64_t n = g.id(i, j, k), nc = g.nc;
  V z(0);
  if (c == 0) {
    V hzm = (j > 0) ? ld(2 * nc + g.id(i, j - 1, k)) : z;
    V hym = (k > 0) ? ld(1 * nc + g.id(i, j, k - 1)) : z;
    return g.rdd(1, j) * (ld(2 * nc + n) - hzm) - g.rdd(2, k) * (ld(1 * nc + n) - hym);
  } else if (c == 1) {
    V hxm = (k > 0) ? ld(0 * nc + g.id(i, j, k - 1)) : z;
    V hzm = (i > 0) ? ld(2 * nc + g.id(i - 1, j, k)) : z;
    return g.rdd(2, k) * (ld(0 * nc + n) - hxm) - g.rdd(0, i) * (ld(2 * nc + n) - hzm);
  } else {
    V hym = (i > 0) ? ld(1 * nc + g.id(i - 1, j, k)) : z;
    V hxm = (j > 0) ? ld(0 * nc + g.id(i, j - 1, k)) : z;
    return g.rdd(0, i) * (ld(1 * nc + n) - hym) - g.rdd(1, j) * (ld(0 * nc + n) - hxm);
  }
}

// All three components of curl E at cell (i, j, k) (linear index n) from the
// nine values they need, each loaded once (values outside the box are zero).
template <typename T, typename V, typename LD>
__device__ __forceinline__ void curl_e3(const Geo<T> &g, LD ld, int i, int j, int k, int64_t n, V out[3]) {
  const int64_t nc = g.nc, sy = g.nx, sz = (int64_t)g.nx * g.ny;
  const V z(0);
  const bool ip = i + 1 < g.nx, jp = j + 1 < g.ny, kp = k + 1 < g.nz;
  const V ex = ld(n), ey = ld(nc + n), ez = ld(2 * nc + n);
  const V ez_jp = jp ? ld(2 * nc + n + sy) : z, ey_kp = kp ? ld(nc + n + sz) : z;
  const V ex_kp = kp ? ld(n + sz) : z, ez_ip = ip ? ld(2 * nc + n + 1) : z;
  const V ey_ip = ip ? ld(nc + n + 1) : z, ex_jp = jp ? ld(n + sy) : z;
  const T rx = g.rd(0, i), ry = g.rd(1, j), rz = g.rd(2, k);
  out[0] = ry * (ez_jp - ez) - rz * (ey_kp - ey);
  out[1] = rz * (ex_kp - ex) - rx * (ez_ip - ez);
  out[2] = rx * (ey_ip - ey) - ry * (ex_jp - ex);
}

// All three components of curl H at cell (i, j, k), each input loaded once.
template <typename T, typename V, typename LD>
__device__ __forceinline__ void curl_h3(const Geo<T> &g, LD ld, int i, int j, int k, int64_t n, V out[3]) {
  const int64_t nc = g.nc, sy = g.nx, sz = (int64_t)g.nx * g.ny;
  const V z(0);
  const V hx = ld(n), hy = ld(nc + n), hz = ld(2 * nc + n);
  const V hz_jm = j > 0 ? ld(2 * nc + n - sy) : z, hy_km = k > 0 ? ld(nc + n - sz) : z;
  const V hx_km = k > 0 ? ld(n - sz) : z, hz_im = i > 0 ? ld(2 * nc + n - 1) : z;
  const V hy_im = i > 0 ? ld(nc + n - 1) : z, hx_jm = j > 0 ? ld(n - sy) : z;
  const T rx = g.rdd(0, i), ry = g.rdd(1, j), rz = g.rdd(2, k);
  out[0] = ry * (hz - hz_jm) - rz * (hy - hy_km);
  out[1] = rz * (hx - hx_km) - rx * (hz - hz_im);
  out[2] = rx * (hy - hy_im) - ry * (hx - hx_jm);
}

// Per-edge material properties of a grid (computed once, field type T) in
// g->eprops: E edges: eps (absolute, 0 on dead edges: walls / PEC), sig;
// H edges: mu (absolute, 0 on dead edges: normal to a wall), sgm; each 3 x nc.
enum EdgeProp { EP_EPS = 0, EP_SIG = 1, EP_MU = 2, EP_SGM = 3 };
fdtd_status ensure_edge_props(fdtd_grid *g, cudaStream_t s);

template <typename T>
Geo<T> make_geo(const fdtd_grid *g) {
  Geo<T> geo;
  geo.nx = g->nx; geo.ny = g->ny; geo.nz = g->nz; geo.nc = g->nc;
  geo.ax = g->axis.as<T>();
  return geo;
}

}  // namespace fdtdmor
