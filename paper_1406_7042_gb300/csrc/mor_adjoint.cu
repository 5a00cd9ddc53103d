// A12 (reduced model): gradient of a probe loss of the reduced leap-frog with
// respect to the per-cell relative permittivity, with the projection V frozen
// (not in the paper).  D~eps = V1^T D_eps V1 is the only reduced matrix that
// depends on eps; K~ (as prepared by mor_perturb) is held fixed.
//
// The reduced recursion, per step,
//   e' = Pe e - Qe h + be u,  h' = Ph h + Qh e' + bh u,  y = C~ e',
// with Pe = Ae^-1 Be, Qe = Ae^-1 K~, Ph = Ah^-1 Bh, Qh = Ah^-1 K~^T,
// Ae = D~e/dt + D~se/2, Be = D~e/dt - D~se/2, has the adjoint (carries eb,
// hb of e^{n+1}, h^{n+1}, backwards in n)
//   ebar = eb + C~^T dL/dy^n + Qh^T hb,  eb <- Pe^T ebar,  hb <- Ph^T hb - Qe^T ebar,
// and dL/dD~e = Ae^-1 [sum_n ebar_n (e^n - e^{n+1})^T] / dt.  One CTA runs the
// recursion forwards (keeping the differences e^n - e^{n+1}) and backwards
// (keeping ebar_n); their outer-product sum is a Gram product over the steps;
// the host applies Ae^-1 / dt to the q1 x q1 result.  Per E edge,
// dL/d eps_e = V_e v_e^T G v_e (v_e the edge's row of V1), and the edges map to
// cells by the area weights of the edge average.
#include <algorithm>
#include <cmath>
#include <vector>

#include "grid_internal.cuh"
#include "mor_common.cuh"
#include "mor_internal.cuh"

namespace fdtdmor {

template <typename T>
struct RedAdjArgs {
  int q1, q2, m, p;
  int64_t nsteps;
  const T *Pe, *Qe, *be, *Ph, *Qh, *bh, *C;
  const T *u, *dldy;
  T *dif;   // [q1][nsteps]: e^n - e^{n+1}
  T *ebar;  // [q1][nsteps]
};

template <typename T>
__device__ __forceinline__ T ra_warp_sum(T v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(1024) reduced_adjoint_kernel(RedAdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  const int q1 = a.q1, q2 = a.q2, m = a.m, p = a.p;
  const int64_t T_ = a.nsteps;
  T *e = sm, *h = e + q1, *en = h + q2, *hn = en + q1, *us = hn + q2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < q1 + q2; t += blockDim.x) sm[t] = T(0);
  __syncthreads();
  // forward from zero state
  for (int64_t n = 0; n < T_; ++n) {
    for (int t = threadIdx.x; t < m; t += blockDim.x) us[t] = a.u[n * m + t];
    __syncthreads();
    for (int r = w; r < q1; r += nw) {
      T acc = 0;
      for (int c = lane; c < q1; c += 32) acc += a.Pe[r * q1 + c] * e[c];
      for (int c = lane; c < q2; c += 32) acc -= a.Qe[r * q2 + c] * h[c];
      for (int c = lane; c < m; c += 32) acc += a.be[r * m + c] * us[c];
      acc = ra_warp_sum(acc);
      if (lane == 0) en[r] = acc;
    }
    __syncthreads();
    for (int r = w; r < q2; r += nw) {
      T acc = 0;
      for (int c = lane; c < q2; c += 32) acc += a.Ph[r * q2 + c] * h[c];
      for (int c = lane; c < q1; c += 32) acc += a.Qh[r * q1 + c] * en[c];
      for (int c = lane; c < m; c += 32) acc += a.bh[r * m + c] * us[c];
      acc = ra_warp_sum(acc);
      if (lane == 0) hn[r] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < q1; t += blockDim.x) a.dif[(int64_t)t * T_ + n] = e[t] - en[t];
    for (int t = threadIdx.x; t < q1 + q2; t += blockDim.x) sm[t] = t < q1 ? en[t] : hn[t - q1];
    __syncthreads();
  }
  // backward: e and h now hold the carries eb, hb; en, hn the new ones
  for (int t = threadIdx.x; t < q1 + q2; t += blockDim.x) sm[t] = T(0);
  T *eb = e, *hb = h, *ebar = en, *hb2 = hn, *ys = us;
  __syncthreads();
  for (int64_t n = T_ - 1; n >= 0; --n) {
    for (int t = threadIdx.x; t < p; t += blockDim.x) ys[t] = a.dldy[n * p + t];
    __syncthreads();
    // ebar = eb + C^T y + Qh^T hb   (C: p x q1, Qh: q2 x q1, row-major)
    for (int c = threadIdx.x; c < q1; c += blockDim.x) {
      T acc = eb[c];
      for (int r = 0; r < p; ++r) acc += a.C[r * q1 + c] * ys[r];
      for (int r = 0; r < q2; ++r) acc += a.Qh[r * q1 + c] * hb[r];
      ebar[c] = acc;
      a.ebar[(int64_t)c * T_ + n] = acc;
    }
    __syncthreads();
    // hb' = Ph^T hb - Qe^T ebar   (Ph: q2 x q2, Qe: q1 x q2)
    for (int c = threadIdx.x; c < q2; c += blockDim.x) {
      T acc = 0;
      for (int r = 0; r < q2; ++r) acc += a.Ph[r * q2 + c] * hb[r];
      for (int r = 0; r < q1; ++r) acc -= a.Qe[r * q2 + c] * ebar[r];
      hb2[c] = acc;
    }
    // eb' = Pe^T ebar   (Pe: q1 x q1)
    __syncthreads();
    for (int c = threadIdx.x; c < q1; c += blockDim.x) {
      T acc = 0;
      for (int r = 0; r < q1; ++r) acc += a.Pe[r * q1 + c] * ebar[r];
      eb[c] = acc;
    }
    for (int c = threadIdx.x; c < q2; c += blockDim.x) hb[c] = hb2[c];
    __syncthreads();
  }
}

// gedge[e] = V_e v_e^T G v_e for every E edge, v_e[a] = V1[a * n3 + e]; a
// block stages the rows of its edges in shared memory; the arithmetic is in
// the basis type (FP32 products summed per row, rows summed in FP64).
template <typename T>
constexpr int qf_edges() { return sizeof(T) == 4 ? 128 : 64; }

template <typename T>
__global__ void __launch_bounds__(qf_edges<T>()) quad_form_kernel(Geo<T> g, int q1, const T *__restrict__ V1,
                                                                  const T *__restrict__ G, double *__restrict__ gedge) {
  extern __shared__ __align__(16) unsigned char qf_raw[];
  T *vs = reinterpret_cast<T *>(qf_raw);  // [edges][q1 + 1]
  constexpr int NE = qf_edges<T>();
  const int64_t nc = g.nc, n3 = 3 * nc;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int ld = q1 + 1;
  for (int a = 0; a < q1; ++a) {
    const int64_t e = e0 + threadIdx.x;
    vs[threadIdx.x * ld + a] = e < n3 ? V1[(size_t)a * n3 + e] : T(0);
  }
  __syncthreads();
  const int64_t e = e0 + threadIdx.x;
  if (e >= n3) return;
  const T *v = vs + threadIdx.x * ld;
  double s = 0.0;
  for (int a = 0; a < q1; ++a) {
    T acc = 0;
    const T *Ga = G + (size_t)a * q1;
    for (int b = 0; b < q1; ++b) acc += __ldg(Ga + b) * v[b];
    s += (double)v[a] * (double)acc;
  }
  const int c = (int)(e / nc);
  const int64_t n = e - c * nc;
  int i, j, k;
  cell_ijk(n, g.nx, g.ny, nc, i, j, k);
  gedge[e] = edge_volume(g.ax, g.nx, g.ny, g.nz, c, i, j, k) * s;
}

// Cholesky solve of the SPD q x q system A X = B in place (host, FP64).
static bool chol_solve_host(std::vector<double> &A, int q, std::vector<double> &B, int nrhs) {
  for (int j = 0; j < q; ++j) {
    double d = A[(size_t)j * q + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * q + k] * A[(size_t)j * q + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * q + j] = d;
    for (int i = j + 1; i < q; ++i) {
      double v = A[(size_t)i * q + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * q + k] * A[(size_t)j * q + k];
      A[(size_t)i * q + j] = v / d;
    }
  }
  for (int c = 0; c < nrhs; ++c) {
    for (int i = 0; i < q; ++i) {  // L y = b
      double v = B[(size_t)i * nrhs + c];
      for (int k = 0; k < i; ++k) v -= A[(size_t)i * q + k] * B[(size_t)k * nrhs + c];
      B[(size_t)i * nrhs + c] = v / A[(size_t)i * q + i];
    }
    for (int i = q - 1; i >= 0; --i) {  // L^T x = y
      double v = B[(size_t)i * nrhs + c];
      for (int k = i + 1; k < q; ++k) v -= A[(size_t)k * q + i] * B[(size_t)k * nrhs + c];
      B[(size_t)i * nrhs + c] = v / A[(size_t)i * q + i];
    }
  }
  return true;
}

template <typename T>
static fdtd_status gradient_t(mor_model *M, const mor_basis *b, fdtd_grid *g, int64_t T_, const void *u,
                              const void *dldy, double *gcell, double *gmat, double *gDe, cudaStream_t s) {
  const int q1 = M->q1, q2 = M->q2, m = M->m, p = M->p;
  DevBuf dif, ebar, Gd, Gf, gedge;
  struct Rel {
    std::vector<DevBuf *> v;
    cudaStream_t s;
    ~Rel() { for (auto *x : v) x->release(s); }
  } rel{{&dif, &ebar, &Gd, &Gf, &gedge}, s};
  FDTD_CHECK(dif.alloc(sizeof(T) * (size_t)q1 * T_, s));
  FDTD_CHECK(ebar.alloc(sizeof(T) * (size_t)q1 * T_, s));
  RedAdjArgs<T> a;
  a.q1 = q1; a.q2 = q2; a.m = m; a.p = p; a.nsteps = T_;
  a.Pe = M->Pe.as<T>(); a.Qe = M->Qe.as<T>(); a.be = M->be.as<T>();
  a.Ph = M->Ph.as<T>(); a.Qh = M->Qh.as<T>(); a.bh = M->bh.as<T>(); a.C = M->Cr.as<T>();
  a.u = static_cast<const T *>(u);
  a.dldy = static_cast<const T *>(dldy);
  a.dif = dif.as<T>();
  a.ebar = ebar.as<T>();
  const size_t smem = sizeof(T) * (2 * (size_t)(q1 + q2) + std::max(m, p) + 2);
  FDTD_REQUIRE(smem <= 220 * 1024, "mor_gradient: reduced order too large");
  FDTD_CHECK_CUDA(cudaFuncSetAttribute(reduced_adjoint_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  reduced_adjoint_kernel<T><<<1, 1024, smem, s>>>(a);
  FDTD_CHECK(after_launch("reduced_adjoint_kernel"));
  // E = sum_n ebar_n (e^n - e^{n+1})^T: a Gram product over the steps
  FDTD_CHECK(Gd.alloc(sizeof(double) * (size_t)q1 * q1, s));
  FDTD_CHECK(gram_native(s, T_, ebar.as<T>(), q1, dif.as<T>(), q1, Gd.as<double>()));
  // G = Ae^-1 E / dt with Ae = D~e/dt + D~se/2 (host FP64)
  std::vector<double> E((size_t)q1 * q1), De((size_t)q1 * q1), Dse((size_t)q1 * q1);
  FDTD_CHECK_CUDA(cudaMemcpyAsync(E.data(), Gd.ptr, sizeof(double) * E.size(), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(De.data(), M->De.ptr, sizeof(double) * De.size(), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(Dse.data(), M->Dse.ptr, sizeof(double) * Dse.size(), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  const double dt = M->dt;
  std::vector<double> Ae((size_t)q1 * q1);
  for (size_t t = 0; t < Ae.size(); ++t) Ae[t] = De[t] / dt + 0.5 * Dse[t];
  FDTD_REQUIRE_STATUS(chol_solve_host(Ae, q1, E, q1), FDTD_EUNSTABLE,
                      "mor_gradient: D~eps/dt + D~se/2 is not positive definite");
  for (double &x : E) x /= dt;
  if (gDe) std::copy(E.begin(), E.end(), gDe);
  if (!gcell && !gmat) return FDTD_OK;
  std::vector<T> Gh(E.begin(), E.end());
  FDTD_CHECK(Gf.alloc(sizeof(T) * Gh.size(), s));
  FDTD_CHECK_CUDA(cudaMemcpyAsync(Gf.ptr, Gh.data(), sizeof(T) * Gh.size(), cudaMemcpyHostToDevice, s));
  const int64_t n3 = 3 * g->nc;
  FDTD_CHECK(gedge.alloc(sizeof(double) * n3, s));
  constexpr int NE = qf_edges<T>();
  const size_t qsm = sizeof(T) * NE * (q1 + 1);
  FDTD_REQUIRE(qsm <= 220 * 1024, "mor_gradient: reduced order too large for the edge quadratic form");
  FDTD_CHECK_CUDA(cudaFuncSetAttribute(quad_form_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm));
  quad_form_kernel<T><<<(int)((n3 + NE - 1) / NE), NE, qsm, s>>>(make_geo<T>(g), q1, b->V1.as<T>(), Gf.as<T>(),
                                                                  gedge.as<double>());
  FDTD_CHECK(after_launch("quad_form_kernel"));
  FDTD_CHECK(edges_to_cells(g, gedge.as<double>(), gcell, gmat, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));  // host staging (Gh) is read by the copy above
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status mor_gradient(mor_model *M, const mor_basis *b, fdtd_grid *g, int64_t nsteps, const void *u,
                         const void *dloss_dy, double *grad_eps_cell, double *grad_eps_mat, double *grad_De,
                         fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(M && b && g, "mor_gradient: NULL argument");
  FDTD_REQUIRE(M->perturbed, "mor_gradient: call mor_perturb first (it prepares the step matrices)");
  FDTD_REQUIRE(nsteps >= 1 && (M->m == 0 || u) && (M->p == 0 || dloss_dy), "mor_gradient: bad arguments");
  FDTD_REQUIRE(b->n3 == 3 * g->nc && b->q1 == M->q1 && b->prec == g->prec && M->prec == g->prec,
               "mor_gradient: model, basis and grid do not belong together");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->prec == FDTD_F64)
    return gradient_t<double>(M, b, g, nsteps, u, dloss_dy, grad_eps_cell, grad_eps_mat, grad_De, s);
  return gradient_t<float>(M, b, g, nsteps, u, dloss_dy, grad_eps_cell, grad_eps_mat, grad_De, s);
}

}  // extern "C"
