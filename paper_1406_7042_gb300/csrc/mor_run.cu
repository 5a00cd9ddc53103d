// A8: reduced leap-frog, Eq. (reducedMNAform) in the block form of
// Eq. (R_and_Freduced), as one persistent kernel; A9: probe comparison.
//
// Per step n (state e ~ E part, h ~ H part of x~^n):
//   e <- Pe e - Qe h + be u^{n+1}
//   h <- Ph h + Qh e + bh u^{n+1}
//   y^n = C~ e
// The two phases depend on each other, so one CTA of 1024 threads runs all
// steps with a block barrier between phases; the step matrices sit in shared
// memory when they fit (q up to about 90 in FP32), else they stream from L2.
#include <algorithm>
#include <vector>

#include "mor_common.cuh"
#include "mor_internal.cuh"

namespace fdtdmor {

template <typename T>
struct RunArgs {
  int q1, q2, m, p;
  int64_t nsteps;
  const T *Pe, *Qe, *be, *Ph, *Qh, *bh, *C;
  const T *u;
  T *y;
  T *state;
  int mats_in_smem;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(1024) reduced_run_kernel(RunArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  const int q1 = a.q1, q2 = a.q2, m = a.m, p = a.p;
  T *e = sm, *h = e + q1, *en = h + q2, *hn = en + q1, *us = hn + q2;
  T *mats = us + ((m + 1) & ~1);
  const T *Pe = a.Pe, *Qe = a.Qe, *be = a.be, *Ph = a.Ph, *Qh = a.Qh, *bh = a.bh, *C = a.C;
  if (a.mats_in_smem) {
    T *d = mats;
    auto cp = [&](const T *src, int n) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) d[t] = src[t];
      T *r = d;
      d += n;
      return (const T *)r;
    };
    Pe = cp(a.Pe, q1 * q1); Qe = cp(a.Qe, q1 * q2); be = cp(a.be, q1 * m);
    Ph = cp(a.Ph, q2 * q2); Qh = cp(a.Qh, q2 * q1); bh = cp(a.bh, q2 * m); C = cp(a.C, p * q1);
  }
  for (int t = threadIdx.x; t < q1 + q2; t += blockDim.x) sm[t] = a.state[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t n = 0; n < a.nsteps; ++n) {
    for (int t = threadIdx.x; t < m; t += blockDim.x) us[t] = a.u[n * m + t];
    __syncthreads();
    for (int r = w; r < q1; r += nw) {
      T acc = 0;
      for (int c = lane; c < q1; c += 32) acc += Pe[r * q1 + c] * e[c];
      for (int c = lane; c < q2; c += 32) acc -= Qe[r * q2 + c] * h[c];
      for (int c = lane; c < m; c += 32) acc += be[r * m + c] * us[c];
      acc = warp_sum(acc);
      if (lane == 0) en[r] = acc;
    }
    __syncthreads();
    for (int r = w; r < q2; r += nw) {
      T acc = 0;
      for (int c = lane; c < q2; c += 32) acc += Ph[r * q2 + c] * h[c];
      for (int c = lane; c < q1; c += 32) acc += Qh[r * q1 + c] * en[c];
      for (int c = lane; c < m; c += 32) acc += bh[r * m + c] * us[c];
      acc = warp_sum(acc);
      if (lane == 0) hn[r] = acc;
    }
    for (int r = w; r < p; r += nw) {
      T acc = 0;
      for (int c = lane; c < q1; c += 32) acc += C[r * q1 + c] * en[c];
      acc = warp_sum(acc);
      if (lane == 0) a.y[n * p + r] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < q1 + q2; t += blockDim.x) sm[t] = t < q1 ? en[t] : hn[t - q1];
    __syncthreads();
  }
  for (int t = threadIdx.x; t < q1 + q2; t += blockDim.x) a.state[t] = sm[t];
}

template <typename T>
static fdtd_status run_t(mor_model *M, int64_t nsteps, const void *u, void *y, int reset, cudaStream_t s) {
  const int q1 = M->q1, q2 = M->q2, m = M->m, p = M->p;
  FDTD_CHECK(M->state.alloc(sizeof(T) * std::max(1, q1 + q2), s));
  if (reset) FDTD_CHECK_CUDA(cudaMemsetAsync(M->state.ptr, 0, sizeof(T) * (q1 + q2), s));
  if (nsteps == 0) return FDTD_OK;
  RunArgs<T> a;
  a.q1 = q1; a.q2 = q2; a.m = m; a.p = p; a.nsteps = nsteps;
  a.Pe = M->Pe.as<T>(); a.Qe = M->Qe.as<T>(); a.be = M->be.as<T>();
  a.Ph = M->Ph.as<T>(); a.Qh = M->Qh.as<T>(); a.bh = M->bh.as<T>(); a.C = M->Cr.as<T>();
  a.u = static_cast<const T *>(u);
  a.y = static_cast<T *>(y);
  a.state = M->state.as<T>();
  const size_t vec = sizeof(T) * (2 * (size_t)(q1 + q2) + ((m + 1) & ~1));
  const size_t mats = sizeof(T) * ((size_t)q1 * q1 + 2 * (size_t)q1 * q2 + (size_t)q2 * q2 + (size_t)(q1 + q2) * m + (size_t)p * q1);
  const size_t limit = 220 * 1024;
  a.mats_in_smem = vec + mats <= limit;
  const size_t smem = a.mats_in_smem ? vec + mats : vec;
  FDTD_REQUIRE(vec <= limit, "reduced order too large for the reduced-run kernel");
  FDTD_CHECK_CUDA(cudaFuncSetAttribute(reduced_run_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  reduced_run_kernel<T><<<1, 1024, smem, s>>>(a);
  return after_launch("reduced_run_kernel");
}

// sum over the common samples of (y_red - y_ref)^2 and y_ref^2
template <typename T>
__global__ void compare_kernel(const T *__restrict__ yr, const T *__restrict__ yf, int64_t n, int64_t stride,
                               int64_t offset, int p, double *out) {
  __shared__ double sh[2][32];
  double d2 = 0, r2 = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * p; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / p, c = t % p;
    const double a = (double)yr[i * p + c], b = (double)yf[(offset + i * stride) * p + c];
    d2 += (a - b) * (a - b);
    r2 += b * b;
  }
  for (int o = 16; o; o >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, o);
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = d2; sh[1][threadIdx.x >> 5] = r2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int wq = 0; wq < (int)(blockDim.x >> 5); ++wq) { a += sh[0][wq]; b += sh[1][wq]; }
    atomicAdd(&out[0], a);
    atomicAdd(&out[1], b);
  }
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status mor_run(mor_model *M, int64_t nsteps, const void *u, void *y, int reset_state, fdtd_stream_t stream) {
  FDTD_REQUIRE(M, "mor_run: NULL model");
  FDTD_REQUIRE(M->perturbed, "mor_run: call mor_perturb first (it fixes dt and builds the step matrices)");
  FDTD_REQUIRE(nsteps >= 0, "nsteps must be >= 0");
  FDTD_REQUIRE(nsteps == 0 || ((M->m == 0 || u) && (M->p == 0 || y)), "mor_run: u / y required");
  cudaStream_t s = (cudaStream_t)stream;
  return M->prec == FDTD_F64 ? run_t<double>(M, nsteps, u, y, reset_state, s)
                             : run_t<float>(M, nsteps, u, y, reset_state, s);
}

fdtd_status mor_model_get(const mor_model *M, int which, double *host_out, int *rows, int *cols,
                          fdtd_stream_t stream) {
  FDTD_REQUIRE(M, "mor_model_get: NULL model");
  const DevBuf *src = nullptr;
  int r = 0, c = 0;
  switch (which) {
    case 0: src = &M->De; r = M->q1; c = M->q1; break;
    case 1: src = &M->Dse; r = M->q1; c = M->q1; break;
    case 2: src = &M->Dm; r = M->q2; c = M->q2; break;
    case 3: src = &M->Dsm; r = M->q2; c = M->q2; break;
    case 4: src = &M->K; r = M->q1; c = M->q2; break;
    case 5: src = &M->Kp; r = M->q1; c = M->q2; break;
    case 6: src = &M->BE; r = M->q1; c = M->m; break;
    case 7: src = &M->CE; r = M->p; c = M->q1; break;
    case 8: src = &M->sigma; r = 1; c = M->perturbed ? M->q2 : 0; break;
    default: FDTD_REQUIRE(false, "mor_model_get: which must be 0..8");
  }
  if (rows) *rows = r;
  if (cols) *cols = c;
  if (host_out && r * c > 0) {
    cudaStream_t s = (cudaStream_t)stream;
    FDTD_CHECK_CUDA(cudaMemcpyAsync(host_out, src->ptr, sizeof(double) * r * c, cudaMemcpyDeviceToHost, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  return FDTD_OK;
}

fdtd_status mor_model_destroy(mor_model *M) {
  if (!M) return FDTD_OK;
  cudaStream_t s = M->stream;
  cudaStreamSynchronize(s);
  for (DevBuf *d : {&M->De, &M->Dse, &M->Dm, &M->Dsm, &M->K, &M->Kp, &M->BE, &M->BH, &M->CE, &M->sigma, &M->Pe,
                    &M->Qe, &M->be, &M->Ph, &M->Qh, &M->bh, &M->Cr, &M->state})
    d->release(s);
  cudaStreamSynchronize(s);
  delete M;
  return FDTD_OK;
}

fdtd_status mor_compare(const void *y_red, const void *y_ref, int64_t n, int64_t stride, int64_t offset, int p,
                        fdtd_prec prec, double *err, fdtd_stream_t stream) {
  FDTD_REQUIRE(y_red && y_ref && err && n >= 1 && stride >= 1 && offset >= 0 && p >= 1, "mor_compare: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf acc;
  FDTD_CHECK(acc.alloc(2 * sizeof(double), s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(acc.ptr, 0, 2 * sizeof(double), s));
  const int blocks = (int)std::min<int64_t>(1024, (n * p + 255) / 256);
  if (prec == FDTD_F64)
    compare_kernel<double><<<blocks, 256, 0, s>>>((const double *)y_red, (const double *)y_ref, n, stride, offset, p, acc.as<double>());
  else
    compare_kernel<float><<<blocks, 256, 0, s>>>((const float *)y_red, (const float *)y_ref, n, stride, offset, p, acc.as<double>());
  FDTD_CHECK(after_launch("compare_kernel"));
  double h[2];
  FDTD_CHECK_CUDA(cudaMemcpyAsync(h, acc.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  acc.release(s);
  *err = h[1] > 0 ? std::sqrt(h[0] / h[1]) : (h[0] > 0 ? INFINITY : 0.0);
  return FDTD_OK;
}

}  // extern "C"
