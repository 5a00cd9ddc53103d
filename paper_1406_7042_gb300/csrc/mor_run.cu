// A8: reduced leap-frog, Eq. (reducedMNAform) in the block form of
// Eq. (R_and_Freduced), as one persistent kernel; A9: probe comparison.
//
// Per step n (state e ~ E part, h ~ H part of x~^n):
//   e <- Pe e - Qe h + be u^{n+1}
//   h <- Ph h + Qh e + bh u^{n+1}
//   y^n = C~ e
// The two phases depend on each other.  The model runs on a thread block
// cluster whose CTAs each hold a slice of rows of the step matrices in shared
// memory (resident for the whole run); each phase's new state slice is stored
// into every CTA's copy of the state through distributed shared memory, with
// one cluster barrier per phase.  Where no cluster can be scheduled, or for
// models too large for 16 CTAs, one CTA of 1024 threads runs all steps with a
// block barrier between phases (the matrices in its shared memory when they
// fit, q up to about 90 in FP32, else streamed from L2).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cooperative_groups.h>
#include <cstdlib>
#include <string>
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

// Cluster form.  CTA `rank` of the cluster owns rows [rank*er, rank*er + er)
// of e and [rank*hr, ...) of h, with those rows of Pe, Qe, be and of Ph, Qh,
// bh in its shared memory, and a double-buffered copy of the whole state
// (slot n & 1 is read in step n, slot (n+1) & 1 written).  Per step: phase E
// computes its rows of e^{n+1} and stores them into slot (n+1)&1 of every
// CTA (DSMEM); cluster barrier; phase H computes its rows of h^{n+1} from
// e^{n+1} likewise and rank 0 forms y^n = C~ e^{n+1}; cluster barrier.  A
// slot is rewritten only two barriers after its last read, so the two
// barriers per step are all the ordering the exchange needs.
constexpr int kRunClusterThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kRunClusterThreads) reduced_run_cluster_kernel(RunArgs<T> a, int er, int hr) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), ncta = (int)cluster.num_blocks();
  const int q1 = a.q1, q2 = a.q2, m = a.m, p = a.p;
  const int e0 = rank * er, ne = max(0, min(q1, e0 + er) - e0);
  const int h0 = rank * hr, nh = max(0, min(q2, h0 + hr) - h0);
  const int mp = (m + 1) & ~1;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *E = reinterpret_cast<T *>(smraw);  // [2][q1]
  T *H = E + 2 * q1;                     // [2][q2]
  T *us = H + 2 * q2;                    // [mp]
  T *Pe = us + mp, *Qe = Pe + (size_t)er * q1, *be = Qe + (size_t)er * q2;
  T *Ph = be + (size_t)er * m, *Qh = Ph + (size_t)hr * q2, *bh = Qh + (size_t)hr * q1, *C = bh + (size_t)hr * m;
  for (int t = threadIdx.x; t < ne * q1; t += blockDim.x) Pe[t] = a.Pe[(size_t)e0 * q1 + t];
  for (int t = threadIdx.x; t < ne * q2; t += blockDim.x) Qe[t] = a.Qe[(size_t)e0 * q2 + t];
  for (int t = threadIdx.x; t < ne * m; t += blockDim.x) be[t] = a.be[(size_t)e0 * m + t];
  for (int t = threadIdx.x; t < nh * q2; t += blockDim.x) Ph[t] = a.Ph[(size_t)h0 * q2 + t];
  for (int t = threadIdx.x; t < nh * q1; t += blockDim.x) Qh[t] = a.Qh[(size_t)h0 * q1 + t];
  for (int t = threadIdx.x; t < nh * m; t += blockDim.x) bh[t] = a.bh[(size_t)h0 * m + t];
  if (rank == 0)
    for (int t = threadIdx.x; t < p * q1; t += blockDim.x) C[t] = a.C[t];
  for (int t = threadIdx.x; t < q1; t += blockDim.x) E[t] = a.state[t];
  for (int t = threadIdx.x; t < q2; t += blockDim.x) H[t] = a.state[q1 + t];
  cluster.sync();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t n = 0; n < a.nsteps; ++n) {
    const int cur = (int)(n & 1), nxt = cur ^ 1;
    const T *e = E + cur * q1, *h = H + cur * q2;
    for (int t = threadIdx.x; t < m; t += blockDim.x) us[t] = a.u[n * m + t];
    __syncthreads();
    for (int r = w; r < ne; r += nw) {
      T acc = 0;
      for (int c = lane; c < q1; c += 32) acc += Pe[r * q1 + c] * e[c];
      for (int c = lane; c < q2; c += 32) acc -= Qe[r * q2 + c] * h[c];
      for (int c = lane; c < m; c += 32) acc += be[r * m + c] * us[c];
      acc = warp_sum(acc);
      for (int d = lane; d < ncta; d += 32) cluster.map_shared_rank(E, d)[nxt * q1 + e0 + r] = acc;
    }
    cluster.sync();
    const T *en = E + nxt * q1;
    for (int r = w; r < nh; r += nw) {
      T acc = 0;
      for (int c = lane; c < q2; c += 32) acc += Ph[r * q2 + c] * h[c];
      for (int c = lane; c < q1; c += 32) acc += Qh[r * q1 + c] * en[c];
      for (int c = lane; c < m; c += 32) acc += bh[r * m + c] * us[c];
      acc = warp_sum(acc);
      for (int d = lane; d < ncta; d += 32) cluster.map_shared_rank(H, d)[nxt * q2 + h0 + r] = acc;
    }
    if (rank == 0)
      for (int r = w; r < p; r += nw) {
        T acc = 0;
        for (int c = lane; c < q1; c += 32) acc += C[r * q1 + c] * en[c];
        acc = warp_sum(acc);
        if (lane == 0) a.y[n * p + r] = acc;
      }
    cluster.sync();
  }
  if (rank == 0) {
    const int fin = (int)(a.nsteps & 1);
    for (int t = threadIdx.x; t < q1; t += blockDim.x) a.state[t] = E[fin * q1 + t];
    for (int t = threadIdx.x; t < q2; t += blockDim.x) a.state[q1 + t] = H[fin * q2 + t];
  }
}

// Shared memory of the cluster form with cl CTAs (row slices er, hr); 0 if
// it exceeds 200 KB per CTA.
template <typename T>
static size_t run_cluster_smem(int cl, int q1, int q2, int m, int p, int &er, int &hr) {
  er = (q1 + cl - 1) / cl;
  hr = (q2 + cl - 1) / cl;
  const size_t smem = sizeof(T) * (2 * (size_t)(q1 + q2) + ((m + 1) & ~1) + (size_t)er * (q1 + q2 + m) +
                                   (size_t)hr * (q2 + q1 + m) + (size_t)p * q1);
  return smem <= 200 * 1024 ? smem : 0;
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
  // Cluster form whenever it can be scheduled (FDTDMOR_RUN=cta / cluster
  // forces a form), the one-CTA form as the fallback.  Measured (FP32, us per
  // step, one CTA against a cluster of 16): q = 40 3.27 / 2.76, q = 80
  // 4.61 / 2.89, q = 200 21.3 / 3.33 (clusters of 4 and 8: 7.3, 4.4),
  // q = 400 46.4 / 5.34; FDTDMOR_RUN_CL caps the size.
  const char *env = getenv("FDTDMOR_RUN");
  const std::string form = env ? env : "";
  const char *envc = getenv("FDTDMOR_RUN_CL");
  const int cl_max = envc ? std::max(2, std::min(16, atoi(envc))) : 16;
  if (form != "cta") {
    auto kern = reduced_run_cluster_kernel<T>;
    for (int cl = cl_max; cl >= 2; cl /= 2) {
      int er = 0, hr = 0;
      const size_t csm = run_cluster_smem<T>(cl, q1, q2, m, p, er, hr);
      if (csm == 0) break;  // smaller clusters need even more per CTA
      FDTD_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
      if (cl > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(kRunClusterThreads);
      cfg.dynamicSmemBytes = csm;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cl;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();  // not schedulable: try a smaller cluster
        continue;
      }
      FDTD_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, a, er, hr));
      return after_launch("reduced_run_cluster_kernel");
    }
  }
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
  FDTD_API_RANGE(__func__);
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

// File of a projected model: "FDTDMOR1", int32 version (1), q1, q2, m, p,
// prec, then the FP64 matrices D~eps, D~se (q1 x q1), D~mu, D~sm (q2 x q2),
// K~ (q1 x q2), B~_E (q1 x m), B~_H (q2 x m), C~_E (p x q1), row-major, in
// the little-endian byte order of the hosts this library builds for.
static const char kModelMagic[8] = {'F', 'D', 'T', 'D', 'M', 'O', 'R', '1'};

fdtd_status mor_model_save(const mor_model *M, const char *path, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(M && path, "mor_model_save: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t hdr[6] = {1, M->q1, M->q2, M->m, M->p, (int32_t)M->prec};
  const DevBuf *bufs[8] = {&M->De, &M->Dse, &M->Dm, &M->Dsm, &M->K, &M->BE, &M->BH, &M->CE};
  const size_t cnt[8] = {(size_t)M->q1 * M->q1, (size_t)M->q1 * M->q1, (size_t)M->q2 * M->q2, (size_t)M->q2 * M->q2,
                         (size_t)M->q1 * M->q2, (size_t)M->q1 * M->m, (size_t)M->q2 * M->m, (size_t)M->p * M->q1};
  std::vector<double> host;
  for (int i = 0; i < 8; ++i) {
    const size_t off = host.size();
    host.resize(off + cnt[i]);
    if (cnt[i]) FDTD_CHECK_CUDA(cudaMemcpyAsync(host.data() + off, bufs[i]->ptr, cnt[i] * sizeof(double),
                                                cudaMemcpyDeviceToHost, s));
  }
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  FILE *f = fopen(path, "wb");
  FDTD_REQUIRE(f, "mor_model_save: cannot open %s for writing", path);
  const bool ok = fwrite(kModelMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
                  (host.empty() || fwrite(host.data(), sizeof(double), host.size(), f) == host.size());
  const bool closed = fclose(f) == 0;
  FDTD_REQUIRE(ok && closed, "mor_model_save: write to %s failed", path);
  return FDTD_OK;
}

fdtd_status mor_model_load(const char *path, fdtd_stream_t stream, mor_model **out) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(path && out, "mor_model_load: NULL argument");
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  FDTD_REQUIRE(f, "mor_model_load: cannot open %s", path);
  char magic[8];
  int32_t hdr[6];
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kModelMagic, 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
            hdr[0] == 1 && hdr[1] >= 0 && hdr[2] >= 0 && hdr[3] >= 0 && hdr[4] >= 0 &&
            (hdr[5] == FDTD_F32 || hdr[5] == FDTD_F64) && hdr[1] <= 65535 && hdr[2] <= 65535;
  const int q1 = ok ? hdr[1] : 0, q2 = ok ? hdr[2] : 0, m = ok ? hdr[3] : 0, p = ok ? hdr[4] : 0;
  const size_t cnt[8] = {(size_t)q1 * q1, (size_t)q1 * q1, (size_t)q2 * q2, (size_t)q2 * q2,
                         (size_t)q1 * q2, (size_t)q1 * m, (size_t)q2 * m, (size_t)p * q1};
  size_t total = 0;
  for (size_t c : cnt) total += c;
  std::vector<double> host(ok ? total : 0);
  if (ok && total) ok = fread(host.data(), sizeof(double), total, f) == total;
  fclose(f);
  FDTD_REQUIRE(ok, "mor_model_load: %s is not a reduced-model file of this library", path);
  cudaStream_t s = (cudaStream_t)stream;
  mor_model *M = new mor_model();
  M->q1 = q1; M->q2 = q2; M->m = m; M->p = p;
  M->prec = (fdtd_prec)hdr[5];
  M->elem = M->prec == FDTD_F64 ? 8 : 4;
  M->stream = s;
  DevBuf *bufs[8] = {&M->De, &M->Dse, &M->Dm, &M->Dsm, &M->K, &M->BE, &M->BH, &M->CE};
  fdtd_status st = FDTD_OK;
  size_t off = 0;
  for (int i = 0; i < 8 && st == FDTD_OK; ++i) {
    st = bufs[i]->alloc(sizeof(double) * std::max<size_t>(1, cnt[i]), s);
    if (st == FDTD_OK && cnt[i] &&
        cudaMemcpyAsync(bufs[i]->ptr, host.data() + off, cnt[i] * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
      st = cuda_fail(cudaGetLastError(), "mor_model_load copy");
    off += cnt[i];
  }
  if (st == FDTD_OK) st = M->Kp.alloc(sizeof(double) * std::max<size_t>(1, cnt[4]), s);
  if (st == FDTD_OK && cnt[4] &&
      cudaMemcpyAsync(M->Kp.ptr, M->K.ptr, cnt[4] * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "mor_model_load copy");
  if (st == FDTD_OK) st = M->sigma.alloc(sizeof(double) * std::max(1, std::min(q1, q2)), s);
  if (st == FDTD_OK && cudaStreamSynchronize(s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "sync");
  if (st != FDTD_OK) {
    mor_model_destroy(M);
    return st;
  }
  *out = M;
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
  FDTD_API_RANGE(__func__);
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
