// mor_compare_noalloc: the probe comparison of mor_compare for callers that
// cannot allocate device memory, with its scratch in a static device array.
//
// Who needs it: a host application or plugin that owns all device memory
// itself and may not have a library allocate behind its back, or a run under
// an allocator that must not grow while it runs.  The caller still provides
// y_red and y_ref; only the reduction scratch moves into the library image.
// The call reads its result back to the host and synchronises the stream.
//
// Scratch: g_noalloc_scratch holds one pair of partial sums per block of the
// first pass (at most kNoAllocMaxBlocks blocks of kNoAllocBlock threads, each
// thread covering kNoAllocItems samples, so n*p <= kNoAllocMaxSamples) and the
// final pair written by the second pass.  Every slot a call reads is written
// earlier in the same call, so no clearing is needed; the array keeps the last
// call's contents.  Calls that overlap on the GPU (different streams, or
// different host threads) share the array and race: serialise them.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace fdtdmor {

constexpr int kNoAllocBlock = 256;
constexpr int kNoAllocItems = 16;
constexpr int kNoAllocMaxBlocks = 4096;
constexpr int64_t kNoAllocMaxSamples = (int64_t)kNoAllocMaxBlocks * kNoAllocBlock * kNoAllocItems;  // 16.7 M
constexpr int kNoAllocDoubles = 2 * kNoAllocMaxBlocks + 2;  // 64 KiB + 16 B

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch, looked up once per device.
static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[64] = {nullptr};

static fdtd_status noalloc_scratch(double **out) {
  int dev = 0;
  FDTD_CHECK_CUDA(cudaGetDevice(&dev));
  FDTD_REQUIRE(dev >= 0 && dev < 64, "mor_compare_noalloc: device ordinal %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    FDTD_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return FDTD_OK;
}

// Pass 1: block b sums (y_red - y_ref)^2 and y_ref^2 over its samples into
// scratch[2b], scratch[2b+1].
template <typename T>
__global__ void __launch_bounds__(kNoAllocBlock) noalloc_compare_pass1(const T *__restrict__ yr,
                                                                       const T *__restrict__ yf, int64_t n,
                                                                       int64_t stride, int64_t offset, int p,
                                                                       double *__restrict__ scratch) {
  __shared__ double sh[2][kNoAllocBlock / 32];
  double d2 = 0, r2 = 0;
  const int64_t total = n * p;
  const int64_t base = (int64_t)blockIdx.x * kNoAllocBlock * kNoAllocItems + threadIdx.x;
  for (int it = 0; it < kNoAllocItems; ++it) {
    const int64_t t = base + (int64_t)it * kNoAllocBlock;
    if (t < total) {
      const int64_t i = t / p, c = t % p;
      const double a = (double)yr[i * p + c], b = (double)yf[(offset + i * stride) * p + c];
      d2 += (a - b) * (a - b);
      r2 += b * b;
    }
  }
  for (int o = 16; o; o >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, o);
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = d2;
    sh[1][threadIdx.x >> 5] = r2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < kNoAllocBlock / 32; ++w) { a += sh[0][w]; b += sh[1][w]; }
    scratch[2 * blockIdx.x] = a;
    scratch[2 * blockIdx.x + 1] = b;
  }
}

// Pass 2: one block adds the nblk pairs in a fixed order into the last slot.
__global__ void __launch_bounds__(kNoAllocBlock) noalloc_compare_pass2(int nblk, double *__restrict__ scratch) {
  __shared__ double sh[2][kNoAllocBlock];
  double a = 0, b = 0;
  for (int k = threadIdx.x; k < nblk; k += kNoAllocBlock) {
    a += scratch[2 * k];
    b += scratch[2 * k + 1];
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int s = kNoAllocBlock / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[kNoAllocDoubles - 2] = sh[0][0];
    scratch[kNoAllocDoubles - 1] = sh[1][0];
  }
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status mor_compare_noalloc(const void *y_red, const void *y_ref, int64_t n, int64_t stride, int64_t offset,
                                int p, fdtd_prec prec, double *err, fdtd_stream_t stream) {
  FDTD_REQUIRE(y_red && y_ref && err && n >= 1 && stride >= 1 && offset >= 0 && p >= 1,
               "mor_compare_noalloc: bad argument");
  FDTD_REQUIRE(prec == FDTD_F32 || prec == FDTD_F64, "mor_compare_noalloc: prec must be FDTD_F32 or FDTD_F64");
  FDTD_REQUIRE(n <= kNoAllocMaxSamples / p,
               "mor_compare_noalloc: n*p = %lld exceeds the no-allocation maximum of %lld samples",
               (long long)n * p, (long long)kNoAllocMaxSamples);
  double *scratch = nullptr;
  FDTD_CHECK(noalloc_scratch(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t per_block = (int64_t)kNoAllocBlock * kNoAllocItems;
  const int nblk = (int)((n * p + per_block - 1) / per_block);
  if (prec == FDTD_F64)
    noalloc_compare_pass1<double><<<nblk, kNoAllocBlock, 0, s>>>((const double *)y_red, (const double *)y_ref, n,
                                                                 stride, offset, p, scratch);
  else
    noalloc_compare_pass1<float><<<nblk, kNoAllocBlock, 0, s>>>((const float *)y_red, (const float *)y_ref, n,
                                                                stride, offset, p, scratch);
  FDTD_CHECK(after_launch("noalloc_compare_pass1"));
  noalloc_compare_pass2<<<1, kNoAllocBlock, 0, s>>>(nblk, scratch);
  FDTD_CHECK(after_launch("noalloc_compare_pass2"));
  double h[2];
  FDTD_CHECK_CUDA(cudaMemcpyAsync(h, scratch + kNoAllocDoubles - 2, sizeof(h), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  *err = h[1] > 0 ? std::sqrt(h[0] / h[1]) : (h[0] > 0 ? INFINITY : 0.0);
  return FDTD_OK;
}

}  // extern "C"
