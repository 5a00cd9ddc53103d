// Field watchdog of fdtd_step and the settable wait limit of the dataflow
// stepping kernel.
//
// After every public fdtd_step call (unless switched off) one reduction sums
// the squares of the six field arrays in FP64 and a one-thread kernel sets bit
// 4 of the grid's error flag when the sum is not finite -- a leap-frog run
// beyond its stability limit (Eq. (singular_limit): R loses positive
// definiteness above the exact Delta t limit) overflows to Inf and NaN.  With
// a growth limit set, a source-free call (no sources, or u = NULL) also sums
// the fields before stepping and sets bit 8 when the sum grew by more than
// the limit: without sources the discrete energy x^T R x is conserved
// (lossless) or decays, and the sum of E^2 + eta0^2 H^2 (the vacuum energy
// density over eps0) stays within the ratio of the largest to the smallest
// relative material constant of it.  fdtd_check reports
// either bit as FDTD_EUNSTABLE; in synchronous mode fdtd_step itself returns it.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "grid_internal.cuh"

namespace fdtdmor {

// sum of E^2 + eta0^2 H^2 over the six arrays (the vacuum field energy over
// eps0 per unit volume): blockIdx.y = 0 sums the three E arrays, 1 the three
// H arrays.  Each thread sums its values in the field type (FP32 grids: float4
// loads, a few hundred values per thread, finite for values below 1e19) and
// the block totals go to FP64; FP64 arithmetic on every value would make this
// pass FP64-throughput-bound instead of memory-bound.
template <typename T>
__global__ void field_energy_kernel(const T *__restrict__ f, int64_t half, double *__restrict__ out) {
  __shared__ double sh[32];
  const double eta2 = kMu0 / kEps0;
  const T *p = f + blockIdx.y * half;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T acc = T(0);
  int64_t done = 0;
  if constexpr (sizeof(T) == 4) {
    if (((uintptr_t)p & 15) == 0) {
      const float4 *p4 = reinterpret_cast<const float4 *>(p);
      const int64_t n4 = half / 4;
      for (int64_t i = t0; i < n4; i += stride) {
        const float4 v = __ldg(p4 + i);
        acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
      }
      done = 4 * n4;
    }
  }
  for (int64_t i = done + t0; i < half; i += stride) {
    const T v = p[i];
    acc += v * v;
  }
  double d = (double)acc;
  for (int o = 16; o; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    atomicAdd(out, (blockIdx.y ? eta2 : 1.0) * t);
  }
}

__global__ void watchdog_decide_kernel(const double *__restrict__ acc, double growth, unsigned *err) {
  const double before = acc[0], after = acc[1];
  if (!isfinite(after)) atomicOr(err, 4u);
  else if (growth > 0 && before > 0 && after > growth * before) atomicOr(err, 8u);
}

static fdtd_status field_energy(fdtd_grid *g, double *slot, cudaStream_t s) {
  const int64_t half = 3 * g->nc;
  const dim3 blocks((unsigned)std::min<int64_t>(152 * 4, (half + 1023) / 1024), 2);
  if (g->prec == FDTD_F64)
    field_energy_kernel<double><<<blocks, 256, 0, s>>>(g->fields[g->cur].as<double>(), half, slot);
  else
    field_energy_kernel<float><<<blocks, 256, 0, s>>>(g->fields[g->cur].as<float>(), half, slot);
  return after_launch("field_energy_kernel");
}

static bool source_free(const fdtd_grid *g, const void *u) { return g->ports.empty() || !u; }

fdtd_status watchdog_before(fdtd_grid *g, const void *u, int reset_fields, cudaStream_t s) {
  if (!g->wd_on) return FDTD_OK;
  FDTD_CHECK(g->wd_acc.alloc(2 * sizeof(double), s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(g->wd_acc.ptr, 0, 2 * sizeof(double), s));
  if (g->wd_growth > 0 && source_free(g, u) && !reset_fields) FDTD_CHECK(field_energy(g, g->wd_acc.as<double>(), s));
  return FDTD_OK;
}

fdtd_status watchdog_after(fdtd_grid *g, const void *u, int reset_fields, cudaStream_t s) {
  if (!g->wd_on) return FDTD_OK;
  double *acc = g->wd_acc.as<double>();
  FDTD_CHECK(field_energy(g, acc + 1, s));
  const double growth = (g->wd_growth > 0 && source_free(g, u) && !reset_fields) ? g->wd_growth : 0.0;
  watchdog_decide_kernel<<<1, 1, 0, s>>>(acc, growth, g->errflag.as<unsigned>());
  FDTD_CHECK(after_launch("watchdog_decide_kernel"));
  if (!g->wd_sync) return FDTD_OK;
  unsigned h = 0;
  FDTD_CHECK_CUDA(cudaMemcpyAsync(&h, g->errflag.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  FDTD_CHECK_CUDA(cudaStreamSynchronize(s));
  if (h & 12u) {
    FDTD_CHECK_CUDA(cudaMemsetAsync(g->errflag.ptr, 0, sizeof(unsigned), s));
    set_error("fdtd_step: the field watchdog fired: %s",
              (h & 4u) ? "NaN or Inf in the fields" : "field energy of a source-free call grew beyond the limit");
    return FDTD_EUNSTABLE;
  }
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status fdtd_grid_set_watchdog(fdtd_grid *g, int enable, double growth, int sync) {
  FDTD_REQUIRE(g, "fdtd_grid_set_watchdog: NULL grid");
  FDTD_REQUIRE(growth >= 0 && std::isfinite(growth), "fdtd_grid_set_watchdog: growth must be finite and >= 0");
  g->wd_on = enable != 0;
  g->wd_growth = growth;
  g->wd_sync = sync != 0;
  return FDTD_OK;
}

fdtd_status fdtd_grid_set_wait_limit(fdtd_grid *g, long long polls) {
  FDTD_REQUIRE(g, "fdtd_grid_set_wait_limit: NULL grid");
  g->wait_limit = polls < 0 ? ((int64_t)1 << 24) : (int64_t)polls;
  return FDTD_OK;
}

}  // extern "C"
