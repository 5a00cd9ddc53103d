// Internal helpers shared by the library's translation units: status and error
// messages, the device allocator hooks, launch accounting and the grid handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/fdtdmor.h"

namespace fdtdmor {

// ------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
fdtd_status cuda_fail(cudaError_t e, const char *what);

#define FDTD_CHECK_CUDA(expr)                                 \
  do {                                                        \
    cudaError_t e__ = (expr);                                 \
    if (e__ != cudaSuccess) return ::fdtdmor::cuda_fail(e__, #expr); \
  } while (0)

#define FDTD_CHECK(expr)                     \
  do {                                       \
    fdtd_status s__ = (expr);                \
    if (s__ != FDTD_OK) return s__;          \
  } while (0)

#define FDTD_REQUIRE(cond, ...)              \
  do {                                       \
    if (!(cond)) {                           \
      ::fdtdmor::set_error(__VA_ARGS__);     \
      return FDTD_EINVAL;                    \
    }                                        \
  } while (0)

#define FDTD_REQUIRE_STATUS(cond, status, ...) \
  do {                                         \
    if (!(cond)) {                             \
      ::fdtdmor::set_error(__VA_ARGS__);       \
      return (status);                         \
    }                                          \
  } while (0)

// Checked build (-DFDTD_CHECKED, libfdtdmor_checked.so): every launch is
// followed by a device synchronisation, so an asynchronous fault is reported
// with the kernel that caused it; no CUDA graph is captured; and the stepping
// kernels check the indices they take from the port lists, recording bit 16
// of the grid's error flag (FDTD_ECUDA from fdtd_check) and skipping the
// access instead of making it.
#ifdef FDTD_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
inline bool graphs_off() { return kChecked || getenv("FDTDMOR_NO_GRAPH") != nullptr; }
#ifdef __CUDACC__
__device__ __forceinline__ bool dcheck(unsigned *err, bool ok) {
#ifdef FDTD_CHECKED
  if (!ok && err) atomicOr(err, 16u);
  return ok;
#else
  (void)err;
  (void)ok;
  return true;
#endif
}
#endif

// After a kernel launch: count it and surface launch-configuration errors
// (and, in the checked build, execution errors).
fdtd_status after_launch(const char *name);
void add_launches(int64_t n);  // kernel launches made by a graph replay

// NVTX range over one C-ABI call, in the domain "fdtdmor" (a no-op unless a
// profiler is attached): profiles and traces show which call a kernel ran in.
struct ApiRange {
  explicit ApiRange(const char *name);
  ~ApiRange();
  ApiRange(const ApiRange &) = delete;
  ApiRange &operator=(const ApiRange &) = delete;
};
#define FDTD_API_RANGE(name) ::fdtdmor::ApiRange fdtd_api_range_(name)

// ------------------------------------------------------------ memory
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// Device buffer owned by a handle.
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
  fdtd_status alloc(size_t n, cudaStream_t s);
  void release(cudaStream_t s);
  template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// ------------------------------------------------------------ physics constants
constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;
constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);

// ------------------------------------------------------------ grid handle
// Per-axis tables (precision T), packed in one buffer, each of length n_axis:
//   rd   = 1/d[i]                         (primal spacing)
//   rdd  = 2/(d[i-1]+d[i]), 0 at i = 0     (dual spacing)
//   wlo  = d[i-1]/(d[i-1]+d[i]), whi = d[i]/(d[i-1]+d[i])   (cell weights)
enum AxisTable { AX_RD = 0, AX_RDD = 1, AX_WLO = 2, AX_WHI = 3, AX_COUNT = 4 };

// Source/probe entry in the per-tile lists used by the fused kernels.
struct PortEntry {
  int32_t k;      // plane
  int16_t lx, ly; // local coordinates in the tile's extended region
  int16_t comp;   // 0..2
  int16_t pad;
  int32_t port;   // column of B / row of C
  double w;       // weight
};

struct TileLists {
  int tx = 0, ty = 0;       // tile shape the lists were built for
  int ntx = 0, nty = 0;
  DevBuf src_ptr, src;      // CSR over xy-tiles, entries sorted by k
  DevBuf prb_ptr, prb;
  int64_t nsrc = 0, nprb = 0;
};

struct HostPort {
  int comp;
  std::vector<int64_t> cell;
  std::vector<double> w;
};

}  // namespace fdtdmor

struct fdtd_grid {
  int nx = 0, ny = 0, nz = 0;
  int64_t nc = 0;
  fdtd_prec prec = FDTD_F32;
  int elem = 4;                 // bytes per field value
  int nmat = 0;
  int id_bytes = 1;             // 1 (uint8) or 2 (uint16)
  bool homog_h = true;          // every material has the same mu_r, sig_m
  std::vector<double> dx, dy, dz, eps_r, mu_r, sig_e, sig_m;
  std::vector<uint8_t> pec;
  std::vector<uint16_t> used_mats;
  std::vector<fdtdmor::HostPort> ports, probes;
  double cfl = 0;

  fdtdmor::DevBuf fields[2];    // ping-pong: 6*nc values each
  int cur = 0;                  // buffer holding the current state
  fdtdmor::DevBuf mat;          // per-cell material id
  fdtdmor::DevBuf axis;         // AX_COUNT * (nx + ny + nz) values of the field type
  fdtdmor::DevBuf mtab;         // per-material properties in the field type: eps, sig, mu, sigm, pec
  fdtdmor::DevBuf mraw;         // the same table in double, relative eps/mu (source of ctab)
  fdtdmor::DevBuf ctab;         // per-material coefficients for the cached dt: ca, cb, da, db
  double ctab_dt = -1;
  fdtdmor::TileLists lists;
  fdtdmor::DevBuf u_stage, y_stage;  // device staging for fdtd_step_host
  // captured chunks of leap-frog steps (by parity of cur at their start) and
  // what they were captured for; fixed staging rows for their u and y
  cudaGraphExec_t ygraph[2] = {nullptr, nullptr};
  uint64_t ygraph_key[2][12] = {};
  int64_t ygraph_launches[2] = {0, 0};
  cudaStream_t cap_stream = nullptr;
  fdtdmor::DevBuf u_graph, y_graph;
  fdtdmor::DevBuf gsync;        // ticket and per-slab completion counters of the dataflow kernel
  int kernel = 0;               // fdtd_kernel chosen by fdtd_grid_set_kernel (0 = automatic)
  int tune_vw = 0, tune_lz = 0; // split-kernel tile: x cells per thread, z planes per thread (0 = heuristic)
  int tune_slab = 0;            // split-kernel z slab per launch pair (0 = the whole grid)
  fdtdmor::DevBuf flat_src, flat_prb;  // flat (cell, comp, port, w) lists of the fused z-march form
  int nflat_src = 0, nflat_prb = 0;
  bool flat_ready = false;
  // the sources' terms gathered per (field value, port) for the coefficients
  // of ctab_version fix_version (z-march form); fix_one: sources and probes
  // in one launch (no probe edge carries a source term)
  fdtdmor::DevBuf fix_off, fix_fac, fix_port;
  int nfix = 0;
  int64_t fix_version = -1;
  bool fix_one = false;
  fdtdmor::DevBuf emat;         // per cell: material of its uniform E neighbourhood, or ~0
  bool emat_ready = false;
  fdtdmor::DevBuf ecoef;        // per E edge (Ca x3, Cb x3 by cell) for small grids
  int64_t ecoef_version = -1;   // ctab_version it was built from
  int64_t ctab_version = 0;     // bumped by every rebuild of ctab
  fdtdmor::DevBuf uflag;        // per (tile, plane) uniform material id or -1 (fast Yee kernel)
  bool uflag_ready = false;
  fdtdmor::DevBuf errflag;      // bit 2: a bounded device wait gave up; bits 4, 8: watchdog (NaN/Inf, growth)
  int64_t wait_limit = (int64_t)1 << 24;  // polls of a dataflow-kernel counter wait before it gives up
  bool wd_on = true;            // field watchdog after every fdtd_step call
  double wd_growth = 0;         // > 0: flag source-free calls whose field energy grows by more than this factor
  bool wd_sync = false;         // synchronise and return FDTD_EUNSTABLE from fdtd_step when flagged
  fdtdmor::DevBuf wd_acc;       // 2 doubles: field energy before and after the call
  fdtdmor::DevBuf eprops;       // per-edge eps, sig (E) and mu, sgm (H), 4 x 3 x nc (reduction kernels)
  bool eprops_ready = false;
  cudaStream_t create_stream = nullptr;
};
