// A11: many grids of uneven size stepped in lockstep by shared launches.
//
// Each leap-frog step is one E launch and one H launch per group of grids
// that share a kernel instantiation (field type, id width, uniform mu, x
// cells per thread).  A launch walks a work list of (grid, tile, z range)
// units -- the split kernels' units of every grid in the group -- so a batch
// of small cavities fills the GPU as one large grid would.  The step number
// comes from a device counter that the last kernel of each step advances, and
// a grid's input and output buffers follow its step parity, so a captured
// chunk of steps replays without host changes.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "yee_units.cuh"

namespace fdtdmor {

fdtd_status ensure_coef_table(fdtd_grid *g, double dt, cudaStream_t s);

template <typename T, typename ID>
struct BatchGrid {
  YeeArgs<T, ID> a;      // geometry, tables, lists; field pointers set per step
  T *f[2];               // the grid's two state buffers; step n reads f[(c0 + n) & 1]
  int c0;                // parity of the buffer holding the state at step 0
  const ID *emat;
  const T *u;            // [nsteps][m] or null
  T *y;                  // [nsteps][p] or null
  int m, p;
};

struct BatchUnit {
  int grid;
  int bx, by;
  int k0, k1;
};

template <typename T, typename ID>
__device__ __forceinline__ YeeArgs<T, ID> batch_args(const BatchGrid<T, ID> &bg, long long n) {
  YeeArgs<T, ID> a = bg.a;
  const int par = (int)((bg.c0 + n) & 1);
  const int64_t nc = a.nc;
  a.Ein = bg.f[par];
  a.Hin = bg.f[par] + 3 * nc;
  a.Eout = bg.f[par ^ 1];
  a.Hout = bg.f[par ^ 1] + 3 * nc;
  a.u = bg.u ? bg.u + n * bg.m : nullptr;
  a.y = bg.y ? bg.y + n * bg.p : nullptr;
  return a;
}

template <typename T, typename ID, int VW, bool PRE>
__global__ void __launch_bounds__(LTX *LTY, 3) yee_batch_e_kernel(const BatchGrid<T, ID> *__restrict__ grids,
                                                                 const BatchUnit *__restrict__ units, int nunits,
                                                                 const long long *__restrict__ step) {
  wait_prior_grid();
  const long long n = *step;
  for (int w = blockIdx.x; w < nunits; w += gridDim.x) {
    const BatchUnit un = units[w];
    const BatchGrid<T, ID> &bg = grids[un.grid];
    const YeeArgs<T, ID> a = batch_args(bg, n);
    e_unit<T, ID, false, VW, PRE>(a, bg.emat, un.bx, un.by, un.k0, un.k1);
  }
  allow_next_grid();
}

template <typename T, typename ID, bool HOMOG_H, int VW>
__global__ void __launch_bounds__(LTX *LTY) yee_batch_h_kernel(const BatchGrid<T, ID> *__restrict__ grids,
                                                              const BatchUnit *__restrict__ units, int nunits,
                                                              const long long *__restrict__ step) {
  wait_prior_grid();
  const long long n = *step;
  for (int w = blockIdx.x; w < nunits; w += gridDim.x) {
    const BatchUnit un = units[w];
    const BatchGrid<T, ID> &bg = grids[un.grid];
    const YeeArgs<T, ID> a = batch_args(bg, n);
    h_unit<T, ID, HOMOG_H, false, VW>(a, un.bx, un.by, un.k0, un.k1);
  }
  allow_next_grid();
}

// *step += 1 after the last H launch of a step.
__global__ void batch_advance_kernel(long long *step) {
  wait_prior_grid();
  if (threadIdx.x == 0) *step += 1;
  allow_next_grid();
}

// One group's device tables and launchers.
struct BatchGroup {
  virtual ~BatchGroup() = default;
  virtual fdtd_status build(const std::vector<fdtd_grid *> &gs, const std::vector<const void *> &us,
                            const std::vector<void *> &ys, cudaStream_t s) = 0;
  virtual fdtd_status launch_e(cudaStream_t s, const long long *step) = 0;
  virtual fdtd_status launch_h(cudaStream_t s, const long long *step) = 0;
  virtual void release(cudaStream_t s) = 0;
};

template <typename T, typename ID, bool HH, int VW, bool PRE>
struct BatchGroupT : BatchGroup {
  DevBuf grids, units;
  int nunits = 0;
  fdtd_status build(const std::vector<fdtd_grid *> &gs, const std::vector<const void *> &us,
                    const std::vector<void *> &ys, cudaStream_t s) override {
    std::vector<BatchGrid<T, ID>> hg(gs.size());
    std::vector<BatchUnit> hu;
    for (size_t q = 0; q < gs.size(); ++q) {
      fdtd_grid *g = gs[q];
      FDTD_CHECK(ensure_emat<ID>(g, s));
      BatchGrid<T, ID> &b = hg[q];
      b.a = split_args<T, ID>(g);
      if (PRE) {
        const fdtd_status st = ensure_ecoef<T, ID>(g, b.a, s);
        FDTD_CHECK(st);
        b.a.ecoef = g->ecoef.as<T>();
      }
      b.f[0] = g->fields[0].as<T>();
      b.f[1] = g->fields[1].as<T>();
      b.c0 = g->cur;
      b.emat = g->emat.as<ID>();
      b.m = (int)g->ports.size();
      b.p = (int)g->probes.size();
      b.u = static_cast<const T *>(us[q]);
      b.y = static_cast<T *>(ys[q]);
      // four z planes per thread unless tuned: the batch as a whole has many
      // waves of units even when each grid alone has few
      const int lz = g->tune_lz > 0 ? std::min(g->nz, g->tune_lz) : std::min(g->nz, env_int("FDTDMOR_LZ", 4));
      for (int k0 = 0; k0 < g->nz; k0 += lz)
        for (int by = 0; by < g->lists.nty; ++by)
          for (int bx = 0; bx < g->lists.ntx; ++bx) hu.push_back(BatchUnit{(int)q, bx, by, k0, std::min(g->nz, k0 + lz)});
    }
    nunits = (int)hu.size();
    FDTD_CHECK(grids.alloc(hg.size() * sizeof(BatchGrid<T, ID>), s));
    FDTD_CHECK(units.alloc(std::max<size_t>(1, hu.size()) * sizeof(BatchUnit), s));
    FDTD_CHECK_CUDA(cudaMemcpyAsync(grids.ptr, hg.data(), hg.size() * sizeof(BatchGrid<T, ID>), cudaMemcpyHostToDevice, s));
    if (!hu.empty())
      FDTD_CHECK_CUDA(cudaMemcpyAsync(units.ptr, hu.data(), hu.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice, s));
    FDTD_CHECK_CUDA(cudaStreamSynchronize(s));  // host staging vectors go out of scope
    return FDTD_OK;
  }
  int blocks() const { return std::max(1, std::min(nunits, 16 * device_sms())); }
  fdtd_status launch_e(cudaStream_t s, const long long *step) override {
    if (!nunits) return FDTD_OK;
    FDTD_CHECK_CUDA(launch_dependent(yee_batch_e_kernel<T, ID, VW, PRE>, dim3(blocks()), dim3(LTX, LTY), s,
                                     grids.as<const BatchGrid<T, ID>>(), units.as<const BatchUnit>(), nunits, step));
    return after_launch("yee_batch_e_kernel");
  }
  fdtd_status launch_h(cudaStream_t s, const long long *step) override {
    if (!nunits) return FDTD_OK;
    FDTD_CHECK_CUDA(launch_dependent(yee_batch_h_kernel<T, ID, HH, VW>, dim3(blocks()), dim3(LTX, LTY), s,
                                     grids.as<const BatchGrid<T, ID>>(), units.as<const BatchUnit>(), nunits, step));
    return after_launch("yee_batch_h_kernel");
  }
  void release(cudaStream_t s) override {
    grids.release(s);
    units.release(s);
  }
};

template <typename T, typename ID, bool HH, bool PRE>
static BatchGroup *make_group_vw(int vw) {
  if constexpr (sizeof(T) == 4) {
    if (vw == 4) return new BatchGroupT<T, ID, HH, 4, PRE>();
  }
  if (vw == 2) return new BatchGroupT<T, ID, HH, 2, PRE>();
  return new BatchGroupT<T, ID, HH, 1, PRE>();
}

template <typename T, typename ID, bool HH>
static BatchGroup *make_group_pre(int vw, bool pre) {
  return pre ? make_group_vw<T, ID, HH, true>(vw) : make_group_vw<T, ID, HH, false>(vw);
}

static BatchGroup *make_group(fdtd_prec prec, int id_bytes, bool hh, int vw, bool pre) {
  if (prec == FDTD_F64) {
    if (id_bytes == 1)
      return hh ? make_group_pre<double, uint8_t, true>(vw, pre) : make_group_pre<double, uint8_t, false>(vw, pre);
    return hh ? make_group_pre<double, uint16_t, true>(vw, pre) : make_group_pre<double, uint16_t, false>(vw, pre);
  }
  if (id_bytes == 1)
    return hh ? make_group_pre<float, uint8_t, true>(vw, pre) : make_group_pre<float, uint8_t, false>(vw, pre);
  return hh ? make_group_pre<float, uint16_t, true>(vw, pre) : make_group_pre<float, uint16_t, false>(vw, pre);
}

// Leap-frog steps per captured graph.
constexpr int kBatchGraphSteps = 16;

static fdtd_status step_batched(fdtd_grid *const *grids, int ngrids, const double *dt, int64_t nsteps,
                                const void *const *u, void *const *y, int reset_fields, cudaStream_t s) {
  // checks and per-grid preparation
  for (int q = 0; q < ngrids; ++q) {
    fdtd_grid *g = grids[q];
    FDTD_REQUIRE(g, "fdtd_step_batched: NULL grid %d", q);
    for (int r = 0; r < q; ++r) FDTD_REQUIRE(grids[r] != g, "fdtd_step_batched: grid %d repeated", q);
    FDTD_REQUIRE(dt[q] > 0, "fdtd_step_batched: dt[%d] must be > 0", q);
    FDTD_REQUIRE(nsteps == 0 || g->ports.empty() || (u && u[q]), "fdtd_step_batched: u[%d] is required", q);
    FDTD_REQUIRE(nsteps == 0 || g->probes.empty() || (y && y[q]), "fdtd_step_batched: y[%d] is required", q);
  }
  if (nsteps == 0) return FDTD_OK;
  std::map<std::tuple<int, int, int, int, int>, std::vector<int>> groups;
  for (int q = 0; q < ngrids; ++q) {
    fdtd_grid *g = grids[q];
    FDTD_CHECK(ensure_coef_table(g, dt[q], s));
    const int vw = yee_split_vw(g);
    FDTD_CHECK(build_tile_lists(g, LTX * vw, LTY, s));
    if (reset_fields) FDTD_CHECK_CUDA(cudaMemsetAsync(g->fields[g->cur].ptr, 0, (size_t)6 * g->nc * g->elem, s));
    const int p = (int)g->probes.size();
    if (p) FDTD_CHECK_CUDA(cudaMemsetAsync(y[q], 0, (size_t)nsteps * p * g->elem, s));
    groups[std::make_tuple((int)g->prec, g->id_bytes, (int)g->homog_h, vw, (int)yee_split_precoef(g))].push_back(q);
  }
  std::vector<BatchGroup *> gl;
  DevBuf step;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> gstr;  // per-group branches of the captured step
  std::vector<cudaEvent_t> gev;    // fork event, then one join event per group
  struct Cleanup {
    std::vector<BatchGroup *> &gl;
    DevBuf &step;
    cudaStream_t &cap;
    cudaGraphExec_t &exec;
    std::vector<cudaStream_t> &gstr;
    std::vector<cudaEvent_t> &gev;
    cudaStream_t s;
    ~Cleanup() {
      for (auto *b : gl) { b->release(s); delete b; }
      step.release(s);
      if (exec) cudaGraphExecDestroy(exec);
      if (cap) cudaStreamDestroy(cap);
      for (auto x : gstr) cudaStreamDestroy(x);
      for (auto e : gev) cudaEventDestroy(e);
    }
  } cleanup{gl, step, cap, exec, gstr, gev, s};
  for (auto &kv : groups) {
    const int prec = std::get<0>(kv.first), idb = std::get<1>(kv.first), hh = std::get<2>(kv.first),
              vw = std::get<3>(kv.first), pre = std::get<4>(kv.first);
    std::vector<fdtd_grid *> gs;
    std::vector<const void *> us;
    std::vector<void *> ys;
    for (int q : kv.second) {
      gs.push_back(grids[q]);
      us.push_back(grids[q]->ports.empty() ? nullptr : u[q]);
      ys.push_back(grids[q]->probes.empty() ? nullptr : y[q]);
    }
    BatchGroup *b = make_group((fdtd_prec)prec, idb, hh != 0, vw, pre != 0);
    gl.push_back(b);
    FDTD_CHECK(b->build(gs, us, ys, s));
  }
  FDTD_CHECK(step.alloc(sizeof(long long), s));
  FDTD_CHECK_CUDA(cudaMemsetAsync(step.ptr, 0, sizeof(long long), s));
  const long long *sp = step.as<const long long>();
  auto one_step = [&](cudaStream_t st) -> fdtd_status {
    for (auto *b : gl) FDTD_CHECK(b->launch_e(st, sp));
    for (auto *b : gl) FDTD_CHECK(b->launch_h(st, sp));
    FDTD_CHECK_CUDA(launch_dependent(batch_advance_kernel, dim3(1), dim3(32), st, step.as<long long>()));
    return after_launch("batch_advance_kernel");
  };
  // In the captured graph the groups (different grids, so independent until
  // the step counter advances) run as parallel branches: each group's E and
  // H launches on a stream of its own, forked from and joined back into the
  // capture stream around the counter's advance.
  auto one_step_branched = [&](cudaStream_t st) -> fdtd_status {
    const int ng = (int)gl.size();
    FDTD_CHECK_CUDA(cudaEventRecord(gev[0], st));
    for (int q = 0; q < ng; ++q) {
      FDTD_CHECK_CUDA(cudaStreamWaitEvent(gstr[q], gev[0], 0));
      FDTD_CHECK(gl[q]->launch_e(gstr[q], sp));
      FDTD_CHECK(gl[q]->launch_h(gstr[q], sp));
      FDTD_CHECK_CUDA(cudaEventRecord(gev[1 + q], gstr[q]));
      FDTD_CHECK_CUDA(cudaStreamWaitEvent(st, gev[1 + q], 0));
    }
    FDTD_CHECK_CUDA(launch_dependent(batch_advance_kernel, dim3(1), dim3(32), st, step.as<long long>()));
    return after_launch("batch_advance_kernel");
  };
  int64_t n = 0;
  if (nsteps >= 2 * kBatchGraphSteps && !graphs_off()) {
    FDTD_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const bool branched = gl.size() > 1 && !(getenv("FDTDMOR_BATCH_SERIAL") && atoi(getenv("FDTDMOR_BATCH_SERIAL")));
    if (branched) {
      for (size_t q = 0; q < gl.size(); ++q) {
        cudaStream_t x;
        FDTD_CHECK_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        gstr.push_back(x);
      }
      for (size_t q = 0; q <= gl.size(); ++q) {
        cudaEvent_t e;
        FDTD_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        gev.push_back(e);
      }
    }
    const int64_t before = fdtd_launch_count(0);
    FDTD_CHECK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    fdtd_status st = FDTD_OK;
    for (int t = 0; t < kBatchGraphSteps && st == FDTD_OK; ++t) st = branched ? one_step_branched(cap) : one_step(cap);
    const int64_t per_replay = fdtd_launch_count(0) - before;
    add_launches(-per_replay);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (st != FDTD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched graph capture");
    const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) {
      exec = nullptr;
      return cuda_fail(e2, "batched graph instantiate");
    }
    for (; n + kBatchGraphSteps <= nsteps; n += kBatchGraphSteps) {
      FDTD_CHECK_CUDA(cudaGraphLaunch(exec, s));
      add_launches(per_replay);
    }
  }
  for (; n < nsteps; ++n) FDTD_CHECK(one_step(s));
  for (int q = 0; q < ngrids; ++q) grids[q]->cur ^= (int)(nsteps & 1);
  return FDTD_OK;
}

}  // namespace fdtdmor

using namespace fdtdmor;

extern "C" {

fdtd_status fdtd_step_batched(fdtd_grid *const *grids, int ngrids, const double *dt, int64_t nsteps,
                              const void *const *u, void *const *y, int reset_fields, fdtd_stream_t stream) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(grids && dt && ngrids >= 1, "fdtd_step_batched: need grids, dt and ngrids >= 1");
  FDTD_REQUIRE(nsteps >= 0, "fdtd_step_batched: nsteps must be >= 0");
  return step_batched(grids, ngrids, dt, nsteps, u, y, reset_fields, (cudaStream_t)stream);
}

}  // extern "C"
