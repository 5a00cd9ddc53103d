// Batched SPRIM basis build (Sec. IV on many grids at once).
//
// One basis build is a chain of small kernels: shifted solves of a few
// right-hand sides, iteration blocks replayed from a captured graph with a
// host poll of the residuals between blocks, then CGS2.  On a grid of 10^4 to
// 10^6 cells each kernel fills a fraction of the 152 SMs, and the host polls
// leave the GPU idle between blocks.  A batch of uneven grids therefore runs
// its builds side by side: a few host workers, each with a stream of its own,
// take the grids largest first from a shared counter and run the ordinary
// build on them, so that the kernels and polls of different grids overlap.
// The caller's stream is joined before (each worker stream waits for its
// event) and after (it waits for the workers' events).  The arithmetic is the
// ordinary build's, grid by grid.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "grid_internal.cuh"
#include "mor_internal.cuh"

using namespace fdtdmor;

namespace {

constexpr int kMaxWorkers = 32;

// Worker streams, created once per device and kept: the caching allocator
// keys its free blocks by stream, so reusing the streams lets later batches
// reuse the memory of earlier ones.
struct StreamPool {
  std::mutex mu;
  std::vector<std::pair<int, cudaStream_t>> streams;  // (device, stream)

  fdtd_status get(int dev, int count, std::vector<cudaStream_t> &out) {
    std::lock_guard<std::mutex> lock(mu);
    out.clear();
    for (auto &ds : streams)
      if (ds.first == dev && (int)out.size() < count) out.push_back(ds.second);
    while ((int)out.size() < count) {
      cudaStream_t s;
      FDTD_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      streams.emplace_back(dev, s);
      out.push_back(s);
    }
    return FDTD_OK;
  }
};

StreamPool &stream_pool() {
  static StreamPool pool;
  return pool;
}

int worker_count(int n) {
  int w = 8;  // the default number of hardware work queues a context uses
  if (const char *e = getenv("FDTDMOR_BATCH_WORKERS")) w = atoi(e);
  return std::max(1, std::min({w, n, kMaxWorkers}));
}

struct Result {
  fdtd_status st = FDTD_OK;
  std::string err;
};

}  // namespace

extern "C" {

fdtd_status mor_build_basis_batched(int n, fdtd_grid *const *grids, const mor_opts *opts, fdtd_stream_t stream,
                                    mor_basis **out, fdtd_status *status) {
  FDTD_API_RANGE(__func__);
  FDTD_REQUIRE(n >= 0 && (n == 0 || (grids && opts && out)), "mor_build_basis_batched: NULL argument");
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  if (n == 0) return FDTD_OK;
  for (int i = 0; i < n; ++i) {
    FDTD_REQUIRE(grids[i], "mor_build_basis_batched: grid %d is NULL", i);
    for (int j = 0; j < i; ++j)
      FDTD_REQUIRE(grids[j] != grids[i], "mor_build_basis_batched: grid %d appears twice (%d)", i, j);
  }
  cudaStream_t cs = (cudaStream_t)stream;
  int dev = 0;
  FDTD_CHECK_CUDA(cudaGetDevice(&dev));
  const int nw = worker_count(n);
  std::vector<cudaStream_t> ws;
  FDTD_CHECK(stream_pool().get(dev, nw, ws));

  // Every worker stream starts after the work already queued on the caller's.
  cudaEvent_t start;
  FDTD_CHECK_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  fdtd_status st0 = FDTD_OK;
  if (cudaEventRecord(start, cs) != cudaSuccess) st0 = cuda_fail(cudaGetLastError(), "event record");
  for (int w = 0; w < nw && st0 == FDTD_OK; ++w)
    if (cudaStreamWaitEvent(ws[w], start, 0) != cudaSuccess) st0 = cuda_fail(cudaGetLastError(), "stream wait");
  cudaEventDestroy(start);
  if (st0 != FDTD_OK) return st0;

  // Largest grid first, so that the longest builds do not start last.
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return grids[a]->nc > grids[b]->nc; });

  std::atomic<int> next(0);
  std::vector<Result> res(n);
  std::vector<int64_t> launches(nw, 0);
  auto work = [&](int w) {
    cudaSetDevice(dev);
    const int64_t l0 = fdtd_launch_count(0);
    for (int t = next.fetch_add(1); t < n; t = next.fetch_add(1)) {
      const int i = order[t];
      res[i].st = mor_build_basis(grids[i], &opts[i], (fdtd_stream_t)ws[w], &out[i]);
      if (res[i].st != FDTD_OK) res[i].err = fdtd_last_error();
      // The basis is used and released on the caller's stream from here on.
      if (out[i]) out[i]->stream = cs;
    }
    launches[w] = fdtd_launch_count(0) - l0;
  };
  std::vector<std::thread> threads;
  threads.reserve(nw - 1);
  for (int w = 1; w < nw; ++w) threads.emplace_back(work, w);
  work(0);
  for (auto &t : threads) t.join();

  // The caller's stream continues after every build.
  fdtd_status st = FDTD_OK;
  for (int w = 0; w < nw; ++w) {
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(done, ws[w]) != cudaSuccess || cudaStreamWaitEvent(cs, done, 0) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "stream join");
      cudaStreamSynchronize(ws[w]);
    }
    if (done) cudaEventDestroy(done);
  }
  for (int w = 1; w < nw; ++w) add_launches(launches[w]);

  // Worst status: a hard error over ENOCONV over OK; its message is kept.
  int worst = -1;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = res[i].st;
    if (res[i].st == FDTD_OK) continue;
    const bool hard = res[i].st != FDTD_ENOCONV;
    if (worst < 0 || (hard && res[worst].st == FDTD_ENOCONV)) worst = i;
  }
  if (st != FDTD_OK) return st;
  if (worst >= 0) {
    set_error("mor_build_basis_batched: grid %d: %s", worst, res[worst].err.c_str());
    return res[worst].st;
  }
  return FDTD_OK;
}

}  // extern "C"
