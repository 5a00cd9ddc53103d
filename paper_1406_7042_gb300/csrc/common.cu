// Error reporting, allocator hooks, launch accounting and NVTX ranges of the C ABI.
#include <cstdarg>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace fdtdmor {

static thread_local char g_err[1024] = "";
static thread_local int64_t g_launches = 0;
static fdtd_alloc_fn g_alloc = nullptr;
static fdtd_free_fn g_free = nullptr;

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

fdtd_status cuda_fail(cudaError_t e, const char *what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  if (e == cudaErrorMemoryAllocation) return FDTD_ENOMEM;
  return FDTD_ECUDA;
}

fdtd_status after_launch(const char *name) {
  ++g_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, name);
  if (kChecked && (e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, name);
  return FDTD_OK;
}

void add_launches(int64_t n) { g_launches += n; }

static nvtxDomainHandle_t api_domain() {
  static const nvtxDomainHandle_t d = nvtxDomainCreateA("fdtdmor");  // thread-safe one-time creation
  return d;
}

ApiRange::ApiRange(const char *name) {
  nvtxEventAttributes_t at = {};
  at.version = NVTX_VERSION;
  at.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  at.messageType = NVTX_MESSAGE_TYPE_ASCII;
  at.message.ascii = name;
  nvtxDomainRangePushEx(api_domain(), &at);
}

ApiRange::~ApiRange() { nvtxDomainRangePop(api_domain()); }

void *dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc(bytes, (fdtd_stream_t)s);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void *p, cudaStream_t s) {
  if (!p) return;
  if (g_free) {
    g_free(p, (fdtd_stream_t)s);
    return;
  }
  cudaFreeAsync(p, s);
}

fdtd_status DevBuf::alloc(size_t n, cudaStream_t s) {
  if (ptr && bytes >= n) return FDTD_OK;
  release(s);
  ptr = dev_alloc(n, s);
  if (!ptr) {
    set_error("device allocation of %zu bytes failed", n);
    return FDTD_ENOMEM;
  }
  bytes = n;
  return FDTD_OK;
}

void DevBuf::release(cudaStream_t s) {
  if (ptr) dev_free(ptr, s);
  ptr = nullptr;
  bytes = 0;
}

}  // namespace fdtdmor

extern "C" {

const char *fdtd_last_error(void) { return fdtdmor::g_err; }

fdtd_status fdtd_set_allocator(fdtd_alloc_fn alloc, fdtd_free_fn release) {
  if ((alloc == nullptr) != (release == nullptr)) {
    fdtdmor::set_error("fdtd_set_allocator: give both hooks or neither");
    return FDTD_EINVAL;
  }
  fdtdmor::g_alloc = alloc;
  fdtdmor::g_free = release;
  return FDTD_OK;
}

int64_t fdtd_launch_count(int reset) {
  int64_t n = fdtdmor::g_launches;
  if (reset) fdtdmor::g_launches = 0;
  return n;
}

}  // extern "C"
