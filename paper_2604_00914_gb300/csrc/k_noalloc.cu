// apf_gram_noalloc: the Gram product G = X^H Y for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA graph
// that is being captured, an allocator's own callbacks, or a host that hands
// the library a fixed memory budget.  apf_gram needs a per-call workspace for
// the partial sums of its row splits and allocates it; this variant keeps
// that workspace in one file-scope device array of fixed size instead.
//
// The array is loaded with the library: every GPU that loads libapf.so holds
// kNoAllocScratchBytes of device memory until the process exits.  Host code
// cannot use the array's name as a device address (it denotes a host-side
// stand-in), so the first call on each device looks up the device address
// with cudaGetSymbolAddress while that device is current and caches it.  The
// cache remembers the context the address belongs to: after a device reset
// (cudaDeviceReset) the runtime creates a new context and loads the module
// again, and the next call looks the address up again instead of using the
// stale one.
#include <cuda.h>

#include <mutex>

#include "apf_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_gram_scratch[kNoAllocScratchBytes];

struct DeviceScratch {
  void* ptr = nullptr;
  int num_sms = 0;
  unsigned long long ctx_id = 0;  // context the address belongs to
  bool ready = false;
};
std::mutex g_scratch_mutex;
DeviceScratch g_scratch[kMaxDevices];

// The unique id of the calling thread's current context, 0 when there is none
// (driver entry points through the runtime: nothing links libcuda directly).
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Set-up for the current device (first call, and the first call in a new
// context of it): the device address of the array and the SM count.
apf_status scratch_for_current_device(DeviceScratch* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APF_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return APF_ERR_ARG;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  DeviceScratch& d = g_scratch[dev];
  if (!d.ready || id == 0 || id != d.ctx_id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess) return APF_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APF_ERR_CUDA;
    d.ptr = p;
    d.num_sms = sms;
    d.ctx_id = current_context_id();  // the context now exists
    d.ready = true;
  }
  *out = d;
  return APF_OK;
}

}  // namespace

extern "C" apf_status apf_gram_noalloc(int32_t dtype, int64_t n, int64_t pa, int64_t pb, const void* X,
                                       int64_t ldx, const void* Y, int64_t ldy, void* G, int64_t ldg,
                                       void* cuda_stream) {
  if (!X || !Y || !G || n < 1 || pa < 1 || pb < 1 || ldx < pa || ldy < pb || ldg < pb) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  const size_t elem = dtype == APF_C128 ? 16 : 8;
  if ((size_t)pa * (size_t)pb * elem > kNoAllocScratchBytes) return APF_ERR_ARG;
  DeviceScratch d;
  const apf_status st = scratch_for_current_device(&d);
  if (st != APF_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  try {
    if (dtype == APF_C128)
      apf::gram_scratch<double2>(stream, d.num_sms, n, pa, pb, static_cast<const double2*>(X), ldx,
                                 static_cast<const double2*>(Y), ldy, static_cast<double2*>(G), ldg, d.ptr,
                                 kNoAllocScratchBytes);
    else
      apf::gram_scratch<double>(stream, d.num_sms, n, pa, pb, static_cast<const double*>(X), ldx,
                                static_cast<const double*>(Y), ldy, static_cast<double*>(G), ldg, d.ptr,
                                kNoAllocScratchBytes);
  } catch (const ApfError& e) {
    return e.status;
  } catch (...) {
    return APF_ERR_CUDA;
  }
  return APF_OK;
}
