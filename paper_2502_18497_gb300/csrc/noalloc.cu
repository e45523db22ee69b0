// Allocation-free copy of the last batch's changed labels.
//
// Some callers cannot allocate device memory once they are running: a
// serving loop that reserved all of its memory at start-up, a process whose
// device memory is fully held by another framework's caching allocator, or a
// real-time path that forbids allocator calls.  ldl_copy_changed_noalloc gives
// them the same result as ldl_copy_changed while touching no allocator: the
// labels of the changed vertices are gathered into a fixed static device
// array and copied to the caller's host arrays from there.
#include <algorithm>
#include <mutex>

#include "kern.cuh"

// Largest number of changed vertices one call can return.
#define LDL_NOALLOC_MAX_CHANGED (1 << 20)

// The scratch array: 4 MiB per device that loads this library, held until the
// process exits.  Every call uses the same array, so calls whose GPU work
// overlaps (for example on two streams) race on it and must be serialised by
// the caller.  The gather overwrites every slot it returns, so nothing has to
// start at zero.
static __device__ __align__(256) int32_t g_noalloc_labels[LDL_NOALLOC_MAX_CHANGED];

namespace {

constexpr int kMaxDevices = 64;
// Device address of the array on each device, resolved once per device (the
// host-side symbol is only a stand-in and must never reach a kernel).
std::once_flag g_once[kMaxDevices];
int32_t* g_ptr[kMaxDevices] = {nullptr};
cudaError_t g_ptr_err[kMaxDevices] = {cudaSuccess};

__global__ void k_gather_noalloc(const int32_t* ids, int32_t k, const int32_t* lab, int32_t* out) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) out[i] = lab[ids[i]];
}

}  // namespace

extern "C" ldl_status ldl_copy_changed_noalloc(const ldl_ctx* cc, int32_t* ids, int32_t* labels) {
  if (!cc) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  const int64_t k = c.res.n_changed;
  if (k == 0) return LDL_OK;
  if (!ids || !labels) {
    c.err = "ldl_copy_changed_noalloc: ids and labels must both be given";
    return LDL_E_INVALID;
  }
  if (k > LDL_NOALLOC_MAX_CHANGED) {
    c.err = "ldl_copy_changed_noalloc: " + std::to_string(k) + " changed vertices exceed the limit of " +
            std::to_string(LDL_NOALLOC_MAX_CHANGED) + "; use ldl_copy_changed";
    return LDL_E_INVALID;
  }
  const int dev = c.dev;
  if (dev < 0 || dev >= kMaxDevices) {
    c.err = "ldl_copy_changed_noalloc: device ordinal out of range";
    return LDL_E_CUDA;
  }
  // the context's device is current for the whole call (and the caller's
  // device is restored on return), so the address looked up below and the
  // kernel's launch both belong to the device that holds the context
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
  if (e != cudaSuccess) {
    c.err = std::string("ldl_copy_changed_noalloc: cannot make the context's device current: ") +
            cudaGetErrorString(e);
    return LDL_E_CUDA;
  }
  std::call_once(g_once[dev], [dev] {
    void* p = nullptr;
    g_ptr_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_labels);
    if (g_ptr_err[dev] == cudaSuccess && !p) g_ptr_err[dev] = cudaErrorInvalidSymbol;
    if (g_ptr_err[dev] == cudaSuccess) g_ptr[dev] = (int32_t*)p;
  });
  if (g_ptr_err[dev] != cudaSuccess) {
    c.err = std::string("ldl_copy_changed_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(g_ptr_err[dev]);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return LDL_E_CUDA;
  }
  int32_t* scratch = g_ptr[dev];
  const int32_t kk = (int32_t)k;
  const int grid = (int)std::min<int64_t>(((int64_t)kk + 255) / 256, 4096);
  k_gather_noalloc<<<grid, 256, 0, c.s>>>(c.lChg.p, kk, c.lv[0].lab.p, scratch);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(ids, c.lChg.p, sizeof(int32_t) * (size_t)kk, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(labels, scratch, sizeof(int32_t) * (size_t)kk, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    c.err = std::string("ldl_copy_changed_noalloc: ") + cudaGetErrorString(e);
    return LDL_E_CUDA;
  }
  return LDL_OK;
}
