// Allocation-free entry point of the dense contraction (one trajectory).
//
// Some callers cannot let a library call cudaMalloc: an application whose
// device memory is owned by another allocator (a framework's caching
// allocator that reserves the HBM up front, or a host program that fixes its
// memory budget at start-up), or code that issues work from a hard real-time
// control loop, where an allocation can synchronise the device or take an
// unbounded time.  grom_nonlinear_full_noalloc serves them: it runs the same
// K1 streaming kernel as grom_nonlinear on a tensor the caller owns, and its
// scratch (the per-warp partial sums of the streaming kernel and the timeout
// flag) lives in the file-scope device array below instead of memory the
// library allocates.
#include <mutex>
#include <string>

#include "grom_internal.h"

namespace grom {

// 1 MiB of partial sums: the K1 partition needs grid * maxseg * 8 doubles for
// one trajectory, about 8 n + 16 * grid, i.e. < 0.6 MiB for n <= 8192 on a
// 152-SM GB300.  Every GPU that loads the library holds this array until the
// process exits.
constexpr size_t kNoAllocScratchDoubles = 131072;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles + 32];

namespace {
struct DeviceSlot {
  bool ready = false;
  double* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sm_count = 0;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;
}  // namespace

}  // namespace grom

using namespace grom;

extern "C" grom_status grom_nonlinear_full_noalloc(int32_t n, int32_t storage, const void* tensor, const double* u,
                                                   double* c, void* stream) {
  if (!tensor || !u || !c) return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear_full_noalloc: null pointer");
  if (n < 1) return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear_full_noalloc: n must be >= 1");
  if (storage_elem_bytes(storage) == 0) return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear_full_noalloc: bad storage");
  if (n > grom_max_n(GROM_FORM_FULL, storage))
    return fail(GROM_ERR_UNSUPPORTED, "grom_nonlinear_full_noalloc: n exceeds grom_max_n");
  if (reinterpret_cast<uintptr_t>(tensor) % 16 != 0)
    return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear_full_noalloc: tensor must be 16-byte aligned");
  int dev = 0;
  GROM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(GROM_ERR_UNSUPPORTED, "grom_nonlinear_full_noalloc: device index");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (s != nullptr) {
    // the scratch address below belongs to the current device; a stream of
    // another device would run the kernel against that device's memory
    int sdev = -1;
    GROM_CUDA_TRY(cudaStreamGetDevice(s, &sdev));
    if (sdev != dev)
      return fail(GROM_ERR_INVALID_ARG, "grom_nonlinear_full_noalloc: the stream belongs to device " +
                                            std::to_string(sdev) + ", the current device is " + std::to_string(dev));
  }
  DeviceSlot slot;
  {
    // Once per device, with that device current: resolve the device address
    // of the file-scope scratch array (host code cannot use its name).
    std::lock_guard<std::mutex> lock(g_slots_mu);
    DeviceSlot& s = g_slots[dev];
    if (!s.ready) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "grom_nonlinear_full_noalloc: cudaGetSymbolAddress");
      e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return cuda_fail(e, "grom_nonlinear_full_noalloc: cudaDeviceGetAttribute");
      s.scratch = static_cast<double*>(p);
      s.ready = true;
    }
    slot = s;
  }
  const K1Plan plan = k1_plan(n, storage, slot.sm_count);
  const size_t need = (size_t)plan.grid * plan.maxseg * (K1_CONSUMERS / 32);
  if (need > kNoAllocScratchDoubles)
    return fail(GROM_ERR_UNSUPPORTED, "grom_nonlinear_full_noalloc: needs " + std::to_string(need * 8) +
                                          " bytes of scratch, more than the fixed 1 MiB");
  // The timeout flag sits after the partials and must start at zero; every
  // partial the finalize step reads is written earlier in the same call.
  int* err = reinterpret_cast<int*>(slot.scratch + kNoAllocScratchDoubles);
  GROM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  K1Args a{};
  a.tensor = static_cast<const uint8_t*>(tensor);
  a.u = u;
  a.u_stride = n;
  a.c = c;
  a.c_stride = n;
  a.part = slot.scratch;
  a.err = err;
  cudaError_t e = k1_launch(plan, storage, a, 1, s);
  if (e != cudaSuccess) return cuda_fail(e, "grom_nonlinear_full_noalloc launch");
  return GROM_OK;
}

extern "C" grom_status grom_nonlinear_full_noalloc_status(void* stream) {
  int dev = 0;
  GROM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(GROM_ERR_UNSUPPORTED, "grom_nonlinear_full_noalloc_status: device index");
  DeviceSlot slot;
  {
    std::lock_guard<std::mutex> lock(g_slots_mu);
    slot = g_slots[dev];
  }
  if (!slot.ready) return GROM_OK;  // no call has run on this device
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int flag = 0;
  const int* err = reinterpret_cast<const int*>(slot.scratch + kNoAllocScratchDoubles);
  GROM_CUDA_TRY(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GROM_CUDA_TRY(cudaStreamSynchronize(s));
  if (flag & DEV_ERR_TIMEOUT)
    return fail(GROM_ERR_TIMEOUT, "grom_nonlinear_full_noalloc: a device wait of the last call timed out; c is unspecified");
  if (flag) return fail(GROM_ERR_CUDA, "grom_nonlinear_full_noalloc: device error flags " + std::to_string(flag));
  return GROM_OK;
}
