// vmc_loss_weights_noalloc: the clipped-energy gradient weights without a
// caller-provided workspace.
//
// vmc_loss_weights needs scratch memory for its sort, which the caller
// allocates and passes in.  Some callers have no way to allocate device
// memory: a plugin whose host framework owns every device allocation and
// hands out only the tensors it passes in, or a long-running service that
// allocates once at start-up and must not touch the allocator afterwards.
// This entry point serves them: its scratch is a fixed array in the
// library's own device memory, so a call needs only the input and output
// arrays.
//
// The array holds kNoAllocMaxWalkers doubles (512 KB).  Every GPU that loads
// the library holds its own copy until the process exits.  All calls on a
// device share that copy and it keeps the previous call's contents; the
// kernel overwrites every element it reads (the sort pads with +inf), so
// nothing has to be cleared, but two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on the array.
//
// Host code cannot pass the array's name to a kernel: in host code that name
// is only a stand-in for the symbol, not a device address.  The first call on
// a device, made with that device current, looks the address up with
// cudaGetSymbolAddress and caches it for the life of the process; that first
// call may load the module and should therefore come before any stream
// capture.  A device reset (cudaDeviceReset, or a reset of the primary
// context) destroys the array with the context that holds it, and the cached
// address with it: like a handle's device buffers, it must not be used on
// that device afterwards.  No call allocates.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kNoAllocMaxWalkers = 65536;
static __device__ __align__(256) double g_loss_scratch[kNoAllocMaxWalkers];

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

dq_status scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (device < 0 || device >= kMaxDevices) return DQ_ERR_ARG;
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_loss_scratch) != cudaSuccess || p == nullptr) return DQ_ERR_CUDA;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return DQ_OK;
}

}  // namespace

extern "C" dq_status vmc_loss_weights_noalloc(dq_handle h, const void* e_loc, int64_t B, double clip_k,
                                              void* weights, double* stats, void* stream) {
  if (h == nullptr) return DQ_ERR_ARG;
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) return DQ_ERR_CUDA;
  if (device != h->device) return DQ_ERR_ARG;
  if (B < 1 || !e_loc || !weights || !(clip_k > 0)) return DQ_ERR_ARG;
  if (B > kNoAllocMaxWalkers) return DQ_ERR_SHAPE;
  double* scratch = nullptr;
  const dq_status st = scratch_address(device, &scratch);
  if (st != DQ_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // timed like the workspace form when the handle's per-launch profiling is on
  if (h->prof) h->prof->begin(dq::PK_LOSS_WEIGHTS, s);
  if (h->precision == DQ_FP64)
    e = dq::launch_loss_weights<double>(static_cast<const double*>(e_loc), B, clip_k, static_cast<double*>(weights),
                                        stats, scratch, s);
  else
    e = dq::launch_loss_weights<float>(static_cast<const float*>(e_loc), B, clip_k, static_cast<float*>(weights),
                                       stats, scratch, s);
  if (h->prof) h->prof->end(s);
  return e == cudaSuccess ? DQ_OK : DQ_ERR_CUDA;
}
