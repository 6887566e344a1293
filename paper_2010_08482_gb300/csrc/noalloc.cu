// ctq_eval_traces_static: ctq_eval_traces with its scratch in a fixed,
// library-owned device array instead of a caller-provided workspace.
//
// Some callers cannot hand the library a workspace: a Monte Carlo driver
// written in C or Fortran that owns no device allocator, code whose device
// memory is entirely managed by another runtime's pool, or code that must not
// call cudaMalloc on a latency-critical path (it may synchronise the device).
// For them the scratch lives in g_static_scratch below: a file-scope __device__
// array of CTQ_STATIC_SCRATCH_BYTES that every GPU which loads this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ctq_internal.h"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[CTQ_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `device` (which must be current).
// In host code the symbol name is only a host-side stand-in, so the address
// is looked up once per device and cached for the life of the process; a
// device reset invalidates it (the header says so to the caller).
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return CTQ_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return CTQ_ERR_CUDA;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return CTQ_OK;
}

}  // namespace

extern "C" int ctq_eval_traces_static(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                                      const ctq_result* result, void* stream) {
  if (!imp || !batch || !opts) return ctq_eval_traces(imp, batch, opts, result, nullptr, 0, stream);
  ctq_info info;
  if (ctq_impurity_info(imp, &info) != CTQ_OK) return CTQ_ERR_ARG;
  const size_t need = ctq_workspace_size(imp, batch->n_chains, opts);
  if (need > CTQ_STATIC_SCRATCH_BYTES) {
    ctq::set_last_error("batch needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                        std::to_string(size_t(CTQ_STATIC_SCRATCH_BYTES)) + " (use ctq_eval_traces with a workspace)");
    return CTQ_ERR_WORKSPACE;
  }
  int device = -1;
  if (ctq::impurity_device(imp, &device) != CTQ_OK || device < 0) return CTQ_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return CTQ_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return CTQ_ERR_CUDA;
  void* scratch = nullptr;
  const int st = scratch_address(device, &scratch);
  if (prev != device) cudaSetDevice(prev);
  if (st != CTQ_OK) {
    ctq::set_last_error("cannot resolve the static scratch on this device");
    return st;
  }
  return ctq_eval_traces(imp, batch, opts, result, scratch, CTQ_STATIC_SCRATCH_BYTES, stream);
}
