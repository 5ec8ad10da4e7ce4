// msm_static.cu -- msm_forward_noalloc: the forward pass with its workspace in
// a fixed device array that the library owns, for callers that cannot
// allocate device memory themselves.
//
// Who needs this: code that runs where it may not call cudaMalloc, e.g. a
// host application whose own allocator owns all device memory and forbids
// outside allocations, or a real-time loop that must not pay for (or fail
// on) an allocation. Such a caller passes only its inputs and outputs.
//
// The array is a file-scope __device__ symbol of MSM_NOALLOC_SCRATCH_BYTES;
// every GPU that loads the library keeps it until the process exits. In host
// code its name is only a stand-in, so its device address is looked up once
// per device (cudaGetSymbolAddress, with that device current) on the first
// call made on that device, and that address is what the kernels receive.
// All calls share the one array, which keeps the previous call's contents:
// the forward pass clears what must start at zero (cell counters, status
// word) itself, and two calls that overlap on the GPU race on the array.
#include <mutex>
#include <string>

#include "msm_plan.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MSM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once per device)
int scratch_address(void** out, std::string* err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return MSM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *err = "device ordinal beyond the supported range";
    return MSM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      *err = std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e);
      return MSM_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MSM_OK;
}

}  // namespace

extern "C" int msm_forward_noalloc(msm_plan plan, int n, const float* pos, const float* q, double* energy, float* phi,
                                   float* forces, int flags, void* stream) {
  if (!plan) return msm::api_error(MSM_ERR_INVALID_ARG, "plan must not be NULL");
  size_t need = 0;
  int rc = msm_workspace_bytes(plan, &need);
  if (rc) return rc;
  if (need > (size_t)MSM_NOALLOC_SCRATCH_BYTES)
    return msm::api_error(MSM_ERR_CAPACITY, "msm_forward_noalloc: this plan needs " + std::to_string(need) +
                                                " bytes of workspace; the fixed scratch holds " +
                                                std::to_string((size_t)MSM_NOALLOC_SCRATCH_BYTES) +
                                                " (use msm_forward with a caller-allocated workspace)");
  void* ws = nullptr;
  std::string err;
  rc = scratch_address(&ws, &err);
  if (rc) return msm::api_error(rc, err);
  return msm_forward(plan, ws, (size_t)MSM_NOALLOC_SCRATCH_BYTES, n, pos, q, energy, phi, forces, flags, stream);
}
