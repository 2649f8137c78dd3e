// psp_apply_noalloc: the preconditioner application with its work vectors in a fixed device array.
//
// Some callers cannot allocate device memory while they run: a framework whose caching allocator
// already holds the free memory (a cudaMalloc then fails although the caller has room), a process
// held to a fixed device-memory budget, or a loop timed as one stream-ordered region in which a
// cudaMalloc would synchronise the device.  psp_apply grows its work vectors on demand; this entry
// point instead uses one file-scope __device__ array, so it never calls cudaMalloc, cudaFree or any
// other allocating routine.
#include <mutex>
#include <string>

#include "cplx.cuh"
#include "psp_internal.h"

// Work vectors of psp_apply_noalloc: 16 MiB, reserved in every GPU context that loads the library
// and held until the process exits.  In host code this name is only a stand-in for the symbol, not a
// device address; the device address is looked up with cudaGetSymbolAddress below.
static constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char psp_apply_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 128;
void* g_scratch_addr[kMaxDevices] = {};  // device address of psp_apply_scratch, per device ordinal

// Once per device, with that device current: resolve the array's device address.
psp_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return psp::set_error(PSP_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return psp::set_error(PSP_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, psp_apply_scratch);
    if (e != cudaSuccess || !p)
      return psp::set_error(PSP_ERR_CUDA, (std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)).c_str());
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PSP_OK;
}

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" psp_status psp_apply_noalloc(psp_handle h, const double* rhs, double* out, int nrhs, void* stream) {
  if (!h || !rhs || !out || nrhs < 1) return psp::set_error(PSP_ERR_ARG, "bad apply arguments");
  const int64_t N = psp::handle_points(h);
  if (N < 0) return psp::set_error(PSP_ERR_STATE, "handle has no factorisation");
  if (!is_device(rhs) || !is_device(out))
    return psp::set_error(PSP_ERR_ARG, "psp_apply_noalloc needs device pointers for rhs and out");
  const size_t need = psp::apply_workspace_bytes(h, nrhs);
  if (need > kNoAllocScratchBytes)
    return psp::set_error(PSP_ERR_ARG, ("psp_apply_noalloc needs " + std::to_string(need) +
                                        " bytes of work vectors for this problem and nrhs, more than its fixed " +
                                        std::to_string(kNoAllocScratchBytes) + "; use psp_apply")
                                           .c_str());
  void* ws = nullptr;
  psp_status st = scratch_address(&ws);
  if (st != PSP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((const void*)rhs != (const void*)out) {
    cudaError_t e = cudaMemcpyAsync(out, rhs, (size_t)N * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return psp::set_error(PSP_ERR_CUDA, cudaGetErrorString(e));
  }
  return psp::apply_with_workspace(h, reinterpret_cast<double2*>(out), nrhs, ws, s);
}
