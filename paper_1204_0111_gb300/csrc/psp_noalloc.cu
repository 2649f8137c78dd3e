// psp_apply_noalloc: the preconditioner application with its work vectors in a fixed device array.
//
// Some callers cannot allocate device memory while they run: a framework whose caching allocator
// already holds the free memory (a cudaMalloc then fails although the caller has room), a process
// held to a fixed device-memory budget, or a loop timed as one stream-ordered region in which a
// cudaMalloc would synchronise the device.  psp_apply grows its work vectors on demand; this entry
// point instead uses one file-scope __device__ array, so it never calls cudaMalloc, cudaFree or any
// other allocating routine.
#include <cuda.h>

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
// device address of psp_apply_scratch per device ordinal, and the context it was resolved in: a
// context created anew on that device (after cudaDeviceReset, say) loads the module again, and the
// address is then resolved again
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrent = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry-point table (the library does not link libcuda)
CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<CtxGetCurrent>(p);
  }();
  return fn;
}

// With the handle's device current: the array's device address in the current context, resolved on
// the first call in that context.
psp_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return psp::set_error(PSP_ERR_CUDA, "device ordinal out of range");
  CtxGetCurrent get = ctx_get_current();
  if (!get) return psp::set_error(PSP_ERR_CUDA, "cuCtxGetCurrent is not available");
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS || !ctx) return psp::set_error(PSP_ERR_CUDA, "no current CUDA context");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, psp_apply_scratch);
    if (e != cudaSuccess || !p)
      return psp::set_error(PSP_ERR_CUDA, (std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)).c_str());
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return PSP_OK;
}

// device memory of device `dev` (memory of another device is not accepted)
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" psp_status psp_apply_noalloc(psp_handle h, const double* rhs, double* out, int nrhs, void* stream) {
  if (!h || !rhs || !out || nrhs < 1) return psp::set_error(PSP_ERR_ARG, "bad apply arguments");
  const int64_t N = psp::handle_points(h);
  if (N < 0) return psp::set_error(PSP_ERR_STATE, "handle has no factorisation");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return psp::set_error(PSP_ERR_CUDA, cudaGetErrorString(e));
  if (dev != psp::handle_device(h))
    return psp::set_error(PSP_ERR_ARG, ("the handle was set up on device " + std::to_string(psp::handle_device(h)) +
                                        ", but device " + std::to_string(dev) + " is current").c_str());
  if (!on_device(rhs, dev) || !on_device(out, dev))
    return psp::set_error(PSP_ERR_ARG, "psp_apply_noalloc needs device pointers of the handle's device for rhs and out");
  const size_t need = psp::apply_workspace_bytes(h, nrhs);
  if (need > kNoAllocScratchBytes)
    return psp::set_error(PSP_ERR_ARG, ("psp_apply_noalloc needs " + std::to_string(need) +
                                        " bytes of work vectors for this problem and nrhs, more than its fixed " +
                                        std::to_string(kNoAllocScratchBytes) + "; use psp_apply")
                                           .c_str());
  void* ws = nullptr;
  psp_status st = scratch_address(dev, &ws);
  if (st != PSP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((const void*)rhs != (const void*)out) {
    e = cudaMemcpyAsync(out, rhs, (size_t)N * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return psp::set_error(PSP_ERR_CUDA, cudaGetErrorString(e));
  }
  return psp::apply_with_workspace(h, reinterpret_cast<double2*>(out), nrhs, ws, s);
}
