// pic_noalloc.cu -- pic_diag_noalloc: the diagnostics of pic_diag computed
// without any device allocation.
//
// pic_diag keeps its reduction scratch in device memory that the library
// allocates (through cudaMalloc or the pic_alloc hooks) the first time a
// diagnostic of a given size is requested.  Some callers cannot allow that:
// a host framework that hands the library a fixed device-memory budget at
// set-up and forbids any later growth, a latency-critical loop in which a
// cudaMalloc/cudaFree (which may synchronise the whole device) would stall
// other streams, or code called back from another library where touching the
// CUDA allocator is not permitted.  For them this entry point runs the same
// reduction kernels as pic_diag (shared through pic_host.h) with the scratch
// placed in a fixed file-scope __device__ array, so it calls no cudaMalloc,
// cudaFree or allocating routine.
//
// Costs and limits: the array (PIC_NOALLOC_MAX_LEN doubles, 512 KiB) exists
// on every GPU that loads the library, for as long as the library stays
// loaded.  All calls share it: the part a call uses is cleared at the start of
// the call, and calls that overlap on the GPU (other streams, other threads,
// other handles on the same device) race on it and give wrong results.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/pic.h"
#include "pic_host.h"
#include "pic_runtime.h"

using namespace pic;

namespace {

constexpr size_t kNoallocMaxLen = PIC_NOALLOC_MAX_LEN;

// The scratch itself.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_diag_scratch[kNoallocMaxLen];

int bad(pic_t* h, int code, const char* msg) {
  h->err = msg;
  return code;
}

// Makes the handle's device current for the duration of a call.
struct DeviceScope {
  int prev = -1;
  cudaError_t status = cudaSuccess;
  explicit DeviceScope(int dev) {
    status = cudaGetDevice(&prev);
    if (status == cudaSuccess && prev != dev) status = cudaSetDevice(dev);
    else if (status == cudaSuccess) prev = -1;  // nothing to restore
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename T>
int diag_noalloc(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a) {
  if (!is_basic_diag(kind)) return bad(h, PIC_ERR_ARG, "pic_diag_noalloc: kind not supported");
  size_t nout = 1;
  double scale = 1.0;
  int rc = basic_diag_check(h, kind, len, a, &nout, &scale, &h->err);
  if (rc) return rc;
  if (nout > kNoallocMaxLen)
    return bad(h, PIC_ERR_ARG, "pic_diag_noalloc: result longer than PIC_NOALLOC_MAX_LEN (65536) values");
  double* scratch = h->noalloc_scratch;
  if (!scratch) return bad(h, PIC_ERR_CUDA, "pic_diag_noalloc: no device address of the scratch array");
  DeviceScope dev(h->device);
  if (dev.status != cudaSuccess) return bad(h, PIC_ERR_CUDA, "pic_diag_noalloc: cannot select the handle's device");
  // the previous call's contents stay in the array: clear what this call sums into
  if (cudaMemsetAsync(scratch, 0, nout * sizeof(double), h->stream) != cudaSuccess)
    return bad(h, PIC_ERR_CUDA, "cudaMemsetAsync of the diagnostic scratch failed");
  basic_diag_launch<T>(h, kind, len, a, scratch);
  if (cudaGetLastError() != cudaSuccess) return bad(h, PIC_ERR_CUDA, "diagnostic kernel launch failed");
  if (cudaMemcpyAsync(out, scratch, nout * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return bad(h, PIC_ERR_CUDA, "reading the diagnostic back failed");
  for (size_t i = 0; i < nout; ++i) {
    out[i] *= scale;
    if (!std::isfinite(out[i])) return bad(h, PIC_ERR_NUMERIC, "diagnostic is not finite");
  }
  return PIC_OK;
}

}  // namespace

namespace pic {

// Set-up of a handle (pic_create, with the handle's device current): the
// device address of the scratch array on that device.  Kept in the handle, so
// it lives exactly as long as the handle and its device memory.
cudaError_t noalloc_attach(pic_t* h) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_diag_scratch);
  h->noalloc_scratch = e == cudaSuccess ? p : nullptr;
  return e;
}

}  // namespace pic

extern "C" int pic_diag_noalloc(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a) {
  if (!h || !out) return PIC_ERR_ARG;
  return h->precision == PIC_FP64 ? diag_noalloc<double>(h, kind, out, len, a)
                                  : diag_noalloc<float>(h, kind, out, len, a);
}
