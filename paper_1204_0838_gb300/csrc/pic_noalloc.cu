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
// reduction kernels with the scratch placed in a fixed file-scope __device__
// array, so it calls no cudaMalloc, cudaFree or allocating routine.
//
// Costs and limits: the array (kNoallocMaxLen doubles, 512 KiB) exists on
// every GPU that loads the library, for as long as the library stays loaded.
// All calls share it: the part a call uses is cleared at the start of the
// call, and calls that overlap on the GPU (other streams, other threads,
// other handles on the same device) race on it and give wrong results.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/pic.h"
#include "pic_kernels.cuh"
#include "pic_runtime.h"

using namespace pic;

namespace {

constexpr size_t kNoallocMaxLen = PIC_NOALLOC_MAX_LEN;

// The scratch itself.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_diag_scratch[kNoallocMaxLen];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (on the first call made with that device current).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_diag_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

int bad(pic_t* h, int code, const char* msg) {
  h->err = msg;
  return code;
}

template <typename T>
int diag_noalloc(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a) {
  constexpr double kC = 299792458.0, kQe = 1.602176634e-19, kMe = 9.1093837015e-31, kEps0 = 8.8541878128e-12;
  const double omega0 = h->omega0;
  const double Eunit = kMe * kC * omega0 / kQe;
  const double Lunit = kC / omega0;
  const double nc = kEps0 * kMe * omega0 * omega0 / (kQe * kQe);
  const double Qunit = kQe * nc * Lunit * Lunit * Lunit;
  const double mc2 = kMe * kC * kC / (kQe * 1e6) * h->m;

  size_t nout = 1;
  switch (kind) {
    case PIC_DIAG_EX_LINEOUT:
      if (len < (size_t)h->nx) return bad(h, PIC_ERR_ARG, "lineout needs len >= nx");
      nout = h->nx;
      break;
    case PIC_DIAG_FIELD_ENERGY:
      if (len < 1) return bad(h, PIC_ERR_ARG, "len < 1");
      break;
    case PIC_DIAG_CHARGE:
    case PIC_DIAG_SPECTRUM:
      if (len < 1) return bad(h, PIC_ERR_ARG, "len < 1");
      if (!a) return bad(h, PIC_ERR_ARG, "diagnostic arguments required");
      if (kind == PIC_DIAG_SPECTRUM && !(a->e_max > a->e_min)) return bad(h, PIC_ERR_ARG, "e_max <= e_min");
      if (kind == PIC_DIAG_SPECTRUM) nout = len;
      break;
    default:
      return bad(h, PIC_ERR_ARG, "unknown diagnostic kind");
  }
  if (nout > kNoallocMaxLen)
    return bad(h, PIC_ERR_ARG, "pic_diag_noalloc: result longer than PIC_NOALLOC_MAX_LEN (65536) values");

  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return bad(h, PIC_ERR_CUDA, "cudaGetSymbolAddress of the diagnostic scratch failed");

  Geom<T> g;
  g.nx = h->nx;
  g.ny = h->ny;
  g.nz = h->nz;
  g.origin = h->origin;
  g.periodic_x = h->periodic_x;
  g.nyz = h->ny * h->nz;
  g.dt = (T)h->dt;
  g.dx = (T)h->dx;
  g.dy = (T)h->dy;
  g.dz = (T)h->dz;
  g.dyn = nullptr;
  g.gate = 0;
  g.pml = h->pml;
  Fields<T> f;
  for (int c = 0; c < NCOMP; ++c) f.c[c] = (T*)h->fields + (size_t)c * h->ncell;
  Parts<T> p;
  const PartBuf& pb = h->pb[h->cur];
  p.cell = pb.cell;
  for (int d = 0; d < 3; ++d) {
    p.o[d] = (T*)pb.o[d];
    p.u[d] = (T*)pb.u[d];
  }
  p.w = (T*)pb.w;
  p.id = pb.id;

  // the previous call's contents stay in the array: clear what this call sums into
  if (cudaMemsetAsync(scratch, 0, nout * sizeof(double), h->stream) != cudaSuccess)
    return bad(h, PIC_ERR_CUDA, "cudaMemsetAsync of the diagnostic scratch failed");
  double scale = 1.0;
  auto blocks = [](long long n, int cap) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
  };
  switch (kind) {
    case PIC_DIAG_EX_LINEOUT:
      k_lineout<T><<<blocks(h->nx, 152 * 32), 256, 0, h->stream>>>(g, f.c[EX], scratch);
      scale = Eunit;
      break;
    case PIC_DIAG_FIELD_ENERGY:
      k_field_energy<T><<<blocks((long long)h->ncell, 152 * 8), 256, 0, h->stream>>>(g, f, scratch);
      scale = 0.5 * h->dx * h->dy * h->dz * kEps0 * Eunit * Eunit * Lunit * Lunit * Lunit;
      break;
    default:
      if (h->capacity > 0)
        k_particle_diag<T><<<blocks(h->capacity, 152 * 8), 256, 0, h->stream>>>(
            p, h->d_ctrl + h->cur, kind == PIC_DIAG_SPECTRUM ? 1 : 0, a->gamma_min, mc2, a->e_min, a->e_max,
            (int)len, scratch);
      scale = std::fabs(h->q) * Qunit;
      break;
  }
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

extern "C" int pic_diag_noalloc(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a) {
  if (!h || !out) return PIC_ERR_ARG;
  return h->precision == PIC_FP64 ? diag_noalloc<double>(h, kind, out, len, a)
                                  : diag_noalloc<float>(h, kind, out, len, a);
}
