// pic_host.h -- host-side helpers shared by the translation units of the
// library: physical constants, launch accounting, the device views of a
// handle's arrays, and the reductions behind the field and particle
// diagnostics (used by pic_diag and by pic_diag_noalloc, which differ only in
// where their reduction scratch lives).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/pic.h"
#include "pic_kernels.cuh"
#include "pic_runtime.h"

namespace pic {

constexpr double kC = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

// Launch accounting: kernels per timing group (pic_timing_read).
enum { G_PUSH = 0, G_FIELD = 1, G_PART = 2, G_OTHER = 3 };

inline void counted(pic_t* h, int group, int n = 1) {
  h->launches[group] += n;
  h->kernels += n;
}

inline int grid_for(long long n, int per_block = 256, int cap = 152 * 32) {
  long long b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

template <typename T>
Geom<T> geom(const pic_t* h) {
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
  return g;
}

template <typename T>
Fields<T> fields(const pic_t* h) {
  Fields<T> f;
  for (int c = 0; c < NCOMP; ++c) f.c[c] = (T*)h->fields + (size_t)c * h->ncell;
  return f;
}

template <typename T>
Parts<T> parts(const pic_t* h, int b) {
  const PartBuf& pb = h->pb[b];
  Parts<T> p;
  p.cell = pb.cell;
  for (int d = 0; d < 3; ++d) {
    p.o[d] = (T*)pb.o[d];
    p.u[d] = (T*)pb.u[d];
  }
  p.w = (T*)pb.w;
  p.id = pb.id;
  return p;
}

// SI units of the normalised quantities (omega0 of the handle's grid).
struct DiagUnits {
  double E;        // V/m per m_e c omega0 / e
  double L;        // m per c / omega0
  double nc;       // critical density, 1/m^3
  double Q;        // C per unit of macroparticle weight (n_c (c/omega0)^3 electrons)
  double mc2_mev;  // rest energy of the species, MeV
};

inline DiagUnits diag_units(const pic_t* h) {
  DiagUnits u;
  u.E = kMe * kC * h->omega0 / kQe;
  u.L = kC / h->omega0;
  u.nc = kEps0 * kMe * h->omega0 * h->omega0 / (kQe * kQe);
  u.Q = kQe * u.nc * u.L * u.L * u.L;
  u.mc2_mev = kMe * kC * kC / (kQe * 1e6) * h->m;
  return u;
}

// The field and particle reductions of EX_LINEOUT, FIELD_ENERGY, CHARGE and
// SPECTRUM.  basic_diag_check validates a request and returns the number of
// result values and the factor that turns the scratch sums into SI units;
// basic_diag_launch queues the reduction into `scratch` (which the caller has
// cleared over nout values) on the handle's stream.
inline bool is_basic_diag(int kind) {
  return kind == PIC_DIAG_EX_LINEOUT || kind == PIC_DIAG_FIELD_ENERGY || kind == PIC_DIAG_CHARGE ||
         kind == PIC_DIAG_SPECTRUM;
}

inline int basic_diag_check(const pic_t* h, int kind, size_t len, const pic_diag_args* a, size_t* nout,
                            double* scale, std::string* err) {
  const DiagUnits u = diag_units(h);
  switch (kind) {
    case PIC_DIAG_EX_LINEOUT:
      if (len < (size_t)h->nx) return *err = "lineout needs len >= nx", PIC_ERR_ARG;
      *nout = h->nx;
      *scale = u.E;
      return PIC_OK;
    case PIC_DIAG_FIELD_ENERGY:
      if (len < 1) return *err = "len < 1", PIC_ERR_ARG;
      *nout = 1;
      *scale = 0.5 * h->dx * h->dy * h->dz * kEps0 * u.E * u.E * u.L * u.L * u.L;
      return PIC_OK;
    case PIC_DIAG_CHARGE:
    case PIC_DIAG_SPECTRUM:
      if (len < 1) return *err = "len < 1", PIC_ERR_ARG;
      if (!a) return *err = "diagnostic arguments required", PIC_ERR_ARG;
      if (kind == PIC_DIAG_SPECTRUM && !(a->e_max > a->e_min)) return *err = "e_max <= e_min", PIC_ERR_ARG;
      *nout = kind == PIC_DIAG_SPECTRUM ? len : 1;
      *scale = std::fabs(h->q) * u.Q;
      return PIC_OK;
    default:
      return *err = "unknown diagnostic kind", PIC_ERR_ARG;
  }
}

template <typename T>
void basic_diag_launch(pic_t* h, int kind, size_t len, const pic_diag_args* a, double* scratch) {
  const Geom<T> g = geom<T>(h);
  const Fields<T> f = fields<T>(h);
  switch (kind) {
    case PIC_DIAG_EX_LINEOUT:
      counted(h, G_OTHER);
      k_lineout<T><<<grid_for(h->nx), 256, 0, h->stream>>>(g, f.c[EX], scratch);
      break;
    case PIC_DIAG_FIELD_ENERGY:
      counted(h, G_OTHER);
      k_field_energy<T><<<grid_for((long long)h->ncell, 256, 152 * 8), 256, 0, h->stream>>>(g, f, scratch);
      break;
    default:  // CHARGE, SPECTRUM
      if (h->capacity > 0) {
        counted(h, G_OTHER);
        const size_t smem = kind == PIC_DIAG_SPECTRUM && len <= (size_t)kDiagSharedBins ? len * sizeof(double) : 0;
        k_particle_diag<T><<<grid_for(h->capacity, 256, 152 * 8), 256, smem, h->stream>>>(
            parts<T>(h, h->cur), h->d_ctrl + h->cur, kind == PIC_DIAG_SPECTRUM ? 1 : 0, a->gamma_min,
            diag_units(h).mc2_mev, a->e_min, a->e_max, (int)len, scratch);
      }
      break;
  }
}

// Look up the device address of the file-scope scratch array behind
// pic_diag_noalloc for the handle (pic_noalloc.cu; called by pic_create with
// the handle's device current).
cudaError_t noalloc_attach(pic_t* h);

}  // namespace pic
