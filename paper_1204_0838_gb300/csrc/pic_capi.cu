// pic_capi.cu -- host runtime and C-ABI of the GB300 perfect-dispersion PIC
// library (see include/pic.h).  The runtime owns device memory, sequences the
// kernels of one step on the handle's stream, keeps the moving-window
// accumulator in FP64 on the host and checks the device error word.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost nothing unless a tool is attached

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_host.h"
#include "pic_runtime.h"
#include "pic_tiled.cuh"

using namespace pic;

namespace {

int fail(pic_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(h, call)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail((h), PIC_ERR_CUDA, std::string(#call) + ": " +      \
                                       cudaGetErrorString(e_));                             \
  } while (0)

void* dalloc(pic_t* h, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(bytes, h->alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->owned.push_back(p);
  return p;
}

void dfree(pic_t* h, void* p) {
  if (!p) return;
  auto it = std::find(h->owned.begin(), h->owned.end(), p);
  if (it != h->owned.end()) h->owned.erase(it);
  if (h->has_alloc)
    h->alloc.free(p, h->alloc.ctx);
  else
    cudaFree(p);
}

// k_e_update: one thread per cell, blocks of up to 256 threads along z (a
// multiple of 32 covering nz when it is shorter), block (., j, i).
int e_update_block(const pic_t* h) { return std::min(256, (h->nz + 31) / 32 * 32); }
dim3 e_update_grid(const pic_t* h) {
  const int b = e_update_block(h);
  return dim3((h->nz + b - 1) / b, h->ny, h->nx);
}

// Optional per-group timing.
cudaEvent_t take_event(pic_t* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Per-group event timing (when enabled) and an NVTX range named for the group,
// so that profilers can select one part of the step.
struct GroupTimer {
  pic_t* h;
  int group;
  cudaEvent_t a = nullptr;
  GroupTimer(pic_t* hh, int g) : h(hh), group(g) {
    static const char* const names[4] = {"pic:gather_push_deposit", "pic:field_update", "pic:window_inject_bin",
                                         "pic:other"};
    nvtxRangePushA(names[g]);
    if (h->profiling && (a = take_event(h))) cudaEventRecord(a, h->stream);
  }
  ~GroupTimer() {
    nvtxRangePop();
    if (!a) return;
    cudaEvent_t b = take_event(h);
    if (!b) {
      h->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, h->stream);
    h->ev_pairs[group].push_back({a, b});
  }
};

// Memory variables and coefficients of the absorbing layers (L = 0: none).
template <typename T>
Pml<T> pml_view(const pic_t* h) {
  Pml<T> pm;
  pm.L = h->pml;
  pm.rows = 2 * h->pml + 1;
  T* base = (T*)h->psi;
  const size_t ny_ = (size_t)h->nx * pm.rows * h->nz, nz_ = (size_t)h->nx * h->ny * pm.rows;
  for (int c = 0; c < 4; ++c) {
    pm.py[c] = base ? base + c * ny_ : nullptr;
    pm.pz[c] = base ? base + 4 * ny_ + c * nz_ : nullptr;
  }
  pm.cy = (const T*)h->pml_coef;
  pm.cz = h->pml_coef ? (const T*)h->pml_coef + 4 * h->ny : nullptr;
  if (!base) pm.L = 0;
  return pm;
}

size_t psi_values(const pic_t* h) {
  if (!h->pml) return 0;
  const size_t rows = 2 * (size_t)h->pml + 1;
  return 4 * ((size_t)h->nx * rows * h->nz + (size_t)h->nx * h->ny * rows);
}

// Coefficients of the convolutional layer (kappa = 1, no frequency shift):
// sigma = sigma_max (depth / L)^3, sigma_max = 4 ln(1e6) / (2 L d) (a
// continuous layer reflects 1e-6 at normal incidence), b = exp(-sigma dt),
// a = b - 1.  Depth in cells at position pos (nodes integer, half nodes
// + 1/2) of an axis of n cells: max(L - pos, pos - (n - 1 - L), 0).
void pml_coefficients(const pic_t* h, int n, double d, double* out /* [4][n] */) {
  const double L = h->pml;
  const double sig_max = 4.0 * std::log(1e6) / (2.0 * L * d);
  for (int j = 0; j < n; ++j)
    for (int half = 0; half < 2; ++half) {
      const double pos = j + 0.5 * half;
      const double depth = std::max(std::max(L - pos, pos - (n - 1.0 - L)), 0.0);
      const double r = depth / L;
      const double b = std::exp(-sig_max * r * r * r * h->dt);
      out[(2 * half) * n + j] = b - 1.0;
      out[(2 * half + 1) * n + j] = b;
    }
}

template <typename T>
Smooth<T> smooth(const pic_t* h) {
  Smooth<T> s;
  for (int a = 0; a < 3; ++a) {
    s.a[a] = (T)h->sm_a[a];
    s.b1[a] = (T)h->sm_b1[a];
    s.b2[a] = (T)h->sm_b2[a];
    s.g[a] = (T)h->sm_g[a];
  }
  return s;
}

size_t esize(const pic_t* h) { return h->precision == PIC_FP64 ? 8 : 4; }

// Smoothing coefficients: a family with no dispersion along x at c dt = dx
// that is stable for every dx <= dy, dz (Sec. 2 constraint).  With
// r_b = (dx/d_b)^2: gamma_x = r_y r_z / 48, gamma_y = r_z / 48,
// gamma_z = r_y / 48, beta_a(b) = r_b / 8 - 2 gamma_a, alpha_a from
// alpha + 2 beta + 2 beta + 4 gamma = 1; the dispersion function is then
// 1 - (1 - s_x^2)(1 - r_y s_y^2)(1 - r_z s_z^2).
void set_coefficients(pic_t* h) {
  if (h->solver == PIC_SOLVER_YEE) {  // standard curl: every S_i is the identity
    for (int a = 0; a < 3; ++a) {
      h->sm_a[a] = 1.0;
      h->sm_b1[a] = h->sm_b2[a] = h->sm_g[a] = 0.0;
    }
    return;
  }
  const double r[3] = {1.0, (h->dx / h->dy) * (h->dx / h->dy), (h->dx / h->dz) * (h->dx / h->dz)};
  const int t1[3] = {1, 0, 0}, t2[3] = {2, 2, 1};
  for (int a = 0; a < 3; ++a) {
    const double g = r[t1[a]] * r[t2[a]] / 48.0;
    h->sm_g[a] = g;
    h->sm_b1[a] = r[t1[a]] / 8.0 - 2.0 * g;
    h->sm_b2[a] = r[t2[a]] / 8.0 - 2.0 * g;
    h->sm_a[a] = 1.0 - 2.0 * h->sm_b1[a] - 2.0 * h->sm_b2[a] - 4.0 * g;
  }
}

int ensure_particles(pic_t* h, long long cap) {
  if (cap <= h->capacity) return PIC_OK;
  if (cap > 0x7fffffffLL) return fail(h, PIC_ERR_ARG, "particle capacity above 2^31-1");
  const size_t es = esize(h);
  const bool ids = (h->flags & PIC_FLAG_TRACK_IDS) != 0;
  const size_t per = 4 + 7 * es + (ids ? 4 : 0);
  PartBuf nb[2];
  for (int b = 0; b < 2; ++b) {
    char* base = (char*)dalloc(h, per * (size_t)cap + 8 * 256);
    if (!base) return fail(h, PIC_ERR_OOM, "particle buffer allocation failed");
    nb[b].base = base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
      char* p = base + off;
      off += (bytes + 255) & ~size_t(255);
      return (void*)p;
    };
    nb[b].cell = (int*)take(4 * (size_t)cap);
    for (int d = 0; d < 3; ++d) nb[b].o[d] = take(es * cap);
    for (int d = 0; d < 3; ++d) nb[b].u[d] = take(es * cap);
    nb[b].w = take(es * cap);
    nb[b].id = ids ? (uint32_t*)take(4 * (size_t)cap) : nullptr;
  }
  int* nkeys = (int*)dalloc(h, 4 * (size_t)cap);
  if (!nkeys) return fail(h, PIC_ERR_OOM, "particle key allocation failed");
  // carry the live particles over
  int np = 0;
  if (h->capacity > 0) {
    CK(h, cudaMemcpyAsync(&np, h->d_ctrl + h->cur, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const PartBuf& ob = h->pb[h->cur];
    if (np > 0) {
      CK(h, cudaMemcpyAsync(nb[0].cell, ob.cell, 4 * (size_t)np, cudaMemcpyDeviceToDevice, h->stream));
      for (int d = 0; d < 3; ++d) {
        CK(h, cudaMemcpyAsync(nb[0].o[d], ob.o[d], es * np, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, cudaMemcpyAsync(nb[0].u[d], ob.u[d], es * np, cudaMemcpyDeviceToDevice, h->stream));
      }
      CK(h, cudaMemcpyAsync(nb[0].w, ob.w, es * np, cudaMemcpyDeviceToDevice, h->stream));
      if (ids) CK(h, cudaMemcpyAsync(nb[0].id, ob.id, 4 * (size_t)np, cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    dfree(h, h->pb[0].base);
    dfree(h, h->pb[1].base);
    dfree(h, h->keys);
  }
  h->pb[0] = nb[0];
  h->pb[1] = nb[1];
  h->keys = nkeys;
  h->cur = 0;
  h->capacity = cap;
  h->need_sort = true;
  CK(h, cudaMemcpyAsync(h->d_ctrl, &np, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

Laser laser_params(const pic_t* h) {
  Laser L;
  L.a0k = h->las_a0 * h->las_k;
  L.k = h->las_k;
  L.w0 = h->las_w0;
  L.zr = 0.5 * h->las_k * h->las_w0 * h->las_w0;
  L.tau = h->las_tau;
  L.xf = h->las_xf;
  L.tpk = h->las_tpk;
  L.yc = 0.5 * h->ny * h->dy;
  L.zc = 0.5 * h->nz * h->dz;
  return L;
}

int x_lo(const pic_t* h) { return h->periodic_x ? 0 : 2; }
int x_hi(const pic_t* h) { return h->periodic_x ? h->nx - 1 : h->nx - 4; }

// Loading parameters for window-relative x cells [lo, hi].
LoadSpec load_spec(const pic_t* h, int lo, int hi) {
  LoadSpec L;
  L.shifts = h->shifts;
  L.lo = lo;
  L.hi = hi;
  L.ppc = h->ppc;
  L.lattice = h->loading == PIC_LOAD_LATTICE;
  for (int d = 0; d < 3; ++d) L.ns[d] = h->lat[d];
  L.seed = h->seed;
  L.x0 = h->x0;
  L.dx = h->dx;
  L.dVppc = h->dx * h->dy * h->dz / h->ppc;
  L.px = h->d_prof;
  L.pn = h->d_prof + h->nprof;
  L.np = h->nprof;
  L.capacity = (int)h->capacity;
  L.pml = h->pml;
  return L;
}

template <typename T>
int load_cells(pic_t* h, int lo, int hi) {
  const LoadSpec L = load_spec(h, lo, hi);
  const long long nslot = (long long)(hi - lo + 1) * h->ny * h->nz * h->ppc;
  GroupTimer tm(h, G_PART);
  k_load<T><<<grid_for(nslot, 256, 152 * 64), 256, 0, h->stream>>>(geom<T>(h), parts<T>(h, h->cur),
                                                                     h->d_ctrl + h->cur, h->d_ctrl + 2, L);
  k_clamp_count<<<1, 32, 0, h->stream>>>(h->d_ctrl + h->cur, (int)h->capacity);
  counted(h, G_PART, 2);
  CK(h, cudaGetLastError());
  return PIC_OK;
}

template <typename T>
int hard_source(pic_t* h, double t) {
  const Laser L = laser_params(h);
  const double xplane = h->x0 + (double)h->shifts * h->dx;
  GroupTimer tm(h, G_OTHER);
  counted(h, G_OTHER);
  k_hard_source<T><<<grid_for(h->ny * h->nz), 256, 0, h->stream>>>(geom<T>(h), fields<T>(h).c[EY], L, xplane, t,
                                                                    h->dy, h->dz);
  CK(h, cudaGetLastError());
  return PIC_OK;
}

template <typename T>
int laser_in_box(pic_t* h) {
  const size_t n = h->ncell;
  T* tmp = (T*)dalloc(h, 6 * n * sizeof(T));
  if (!tmp) return fail(h, PIC_ERR_OOM, "laser scratch allocation failed");
  CK(h, cudaMemsetAsync(tmp, 0, 6 * n * sizeof(T), h->stream));
  T* E[3] = {tmp, tmp + n, tmp + 2 * n};
  T* B[3] = {tmp + 3 * n, tmp + 4 * n, tmp + 5 * n};
  const Geom<T> g = geom<T>(h);
  const Laser L = laser_params(h);
  const double t = (double)h->step * h->dt;
  const double xnode0 = h->x0 + (double)h->shifts * h->dx;
  counted(h, G_OTHER, 9);
  k_laser_fill<T><<<grid_for(n), 256, 0, h->stream>>>(g, E[1], B[2], L, xnode0, h->dx, h->dy, h->dz, t, h->dt);
  k_laser_scan<T><<<grid_for(h->ny * h->nz, 128), 128, 0, h->stream>>>(g, E[1], E[0], B[2], B[0]);
  k_curl_e<T><<<grid_for(n), 256, 0, h->stream>>>(g, smooth<T>(h), E[0], E[1], E[2], B[0], B[1], B[2],
                                                   (T)(0.5 * h->dt));
  Fields<T> f = fields<T>(h);
  for (int c = 0; c < 3; ++c) {
    k_add<T><<<grid_for(n), 256, 0, h->stream>>>(f.c[EX + c], E[c], (long long)n);
    k_add<T><<<grid_for(n), 256, 0, h->stream>>>(f.c[BX + c], B[c], (long long)n);
  }
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->stream));
  dfree(h, tmp);
  return PIC_OK;
}

template <typename T>
FieldCoef<T> field_coef(const pic_t* h) {
  FieldCoef<T> c;
  c.dt = (T)h->dt;
  c.hdt = (T)(0.5 * h->dt);
  c.idx = (T)(1.0 / h->dx);
  c.idy = (T)(1.0 / h->dy);
  c.idz = (T)(1.0 / h->dz);
  return c;
}

template <typename T>
Fields<T> curl_view(const pic_t* h) {
  Fields<T> c;
  for (int i = 0; i < NCOMP; ++i) c.c[i] = nullptr;
  for (int i = 0; i < 3; ++i) c.c[i] = (T*)h->curl + (size_t)i * h->ncell;
  return c;
}

// Launch of the tiled smoothed curl over window-relative slabs [i0, i0 + ni).
template <typename T>
void launch_curl(const pic_t* h, const Geom<T>& g, int mode, int i0, int ni, cudaStream_t s) {
  const dim3 grid((ni + CB_X - 1) / CB_X, (h->ny + CB_Y - 1) / CB_Y, (h->nz + CB_Z - 1) / CB_Z);
  k_curl_tiled<T><<<grid, 256, curl_tiled_smem_bytes<T>(), s>>>(g, smooth<T>(h), fields<T>(h), curl_view<T>(h),
                                                               field_coef<T>(h), mode, i0, ni, pml_view<T>(h));
}

// C = curl'(E) over window-relative slabs [i0, i0 + ni).
template <typename T>
int curl_only(pic_t* h, int i0, int ni) {
  GroupTimer tm(h, G_FIELD);
  counted(h, G_FIELD);
  launch_curl<T>(h, geom<T>(h), 0, i0, ni, h->stream);
  CK(h, cudaGetLastError());
  return PIC_OK;
}

// Counting sort of the current buffer by tile into the other buffer.
template <typename T>
int resort_all(pic_t* h) {
  if (h->capacity == 0) return PIC_OK;
  const int nb = 1 - h->cur;
  const Tiles tl = h->tiles;
  GroupTimer tm(h, G_PART);
  CK(h, cudaMemsetAsync(h->tcnt, 0, sizeof(int) * tl.n, h->stream));
  CK(h, cudaMemsetAsync(h->tfill, 0, sizeof(int) * tl.n, h->stream));
  k_keys<T><<<grid_for(h->capacity, 256, 152 * 16), 256, 0, h->stream>>>(geom<T>(h), tl, parts<T>(h, h->cur),
                                                                         h->d_ctrl + h->cur, h->keys, h->tcnt);
  k_scan_tiles<<<1, 1024, 0, h->stream>>>(h->tcnt, h->tstart[nb], tl.n, h->d_ctrl + nb, (int)h->capacity,
                                          h->d_ctrl + 2);
  k_scatter<T><<<grid_for(h->capacity, 256, 152 * 16), 256, 0, h->stream>>>(
      parts<T>(h, h->cur), h->keys, h->d_ctrl + h->cur, parts<T>(h, nb), h->tstart[nb], h->tfill, h->d_ctrl + 2);
  counted(h, G_PART, 3);
  CK(h, cudaGetLastError());
  h->cur = nb;
  return PIC_OK;
}

// Window decision for the step that ends at t_new: returns 1 if the window
// moves one cell at the end of this step (v <= c and c dt <= dx: at most one).
int window_due(pic_t* h, double t_old, double t_new, double* frac_new) {
  *frac_new = h->win_frac;
  if (!h->has_window || !(t_new > h->win_t0)) return 0;
  *frac_new = h->win_frac + h->win_v * (t_old >= h->win_t0 ? h->dt : (t_new - h->win_t0)) / h->dx;
  return *frac_new >= 1.0 ? 1 : 0;
}

template <typename T>
int zero_front_slab(pic_t* h, int storage_slab) {
  Fields<T> f = fields<T>(h);
  const size_t slab = (size_t)h->ny * h->nz;
  for (int c = 0; c < NCOMP; ++c)
    CK(h, cudaMemsetAsync(f.c[c] + (size_t)storage_slab * slab, 0, slab * sizeof(T), h->stream));
  const Pml<T> pm = pml_view<T>(h);
  for (int c = 0; c < 4 && pm.L; ++c) {
    const size_t ny_ = (size_t)pm.rows * h->nz, nz_ = (size_t)h->ny * pm.rows;
    CK(h, cudaMemsetAsync(pm.py[c] + (size_t)storage_slab * ny_, 0, ny_ * sizeof(T), h->stream));
    CK(h, cudaMemsetAsync(pm.pz[c] + (size_t)storage_slab * nz_, 0, nz_ * sizeof(T), h->stream));
  }
  return PIC_OK;
}

template <typename T>
int field_first_half(pic_t* h) {
  if (!h->curl_valid) {
    int rc = curl_only<T>(h, 0, h->nx);
    if (rc) return rc;
    h->curl_valid = true;
  }
  GroupTimer tm(h, G_FIELD);
  counted(h, G_FIELD);
  k_e_update<T><<<e_update_grid(h), e_update_block(h), 0, h->stream>>>(geom<T>(h), fields<T>(h), curl_view<T>(h),
                                                         field_coef<T>(h), pml_view<T>(h));
  CK(h, cudaGetLastError());
  return PIC_OK;
}

template <typename T>
int field_second_half(pic_t* h) {
  GroupTimer tm(h, G_FIELD);
  counted(h, G_FIELD);
  launch_curl<T>(h, geom<T>(h), 1, 0, h->nx, h->stream);
  CK(h, cudaGetLastError());
  return PIC_OK;
}

// After a shift the storage slab that left at the back is the new, zeroed
// front slab; the cached curl is recomputed where the window edges moved.
template <typename T>
int after_shift_fields(pic_t* h, int old_origin) {
  int rc = zero_front_slab<T>(h, old_origin);
  if (rc) return rc;
  if (h->curl_valid) {
    rc = curl_only<T>(h, 0, 1);
    if (!rc) rc = curl_only<T>(h, h->nx - 1, 1);
  }
  return rc;
}

// One step with tile-sorted particles.
template <typename T>
int step_tiled(pic_t* h) {
  const size_t n = h->ncell;
  Fields<T> f = fields<T>(h);
  const double t_old = (double)h->step * h->dt, t_new = (double)(h->step + 1) * h->dt;
  double frac_new;
  const int shift = window_due(h, t_old, t_new, &frac_new);
  const int origin_after = shift ? (h->origin + 1) % h->nx : h->origin;
  const Tiles tl = h->tiles;
  const int nb = 1 - h->cur;
  CK(h, cudaMemsetAsync(f.c[JX], 0, 3 * n * sizeof(T), h->stream));
  if (h->capacity > 0) {
    CK(h, cudaMemsetAsync(h->tcnt, 0, sizeof(int) * tl.n, h->stream));
    GroupTimer tm(h, G_PUSH);
    counted(h, G_PUSH);
    const T hq = (T)(h->q * h->dt / (2.0 * h->m));
    k_push_tiled<T><<<tl.n, push_threads<T>(), tiled_smem_bytes<T>(tl), h->stream>>>(
        geom<T>(h), tl, f, parts<T>(h, h->cur), h->tstart[h->cur], (int)h->capacity, h->keys, h->tcnt, hq,
        (T)h->q, origin_after, x_lo(h), x_hi(h), h->d_pushed, h->d_ctrl + 2);
    CK(h, cudaGetLastError());
  }
  int rc = field_first_half<T>(h);
  if (rc) return rc;
  h->step += 1;
  if (h->laser_mode == PIC_LASER_HARD_SOURCE) {
    rc = hard_source<T>(h, t_new);
    if (rc) return rc;
  }
  rc = field_second_half<T>(h);
  if (rc) return rc;
  h->win_frac = frac_new;
  LoadSpec L;
  if (shift) {
    h->win_frac -= 1.0;
    const int old_origin = h->origin;
    h->origin = origin_after;
    h->shifts += 1;
    rc = after_shift_fields<T>(h, old_origin);
    if (rc) return rc;
  }
  if (h->capacity == 0) return PIC_OK;
  GroupTimer tm(h, G_PART);
  const bool inject = shift && h->has_species;
  if (inject) {
    L = load_spec(h, x_hi(h), x_hi(h));
    const long long nslot = (long long)h->ny * h->nz * h->ppc;
    k_inject_tiled<T><<<grid_for(nslot, 256, 152 * 16), 256, 0, h->stream>>>(
        geom<T>(h), tl, parts<T>(h, nb), L, 0, h->tcnt, h->tstart[nb], h->tfill, h->d_ctrl + 2);
    counted(h, G_PART);
  }
  k_scan_tiles<<<1, 1024, 0, h->stream>>>(h->tcnt, h->tstart[nb], tl.n, h->d_ctrl + nb, (int)h->capacity,
                                          h->d_ctrl + 2);
  CK(h, cudaMemsetAsync(h->tfill, 0, sizeof(int) * tl.n, h->stream));
  k_scatter<T><<<grid_for(h->capacity, 256, 152 * 16), 256, 0, h->stream>>>(
      parts<T>(h, h->cur), h->keys, h->d_ctrl + h->cur, parts<T>(h, nb), h->tstart[nb], h->tfill, h->d_ctrl + 2);
  counted(h, G_PART, 2);
  if (inject) {
    const long long nslot = (long long)h->ny * h->nz * h->ppc;
    k_inject_tiled<T><<<grid_for(nslot, 256, 152 * 16), 256, 0, h->stream>>>(
        geom<T>(h), tl, parts<T>(h, nb), L, 1, h->tcnt, h->tstart[nb], h->tfill, h->d_ctrl + 2);
    counted(h, G_PART);
  }
  CK(h, cudaGetLastError());
  h->cur = nb;
  return PIC_OK;
}

template <typename T>
int step_impl(pic_t* h, int nsteps) {
  if (h->need_sort && nsteps > 0) {
    int rc = resort_all<T>(h);
    if (rc) return rc;
    h->need_sort = false;
  }
  for (int it = 0; it < nsteps; ++it) {
    int rc = step_tiled<T>(h);
    if (rc) return rc;
  }
  return PIC_OK;
}

int check_device_error(pic_t* h);

// Between calls: if the live count is within 20% of the capacity and the
// caller did not fix the capacity, grow the buffers by half.
int grow_if_needed(pic_t* h) {
  if (h->capacity == 0 || h->max_particles > 0) return PIC_OK;
  if ((double)h->np_host < 0.8 * (double)h->capacity) return PIC_OK;
  return ensure_particles(h, std::min<long long>(0x7fffffffLL, h->capacity * 3 / 2 + 4096));
}

int check_device_error(pic_t* h) {
  int ctrl[6];
  CK(h, cudaMemcpyAsync(ctrl, h->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->np_host = ctrl[h->cur];
  unsigned long long pushed;
  std::memcpy(&pushed, ctrl + 4, sizeof(pushed));
  h->pushed_host = (long long)pushed;
  if (ctrl[2] & 1) {
    return fail(h, PIC_ERR_CAPACITY, "particle capacity exceeded during loading/injection");
  }
  if (ctrl[2] & 6) return fail(h, PIC_ERR_STATE, "tile bookkeeping error in the particle binning");
  if (ctrl[2] & 16) return fail(h, PIC_ERR_STATE, "a tile held 2^20 or more particles (FP32 current tile range)");
  if (ctrl[2] & 8) {
    // reported once: the offending particles were absorbed
    const int zero = 0;
    CK(h, cudaMemcpyAsync(h->d_ctrl + 2, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return fail(h, PIC_ERR_NUMERIC, "non-finite particle momentum: the particle was absorbed");
  }
  return PIC_OK;
}

// Gauss-law residual: out[0] = max |div E - rho| / max |rho_e| over the nodes
// (rho = electrons plus immobile ions; max |div E - rho| itself when there is
// no electron charge); with len >= 3 also out[1] = max |div E - rho| and
// out[2] = max |rho_e|, in C/m^3.  Scratch: [2 words][rho_e][rho_i].
template <typename T>
int gauss_residual(pic_t* h, double* out, size_t len) {
  const Geom<T> g = geom<T>(h);
  double* rho_e = h->d_diag + 2;
  double* rho_i = rho_e + h->ncell;
  const double dV = h->dx * h->dy * h->dz;
  if (h->capacity > 0) {
    counted(h, G_OTHER);
    k_rho_particles<T><<<grid_for(h->capacity, 256, 152 * 8), 256, 0, h->stream>>>(
        g, parts<T>(h, h->cur), h->d_ctrl + h->cur, h->q / dV, rho_e);
  }
  if (h->has_species) {
    // every lab cell loaded so far: the set-up load and one front slab per shift
    const int lo = h->periodic_x ? 0 : (int)std::max<long long>(h->ion_lab_lo - h->shifts, -2);
    const int hi = x_hi(h);
    if (lo <= hi) {
      const LoadSpec L = load_spec(h, lo, hi);
      counted(h, G_OTHER);
      k_rho_ions<T><<<grid_for((long long)(hi - lo + 1) * h->ny * h->nz * h->ppc, 256, 152 * 8), 256, 0,
                      h->stream>>>(g, L, -h->q / dV, rho_i);
    }
  }
  counted(h, G_OTHER);
  k_gauss_residual<T><<<grid_for((long long)h->ncell, 256, 152 * 8), 256, 0, h->stream>>>(
      g, fields<T>(h), rho_e, rho_i, 1.0 / h->dx, 1.0 / h->dy, 1.0 / h->dz, (unsigned long long*)h->d_diag);
  CK(h, cudaGetLastError());
  double m[2];
  CK(h, cudaMemcpyAsync(m, h->d_diag, sizeof(m), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  const double qsi = kQe * diag_units(h).nc;  // e n_c: C/m^3 per normalised charge density
  out[0] = m[1] > 0 ? m[0] / m[1] : m[0];
  if (len >= 3) {
    out[1] = m[0] * qsi;
    out[2] = m[1] * qsi;
  }
  for (size_t i = 0; i < std::min<size_t>(len, 3); ++i)
    if (!std::isfinite(out[i])) return fail(h, PIC_ERR_NUMERIC, "diagnostic is not finite");
  return PIC_OK;
}

template <typename T>
int diag_impl(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a) {
  const DiagUnits un = diag_units(h);
  size_t need = std::max<size_t>(std::max<size_t>(len, 11), (size_t)h->nx * h->ny);
  if (kind == PIC_DIAG_DIVE_RESIDUAL) {
    if (len < 1) return fail(h, PIC_ERR_ARG, "len < 1");
    need = std::max(need, 2 + 2 * h->ncell);
  }
  if (need > h->diag_cap) {
    dfree(h, h->d_diag);
    h->d_diag = (double*)dalloc(h, need * sizeof(double));
    if (!h->d_diag) {
      h->diag_cap = 0;
      return fail(h, PIC_ERR_OOM, "diagnostic scratch allocation failed");
    }
    h->diag_cap = need;
  }
  CK(h, cudaMemsetAsync(h->d_diag, 0, need * sizeof(double), h->stream));
  if (kind == PIC_DIAG_DIVE_RESIDUAL) return gauss_residual<T>(h, out, len);
  const Geom<T> g = geom<T>(h);
  double scale = 1.0;
  size_t nout = 1;
  if (is_basic_diag(kind)) {
    int rc = basic_diag_check(h, kind, len, a, &nout, &scale, &h->err);
    if (rc) return rc;
    basic_diag_launch<T>(h, kind, len, a, h->d_diag);
  } else switch (kind) {
    case PIC_DIAG_EMITTANCE: {
      if (len < 2) return fail(h, PIC_ERR_ARG, "emittance needs len >= 2");
      if (!a) return fail(h, PIC_ERR_ARG, "diagnostic arguments required");
      if (need < 11) return fail(h, PIC_ERR_ARG, "internal: scratch");
      if (h->capacity > 0) {
        counted(h, G_OTHER);
        k_emittance_moments<T><<<grid_for(h->capacity, 256, 152 * 8), 256, 0, h->stream>>>(
            g, parts<T>(h, h->cur), h->d_ctrl + h->cur, a->gamma_min, h->d_diag);
      }
      CK(h, cudaGetLastError());
      double m[11];
      CK(h, cudaMemcpyAsync(m, h->d_diag, sizeof(m), cudaMemcpyDeviceToHost, h->stream));
      CK(h, cudaStreamSynchronize(h->stream));
      for (int ax = 0; ax < 2; ++ax) {
        double e = 0.0;
        if (m[0] > 0) {
          const double W = m[0];
          const double mu = m[1 + 5 * ax] / W, mu2 = m[2 + 5 * ax] / W, mr = m[3 + 5 * ax] / W;
          const double mr2 = m[4 + 5 * ax] / W, mur = m[5 + 5 * ax] / W;
          const double var_u = mu2 - mu * mu, var_r = mr2 - mr * mr, cov = mur - mu * mr;
          const double det = var_u * var_r - cov * cov;
          e = det > 0 ? std::sqrt(det) : 0.0;
        }
        out[ax] = e * un.L;  // normalised length -> metres (u is dimensionless)
        if (!std::isfinite(out[ax])) return fail(h, PIC_ERR_NUMERIC, "diagnostic is not finite");
      }
      return PIC_OK;
    }
    case PIC_DIAG_PHASE_X_PX: {
      if (!a || !(a->p_max > a->p_min)) return fail(h, PIC_ERR_ARG, "p_max <= p_min");
      if (len < (size_t)h->nx || len % (size_t)h->nx) return fail(h, PIC_ERR_ARG, "len must be nx * bins");
      if (h->capacity > 0) {
        counted(h, G_OTHER);
        k_phase_x_px<T><<<grid_for(h->capacity, 256, 152 * 8), 256, 0, h->stream>>>(
            g, parts<T>(h, h->cur), h->d_ctrl + h->cur, a->p_min, a->p_max, (int)(len / h->nx), h->d_diag);
      }
      scale = std::fabs(h->q) * un.Q;
      nout = len;
      break;
    }
    case PIC_DIAG_DENSITY_XY: {
      if (len < (size_t)h->nx * h->ny) return fail(h, PIC_ERR_ARG, "density map needs len >= nx * ny");
      if (h->capacity > 0) {
        counted(h, G_OTHER);
        k_density_xy<T><<<grid_for(h->capacity, 256, 152 * 8), 256, 0, h->stream>>>(
            g, parts<T>(h, h->cur), h->d_ctrl + h->cur, h->d_diag);
      }
      scale = 1.0 / (h->dx * h->dy * h->dz);  // weight per cell volume: n / n_c
      nout = (size_t)h->nx * h->ny;
      break;
    }
    default:
      return fail(h, PIC_ERR_ARG, "unknown diagnostic kind");
  }
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(out, h->d_diag, nout * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < nout; ++i) {
    out[i] *= scale;
    if (!std::isfinite(out[i])) return fail(h, PIC_ERR_NUMERIC, "diagnostic is not finite");
  }
  return PIC_OK;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

const char* pic_version(void) { return "paper_1204_0838_gb300 0.1 (sm_103a)"; }

const char* pic_last_error(const pic_t* h) { return h ? h->err.c_str() : "null handle"; }

int pic_create(const pic_grid* g, double dt, const pic_window* w, pic_t** out) {
  if (!g || !out) return PIC_ERR_ARG;
  *out = nullptr;
  if (g->nx < 16 || g->ny < 4 || g->nz < 4) return PIC_ERR_ARG;
  if (g->nx > 65535 || g->ny > 65535) return PIC_ERR_ARG;  // launch grid extents of the field kernels
  if ((long long)g->nx * g->ny * g->nz > 0x7fffffffLL) return PIC_ERR_ARG;
  if (!(g->dx > 0 && g->dy > 0 && g->dz > 0 && g->lambda0 > 0)) return PIC_ERR_ARG;
  if (g->dx > g->dy || g->dx > g->dz) return PIC_ERR_ARG;  // Sec. 2: dx <= dy, dz
  if (g->precision != PIC_FP64 && g->precision != PIC_FP32) return PIC_ERR_ARG;
  if (g->bc_x != PIC_BC_PERIODIC && g->bc_x != PIC_BC_OPEN) return PIC_ERR_ARG;
  if (g->solver != PIC_SOLVER_PERFECT && g->solver != PIC_SOLVER_YEE) return PIC_ERR_ARG;
  if (w && g->bc_x != PIC_BC_OPEN) return PIC_ERR_ARG;
  if (g->alloc && (!g->alloc->alloc || !g->alloc->free)) return PIC_ERR_ARG;
  // absorbing layers: room for the particles' cubic stencils inside the grid
  if (g->pml < 0 || (g->pml > 0 && (g->pml < 3 || g->ny < 2 * g->pml + 4 || g->nz < 2 * g->pml + 4)))
    return PIC_ERR_ARG;
  pic_t* h = new (std::nothrow) pic_t();
  if (!h) return PIC_ERR_OOM;
  h->precision = g->precision;
  h->nx = g->nx;
  h->ny = g->ny;
  h->nz = g->nz;
  h->ncell = (size_t)g->nx * g->ny * g->nz;
  h->periodic_x = g->bc_x == PIC_BC_PERIODIC;
  h->lambda0 = g->lambda0;
  h->k0 = 2.0 * kPi / g->lambda0;
  h->omega0 = h->k0 * kC;
  h->dx = g->dx * h->k0;
  h->dy = g->dy * h->k0;
  h->dz = g->dz * h->k0;
  h->x0 = g->x0 * h->k0;
  h->seed = g->seed;
  h->flags = g->flags;
  h->max_particles = g->max_particles;
  h->solver = g->solver;
  h->pml = g->pml;
  if (h->solver == PIC_SOLVER_YEE) {
    const double lim = 1.0 / std::sqrt(1.0 / (h->dx * h->dx) + 1.0 / (h->dy * h->dy) + 1.0 / (h->dz * h->dz));
    h->dt = dt > 0 ? dt * h->omega0 : 0.999 * lim;
    if (h->dt > lim * (1.0 + 1e-12)) {
      delete h;
      return PIC_ERR_ARG;  // Courant limit of the standard Yee scheme
    }
  } else {
    h->dt = dt > 0 ? dt * h->omega0 : h->dx;
    if (h->dt > h->dx * (1.0 + 1e-12)) {
      delete h;
      return PIC_ERR_ARG;  // c dt <= dx keeps the scheme stable for dx <= dy, dz
    }
  }
  if (g->alloc) {
    h->alloc = *g->alloc;
    h->has_alloc = true;
  }
  if (w) {
    if (!(w->v >= 0.0 && w->v <= 1.0)) {
      delete h;
      return PIC_ERR_ARG;  // the window moves at most at c (one cell per step)
    }
    h->has_window = true;
    h->win_v = w->v;
    h->win_t0 = w->t_start * h->omega0;
  }
  {
    int t3[3] = {8, 8, 8};
    const char* ts = std::getenv("PIC_TILE");
    if (ts) std::sscanf(ts, "%d,%d,%d", &t3[0], &t3[1], &t3[2]);
    const int n3[3] = {h->nx, h->ny, h->nz};
    for (int d = 0; d < 3; ++d) t3[d] = std::max(1, std::min(t3[d], n3[d]));
    Tiles& tl = h->tiles;
    tl.tx = t3[0];
    tl.ty = t3[1];
    tl.tz = t3[2];
    // keep the shared-memory tile within the 227 KB a CTA may use
    auto smem = [&]() {
      return h->precision == PIC_FP64 ? tiled_smem_bytes<double>(tl) : tiled_smem_bytes<float>(tl);
    };
    while (smem() > 227 * 1024) {
      if (tl.tx >= tl.ty && tl.tx >= tl.tz) tl.tx /= 2;
      else if (tl.ty >= tl.tz) tl.ty /= 2;
      else tl.tz /= 2;
    }
    tl.ntx = (h->nx + tl.tx - 1) / tl.tx;
    tl.nty = (h->ny + tl.ty - 1) / tl.ty;
    tl.ntz = (h->nz + tl.tz - 1) / tl.tz;
    tl.n = tl.ntx * tl.nty * tl.ntz;
  }
  set_coefficients(h);
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return PIC_ERR_CUDA;
  }
  // pic_diag_noalloc's scratch address on this device; a failure here only
  // disables that call (it then returns PIC_ERR_CUDA)
  if (noalloc_attach(h) != cudaSuccess) cudaGetLastError();
  h->stream = h->own_stream;
  h->fields = dalloc(h, NCOMP * h->ncell * esize(h));
  h->curl = dalloc(h, 3 * h->ncell * esize(h));
  h->tstart[0] = (int*)dalloc(h, sizeof(int) * (h->tiles.n + 1));
  h->tstart[1] = (int*)dalloc(h, sizeof(int) * (h->tiles.n + 1));
  h->tcnt = (int*)dalloc(h, sizeof(int) * h->tiles.n);
  h->tfill = (int*)dalloc(h, sizeof(int) * h->tiles.n);
  h->tiles_alloc = h->tiles.n;
  if (!h->curl || !h->tstart[0] || !h->tstart[1] || !h->tcnt || !h->tfill) {
    pic_destroy(h);
    return PIC_ERR_OOM;
  }
  {
    // the limit is a property of the kernel, shared by every handle: allow the
    // largest tile any handle may pick (227 KB); each launch asks for its own
    const int sm = 227 * 1024;
    cudaError_t e = h->precision == PIC_FP64
                        ? cudaFuncSetAttribute(k_push_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)
                        : cudaFuncSetAttribute(k_push_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = h->precision == PIC_FP64 ? cudaFuncSetAttribute(k_curl_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)curl_tiled_smem_bytes<double>())
                                   : cudaFuncSetAttribute(k_curl_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)curl_tiled_smem_bytes<float>());
    if (e != cudaSuccess) {
      cudaGetLastError();
      pic_destroy(h);
      return PIC_ERR_CUDA;
    }
  }
  h->d_ctrl = (int*)dalloc(h, 64);
  h->d_pushed = h->d_ctrl ? (unsigned long long*)(h->d_ctrl + 4) : nullptr;
  if (!h->fields || !h->d_ctrl) {
    pic_destroy(h);
    return PIC_ERR_OOM;
  }
  if (h->pml) {
    h->psi = dalloc(h, psi_values(h) * esize(h));
    h->pml_coef = dalloc(h, 4 * (size_t)(h->ny + h->nz) * esize(h));
    if (!h->psi || !h->pml_coef) {
      pic_destroy(h);
      return PIC_ERR_OOM;
    }
    std::vector<double> c(4 * (size_t)(h->ny + h->nz));
    pml_coefficients(h, h->ny, h->dy, c.data());
    pml_coefficients(h, h->nz, h->dz, c.data() + 4 * h->ny);
    std::vector<float> cf(c.begin(), c.end());
    const void* src = h->precision == PIC_FP64 ? (const void*)c.data() : (const void*)cf.data();
    cudaError_t e = cudaMemcpyAsync(h->pml_coef, src, c.size() * esize(h), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->psi, 0, psi_values(h) * esize(h), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // the host copies die here
    if (e != cudaSuccess) {
      cudaGetLastError();
      pic_destroy(h);
      return PIC_ERR_CUDA;
    }
  }
  if (cudaMemsetAsync(h->fields, 0, NCOMP * h->ncell * esize(h), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->tstart[0], 0, sizeof(int) * (h->tiles.n + 1), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->tstart[1], 0, sizeof(int) * (h->tiles.n + 1), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_ctrl, 0, 64, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    pic_destroy(h);
    return PIC_ERR_CUDA;
  }
  *out = h;
  return PIC_OK;
}

int pic_set_stream(pic_t* h, void* stream) {
  if (!h) return PIC_ERR_ARG;
  CK(h, cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  return PIC_OK;
}

int pic_add_species(pic_t* h, const pic_profile* n, int ppc, int spline_order, double q, double m,
                    int loading) {
  if (!h) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  if (h->has_species) return fail(h, PIC_ERR_STATE, "one species per handle");
  if (!n || n->n < 1 || !n->x || !n->dens) return fail(h, PIC_ERR_ARG, "bad profile");
  if (spline_order != 3) return fail(h, PIC_ERR_ARG, "only cubic (order 3) splines");
  if (ppc < 1 || !(m > 0)) return fail(h, PIC_ERR_ARG, "bad ppc or mass");
  int lat[3] = {1, 1, 1};
  if (loading == PIC_LOAD_LATTICE) {
    switch (ppc) {
      case 1: break;
      case 2: lat[1] = 2; break;
      case 4: lat[1] = 2; lat[2] = 2; break;
      case 8: lat[0] = 2; lat[1] = 2; lat[2] = 2; break;
      default: return fail(h, PIC_ERR_ARG, "lattice loading needs ppc in {1,2,4,8}");
    }
  } else if (loading != PIC_LOAD_RANDOM) {
    return fail(h, PIC_ERR_ARG, "unknown loading");
  }
  for (int i = 0; i + 1 < n->n; ++i)
    if (n->x[i + 1] < n->x[i]) return fail(h, PIC_ERR_ARG, "profile x must be non-decreasing");
  std::vector<double> prof(2 * (size_t)n->n);
  for (int i = 0; i < n->n; ++i) {
    prof[i] = n->x[i] * h->k0;
    prof[n->n + i] = n->dens[i];
  }
  h->d_prof = (double*)dalloc(h, prof.size() * sizeof(double));
  if (!h->d_prof) return fail(h, PIC_ERR_OOM, "profile allocation failed");
  CK(h, cudaMemcpyAsync(h->d_prof, prof.data(), prof.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  h->nprof = n->n;
  h->ppc = ppc;
  h->loading = loading;
  for (int d = 0; d < 3; ++d) h->lat[d] = lat[d];
  h->q = q;
  h->m = m;
  // default capacity: 25% above one full load, for compression by the wake
  long long cap = h->max_particles > 0 ? h->max_particles : (long long)h->ncell * ppc * 5 / 4 + 4096;
  int rc = ensure_particles(h, cap);
  if (rc) return rc;
  h->has_species = true;
  h->ion_lab_lo = h->shifts + x_lo(h);
  rc = h->precision == PIC_FP64 ? load_cells<double>(h, x_lo(h), x_hi(h)) : load_cells<float>(h, x_lo(h), x_hi(h));
  if (rc) return rc;
  h->need_sort = true;
  return check_device_error(h);
}

int pic_add_laser(pic_t* h, double a0, double waist, double duration_fwhm, double lambda0,
                  const pic_laser_opts* opts) {
  if (!h) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  if (!(waist > 0) || !(duration_fwhm > 0) || !(lambda0 > 0)) return fail(h, PIC_ERR_ARG, "bad laser parameters");
  h->las_a0 = a0;
  h->las_w0 = waist * h->k0;
  h->las_tau = duration_fwhm * h->omega0;
  h->las_k = h->lambda0 / lambda0;
  h->las_xf = (opts ? opts->x_focus : 0.0) * h->k0;
  h->las_tpk = (opts && opts->t_peak != 0.0 ? opts->t_peak : 2.0 * duration_fwhm) * h->omega0;
  int mode = opts ? opts->mode : PIC_LASER_AUTO;
  if (mode == PIC_LASER_AUTO)
    mode = (!h->has_window && !h->periodic_x) ? PIC_LASER_HARD_SOURCE : PIC_LASER_IN_BOX;
  if (mode == PIC_LASER_HARD_SOURCE && (h->has_window || h->periodic_x))
    return fail(h, PIC_ERR_ARG, "hard source needs open x and no window");
  if (mode != PIC_LASER_HARD_SOURCE && mode != PIC_LASER_IN_BOX) return fail(h, PIC_ERR_ARG, "bad laser mode");
  h->laser_mode = mode;
  int rc;
  const double t = (double)h->step * h->dt;
  h->curl_valid = false;
  if (mode == PIC_LASER_HARD_SOURCE)
    rc = h->precision == PIC_FP64 ? hard_source<double>(h, t) : hard_source<float>(h, t);
  else
    rc = h->precision == PIC_FP64 ? laser_in_box<double>(h) : laser_in_box<float>(h);
  if (rc) return rc;
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int pic_step(pic_t* h, int n) {
  if (!h || n < 0) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  int rc = grow_if_needed(h);
  if (rc) return rc;
  rc = h->precision == PIC_FP64 ? step_impl<double>(h, n) : step_impl<float>(h, n);
  if (rc) return rc;
  return check_device_error(h);
}

int pic_diag(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a) {
  if (!h || !out) return PIC_ERR_ARG;
  return h->precision == PIC_FP64 ? diag_impl<double>(h, kind, out, len, a) : diag_impl<float>(h, kind, out, len, a);
}

int pic_get_info(const pic_t* hc, pic_info* out) {
  if (!hc || !out) return PIC_ERR_ARG;
  pic_t* h = const_cast<pic_t*>(hc);
  int rc = check_device_error(h);
  if (rc && rc != PIC_ERR_CAPACITY) return rc;
  out->dt = h->dt;
  out->dx = h->dx;
  out->dy = h->dy;
  out->dz = h->dz;
  out->t = (double)h->step * h->dt;
  out->step = h->step;
  out->shifts = h->shifts;
  out->np = h->capacity > 0 ? h->np_host : 0;
  out->capacity = h->capacity;
  out->pushed = h->pushed_host;
  out->precision = h->precision;
  return PIC_OK;
}

int pic_get_field(pic_t* h, int comp, double* host_out) {
  if (!h || !host_out || comp < 0 || comp >= NCOMP) return PIC_ERR_ARG;
  const size_t es = esize(h), slab = (size_t)h->ny * h->nz;
  std::vector<char> buf(h->ncell * es);
  CK(h, cudaMemcpyAsync(buf.data(), (char*)h->fields + comp * h->ncell * es, h->ncell * es, cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->nx; ++i) {
    const size_t s = (size_t)((i + h->origin) % h->nx);
    for (size_t r = 0; r < slab; ++r)
      host_out[i * slab + r] = es == 8 ? ((const double*)buf.data())[s * slab + r]
                                       : (double)((const float*)buf.data())[s * slab + r];
  }
  return PIC_OK;
}

int pic_set_field(pic_t* h, int comp, const double* host_in) {
  if (!h || !host_in || comp < 0 || comp >= NCOMP) return PIC_ERR_ARG;
  const size_t es = esize(h), slab = (size_t)h->ny * h->nz;
  std::vector<char> buf(h->ncell * es);
  for (int i = 0; i < h->nx; ++i) {
    const size_t s = (size_t)((i + h->origin) % h->nx);
    for (size_t r = 0; r < slab; ++r) {
      if (es == 8)
        ((double*)buf.data())[s * slab + r] = host_in[i * slab + r];
      else
        ((float*)buf.data())[s * slab + r] = (float)host_in[i * slab + r];
    }
  }
  CK(h, cudaMemcpyAsync((char*)h->fields + comp * h->ncell * es, buf.data(), h->ncell * es, cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  if (comp <= EZ) h->curl_valid = false;
  return PIC_OK;
}

int pic_get_particles(pic_t* h, pic_particles* p) {
  if (!h || !p) return PIC_ERR_ARG;
  int rc = check_device_error(h);
  if (rc && rc != PIC_ERR_CAPACITY) return rc;
  const long long np = h->capacity > 0 ? h->np_host : 0;
  const long long room = p->n;
  p->n = np;
  if (room < np) return fail(h, PIC_ERR_CAPACITY, "host particle buffers too small");
  if (np == 0) return PIC_OK;
  const size_t es = esize(h);
  const PartBuf& b = h->pb[h->cur];
  std::vector<int> cell(np);
  std::vector<char> tmp(np * es);
  CK(h, cudaMemcpyAsync(cell.data(), b.cell, 4 * np, cudaMemcpyDeviceToHost, h->stream));
  auto fetch = [&](const void* src, double* dst) -> int {
    CK(h, cudaMemcpyAsync(tmp.data(), src, es * np, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < np; ++i)
      dst[i] = es == 8 ? ((const double*)tmp.data())[i] : (double)((const float*)tmp.data())[i];
    return PIC_OK;
  };
  for (int d = 0; d < 3; ++d) {
    if (p->xi[d] && fetch(b.o[d], p->xi[d])) return PIC_ERR_CUDA;
    if (p->u[d] && fetch(b.u[d], p->u[d])) return PIC_ERR_CUDA;
  }
  if (p->w && fetch(b.w, p->w)) return PIC_ERR_CUDA;
  if (p->id) {
    if (b.id)
      CK(h, cudaMemcpyAsync(p->id, b.id, 4 * np, cudaMemcpyDeviceToHost, h->stream));
    else
      for (long long i = 0; i < np; ++i) p->id[i] = 0xffffffffu;
  }
  CK(h, cudaStreamSynchronize(h->stream));
  const int nyz = h->ny * h->nz;
  for (long long i = 0; i < np; ++i) {
    const int c = cell[i];
    int cx = c / nyz;
    const int r = c - cx * nyz;
    const int cy = r / h->nz, cz = r - cy * h->nz;
    cx = (cx - h->origin + h->nx) % h->nx;
    if (p->xi[0]) p->xi[0][i] += cx;
    if (p->xi[1]) p->xi[1][i] += cy;
    if (p->xi[2]) p->xi[2][i] += cz;
  }
  return PIC_OK;
}

int pic_set_particles(pic_t* h, const pic_particles* p) {
  if (!h || !p || p->n < 0) return PIC_ERR_ARG;
  if (p->n > 0 && (!p->xi[0] || !p->xi[1] || !p->xi[2] || !p->u[0] || !p->u[1] || !p->u[2] || !p->w))
    return fail(h, PIC_ERR_ARG, "null particle array");
  const long long np = p->n;
  const int N[3] = {h->nx, h->ny, h->nz};
  for (long long i = 0; i < np; ++i)
    for (int d = 0; d < 3; ++d) {
      const double x = p->xi[d][i];
      if (d == 0 && !h->periodic_x) {
        const double c = std::floor(x);
        if (!(c >= x_lo(h) && c <= x_hi(h))) return fail(h, PIC_ERR_ARG, "particle outside the allowed x range");
      } else if (d > 0 && h->pml) {
        if (!(x >= h->pml && x < N[d] - h->pml)) return fail(h, PIC_ERR_ARG, "particle inside an absorbing layer");
      } else if (!(x >= 0.0 && x < N[d])) {
        return fail(h, PIC_ERR_ARG, "particle outside the box");
      }
    }
  if (!h->has_species) {
    if (h->q == 0.0) {
      h->q = -1.0;
      h->m = 1.0;
    }
  }
  long long cap = std::max<long long>(np, h->max_particles > 0 ? h->max_particles : 0);
  if (cap < 1) cap = 1;
  int rc = ensure_particles(h, cap);
  if (rc) return rc;
  const size_t es = esize(h);
  const PartBuf& b = h->pb[h->cur];
  std::vector<int> cell(np);
  std::vector<char> tmp(std::max<long long>(np, 1) * es);
  std::vector<double> off[3];
  for (int d = 0; d < 3; ++d) off[d].resize(np);
  for (long long i = 0; i < np; ++i) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      const double x = p->xi[d][i];
      const double fl = std::floor(x);
      c[d] = (int)fl;
      off[d][i] = x - fl;
    }
    const int sx = (c[0] + h->origin) % h->nx;
    cell[i] = (sx * h->ny + c[1]) * h->nz + c[2];
  }
  auto put = [&](void* dst, const double* src) -> int {
    for (long long i = 0; i < np; ++i) {
      if (es == 8)
        ((double*)tmp.data())[i] = src[i];
      else {
        float v = (float)src[i];
        ((float*)tmp.data())[i] = v;
      }
    }
    CK(h, cudaMemcpyAsync(dst, tmp.data(), es * np, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PIC_OK;
  };
  CK(h, cudaStreamSynchronize(h->stream));
  if (np > 0) {
    CK(h, cudaMemcpyAsync(b.cell, cell.data(), 4 * np, cudaMemcpyHostToDevice, h->stream));
    for (int d = 0; d < 3; ++d) {
      if (es == 4)
        for (long long i = 0; i < np; ++i)
          if ((float)off[d][i] >= 1.0f) off[d][i] = 0.99999994;
      if (put(b.o[d], off[d].data())) return PIC_ERR_CUDA;
      if (put(b.u[d], p->u[d])) return PIC_ERR_CUDA;
    }
    if (put(b.w, p->w)) return PIC_ERR_CUDA;
    if (b.id) {
      std::vector<uint32_t> ids(np);
      for (long long i = 0; i < np; ++i) ids[i] = p->id ? p->id[i] : (uint32_t)i;
      CK(h, cudaMemcpyAsync(b.id, ids.data(), 4 * np, cudaMemcpyHostToDevice, h->stream));
      CK(h, cudaStreamSynchronize(h->stream));
    }
  }
  int npi = (int)np;
  CK(h, cudaMemcpyAsync(h->d_ctrl + h->cur, &npi, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->np_host = npi;
  h->need_sort = true;
  return PIC_OK;
}

namespace {
struct CkptHeader {
  char magic[8];  // "PICCKPT1"
  int version, precision, nx, ny, nz, ppc, has_ids, pml;
  long long step, shifts, np, pushed;
  double win_frac;
};

// Memory variables of the absorbing layers in window-relative slab order, as
// doubles (to_host) or back into the storage slabs (from host).
int psi_io(pic_t* h, std::vector<double>& host, bool to_host) {
  const size_t n = psi_values(h);
  if (!n) return PIC_OK;
  const size_t es = esize(h);
  std::vector<unsigned char> raw(n * es);
  if (to_host) {
    CK(h, cudaMemcpyAsync(raw.data(), h->psi, raw.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    host.assign(n, 0.0);
  } else if (host.size() != n) {
    return fail(h, PIC_ERR_STATE, "absorbing-layer state of the wrong size");
  }
  const size_t rows = 2 * (size_t)h->pml + 1;
  const size_t per_slab[2] = {rows * h->nz, (size_t)h->ny * rows};  // y arrays, z arrays
  size_t off = 0;
  for (int c = 0; c < 8; ++c) {
    const size_t ps = per_slab[c / 4];
    for (int i = 0; i < h->nx; ++i) {
      const size_t st = off + (size_t)((i + h->origin) % h->nx) * ps, wr = off + (size_t)i * ps;
      for (size_t q = 0; q < ps; ++q) {
        double* hv = &host[wr + q];
        unsigned char* rv = &raw[(st + q) * es];
        if (to_host) {
          if (es == 8) std::memcpy(hv, rv, 8);
          else { float v; std::memcpy(&v, rv, 4); *hv = v; }
        } else {
          if (es == 8) std::memcpy(rv, hv, 8);
          else { const float v = (float)*hv; std::memcpy(rv, &v, 4); }
        }
      }
    }
    off += ps * h->nx;
  }
  if (!to_host) {
    CK(h, cudaMemcpyAsync(h->psi, raw.data(), raw.size(), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
  }
  return PIC_OK;
}
}  // namespace

int pic_save(pic_t* h, const char* path) {
  if (!h || !path) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  int rc = check_device_error(h);
  if (rc) return rc;
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "PICCKPT1", 8);
  hd.version = 1;
  hd.precision = h->precision;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.nz = h->nz;
  hd.ppc = h->ppc;
  hd.has_ids = h->pb[0].id != nullptr;
  hd.pml = h->pml;
  hd.step = h->step;
  hd.shifts = h->shifts;
  hd.np = h->capacity > 0 ? h->np_host : 0;
  hd.pushed = h->pushed_host;
  hd.win_frac = h->win_frac;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, PIC_ERR_ARG, "cannot open checkpoint file for writing");
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  std::vector<double> buf(h->ncell);
  for (int c = 0; c < NCOMP && ok; ++c) {
    rc = pic_get_field(h, c, buf.data());
    ok = rc == PIC_OK && std::fwrite(buf.data(), sizeof(double), h->ncell, f) == h->ncell;
  }
  if (ok && hd.np > 0) {
    std::vector<double> a(7 * (size_t)hd.np);
    std::vector<uint32_t> ids(hd.has_ids ? hd.np : 0);
    pic_particles pp;
    pp.n = hd.np;
    for (int d = 0; d < 3; ++d) {
      pp.xi[d] = a.data() + d * hd.np;
      pp.u[d] = a.data() + (3 + d) * hd.np;
    }
    pp.w = a.data() + 6 * hd.np;
    pp.id = hd.has_ids ? ids.data() : nullptr;
    rc = pic_get_particles(h, &pp);
    ok = rc == PIC_OK && std::fwrite(a.data(), sizeof(double), a.size(), f) == a.size();
    if (ok && hd.has_ids) ok = std::fwrite(ids.data(), sizeof(uint32_t), ids.size(), f) == ids.size();
  }
  if (ok && h->pml) {
    std::vector<double> ps;
    rc = psi_io(h, ps, true);
    ok = rc == PIC_OK && std::fwrite(ps.data(), sizeof(double), ps.size(), f) == ps.size();
  }
  if (std::fclose(f) != 0) ok = false;
  if (!ok) return rc ? rc : fail(h, PIC_ERR_ARG, "writing the checkpoint failed");
  return PIC_OK;
}

int pic_load(pic_t* h, const char* path) {
  if (!h || !path) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(h, PIC_ERR_ARG, "cannot open checkpoint file");
  CkptHeader hd;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "PICCKPT1", 8) != 0 || hd.version != 1) {
    std::fclose(f);
    return fail(h, PIC_ERR_STATE, "not a checkpoint of this library");
  }
  if (hd.precision != h->precision || hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz || hd.ppc != h->ppc ||
      hd.pml != h->pml) {
    std::fclose(f);
    return fail(h, PIC_ERR_ARG, "checkpoint grid, precision, ppc or absorbing layers differ from the handle");
  }
  std::vector<double> buf(h->ncell);
  int rc = PIC_OK;
  for (int c = 0; c < NCOMP && rc == PIC_OK; ++c) {
    if (std::fread(buf.data(), sizeof(double), h->ncell, f) != h->ncell) rc = fail(h, PIC_ERR_STATE, "truncated checkpoint");
    if (rc == PIC_OK) rc = pic_set_field(h, c, buf.data());
  }
  if (rc == PIC_OK) {
    std::vector<double> a(7 * (size_t)hd.np);
    std::vector<uint32_t> ids(hd.has_ids ? hd.np : 0);
    if (std::fread(a.data(), sizeof(double), a.size(), f) != a.size() ||
        (hd.has_ids && std::fread(ids.data(), sizeof(uint32_t), ids.size(), f) != ids.size()))
      rc = fail(h, PIC_ERR_STATE, "truncated checkpoint");
    if (rc == PIC_OK) {
      pic_particles pp;
      pp.n = hd.np;
      for (int d = 0; d < 3; ++d) {
        pp.xi[d] = a.data() + d * hd.np;
        pp.u[d] = a.data() + (3 + d) * hd.np;
      }
      pp.w = a.data() + 6 * hd.np;
      pp.id = hd.has_ids ? ids.data() : nullptr;
      rc = pic_set_particles(h, &pp);
    }
  }
  if (rc == PIC_OK && h->pml) {
    std::vector<double> ps(psi_values(h));
    if (std::fread(ps.data(), sizeof(double), ps.size(), f) != ps.size())
      rc = fail(h, PIC_ERR_STATE, "truncated checkpoint");
    else
      rc = psi_io(h, ps, false);
  }
  std::fclose(f);
  if (rc) return rc;
  h->step = hd.step;
  h->shifts = hd.shifts;
  h->win_frac = hd.win_frac;
  h->curl_valid = false;
  unsigned long long pushed = (unsigned long long)hd.pushed;
  CK(h, cudaMemcpyAsync(h->d_pushed, &pushed, sizeof(pushed), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  h->pushed_host = hd.pushed;
  return PIC_OK;
}

int pic_timing_start(pic_t* h, int enable) {
  if (!h) return PIC_ERR_ARG;
  CK(h, cudaStreamSynchronize(h->stream));
  for (int g = 0; g < 4; ++g) {
    for (auto& pr : h->ev_pairs[g]) {
      h->ev_pool.push_back(pr.first);
      h->ev_pool.push_back(pr.second);
    }
    h->ev_pairs[g].clear();
    h->launches[g] = 0;
  }
  h->kernels = 0;
  h->profiling = enable != 0;
  return PIC_OK;
}

int pic_timing_read(pic_t* h, pic_timing* out) {
  if (!h || !out) return PIC_ERR_ARG;
  CK(h, cudaStreamSynchronize(h->stream));
  for (int g = 0; g < 4; ++g) {
    double ms = 0.0;
    for (auto& pr : h->ev_pairs[g]) {
      float t = 0.f;
      CK(h, cudaEventElapsedTime(&t, pr.first, pr.second));
      ms += t;
    }
    out->ms[g] = ms;
    out->launches[g] = h->launches[g];
  }
  out->kernels = h->kernels;
  return PIC_OK;
}

int pic_destroy(pic_t* h) {
  if (!h) return PIC_ERR_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int g = 0; g < 4; ++g)
    for (auto& pr : h->ev_pairs[g]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  std::vector<void*> own = h->owned;
  for (void* p : own) dfree(h, p);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return PIC_OK;
}

}  // extern "C"

// ===========================================================================
// Tile shapes and the autotuner
// ===========================================================================
namespace {

int set_tiles(pic_t* h, int tx, int ty, int tz) {
  const int n3[3] = {h->nx, h->ny, h->nz};
  int t3[3] = {tx, ty, tz};
  for (int d = 0; d < 3; ++d) t3[d] = std::max(1, std::min(t3[d], n3[d]));
  Tiles tl;
  tl.tx = t3[0];
  tl.ty = t3[1];
  tl.tz = t3[2];
  tl.ntx = (h->nx + tl.tx - 1) / tl.tx;
  tl.nty = (h->ny + tl.ty - 1) / tl.ty;
  tl.ntz = (h->nz + tl.tz - 1) / tl.tz;
  tl.n = tl.ntx * tl.nty * tl.ntz;
  const size_t sm = h->precision == PIC_FP64 ? tiled_smem_bytes<double>(tl) : tiled_smem_bytes<float>(tl);
  if (sm > 227 * 1024) return fail(h, PIC_ERR_ARG, "tile too large for shared memory");
  CK(h, cudaStreamSynchronize(h->stream));
  if (tl.n > h->tiles_alloc) {
    int* a0 = (int*)dalloc(h, sizeof(int) * (tl.n + 1));
    int* a1 = (int*)dalloc(h, sizeof(int) * (tl.n + 1));
    int* c = (int*)dalloc(h, sizeof(int) * tl.n);
    int* f = (int*)dalloc(h, sizeof(int) * tl.n);
    if (!a0 || !a1 || !c || !f) return fail(h, PIC_ERR_OOM, "tile arrays");
    dfree(h, h->tstart[0]);
    dfree(h, h->tstart[1]);
    dfree(h, h->tcnt);
    dfree(h, h->tfill);
    h->tstart[0] = a0;
    h->tstart[1] = a1;
    h->tcnt = c;
    h->tfill = f;
    h->tiles_alloc = tl.n;
  }
  h->tiles = tl;
  h->need_sort = true;
  return PIC_OK;
}

// Device copy of the state that a trial step changes.
struct Snapshot {
  void* fields = nullptr;
  void* curl = nullptr;
  void* psi = nullptr;  // absorbing-layer memory variables (none without layers)
  void* part = nullptr;
  int ctrl[6];
  int cur = 0;
  int64_t step = 0, shifts = 0;
  int origin = 0;
  double win_frac = 0;
  bool curl_valid = false, need_sort = false;
  int np = 0;
};

int snapshot_take(pic_t* h, Snapshot* sn) {
  const size_t es = esize(h);
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(sn->ctrl, h->d_ctrl, sizeof(sn->ctrl), cudaMemcpyDeviceToHost));
  sn->np = sn->ctrl[h->cur];
  sn->fields = dalloc(h, NCOMP * h->ncell * es);
  sn->curl = dalloc(h, 3 * h->ncell * es);
  const size_t per = 4 + 7 * es + (h->pb[0].id ? 4 : 0);
  sn->part = dalloc(h, per * (size_t)std::max(sn->np, 1));
  if (!sn->fields || !sn->curl || !sn->part) return fail(h, PIC_ERR_OOM, "autotune snapshot");
  CK(h, cudaMemcpyAsync(sn->fields, h->fields, NCOMP * h->ncell * es, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(sn->curl, h->curl, 3 * h->ncell * es, cudaMemcpyDeviceToDevice, h->stream));
  if (h->psi) {
    sn->psi = dalloc(h, psi_values(h) * es);
    if (!sn->psi) return fail(h, PIC_ERR_OOM, "autotune snapshot");
    CK(h, cudaMemcpyAsync(sn->psi, h->psi, psi_values(h) * es, cudaMemcpyDeviceToDevice, h->stream));
  }
  const PartBuf& b = h->pb[h->cur];
  char* dst = (char*)sn->part;
  const size_t n = sn->np;
  CK(h, cudaMemcpyAsync(dst, b.cell, 4 * n, cudaMemcpyDeviceToDevice, h->stream));
  dst += 4 * n;
  for (int d = 0; d < 3; ++d, dst += es * n) CK(h, cudaMemcpyAsync(dst, b.o[d], es * n, cudaMemcpyDeviceToDevice, h->stream));
  for (int d = 0; d < 3; ++d, dst += es * n) CK(h, cudaMemcpyAsync(dst, b.u[d], es * n, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dst, b.w, es * n, cudaMemcpyDeviceToDevice, h->stream));
  dst += es * n;
  if (b.id) CK(h, cudaMemcpyAsync(dst, b.id, 4 * n, cudaMemcpyDeviceToDevice, h->stream));
  sn->cur = h->cur;
  sn->step = h->step;
  sn->shifts = h->shifts;
  sn->origin = h->origin;
  sn->win_frac = h->win_frac;
  sn->curl_valid = h->curl_valid;
  sn->need_sort = h->need_sort;
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

// Restore into buffer 0 (unsorted order is kept; a re-sort follows).
int snapshot_restore(pic_t* h, Snapshot* sn) {
  const size_t es = esize(h);
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpyAsync(h->fields, sn->fields, NCOMP * h->ncell * es, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->curl, sn->curl, 3 * h->ncell * es, cudaMemcpyDeviceToDevice, h->stream));
  if (sn->psi) CK(h, cudaMemcpyAsync(h->psi, sn->psi, psi_values(h) * es, cudaMemcpyDeviceToDevice, h->stream));
  const PartBuf& b = h->pb[0];
  const char* src = (const char*)sn->part;
  const size_t n = sn->np;
  CK(h, cudaMemcpyAsync(b.cell, src, 4 * n, cudaMemcpyDeviceToDevice, h->stream));
  src += 4 * n;
  for (int d = 0; d < 3; ++d, src += es * n) CK(h, cudaMemcpyAsync(b.o[d], src, es * n, cudaMemcpyDeviceToDevice, h->stream));
  for (int d = 0; d < 3; ++d, src += es * n) CK(h, cudaMemcpyAsync(b.u[d], src, es * n, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(b.w, src, es * n, cudaMemcpyDeviceToDevice, h->stream));
  src += es * n;
  if (b.id) CK(h, cudaMemcpyAsync(b.id, src, 4 * n, cudaMemcpyDeviceToDevice, h->stream));
  int ctrl[6];
  std::memcpy(ctrl, sn->ctrl, sizeof(ctrl));
  ctrl[0] = sn->np;
  ctrl[1] = 0;
  CK(h, cudaMemcpyAsync(h->d_ctrl, ctrl, sizeof(ctrl), cudaMemcpyHostToDevice, h->stream));
  h->cur = 0;
  h->step = sn->step;
  h->shifts = sn->shifts;
  h->origin = sn->origin;
  h->win_frac = sn->win_frac;
  h->curl_valid = sn->curl_valid;
  h->need_sort = true;
  CK(h, cudaStreamSynchronize(h->stream));
  dfree(h, sn->fields);
  dfree(h, sn->curl);
  dfree(h, sn->psi);
  dfree(h, sn->part);
  return PIC_OK;
}

std::string tune_key(const pic_t* h) {
  char buf[128];
  std::snprintf(buf, sizeof(buf), "%s:ppc%d:%dx%dx%d%s", h->precision == PIC_FP64 ? "fp64" : "fp32", h->ppc, h->nx,
                h->ny, h->nz, h->pml ? ":pml" : "");
  return buf;
}

// Tiny JSON cache {"key": [tx, ty, tz], ...}.
bool cache_lookup(const char* path, const std::string& key, int t3[3]) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
  std::fclose(f);
  const std::string pat = "\"" + key + "\"";
  size_t p = txt.find(pat);
  if (p == std::string::npos) return false;
  p = txt.find('[', p);
  if (p == std::string::npos) return false;
  return std::sscanf(txt.c_str() + p, "[%d, %d, %d]", &t3[0], &t3[1], &t3[2]) == 3;
}

void cache_store(const char* path, const std::string& key, const int t3[3]) {
  if (!path) return;
  std::string txt;
  if (FILE* f = std::fopen(path, "r")) {
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
    std::fclose(f);
  }
  std::vector<std::string> entries;
  // keep the other entries (one per line between the braces)
  size_t a = 0;
  while ((a = txt.find('"', a)) != std::string::npos) {
    size_t b = txt.find(']', a);
    if (b == std::string::npos) break;
    std::string e = txt.substr(a, b - a + 1);
    if (e.find("\"" + key + "\"") != 0) entries.push_back(e);
    a = b + 1;
  }
  char buf[160];
  std::snprintf(buf, sizeof(buf), "\"%s\": [%d, %d, %d]", key.c_str(), t3[0], t3[1], t3[2]);
  entries.push_back(buf);
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  std::fputs("{\n", f);
  for (size_t i = 0; i < entries.size(); ++i) std::fprintf(f, "  %s%s\n", entries[i].c_str(), i + 1 < entries.size() ? "," : "");
  std::fputs("}\n", f);
  std::fclose(f);
}

template <typename T>
int autotune_impl(pic_t* h, int steps, const char* cache_path, int out3[3], double* best_ms) {
  const std::string key = tune_key(h);
  int t3[3];
  if (cache_lookup(cache_path, key, t3)) {
    int rc = set_tiles(h, t3[0], t3[1], t3[2]);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d) out3[d] = t3[d];
    *best_ms = -1.0;
    return PIC_OK;
  }
  static const int cand[][3] = {{8, 8, 8}, {16, 8, 8}, {8, 8, 16}, {4, 8, 16}, {8, 4, 4}, {16, 4, 4},
                                {32, 4, 4}, {4, 8, 8}, {8, 8, 4}, {16, 8, 4}, {4, 4, 4}, {12, 6, 6}};
  const Tiles orig = h->tiles;
  double best = 1e300;
  int bi = -1;
  const bool prof = h->profiling;
  for (int c = 0; c < (int)(sizeof(cand) / sizeof(cand[0])); ++c) {
    Tiles trial = h->tiles;
    (void)trial;
    if (set_tiles(h, cand[c][0], cand[c][1], cand[c][2]) != PIC_OK) continue;
    Snapshot sn;
    int rc = snapshot_take(h, &sn);
    if (rc) return rc;
    rc = resort_all<T>(h);
    if (rc) return rc;
    h->need_sort = false;
    rc = step_impl<T>(h, 1);  // warm-up
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    CK(h, cudaEventRecord(e0, h->stream));
    rc = step_impl<T>(h, steps);
    if (rc) return rc;
    CK(h, cudaEventRecord(e1, h->stream));
    CK(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rc = snapshot_restore(h, &sn);
    if (rc) return rc;
    const double per = ms / std::max(steps, 1);
    if (per < best) {
      best = per;
      bi = c;
    }
  }
  h->profiling = prof;
  int rc;
  if (bi < 0)
    rc = set_tiles(h, orig.tx, orig.ty, orig.tz);
  else
    rc = set_tiles(h, cand[bi][0], cand[bi][1], cand[bi][2]);
  if (rc) return rc;
  out3[0] = h->tiles.tx;
  out3[1] = h->tiles.ty;
  out3[2] = h->tiles.tz;
  *best_ms = best;
  cache_store(cache_path, key, out3);
  return check_device_error(h);
}

}  // namespace

extern "C" int pic_autotune(pic_t* h, int steps, const char* cache_path, int* tile_out, double* ms_out) {
  if (!h || steps < 1) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  if (!cache_path) cache_path = std::getenv("PIC_AUTOTUNE_CACHE");
  int t3[3];
  double ms = 0.0;
  int rc = h->precision == PIC_FP64 ? autotune_impl<double>(h, steps, cache_path, t3, &ms)
                                    : autotune_impl<float>(h, steps, cache_path, t3, &ms);
  if (rc) return rc;
  if (tile_out)
    for (int d = 0; d < 3; ++d) tile_out[d] = t3[d];
  if (ms_out) *ms_out = ms;
  return PIC_OK;
}

extern "C" int pic_set_tiles(pic_t* h, int tx, int ty, int tz) {
  if (!h || tx < 1 || ty < 1 || tz < 1) return PIC_ERR_ARG;
  if (h->batched) return fail(h, PIC_ERR_STATE, "handle is part of a batch");
  return set_tiles(h, tx, ty, tz);
}

// ===========================================================================
// Batched instances: one CUDA graph launch per step for all members.
// ===========================================================================
struct pic_batch_t {
  std::vector<pic_t*> sims;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<int> cur0;
  int parity = 0;
  bool stale = true;
  long long kernels_per_step = 0;
  long long graph_launches = 0, kernel_launches = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  double last_ms = 0.0;
  std::string err;
};

namespace {

int bfail(pic_batch_t* b, int code, const std::string& m) {
  b->err = m;
  return code;
}

// One step of member h on stream s, every step parameter read from the
// device-side state (so the same captured launches replay every step).
int enqueue_step_dyn(pic_t* h, cudaStream_t s, int cur, long long* kernels) {
  using T = float;
  const size_t n = h->ncell;
  const Tiles tl = h->tiles;
  const int nb = 1 - cur;
  Geom<T> g = geom<T>(h);
  g.dyn = h->d_dyn;
  Geom<T> gs = g;
  gs.gate = 1;
  Fields<T> f = fields<T>(h);
  const FieldCoef<T> fc = field_coef<T>(h);
  const Smooth<T> S = smooth<T>(h);
  CK(h, cudaMemsetAsync(f.c[JX], 0, 3 * n * sizeof(T), s));
  CK(h, cudaMemsetAsync(h->tcnt, 0, sizeof(int) * tl.n, s));
  k_step_begin<<<1, 32, 0, s>>>(h->d_dyn);
  const T hq = (T)(h->q * h->dt / (2.0 * h->m));
  k_push_tiled<T><<<tl.n, push_threads<T>(), tiled_smem_bytes<T>(tl), s>>>(g, tl, f, parts<T>(h, cur), h->tstart[cur],
                                                            (int)h->capacity, h->keys, h->tcnt, hq, (T)h->q, 0,
                                                            x_lo(h), x_hi(h), h->d_pushed, h->d_ctrl + 2);
  k_e_update<T><<<e_update_grid(h), e_update_block(h), 0, s>>>(g, f, curl_view<T>(h), fc, pml_view<T>(h));
  launch_curl<T>(h, g, 1, 0, h->nx, s);
  k_window_commit<<<1, 32, 0, s>>>(h->d_dyn);
  k_zero_front_slab<T><<<grid_for((long long)NCOMP * h->ny * h->nz), 256, 0, s>>>(gs, f, pml_view<T>(h));
  launch_curl<T>(h, gs, 0, 0, 1, s);
  launch_curl<T>(h, gs, 0, h->nx - 1, 1, s);
  (void)S;
  LoadSpec L;
  const bool inject = h->has_species;
  const long long nslot = (long long)h->ny * h->nz * std::max(h->ppc, 1);
  if (inject) {
    L = load_spec(h, x_hi(h), x_hi(h));
    k_inject_tiled<T><<<grid_for(nslot, 256, 152 * 16), 256, 0, s>>>(gs, tl, parts<T>(h, nb), L, 0, h->tcnt,
                                                                     h->tstart[nb], h->tfill, h->d_ctrl + 2);
  }
  k_scan_tiles<<<1, 1024, 0, s>>>(h->tcnt, h->tstart[nb], tl.n, h->d_ctrl + nb, (int)h->capacity, h->d_ctrl + 2);
  CK(h, cudaMemsetAsync(h->tfill, 0, sizeof(int) * tl.n, s));
  k_scatter<T><<<grid_for(h->capacity, 256, 152 * 16), 256, 0, s>>>(parts<T>(h, cur), h->keys, h->d_ctrl + cur,
                                                                     parts<T>(h, nb), h->tstart[nb], h->tfill,
                                                                     h->d_ctrl + 2);
  if (inject)
    k_inject_tiled<T><<<grid_for(nslot, 256, 152 * 16), 256, 0, s>>>(gs, tl, parts<T>(h, nb), L, 1, h->tcnt,
                                                                     h->tstart[nb], h->tfill, h->d_ctrl + 2);
  *kernels += 11 + (inject ? 2 : 0);
  CK(h, cudaGetLastError());
  return PIC_OK;
}

int dyn_to_device(pic_t* h) {
  DynState d;
  d.frac = h->win_frac;
  d.frac_new = h->win_frac;
  d.v = h->win_v;
  d.dt = h->dt;
  d.dx = h->dx;
  d.t0 = h->win_t0;
  d.step = h->step;
  d.shifts = h->shifts;
  d.origin = h->origin;
  d.origin_after = h->origin;
  d.shift = 0;
  d.has_window = h->has_window ? 1 : 0;
  d.nx = h->nx;
  CK(h, cudaMemcpyAsync(h->d_dyn, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

int dyn_to_host(pic_t* h) {
  DynState d;
  CK(h, cudaMemcpy(&d, h->d_dyn, sizeof(d), cudaMemcpyDeviceToHost));
  h->win_frac = d.frac;
  h->step = d.step;
  h->shifts = d.shifts;
  h->origin = d.origin;
  return PIC_OK;
}

void drop_graphs(pic_batch_t* b) {
  for (int p = 0; p < 2; ++p)
    if (b->exec[p]) {
      cudaGraphExecDestroy(b->exec[p]);
      b->exec[p] = nullptr;
    }
  b->stale = true;
}

// Bring every member to a capturable state and capture the two step graphs
// (members alternate their particle buffers, so even and odd steps differ).
int prepare_and_capture(pic_batch_t* b) {
  drop_graphs(b);
  b->cur0.assign(b->sims.size(), 0);
  for (size_t i = 0; i < b->sims.size(); ++i) {
    pic_t* h = b->sims[i];
    if (h->need_sort) {
      int rc = resort_all<float>(h);
      if (rc) return bfail(b, rc, h->err);
      h->need_sort = false;
    }
    if (!h->curl_valid) {
      int rc = curl_only<float>(h, 0, h->nx);
      if (rc) return bfail(b, rc, h->err);
      h->curl_valid = true;
    }
    int rc = dyn_to_device(h);
    if (rc) return bfail(b, rc, h->err);
    b->cur0[i] = h->cur;
  }
  for (int p = 0; p < 2; ++p) {
    long long kernels = 0;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return bfail(b, PIC_ERR_CUDA, "cudaStreamBeginCapture failed");
    cudaEventRecord(b->fork, b->stream);
    int rc = PIC_OK;
    for (size_t i = 0; i < b->sims.size() && rc == PIC_OK; ++i) {
      cudaStreamWaitEvent(b->side[i], b->fork, 0);
      rc = enqueue_step_dyn(b->sims[i], b->side[i], b->cur0[i] ^ p, &kernels);
      cudaEventRecord(b->join[i], b->side[i]);
      cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(b, rc, "capture of a member step failed");
    }
    if (e != cudaSuccess || !graph) return bfail(b, PIC_ERR_CUDA, "cudaStreamEndCapture failed");
    e = cudaGraphInstantiate(&b->exec[p], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, PIC_ERR_CUDA, "cudaGraphInstantiate failed");
    b->kernels_per_step = kernels;
  }
  b->parity = 0;
  b->stale = false;
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_create(int n, pic_t* const* sims, pic_batch_t** out) {
  if (n < 1 || !sims || !out) return PIC_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!sims[i]) return PIC_ERR_ARG;
    if (sims[i]->precision != PIC_FP32 || sims[i]->batched) return PIC_ERR_STATE;
    if (sims[i]->laser_mode == PIC_LASER_HARD_SOURCE) return PIC_ERR_STATE;  // time-driven source: host path only
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return PIC_ERR_ARG;
  }
  pic_batch_t* b = new (std::nothrow) pic_batch_t();
  if (!b) return PIC_ERR_OOM;
  b->sims.assign(sims, sims + n);
  bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreate(&b->t0) == cudaSuccess && cudaEventCreate(&b->t1) == cudaSuccess;
  b->side.assign(n, nullptr);
  b->join.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i)
    ok = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i) {
    pic_t* h = sims[i];
    if (!h->d_dyn) h->d_dyn = (DynState*)dalloc(h, sizeof(DynState));
    ok = h->d_dyn != nullptr && cudaStreamSynchronize(h->stream) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    pic_batch_destroy(b);
    return PIC_ERR_CUDA;
  }
  for (pic_t* s : b->sims) s->batched = true;
  *out = b;
  return PIC_OK;
}

int pic_batch_step(pic_batch_t* b, int n) {
  if (!b || n < 0) return PIC_ERR_ARG;
  if (n == 0) return PIC_OK;
  for (pic_t* s : b->sims) {
    int rc = grow_if_needed(s);
    if (rc) return bfail(b, rc, s->err);
    if (s->need_sort) b->stale = true;
  }
  if (b->stale) {
    int rc = prepare_and_capture(b);
    if (rc) return rc;
  }
  cudaEventRecord(b->t0, b->stream);
  for (int it = 0; it < n; ++it) {
    if (cudaGraphLaunch(b->exec[b->parity], b->stream) != cudaSuccess)
      return bfail(b, PIC_ERR_CUDA, "cudaGraphLaunch failed");
    b->parity ^= 1;
    b->graph_launches += 1;
    b->kernel_launches += b->kernels_per_step;
  }
  cudaEventRecord(b->t1, b->stream);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, PIC_ERR_CUDA, "batch step failed");
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, b->t0, b->t1) == cudaSuccess) b->last_ms = ms;
  for (size_t i = 0; i < b->sims.size(); ++i) {
    pic_t* h = b->sims[i];
    h->cur = b->cur0[i] ^ b->parity;
    int rc = dyn_to_host(h);
    if (!rc) rc = check_device_error(h);
    if (rc) return bfail(b, rc, h->err);
  }
  return PIC_OK;
}

int pic_batch_info(const pic_batch_t* b, int64_t* graph_launches, int64_t* kernel_launches,
                   double* last_step_ms) {
  if (!b) return PIC_ERR_ARG;
  if (graph_launches) *graph_launches = b->graph_launches;
  if (kernel_launches) *kernel_launches = b->kernel_launches;
  if (last_step_ms) *last_step_ms = b->last_ms;
  return PIC_OK;
}

int pic_batch_diag(pic_batch_t* b, int instance, int kind, double* out, size_t len, const pic_diag_args* a) {
  if (!b || instance < 0 || instance >= (int)b->sims.size()) return PIC_ERR_ARG;
  return pic_diag(b->sims[instance], kind, out, len, a);
}

int pic_batch_destroy(pic_batch_t* b) {
  if (!b) return PIC_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (pic_t* s : b->sims) s->batched = false;
  for (cudaStream_t s : b->side)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return PIC_OK;
}

}  // extern "C"
