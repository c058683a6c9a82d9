// pic_kernels.cuh -- CUDA kernels of one perfect-dispersion PIC step
// (Cowan, Kalmykov et al., J. Plasma Phys. 2012), templated on the
// arithmetic type (double or float).
#pragma once

#include "pic_device.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// Field access helpers.  `s` is a storage slab, or -1 outside an open window.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ld(const T* __restrict__ a, const Geom<T>& g, int s, int j, int k) {
  if (s < 0) return T(0);
  if (g.pml) {
    if (j < 0 || j >= g.ny || k < 0 || k >= g.nz) return T(0);
  } else {
    j = (j < 0) ? j + g.ny : (j >= g.ny ? j - g.ny : j);
    k = (k < 0) ? k + g.nz : (k >= g.nz ? k - g.nz : k);
  }
  return a[(size_t)s * g.nyz + (size_t)j * g.nz + k];
}

// storage slab of window-relative slab i (may be out of range for open x)
template <typename T>
__device__ __forceinline__ int slab_of(const Geom<T>& g, int i) {
  if (g.periodic_x) return wrapi(i + g.origin, g.nx);
  if (i < 0 || i >= g.nx) return -1;
  int s = i + g.origin;
  return s >= g.nx ? s - g.nx : s;
}

// S_x: smoothing transverse to x (in y and z) at one slab.
template <typename T>
__device__ __forceinline__ T smooth_x(const T* a, const Geom<T>& g, const Smooth<T>& S, int s, int j, int k) {
  if (s < 0) return T(0);
  const T c = ld(a, g, s, j, k);
  const T ey = ld(a, g, s, j + 1, k) + ld(a, g, s, j - 1, k);
  const T ez = ld(a, g, s, j, k + 1) + ld(a, g, s, j, k - 1);
  const T cr = ld(a, g, s, j + 1, k + 1) + ld(a, g, s, j + 1, k - 1) + ld(a, g, s, j - 1, k + 1) +
               ld(a, g, s, j - 1, k - 1);
  return S.a[0] * c + S.b1[0] * ey + S.b2[0] * ez + S.g[0] * cr;
}

// S_y: smoothing transverse to y (in x and z); sm, s, sp = slabs i-1, i, i+1.
template <typename T>
__device__ __forceinline__ T smooth_y(const T* a, const Geom<T>& g, const Smooth<T>& S, int sm, int s, int sp,
                                      int j, int k) {
  const T c = ld(a, g, s, j, k);
  const T ex = ld(a, g, sp, j, k) + ld(a, g, sm, j, k);
  const T ez = ld(a, g, s, j, k + 1) + ld(a, g, s, j, k - 1);
  const T cr = ld(a, g, sp, j, k + 1) + ld(a, g, sp, j, k - 1) + ld(a, g, sm, j, k + 1) + ld(a, g, sm, j, k - 1);
  return S.a[1] * c + S.b1[1] * ex + S.b2[1] * ez + S.g[1] * cr;
}

// S_z: smoothing transverse to z (in x and y).
template <typename T>
__device__ __forceinline__ T smooth_z(const T* a, const Geom<T>& g, const Smooth<T>& S, int sm, int s, int sp,
                                      int j, int k) {
  const T c = ld(a, g, s, j, k);
  const T ex = ld(a, g, sp, j, k) + ld(a, g, sm, j, k);
  const T ey = ld(a, g, s, j + 1, k) + ld(a, g, s, j - 1, k);
  const T cr = ld(a, g, sp, j + 1, k) + ld(a, g, sp, j - 1, k) + ld(a, g, sm, j + 1, k) + ld(a, g, sm, j - 1, k);
  return S.a[2] * c + S.b1[2] * ex + S.b2[2] * ey + S.g[2] * cr;
}

// ---------------------------------------------------------------------------
// Eq. (perfDispMaxwell), magnetic half step: B += coef * curl'(E), with the
// smoothed curl of Sec. 2 (D_i replaced by D_i S_i).  One thread per cell,
// k fastest so that a warp reads consecutive addresses.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_curl_e(Geom<T> g, Smooth<T> S, const T* __restrict__ Ex,
                                               const T* __restrict__ Ey, const T* __restrict__ Ez, T* Bx, T* By,
                                               T* Bz, T coef) {
  const int nyz = g.nyz;
  const long long ncell = (long long)g.nx * nyz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / nyz);
    const int r = (int)(q - (long long)i * nyz);
    const int j = r / g.nz, k = r - j * g.nz;
    const int s = slab_of(g, i), sm = slab_of(g, i - 1), sp = slab_of(g, i + 1);
    // Bx(i, j+1/2, k+1/2): D_y S_y Ez - D_z S_z Ey
    const T cx = (smooth_y(Ez, g, S, sm, s, sp, j + 1, k) - smooth_y(Ez, g, S, sm, s, sp, j, k)) / g.dy -
                 (smooth_z(Ey, g, S, sm, s, sp, j, k + 1) - smooth_z(Ey, g, S, sm, s, sp, j, k)) / g.dz;
    // By(i+1/2, j, k+1/2): D_z S_z Ex - D_x S_x Ez
    const T cy = (smooth_z(Ex, g, S, sm, s, sp, j, k + 1) - smooth_z(Ex, g, S, sm, s, sp, j, k)) / g.dz -
                 (smooth_x(Ez, g, S, sp, j, k) - smooth_x(Ez, g, S, s, j, k)) / g.dx;
    // Bz(i+1/2, j+1/2, k): D_x S_x Ey - D_y S_y Ex
    const T cz = (smooth_x(Ey, g, S, sp, j, k) - smooth_x(Ey, g, S, s, j, k)) / g.dx -
                 (smooth_y(Ex, g, S, sm, s, sp, j + 1, k) - smooth_y(Ex, g, S, sm, s, sp, j, k)) / g.dy;
    const size_t id = (size_t)s * nyz + r;
    Bx[id] += coef * cx;
    By[id] += coef * cy;
    Bz[id] += coef * cz;
  }
}

// ---------------------------------------------------------------------------
// Field update with a cached smoothed curl.  The two magnetic half steps of
// consecutive steps use the same curl'(E^{n+1}), so it is computed once per
// step and kept in C:
//   k_e_update:     B^{n+1/2} = B^n - (dt/2) C^n (formed on the fly),
//                   E^{n+1} = E^n + dt (curl B^{n+1/2} - J)
//   k_curl_tiled:   C^{n+1} = curl'(E^{n+1}),
//                   B^{n+1} = (B^n - (dt/2) C^n) - (dt/2) C^{n+1}
// Reciprocal spacings are precomputed (no divisions in the loops).
// ---------------------------------------------------------------------------
template <typename T>
struct FieldCoef {
  T dt, hdt;             // dt, dt/2
  T idx, idy, idz;       // 1/dx, 1/dy, 1/dz
};

template <typename T>
__device__ __forceinline__ T bhalf(const T* __restrict__ B, const T* __restrict__ C, const Geom<T>& g, int s,
                                   int j, int k, T hdt) {
  if (s < 0) return T(0);
  if (g.pml && (j < 0 || k < 0)) return T(0);
  j = (j < 0) ? j + g.ny : j;
  k = (k < 0) ? k + g.nz : k;
  const size_t id = (size_t)s * g.nyz + (size_t)j * g.nz + k;
  return B[id] - hdt * C[id];
}

// Launch: grid (ceil(nz / blockDim.x), ny, nx), one thread per cell; k from
// the thread, j and the window-relative slab i from the block (no division).
template <typename T>
__global__ void __launch_bounds__(256) k_e_update(Geom<T> g, Fields<T> f, Fields<T> cc, FieldCoef<T> fc, Pml<T> pm) {
  if (!dyn_prologue(g)) return;
  const int nyz = g.nyz;
  const T *Bx = f.c[BX], *By = f.c[BY], *Bz = f.c[BZ];
  const T *Cx = cc.c[0], *Cy = cc.c[1], *Cz = cc.c[2];
  {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
    if (k >= g.nz) return;
    const int r = j * g.nz + k;
    const int s = slab_of(g, i), sm = slab_of(g, i - 1);
    const size_t id = (size_t)s * nyz + r;
    const T bx = Bx[id] - fc.hdt * Cx[id];
    const T by = By[id] - fc.hdt * Cy[id];
    const T bz = Bz[id] - fc.hdt * Cz[id];
    T dyBz = (bz - bhalf(Bz, Cz, g, s, j - 1, k, fc.hdt)) * fc.idy;
    T dzBy = (by - bhalf(By, Cy, g, s, j, k - 1, fc.hdt)) * fc.idz;
    T dzBx = (bx - bhalf(Bx, Cx, g, s, j, k - 1, fc.hdt)) * fc.idz;
    const T dxBz = (bz - bhalf(Bz, Cz, g, sm, j, k, fc.hdt)) * fc.idx;
    const T dxBy = (by - bhalf(By, Cy, g, sm, j, k, fc.hdt)) * fc.idx;
    T dyBx = (bx - bhalf(Bx, Cx, g, s, j - 1, k, fc.hdt)) * fc.idy;
    if (pm.L) {  // Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2): y and z at nodes
      const int jr = pml_row(j, g.ny, pm.L);
      if (jr >= 0) {
        const T a = pm.cy[j], b = pm.cy[g.ny + j];
        const size_t pi = ((size_t)s * pm.rows + jr) * g.nz + k;
        const T p0 = b * pm.py[0][pi] + a * dyBz, p1 = b * pm.py[1][pi] + a * dyBx;
        pm.py[0][pi] = p0;
        pm.py[1][pi] = p1;
        dyBz += p0;
        dyBx += p1;
      }
      const int kr = pml_row(k, g.nz, pm.L);
      if (kr >= 0) {
        const T a = pm.cz[k], b = pm.cz[g.nz + k];
        const size_t pi = ((size_t)s * g.ny + j) * pm.rows + kr;
        const T p0 = b * pm.pz[0][pi] + a * dzBy, p1 = b * pm.pz[1][pi] + a * dzBx;
        pm.pz[0][pi] = p0;
        pm.pz[1][pi] = p1;
        dzBy += p0;
        dzBx += p1;
      }
    }
    f.c[EX][id] += fc.dt * ((dyBz - dzBy) - f.c[JX][id]);
    f.c[EY][id] += fc.dt * ((dzBx - dxBz) - f.c[JY][id]);
    f.c[EZ][id] += fc.dt * ((dxBy - dyBx) - f.c[JZ][id]);
  }
}

// ---------------------------------------------------------------------------
// Smoothed curl, shared-memory tiled.  A CTA covers a block of CB_X x CB_Y x
// CB_Z cells (window-relative slabs i0 + blockIdx.x * CB_X ...).  It stages E
// over the block plus one cell on every side, evaluates each of the six
// smoothed fields (S_x Ey, S_x Ez over x = i .. i+CB_X; S_y Ez, S_y Ex over
// y = j .. j+CB_Y; S_z Ex, S_z Ey over z = k .. k+CB_Z) once per point, and
// forms curl'(E) from their differences.
// mode 0: C = curl'(E) only (start, after E changed outside a step, or the
//         slabs next to a moved window edge), over window-relative slabs
//         [i0, i0 + ni);
// mode 1: C^{n+1} = curl'(E^{n+1}) and the two B half steps.
// ---------------------------------------------------------------------------
constexpr int CB_X = 4, CB_Y = 8, CB_Z = 32;
constexpr int CE_X = CB_X + 2, CE_Y = CB_Y + 2, CE_Z = CB_Z + 2;  // staged E extents
constexpr int CE_N = CE_X * CE_Y * CE_Z;
// smoothed-field extents
constexpr int SXN = (CB_X + 1) * CB_Y * CB_Z;  // S_x Ey, S_x Ez
constexpr int SYN = CB_X * (CB_Y + 1) * CB_Z;  // S_y Ez, S_y Ex
constexpr int SZN = CB_X * CB_Y * (CB_Z + 1);  // S_z Ex, S_z Ey

template <typename T>
size_t curl_tiled_smem_bytes() {
  return sizeof(T) * (3 * (size_t)CE_N + 2 * (size_t)(SXN + SYN + SZN));
}

template <typename T>
__global__ void __launch_bounds__(256) k_curl_tiled(Geom<T> g, Smooth<T> S, Fields<T> f, Fields<T> cc,
                                                   FieldCoef<T> fc, int mode, int i0, int ni, Pml<T> pm) {
  if (!dyn_prologue(g)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sE = reinterpret_cast<T*>(smem_raw);  // [3][CE_X][CE_Y][CE_Z], origin (bx-1, by-1, bz-1)
  T* sSxEy = sE + 3 * CE_N;                // [CB_X+1][CB_Y][CB_Z]
  T* sSxEz = sSxEy + SXN;
  T* sSyEz = sSxEz + SXN;                  // [CB_X][CB_Y+1][CB_Z]
  T* sSyEx = sSyEz + SYN;
  T* sSzEx = sSyEx + SYN;                  // [CB_X][CB_Y][CB_Z+1]
  T* sSzEy = sSzEx + SZN;
  const int bx = i0 + blockIdx.x * CB_X, by = blockIdx.y * CB_Y, bz = blockIdx.z * CB_Z;
  const int tid = threadIdx.x;

  // stage E with a one-cell halo (zero outside an open window)
  for (int q = tid; q < CE_N; q += blockDim.x) {
    const int lz = q % CE_Z, r = q / CE_Z;
    const int ly = r % CE_Y, lx = r / CE_Y;
    int s = slab_of(g, bx - 1 + lx);
    int j = by - 1 + ly, k = bz - 1 + lz;
    if (g.pml) {  // zero beyond the grid
      if (j < 0 || j >= g.ny || k < 0 || k >= g.nz) s = -1;
      j = min(max(j, 0), g.ny - 1);
      k = min(max(k, 0), g.nz - 1);
    } else {  // periodic; a block may exceed a small ny or nz more than once
      j = j < 0 ? j + g.ny : (j >= g.ny ? j - g.ny : j);
      k = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
      if ((unsigned)j >= (unsigned)g.ny) j = wrapi(j, g.ny);
      if ((unsigned)k >= (unsigned)g.nz) k = wrapi(k, g.nz);
    }
    const size_t gi = (size_t)(s < 0 ? 0 : s) * g.nyz + (size_t)j * g.nz + k;
#pragma unroll
    for (int c = 0; c < 3; ++c) sE[c * CE_N + q] = s < 0 ? T(0) : f.c[EX + c][gi];
  }
  // Read what the output step needs from global memory (C, and B in mode 1)
  // now, so that these loads overlap the shared-memory smoothing below.
  // blockDim.x is 256: each thread owns kPer cells of the block.
  constexpr int kPer = CB_X * CB_Y * CB_Z / 256;
  static_assert(CB_X * CB_Y * CB_Z % 256 == 0, "whole cells per thread");
  T pb[kPer][3], pc[kPer][3];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int q = tid + 256 * t;
    const int lz = q % CB_Z, r = q / CB_Z;
    const int ly = r % CB_Y, lx = r / CB_Y;
    const int i = bx + lx, j = by + ly, k = bz + lz;
    const bool in = i < i0 + ni && j < g.ny && k < g.nz;
    const size_t id = in ? (size_t)slab_of(g, i) * g.nyz + (size_t)j * g.nz + k : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pc[t][c] = in && mode == 1 ? cc.c[c][id] : T(0);
      pb[t][c] = in && mode == 1 ? f.c[BX + c][id] : T(0);
    }
  }
  __syncthreads();

  auto E = [&](int c, int lx, int ly, int lz) -> T { return sE[c * CE_N + (lx * CE_Y + ly) * CE_Z + lz]; };
  // S_x at staged (lx, ly, lz): smoothing in y and z
  auto sx = [&](int c, int lx, int ly, int lz) -> T {
    const T ctr = E(c, lx, ly, lz);
    const T ey = E(c, lx, ly + 1, lz) + E(c, lx, ly - 1, lz);
    const T ez = E(c, lx, ly, lz + 1) + E(c, lx, ly, lz - 1);
    const T cr = E(c, lx, ly + 1, lz + 1) + E(c, lx, ly + 1, lz - 1) + E(c, lx, ly - 1, lz + 1) + E(c, lx, ly - 1, lz - 1);
    return S.a[0] * ctr + S.b1[0] * ey + S.b2[0] * ez + S.g[0] * cr;
  };
  auto sy = [&](int c, int lx, int ly, int lz) -> T {  // smoothing in x and z
    const T ctr = E(c, lx, ly, lz);
    const T ex = E(c, lx + 1, ly, lz) + E(c, lx - 1, ly, lz);
    const T ez = E(c, lx, ly, lz + 1) + E(c, lx, ly, lz - 1);
    const T cr = E(c, lx + 1, ly, lz + 1) + E(c, lx + 1, ly, lz - 1) + E(c, lx - 1, ly, lz + 1) + E(c, lx - 1, ly, lz - 1);
    return S.a[1] * ctr + S.b1[1] * ex + S.b2[1] * ez + S.g[1] * cr;
  };
  auto sz = [&](int c, int lx, int ly, int lz) -> T {  // smoothing in x and y
    const T ctr = E(c, lx, ly, lz);
    const T ex = E(c, lx + 1, ly, lz) + E(c, lx - 1, ly, lz);
    const T ey = E(c, lx, ly + 1, lz) + E(c, lx, ly - 1, lz);
    const T cr = E(c, lx + 1, ly + 1, lz) + E(c, lx + 1, ly - 1, lz) + E(c, lx - 1, ly + 1, lz) + E(c, lx - 1, ly - 1, lz);
    return S.a[2] * ctr + S.b1[2] * ex + S.b2[2] * ey + S.g[2] * cr;
  };
  // each smoothed value once (block-local coordinates; staged = local + 1)
  for (int q = tid; q < SXN; q += blockDim.x) {
    const int lz = q % CB_Z, r = q / CB_Z;
    const int ly = r % CB_Y, lx = r / CB_Y;
    sSxEy[q] = sx(1, lx + 1, ly + 1, lz + 1);
    sSxEz[q] = sx(2, lx + 1, ly + 1, lz + 1);
  }
  for (int q = tid; q < SYN; q += blockDim.x) {
    const int lz = q % CB_Z, r = q / CB_Z;
    const int ly = r % (CB_Y + 1), lx = r / (CB_Y + 1);
    sSyEz[q] = sy(2, lx + 1, ly + 1, lz + 1);
    sSyEx[q] = sy(0, lx + 1, ly + 1, lz + 1);
  }
  for (int q = tid; q < SZN; q += blockDim.x) {
    const int lz = q % (CB_Z + 1), r = q / (CB_Z + 1);
    const int ly = r % CB_Y, lx = r / CB_Y;
    sSzEx[q] = sz(0, lx + 1, ly + 1, lz + 1);
    sSzEy[q] = sz(1, lx + 1, ly + 1, lz + 1);
  }
  __syncthreads();

#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int q = tid + 256 * t;
    const int lz = q % CB_Z, r = q / CB_Z;
    const int ly = r % CB_Y, lx = r / CB_Y;
    const int i = bx + lx, j = by + ly, k = bz + lz;
    if (i >= i0 + ni || j >= g.ny || k >= g.nz) continue;
    const int x0 = (lx * CB_Y + ly) * CB_Z + lz, x1 = ((lx + 1) * CB_Y + ly) * CB_Z + lz;
    const int y0 = (lx * (CB_Y + 1) + ly) * CB_Z + lz, y1 = (lx * (CB_Y + 1) + ly + 1) * CB_Z + lz;
    const int z0 = (lx * CB_Y + ly) * (CB_Z + 1) + lz;
    // Bx: D_y S_y Ez - D_z S_z Ey; By: D_z S_z Ex - D_x S_x Ez; Bz: D_x S_x Ey - D_y S_y Ex
    T dyEz = (sSyEz[y1] - sSyEz[y0]) * fc.idy, dzEy = (sSzEy[z0 + 1] - sSzEy[z0]) * fc.idz;
    T dzEx = (sSzEx[z0 + 1] - sSzEx[z0]) * fc.idz;
    const T dxEz = (sSxEz[x1] - sSxEz[x0]) * fc.idx, dxEy = (sSxEy[x1] - sSxEy[x0]) * fc.idx;
    T dyEx = (sSyEx[y1] - sSyEx[y0]) * fc.idy;
    const int slab = slab_of(g, i);
    if (pm.L) {  // Bx (i, j+1/2, k+1/2), By (i+1/2, j, k+1/2), Bz (i+1/2, j+1/2, k): half nodes
      // mode 1 advances the memory variables with E^{n+1}; mode 0 uses them as stored
      const int jr = pml_row(j, g.ny, pm.L);
      if (jr >= 0) {
        const size_t pi = ((size_t)slab * pm.rows + jr) * g.nz + k;
        T p2 = pm.py[2][pi], p3 = pm.py[3][pi];
        if (mode == 1) {
          const T a = pm.cy[2 * g.ny + j], b = pm.cy[3 * g.ny + j];
          p2 = b * p2 + a * dyEz;
          p3 = b * p3 + a * dyEx;
          pm.py[2][pi] = p2;
          pm.py[3][pi] = p3;
        }
        dyEz += p2;
        dyEx += p3;
      }
      const int kr = pml_row(k, g.nz, pm.L);
      if (kr >= 0) {
        const size_t pi = ((size_t)slab * g.ny + j) * pm.rows + kr;
        T p2 = pm.pz[2][pi], p3 = pm.pz[3][pi];
        if (mode == 1) {
          const T a = pm.cz[2 * g.nz + k], b = pm.cz[3 * g.nz + k];
          p2 = b * p2 + a * dzEy;
          p3 = b * p3 + a * dzEx;
          pm.pz[2][pi] = p2;
          pm.pz[3][pi] = p3;
        }
        dzEy += p2;
        dzEx += p3;
      }
    }
    const T cx = dyEz - dzEy, cy = dzEx - dxEz, cz = dxEy - dyEx;
    const size_t id = (size_t)slab * g.nyz + (size_t)j * g.nz + k;
    if (mode == 1) {
      f.c[BX][id] = (pb[t][0] - fc.hdt * pc[t][0]) - fc.hdt * cx;
      f.c[BY][id] = (pb[t][1] - fc.hdt * pc[t][1]) - fc.hdt * cy;
      f.c[BZ][id] = (pb[t][2] - fc.hdt * pc[t][2]) - fc.hdt * cz;
    }
    cc.c[0][id] = cx;
    cc.c[1][id] = cy;
    cc.c[2][id] = cz;
  }
}

// ---------------------------------------------------------------------------
// Laser: boundary source on the window's back plane, and in-box start.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_hard_source(Geom<T> g, T* Ey, Laser L, double x_plane, double t, double dy, double dz) {
  const int n = g.nyz;
  const int s = slab_of(g, 0);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int j = r / g.nz, k = r - j * g.nz;
    Ey[(size_t)s * n + r] = (T)laser_ey(L, x_plane, (j + 0.5) * dy, k * dz, t);
  }
}

// In-box start, part 1: Ey(t) at its nodes and Bz(t + dt/2) at its nodes.
template <typename T>
__global__ void k_laser_fill(Geom<T> g, T* Ey, T* Bz, Laser L, double xnode0, double dx, double dy, double dz,
                             double t, double dt) {
  const long long ncell = (long long)g.nx * g.nyz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / g.nyz);
    const int r = (int)(q - (long long)i * g.nyz);
    const int j = r / g.nz, k = r - j * g.nz;
    const size_t id = (size_t)slab_of(g, i) * g.nyz + r;
    Ey[id] = (T)laser_ey(L, xnode0 + i * dx, (j + 0.5) * dy, k * dz, t);
    Bz[id] = (T)laser_ey(L, xnode0 + (i + 0.5) * dx, (j + 0.5) * dy, k * dz, t + 0.5 * dt);
  }
}

// In-box start, part 2: Ex from the discrete Gauss law and Bx from the
// discrete div B = 0, integrated from the back face (one thread per line).
template <typename T>
__global__ void k_laser_scan(Geom<T> g, const T* Ey, T* Ex, const T* Bz, T* Bx) {
  const int n = g.nyz;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int j = r / g.nz, k = r - j * g.nz;
    const int jm = j == 0 ? g.ny - 1 : j - 1, kp = k + 1 == g.nz ? 0 : k + 1;
    // with absorbing layers the neighbours beyond the grid are zero, not wrapped
    const bool jm_in = !(g.pml && j == 0), kp_in = !(g.pml && k + 1 == g.nz);
    T ex = T(0), bx = T(0);
    for (int i = 0; i < g.nx; ++i) {
      const size_t sb = (size_t)slab_of(g, i) * n;
      ex -= g.dx * (Ey[sb + j * g.nz + k] - (jm_in ? Ey[sb + jm * g.nz + k] : T(0))) / g.dy;
      Ex[sb + r] = ex;
      Bx[sb + r] = bx;
      bx -= g.dx * ((kp_in ? Bz[sb + j * g.nz + kp] : T(0)) - Bz[sb + j * g.nz + k]) / g.dz;
    }
  }
}

template <typename T>
__global__ void k_add(T* dst, const T* src, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] += src[q];
}

// ---------------------------------------------------------------------------
// Plasma loading / window injection (Sec. 3.1 profile, SplitMix64 keys).
// One thread per (cell, slot) of relative x cells [lo, hi].
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T one_below();
template <>
__device__ __forceinline__ float one_below<float>() { return 0.99999994f; }
template <>
__device__ __forceinline__ double one_below<double>() { return 0.99999999999999989; }

struct LoadSpec {
  long long shifts;   // window shifts so far: lab cell = shifts + relative cell
  int lo, hi;         // relative x cells to load
  int ppc, lattice;
  int ns[3];          // sub-lattice of the jittered lattice
  uint64_t seed;
  double x0, dx, dVppc;  // normalised; dV / ppc
  const double* px;
  const double* pn;
  int np;
  int capacity;
  int pml;            // plasma only in y, z cells [pml, n - pml)
};

template <typename T>
__global__ void k_load(Geom<T> g, Parts<T> p, int* d_np, int* d_err, LoadSpec L) {
  const long long nslot = (long long)(L.hi - L.lo + 1) * g.nyz * L.ppc;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q0 = (long long)blockIdx.x * blockDim.x; q0 < nslot; q0 += stride) {
    const long long q = q0 + threadIdx.x;
    bool want = false;
    double o[3] = {0, 0, 0}, n = 0;
    int ci = 0, j = 0, k = 0, sl = 0;
    unsigned long long cell = 0;
    if (q < nslot) {
      sl = (int)(q % L.ppc);
      const long long c = q / L.ppc;
      const int r = (int)(c % g.nyz);
      ci = L.lo + (int)(c / g.nyz);
      j = r / g.nz;
      k = r - j * g.nz;
      const long long lab = L.shifts + ci;
      cell = ((unsigned long long)lab * g.ny + j) * g.nz + k;
      const unsigned long long ctr = (cell * L.ppc + sl) * 3ull;
      double rr[3];
      for (int d = 0; d < 3; ++d) rr[d] = unit_uniform(L.seed, ctr + d);
      if (L.lattice) {
        const int sx = sl / (L.ns[1] * L.ns[2]), sy = (sl / L.ns[2]) % L.ns[1], sz = sl % L.ns[2];
        o[0] = (sx + rr[0]) / L.ns[0];
        o[1] = (sy + rr[1]) / L.ns[1];
        o[2] = (sz + rr[2]) / L.ns[2];
      } else {
        o[0] = rr[0];
        o[1] = rr[1];
        o[2] = rr[2];
      }
      const bool inner = j >= L.pml && j < g.ny - L.pml && k >= L.pml && k < g.nz - L.pml;
      n = inner ? profile_at(L.px, L.pn, L.np, L.x0 + ((double)lab + o[0]) * L.dx) : 0.0;
      want = n > 0.0;
    }
    const int slot = warp_append(d_np, want);
    if (want) {
      if (slot >= L.capacity) {
        atomicOr(d_err, 1);
      } else {
        const int s = slab_of(g, ci);
        p.cell[slot] = s * g.nyz + j * g.nz + k;
        for (int d = 0; d < 3; ++d) {
          T od = (T)o[d];
          if (od >= T(1)) od = one_below<T>();  // rounding to float may reach 1
          p.o[d][slot] = od;
          p.u[d][slot] = T(0);
        }
        p.w[slot] = (T)(n * L.dVppc);
        if (p.id) p.id[slot] = (uint32_t)(cell * L.ppc + sl);
      }
    }
  }
}

// After loading or injection the counter may exceed the capacity (the
// overflowing particles were not written and the error bit is set): clamp it.
static __global__ void k_clamp_count(int* d_np, int capacity) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *d_np > capacity) *d_np = capacity;
}

// ---------------------------------------------------------------------------
// Diagnostics (FP64 reductions).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[lane] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_field_energy(Geom<T> g, Fields<T> f, double* out) {
  const long long n = (long long)g.nx * g.nyz;
  double acc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    for (int c = EX; c <= BZ; ++c) {
      const double v = (double)f.c[c][q];
      acc += v * v;
    }
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

template <typename T>
__global__ void k_lineout(Geom<T> g, const T* Ex, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += gridDim.x * blockDim.x)
    out[i] = (double)Ex[(size_t)slab_of(g, i) * g.nyz + (size_t)(g.ny / 2) * g.nz + g.nz / 2];
}

// Weighted transverse moments of the particles with gamma > gmin for the
// normalised emittance (Sec. 3.2): out[0] = sum w, then per axis y, z:
// sum w u, w u^2, w r, w r^2, w u r with r the distance from the box axis
// (normalised units).
template <typename T>
__global__ void __launch_bounds__(256) k_emittance_moments(Geom<T> g, Parts<T> p, const int* __restrict__ d_np,
                                                          double gmin, double* out) {
  const int n = *d_np;
  double acc[11];
#pragma unroll
  for (int i = 0; i < 11; ++i) acc[i] = 0.0;
  const double d[2] = {(double)g.dy, (double)g.dz};
  const int nn[2] = {g.ny, g.nz};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const double ux = p.u[0][q], uy = p.u[1][q], uz = p.u[2][q];
    if (!(sqrt(1.0 + ux * ux + uy * uy + uz * uz) > gmin)) continue;
    const double w = (double)p.w[q];
    const int cell = p.cell[q];
    const int r = cell % g.nyz;
    const int cyz[2] = {r / g.nz, r % g.nz};
    acc[0] += w;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const double uu = (double)p.u[1 + a][q];
      const double rr = ((double)cyz[a] + (double)p.o[1 + a][q] - 0.5 * nn[a]) * d[a];
      acc[1 + 5 * a] += w * uu;
      acc[2 + 5 * a] += w * uu * uu;
      acc[3 + 5 * a] += w * rr;
      acc[4 + 5 * a] += w * rr * rr;
      acc[5 + 5 * a] += w * uu * rr;
    }
  }
#pragma unroll
  for (int i = 0; i < 11; ++i) {
    const double v = block_sum(acc[i]);
    if (threadIdx.x == 0) atomicAdd(out + i, v);
  }
}

// Charge per (window x cell, p_x bin): out[i * nb + b].
template <typename T>
__global__ void k_phase_x_px(Geom<T> g, Parts<T> p, const int* __restrict__ d_np, double pmin, double pmax, int nb,
                             double* out) {
  const int n = *d_np;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const double ux = p.u[0][q];
    if (!(ux >= pmin && ux < pmax)) continue;
    int b = (int)floor((ux - pmin) / (pmax - pmin) * nb);
    if (b >= nb) b = nb - 1;
    int i = p.cell[q] / g.nyz - g.origin;
    if (i < 0) i += g.nx;
    atomicAdd(out + (size_t)i * nb + b, (double)p.w[q]);
  }
}

// Electron weight per cell of the z = nz/2 plane: out[i * ny + j].
template <typename T>
__global__ void k_density_xy(Geom<T> g, Parts<T> p, const int* __restrict__ d_np, double* out) {
  const int n = *d_np;
  const int kz = g.nz / 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int cell = p.cell[q];
    const int r = cell % g.nyz;
    if (r % g.nz != kz) continue;
    int i = cell / g.nyz - g.origin;
    if (i < 0) i += g.nx;
    atomicAdd(out + (size_t)i * g.ny + r / g.nz, (double)p.w[q]);
  }
}

// ---------------------------------------------------------------------------
// Gauss-law residual (Sec. 2: the field update takes its current from the
// particles' motion, and a charge-conserving deposit keeps div E - rho fixed
// in time).  rho is the node charge density of the cubic shapes in FP64,
// window-relative [i][j][k]; the immobile ions (Sec. 1) are the frozen
// negative of the electrons as loaded, regenerated here from the same
// counter-based draws (and the same rounding of offsets and weights) as the
// loading, for every lab cell that has been loaded and can reach a node of
// the window.  Nodes beyond an open x end or an absorbing-layer grid edge are
// dropped, periodic axes wrap.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void rho_deposit_cubic(const Geom<T>& g, double* rho, int ci, int cj, int ck,
                                                  const double o[3], double qd) {
  double w[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) bspline3(o[d], w[d]);
  for (int a = 0; a < 4; ++a) {
    int i = ci - 1 + a;
    if (g.periodic_x)
      i = wrapi(i, g.nx);
    else if (i < 0 || i >= g.nx)
      continue;
    for (int b = 0; b < 4; ++b) {
      int j = cj - 1 + b;
      if (g.pml) {
        if (j < 0 || j >= g.ny) continue;
      } else {
        j = wrapi(j, g.ny);
      }
      for (int c = 0; c < 4; ++c) {
        int k = ck - 1 + c;
        if (g.pml) {
          if (k < 0 || k >= g.nz) continue;
        } else {
          k = wrapi(k, g.nz);
        }
        atomicAdd(rho + ((size_t)i * g.ny + j) * g.nz + k, qd * w[0][a] * w[1][b] * w[2][c]);
      }
    }
  }
}

// Electrons: qdv = q / dV (the weight carries the number of electrons).
template <typename T>
__global__ void k_rho_particles(Geom<T> g, Parts<T> p, const int* __restrict__ d_np, double qdv, double* rho) {
  const int n = *d_np;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int cell = p.cell[q];
    int ci = cell / g.nyz - g.origin;
    if (ci < 0) ci += g.nx;
    const int r = cell - (cell / g.nyz) * g.nyz;
    const double o[3] = {(double)p.o[0][q], (double)p.o[1][q], (double)p.o[2][q]};
    rho_deposit_cubic(g, rho, ci, r / g.nz, r % g.nz, o, qdv * (double)p.w[q]);
  }
}

// Immobile ions of window-relative cells [L.lo, L.hi] (L.lo may be negative
// for an open window: those cells still reach nodes 0 and 1): qdv = -q / dV.
template <typename T>
__global__ void k_rho_ions(Geom<T> g, LoadSpec L, double qdv, double* rho) {
  const long long nslot = (long long)(L.hi - L.lo + 1) * g.nyz * L.ppc;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nslot;
       q += (long long)gridDim.x * blockDim.x) {
    const int sl = (int)(q % L.ppc);
    const long long c = q / L.ppc;
    const int r = (int)(c % g.nyz);
    const int ci = L.lo + (int)(c / g.nyz);
    const int j = r / g.nz, k = r - (r / g.nz) * g.nz;
    const long long lab = L.shifts + ci;
    const unsigned long long cell = ((unsigned long long)lab * g.ny + j) * g.nz + k;
    const unsigned long long ctr = (cell * L.ppc + sl) * 3ull;
    double rr[3], o[3];
    for (int d = 0; d < 3; ++d) rr[d] = unit_uniform(L.seed, ctr + d);
    if (L.lattice) {
      const int sx = sl / (L.ns[1] * L.ns[2]), sy = (sl / L.ns[2]) % L.ns[1], sz = sl % L.ns[2];
      o[0] = (sx + rr[0]) / L.ns[0];
      o[1] = (sy + rr[1]) / L.ns[1];
      o[2] = (sz + rr[2]) / L.ns[2];
    } else {
      o[0] = rr[0];
      o[1] = rr[1];
      o[2] = rr[2];
    }
    const bool inner = j >= L.pml && j < g.ny - L.pml && k >= L.pml && k < g.nz - L.pml;
    const double n = inner ? profile_at(L.px, L.pn, L.np, L.x0 + ((double)lab + o[0]) * L.dx) : 0.0;
    if (!(n > 0.0)) continue;
    double os[3];
    for (int d = 0; d < 3; ++d) {  // the offsets and weight as the loading stored them
      T od = (T)o[d];
      if (od >= T(1)) od = one_below<T>();
      os[d] = (double)od;
    }
    rho_deposit_cubic(g, rho, ci, j, k, os, qdv * (double)(T)(n * L.dVppc));
  }
}

// max |div E - rho_e - rho_i| and max |rho_e| over the nodes, as the bit
// patterns of non-negative doubles (which order like the values) in out[0..1].
template <typename T>
__global__ void __launch_bounds__(256) k_gauss_residual(Geom<T> g, Fields<T> f, const double* __restrict__ rho_e,
                                                        const double* __restrict__ rho_i, double idx, double idy,
                                                        double idz, unsigned long long* out) {
  const long long n = (long long)g.nx * g.nyz;
  double rmax = 0.0, emax = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / g.nyz), r = (int)(q - (long long)i * g.nyz);
    const int j = r / g.nz, k = r - (r / g.nz) * g.nz;
    const int s = slab_of(g, i), sm = slab_of(g, i - 1);
    const double div = ((double)ld(f.c[EX], g, s, j, k) - (double)ld(f.c[EX], g, sm, j, k)) * idx +
                       ((double)ld(f.c[EY], g, s, j, k) - (double)ld(f.c[EY], g, s, j - 1, k)) * idy +
                       ((double)ld(f.c[EZ], g, s, j, k) - (double)ld(f.c[EZ], g, s, j, k - 1)) * idz;
    rmax = fmax(rmax, fabs(div - rho_e[q] - rho_i[q]));
    emax = fmax(emax, fabs(rho_e[q]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
    emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(rmax));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(emax));
  }
}

// kind 0: sum of w over gamma > gmin into out[0]; kind 1: histogram of
// (gamma - 1) * mc2 over [e0, e1) into nb bins, accumulated per block in
// shared memory (dynamic, nb doubles) when nb <= kDiagSharedBins, then added
// to out once per nonzero bin.
constexpr int kDiagSharedBins = 4096;
template <typename T>
__global__ void __launch_bounds__(256) k_particle_diag(Parts<T> p, const int* __restrict__ d_np, int kind,
                                                      double gmin, double mc2, double e0, double e1, int nb,
                                                      double* out) {
  extern __shared__ double sbins[];
  const bool local = kind == 1 && nb <= kDiagSharedBins;
  if (local) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sbins[b] = 0.0;
    __syncthreads();
  }
  const int n = *d_np;
  double acc = 0.0;
  // gamma and the bin in the particles' own precision; the sums in FP64.  A
  // thread adds a run of particles that fall in the same bin before touching
  // the histogram: most particles of a plasma sit in the lowest bin, where the
  // lanes of a warp would otherwise all add to one address.
  const T te0 = (T)e0, te1 = (T)e1, tmc2 = (T)mc2;
  int run_b = -1;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const T ux = p.u[0][q], uy = p.u[1][q], uz = p.u[2][q];
    const T gam = sqrt(T(1) + ux * ux + uy * uy + uz * uz);
    const double w = (double)p.w[q];
    if (kind == 0) {
      if ((double)gam > gmin) acc += w;
    } else {
      const T e = (gam - T(1)) * tmc2;
      if (e >= te0 && e < te1) {
        int b = (int)floor((e - te0) / (te1 - te0) * (T)nb);
        if (b >= nb) b = nb - 1;
        if (b != run_b) {
          if (run_b >= 0) atomicAdd(local ? sbins + run_b : out + run_b, acc);
          run_b = b;
          acc = 0.0;
        }
        acc += w;
      }
    }
  }
  if (kind == 1 && run_b >= 0) atomicAdd(local ? sbins + run_b : out + run_b, acc);
  if (kind == 0) {
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(out, acc);
  } else if (local) {
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      if (sbins[b] != 0.0) atomicAdd(out + b, sbins[b]);
  }
}

// ---------------------------------------------------------------------------
// Device-side step state (graph-replayed batch steps).
// ---------------------------------------------------------------------------
// Start of a step: decide whether it ends with a window shift (the same FP64
// accumulator arithmetic as the host path, without contraction).
static __global__ void k_step_begin(DynState* d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double t_old = __dmul_rn((double)d->step, d->dt);
  const double t_new = __dmul_rn((double)(d->step + 1), d->dt);
  double fn = d->frac;
  if (d->has_window && t_new > d->t0) {
    const double span = t_old >= d->t0 ? d->dt : __dsub_rn(t_new, d->t0);
    fn = __dadd_rn(d->frac, __ddiv_rn(__dmul_rn(d->v, span), d->dx));
  }
  d->frac_new = fn;
  d->shift = fn >= 1.0 ? 1 : 0;
  d->origin_after = d->shift ? (d->origin + 1) % d->nx : d->origin;
}

// After the field update: commit the step and the shift.
static __global__ void k_window_commit(DynState* d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  d->step += 1;
  if (d->shift) {
    d->frac = __dsub_rn(d->frac_new, 1.0);
    d->origin = d->origin_after;
    d->shifts += 1;
  } else {
    d->frac = d->frac_new;
  }
}

// On a shift step: zero all components of the storage slab that left the
// window at the back (it is the new front slab).
template <typename T>
__global__ void k_zero_front_slab(Geom<T> g, Fields<T> f, Pml<T> pm) {
  if (!dyn_prologue(g)) return;
  const int slab = (g.origin + g.nx - 1) % g.nx;
  const long long n = (long long)NCOMP * g.nyz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(q / g.nyz), r = (int)(q - (long long)c * g.nyz);
    f.c[c][(size_t)slab * g.nyz + r] = T(0);
  }
  if (!pm.L) return;
  const long long ny_ = (long long)pm.rows * g.nz, nz_ = (long long)g.ny * pm.rows;  // per slab and array
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 4 * (ny_ + nz_);
       q += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(q / (ny_ + nz_));
    const long long r = q - c * (ny_ + nz_);
    if (r < ny_)
      pm.py[c][(size_t)slab * ny_ + r] = T(0);
    else
      pm.pz[c][(size_t)slab * nz_ + (r - ny_)] = T(0);
  }
}

}  // namespace pic
