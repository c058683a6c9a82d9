// pic_device.cuh -- device-side data views and small helpers shared by the
// kernels of the perfect-dispersion PIC step (Cowan, Kalmykov et al. 2012).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

// Component order of the field block.
enum { EX = 0, EY, EZ, BX, BY, BZ, JX, JY, JZ, NCOMP };

// Grid geometry as the kernels see it.  Field arrays are [slab][j][k] with
// the x slab stored in a ring: window-relative slab i lives at storage slab
// (i + origin) mod nx, so the moving window never copies a field.
// Per-instance step state kept on the device, so that a captured CUDA graph
// can replay steps: the FP64 window accumulator, the ring origin and the
// shift decision of the current step.
struct DynState {
  double frac;      // window accumulator, cells
  double frac_new;  // accumulator at the end of the current step
  double v, dt, dx, t0;  // window speed (c), time step, cell, start time
  long long step, shifts;
  int origin;        // storage slab of window-relative slab 0
  int origin_after;  // origin once the current step's shift is applied
  int shift;         // 1 if the current step ends with a window shift
  int has_window;
  int nx;
};

template <typename T>
struct Geom {
  int nx, ny, nz;
  int origin;      // storage slab of window-relative slab 0
  int periodic_x;  // 1: x periodic; 0: open (zero outside the window)
  int nyz;         // ny * nz
  T dt, dx, dy, dz;
  const DynState* dyn;  // non-null: origin (and shift) come from the device
  int gate;             // with dyn: 1 = the kernel runs only on a shift step
  int pml;              // 0: y, z periodic; L > 0: absorbing layers, zero beyond the grid
};

// Transverse absorbing layers (convolutional PML, Sec. 3.1).  In the outer L
// cells of y (and of z) a y derivative dF/dy of the field update becomes
// dF/dy + psi with psi <- b psi + a dF/dy, once per step at the derivative's
// time level; b = exp(-sigma dt), a = b - 1 (kappa = 1, no frequency shift).
// The memory variables live in compact arrays over the rows that can have
// sigma > 0: y index j < L or j >= ny - 1 - L (2 L + 1 rows), likewise z.
template <typename T>
struct Pml {
  int L;                 // 0: no layers (all pointers null)
  int rows;              // 2 L + 1
  T* py[4];              // [slab][row][nz]: d_y Bz in Ex, d_y Bx in Ez, D_y S_y Ez in Bx, D_y S_y Ex in Bz
  T* pz[4];              // [slab][ny][row]: d_z By in Ex, d_z Bx in Ey, D_z S_z Ey in Bx, D_z S_z Ex in By
  const T* cy;           // [4][ny]: a at node j, b at node j, a at j + 1/2, b at j + 1/2
  const T* cz;           // [4][nz], the same for z
};

// Compact row of index j on an axis of n cells with L-cell layers, or -1.
__device__ __forceinline__ int pml_row(int j, int n, int L) {
  if (j < L) return j;
  if (j >= n - 1 - L) return j - (n - 1 - L) + L;
  return -1;
}

// Apply the device-side step state to a kernel's geometry; false means the
// kernel has nothing to do this step.
template <typename T>
__device__ __forceinline__ bool dyn_prologue(Geom<T>& g) {
  if (!g.dyn) return true;
  if (g.gate && !g.dyn->shift) return false;
  g.origin = g.dyn->origin;
  return true;
}

// Smoothing stencils S_x, S_y, S_z of Sec. 2 (centre, first-transverse edge,
// second-transverse edge, corner); transverse order (y,z), (x,z), (x,y).
template <typename T>
struct Smooth {
  T a[3], b1[3], b2[3], g[3];
};

// Tiling of the storage-frame grid (x slabs in ring order) used to keep the
// particles grouped; tiles at the high end of an axis may be ragged.
struct Tiles {
  int tx, ty, tz;     // tile extent in cells
  int ntx, nty, ntz;  // tiles per axis
  int n;              // ntx * nty * ntz
};

template <typename T>
struct Fields {
  T* c[NCOMP];
};

// Structure-of-arrays macroparticles: storage-frame linear cell index
// (slab*ny + j)*nz + k, offsets in [0,1) per axis, u = gamma v / c, weight.
template <typename T>
struct Parts {
  int* cell;
  T* o[3];
  T* u[3];
  T* w;
  uint32_t* id;  // may be null
};

// Cubic B-spline weights of the four nodes c-1, c, c+1, c+2 for a particle
// at offset t in [0,1) of cell c (the uniform cubic B-spline evaluated at the
// node distances 1+t, t, 1-t, 2-t).
// With s = 1 - t: w0 = s^3/6, w1 = 2/3 - t^2 + t^3/2, w2 = 2/3 - s^2 + s^3/2,
// w3 = t^3/6 (the kernel's two polynomial pieces at those distances).
template <typename T>
__device__ __forceinline__ void bspline3(T t, T w[4]) {
  const T s = T(1) - t, t2 = t * t, s2 = s * s, t3 = t2 * t, s3 = s2 * s;
  const T sixth = T(1) / T(6), two3 = T(2) / T(3);
  w[0] = s3 * sixth;
  w[1] = fma(t3, T(0.5), two3 - t2);
  w[2] = fma(s3, T(0.5), two3 - s2);
  w[3] = t3 * sixth;
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator: the
// (n+1)-th output of the stream seeded with `seed`.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ double unit_uniform(uint64_t seed, uint64_t n) {
  return (double)(splitmix64_at(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

// Laser parameters (normalised units) of the linearly y-polarised paraxial
// Gaussian pulse of Sec. 3.1.
struct Laser {
  double a0k;   // peak field a0 * k_laser
  double k;     // laser wavenumber (omega0 units)
  double w0;    // 1/e field radius
  double zr;    // Rayleigh length k w0^2 / 2
  double tau;   // intensity FWHM duration
  double xf;    // focus (lab x)
  double tpk;   // time at which the envelope peak passes xf
  double yc, zc;  // transverse axis
};

// E_y of the forward paraxial Gaussian beam at lab point (x, y, z), time t.
__device__ __forceinline__ double laser_ey(const Laser& L, double x, double y, double z, double t) {
  const double xi = x - L.xf;
  const double q = xi / L.zr;
  const double w = L.w0 * sqrt(1.0 + q * q);
  const double curv = xi / (xi * xi + L.zr * L.zr);  // 1 / R(x)
  const double gouy = atan2(xi, L.zr);
  const double r2 = (y - L.yc) * (y - L.yc) + (z - L.zc) * (z - L.zc);
  const double lag = xi - (t - L.tpk);  // position relative to the envelope centre
  const double env = exp(-1.3862943611198906 * lag * lag / (L.tau * L.tau));  // 2 ln 2
  const double ph = gouy - L.k * lag - 0.5 * L.k * r2 * curv;
  return L.a0k * (L.w0 / w) * exp(-r2 / (w * w)) * env * sin(ph);
}

// Piecewise-linear density profile n(x_lab), zero outside its range.
__device__ __forceinline__ double profile_at(const double* px, const double* pn, int np, double x) {
  if (np <= 0 || x < px[0] || x > px[np - 1]) return 0.0;
  for (int i = 0; i + 1 < np; ++i) {
    if (x <= px[i + 1]) {
      const double x0 = px[i], x1 = px[i + 1];
      if (x1 <= x0) return pn[i + 1];
      return pn[i] + (x - x0) / (x1 - x0) * (pn[i + 1] - pn[i]);
    }
  }
  return pn[np - 1];
}

// Warp-aggregated atomic increment: returns this lane's slot.
__device__ __forceinline__ int warp_append(int* counter, bool want) {
  const unsigned mask = __ballot_sync(0xffffffffu, want);
  if (!want) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

}  // namespace pic
