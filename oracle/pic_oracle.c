/*
 * pic_oracle.c -- plain FP64 CPU oracle of the perfect-dispersion 3D
 * electromagnetic PIC step (Cowan, Kalmykov et al., J. Plasma Phys. 2012).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library.  Everything is written as plain nested loops in
 * the order the method states, with the closed-form kernels evaluated
 * directly, so that it can be read against the paper.
 *
 * One step (stored E^n, B^n at integer time, u at half time, x at integer
 * time):
 *   1. gather E^n, B^n at x^n with the cubic spline shape (abstract, Sec. 3.1:
 *      third-order spline shapes for the macroparticles);
 *   2. relativistic Boris push u^{n-1/2} -> u^{n+1/2}, x^{n+1} = x^n + dt u/gamma
 *      (the PIC particle advance of Sec. 1);
 *   3. charge-conserving (Esirkepov) deposit of J^{n+1/2} from the motion
 *      x^n -> x^{n+1} (Sec. 2: the field update takes its current from the
 *      particles' motion);
 *   4. field update of Eq. (perfDispMaxwell), Sec. 2: B is advanced in two
 *      half steps with the smoothed curl of E, E in one step with the standard
 *      curl of B and the deposited J;
 *   5. laser boundary source (Sec. 3.1 set-up), moving-window shift at the
 *      window speed (Sec. 1) with injection of fresh plasma at the front, and
 *      absorption of particles that leave an open x range.
 *
 * Readings of the paper that the code takes (the paper is silent or defers
 * the detail to an unpublished reference):
 *   - smoothing coefficients: the family in smoothing_coefficients() below,
 *     which has no dispersion along x for c dt = dx and is stable for every
 *     dx <= dy, dz (Sec. 2 constraint);
 *   - third-order spline shapes read as the cubic B-spline, 4-node support;
 *   - the same cubic weights at each field component's own staggered
 *     position for the gather;
 *   - Boris push and Esirkepov deposit (the paper names neither);
 *   - ions immobile (Sec. 1): they carry no current and are implicit.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 values (exact for e and c). */
#define OC_C 299792458.0
#define OC_QE 1.602176634e-19
#define OC_ME 9.1093837015e-31
#define OC_EPS0 8.8541878128e-12
#define OC_PI 3.14159265358979323846

struct or_sim {
  int nx, ny, nz, periodic_x, solver;
  double dx, dy, dz, dt; /* normalised */
  double lambda0, omega0, k0; /* SI: m, 1/s, 1/m */
  double x0;                  /* normalised lab x of node 0 at t = 0 */
  uint64_t seed;
  double alpha[3], beta[3][3], gam[3];
  double* F[OR_NCOMP];
  double* rho_ion;
  /* particles */
  size_t np, cap;
  double* xi[3];
  double* u[3];
  double* w;
  uint32_t* id;
  double q, m;
  int has_species, ppc, loading;
  int nprof;
  double* prof_x;
  double* prof_n;
  /* laser */
  int laser_mode;
  double a0, w0, tau, kl, xf, tpk;
  /* time and window */
  long long step, shifts;
  int has_window;
  double win_v, win_t0, win_frac;
  /* transverse absorbing layers: pml cells at each y and z end, and the
   * memory variables of the convolutional PML (see pml_coef) */
  int pml;
  double* psi[8];
};

/* Memory variables, one per stretched derivative (name: field it enters, axis):
 * E update: d_y Bz in Ex, d_y Bx in Ez, d_z By in Ex, d_z Bx in Ey;
 * B update (smoothed curl): D_y S_y Ez in Bx, D_y S_y Ex in Bz,
 * D_z S_z Ey in Bx, D_z S_z Ex in By. */
enum { PSI_EX_Y = 0, PSI_EZ_Y, PSI_EX_Z, PSI_EY_Z, PSI_CX_Y, PSI_CZ_Y, PSI_CX_Z, PSI_CY_Z };

/* ------------------------------------------------------------------ */
/* Cubic B-spline kernel M4 (abstract, Sec. 3.1 third-order splines):  */
/* the centred uniform B-spline of degree 3, support (-2, 2).          */
/* ------------------------------------------------------------------ */
double or_m4(double d) {
  double a = fabs(d);
  if (a < 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
  if (a < 2.0) {
    double b = 2.0 - a;
    return b * b * b / 6.0;
  }
  return 0.0;
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the (n+1)-th output of the
 * generator seeded with `seed`, i.e. the finaliser applied to
 * seed + (n+1) * golden_gamma.  Used as a counter-based generator so that
 * particle loading is reproducible independently of order. */
uint64_t or_splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double uniform01(uint64_t seed, uint64_t n) {
  return (double)(or_splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* Smoothing operators S_x, S_y, S_z of Sec. 2.                        */
/* S_a acts in the two directions transverse to a with centre alpha_a, */
/* edge weights beta_a[b] for the +-b neighbours and corner gamma_a.   */
/* Reading of the coefficients (the paper defers them): with           */
/* r_b = (dx/d_b)^2, gamma_x = r_y r_z/48, gamma_y = r_z/48,           */
/* gamma_z = r_y/48, beta_a[b] = r_b/8 - 2 gamma_a, alpha from         */
/* alpha_a + 2 beta_a[b] + 2 beta_a[c] + 4 gamma_a = 1.  Then the      */
/* scheme's dispersion function is 1 - (1-s_x^2)(1-r_y s_y^2)(1-r_z    */
/* s_z^2), which is in [0,1] for dx <= dy, dz and equals s_x^2 for     */
/* waves along x, so c dt = dx propagates them without dispersion.     */
/* ------------------------------------------------------------------ */
static void smoothing_coefficients(or_sim* s) {
  double r[3];
  if (s->solver == 1) { /* standard Yee curl: no smoothing */
    for (int a = 0; a < 3; ++a) {
      s->alpha[a] = 1.0;
      s->gam[a] = 0.0;
      for (int b = 0; b < 3; ++b) s->beta[a][b] = 0.0;
    }
    return;
  }
  r[0] = 1.0;
  r[1] = (s->dx / s->dy) * (s->dx / s->dy);
  r[2] = (s->dx / s->dz) * (s->dx / s->dz);
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    s->gam[a] = r[b] * r[c] / 48.0;
    s->beta[a][a] = 0.0;
    s->beta[a][b] = r[b] / 8.0 - 2.0 * s->gam[a];
    s->beta[a][c] = r[c] / 8.0 - 2.0 * s->gam[a];
    s->alpha[a] = 1.0 - 2.0 * s->beta[a][b] - 2.0 * s->beta[a][c] - 4.0 * s->gam[a];
  }
}

void or_smoothing(const or_sim* s, double out[12]) {
  /* per axis a: alpha_a, beta_a[first transverse], beta_a[second], gamma_a
   * with transverse order (y,z) for x, (x,z) for y, (x,y) for z. */
  static const int t1[3] = {1, 0, 0}, t2[3] = {2, 2, 1};
  for (int a = 0; a < 3; ++a) {
    out[4 * a + 0] = s->alpha[a];
    out[4 * a + 1] = s->beta[a][t1[a]];
    out[4 * a + 2] = s->beta[a][t2[a]];
    out[4 * a + 3] = s->gam[a];
  }
}

/* ------------------------------------------------------------------ */
/* Grid access.                                                        */
/* ------------------------------------------------------------------ */
static inline size_t ix3(const or_sim* s, int i, int j, int k) {
  return ((size_t)i * (size_t)s->ny + (size_t)j) * (size_t)s->nz + (size_t)k;
}

static inline int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

/* Value of a component array at storage index (i,j,k).  x is periodic or
 * else zero outside the window; y and z are periodic, or (with absorbing
 * layers) zero outside the grid. */
static double fv(const or_sim* s, const double* a, int i, int j, int k) {
  if (s->periodic_x)
    i = wrap(i, s->nx);
  else if (i < 0 || i >= s->nx)
    return 0.0;
  if (s->pml) {
    if (j < 0 || j >= s->ny || k < 0 || k >= s->nz) return 0.0;
  } else {
    j = wrap(j, s->ny);
    k = wrap(k, s->nz);
  }
  return a[ix3(s, i, j, k)];
}

static void fadd(or_sim* s, double* a, int i, int j, int k, double v) {
  if (s->periodic_x)
    i = wrap(i, s->nx);
  else if (i < 0 || i >= s->nx)
    return; /* never reached for particles inside the allowed range */
  if (s->pml) {
    if (j < 0 || j >= s->ny || k < 0 || k >= s->nz) return; /* never reached either */
  } else {
    j = wrap(j, s->ny);
    k = wrap(k, s->nz);
  }
  a[ix3(s, i, j, k)] += v;
}

/* ------------------------------------------------------------------ */
/* Transverse absorbing layers (Sec. 3.1: a 16-layer perfectly matched */
/* layer surrounds the box transversely; the paper gives no form).     */
/* Reading: a convolutional PML with kappa = 1 and no frequency shift  */
/* (Roden & Gedney 2000).  In the outer L cells of y (and of z) each   */
/* derivative d/dy of the field update becomes d/dy + psi, with        */
/* psi <- b psi + a (d/dy F), b = exp(-sigma dt), a = b - 1, updated   */
/* once per step at the derivative's time level.  sigma grows as the   */
/* cube of the depth into the layer: sigma = sigma_max (depth / L)^3,  */
/* sigma_max = 4 ln(1e6) / (2 L d) (normal-incidence reflection 1e-6   */
/* of the continuous layer).  The smoothed derivatives D_y S_y of the  */
/* perfect-dispersion curl are stretched the same way.  Depth, in      */
/* cells, at position pos (nodes integer, half nodes + 1/2) of an axis */
/* of n cells: max(L - pos, pos - (n - 1 - L), 0).                     */
/* ------------------------------------------------------------------ */
static void pml_coef(const or_sim* s, double pos, int n, double d, double* a, double* b) {
  const double L = (double)s->pml;
  double depth = L - pos;
  if (pos - ((double)n - 1.0 - L) > depth) depth = pos - ((double)n - 1.0 - L);
  if (depth < 0.0) depth = 0.0;
  const double sig_max = 4.0 * log(1e6) / (2.0 * L * d);
  const double r = depth / L;
  *b = exp(-sig_max * r * r * r * s->dt);
  *a = *b - 1.0;
}

/* S_axis applied to component array a at storage index (i,j,k). */
static double smooth(const or_sim* s, int axis, const double* a, int i, int j, int k) {
  static const int t1[3] = {1, 0, 0}, t2[3] = {2, 2, 1};
  int d1[3] = {0, 0, 0}, d2[3] = {0, 0, 0};
  d1[t1[axis]] = 1;
  d2[t2[axis]] = 1;
  double c = fv(s, a, i, j, k);
  double e1 = fv(s, a, i + d1[0], j + d1[1], k + d1[2]) + fv(s, a, i - d1[0], j - d1[1], k - d1[2]);
  double e2 = fv(s, a, i + d2[0], j + d2[1], k + d2[2]) + fv(s, a, i - d2[0], j - d2[1], k - d2[2]);
  double cr = fv(s, a, i + d1[0] + d2[0], j + d1[1] + d2[1], k + d1[2] + d2[2]) +
              fv(s, a, i + d1[0] - d2[0], j + d1[1] - d2[1], k + d1[2] - d2[2]) +
              fv(s, a, i - d1[0] + d2[0], j - d1[1] + d2[1], k - d1[2] + d2[2]) +
              fv(s, a, i - d1[0] - d2[0], j - d1[1] - d2[1], k - d1[2] - d2[2]);
  return s->alpha[axis] * c + s->beta[axis][t1[axis]] * e1 + s->beta[axis][t2[axis]] * e2 +
         s->gam[axis] * cr;
}

/* B += coef * curl'(E) with the smoothed curl of Sec. 2: D_i is replaced by
 * D_i S_i.  Writes into separate output arrays so that the input E is read
 * unmodified.  With absorbing layers the y and z derivatives carry their
 * memory variables: psi_mode 2 first advances them with this E (the second
 * half step of a step, whose curl the next step's first half step reuses
 * with the variables as stored: psi_mode 1); psi_mode 0 leaves them out (the
 * curl of a field increment with no history, as at the laser's set-up). */
static void curl_e_add(or_sim* s, double* const E[3], double* B[3], double coef, int psi_mode) {
  const double dx = s->dx, dy = s->dy, dz = s->dz;
  for (int i = 0; i < s->nx; ++i)
    for (int j = 0; j < s->ny; ++j)
      for (int k = 0; k < s->nz; ++k) {
        size_t id = ix3(s, i, j, k);
        /* Bx at (i, j+1/2, k+1/2): D_y S_y Ez - D_z S_z Ey */
        double dyEz = (smooth(s, 1, E[2], i, j + 1, k) - smooth(s, 1, E[2], i, j, k)) / dy;
        double dzEy = (smooth(s, 2, E[1], i, j, k + 1) - smooth(s, 2, E[1], i, j, k)) / dz;
        /* By at (i+1/2, j, k+1/2): D_z S_z Ex - D_x S_x Ez */
        double dzEx = (smooth(s, 2, E[0], i, j, k + 1) - smooth(s, 2, E[0], i, j, k)) / dz;
        double dxEz = (smooth(s, 0, E[2], i + 1, j, k) - smooth(s, 0, E[2], i, j, k)) / dx;
        /* Bz at (i+1/2, j+1/2, k): D_x S_x Ey - D_y S_y Ex */
        double dxEy = (smooth(s, 0, E[1], i + 1, j, k) - smooth(s, 0, E[1], i, j, k)) / dx;
        double dyEx = (smooth(s, 1, E[0], i, j + 1, k) - smooth(s, 1, E[0], i, j, k)) / dy;
        if (s->pml && psi_mode) {
          double ay, by, az, bz;
          pml_coef(s, j + 0.5, s->ny, dy, &ay, &by);
          pml_coef(s, k + 0.5, s->nz, dz, &az, &bz);
          if (psi_mode == 2) {
            s->psi[PSI_CX_Y][id] = by * s->psi[PSI_CX_Y][id] + ay * dyEz;
            s->psi[PSI_CZ_Y][id] = by * s->psi[PSI_CZ_Y][id] + ay * dyEx;
            s->psi[PSI_CX_Z][id] = bz * s->psi[PSI_CX_Z][id] + az * dzEy;
            s->psi[PSI_CY_Z][id] = bz * s->psi[PSI_CY_Z][id] + az * dzEx;
          }
          dyEz += s->psi[PSI_CX_Y][id];
          dyEx += s->psi[PSI_CZ_Y][id];
          dzEy += s->psi[PSI_CX_Z][id];
          dzEx += s->psi[PSI_CY_Z][id];
        }
        B[0][id] += coef * (dyEz - dzEy);
        B[1][id] += coef * (dzEx - dxEz);
        B[2][id] += coef * (dxEy - dyEx);
      }
}

/* E += dt * (curl B - J) with the standard Yee curl (Eq. perfDispMaxwell). */
static void e_update(or_sim* s) {
  const double dx = s->dx, dy = s->dy, dz = s->dz, dt = s->dt;
  double *Ex = s->F[OR_EX], *Ey = s->F[OR_EY], *Ez = s->F[OR_EZ];
  const double *Bx = s->F[OR_BX], *By = s->F[OR_BY], *Bz = s->F[OR_BZ];
  const double *Jx = s->F[OR_JX], *Jy = s->F[OR_JY], *Jz = s->F[OR_JZ];
  for (int i = 0; i < s->nx; ++i)
    for (int j = 0; j < s->ny; ++j)
      for (int k = 0; k < s->nz; ++k) {
        size_t id = ix3(s, i, j, k);
        double dyBz = (fv(s, Bz, i, j, k) - fv(s, Bz, i, j - 1, k)) / dy;
        double dzBy = (fv(s, By, i, j, k) - fv(s, By, i, j, k - 1)) / dz;
        double dzBx = (fv(s, Bx, i, j, k) - fv(s, Bx, i, j, k - 1)) / dz;
        double dxBz = (fv(s, Bz, i, j, k) - fv(s, Bz, i - 1, j, k)) / dx;
        double dxBy = (fv(s, By, i, j, k) - fv(s, By, i - 1, j, k)) / dx;
        double dyBx = (fv(s, Bx, i, j, k) - fv(s, Bx, i, j - 1, k)) / dy;
        if (s->pml) { /* Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2) */
          double ay, by, az, bz;
          pml_coef(s, (double)j, s->ny, dy, &ay, &by);
          pml_coef(s, (double)k, s->nz, dz, &az, &bz);
          s->psi[PSI_EX_Y][id] = by * s->psi[PSI_EX_Y][id] + ay * dyBz;
          s->psi[PSI_EZ_Y][id] = by * s->psi[PSI_EZ_Y][id] + ay * dyBx;
          s->psi[PSI_EX_Z][id] = bz * s->psi[PSI_EX_Z][id] + az * dzBy;
          s->psi[PSI_EY_Z][id] = bz * s->psi[PSI_EY_Z][id] + az * dzBx;
          dyBz += s->psi[PSI_EX_Y][id];
          dyBx += s->psi[PSI_EZ_Y][id];
          dzBy += s->psi[PSI_EX_Z][id];
          dzBx += s->psi[PSI_EY_Z][id];
        }
        Ex[id] += dt * (dyBz - dzBy - Jx[id]);
        Ey[id] += dt * (dzBx - dxBz - Jy[id]);
        Ez[id] += dt * (dxBy - dyBx - Jz[id]);
      }
}

/* Eq. (perfDispMaxwell): B half step, E full step, B half step. */
void or_field_update(or_sim* s) {
  double* E[3] = {s->F[OR_EX], s->F[OR_EY], s->F[OR_EZ]};
  double* B[3] = {s->F[OR_BX], s->F[OR_BY], s->F[OR_BZ]};
  curl_e_add(s, E, B, -0.5 * s->dt, 1);
  e_update(s);
  curl_e_add(s, E, B, -0.5 * s->dt, 2);
}

/* ------------------------------------------------------------------ */
/* Particles: gather, push, deposit.                                   */
/* ------------------------------------------------------------------ */

/* Interpolate component array a, whose values sit at (i+ox, j+oy, k+oz), at
 * the grid-unit position xi with the cubic B-spline weights: the sum over the
 * 4x4x4 nearest nodes of value * M4 * M4 * M4. */
static double interp(const or_sim* s, const double* a, const double xi[3], const double off[3]) {
  int base[3];
  double wgt[3][4];
  for (int d = 0; d < 3; ++d) {
    base[d] = (int)floor(xi[d] - off[d]) - 1;
    for (int m = 0; m < 4; ++m) wgt[d][m] = or_m4(xi[d] - (base[d] + m) - off[d]);
  }
  double acc = 0.0;
  for (int a0 = 0; a0 < 4; ++a0)
    for (int b0 = 0; b0 < 4; ++b0)
      for (int c0 = 0; c0 < 4; ++c0)
        acc += fv(s, a, base[0] + a0, base[1] + b0, base[2] + c0) * wgt[0][a0] * wgt[1][b0] *
               wgt[2][c0];
  return acc;
}

static const double STAG[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}, /* Ex Ey Ez */
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}  /* Bx By Bz */
};

void or_gather(const or_sim* s, const double xi[3], double E[3], double B[3]) {
  for (int c = 0; c < 3; ++c) E[c] = interp(s, s->F[OR_EX + c], xi, STAG[c]);
  for (int c = 0; c < 3; ++c) B[c] = interp(s, s->F[OR_BX + c], xi, STAG[3 + c]);
}

/* Relativistic Boris rotation; h = q dt / (2 m).  u = gamma v / c. */
void or_boris(double u[3], const double E[3], const double B[3], double h) {
  double um[3], up[3], t[3], sv[3], uprime[3];
  for (int c = 0; c < 3; ++c) um[c] = u[c] + h * E[c];
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  for (int c = 0; c < 3; ++c) t[c] = h * B[c] / gm;
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int c = 0; c < 3; ++c) sv[c] = 2.0 * t[c] / (1.0 + t2);
  uprime[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  uprime[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  uprime[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  up[0] = um[0] + (uprime[1] * sv[2] - uprime[2] * sv[1]);
  up[1] = um[1] + (uprime[2] * sv[0] - uprime[0] * sv[2]);
  up[2] = um[2] + (uprime[0] * sv[1] - uprime[1] * sv[0]);
  for (int c = 0; c < 3; ++c) u[c] = up[c] + h * E[c];
}

/* Esirkepov charge-conserving deposit of one macroparticle of charge q*w
 * moving xi0 -> xi1 (grid units, |xi1 - xi0| < 1 per axis) during dt.
 * With S0, S1 the cubic shapes before and after the move on a 6-node window
 * per axis and DS = S1 - S0:
 *   Wx = DSx [S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3], cyclic for Wy, Wz,
 *   Jx(i+1/2,j,k) = -(q w / (dt dy dz)) sum_{i' <= i} Wx(i',j,k), likewise y, z. */
void or_deposit_one(or_sim* s, const double xi0[3], const double xi1[3], double qw) {
  int base[3];
  double S0[3][6], DS[3][6];
  for (int d = 0; d < 3; ++d) {
    base[d] = (int)floor(xi0[d]) - 2;
    for (int m = 0; m < 6; ++m) {
      double n = (double)(base[d] + m);
      S0[d][m] = or_m4(xi0[d] - n);
      DS[d][m] = or_m4(xi1[d] - n) - S0[d][m];
    }
  }
  const double dx = s->dx, dy = s->dy, dz = s->dz, dt = s->dt;
  const double cx = -qw / (dt * dy * dz), cy = -qw / (dt * dx * dz), cz = -qw / (dt * dx * dy);
  /* Jx: running sum along x */
  for (int b = 0; b < 6; ++b)
    for (int c = 0; c < 6; ++c) {
      double t = S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c] + 0.5 * S0[1][b] * DS[2][c] +
                 DS[1][b] * DS[2][c] / 3.0;
      double run = 0.0;
      for (int a = 0; a < 6; ++a) {
        run += DS[0][a] * t;
        if (run != 0.0) fadd(s, s->F[OR_JX], base[0] + a, base[1] + b, base[2] + c, cx * run);
      }
    }
  /* Jy: running sum along y */
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 6; ++c) {
      double t = S0[0][a] * S0[2][c] + 0.5 * DS[0][a] * S0[2][c] + 0.5 * S0[0][a] * DS[2][c] +
                 DS[0][a] * DS[2][c] / 3.0;
      double run = 0.0;
      for (int b = 0; b < 6; ++b) {
        run += DS[1][b] * t;
        if (run != 0.0) fadd(s, s->F[OR_JY], base[0] + a, base[1] + b, base[2] + c, cy * run);
      }
    }
  /* Jz: running sum along z */
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double t = S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b] + 0.5 * S0[0][a] * DS[1][b] +
                 DS[0][a] * DS[1][b] / 3.0;
      double run = 0.0;
      for (int c = 0; c < 6; ++c) {
        run += DS[2][c] * t;
        if (run != 0.0) fadd(s, s->F[OR_JZ], base[0] + a, base[1] + b, base[2] + c, cz * run);
      }
    }
}

static void push_and_deposit(or_sim* s) {
  size_t n = (size_t)s->nx * s->ny * s->nz;
  for (int c = OR_JX; c <= OR_JZ; ++c) memset(s->F[c], 0, n * sizeof(double));
  const double h = s->q * s->dt / (2.0 * s->m);
  const double d[3] = {s->dx, s->dy, s->dz};
  const int N[3] = {s->nx, s->ny, s->nz};
  for (size_t p = 0; p < s->np; ++p) {
    double xi0[3] = {s->xi[0][p], s->xi[1][p], s->xi[2][p]};
    double E[3], B[3], u[3] = {s->u[0][p], s->u[1][p], s->u[2][p]};
    or_gather(s, xi0, E, B);
    or_boris(u, E, B, h);
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double xi1[3];
    for (int c = 0; c < 3; ++c) xi1[c] = xi0[c] + s->dt * u[c] / (g * d[c]);
    or_deposit_one(s, xi0, xi1, s->q * s->w[p]);
    for (int c = 0; c < 3; ++c) {
      double x = xi1[c];
      if (c == 0 ? s->periodic_x : !s->pml) {
        if (x < 0.0) x += N[c];
        if (x >= N[c]) x -= N[c];
      }
      s->xi[c][p] = x;
      s->u[c][p] = u[c];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Plasma loading (Sec. 3.1 density profile), with the counter-based   */
/* SplitMix64 draws keyed on (seed, lab cell, slot, component).        */
/* ------------------------------------------------------------------ */
static double profile(const or_sim* s, double x) {
  if (s->nprof <= 0) return 0.0;
  if (x < s->prof_x[0] || x > s->prof_x[s->nprof - 1]) return 0.0;
  for (int i = 0; i + 1 < s->nprof; ++i) {
    if (x <= s->prof_x[i + 1]) {
      double x0 = s->prof_x[i], x1 = s->prof_x[i + 1];
      if (x1 <= x0) return s->prof_n[i + 1];
      double f = (x - x0) / (x1 - x0);
      return s->prof_n[i] + f * (s->prof_n[i + 1] - s->prof_n[i]);
    }
  }
  return s->prof_n[s->nprof - 1];
}

static void reserve(or_sim* s, size_t need) {
  if (need <= s->cap) return;
  size_t cap = s->cap ? s->cap : 1024;
  while (cap < need) cap *= 2;
  for (int c = 0; c < 3; ++c) {
    s->xi[c] = (double*)realloc(s->xi[c], cap * sizeof(double));
    s->u[c] = (double*)realloc(s->u[c], cap * sizeof(double));
  }
  s->w = (double*)realloc(s->w, cap * sizeof(double));
  s->id = (uint32_t*)realloc(s->id, cap * sizeof(uint32_t));
  s->cap = cap;
}

static int lattice_dims(int ppc, int ns[3]) {
  switch (ppc) {
    case 1: ns[0] = 1; ns[1] = 1; ns[2] = 1; return 0;
    case 2: ns[0] = 1; ns[1] = 2; ns[2] = 1; return 0;
    case 4: ns[0] = 1; ns[1] = 2; ns[2] = 2; return 0;
    case 8: ns[0] = 2; ns[1] = 2; ns[2] = 2; return 0;
    default: return -1;
  }
}

/* Node charge density of the given particles added into rho with sign sgn. */
static void rho_add(or_sim* s, double* rho, size_t p0, size_t p1, double sgn) {
  double dV = s->dx * s->dy * s->dz;
  for (size_t p = p0; p < p1; ++p) {
    int base[3];
    double wg[3][4];
    double xi[3] = {s->xi[0][p], s->xi[1][p], s->xi[2][p]};
    for (int d = 0; d < 3; ++d) {
      base[d] = (int)floor(xi[d]) - 1;
      for (int m = 0; m < 4; ++m) wg[d][m] = or_m4(xi[d] - (base[d] + m));
    }
    double qd = sgn * s->q * s->w[p] / dV;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int c = 0; c < 4; ++c)
          fadd(s, rho, base[0] + a, base[1] + b, base[2] + c, qd * wg[0][a] * wg[1][b] * wg[2][c]);
  }
}

/* Load relative x cells [lo, hi] (lab cell = shifts + relative cell). */
static void load_cells(or_sim* s, int lo, int hi) {
  int ns[3] = {1, 1, 1};
  if (s->loading == OR_LOAD_LATTICE) lattice_dims(s->ppc, ns);
  size_t first = s->np;
  for (int ci = lo; ci <= hi; ++ci) {
    long long L = s->shifts + ci;
    for (int j = s->pml; j < s->ny - s->pml; ++j)
      for (int k = s->pml; k < s->nz - s->pml; ++k) {
        uint64_t cell = ((uint64_t)L * (uint64_t)s->ny + (uint64_t)j) * (uint64_t)s->nz + (uint64_t)k;
        for (int sl = 0; sl < s->ppc; ++sl) {
          uint64_t ctr = (cell * (uint64_t)s->ppc + (uint64_t)sl) * 3u;
          double r[3], o[3];
          for (int c = 0; c < 3; ++c) r[c] = uniform01(s->seed, ctr + (uint64_t)c);
          if (s->loading == OR_LOAD_LATTICE) {
            int sx = sl / (ns[1] * ns[2]), sy = (sl / ns[2]) % ns[1], sz = sl % ns[2];
            o[0] = (sx + r[0]) / ns[0];
            o[1] = (sy + r[1]) / ns[1];
            o[2] = (sz + r[2]) / ns[2];
          } else {
            o[0] = r[0];
            o[1] = r[1];
            o[2] = r[2];
          }
          double xlab = s->x0 + ((double)L + o[0]) * s->dx;
          double n = profile(s, xlab);
          if (!(n > 0.0)) continue;
          reserve(s, s->np + 1);
          size_t p = s->np++;
          s->xi[0][p] = ci + o[0];
          s->xi[1][p] = j + o[1];
          s->xi[2][p] = k + o[2];
          s->u[0][p] = s->u[1][p] = s->u[2][p] = 0.0;
          s->w[p] = n * s->dx * s->dy * s->dz / s->ppc;
          s->id[p] = (uint32_t)(cell * (uint64_t)s->ppc + (uint64_t)sl);
        }
      }
  }
  /* immobile ions: a frozen neutralising copy of the loaded electrons */
  rho_add(s, s->rho_ion, first, s->np, -1.0);
}

/* Allowed x cell range for open x: the cubic shapes of a particle in cell
 * c touch x indices c-2 .. c+3 during one step, which stay in the window for
 * 2 <= c <= nx - 4. */
static int x_lo(const or_sim* s) { return s->periodic_x ? 0 : 2; }
static int x_hi(const or_sim* s) { return s->periodic_x ? s->nx - 1 : s->nx - 4; }

/* With absorbing layers, particles live in the y, z cells [L, n - L) and are
 * absorbed when they leave them; the cubic shapes of such a particle stay
 * inside the grid during a step for L >= 3. */
static int inside_yz(const or_sim* s, size_t p) {
  if (!s->pml) return 1;
  int cy = (int)floor(s->xi[1][p]), cz = (int)floor(s->xi[2][p]);
  return cy >= s->pml && cy < s->ny - s->pml && cz >= s->pml && cz < s->nz - s->pml;
}

static void drop_outside(or_sim* s) {
  if (s->periodic_x && !s->pml) return;
  size_t q = 0;
  int lo = x_lo(s), hi = x_hi(s);
  for (size_t p = 0; p < s->np; ++p) {
    int c = (int)floor(s->xi[0][p]);
    if (!s->periodic_x && (c < lo || c > hi)) continue;
    if (!inside_yz(s, p)) continue;
    if (q != p) {
      for (int d = 0; d < 3; ++d) {
        s->xi[d][q] = s->xi[d][p];
        s->u[d][q] = s->u[d][p];
      }
      s->w[q] = s->w[p];
      s->id[q] = s->id[p];
    }
    ++q;
  }
  s->np = q;
}

/* ------------------------------------------------------------------ */
/* Moving window (Sec. 1): the box advances one cell, the back slab    */
/* leaves, the front slab enters empty and fresh plasma is loaded.     */
/* ------------------------------------------------------------------ */
static void shift_window(or_sim* s) {
  size_t slab = (size_t)s->ny * s->nz, n = slab * s->nx;
  for (int c = 0; c < OR_NCOMP; ++c) {
    memmove(s->F[c], s->F[c] + slab, (n - slab) * sizeof(double));
    memset(s->F[c] + (n - slab), 0, slab * sizeof(double));
  }
  memmove(s->rho_ion, s->rho_ion + slab, (n - slab) * sizeof(double));
  memset(s->rho_ion + (n - slab), 0, slab * sizeof(double));
  for (int c = 0; c < 8 && s->pml; ++c) {
    memmove(s->psi[c], s->psi[c] + slab, (n - slab) * sizeof(double));
    memset(s->psi[c] + (n - slab), 0, slab * sizeof(double));
  }
  for (size_t p = 0; p < s->np; ++p) s->xi[0][p] -= 1.0;
  s->shifts += 1;
  drop_outside(s);
  if (s->has_species) load_cells(s, x_hi(s), x_hi(s));
}

/* ------------------------------------------------------------------ */
/* Laser (Sec. 3.1): linearly y-polarised Gaussian, focus x_focus,     */
/* 1/e field radius w0, intensity FWHM tau, paraxial Gaussian beam.    */
/* Envelope peak passes x_focus at t_peak.                             */
/* ------------------------------------------------------------------ */
double or_laser_ey(const or_sim* s, double x, double y, double z, double t) {
  double k = s->kl;
  double zr = 0.5 * k * s->w0 * s->w0;
  double xi = x - s->xf;
  double w = s->w0 * sqrt(1.0 + (xi / zr) * (xi / zr));
  double invR = xi / (xi * xi + zr * zr);
  double psi = atan2(xi, zr);
  double yc = 0.5 * s->ny * s->dy, zc = 0.5 * s->nz * s->dz;
  double r2 = (y - yc) * (y - yc) + (z - zc) * (z - zc);
  double sh = xi - (t - s->tpk); /* distance behind/ahead of the envelope centre */
  double env = exp(-2.0 * log(2.0) * sh * sh / (s->tau * s->tau));
  double phase = -k * sh - 0.5 * k * r2 * invR + psi;
  return s->a0 * k * (s->w0 / w) * exp(-r2 / (w * w)) * env * sin(phase);
}

static double node_x(const or_sim* s, double i) { return s->x0 + ((double)s->shifts + i) * s->dx; }

static void hard_source(or_sim* s) {
  double t = (double)s->step * s->dt;
  double x = node_x(s, 0.0);
  for (int j = 0; j < s->ny; ++j)
    for (int k = 0; k < s->nz; ++k)
      s->F[OR_EY][ix3(s, 0, j, k)] = or_laser_ey(s, x, (j + 0.5) * s->dy, k * s->dz, t);
}

/* In-box initialisation: E^n from the paraxial formula with Ex from the
 * discrete Gauss law; B^{n+1/2} from the formula (Bz = Ey of the forward
 * wave, half a step later) with Bx from the discrete div B = 0; then
 * B^n = B^{n+1/2} + (dt/2) curl' E^n so that the first half push of the
 * scheme reproduces B^{n+1/2}. */
static void laser_in_box(or_sim* s) {
  size_t n = (size_t)s->nx * s->ny * s->nz;
  double* tmp = (double*)calloc(6 * n, sizeof(double));
  double* E[3] = {tmp, tmp + n, tmp + 2 * n};
  double* B[3] = {tmp + 3 * n, tmp + 4 * n, tmp + 5 * n};
  double t = (double)s->step * s->dt;
  for (int i = 0; i < s->nx; ++i)
    for (int j = 0; j < s->ny; ++j)
      for (int k = 0; k < s->nz; ++k) {
        E[1][ix3(s, i, j, k)] = or_laser_ey(s, node_x(s, i), (j + 0.5) * s->dy, k * s->dz, t);
        B[2][ix3(s, i, j, k)] =
            or_laser_ey(s, node_x(s, i + 0.5), (j + 0.5) * s->dy, k * s->dz, t + 0.5 * s->dt);
      }
  for (int j = 0; j < s->ny; ++j)
    for (int k = 0; k < s->nz; ++k) {
      double ex = 0.0, bx = 0.0;
      for (int i = 0; i < s->nx; ++i) {
        ex -= s->dx * (fv(s, E[1], i, j, k) - fv(s, E[1], i, j - 1, k)) / s->dy;
        E[0][ix3(s, i, j, k)] = ex;
        B[0][ix3(s, i, j, k)] = bx;
        bx -= s->dx * (fv(s, B[2], i, j, k + 1) - fv(s, B[2], i, j, k)) / s->dz;
      }
    }
  curl_e_add(s, E, B, 0.5 * s->dt, 0);
  for (int c = 0; c < 3; ++c)
    for (size_t q = 0; q < n; ++q) {
      s->F[OR_EX + c][q] += E[c][q];
      s->F[OR_BX + c][q] += B[c][q];
    }
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* Public API.                                                         */
/* ------------------------------------------------------------------ */
or_sim* or_create(const or_grid* g, double dt_si, const or_window* w) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return NULL;
  if (!(g->dx > 0 && g->dy > 0 && g->dz > 0 && g->lambda0 > 0)) return NULL;
  if (g->dx > g->dy || g->dx > g->dz) return NULL; /* Sec. 2 constraint */
  if (!g->periodic_x && g->nx < 8) return NULL;
  if (w && g->periodic_x) return NULL;
  if (g->pml < 0 || (g->pml > 0 && (g->pml < 3 || g->ny < 2 * g->pml + 4 || g->nz < 2 * g->pml + 4)))
    return NULL;
  or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
  s->nx = g->nx;
  s->ny = g->ny;
  s->nz = g->nz;
  s->periodic_x = g->periodic_x ? 1 : 0;
  s->lambda0 = g->lambda0;
  s->k0 = 2.0 * OC_PI / g->lambda0;
  s->omega0 = s->k0 * OC_C;
  s->dx = g->dx * s->k0;
  s->dy = g->dy * s->k0;
  s->dz = g->dz * s->k0;
  s->x0 = g->x0 * s->k0;
  s->seed = g->seed;
  if (g->solver != 0 && g->solver != 1) {
    free(s);
    return NULL;
  }
  s->solver = g->solver;
  if (s->solver == 1) { /* Yee: Courant limit 1 / sqrt(sum 1/d^2) */
    double lim = 1.0 / sqrt(1.0 / (s->dx * s->dx) + 1.0 / (s->dy * s->dy) + 1.0 / (s->dz * s->dz));
    s->dt = dt_si > 0 ? dt_si * s->omega0 : 0.999 * lim;
    if (s->dt > lim * (1.0 + 1e-12)) {
      free(s);
      return NULL;
    }
  } else {
    s->dt = dt_si > 0 ? dt_si * s->omega0 : s->dx;
    if (s->dt > s->dx * (1.0 + 1e-12)) {
      free(s);
      return NULL;
    }
  }
  smoothing_coefficients(s);
  size_t n = (size_t)s->nx * s->ny * s->nz;
  for (int c = 0; c < OR_NCOMP; ++c) s->F[c] = (double*)calloc(n, sizeof(double));
  s->rho_ion = (double*)calloc(n, sizeof(double));
  s->pml = g->pml;
  for (int c = 0; c < 8 && s->pml; ++c) s->psi[c] = (double*)calloc(n, sizeof(double));
  if (w) {
    s->has_window = 1;
    s->win_v = w->v;
    s->win_t0 = w->t_start * s->omega0;
  }
  return s;
}

void or_destroy(or_sim* s) {
  if (!s) return;
  for (int c = 0; c < OR_NCOMP; ++c) free(s->F[c]);
  free(s->rho_ion);
  for (int c = 0; c < 8; ++c) free(s->psi[c]);
  for (int c = 0; c < 3; ++c) {
    free(s->xi[c]);
    free(s->u[c]);
  }
  free(s->w);
  free(s->id);
  free(s->prof_x);
  free(s->prof_n);
  free(s);
}

int or_add_species(or_sim* s, const or_profile* prof, int ppc, double q, double m, int loading) {
  int ns[3];
  if (!s || !prof || prof->n < 1 || ppc < 1 || m <= 0 || s->has_species) return -1;
  if (loading == OR_LOAD_LATTICE && lattice_dims(ppc, ns) != 0) return -1;
  if (loading != OR_LOAD_LATTICE && loading != OR_LOAD_RANDOM) return -1;
  s->nprof = prof->n;
  s->prof_x = (double*)malloc(prof->n * sizeof(double));
  s->prof_n = (double*)malloc(prof->n * sizeof(double));
  for (int i = 0; i < prof->n; ++i) {
    s->prof_x[i] = prof->x[i] * s->k0;
    s->prof_n[i] = prof->dens[i];
  }
  s->ppc = ppc;
  s->q = q;
  s->m = m;
  s->loading = loading;
  s->has_species = 1;
  load_cells(s, x_lo(s), x_hi(s));
  return 0;
}

int or_add_laser(or_sim* s, double a0, double waist, double fwhm, double lambda_l, double x_focus,
                 double t_peak, int mode) {
  if (!s || !(waist > 0) || !(fwhm > 0) || !(lambda_l > 0)) return -1;
  s->a0 = a0;
  s->w0 = waist * s->k0;
  s->tau = fwhm * s->omega0;
  s->kl = s->lambda0 / lambda_l;
  s->xf = x_focus * s->k0;
  s->tpk = t_peak * s->omega0;
  if (mode == OR_LASER_AUTO) mode = (!s->has_window && !s->periodic_x) ? OR_LASER_HARD_SOURCE : OR_LASER_IN_BOX;
  if (mode == OR_LASER_HARD_SOURCE && (s->has_window || s->periodic_x)) return -1;
  s->laser_mode = mode;
  if (mode == OR_LASER_HARD_SOURCE)
    hard_source(s);
  else
    laser_in_box(s);
  return 0;
}

static void step_once(or_sim* s) {
  double t_old = (double)s->step * s->dt;
  double* E[3] = {s->F[OR_EX], s->F[OR_EY], s->F[OR_EZ]};
  double* B[3] = {s->F[OR_BX], s->F[OR_BY], s->F[OR_BZ]};
  push_and_deposit(s);
  /* Eq. (perfDispMaxwell); the boundary source imposes E_y^{n+1} on the
   * i = 0 plane after the E update and before the second B half step. */
  curl_e_add(s, E, B, -0.5 * s->dt, 1);
  e_update(s);
  s->step += 1;
  double t_new = (double)s->step * s->dt;
  if (s->laser_mode == OR_LASER_HARD_SOURCE) hard_source(s);
  curl_e_add(s, E, B, -0.5 * s->dt, 2);
  if (s->has_window && t_new > s->win_t0) {
    double tb = t_old > s->win_t0 ? t_old : s->win_t0;
    s->win_frac += s->win_v * (t_old >= s->win_t0 ? s->dt : (t_new - tb)) / s->dx;
    while (s->win_frac >= 1.0) {
      s->win_frac -= 1.0;
      shift_window(s);
    }
  }
  drop_outside(s);
}

void or_step(or_sim* s, int n) {
  for (int i = 0; i < n; ++i) step_once(s);
}

void or_info_get(const or_sim* s, or_info* info) {
  info->dt = s->dt;
  info->dx = s->dx;
  info->dy = s->dy;
  info->dz = s->dz;
  info->t = (double)s->step * s->dt;
  info->step = s->step;
  info->shifts = s->shifts;
  info->np = s->np;
}

double* or_field(or_sim* s, int comp) {
  if (comp < 0 || comp >= OR_NCOMP) return NULL;
  return s->F[comp];
}

size_t or_particles(or_sim* s, double** xi3, double** u3, double** w, uint32_t** id) {
  for (int c = 0; c < 3; ++c) {
    if (xi3) xi3[c] = s->xi[c];
    if (u3) u3[c] = s->u[c];
  }
  if (w) *w = s->w;
  if (id) *id = s->id;
  return s->np;
}

int or_set_particles(or_sim* s, size_t n, const double* const* xi3, const double* const* u3,
                     const double* w, const uint32_t* id) {
  const int N[3] = {s->nx, s->ny, s->nz};
  for (size_t p = 0; p < n; ++p)
    for (int c = 0; c < 3; ++c) {
      double x = xi3[c][p];
      if (c == 0 && !s->periodic_x) {
        int cl = (int)floor(x);
        if (cl < x_lo(s) || cl > x_hi(s)) return -1;
      } else if (c > 0 && s->pml) {
        if (!(x >= s->pml && x < N[c] - s->pml)) return -1;
      } else if (!(x >= 0.0 && x < N[c])) {
        return -1;
      }
    }
  s->np = 0;
  reserve(s, n);
  for (size_t p = 0; p < n; ++p) {
    for (int c = 0; c < 3; ++c) {
      s->xi[c][p] = xi3[c][p];
      s->u[c][p] = u3[c][p];
    }
    s->w[p] = w[p];
    s->id[p] = id ? id[p] : (uint32_t)p;
  }
  s->np = n;
  if (!s->has_species) {
    s->q = -1.0;
    s->m = 1.0;
  }
  return 0;
}

void or_rho(const or_sim* s, double* rho) {
  size_t n = (size_t)s->nx * s->ny * s->nz;
  memset(rho, 0, n * sizeof(double));
  rho_add((or_sim*)s, rho, 0, s->np, 1.0);
}

/* Standard discrete divergence of E at the nodes. */
void or_div_e(const or_sim* s, double* div) {
  const double *Ex = s->F[OR_EX], *Ey = s->F[OR_EY], *Ez = s->F[OR_EZ];
  for (int i = 0; i < s->nx; ++i)
    for (int j = 0; j < s->ny; ++j)
      for (int k = 0; k < s->nz; ++k)
        div[ix3(s, i, j, k)] = (fv(s, Ex, i, j, k) - fv(s, Ex, i - 1, j, k)) / s->dx +
                               (fv(s, Ey, i, j, k) - fv(s, Ey, i, j - 1, k)) / s->dy +
                               (fv(s, Ez, i, j, k) - fv(s, Ez, i, j, k - 1)) / s->dz;
}

/* Diagnostics (Fig. 1a lineout, Fig. 4 spectra, Table 1 charge), SI units. */
int or_diag(or_sim* s, int kind, double* out, size_t len, double p0, double p1) {
  const double Eunit = OC_ME * OC_C * s->omega0 / OC_QE;            /* V/m */
  const double Lunit = OC_C / s->omega0;                             /* m */
  const double nc = OC_EPS0 * OC_ME * s->omega0 * s->omega0 / (OC_QE * OC_QE); /* 1/m^3 */
  const double Qunit = OC_QE * nc * Lunit * Lunit * Lunit;           /* C per unit weight */
  const double mc2_MeV = OC_ME * OC_C * OC_C / (OC_QE * 1e6);
  size_t ncell = (size_t)s->nx * s->ny * s->nz;
  switch (kind) {
    case OR_DIAG_EX_LINEOUT:
      if (len < (size_t)s->nx) return -1;
      for (int i = 0; i < s->nx; ++i) out[i] = s->F[OR_EX][ix3(s, i, s->ny / 2, s->nz / 2)] * Eunit;
      return 0;
    case OR_DIAG_FIELD_ENERGY: {
      if (len < 1) return -1;
      double acc = 0.0;
      for (int c = OR_EX; c <= OR_BZ; ++c)
        for (size_t q = 0; q < ncell; ++q) acc += s->F[c][q] * s->F[c][q];
      out[0] = 0.5 * acc * s->dx * s->dy * s->dz * OC_EPS0 * Eunit * Eunit * Lunit * Lunit * Lunit;
      return 0;
    }
    case OR_DIAG_CHARGE: {
      if (len < 1) return -1;
      double acc = 0.0;
      for (size_t p = 0; p < s->np; ++p) {
        double g = sqrt(1.0 + s->u[0][p] * s->u[0][p] + s->u[1][p] * s->u[1][p] + s->u[2][p] * s->u[2][p]);
        if (g > p0) acc += fabs(s->q) * s->w[p];
      }
      out[0] = acc * Qunit;
      return 0;
    }
    case OR_DIAG_SPECTRUM: {
      if (len < 1 || !(p1 > p0)) return -1;
      for (size_t b = 0; b < len; ++b) out[b] = 0.0;
      for (size_t p = 0; p < s->np; ++p) {
        double g = sqrt(1.0 + s->u[0][p] * s->u[0][p] + s->u[1][p] * s->u[1][p] + s->u[2][p] * s->u[2][p]);
        double e = (g - 1.0) * s->m * mc2_MeV;
        if (e < p0 || e >= p1) continue;
        size_t b = (size_t)floor((e - p0) / (p1 - p0) * (double)len);
        if (b >= len) b = len - 1;
        out[b] += fabs(s->q) * s->w[p] * Qunit;
      }
      return 0;
    }
    case OR_DIAG_EMITTANCE: {
      /* Sec. 3.2: eps_N,i = (m_e c)^-1 [(<p_i^2> - <p_i>^2)(<r_i^2> - <r_i>^2)
       * - (<p_i r_i> - <r_i><p_i>)^2]^(1/2), averages weighted by the
       * macroparticle weights, over particles with gamma > p0; r_i measured
       * from the box axis.  Result in metres (x 1e6 = mm mrad). */
      if (len < 2) return -1;
      for (int ax = 1; ax <= 2; ++ax) {
        double W = 0, su = 0, suu = 0, sr = 0, srr = 0, sur = 0;
        const double d = ax == 1 ? s->dy : s->dz;
        const int N = ax == 1 ? s->ny : s->nz;
        for (size_t p = 0; p < s->np; ++p) {
          double g = sqrt(1.0 + s->u[0][p] * s->u[0][p] + s->u[1][p] * s->u[1][p] + s->u[2][p] * s->u[2][p]);
          if (!(g > p0)) continue;
          double w = s->w[p], u = s->u[ax][p], r = (s->xi[ax][p] - 0.5 * N) * d;
          W += w;
          su += w * u;
          suu += w * u * u;
          sr += w * r;
          srr += w * r * r;
          sur += w * u * r;
        }
        double e = 0.0;
        if (W > 0) {
          double mu = su / W, mr = sr / W;
          double det = (suu / W - mu * mu) * (srr / W - mr * mr) - (sur / W - mu * mr) * (sur / W - mu * mr);
          e = det > 0 ? sqrt(det) : 0.0;
        }
        out[ax - 1] = e * Lunit;
      }
      return 0;
    }
    case OR_DIAG_PHASE_X_PX: {
      /* charge per (window x cell, p_x bin), p_x / (m c) in [p0, p1) */
      if (len < (size_t)s->nx || len % (size_t)s->nx || !(p1 > p0)) return -1;
      size_t nb = len / (size_t)s->nx;
      for (size_t b = 0; b < len; ++b) out[b] = 0.0;
      for (size_t p = 0; p < s->np; ++p) {
        double ux = s->u[0][p];
        if (ux < p0 || ux >= p1) continue;
        size_t b = (size_t)floor((ux - p0) / (p1 - p0) * (double)nb);
        if (b >= nb) b = nb - 1;
        int i = (int)floor(s->xi[0][p]);
        out[(size_t)i * nb + b] += fabs(s->q) * s->w[p] * Qunit;
      }
      return 0;
    }
    case OR_DIAG_DENSITY_XY: {
      /* electron density (units of n_c) in the z = nz/2 cell plane, [i][j] */
      if (len < (size_t)s->nx * s->ny) return -1;
      for (size_t b = 0; b < (size_t)s->nx * s->ny; ++b) out[b] = 0.0;
      for (size_t p = 0; p < s->np; ++p) {
        if ((int)floor(s->xi[2][p]) != s->nz / 2) continue;
        int i = (int)floor(s->xi[0][p]), j = (int)floor(s->xi[1][p]);
        out[(size_t)i * s->ny + j] += s->w[p] / (s->dx * s->dy * s->dz);
      }
      return 0;
    }
    case OR_DIAG_DIVE_RESIDUAL: {
      if (len < 1) return -1;
      double* div = (double*)malloc(ncell * sizeof(double));
      double* rho = (double*)malloc(ncell * sizeof(double));
      or_div_e(s, div);
      or_rho(s, rho);
      double rmax = 0.0, emax = 0.0;
      for (size_t q = 0; q < ncell; ++q) {
        double r = fabs(div[q] - rho[q] - s->rho_ion[q]);
        if (r > emax) emax = r;
        if (fabs(rho[q]) > rmax) rmax = fabs(rho[q]);
      }
      out[0] = rmax > 0 ? emax / rmax : emax;
      if (len >= 3) { /* the two maxima themselves, C/m^3 */
        out[1] = emax * OC_QE * nc;
        out[2] = rmax * OC_QE * nc;
      }
      free(div);
      free(rho);
      return 0;
    }
    default:
      return -1;
  }
}
