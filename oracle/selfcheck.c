/*
 * selfcheck.c -- a small program that runs every path of the oracle once
 * (periodic and open x, moving window, both laser modes, both solvers,
 * absorbing layers, every diagnostic, particle get/set), for a build with
 * the address and undefined-behaviour sanitizers.
 *
 * TEST INFRASTRUCTURE ONLY (like the oracle itself).  Exit status 0 when every
 * call succeeded and every diagnostic is finite; the sanitizers abort on any
 * out-of-bounds access, use after free, leak or undefined operation.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "pic_oracle.h"

static const double LAM = 0.8e-6;

static double u01(uint64_t n) { return (double)(or_splitmix64(77, n) >> 11) * (1.0 / 9007199254740992.0); }

static int finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!isfinite(a[i])) return 0;
  return 1;
}

/* Random fields and particles inside [lo, hi) per axis. */
static int seed_state(or_sim* s, int nx, int ny, int nz, size_t np, const double lo[3], const double hi[3]) {
  size_t n = (size_t)nx * ny * nz;
  for (int c = 0; c < 6; ++c) {
    double* f = or_field(s, c);
    for (size_t i = 0; i < n; ++i) f[i] = 0.1 * (u01(c * n + i) - 0.5);
  }
  double* xi[3];
  double* u[3];
  double* w = (double*)malloc(np * sizeof(double));
  for (int d = 0; d < 3; ++d) {
    xi[d] = (double*)malloc(np * sizeof(double));
    u[d] = (double*)malloc(np * sizeof(double));
    for (size_t p = 0; p < np; ++p) {
      xi[d][p] = lo[d] + (hi[d] - lo[d]) * u01(1000000 + 3 * p + d);
      u[d][p] = 4.0 * (u01(2000000 + 3 * p + d) - 0.5);
    }
  }
  for (size_t p = 0; p < np; ++p) w[p] = 1e-3 * (0.5 + u01(3000000 + p));
  int rc = or_set_particles(s, np, (const double* const*)xi, (const double* const*)u, w, NULL);
  for (int d = 0; d < 3; ++d) {
    free(xi[d]);
    free(u[d]);
  }
  free(w);
  return rc;
}

static int diags(or_sim* s, int nx, int ny) {
  double out[4096];
  int bad = 0;
  bad |= or_diag(s, OR_DIAG_EX_LINEOUT, out, (size_t)nx, 0, 0) || !finite_all(out, (size_t)nx);
  bad |= or_diag(s, OR_DIAG_FIELD_ENERGY, out, 1, 0, 0) || !finite_all(out, 1);
  bad |= or_diag(s, OR_DIAG_CHARGE, out, 1, 1.0, 0) || !finite_all(out, 1);
  bad |= or_diag(s, OR_DIAG_SPECTRUM, out, 32, 0.0, 1.0) || !finite_all(out, 32);
  bad |= or_diag(s, OR_DIAG_DIVE_RESIDUAL, out, 1, 0, 0) || !finite_all(out, 1);
  bad |= or_diag(s, OR_DIAG_EMITTANCE, out, 2, 1.0, 0) || !finite_all(out, 2);
  bad |= or_diag(s, OR_DIAG_PHASE_X_PX, out, (size_t)nx * 8, -1.0, 1.0) || !finite_all(out, (size_t)nx * 8);
  bad |= or_diag(s, OR_DIAG_DENSITY_XY, out, (size_t)nx * ny, 0, 0) || !finite_all(out, (size_t)nx * ny);
  return bad;
}

int main(void) {
  int fails = 0;
  const double dx = LAM / 8, dy = LAM / 4, dz = LAM / 4;
  for (int solver = 0; solver < 2; ++solver)
    for (int pml = 0; pml <= 4; pml += 4) {
      /* periodic x, random state */
      or_grid g = {16, 12, 12, dx, dy, dz, LAM, 0.0, 1, 5, solver, pml};
      or_sim* s = or_create(&g, 0.0, NULL);
      if (!s) {
        ++fails;
        continue;
      }
      const double lo[3] = {0, pml, pml}, hi[3] = {16, 12 - pml, 12 - pml};
      if (seed_state(s, 16, 12, 12, 500, lo, hi)) ++fails;
      or_step(s, 4);
      fails += diags(s, 16, 12);
      or_destroy(s);

      /* open x, moving window, species, in-box laser */
      or_grid gw = {48, 12, 12, dx, dy, dz, LAM, -24 * dx, 0, 6, solver, pml};
      or_window w = {1.0, 0.0};
      or_sim* sw = or_create(&gw, 0.0, &w);
      double px[3] = {0.0, 1e-6, 1.0}, pn[3] = {0.0, 0.02, 0.02};
      or_profile prof = {3, px, pn};
      if (!sw || or_add_species(sw, &prof, 2, -1.0, 1.0, OR_LOAD_LATTICE) ||
          or_add_laser(sw, 2.0, 2e-6, 4e-15, LAM, 0.0, 20 * dx / 299792458.0, OR_LASER_AUTO)) {
        ++fails;
      } else {
        or_step(sw, 12);
        fails += diags(sw, 48, 12);
      }
      or_destroy(sw);
    }
  /* open x without window: boundary source, random loading */
  or_grid gh = {32, 8, 8, dx, LAM / 2, LAM / 2, LAM, 0.0, 0, 7, 0, 0};
  or_sim* sh = or_create(&gh, 0.0, NULL);
  double px[2] = {-1.0, 1.0}, pn[2] = {0.02, 0.02};
  or_profile prof = {2, px, pn};
  if (!sh || or_add_species(sh, &prof, 1, -1.0, 1.0, OR_LOAD_RANDOM) ||
      or_add_laser(sh, 2.0, 4 * LAM, 4 * LAM / 299792458.0, LAM, 0.0, 8 * LAM / 299792458.0, OR_LASER_AUTO)) {
    ++fails;
  } else {
    or_step(sh, 10);
    fails += diags(sh, 32, 8);
  }
  or_destroy(sh);
  printf("oracle selfcheck: %d failure(s)\n", fails);
  return fails ? 1 : 0;
}
