/*
 * pic_oracle.h -- plain FP64 CPU oracle of one explicit 3D electromagnetic
 * particle-in-cell step of the perfect-dispersion Cartesian LWFA method
 * (Cowan, Kalmykov et al., J. Plasma Phys. 2012, arXiv:1204.0838).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library
 * against the paper.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Units are normalised internally: c = eps0 = m_e = e = 1, lengths in c/omega0,
 * times in 1/omega0 with omega0 = 2 pi c / lambda0, fields in m_e c omega0 / e,
 * densities in the critical density n_c = eps0 m_e omega0^2 / e^2.  The
 * set-up calls take SI lengths and times (like the CUDA C-ABI) and convert.
 *
 * Grid (Yee, Sec. 1): node (i,j,k) sits at (i dx, j dy, k dz); Ex at (i+1/2,j,k),
 * Ey at (i,j+1/2,k), Ez at (i,j,k+1/2); Bx at (i,j+1/2,k+1/2), By at
 * (i+1/2,j,k+1/2), Bz at (i+1/2,j+1/2,k); J sits with E.  Every component
 * array is [nx][ny][nz], C order, index (i*ny + j)*nz + k, i counted from the
 * back (low-x) face of the window.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_EX = 0, OR_EY, OR_EZ, OR_BX, OR_BY, OR_BZ, OR_JX, OR_JY, OR_JZ, OR_NCOMP };
enum { OR_LOAD_RANDOM = 0, OR_LOAD_LATTICE = 1 };
enum { OR_LASER_AUTO = 0, OR_LASER_HARD_SOURCE = 1, OR_LASER_IN_BOX = 2 };
enum {
  OR_DIAG_EX_LINEOUT = 0, OR_DIAG_FIELD_ENERGY = 1, OR_DIAG_CHARGE = 2,
  OR_DIAG_SPECTRUM = 3, OR_DIAG_DIVE_RESIDUAL = 4, OR_DIAG_EMITTANCE = 5,
  OR_DIAG_PHASE_X_PX = 6, OR_DIAG_DENSITY_XY = 7
};

typedef struct {
  int nx, ny, nz;           /* cells of the window along x, y, z            */
  double dx, dy, dz;        /* metres; dx <= dy, dx <= dz (Sec. 2)          */
  double lambda0;           /* metres; sets omega0 and n_c                  */
  double x0;                /* metres; lab x of node 0 at t = 0             */
  int periodic_x;           /* 1: periodic x, 0: open x (y, z periodic)     */
  uint64_t seed;            /* particle-loading seed                        */
  int solver;               /* 0: perfect dispersion (Sec. 2), 1: Yee      */
  int pml;                  /* 0: y, z periodic; L > 0: L-cell absorbing    */
                            /* layers (PML, Sec. 3.1) at both y and z ends  */
} or_grid;

typedef struct {
  double v;                 /* window speed in units of c                   */
  double t_start;           /* seconds; the window moves for t > t_start    */
} or_window;

typedef struct {
  int n;                    /* points of a piecewise-linear n(x_lab)        */
  const double* x;          /* metres, increasing                           */
  const double* dens;       /* in units of n_c; zero outside [x0, x_{n-1}]  */
} or_profile;

typedef struct {
  double dt, dx, dy, dz;    /* normalised                                   */
  double t;                 /* normalised time of the stored E, B           */
  long long step, shifts;   /* steps taken; window shifts taken             */
  size_t np;                /* live macroparticles                          */
} or_info;

typedef struct or_sim or_sim;

/* Set-up.  dt_si <= 0 selects c dt = dx (Sec. 2, with the abstract's time
 * step enlarged in proportion to the coarse cell).  Returns NULL on invalid
 * arguments. */
or_sim* or_create(const or_grid* g, double dt_si, const or_window* w);
void or_destroy(or_sim* s);
int or_add_species(or_sim* s, const or_profile* prof, int ppc, double q, double m, int loading);
int or_add_laser(or_sim* s, double a0, double waist, double fwhm, double lambda_l,
                 double x_focus, double t_peak, int mode);
void or_step(or_sim* s, int n);
int or_diag(or_sim* s, int kind, double* out, size_t len, double p0, double p1);
void or_info_get(const or_sim* s, or_info* info);

/* State access (normalised units). */
double* or_field(or_sim* s, int comp);
size_t or_particles(or_sim* s, double** xi3, double** u3, double** w, uint32_t** id);
int or_set_particles(or_sim* s, size_t n, const double* const* xi3,
                     const double* const* u3, const double* w, const uint32_t* id);

/* Pieces used by the pins. */
double or_m4(double d);
void or_smoothing(const or_sim* s, double out[12]);
void or_boris(double u[3], const double E[3], const double B[3], double q_dt_over_2m);
void or_gather(const or_sim* s, const double xi[3], double E[3], double B[3]);
void or_rho(const or_sim* s, double* rho);
void or_div_e(const or_sim* s, double* div);
void or_deposit_one(or_sim* s, const double xi0[3], const double xi1[3], double qw);
void or_field_update(or_sim* s);
uint64_t or_splitmix64(uint64_t seed, uint64_t n);
double or_laser_ey(const or_sim* s, double x, double y, double z, double t);

#ifdef __cplusplus
}
#endif
#endif
