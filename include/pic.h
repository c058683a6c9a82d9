/*
 * pic.h -- C-ABI of the GB300 (sm_103a) library for the explicit 3D
 * electromagnetic particle-in-cell step of the perfect-dispersion Cartesian
 * laser-wakefield method of Cowan, Kalmykov et al., "Computationally efficient
 * methods for modelling laser wakefield acceleration in the blowout regime",
 * J. Plasma Phys. (2012), arXiv:1204.0838.
 *
 * One step, all on one GPU in hand-written CUDA kernels:
 *   cubic-spline gather of E, B to each macroparticle (abstract and Sec. 3.1:
 *   third-order spline macroparticle shapes), relativistic Boris push,
 *   charge-conserving (Esirkepov) cubic current deposit (Sec. 2: the field
 *   update takes its current from the particles' motion), the perfect-dispersion
 *   field update of Eq. (perfDispMaxwell) with the transversely smoothed curl
 *   of Sec. 2, and the moving window of Sec. 1.
 *
 * Conventions shared by every call:
 *   - Every call returns an int status: PIC_OK (0) or a negative PIC_ERR_*.
 *     pic_last_error() describes the most recent failure of a handle.
 *   - Set-up takes SI units (metres, seconds).  Densities are in units of the
 *     critical density n_c = eps0 m_e omega0^2 / e^2 of the grid wavelength.
 *     Charges are in units of e, masses in units of m_e.
 *   - State accessors (fields, particles) use the normalised units c = eps0 =
 *     m_e = e = 1: lengths in c/omega0, times in 1/omega0, fields in
 *     m_e c omega0 / e, omega0 = 2 pi c / lambda0.  Diagnostics are SI.
 *   - Grid (Yee, Sec. 1): node (i,j,k) at (i dx, j dy, k dz); Ex at
 *     (i+1/2,j,k), Ey at (i,j+1/2,k), Ez at (i,j,k+1/2); Bx at (i,j+1/2,k+1/2),
 *     By at (i+1/2,j,k+1/2), Bz at (i+1/2,j+1/2,k); J with E.  A component
 *     array exchanged with the host is [nx][ny][nz] in C order, index
 *     (i*ny + j)*nz + k, i counted from the back (low-x) face of the window.
 *   - The library owns all device memory (allocated through the optional
 *     pic_alloc hooks, else cudaMalloc).  The caller owns every host struct
 *     and buffer; they are copied, never retained.
 *   - Work is queued on the handle's stream; calls that return host data
 *     synchronise that stream.  A handle is not thread-safe.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PIC_OK 0
#define PIC_ERR_ARG -1      /* invalid argument                                  */
#define PIC_ERR_CUDA -2     /* a CUDA runtime call failed                        */
#define PIC_ERR_OOM -3      /* device allocation failed                          */
#define PIC_ERR_CAPACITY -4 /* particle capacity exceeded (injection/loading)    */
#define PIC_ERR_TIMEOUT -5  /* a bounded device-side wait gave up                */
#define PIC_ERR_NUMERIC -6  /* a diagnostic found NaN or Inf, or a step met a
                               particle with a non-finite momentum (reported
                               once; that particle was absorbed)              */
#define PIC_ERR_STATE -7    /* call not valid in the handle's current state      */

/* ---- enumerations ---- */
#define PIC_FP64 0
#define PIC_FP32 1
#define PIC_BC_PERIODIC 0
#define PIC_BC_OPEN 1 /* x only: fields zero outside the window, particles absorbed */
#define PIC_LOAD_RANDOM 0  /* ppc independent uniform positions per cell      */
#define PIC_LOAD_LATTICE 1 /* jittered sub-lattice: ppc 1,2,4,8 = 1x1x1,1x2x1,1x2x2,2x2x2 */
#define PIC_SOLVER_PERFECT 0 /* Sec. 2 smoothed curl, c dt = dx by default         */
#define PIC_SOLVER_YEE 1     /* standard Yee curl (S_i = 1), Courant-limited dt  */
#define PIC_LASER_AUTO 0
#define PIC_LASER_HARD_SOURCE 1 /* Ey imposed on the i = 0 plane each step   */
#define PIC_LASER_IN_BOX 2      /* paraxial pulse initialised inside the box  */
#define PIC_DIAG_EX_LINEOUT 0   /* len >= nx: Ex(i+1/2, ny/2, nz/2) in V/m     */
#define PIC_DIAG_FIELD_ENERGY 1 /* len >= 1: (1/2) sum eps0 (E^2 + c^2 B^2) dV in J */
#define PIC_DIAG_CHARGE 2       /* len >= 1: sum |q| w over gamma > a->gamma_min, C  */
#define PIC_DIAG_SPECTRUM 3     /* len = bins: charge per bin of (gamma-1) m c^2 in
                                   [a->e_min, a->e_max) MeV, C                     */
#define PIC_DIAG_EMITTANCE 4    /* len >= 2: normalised rms emittance (Sec. 3.2 formula)
                                   in y and z of the particles with gamma >
                                   a->gamma_min, metres (x 1e6 = mm mrad); transverse
                                   positions taken from the box axis                 */
#define PIC_DIAG_PHASE_X_PX 5   /* len = nx * bins: charge per (window x cell, p_x bin),
                                   p_x / (m c) in [a->p_min, a->p_max), C (Fig. 3)     */
#define PIC_DIAG_DENSITY_XY 6   /* len >= nx * ny: electron density in the z = nz/2 cell
                                   plane, [i][j], units of n_c (Fig. 2)               */
#define PIC_DIAG_DIVE_RESIDUAL 7 /* len >= 1: Gauss-law residual max |div E - rho| / max |rho_e|
                                   over the nodes, dimensionless (Sec. 2: the charge-
                                   conserving deposit keeps div E - rho fixed in time).
                                   rho = the electrons' cubic node density plus the
                                   immobile ions (Sec. 1), the frozen negative of the
                                   electrons as loaded; div E is the standard Yee
                                   divergence at the nodes.  len >= 3 adds out[1] =
                                   max |div E - rho| and out[2] = max |rho_e| in C/m^3.
                                   Uses 16 bytes of device scratch per cell.         */
#define PIC_FLAG_TRACK_IDS 1u   /* carry a 32-bit id per particle (tests, tracking) */

/* Optional device-memory hooks (e.g. a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` (256-byte aligned) or
 * NULL; free releases it.  Both are called only from set-up and destroy. */
typedef struct pic_alloc {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} pic_alloc;

typedef struct pic_grid {
  int nx, ny, nz;       /* cells of the window along x, y, z: nx >= 16,
                           ny, nz >= 4, nx, ny <= 65535, nx ny nz < 2^31      */
  double dx, dy, dz;    /* metres; dx <= dy and dx <= dz (Sec. 2 constraint)   */
  double lambda0;       /* metres; reference wavelength: omega0 and n_c        */
  double x0;            /* metres; lab-frame x of node 0 at t = 0              */
  int precision;        /* PIC_FP64 or PIC_FP32 (FP32: fields, momenta, offsets,
                           currents; the window accumulator and diagnostic
                           reductions stay FP64).  FP64 gathers and deposits
                           in 64-bit fixed point scaled per cell tile: the
                           absolute precision of FP64 at the tile's largest
                           field and current values                           */
  int bc_x;             /* PIC_BC_PERIODIC or PIC_BC_OPEN                      */
  int solver;           /* PIC_SOLVER_PERFECT (the paper's method) or
                           PIC_SOLVER_YEE (normal dispersion, for comparison;
                           Sec. 1 and Sec. 3.3 contrast the two)              */
  uint64_t seed;        /* particle-loading seed (SplitMix64 counter keys)     */
  uint32_t flags;       /* PIC_FLAG_*                                          */
  int64_t max_particles;/* particle capacity; <= 0 selects ppc * cells         */
  const pic_alloc* alloc; /* NULL: cudaMalloc / cudaFree                       */
  int pml;              /* transverse boundaries.  0: y and z periodic.  L > 0:
                           the outer L cells at each y and each z end are a
                           perfectly matched absorbing layer (Sec. 3.1 uses
                           16), fields are zero beyond the grid, plasma is
                           loaded only in cells [L, n - L) and particles that
                           leave them are absorbed.  Needs L >= 3 and
                           ny, nz >= 2 L + 4.  Reading (the paper gives no
                           form): a convolutional PML, kappa = 1, no frequency
                           shift, sigma = sigma_max (depth / L)^3 with
                           sigma_max = 2 ln(1e6) / (L d), stretching the y and
                           z derivatives of both curls (the smoothed ones of
                           the perfect-dispersion curl included).             */
} pic_grid;

typedef struct pic_window {
  double v;       /* window speed in units of c (Sec. 1: the box moves at c) */
  double t_start; /* seconds; the window moves while t > t_start              */
} pic_window;

typedef struct pic_profile {
  int n;              /* points of a piecewise-linear density n(x_lab), n >= 1 */
  const double* x;    /* metres, non-decreasing                                */
  const double* dens; /* units of n_c; zero outside [x[0], x[n-1]]             */
} pic_profile;

typedef struct pic_laser_opts {
  double x_focus; /* metres, lab frame (default 0: the plasma edge, Sec. 3.1) */
  double t_peak;  /* seconds: envelope peak passes x_focus (default 2 fwhm)   */
  int mode;       /* PIC_LASER_*                                              */
} pic_laser_opts;

typedef struct pic_diag_args {
  double gamma_min;    /* PIC_DIAG_CHARGE / PIC_DIAG_EMITTANCE threshold     */
  double e_min, e_max; /* PIC_DIAG_SPECTRUM range, MeV                       */
  double p_min, p_max; /* PIC_DIAG_PHASE_X_PX range of p_x / (m c)           */
} pic_diag_args;

typedef struct pic_info {
  double dt, dx, dy, dz; /* normalised                                       */
  double t;              /* normalised time of the stored E, B               */
  int64_t step;          /* steps taken                                      */
  int64_t shifts;        /* window shifts taken                              */
  int64_t np;            /* live macroparticles                              */
  int64_t capacity;      /* particle capacity                                */
  int64_t pushed;        /* particle pushes since creation (particle-steps)  */
  int precision;
} pic_info;

/* Kernel timing collected after pic_timing_start (CUDA events on the handle's stream
 * around each group of launches).  Groups: 0 gather/push/deposit, 1 field
 * update, 2 window shift, absorption, injection and particle re-binning,
 * 3 everything else (laser source, set-up). */
#define PIC_TIMING_GROUPS 4
typedef struct pic_timing {
  double ms[PIC_TIMING_GROUPS];          /* summed device time per group            */
  int64_t launches[PIC_TIMING_GROUPS];   /* kernel launches per group               */
  int64_t kernels;                     /* all kernel launches since the last reset */
} pic_timing;

typedef struct pic_particles {
  int64_t n;        /* in: entries to set / capacity of the get buffers; out: count */
  double* xi[3];    /* grid-unit positions (window-relative x, node i at xi = i)    */
  double* u[3];     /* u = gamma v / c                                              */
  double* w;        /* weights (normalised number of electrons)                     */
  uint32_t* id;     /* optional; NULL to skip                                       */
} pic_particles;

typedef struct pic_t pic_t;
typedef struct pic_batch_t pic_batch_t;

const char* pic_last_error(const pic_t* h);
const char* pic_version(void);

/* Create a simulation (Sec. 2, Sec. 3.1).  With the perfect-dispersion solver
 * dt <= 0 selects c dt = dx (the time step tied to the coarse longitudinal
 * cell) and an explicit dt must satisfy 0 < c dt <= dx.  With the Yee solver
 * dt <= 0 selects 0.999 of the Courant limit 1 / (c sqrt(dx^-2 + dy^-2 +
 * dz^-2)) and an explicit dt must not exceed that limit.  w == NULL: no moving window.
 * A window requires bc_x == PIC_BC_OPEN.  Errors: PIC_ERR_ARG (dx > dy or
 * dx > dz, bad sizes, nx < 16 or ny, nz < 4), PIC_ERR_OOM, PIC_ERR_CUDA. */
int pic_create(const pic_grid* g, double dt, const pic_window* w, pic_t** out);

/* Load one electron-like species from a density profile (Sec. 3.1 plasma
 * ramps) with ppc macroparticles per cell at rest, weight n(x) dV / ppc,
 * positions from SplitMix64 keyed on (seed, lab cell, slot, component).
 * Immobile ions are implicit neutralising charge (Sec. 1).  spline_order must
 * be 3 (cubic).  Only one species per handle: PIC_ERR_STATE otherwise. */
int pic_add_species(pic_t* h, const pic_profile* n, int ppc, int spline_order, double q,
                    double m, int loading);

/* Linearly y-polarised Gaussian laser (Sec. 3.1): peak normalised vector
 * potential a0, 1/e field radius `waist` (m), intensity FWHM duration (s),
 * wavelength lambda0 (m).  opts may be NULL (focus at x = 0, peak at 2 fwhm,
 * hard source on the i = 0 plane without a window and open x, else in box). */
int pic_add_laser(pic_t* h, double a0, double waist, double duration_fwhm, double lambda0,
                  const pic_laser_opts* opts);

/* Advance n steps of the explicit PIC cycle (Sec. 1): per step, gather E and B
 * to every macroparticle with its cubic shape, Boris-push it and move it,
 * deposit its current with the charge-conserving Esirkepov scheme, then
 * update B and E by Eq. (perfDispMaxwell) (Sec. 2: the curl smoothed
 * transversely, c dt = dx), and with a window move the box one cell when the
 * window accumulator crosses a cell, injecting the plasma of the new front
 * slab (Sec. 1).  Asynchronous on the handle's stream; the device error word
 * is read back, and the stream synchronised, before returning.  Errors:
 * PIC_ERR_ARG (n < 0), PIC_ERR_STATE (a batched handle), PIC_ERR_CAPACITY,
 * PIC_ERR_NUMERIC (a non-finite momentum), PIC_ERR_CUDA. */
int pic_step(pic_t* h, int n);

/* Diagnostics into a caller-owned host buffer of len doubles, SI units
 * (Fig. 1a lineout, Fig. 4 spectrum, Table 1 charge).  a may be NULL for
 * kinds that need no arguments.  PIC_ERR_NUMERIC if the result is not finite. */
int pic_diag(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a);

int pic_get_info(const pic_t* h, pic_info* out);

/* Bind the handle to a CUDA stream (cudaStream_t passed as void*; NULL = the
 * library's own stream). */
int pic_set_stream(pic_t* h, void* stream);

/* Field access, normalised units, host buffers of nx*ny*nz doubles.
 * comp: 0..8 = Ex, Ey, Ez, Bx, By, Bz, Jx, Jy, Jz. */
int pic_get_field(pic_t* h, int comp, double* host_out);
int pic_set_field(pic_t* h, int comp, const double* host_in);

/* Particle access.  get: p->n is the capacity of the host arrays on entry and
 * the number of live particles on return (PIC_ERR_CAPACITY if too small; the
 * count is still returned).  set: replaces all particles; positions must lie
 * in the allowed x range (cells 2 .. nx-4 for open x), in [0, n) for
 * periodic axes and in [L, n - L) for y and z with absorbing layers of L
 * cells (PIC_ERR_ARG otherwise). */
int pic_get_particles(pic_t* h, pic_particles* p);
int pic_set_particles(pic_t* h, const pic_particles* p);

/* Reset the launch counters and switch per-group event timing on (1) or off
 * (0).  Timing adds two events per group and step; results via
 * pic_timing_read, which synchronises the stream. */
int pic_timing_start(pic_t* h, int enable);
int pic_timing_read(pic_t* h, pic_timing* out);

/* ---- checkpoint / resume ----
 * pic_save writes the dynamic state (fields in window-relative order,
 * particles, step, window shifts, the FP64 window accumulator, the push
 * count) to a binary file; pic_load reads it into a handle created with the
 * same grid, window, species and laser calls (PIC_ERR_ARG if the grid,
 * precision or ppc differ, PIC_ERR_STATE if the file is not a checkpoint).
 * Both synchronise the stream and stage the state through host memory. */
int pic_save(pic_t* h, const char* path);
int pic_load(pic_t* h, const char* path);

int pic_destroy(pic_t* h);

/* ---- diagnostics that allocate nothing ----
 * The paper has no counterpart to this call; it serves callers of the
 * library.  pic_diag may allocate device scratch (through cudaMalloc or the
 * pic_alloc hooks) the first time a diagnostic is requested.  Callers that
 * must not allocate after set-up -- a host framework with a fixed device
 * memory budget, a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device, code running inside another library's callbacks --
 * use pic_diag_noalloc instead: the kinds EX_LINEOUT, FIELD_ENERGY, CHARGE and
 * SPECTRUM, with the same arguments, units and results as pic_diag (other
 * kinds return PIC_ERR_ARG), and the reduction scratch in a fixed file-scope device array of
 * PIC_NOALLOC_MAX_LEN doubles (512 KiB, present on every GPU that loads the
 * library until it is unloaded).  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  Results longer than PIC_NOALLOC_MAX_LEN values (a
 * lineout of nx > 65536 cells, a spectrum of more bins) return PIC_ERR_ARG.
 * pic_create looks up the array's device address (cudaGetSymbolAddress) on
 * the device current at creation, the handle's device, and keeps it in the
 * handle; each call makes that device current while it runs and synchronises
 * the handle's stream before returning.  All calls share the array: each call
 * clears the part it uses, and calls that overlap on the GPU race on it. */
#define PIC_NOALLOC_MAX_LEN 65536
int pic_diag_noalloc(pic_t* h, int kind, double* out, size_t len, const pic_diag_args* a);

/* ---- tile shape and its autotuner ----
 * Particles are kept sorted by cell tile; one CTA works on one tile with its
 * E/B halo and J tile in shared memory.  pic_set_tiles picks the tile shape
 * (cells per axis; shrunk to the grid).  pic_autotune times a set of
 * candidate shapes on `steps` trial steps each, restoring the state after
 * every trial (the simulation does not advance), keeps the fastest and
 * returns it (tile_out[3], ms_out per step; either may be NULL).  With a
 * cache file (cache_path, else $PIC_AUTOTUNE_CACHE, else none) the choice is
 * read from / written to a JSON object keyed by precision, ppc and grid. */
int pic_set_tiles(pic_t* h, int tx, int ty, int tz);
int pic_autotune(pic_t* h, int steps, const char* cache_path, int* tile_out, double* ms_out);

/* ---- batched instances (a0 / density scans) ----
 * A batch borrows n FP32 handles with tile-sorted particles (they must
 * outlive it and may not be stepped on their own while batched; boundary
 * laser sources are not supported) and advances them together.  The step of
 * every member is captured once into a CUDA graph (members on forked streams
 * so that small instances run concurrently; every step parameter, including
 * the FP64 window accumulator and the ring origin, is read from device
 * memory), and each step is one graph launch.  Graphs are re-captured when a
 * member's particle buffers grow. */
int pic_batch_create(int n, pic_t* const* sims, pic_batch_t** out);
int pic_batch_step(pic_batch_t* b, int n);
/* graph launches and kernel launches issued by the batch since creation, and
 * the device time of the last pic_batch_step call (CUDA events on the batch
 * stream around its graph launches), in ms; any pointer may be NULL. */
int pic_batch_info(const pic_batch_t* b, int64_t* graph_launches, int64_t* kernel_launches,
                   double* last_step_ms);
int pic_batch_diag(pic_batch_t* b, int instance, int kind, double* out, size_t len,
                   const pic_diag_args* a);
int pic_batch_destroy(pic_batch_t* b);

#ifdef __cplusplus
}
#endif
#endif
