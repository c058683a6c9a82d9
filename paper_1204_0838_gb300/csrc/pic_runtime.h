// pic_runtime.h -- the handle behind the opaque pic_t of include/pic.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pic.h"

namespace pic {

// One particle buffer: structure of arrays carved from one allocation.
struct PartBuf {
  void* base = nullptr;
  int* cell = nullptr;
  void* o[3] = {nullptr, nullptr, nullptr};
  void* u[3] = {nullptr, nullptr, nullptr};
  void* w = nullptr;
  uint32_t* id = nullptr;
};

}  // namespace pic

struct pic_t {
  // geometry and time (normalised units: c = eps0 = m_e = e = 1)
  int precision = PIC_FP64;
  int nx = 0, ny = 0, nz = 0;
  size_t ncell = 0;
  bool periodic_x = true;
  int solver = PIC_SOLVER_PERFECT;
  double dx = 0, dy = 0, dz = 0, dt = 0;
  double lambda0 = 0, k0 = 0, omega0 = 0, x0 = 0;
  uint64_t seed = 0;
  uint32_t flags = 0;
  long long max_particles = 0;
  double sm_a[3] = {0, 0, 0}, sm_b1[3] = {0, 0, 0}, sm_b2[3] = {0, 0, 0}, sm_g[3] = {0, 0, 0};
  int64_t step = 0;

  // device memory
  void* fields = nullptr;   // 9 component arrays of ncell values
  void* curl = nullptr;     // cached smoothed curl of E (3 arrays)
  bool curl_valid = false;  // false: recompute before the next step
  // transverse absorbing layers (0: y, z periodic): 8 compact memory-variable
  // arrays (4 of nx (2L+1) nz for y, 4 of nx ny (2L+1) for z) and the
  // per-index coefficients (a, b at nodes and half nodes for y, then z)
  int pml = 0;
  void* psi = nullptr;
  void* pml_coef = nullptr;
  // tile-sorted particles
  pic::Tiles tiles = {1, 1, 1, 1, 1, 1, 1};
  int* keys = nullptr;      // destination tile per particle
  int* tstart[2] = {nullptr, nullptr};  // tile starts of pb[0], pb[1]
  int* tcnt = nullptr;      // per-tile counts of the next buffer
  int* tfill = nullptr;     // per-tile fill counters of the scatter
  bool need_sort = false;   // particles not grouped by tile (after load/set)
  int tiles_alloc = 0;      // tile entries the tile arrays were sized for
  pic::DynState* d_dyn = nullptr;  // device-side step state (batched stepping)
  pic::PartBuf pb[2];       // current and compaction target
  int cur = 0;
  long long capacity = 0;
  int* d_ctrl = nullptr;    // [0], [1]: particle counts of pb[0], pb[1]; [2]: error bits
  int np_host = 0;
  long long pushed_host = 0;
  double* d_diag = nullptr;
  size_t diag_cap = 0;
  std::vector<void*> owned;
  pic_alloc alloc = {nullptr, nullptr, nullptr};
  bool has_alloc = false;

  // species (one electron-like species; ions immobile and implicit)
  bool has_species = false;
  long long ion_lab_lo = 0;  // first lab x cell loaded (the immobile ions start there)
  int ppc = 0, loading = 0, lat[3] = {1, 1, 1};
  double q = 0.0, m = 1.0;
  double* d_prof = nullptr;  // x (normalised) then density (n_c)
  int nprof = 0;

  // laser
  int laser_mode = 0;
  double las_a0 = 0, las_w0 = 0, las_tau = 0, las_k = 1, las_xf = 0, las_tpk = 0;

  // moving window: FP64 accumulator in cells, ring origin of the x slabs
  bool has_window = false;
  double win_v = 0, win_t0 = 0, win_frac = 0;
  int64_t shifts = 0;
  int origin = 0;

  // launch accounting and optional per-group event timing
  long long launches[4] = {0, 0, 0, 0};
  long long kernels = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;      // recycled events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pairs[4];
  unsigned long long* d_pushed = nullptr;  // device-side particle-step counter

  // device, streams, batching, errors
  int device = 0;                       // the CUDA device current at pic_create
  double* noalloc_scratch = nullptr;    // device address of pic_diag_noalloc's array on that device
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  bool batched = false;
  std::string err;
};
