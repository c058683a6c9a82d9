// pic_tiled.cuh -- tile-sorted particle kernels: particles are kept grouped
// by cell tile; one CTA stages its tile's E/B (plus the cubic-stencil halo)
// in shared memory, gathers, pushes, deposits J into a shared-memory tile and
// flushes it with global atomics.  Re-binning after each step is a counting
// sort by tile (count fused into the push, scan, scatter).
#pragma once

#include "pic_fixed64.cuh"
#include "pic_kernels.cuh"

namespace pic {

template <typename T>
__device__ __forceinline__ int tile_of(const Geom<T>& g, const Tiles& tl, int cx, int cy, int cz) {
  return ((cx / tl.tx) * tl.nty + cy / tl.ty) * tl.ntz + cz / tl.tz;
}

// Shared-memory extents: E/B staged over cells [c0-2, c0+t+2) per axis (the
// half-staggered cubic gather reaches c-2 .. c+2), J over [c0-2, c0+t+3)
// (the Esirkepov window of a particle that moves at most one cell reaches
// c-2 .. c+3).
__host__ __device__ __forceinline__ int stage_n(const Tiles& tl) { return (tl.tx + 4) * (tl.ty + 4) * (tl.tz + 4); }
__host__ __device__ __forceinline__ int jtile_n(const Tiles& tl) { return (tl.tx + 5) * (tl.ty + 5) * (tl.tz + 5); }

// FP32 particle layout of the push (FP64 keeps its own, see k_push_tiled):
// - cell rounds: the particles of a tile are taken in rounds, round r holding
//   the r-th particle of every occupied cell (ranks from a shared-memory cell
//   histogram), so that the lanes of a warp sit in distinct cells while
//   consecutive lanes stay on neighbouring cells.  Ranks from kRounds - 1 up
//   share the last round; the order is built for chunks of up to kOrderChunk
//   list entries.
// - fixed-point J tile: the deposit adds each contribution as an exact 64-bit
//   fixed-point integer split over two 32-bit words with native shared-memory
//   integer reductions (a float add on shared memory is a load plus a
//   compare-and-swap loop).  The scale is a power of two 2^s per tile and
//   component with 2^s <= 2^42 / B, B = |q jc| sum_p w_p over the tile: no
//   node of the tile can receive more than B in magnitude (each contribution
//   is bounded by |q w jc|), so the high word stays within 2^30 and the low
//   word (12 bits per contribution) within 2^32 for fewer than 2^20
//   contributions.  The resolution 2^-s is about 2^-42 B, far below the FP32
//   rounding of the contributions themselves, and the tile sum is exact and
//   independent of the order of the adds.
// FP64 push: the gather and the deposit run in 64-bit fixed point on the
// integer pipes (pic_fixed64.cuh).  The staged E/B become int64 at a power of
// two 2^sF per tile and component with max|F| 2^sF < 2^60, and the J tile
// holds exact 64-bit sums as (high, low) 32-bit word pairs at 2^s per tile
// and component with B 2^s < 2^62, B a bound on every node's sum taken from
// the particles' speeds before the push (j_scale): a cold or slow tile gets
// a fine scale, not one sized for moves of a whole cell.  The resolutions,
// 2^-60 of the tile's largest field and 2^-62 of B, are at the level of
// FP64 rounding at those scales, and the deposit's products round without
// bias, so that thousands of contributions to a node add up no drift.
constexpr int kRounds = 32;
constexpr int kOrderChunk = 2048;
constexpr int kFixedLoBits = 12;
constexpr int kFixedRange = 42;
constexpr int kFixed64Range = 60;   // staged fields: 4-term sums need |x| < 2^60
constexpr int kFixed64JRange = 62;  // J sums of single products
constexpr long long kThird62 = 1537228672809129301LL;  // round(2^62 / 3)
template <typename T>
struct LaneLayout {
  static constexpr bool cell_rounds = sizeof(T) == 4;
  static constexpr bool fixed_j = sizeof(T) == 4;   // FP32 J words: 12-bit low part
  static constexpr bool fixed64 = sizeof(T) == 8;   // FP64 fixed-point gather and J words
  // shared ints after the J tile: [0, 3) J scales, FP32 3 weight sum, FP64
  // [4, 10) field exponent maxima, [10, 16) field scales and [16, 18) the
  // sums behind the J bounds
  static constexpr int scale_ints = sizeof(T) == 8 ? 18 : 4;
};

template <typename T>
size_t tiled_smem_bytes(const Tiles& tl) {
  size_t b = sizeof(T) * 6 * (size_t)stage_n(tl) + 8 * 3 * (size_t)jtile_n(tl);
  if (LaneLayout<T>::cell_rounds) b += 4 * ((size_t)tl.tx * tl.ty * tl.tz + 3 * kRounds) + 2 * (size_t)kOrderChunk;
  return b + 4 * LaneLayout<T>::scale_ints;
}

// The J tile's scale exponent s for component threadIdx.x (< 3): B 2^s <
// 2^range for the bound B = 1.001 |q| S / (dt d_b d_c) on every node, where
// S bounds the sum over the tile's particles of |w| times the largest
// running sum of the deposit (FP32: S = sum_p |w|, a move of up to one cell;
// FP64: from each particle's speed bound).  1.001: margin over the float
// rounding of the sums.
template <typename T>
__device__ __forceinline__ int j_scale(const Geom<T>& g, T q, float S, int range) {
  const int c = threadIdx.x;
  const T jcc = c == 0 ? g.dt * g.dy * g.dz : (c == 1 ? g.dt * g.dx * g.dz : g.dt * g.dx * g.dy);
  const float B = 1.001f * fabsf((float)q) * S / (float)jcc;
  const int eb = ((__float_as_int(B) >> 23) & 255) - 127;  // B in [2^eb, 2^(eb+1))
  return B > 0.0f ? range - 1 - eb : 0;
}

// The shared-memory J tile of one CTA: [3][nJ] fixed-point word pairs over
// the cells [o3, o3 + t + 5) per axis, and the tile's scales.
template <typename T>
struct JTile {
  unsigned* hi;
  unsigned* lo;
  const int* s;   // J scale exponent per component
  const int* fs;  // FP64: staged field scale per component
  int nJ, JY, JZ;
};

__device__ __forceinline__ void red_u32(unsigned* a, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(a)), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated add of 1 to counter[key] for every lane with key >= 0;
// returns this lane's rank among the lanes that share its key, and the
// aggregated base offset through *base (only meaningful if want_base).
// All 32 lanes must call it.
__device__ __forceinline__ int warp_count(int* counter, int key, bool want_base, int* base) {
  const unsigned m = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int b = 0;
  if (lane == leader && key >= 0) b = want_base ? atomicAdd(counter + key, __popc(m)) : (atomicAdd(counter + key, __popc(m)), 0);
  b = __shfl_sync(0xffffffffu, b, leader);
  if (base) *base = b;
  return __popc(m & lanemask_lt());
}

// Gather one field component from the staged tile: NA x NB x NC separable
// sum (4 nodes along a node-centred axis; 4, or 5 with one zero weight, along
// a half-staggered one), contracting z first, then y, then x.
template <int NA, int NB, int NC, typename T>
__device__ __forceinline__ T gather_smem(const T* __restrict__ s, int SY, int SZ, int bx, int by, int bz,
                                         const T* wx, const T* wy, const T* wz) {
  T ax = T(0);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    T ay = T(0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const T* row = s + ((bx + a) * SY + (by + b)) * SZ + bz;
      T az = row[0] * wz[0];
#pragma unroll
      for (int c = 1; c < NC; ++c) az = fma(row[c], wz[c], az);
      ay = fma(az, wy[b], ay);
    }
    ax = fma(ay, wx[a], ax);
  }
  return ax;
}

// Comparisons of an offset against 0, 1/2 and 1.  In FP64 they are made on
// the bit pattern with integer instructions, off the slow FP64 pipe: for
// doubles of either sign the int64 view orders non-negative values like the
// values and makes every negative value (and -0) negative.
__device__ __forceinline__ bool lt_zero(double o) { return __double_as_longlong(o) < 0; }
__device__ __forceinline__ bool ge_one(double o) { return __double_as_longlong(o) >= 0x3FF0000000000000LL; }
__device__ __forceinline__ bool lt_half(double o) { return __double_as_longlong(o) < 0x3FE0000000000000LL; }
__device__ __forceinline__ bool lt_zero(float o) { return o < 0.0f; }
__device__ __forceinline__ bool ge_one(float o) { return o >= 1.0f; }
__device__ __forceinline__ bool lt_half(float o) { return o < 0.5f; }

// FP64 Esirkepov deposit of one particle into the fixed-point J tile: old
// cell lc (staged frame) with node weights wn, cell step dc and new offsets
// o1, charge times weight qw (0 for a particle that does not deposit).
template <typename T>
__device__ __forceinline__ void deposit_fixed64(const JTile<T>& jt, const T jc[3], const int lc[3], const int dc[3],
                                                const T wn[3][4], const T o1[3], double qw) {
  int lw[3], nw[3];
  // shape factors at 2^62, the factors A and bk and the running sums
  // P 2^s of the current in 64-bit fixed point, exact 64-bit tile sums
  long long S0i[3][5], DSi[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T w1[4];
    bspline3(o1[d], w1);
    long long wnI[4], w1i[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      wnI[k] = to_fixed(wn[d][k], 62);
      w1i[k] = to_fixed(w1[k], 62);
    }
    const int p0 = dc[d] < 0 ? 1 : 0, p1 = dc[d] > 0 ? 1 : 0;
    lw[d] = lc[d] - 1 - p0;
    nw[d] = dc[d] != 0 ? 5 : 4;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const long long a0 = p0 ? (m > 0 ? wnI[m > 0 ? m - 1 : 0] : 0LL) : (m < 4 ? wnI[m < 4 ? m : 3] : 0LL);
      const long long a1 = p1 ? (m > 0 ? w1i[m > 0 ? m - 1 : 0] : 0LL) : (m < 4 ? w1i[m < 4 ? m : 3] : 0LL);
      S0i[d][m] = a0;
      DSi[d][m] = a1 - a0;
    }
  }
  const W62 third62 = w62(kThird62);
  const int st[3] = {jt.JY * jt.JZ, jt.JZ, 1};
  const int base = lw[0] * st[0] + lw[1] * st[1] + lw[2] * st[2];
  // one copy of the component's deposit in a loop over the three components
  // (the unrolled copies overflow the instruction cache): the axes' factors
  // are selected into comp-relative arrays, m along comp, b along ab, c
  // along ac
#pragma unroll 1
  for (int comp = 0; comp < 3; ++comp) {
    const bool c0 = comp == 0, c1 = comp == 1;
    long long dsm[4], sb[5], db[5], sc[5], dsc[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (k < 4) dsm[k] = c0 ? DSi[0][k] : (c1 ? DSi[1][k] : DSi[2][k]);
      sb[k] = c0 ? S0i[1][k] : S0i[0][k];  // ab = 1 for comp 0, else 0
      db[k] = c0 ? DSi[1][k] : DSi[0][k];
      sc[k] = comp == 2 ? S0i[1][k] : S0i[2][k];  // ac = 1 for comp 2, else 2
      dsc[k] = comp == 2 ? DSi[1][k] : DSi[2][k];
    }
    // P 2^s = q w jc run 2^s, below 2^62 by the choice of the tile's scale
    // (|run| <= 3/4 |displacement| along comp)
    const double cfs = qw * (double)(c0 ? jc[0] : (c1 ? jc[1] : jc[2])) * exp2i(jt.s[comp] - 62);
    long long Pi[4];
    long long run = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      run += dsm[m];
      Pi[m] = to_fixed(__ll2double_rn(run) * cfs, 0);
    }
    // ak = (S0 + S1)/2, bk = (S0 + 2 S1)/6 (the sum S0 + 2 S1 <= 2^63 is
    // formed unsigned)
    W62 akW[5], bkW[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      akW[c] = w62((2 * sc[c] + dsc[c]) >> 1);
      const unsigned long long t2 = 3ull * (unsigned long long)sc[c] + 2ull * (unsigned long long)dsc[c];
      bkW[c] = w62(fix_mul_c((long long)(t2 >> 1), third62));
    }
    const int base0 = comp * jt.nJ + base;
    const int sm_ = c0 ? st[0] : (c1 ? st[1] : 1), sb_ = c0 ? st[1] : st[0], sc_ = comp == 2 ? st[1] : 1;
    const int nm = (c0 ? nw[0] : (c1 ? nw[1] : nw[2])) - 1, nb = c0 ? nw[1] : nw[0], nc = comp == 2 ? nw[1] : nw[2];
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (b < nb) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          if (c < nc) {
            FixAcc acc = fix_init();
            fix_mac_c(acc, sb[b], akW[c]);
            fix_mac_c(acc, db[b], bkW[c]);
            const W62 Aw = w62(max(fix_result(acc), 0LL));  // A >= 0; clamps a rounding below zero
#pragma unroll
            for (int m = 0; m < 4; ++m)
              if (m < nm) {
                const int idx = base0 + m * sm_ + b * sb_ + c * sc_;
                add_fixed64(jt.hi + idx, jt.lo + idx, fix_mul_c(Pi[m], Aw));
              }
          }
        }
      }
    }
  }
}

// Gather, Boris push, move and Esirkepov deposit of particle pi of the tile
// whose staged origin is o3; returns its destination tile key (-1: absorbed).
template <typename T>
__device__ __forceinline__ int push_particle(const Geom<T>& g, const Tiles& tl, const Parts<T>& p, int pi,
                                             const int o3[3], const T* __restrict__ sF, int nS, int SY, int SZ,
                                             const JTile<T>& jt, T h, T q, int origin_after, int xlo, int xhi,
                                             int* __restrict__ keys, int* err) {
  const int N[3] = {g.nx, g.ny, g.nz};
  const T dtd[3] = {g.dt / g.dx, g.dt / g.dy, g.dt / g.dz};
  const T jc[3] = {T(-1) / (g.dt * g.dy * g.dz), T(-1) / (g.dt * g.dx * g.dz), T(-1) / (g.dt * g.dx * g.dy)};
  const T third = T(1) / T(3);
  const int cell = p.cell[pi];
  int c0[3];
  c0[0] = cell / g.nyz;
  const int rem = cell - c0[0] * g.nyz;
  c0[1] = rem / g.nz;
  c0[2] = rem - c0[1] * g.nz;
  int lc[3];
  T o0[3], u[3];
  const int text[3] = {tl.tx, tl.ty, tl.tz};
  bool inside = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lc[d] = c0[d] - o3[d];  // in [2, t+2) for a particle of this tile
    inside = inside && lc[d] >= 2 && lc[d] < text[d] + 2;
    o0[d] = p.o[d][pi];
    u[d] = p.u[d][pi];
  }
  if (!inside) {  // never expected: keeps every shared-memory index in range
    atomicOr(err, 4);
    keys[pi] = -1;
    return -1;
  }
  T wn[3][4];
  int bn[3];
  T E[3], B[3];
  T wh[3][4];
  int bh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    bspline3(o0[d], wn[d]);
    const bool lo = lt_half(o0[d]);
    bspline3(lo ? o0[d] + T(0.5) : o0[d] - T(0.5), wh[d]);
    bn[d] = lc[d] - 1;
    bh[d] = lc[d] - (lo ? 2 : 1);
  }
  if constexpr (LaneLayout<T>::fixed64) {
    // FP64: the weights at 2^62 on the fixed-point staged tile
    const long long* sI = reinterpret_cast<const long long*>(sF);
    W62 Wn[3][4], Wh[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Wn[d][k] = w62(to_fixed(wn[d][k], 62));
        Wh[d][k] = w62(to_fixed(wh[d][k], 62));
      }
    // one copy of the 4x4x4 gather in a loop over the six components (the
    // unrolled six copies overflow the instruction cache); bit d of the
    // component's mask = half-staggered along axis d (Ex x, Ey y, Ez z,
    // Bx yz, By xz, Bz xy)
#pragma unroll 1
    for (int comp = 0; comp < 6; ++comp) {
      const int hm = (0x356421 >> (4 * comp)) & 7;
      W62 wx[4], wy[4], wz[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        wx[k] = (hm & 1) ? Wh[0][k] : Wn[0][k];
        wy[k] = (hm & 2) ? Wh[1][k] : Wn[1][k];
        wz[k] = (hm & 4) ? Wh[2][k] : Wn[2][k];
      }
      const double v = from_fixed(gather_fixed<4, 4, 4>(sI + comp * nS, SY, SZ, (hm & 1) ? bh[0] : bn[0],
                                                        (hm & 2) ? bh[1] : bn[1], (hm & 4) ? bh[2] : bn[2], wx, wy, wz),
                                  jt.fs[comp]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (comp == k) E[k] = v;
        if (comp == k + 3) B[k] = v;
      }
    }
  } else {
    E[0] = gather_smem<4, 4, 4>(sF + 0 * nS, SY, SZ, bh[0], bn[1], bn[2], wh[0], wn[1], wn[2]);
    E[1] = gather_smem<4, 4, 4>(sF + 1 * nS, SY, SZ, bn[0], bh[1], bn[2], wn[0], wh[1], wn[2]);
    E[2] = gather_smem<4, 4, 4>(sF + 2 * nS, SY, SZ, bn[0], bn[1], bh[2], wn[0], wn[1], wh[2]);
    B[0] = gather_smem<4, 4, 4>(sF + 3 * nS, SY, SZ, bn[0], bh[1], bh[2], wn[0], wh[1], wh[2]);
    B[1] = gather_smem<4, 4, 4>(sF + 4 * nS, SY, SZ, bh[0], bn[1], bh[2], wh[0], wn[1], wh[2]);
    B[2] = gather_smem<4, 4, 4>(sF + 5 * nS, SY, SZ, bh[0], bh[1], bn[2], wh[0], wh[1], wn[2]);
  }

  // relativistic Boris push
  T um[3], tv[3], sv[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) um[d] = u[d] + h * E[d];
  const T hg = h * rsqrt(T(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);  // h / gamma-
#pragma unroll
  for (int d = 0; d < 3; ++d) tv[d] = hg * B[d];
  const T s2 = T(2) / (T(1) + tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) sv[d] = s2 * tv[d];
  const T px = um[0] + (um[1] * tv[2] - um[2] * tv[1]);
  const T py = um[1] + (um[2] * tv[0] - um[0] * tv[2]);
  const T pz = um[2] + (um[0] * tv[1] - um[1] * tv[0]);
  u[0] = um[0] + (py * sv[2] - pz * sv[1]) + h * E[0];
  u[1] = um[1] + (pz * sv[0] - px * sv[2]) + h * E[1];
  u[2] = um[2] + (px * sv[1] - py * sv[0]) + h * E[2];
  T ig = rsqrt(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);  // 1 / gamma
  // a non-finite momentum (a blown-up state) is reported and the particle
  // absorbed without moving or depositing, so that the fields stay finite
  const bool bad = !(ig > T(0));
  if (bad) {
    atomicOr(err, 8);
    ig = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = T(0);
  }

  // position update (cell + offset), |move| < 1 cell per axis
  T o1[3];
  int dc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T o = o0[d] + dtd[d] * u[d] * ig;
    int k = 0;
    if (lt_zero(o)) {
      o += T(1);
      k = -1;
    } else if (ge_one(o)) {
      o -= T(1);
      k = 1;
    }
    if (ge_one(o)) {
      o = T(0);
      k += 1;
    }
    o1[d] = o;
    dc[d] = k;
  }

  // Esirkepov deposit into the shared J tile: 5-node window per axis
  // starting at c0 - 1 + min(dc, 0); S0 on window nodes p0..p0+3, S1 on
  // p1..p1+3.  Wx(i,j,k) = DSx(i) A(j,k) with A = S0y S0z + DSy S0z/2 +
  // S0y DSz/2 + DSy DSz/3 = S0y (S0z + DSz/2) + DSy (S0z/2 + DSz/3).
  // A particle that stays in its cell along an axis has a 4-node support
  // there (node 5 of the window carries nothing): nw = 4 or 5 nodes, and
  // the running sum along the current's own axis vanishes on its last
  // node, so only nw - 1 current values are nonzero.
  if constexpr (LaneLayout<T>::fixed64) {
    deposit_fixed64(jt, jc, lc, dc, wn, o1, bad ? 0.0 : (double)q * (double)p.w[pi]);
  } else {
    int lw[3], nw[3];
    T S0[3][5], DS[3][5];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T w1[4];
      bspline3(o1[d], w1);
      const int p0 = dc[d] < 0 ? 1 : 0, p1 = dc[d] > 0 ? 1 : 0;
      lw[d] = lc[d] - 1 - p0;
      nw[d] = dc[d] != 0 ? 5 : 4;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const T a0 = p0 ? (m > 0 ? wn[d][m > 0 ? m - 1 : 0] : T(0)) : (m < 4 ? wn[d][m < 4 ? m : 3] : T(0));
        const T a1 = p1 ? (m > 0 ? w1[m > 0 ? m - 1 : 0] : T(0)) : (m < 4 ? w1[m < 4 ? m : 3] : T(0));
        S0[d][m] = a0;
        DS[d][m] = a1 - a0;
      }
    }
    const T qw = bad ? T(0) : q * p.w[pi];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      // axis `comp` carries the running sum; (b, c) are the other two axes
      const int ab = comp == 0 ? 1 : 0, ac = comp == 2 ? 1 : 2;
      T P[4];
      T run = T(0);
      const T cf = qw * jc[comp];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        run += DS[comp][m];
        P[m] = cf * run;
      }
      T ak[5], bk[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        ak[m] = S0[ac][m] + T(0.5) * DS[ac][m];
        bk[m] = T(0.5) * S0[ac][m] + third * DS[ac][m];
      }
      // strides of the three axes in the J tile; (m, b, c) walk (comp, ab, ac)
      const int st[3] = {jt.JY * jt.JZ, jt.JZ, 1};
      const int base0 = comp * jt.nJ + lw[0] * st[0] + lw[1] * st[1] + lw[2] * st[2];
      const int sm_ = st[comp], sb_ = st[ab], sc_ = st[ac];
      const int nm = nw[comp] - 1, nb = nw[ab], nc = nw[ac];
      // P[m] as integers with a per-particle exponent kp (|P 2^kp| in
      // [2^23, 2^24): the float's 24 significant bits, exactly), A with 2^30
      // (exact for A >= 2^-7, within 2^-31 below); their product carries
      // 2^(kp + 30), shifted to the tile's 2^s with rounding to nearest
      const float pmax = fmaxf(fmaxf(fabsf(P[0]), fabsf(P[1])), fmaxf(fabsf(P[2]), fabsf(P[3])));
      const int ep = ((__float_as_int(pmax) >> 23) & 255) - 127;
      if (ep > -100) {  // else the particle carries no current along this axis (or below 2^-100)
        const int kp = 23 - ep;
        const float sp = __int_as_float((127 + kp) << 23);
        int Pi[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) Pi[m] = __float2int_rn(P[m] * sp);
        const int sh = min(max(kp + 30 - jt.s[comp], 0), 62);
        const long long half = (1LL << sh) >> 1;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          if (b < nb) {
            const T sb = S0[ab][b], db = DS[ab][b];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
              if (c < nc) {
                const int Ai = __float2int_rn((sb * ak[c] + db * bk[c]) * 1073741824.0f);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                  if (m < nm) {
                    const long long X = ((long long)Pi[m] * Ai + half) >> sh;
                    const int idx = base0 + m * sm_ + b * sb_ + c * sc_;
                    red_u32(jt.hi + idx, (unsigned)(X >> kFixedLoBits));
                    red_u32(jt.lo + idx, (unsigned)X & ((1u << kFixedLoBits) - 1u));
                  }
              }
            }
          }
        }
      }
    }
  }

  // store in place; the key is the destination tile (or -1: absorbed)
  const int n0 = wrapi(c0[0] + dc[0], N[0]);
  const int n1 = wrapi(c0[1] + dc[1], N[1]);
  const int n2 = wrapi(c0[2] + dc[2], N[2]);
  p.cell[pi] = n0 * g.nyz + n1 * g.nz + n2;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    p.o[d][pi] = o1[d];
    p.u[d][pi] = u[d];
  }
  int key = tile_of(g, tl, n0, n1, n2);
  if (!g.periodic_x) {
    int rel = n0 - origin_after;
    if (rel < 0) rel += g.nx;
    if (rel < xlo || rel > xhi) key = -1;
  }
  // absorbing layers: a particle that leaves the y, z cells [L, n - L) is absorbed
  if (g.pml && (n1 < g.pml || n1 >= g.ny - g.pml || n2 < g.pml || n2 >= g.nz - g.pml)) key = -1;
  if (bad) key = -1;
  keys[pi] = key;
  return key;
}

// Threads per CTA of the push: FP32 256 (the cell-round order is built for
// 256 threads; two CTAs of about 100 KB of shared memory per SM); FP64 512
// (one CTA per SM, the FP64 tile takes most of the shared memory; 16 warps
// at 128 registers hide the integer and fetch latencies better than 8 at
// 254, despite a few hundred bytes of spills).
template <typename T>
constexpr int push_threads() {
  return sizeof(T) == 8 ? 512 : 256;
}

// One CTA per tile.  keys[p] receives the particle's tile after the move (or
// -1 when it leaves the open-x range once the window has moved to
// origin_after); cnt_next[tile] counts the particles each tile will hold.
// blockDim.x is push_threads<T>().
template <typename T>
__global__ void __launch_bounds__(push_threads<T>(), sizeof(T) == 8 ? 1 : 2) k_push_tiled(Geom<T> g, Tiles tl, Fields<T> f, Parts<T> p,
                                                   const int* __restrict__ tstart, int capacity,
                                                   int* __restrict__ keys, int* __restrict__ cnt_next,
                                                   T h, T q, int origin_after, int xlo, int xhi,
                                                   unsigned long long* pushed, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  if (g.dyn) origin_after = g.dyn->origin_after;
  const int t = blockIdx.x;
  const int pbeg = min(tstart[t], capacity), pend = min(tstart[t + 1], capacity);
  if (pbeg >= pend) return;
  const int tzi = t % tl.ntz, rest = t / tl.ntz;
  const int tyi = rest % tl.nty, txi = rest / tl.nty;
  const int o3[3] = {txi * tl.tx - 2, tyi * tl.ty - 2, tzi * tl.tz - 2};  // staged origin (cells)
  const int SX = tl.tx + 4, SY = tl.ty + 4, SZ = tl.tz + 4;
  const int nS = SX * SY * SZ, nJ = jtile_n(tl);
  T* sF = sm;
  JTile<T> jt;
  jt.nJ = nJ;
  jt.JY = tl.ty + 5;
  jt.JZ = tl.tz + 5;
  jt.hi = reinterpret_cast<unsigned*>(sm + 6 * nS);
  jt.lo = jt.hi + 3 * nJ;
  int* sexp = reinterpret_cast<int*>(jt.lo + 3 * nJ);
  jt.s = sexp;
  jt.fs = sexp + 10;
  unsigned char* after_j = reinterpret_cast<unsigned char*>(sexp + LaneLayout<T>::scale_ints);

  // stage E and B (wrapped storage indices; see the ring note in pic_device.cuh);
  // FP64 also takes the largest exponent of each component
  int emax[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nS; i += blockDim.x) {
    const int lz = i % SZ, r = i / SZ;
    const int ly = r % SY, lx = r / SY;
    const size_t gi = (size_t)wrapi(o3[0] + lx, g.nx) * g.nyz + (size_t)wrapi(o3[1] + ly, g.ny) * g.nz +
                      wrapi(o3[2] + lz, g.nz);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T v = f.c[c][gi];
      sF[c * nS + i] = v;
      if constexpr (LaneLayout<T>::fixed64)
        emax[c] = max(emax[c], (int)((__double_as_longlong(v) >> 52) & 0x7FF));
    }
  }
  if (threadIdx.x < LaneLayout<T>::scale_ints) sexp[threadIdx.x] = 0;
  __syncthreads();
  if constexpr (LaneLayout<T>::fixed64) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const unsigned e = __reduce_max_sync(0xffffffffu, (unsigned)emax[c]);
      if ((threadIdx.x & 31) == 0) atomicMax(sexp + 4 + c, (int)e);
    }
    __syncthreads();
    // bound on each particle's speed after the push: |u'| <= |u| + 2 |h| |E|
    // (the Boris rotation keeps |u|), |E| <= sqrt 3 max_c |E_c| < sqrt 3
    // 2^(emax - 1022); sums of |w| min(1, bound) and of |w| over the tile
    const int eE = max(max(sexp[4], sexp[5]), sexp[6]);
    const float kick = eE == 0 ? 0.0f : ldexpf(3.4642f * fabsf((float)h), eE - 1022);
    float su = 0.0f, sw = 0.0f;
    for (int k = threadIdx.x; k < pend - pbeg; k += blockDim.x) {
      const float wa = fabsf((float)p.w[pbeg + k]);
      const float ux = (float)p.u[0][pbeg + k], uy = (float)p.u[1][pbeg + k], uz = (float)p.u[2][pbeg + k];
      su += wa * fminf(1.0f, sqrtf(ux * ux + uy * uy + uz * uz) + kick);
      sw += wa;
    }
    for (int o = 16; o > 0; o >>= 1) {
      su += __shfl_down_sync(0xffffffffu, su, o);
      sw += __shfl_down_sync(0xffffffffu, sw, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(reinterpret_cast<float*>(sexp + 16), su);
      atomicAdd(reinterpret_cast<float*>(sexp + 17), sw);
    }
  }
  for (int i = threadIdx.x; i < 6 * nJ; i += blockDim.x) jt.hi[i] = 0u;
  if constexpr (!LaneLayout<T>::fixed64) {
    // the scale of the fixed-point J tile: B = |q jc| sum_p w_p bounds every node
    float ws = 0.0f;
    for (int k = threadIdx.x; k < pend - pbeg; k += blockDim.x) ws += fabsf((float)p.w[pbeg + k]);
    for (int o = 16; o > 0; o >>= 1) ws += __shfl_down_sync(0xffffffffu, ws, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(reinterpret_cast<float*>(sexp + 3), ws);
  }
  __syncthreads();
  if constexpr (!LaneLayout<T>::fixed64) {
    if (threadIdx.x < 3) sexp[threadIdx.x] = j_scale(g, q, __int_as_float(sexp[3]), kFixedRange);
  } else {
    // a particle moves at most dt/d |u'| cells along an axis, and a running
    // sum of the deposit changes by at most 3/4 of the move (the slope bound
    // of the cubic spline's partial sums); 2^-20 covers the rounding
    if (threadIdx.x < 3) {
      const int c = threadIdx.x;
      const float dtd = (float)(g.dt / (c == 0 ? g.dx : (c == 1 ? g.dy : g.dz)));
      const float S = 0.75f * (dtd * __int_as_float(sexp[16]) + 0x1p-20f * __int_as_float(sexp[17]));
      sexp[c] = j_scale(g, q, S, kFixed64JRange);
    }
    // staged fields to int64 at 2^sF, max|F| 2^sF < 2^60 (an all-zero
    // component takes sF = 1000; a non-finite value reports a numeric error)
    int sfc[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int e = sexp[4 + c];
      sfc[c] = e == 0 ? 1000 : min(kFixed64Range - 1 - (e - 1023), 1000);
      if (e == 0x7FF && threadIdx.x == 0) atomicOr(err, 8);
    }
    if (threadIdx.x < 6) sexp[10 + threadIdx.x] = sfc[threadIdx.x];
    long long* sI = reinterpret_cast<long long*>(sF);
#pragma unroll
    for (int c = 0; c < 6; ++c)
      for (int i = threadIdx.x; i < nS; i += blockDim.x) sI[c * nS + i] = to_fixed(sF[c * nS + i], sfc[c]);
  }
  if (threadIdx.x == 0) atomicAdd(pushed, (unsigned long long)(pend - pbeg));
  // the fixed-point low words hold up to 2^20 contributions each
  if (LaneLayout<T>::fixed_j && threadIdx.x == 0 && pend - pbeg >= (1 << 20)) atomicOr(err, 16);
  __syncthreads();
  const int ntile = pend - pbeg;

  if constexpr (LaneLayout<T>::cell_rounds) {
    // cell-round order, chunk by chunk of the tile's list
    const int ncell_t = tl.tx * tl.ty * tl.tz;
    int* hist = reinterpret_cast<int*>(after_j);
    int* rtot = hist + ncell_t;
    int* rbase = rtot + kRounds;
    int* rfill = rbase + kRounds;
    unsigned short* order = reinterpret_cast<unsigned short*>(rfill + kRounds);
    constexpr int kPer = kOrderChunk / 256;
    for (int ch0 = 0; ch0 < ntile; ch0 += kOrderChunk) {
      const int nch = min(kOrderChunk, ntile - ch0);
      for (int i = threadIdx.x; i < ncell_t; i += blockDim.x) hist[i] = 0;
      if (threadIdx.x < 3 * kRounds) rtot[threadIdx.x] = 0;
      __syncthreads();
      int rk[kPer];
#pragma unroll
      for (int it = 0; it < kPer; ++it) {
        const int k = it * 256 + threadIdx.x;
        int r = -1;
        if (k < nch) {
          const int cell = p.cell[pbeg + ch0 + k];
          const int cx = cell / g.nyz, rem = cell - cx * g.nyz;
          const int cy = rem / g.nz, cz = rem - cy * g.nz;
          const int lx = cx - o3[0] - 2, ly = cy - o3[1] - 2, lz = cz - o3[2] - 2;
          const bool in = lx >= 0 && lx < tl.tx && ly >= 0 && ly < tl.ty && lz >= 0 && lz < tl.tz;
          const int lcell = in ? (lx * tl.ty + ly) * tl.tz + lz : 0;  // a stray particle (caught later) ranks in cell 0
          r = min(atomicAdd(hist + lcell, 1), kRounds - 1);
        }
        rk[it] = r;
        warp_count(rtot, r, false, nullptr);
      }
      __syncthreads();
      if (threadIdx.x < 32) {  // exclusive scan of the round sizes (kRounds = 32)
        const int v = rtot[threadIdx.x];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int n = __shfl_up_sync(0xffffffffu, incl, o);
          if (threadIdx.x >= o) incl += n;
        }
        rbase[threadIdx.x] = incl - v;
      }
      __syncthreads();
#pragma unroll
      for (int it = 0; it < kPer; ++it) {
        int off;
        const int rank = warp_count(rfill, rk[it], true, &off);
        if (rk[it] >= 0) order[rbase[rk[it]] + off + rank] = (unsigned short)(it * 256 + threadIdx.x);
      }
      __syncthreads();
      for (int base = 0; base < nch; base += blockDim.x) {
        const int k = base + threadIdx.x;
        int key = -2;
        if (k < nch)
          key = push_particle(g, tl, p, pbeg + ch0 + order[k], o3, sF, nS, SY, SZ, jt, h, q, origin_after,
                              xlo, xhi, keys, err);
        warp_count(cnt_next, key, false, nullptr);
      }
      __syncthreads();  // the next chunk reuses the histogram and the order
    }
  } else {
    // FP64: the lanes of a warp take particles mrow apart in the list, which
    // spreads the many particles of a dense cell (bubble walls) over warps.
    const int mrow = (ntile + 31) >> 5;
    const int nloop = 32 * mrow;
    for (int base = 0; base < nloop; base += blockDim.x) {
      const int lane = threadIdx.x & 31;
      const int kk = base + threadIdx.x;
      const int loc = lane * mrow + (kk >> 5);
      int key = -2;
      if (kk < nloop && loc < ntile)
        key = push_particle(g, tl, p, pbeg + loc, o3, sF, nS, SY, SZ, jt, h, q, origin_after, xlo, xhi, keys,
                            err);
      warp_count(cnt_next, key, false, nullptr);
    }
    __syncthreads();
  }

  // flush the J tile (cells [o3, o3 + t + 5) per axis, wrapped)
  for (int i = threadIdx.x; i < 3 * nJ; i += blockDim.x) {
    const int comp = i / nJ, li = i - comp * nJ;
    T v;
    if constexpr (LaneLayout<T>::fixed64) {
      const long long X = (long long)(((unsigned long long)jt.hi[i] << 32) | jt.lo[i]);
      if (X == 0) continue;
      v = from_fixed(X, sexp[comp]);
    } else {
      const long long X = (long long)(int)jt.hi[i] * (1LL << kFixedLoBits) + (long long)jt.lo[i];
      if (X == 0) continue;
      v = ldexpf((float)X, -sexp[comp]);
    }
    const int lz = li % jt.JZ, r = li / jt.JZ;
    const int ly = r % jt.JY, lx = r / jt.JY;
    const size_t gi = (size_t)wrapi(o3[0] + lx, g.nx) * g.nyz + (size_t)wrapi(o3[1] + ly, g.ny) * g.nz +
                      wrapi(o3[2] + lz, g.nz);
    atomicAdd(f.c[JX + comp] + gi, v);
  }
}

// Keys from the current cells (used after loading or set_particles).
template <typename T>
__global__ void k_keys(Geom<T> g, Tiles tl, Parts<T> p, const int* __restrict__ d_np, int* keys, int* cnt) {
  const int n = *d_np;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int pi = base + threadIdx.x;
    int key = -2;
    if (pi < n) {
      const int cell = p.cell[pi];
      const int cx = cell / g.nyz, r = cell - cx * g.nyz;
      key = tile_of(g, tl, cx, r / g.nz, r - (r / g.nz) * g.nz);
      keys[pi] = key;
    }
    warp_count(cnt, key, false, nullptr);
  }
}

// Exclusive scan of the tile counts into tile starts (single CTA of 1024
// threads, contiguous chunk per thread).  Starts are clamped to the capacity;
// a total above it sets the capacity error bit.
__global__ void __launch_bounds__(1024) k_scan_tiles(const int* __restrict__ cnt, int* __restrict__ tstart, int n,
                                                    int* d_np_out, int capacity, int* err) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int b = min(tid * chunk, n), e = min(b + chunk, n);
  long long s = 0;
  for (int i = b; i < e; ++i) s += cnt[i];
  part[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    long long v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long run = part[tid] - s;  // exclusive prefix of this chunk
  for (int i = b; i < e; ++i) {
    tstart[i] = (int)min(run, (long long)capacity);
    run += cnt[i];
  }
  if (tid == 1023) {
    const long long total = part[1023];
    tstart[n] = (int)min(total, (long long)capacity);
    *d_np_out = (int)min(total, (long long)capacity);
    if (total > capacity) atomicOr(err, 1);
  }
}

// Scatter the kept particles into their tiles of the other buffer.
template <typename T>
__global__ void k_scatter(Parts<T> src, const int* __restrict__ keys, const int* __restrict__ d_np_src,
                          Parts<T> dst, const int* __restrict__ tstart, int* fill, int* err) {
  const int n = *d_np_src;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int pi = base + threadIdx.x;
    const int key = pi < n ? keys[pi] : -2;
    // read the record before reserving its slot, so that these loads overlap
    // the reservation's atomic round trip instead of following it
    int cell = 0;
    T o[3] = {T(0), T(0), T(0)}, u[3] = {T(0), T(0), T(0)}, w = T(0);
    uint32_t id = 0;
    if (key >= 0) {
      cell = src.cell[pi];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        o[d] = src.o[d][pi];
        u[d] = src.u[d][pi];
      }
      w = src.w[pi];
      if (src.id) id = src.id[pi];
    }
    int off;
    const int rank = warp_count(fill, key, true, &off);
    if (key >= 0) {
      const int slot = tstart[key] + off + rank;
      if (slot >= tstart[key + 1]) {
        atomicOr(err, 2);
        continue;
      }
      dst.cell[slot] = cell;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dst.o[d][slot] = o[d];
        dst.u[d][slot] = u[d];
      }
      dst.w[slot] = w;
      if (dst.id) dst.id[slot] = id;
    }
  }
}

// Window injection into a tile-sorted buffer: pass 0 counts per tile into
// cnt, pass 1 places the particles with the tile fill counters.  The draws
// are the same counter-based SplitMix64 keys as plain loading, so both
// passes regenerate identical particles.
template <typename T>
__global__ void k_inject_tiled(Geom<T> g, Tiles tl, Parts<T> p, LoadSpec L, int pass, int* cnt,
                               const int* __restrict__ tstart, int* fill, int* err) {
  if (!dyn_prologue(g)) return;
  if (g.dyn) L.shifts = g.dyn->shifts;
  const long long nslot = (long long)(L.hi - L.lo + 1) * g.nyz * L.ppc;
  for (long long q0 = (long long)blockIdx.x * blockDim.x; q0 < nslot; q0 += (long long)gridDim.x * blockDim.x) {
    const long long qq = q0 + threadIdx.x;
    int key = -2;
    double o[3] = {0, 0, 0}, n = 0;
    int sx = 0, j = 0, k = 0, sl = 0;
    unsigned long long cell = 0;
    if (qq < nslot) {
      sl = (int)(qq % L.ppc);
      const long long c = qq / L.ppc;
      const int r = (int)(c % g.nyz);
      const int ci = L.lo + (int)(c / g.nyz);
      j = r / g.nz;
      k = r - j * g.nz;
      const long long lab = L.shifts + ci;
      cell = ((unsigned long long)lab * g.ny + j) * g.nz + k;
      const unsigned long long ctr = (cell * L.ppc + sl) * 3ull;
      double rr[3];
      for (int d = 0; d < 3; ++d) rr[d] = unit_uniform(L.seed, ctr + d);
      if (L.lattice) {
        const int ix = sl / (L.ns[1] * L.ns[2]), iy = (sl / L.ns[2]) % L.ns[1], iz = sl % L.ns[2];
        o[0] = (ix + rr[0]) / L.ns[0];
        o[1] = (iy + rr[1]) / L.ns[1];
        o[2] = (iz + rr[2]) / L.ns[2];
      } else {
        o[0] = rr[0];
        o[1] = rr[1];
        o[2] = rr[2];
      }
      const bool inner = j >= L.pml && j < g.ny - L.pml && k >= L.pml && k < g.nz - L.pml;
      n = inner ? profile_at(L.px, L.pn, L.np, L.x0 + ((double)lab + o[0]) * L.dx) : 0.0;
      sx = slab_of(g, ci);
      if (n > 0.0) key = tile_of(g, tl, sx, j, k);
    }
    if (pass == 0) {
      warp_count(cnt, key, false, nullptr);
      continue;
    }
    int off;
    const int rank = warp_count(fill, key, true, &off);
    if (key >= 0) {
      const int slot = tstart[key] + off + rank;
      if (slot >= tstart[key + 1]) {
        atomicOr(err, 2);
        continue;
      }
      p.cell[slot] = sx * g.nyz + j * g.nz + k;
      for (int d = 0; d < 3; ++d) {
        T od = (T)o[d];
        if (od >= T(1)) od = one_below<T>();
        p.o[d][slot] = od;
        p.u[d][slot] = T(0);
      }
      p.w[slot] = (T)(n * L.dVppc);
      if (p.id) p.id[slot] = (uint32_t)(cell * L.ppc + sl);
    }
  }
}

}  // namespace pic
