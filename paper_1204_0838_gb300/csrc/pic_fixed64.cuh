// pic_fixed64.cuh -- 64-bit fixed-point arithmetic of the FP64 push.
//
// The cubic gather (a 4x4x4 weighted sum per field component) and the
// Esirkepov deposit (products of shape-factor sums) of the FP64 push run as
// exact-range integer arithmetic instead of FP64 multiply-adds: on this GPU
// the integer multiply-add pipe retires 32x32->64-bit products many times
// faster than the FP64 pipe retires FMAs, and a 64-bit integer add into
// shared memory is a native 32-bit atomic plus a carry, where a double add is
// a compare-and-swap loop on the FP64 pipe.
//
// Formats:
// - a "value" x is an int64 with |x| < 2^62, in units of 2^-k for a scale k
//   chosen per tile (fields) or per tile and component (current);
// - a "weight" W is a non-negative int64 below 2^62 holding w 2^62 for
//   0 <= w < 1 (B-spline weights, Esirkepov factors), split as
//   W = hi 2^31 + lo with hi, lo < 2^31.
//
// x W / 2^62 = 2 x1 hi + x1 lo / 2^30 + x0 hi / 2^31 + x0 lo / 2^62, where
// x = x1 2^32 + x0 (x1 signed, 0 <= x0 < 2^32).  A FixAcc sums n such
// products in three 64-bit accumulators (one 32x32->64-bit multiply-add
// each), drops the last term (below 2 units per product) and rounds the two
// shifts, so the result is within 2n + 1 units of the exact sum, and a sum
// of zero products is exactly zero.  The bounds
// |x| < 2^60 and sum W <= 2^62 (weights that sum to one) keep every
// accumulator in range: |H| < 2^59, |M1| < 2^61, M2 < 2^63.
#pragma once

#include <cuda_runtime.h>

namespace pic {

struct W62 {
  int hi;  // W >> 31
  int lo;  // W & (2^31 - 1)
};

__device__ __forceinline__ W62 w62(long long W) { return {(int)(W >> 31), (int)(W & 0x7FFFFFFFLL)}; }

// round(v 2^k) for |v| 2^k < 2^62, from the bit pattern of v (integer
// instructions only; zero and subnormal v give 0).
__device__ __forceinline__ long long to_fixed(double v, int k) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = e - 1075 + k;  // |v| 2^k = m 2^sh, sh <= 9 by the caller's bound
  const int l = max(sh, 0), r = min(max(-sh, 0), 62);
  long long X = ((m << l) + ((1LL << r) >> 1)) >> r;
  X = e == 0 ? 0 : X;
  return b < 0 ? -X : X;
}

// 2^k as a double, for -1022 <= k <= 1023.
__device__ __forceinline__ double exp2i(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// x 2^-k as a double.
__device__ __forceinline__ double from_fixed(long long x, int k) { return __ll2double_rn(x) * exp2i(-k); }

struct FixAcc {
  long long H;
  long long M1;
  unsigned long long M2;
};

// Accumulator for a sum of products: the rounding offsets of the two shifts.
__device__ __forceinline__ FixAcc fix_init() { return {0LL, 1LL << 29, 1ULL << 30}; }

__device__ __forceinline__ void fix_mac(FixAcc& a, long long x, W62 w) {
  const int x1 = (int)(x >> 32);
  const unsigned x0 = (unsigned)x;
  a.H += (long long)x1 * w.hi;
  a.M1 += (long long)x1 * w.lo;
  a.M2 += (unsigned long long)x0 * (unsigned)w.hi;
}

__device__ __forceinline__ long long fix_result(const FixAcc& a) {
  return 2 * a.H + (a.M1 >> 30) + (long long)(a.M2 >> 31);
}

// x W / 2^62 for one product.
__device__ __forceinline__ long long fix_mul(long long x, W62 w) {
  FixAcc a = fix_init();
  fix_mac(a, x, w);
  return fix_result(a);
}

// fix_mac plus the mean of the dropped term over the weight's low bits,
// x0 / 2^32 units: the product's error is then within 2 units and has zero
// mean for weights whose low bits are spread, and x = 0 still adds nothing.
// Used where many products are summed (the current deposit), so that the
// rounding does not accumulate as a bias.
__device__ __forceinline__ void fix_mac_c(FixAcc& a, long long x, W62 w) {
  fix_mac(a, x, w);
  a.M2 += (unsigned)x >> 1;
}

// x W / 2^62 for one product, unbiased (fix_mac_c).  For single products
// the bounds allow |x| <= 2^62.
__device__ __forceinline__ long long fix_mul_c(long long x, W62 w) {
  FixAcc a = fix_init();
  fix_mac_c(a, x, w);
  return fix_result(a);
}

// Separable NA x NB x NC gather from a fixed-point staged tile (contracting
// z, then y, then x); the result has the tile's scale.
template <int NA, int NB, int NC>
__device__ __forceinline__ long long gather_fixed(const long long* __restrict__ s, int SY, int SZ, int bx, int by,
                                                  int bz, const W62* wx, const W62* wy, const W62* wz) {
  FixAcc ax = fix_init();
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    FixAcc ay = fix_init();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const long long* row = s + ((bx + a) * SY + (by + b)) * SZ + bz;
      FixAcc az = fix_init();
#pragma unroll
      for (int c = 0; c < NC; ++c) fix_mac(az, row[c], wz[c]);
      fix_mac(ay, fix_result(az), wy[b]);
    }
    fix_mac(ax, fix_result(ay), wx[a]);
  }
  return fix_result(ax);
}

__device__ __forceinline__ unsigned atom_add_u32_shared(unsigned* a, unsigned v) {
  unsigned old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "r"((unsigned)__cvta_generic_to_shared(a)), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ void red_add_u32_shared(unsigned* a, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(a)), "r"(v) : "memory");
}

// Exact 64-bit add of X into the shared word pair (hi, lo): the low word's
// add returns its old value, which gives the carry into the high word.  The
// pair holds the sum modulo 2^64 whatever the order of the adds.
__device__ __forceinline__ void add_fixed64(unsigned* hi, unsigned* lo, long long X) {
  const unsigned l = (unsigned)X, h = (unsigned)((unsigned long long)X >> 32);
  const unsigned old = atom_add_u32_shared(lo, l);
  red_add_u32_shared(hi, h + (old + l < old ? 1u : 0u));
}

}  // namespace pic
