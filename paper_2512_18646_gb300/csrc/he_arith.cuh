// he_arith.cuh - exact modular arithmetic on 64-bit words for primes q < 2^62.
//
// Published methods, written for this library:
//  - Barrett reduction of a 128-bit value with mu = floor(2^128 / q)
//    (Barrett, CRYPTO 1986), quotient estimate from the high words;
//  - Shoup's multiplication by a fixed operand w with w' = floor(w 2^64 / q)
//    (Shoup, NTL), lazy result in [0, 2q);
//  - Harvey's lazy butterflies (Harvey, "Faster arithmetic for number-theoretic
//    transforms", 2014): values kept in [0, 4q) through the forward transform
//    and [0, 2q) through the inverse, which needs 4q < 2^64.
// All functions are __host__ __device__ so they can be checked on the CPU.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define HE_HD __host__ __device__ __forceinline__
#else
#define HE_HD inline
#endif

namespace he {

typedef uint64_t u64;
typedef uint32_t u32;

HE_HD u64 mulhi64(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (u64)(((unsigned __int128)a * b) >> 64);
#endif
}

// Full 64 x 64 -> 128-bit product from four 32 x 32 -> 64-bit products (one
// wide integer multiply-add each) and carry-free 64-bit additions:
// a b = p11 2^64 + (p01 + p10) 2^32 + p00.
HE_HD void mul128(u64 a, u64 b, u64& hi, u64& lo) {
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
  const u64 p00 = (u64)a0 * b0, p01 = (u64)a0 * b1, p10 = (u64)a1 * b0, p11 = (u64)a1 * b1;
  const u64 mid = p01 + (p00 >> 32);            // < 2^64 - 2^32
  const u64 mid2 = p10 + (mid & 0xffffffffull);  // < 2^64 - 2^32
  lo = (mid2 << 32) | (p00 & 0xffffffffull);
  hi = p11 + (mid >> 32) + (mid2 >> 32);
}

// A prime with its Barrett constant mu = floor(2^128 / q) = mu_hi 2^64 + mu_lo.
struct Mod {
  u64 q, mu_hi, mu_lo;
};

// x mod q for x = xh 2^64 + xl < q 2^64. The estimate qhat of floor(x / q)
// drops the low word of xl * mu_lo and the fractional carries, so
// floor(x/q) - 3 <= qhat <= floor(x/q) and x - qhat q lies in [0, 4q).
HE_HD u64 reduce128(u64 xh, u64 xl, const Mod& m) {
  const u64 t1 = mulhi64(xl, m.mu_lo);
  u64 p1l, p1h, p2l, p2h;
  mul128(xl, m.mu_hi, p1h, p1l);
  mul128(xh, m.mu_lo, p2h, p2l);
  const u64 s = p1l + p2l;
  u64 c = s < p1l;
  const u64 s2 = s + t1;
  c += s2 < s;
  const u64 qhat = xh * m.mu_hi + p1h + p2h + c;
  u64 r = xl - qhat * m.q;
  if (r >= m.q) r -= m.q;
  if (r >= m.q) r -= m.q;
  if (r >= m.q) r -= m.q;
  return r;
}

// a b mod q for a b < q 2^64 (e.g. a < 2^64, b < q).
HE_HD u64 mulmod(u64 a, u64 b, const Mod& m) {
  u64 hi, lo;
  mul128(a, b, hi, lo);
  return reduce128(hi, lo, m);
}

// 128-bit accumulator for sums of products, reduced once.
struct Acc128 {
  u64 hi, lo;
};
HE_HD void mac128(Acc128& acc, u64 a, u64 b) {
  u64 hi, lo;
  mul128(a, b, hi, lo);
  acc.lo += lo;
  acc.hi += hi + (acc.lo < lo);
}

// a w mod q in [0, 2q) for any a < 2^64, w < q, wp = floor(w 2^64 / q).
HE_HD u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) { return a * w - mulhi64(a, wp) * q; }
HE_HD u64 shoup(u64 a, u64 w, u64 wp, u64 q) {
  const u64 r = shoup_lazy(a, w, wp, q);
  return r >= q ? r - q : r;
}

HE_HD u64 addmod(u64 a, u64 b, u64 q) {
  const u64 s = a + b;
  return s >= q ? s - q : s;
}
HE_HD u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
HE_HD u64 negmod(u64 a, u64 q) { return a ? q - a : 0; }

// [0, 4q) -> [0, q)
HE_HD u64 reduce4q(u64 a, u64 q) {
  const u64 q2 = 2 * q;
  if (a >= q2) a -= q2;
  if (a >= q) a -= q;
  return a;
}

}  // namespace he
