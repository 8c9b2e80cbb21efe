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

// Full 64 x 64 -> 128-bit product. Schoolbook on 32-bit words:
// a b = a1 b1 2^64 + (a0 b1 + a1 b0) 2^32 + a0 b0. On the device the word
// products are accumulated with PTX carry chains (mad.lo/madc.hi with .cc);
// on the host, four 32 x 32 -> 64-bit products and carry-free additions.
HE_HD void mul128(u64 a, u64 b, u64& hi, u64& lo) {
#if defined(__CUDA_ARCH__)
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
  u32 w0, w1, w2, w3;
  asm("mul.lo.u32     %0, %4, %6;\n\t"
      "mul.hi.u32     %1, %4, %6;\n\t"
      "mul.lo.u32     %2, %5, %7;\n\t"
      "mul.hi.u32     %3, %5, %7;\n\t"
      "mad.lo.cc.u32  %1, %4, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32       %3, %3, 0;\n\t"
      "mad.lo.cc.u32  %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32       %3, %3, 0;"
      : "=&r"(w0), "=&r"(w1), "=&r"(w2), "=&r"(w3)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  lo = ((u64)w1 << 32) | w0;
  hi = ((u64)w3 << 32) | w2;
#else
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
  const u64 p00 = (u64)a0 * b0, p01 = (u64)a0 * b1, p10 = (u64)a1 * b0, p11 = (u64)a1 * b1;
  const u64 mid = p01 + (p00 >> 32);            // < 2^64 - 2^32
  const u64 mid2 = p10 + (mid & 0xffffffffull);  // < 2^64 - 2^32
  lo = (mid2 << 32) | (p00 & 0xffffffffull);
  hi = p11 + (mid >> 32) + (mid2 >> 32);
#endif
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
// acc += a b; the caller keeps the sum below 2^128.
HE_HD void mac128(Acc128& acc, u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
  // the even word products straight into the accumulator, then the two cross products one word up
  u32 w0 = (u32)acc.lo, w1 = (u32)(acc.lo >> 32), w2 = (u32)acc.hi, w3 = (u32)(acc.hi >> 32);
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
  asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
      "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
      "madc.hi.u32    %3, %5, %7, %3;\n\t"
      "mad.lo.cc.u32  %1, %4, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32       %3, %3, 0;\n\t"
      "mad.lo.cc.u32  %1, %5, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
      "addc.u32       %3, %3, 0;"
      : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
  acc.lo = ((u64)w1 << 32) | w0;
  acc.hi = ((u64)w3 << 32) | w2;
#else
  u64 hi, lo;
  mul128(a, b, hi, lo);
  acc.lo += lo;
  acc.hi += hi + (acc.lo < lo);
#endif
}

// 96-bit accumulator (three 32-bit words) for sums of products of residues below
// kMac96Prime: a product is below 2^92 and its high words' product a1 b1 below 2^28,
// so a b = a0 b0 + (a0 b1 + a1 b0) 2^32 + a1 b1 2^64 needs seven 32-bit multiplies
// (three of them high halves) and no fourth word while the sum stays below 2^96.
struct Acc96 {
  u32 w0, w1, w2;
};
constexpr u64 kMac96Prime = 1ull << 46;
// acc += a b for a, b < kMac96Prime; the caller keeps the sum below 2^96 (every partial
// sum is then below 2^96 too, so the dropped carries out of the top word are zero).
HE_HD void mac96(Acc96& acc, u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
  asm("mad.lo.cc.u32  %0, %3, %5, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %5, %1;\n\t"
      "madc.lo.u32    %2, %4, %6, %2;\n\t"
      "mad.lo.cc.u32  %1, %3, %6, %1;\n\t"
      "madc.hi.u32    %2, %3, %6, %2;\n\t"
      "mad.lo.cc.u32  %1, %4, %5, %1;\n\t"
      "madc.hi.u32    %2, %4, %5, %2;"
      : "+r"(acc.w0), "+r"(acc.w1), "+r"(acc.w2)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
#else
  u64 hi, lo;
  mul128(a, b, hi, lo);
  const u64 l = (((u64)acc.w1 << 32) | acc.w0) + lo;
  const u64 h = (u64)acc.w2 + hi + (l < lo);
  acc.w0 = (u32)l;
  acc.w1 = (u32)(l >> 32);
  acc.w2 = (u32)h;
#endif
}
// the accumulated value mod q in [0, q) (Barrett on the 96-bit value, below q 2^64)
HE_HD u64 reduce96(const Acc96& acc, const Mod& m) {
  return reduce128((u64)acc.w2, ((u64)acc.w1 << 32) | acc.w0, m);
}
// products of residues mod q that fit on top of a reduced sum: floor(2^96 / (q - 1)^2) - 1
// (so that v + room (q - 1)^2 < 2^96 for v < q), computed in double precision with a margin
HE_HD int mac96_room(u64 q) {
  const double r = 79228162514264337593543950336.0 / ((double)(q - 1) * (double)(q - 1)) * (1.0 - 1e-12);
  return r >= (double)(1 << 20) ? (1 << 20) : (int)r - 1;
}

// Montgomery reduction (Montgomery, Math. Comp. 1985) of x = hi 2^64 + lo < q 2^64:
// x 2^{-64} mod q in [0, q), with qneg = -q^{-1} mod 2^64. m = lo qneg makes
// x + m q divisible by 2^64; its low word sums to 2^64 unless lo = 0.
HE_HD u64 redc128(u64 hi, u64 lo, u64 q, u64 qneg) {
  const u64 m = lo * qneg;
  u64 mh, ml;
  mul128(m, q, mh, ml);
  const u64 t = hi + mh + (lo != 0);
  return t >= q ? t - q : t;
}

// a w mod q in [0, 2q) for any a < 2^64, w < q, wp = floor(w 2^64 / q).
HE_HD u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) { return a * w - mulhi64(a, wp) * q; }
HE_HD u64 shoup(u64 a, u64 w, u64 wp, u64 q) {
  const u64 r = shoup_lazy(a, w, wp, q);
  return r >= q ? r - q : r;
}

// a w mod q in [0, 4q) for any a < 2^64, w < q, wp = floor(w 2^64 / q), 4q < 2^64.
// Shoup's product with a cheaper quotient estimate: of the four 32 x 32-bit word
// products of a wp only a1 wp1 and the high halves of a1 wp0 and a0 wp1 are kept
// (dropped: their low halves and a0 wp0, together below 3 2^64). The estimate is
// therefore at most 2 below floor(a wp / 2^64), which is itself at most 1 below
// floor(a w / q) and never above it, so the remainder a w - qhat q is in [0, 4q)
// and exact as a 64-bit word.
HE_HD u64 shoup_approx(u64 a, u64 w, u64 wp, u64 q) {
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), p0 = (u32)wp, p1 = (u32)(wp >> 32);
#if defined(__CUDA_ARCH__)
  const u64 qh = (u64)a1 * p1 + ((u64)__umulhi(a1, p0) + __umulhi(a0, p1));
#else
  const u64 qh = (u64)a1 * p1 + ((((u64)a1 * p0) >> 32) + (((u64)a0 * p1) >> 32));
#endif
  return a * w - qh * q;
}

// Primes below this bound take the transforms' growing-range path: values are
// not reduced between butterfly stages (each forward stage adds at most 4q, each
// inverse stage at most doubles), which stays below 2^64 through 16 stages.
constexpr u64 kNarrowPrime = 1ull << 54;

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

#if defined(__CUDACC__)
// v mod q for v < 2^9 q, q < 2^54 (frd = 2^sh / q rounded to fp32, sh = max(0, bitlen(q) + 9 - 32)):
// the quotient is estimated in fp32 from the top 32 bits of v. The estimate x of v / q has
// |x - v / q| < 2^-13 (three fp32 roundings of a value below 512, and the dropped low bits worth
// below 2^-22), so trunc(x) is floor(v / q) or one off either side; v - trunc(x) q is then in
// [-q, 2q) and one correction makes it exact. One 32 x 64-bit product instead of a Shoup product.
__device__ __forceinline__ u64 reduce_fp32(u64 v, u64 q, float frd, int sh) {
  const u32 hi = (u32)(v >> sh);
  const u32 t = __float2uint_rz(__fmul_rn(__uint2float_rn(hi), frd));
  u64 r = v - (u64)t * q;
  if ((long long)r < 0)
    r += q;
  else if (r >= q)
    r -= q;
  return r;
}

__device__ __forceinline__ u32 brv_bits(u32 x, int bits) { return __brev(x) >> (32 - bits); }

// Index j' with NTT(phi_k(a))[j] = NTT(a)[j'] for the bit-reversed evaluation
// order: slot j holds a(psi^(2 brv(j) + 1)), and phi_k maps that point to
// psi^((2 brv(j) + 1) k).
__device__ __forceinline__ u32 galois_index(u32 j, u64 k, int log_n) {
  const u64 two_n_mask = (2ull << log_n) - 1;
  const u64 e = 2 * (u64)brv_bits(j, log_n) + 1;
  const u64 e2 = (e * k) & two_n_mask;
  return brv_bits((u32)((e2 - 1) >> 1), log_n);
}
#endif

}  // namespace he
