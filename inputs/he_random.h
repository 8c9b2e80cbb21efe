/*
 * he_random.h - seeded random draws for RNS-CKKS key generation and encryption.
 *
 * This is the one module that both the CPU oracle (oracle/) and the CUDA
 * library (paper_2512_18646_gb300/csrc/) use. It holds only the random draws
 * the scheme consumes -- secret, public-key and key-switching-key masks and
 * errors, and encryption randomness -- and none of the scheme's arithmetic.
 * With identical draws on both sides, ciphertext limbs can be compared
 * bit for bit.
 *
 * Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) in counter form. Draw i of a stream with
 * state s is mix(s + (i + 1) * GAMMA), the (i+1)-th output of SplitMix64
 * started at s. Each (seed, purpose tag, object id, sub id) names its own
 * stream, so every coefficient can be drawn independently and in parallel.
 *
 * Distributions:
 *   - uniform mod q : a 128-bit draw (two 64-bit draws) reduced mod q; the
 *                     bias is below q / 2^128.
 *   - ternary       : (d * 3) >> 64 of one 64-bit draw d, minus 1; values in
 *                     {-1, 0, 1}, bias below 2^-62.
 *   - discrete Gaussian, parameter sigma, truncated at |e| <= floor(6 sigma):
 *                     inversion of a cumulative table of exp(-k^2 / (2 sigma^2))
 *                     held as 63-bit thresholds; the low bit of the same draw
 *                     gives the sign.
 *
 * Header-only plain C99 (also valid C++). Needs unsigned __int128 (gcc/clang,
 * x86_64 and aarch64).
 */
#ifndef HE_RANDOM_H
#define HE_RANDOM_H

#include <stdint.h>
#include <math.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Purpose tags: one per kind of random object the scheme draws. */
enum {
  HE_TAG_SECRET = 1, /* secret key s, ternary, one stream                        */
  HE_TAG_PK_A = 2,   /* public-key mask a, uniform, sub = prime index            */
  HE_TAG_PK_E = 3,   /* public-key error e, Gaussian                            */
  HE_TAG_KSK_A = 4,  /* key-switching-key mask a_j, uniform, obj = key id,
                        sub = digit * 256 + prime index                          */
  HE_TAG_KSK_E = 5,  /* key-switching-key error e_j, Gaussian, obj = key id,
                        sub = digit                                             */
  HE_TAG_ENC_V = 6,  /* encryption ephemeral v, ternary, obj = ciphertext id    */
  HE_TAG_ENC_E0 = 7, /* encryption error e0, Gaussian, obj = ciphertext id      */
  HE_TAG_ENC_E1 = 8  /* encryption error e1, Gaussian, obj = ciphertext id      */
};

#define HE_RAND_GAMMA 0x9E3779B97F4A7C15ULL
#define HE_CDT_MAX 64

/* SplitMix64 output function (the variant-13 finaliser). */
static inline uint64_t he_rand_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* State of the stream named by (seed, tag, obj, sub). */
static inline uint64_t he_rand_stream(uint64_t seed, uint64_t tag, uint64_t obj, uint64_t sub) {
  uint64_t s = he_rand_mix(seed + HE_RAND_GAMMA);
  s = he_rand_mix(s ^ he_rand_mix(tag + 0x632BE59BD9B4E019ULL));
  s = he_rand_mix(s ^ he_rand_mix(obj + 0x8CB92BA72F3D8DD7ULL));
  s = he_rand_mix(s ^ he_rand_mix(sub + 0xD1B54A32D192ED03ULL));
  return s;
}

/* Draw i (0-based) of a stream. */
static inline uint64_t he_rand_draw(uint64_t stream, uint64_t i) {
  return he_rand_mix(stream + (i + 1) * HE_RAND_GAMMA);
}

/* Coefficient i of a uniform polynomial mod q: draws 2i and 2i+1. */
static inline uint64_t he_rand_uniform_mod(uint64_t stream, uint64_t i, uint64_t q) {
  unsigned __int128 x = ((unsigned __int128)he_rand_draw(stream, 2 * i) << 64) |
                        (unsigned __int128)he_rand_draw(stream, 2 * i + 1);
  return (uint64_t)(x % q);
}

/* Coefficient i of a ternary polynomial, in {-1, 0, 1}. */
static inline int he_rand_ternary(uint64_t stream, uint64_t i) {
  unsigned __int128 x = (unsigned __int128)he_rand_draw(stream, i) * 3u;
  return (int)(uint64_t)(x >> 64) - 1;
}

/*
 * Cumulative table for the truncated discrete Gaussian with parameter sigma.
 * Writes thresholds t[0..bound] and returns bound = floor(6 sigma) (at most
 * HE_CDT_MAX - 1). P(|e| <= k) is proportional to
 * 1 + 2 * sum_{1<=i<=k} exp(-i^2 / (2 sigma^2)); t[k] = floor(P(|e| <= k) * 2^63)
 * and t[bound] = 2^63.
 */
static inline int he_rand_cdt_init(double sigma, uint64_t* t) {
  int bound = (int)floor(6.0 * sigma);
  if (bound < 1) bound = 1;
  if (bound > HE_CDT_MAX - 1) bound = HE_CDT_MAX - 1;
  double w[HE_CDT_MAX];
  double total = 0.0;
  for (int k = 0; k <= bound; k++) {
    w[k] = (k == 0 ? 1.0 : 2.0) * exp(-(double)k * (double)k / (2.0 * sigma * sigma));
    total += w[k];
  }
  double cum = 0.0;
  for (int k = 0; k < bound; k++) {
    cum += w[k];
    t[k] = (uint64_t)ldexp(cum / total, 63);
  }
  t[bound] = 1ULL << 63;
  return bound;
}

/* Coefficient i of a Gaussian error polynomial, from a table made by he_rand_cdt_init. */
static inline int he_rand_gauss(uint64_t stream, uint64_t i, const uint64_t* t, int bound) {
  uint64_t d = he_rand_draw(stream, i);
  uint64_t u = d >> 1;
  int k = 0;
  while (k < bound && u >= t[k]) k++;
  return (d & 1u) ? -k : k;
}

#ifdef __cplusplus
}
#endif

#endif /* HE_RANDOM_H */
