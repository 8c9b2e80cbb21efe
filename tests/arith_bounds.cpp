// Host check of the library's modular-arithmetic helpers (paper_2512_18646_gb300/csrc/he_arith.cuh)
// against exact 128-bit integer arithmetic: the bounds the kernels rely on.
//  - shoup_approx(a, w, w', q) is a w mod q plus 0..3 q (a < 2^64, w < q, 4q < 2^64);
//  - mac96 sums agree with exact sums, and mac96_room(q) products of residues fit on top of a
//    reduced value: v + room (q - 1)^2 < 2^96;
//  - reduce96 / reduce128 return the residue of the sum.
// Prints "ok" and exits 0, or prints the first failure and exits 1.
#include "he_arith.cuh"

#include <cstdio>
#include <random>

using namespace he;
typedef unsigned __int128 u128;

static Mod make_mod(u64 q) {
  Mod m;
  m.q = q;
  // mu = floor(2^128 / q) = floor((2^128 - 1) / q) for q not a power of two
  const u128 mu = (~(u128)0) / q;
  m.mu_hi = (u64)(mu >> 64);
  m.mu_lo = (u64)mu;
  return m;
}

static bool is_prime(u64 n) {
  if (n < 2) return false;
  for (u64 p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull})
    if (n % p == 0) return n == p;
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) d >>= 1, s++;
  for (u64 a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
    u128 x = 1, b = a % n;
    for (u64 e = d; e; e >>= 1, b = b * b % n)
      if (e & 1) x = x * b % n;
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; r++) {
      x = x * x % n;
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

static u64 prime_below(u64 bound) {
  for (u64 q = bound - 1;; q -= 2)
    if (is_prime(q)) return q;
}

int main() {
  std::mt19937_64 rng(12345);
  const u64 bounds[] = {1ull << 40, 1ull << 45, kMac96Prime, 1ull << 54, 1ull << 60, 1ull << 62};
  for (u64 bound : bounds) {
    const u64 q = prime_below(bound);
    const Mod m = make_mod(q);
    for (int t = 0; t < 200000; t++) {
      const u64 a = t % 3 == 0 ? ~0ull - (rng() & 0xffff) : rng();
      const u64 w = rng() % q;
      const u64 wp = (u64)(((u128)w << 64) / q);
      const u64 r = shoup_approx(a, w, wp, q);
      const u64 exact = (u64)((u128)a * w % q);
      if (r >= 4 * q || r % q != exact) {
        printf("shoup_approx q=%llu a=%llu w=%llu: %llu\n", (unsigned long long)q, (unsigned long long)a,
               (unsigned long long)w, (unsigned long long)r);
        return 1;
      }
      const u64 hi = rng() % q, lo = rng();
      if (reduce128(hi, lo, m) != (u64)((((u128)hi << 64) | lo) % q)) {
        printf("reduce128 q=%llu\n", (unsigned long long)q);
        return 1;
      }
    }
    if (q >= kMac96Prime) continue;
    const int room = mac96_room(q);
    const u128 lim = (u128)1 << 96;
    if (room < 1 || (u128)(q - 1) + (u128)room * (q - 1) * (q - 1) >= lim) {
      printf("mac96_room q=%llu room=%d\n", (unsigned long long)q, room);
      return 1;
    }
    for (int t = 0; t < 2000; t++) {
      Acc96 acc{0, 0, 0};
      u128 sum = 0;
      const u64 v0 = t & 1 ? q - 1 : rng() % q;  // a reduced value, then room products at the top
      acc.w0 = (u32)v0;
      acc.w1 = (u32)(v0 >> 32);
      sum = v0;
      for (int j = 0; j < room; j++) {
        const u64 x = t & 1 ? q - 1 : rng() % q, y = t & 1 ? q - 1 : rng() % q;
        mac96(acc, x, y);
        sum += (u128)x * y;
      }
      const u128 got = ((u128)acc.w2 << 64) | ((u128)acc.w1 << 32) | acc.w0;
      if (got != sum || reduce96(acc, m) != (u64)(sum % q)) {
        printf("mac96 q=%llu\n", (unsigned long long)q);
        return 1;
      }
    }
  }
  printf("ok\n");
  return 0;
}
