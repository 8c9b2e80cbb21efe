// oracle_internal.h - internal declarations of the CPU RNS-CKKS oracle.
//
// TEST INFRASTRUCTURE ONLY. The oracle is a plain, slow, obviously correct
// restatement of the scheme and of the paper's multi-ciphertext layouts. Only
// tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.
// It shares no code with the CUDA library; the one shared module is the seeded
// sampler in inputs/he_random.h, which holds no scheme arithmetic.
//
// Representation: every polynomial is held in the coefficient domain, one
// vector of N residues in [0, q) per prime ("limb"). Ring: Z_q[X] / (X^N + 1).
#pragma once

#include <atomic>
#include <cstdint>
#include <map>
#include <vector>

namespace oracle {

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

typedef std::vector<u64> Poly;       // N residues of one limb
typedef std::vector<Poly> RnsPoly;   // limbs
struct Ct {                          // ciphertext (c0, c1) or (d0, d1, d2)
  std::vector<RnsPoly> c;
  int limbs() const { return c.empty() ? 0 : (int)c[0].size(); }
};

// ---- plain modular arithmetic (128-bit product, then %) ----
inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
inline u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
inline u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : q - b + a; }
inline u64 negmod(u64 a, u64 q) { return a ? q - a : 0; }
u64 powmod(u64 b, u64 e, u64 q);
u64 invmod(u64 a, u64 q);  // q prime
u64 reduce_signed(i64 v, u64 q);
bool is_prime(u64 n);

// Key-switching key: digits j < beta, components c in {0,1}, limbs over the
// full Q*P basis (q_0..q_L, p_0..p_{K-1}); coefficient domain, plus the
// forward NTT of every limb (the key is fixed, so its transform is kept).
struct Ksk {
  std::vector<std::vector<RnsPoly>> d;      // [beta][2] -> RnsPoly (L1+K limbs)
  std::vector<std::vector<RnsPoly>> d_ntt;  // same, NTT domain
};

struct Counters {
  std::atomic<long> rotations{0};   // key switches for Galois automorphisms
  std::atomic<long> modups{0};      // ModUp calls (one per hoisted rotation set / relin)
  std::atomic<long> tensors{0};     // ciphertext-ciphertext tensor products
  std::atomic<long> relins{0};
  std::atomic<long> rescales{0};    // ciphertexts rescaled
  std::atomic<long> ct_scalar{0};   // ciphertext x scalar products
  std::atomic<long> ct_plain{0};    // ciphertext x plaintext products
  void reset() { rotations = 0; modups = 0; tensors = 0; relins = 0; rescales = 0; ct_scalar = 0; ct_plain = 0; }
};

struct Ctx {
  int log_n = 0;
  size_t N = 0;
  int L1 = 0;      // number of Q primes (q_0 .. q_L)
  int K = 0;       // number of special primes
  int alpha = 1;   // primes per digit
  std::vector<u64> q;                        // L1 + K primes: Q then P
  std::vector<u64> psi;                      // primitive 2N-th root per prime
  std::vector<Poly> psi_rev, psi_inv_rev;    // psi^{brv(k)}, psi^{-brv(k)}
  std::vector<u64> n_inv;
  double sigma = 3.2;
  u64 seed = 0;
  uint64_t cdt[64];
  int cdt_bound = 0;

  bool has_keys = false;
  std::vector<i64> s;                        // ternary secret coefficients
  RnsPoly s_res;                             // s mod every prime (L1+K limbs)
  RnsPoly pk0, pk1;                          // public key over Q (L1 limbs)
  std::map<u64, Ksk> ksk;                    // key id -> key (0 = relinearisation)
  Counters cnt;

  int beta_at(int lp) const { return (lp + alpha - 1) / alpha; }
  // global prime index of position pos in the basis {q_0..q_{lp-1}, p_0..p_{K-1}}
  int gidx(int pos, int lp) const { return pos < lp ? pos : L1 + (pos - lp); }
};

// ---- scheme pieces (ckks_oracle.cpp) ----
void ntt_fwd(const Ctx& C, int pi, u64* a);
void ntt_inv(const Ctx& C, int pi, u64* a);
Poly polymul(const Ctx& C, int pi, const Poly& a, const Poly& b);
void automorph(const u64* a, u64* out, size_t N, u64 k, u64 q);
u64 galois_elt(const Ctx& C, long step);

Ct ct_add(const Ctx& C, const Ct& a, const Ct& b);
Ct ct_tensor(Ctx& C, const Ct& a, const Ct& b);
Ct ct_relin(Ctx& C, const Ct& d);
std::vector<Ct> ct_rotate_hoisted(Ctx& C, const Ct& ct, const std::vector<long>& steps);
Ct ct_rescale(Ctx& C, const Ct& ct);
Ct ct_mul_scalar(Ctx& C, const Ct& ct, i64 w);
Ct ct_mul_plain(Ctx& C, const Ct& ct, const std::vector<i64>& pt);
Ct ct_add_const(const Ctx& C, const Ct& ct, i64 c);
std::vector<i64> encode(const Ctx& C, const double* z, size_t nz, double scale);

}  // namespace oracle
