// ckks_oracle.cpp - CPU RNS-CKKS oracle: parameters, NTT, encoding, keys,
// encryption, decryption, and the evaluation primitives of paper Sec. II-A
// (Add, Mul, cMul, Rot, and the rescale the paper leaves implicit).
//
// TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py; never by the CUDA library. It shares no code
// with the CUDA path apart from the seeded sampler inputs/he_random.h.
//
// The paper runs CKKS through HEAAN and states the primitives only as
// Enc/Dec/Add/Mul/cMul/Rot (Sec. II-A); it gives no RNS, NTT or key-switching
// description. What is written here is the standard RNS-CKKS scheme, each step
// in its textbook form:
//   - encoding: canonical embedding, slot j <-> root zeta^(5^j) (CKKS, Cheon et
//     al. 2017, cited in Sec. II-A),
//   - RNS limbs over NTT-friendly primes q = 1 mod 2N, exact modular arithmetic
//     by 128-bit product and remainder,
//   - hybrid key switching with digits of alpha primes (ModUp by fast base
//     conversion, inner product with the key, ModDown),
//   - rescale by the last prime with round-half-up.
// Every polynomial is kept in the coefficient domain; the negacyclic NTT is
// used only as the transform behind polynomial products.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../inputs/he_random.h"
#include "oracle_internal.h"

namespace oracle {

// ---------------------------------------------------------------------------
// Modular arithmetic helpers
// ---------------------------------------------------------------------------
u64 powmod(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
    e >>= 1;
  }
  return r;
}

u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

u64 reduce_signed(i64 v, u64 q) {
  i64 r = v % (i64)q;
  return r < 0 ? (u64)(r + (i64)q) : (u64)r;
}

// Deterministic Miller-Rabin: the first 12 prime bases decide every 64-bit n.
bool is_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : bases)
    if (n % p == 0) return n == p;
  u64 d = n - 1;
  int r = 0;
  while ((d & 1) == 0) { d >>= 1; r++; }
  for (u64 a : bases) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool composite = true;
    for (int i = 1; i < r; i++) {
      x = mulmod(x, x, n);
      if (x == n - 1) { composite = false; break; }
    }
    if (composite) return false;
  }
  return true;
}

static size_t bitrev(size_t x, int bits) {
  size_t r = 0;
  for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

// ---------------------------------------------------------------------------
// Parameters: prime chain and NTT roots
// ---------------------------------------------------------------------------
// Candidates of b bits are 2^b - t * 2N + 1 for t = 1, 2, ..., tested in that
// (descending) order; one cursor per bit size so that every prime is distinct.
struct PrimeCursor {
  std::map<int, u64> t;
  u64 next(int bits, u64 two_n) {
    u64& tt = t[bits];
    for (;;) {
      tt++;
      u64 top = (bits == 64) ? 0 : (1ULL << bits);
      u64 c = top - tt * two_n + 1;
      if (c < (1ULL << (bits - 1))) throw std::runtime_error("prime search ran out of candidates");
      if (is_prime(c)) return c;
    }
  }
};

// psi = x^((q-1)/2N) for the smallest x >= 2 with x^((q-1)/2) = -1 mod q
// (a quadratic non-residue); then psi^N = -1, so psi has order exactly 2N.
static u64 find_psi(u64 q, size_t N) {
  for (u64 x = 2;; x++) {
    if (powmod(x, (q - 1) / 2, q) == q - 1) return powmod(x, (q - 1) / (2 * N), q);
  }
}

static void init_params(Ctx& C, int log_n, int n_q, const int* q_bits, int n_special,
                        int special_bits, int alpha, double sigma, u64 seed) {
  if (log_n < 2 || log_n > 17 || n_q < 1 || n_special < 1 || alpha < 1)
    throw std::runtime_error("bad parameters");
  C.log_n = log_n;
  C.N = (size_t)1 << log_n;
  C.L1 = n_q;
  C.K = n_special;
  C.alpha = alpha;
  C.sigma = sigma;
  C.seed = seed;
  const u64 two_n = 2 * (u64)C.N;
  // Assignment order: the K special primes take the largest special_bits
  // candidates, then q_0, then q_1..q_L, each the largest unused candidate of
  // its own bit size.
  PrimeCursor cur;
  std::vector<u64> P(n_special), Q(n_q);
  for (int k = 0; k < n_special; k++) P[k] = cur.next(special_bits, two_n);
  for (int i = 0; i < n_q; i++) Q[i] = cur.next(q_bits[i], two_n);
  C.q = Q;
  C.q.insert(C.q.end(), P.begin(), P.end());
  const int np = n_q + n_special;
  C.psi.resize(np);
  C.psi_rev.assign(np, Poly(C.N));
  C.psi_inv_rev.assign(np, Poly(C.N));
  C.n_inv.resize(np);
  for (int pi = 0; pi < np; pi++) {
    u64 q = C.q[pi];
    u64 psi = find_psi(q, C.N);
    u64 psi_inv = invmod(psi, q);
    C.psi[pi] = psi;
    for (size_t k = 0; k < C.N; k++) {
      size_t e = bitrev(k, log_n);
      C.psi_rev[pi][k] = powmod(psi, e, q);
      C.psi_inv_rev[pi][k] = powmod(psi_inv, e, q);
    }
    C.n_inv[pi] = invmod(C.N % q, q);
  }
  C.cdt_bound = he_rand_cdt_init(sigma, C.cdt);
}

// ---------------------------------------------------------------------------
// Negacyclic NTT. NTT(a)[j] = sum_i a_i psi^((2 brv(j) + 1) i) mod q: the
// evaluations of a(X) at the odd powers of psi, in bit-reversed order.
// Forward: Cooley-Tukey butterflies with psi merged in; inverse: Gentleman-
// Sande butterflies, then a multiply by N^{-1}.
// ---------------------------------------------------------------------------
void ntt_fwd(const Ctx& C, int pi, u64* a) {
  const u64 q = C.q[pi];
  const size_t N = C.N;
  const Poly& W = C.psi_rev[pi];
  for (size_t m = 1, t = N / 2; m < N; m <<= 1, t >>= 1) {
    for (size_t i = 0; i < m; i++) {
      const u64 w = W[m + i];
      const size_t j1 = 2 * i * t;
      for (size_t j = j1; j < j1 + t; j++) {
        u64 u = a[j], v = mulmod(a[j + t], w, q);
        a[j] = addmod(u, v, q);
        a[j + t] = submod(u, v, q);
      }
    }
  }
}

void ntt_inv(const Ctx& C, int pi, u64* a) {
  const u64 q = C.q[pi];
  const size_t N = C.N;
  const Poly& W = C.psi_inv_rev[pi];
  for (size_t m = N / 2, t = 1; m >= 1; m >>= 1, t <<= 1) {
    for (size_t i = 0; i < m; i++) {
      const u64 w = W[m + i];
      const size_t j1 = 2 * i * t;
      for (size_t j = j1; j < j1 + t; j++) {
        u64 u = a[j], v = a[j + t];
        a[j] = addmod(u, v, q);
        a[j + t] = mulmod(submod(u, v, q), w, q);
      }
    }
  }
  for (size_t j = 0; j < N; j++) a[j] = mulmod(a[j], C.n_inv[pi], q);
}

// a * b in Z_q[X]/(X^N + 1), via the transform.
Poly polymul(const Ctx& C, int pi, const Poly& a, const Poly& b) {
  const u64 q = C.q[pi];
  Poly x = a, y = b;
  ntt_fwd(C, pi, x.data());
  ntt_fwd(C, pi, y.data());
  for (size_t j = 0; j < C.N; j++) x[j] = mulmod(x[j], y[j], q);
  ntt_inv(C, pi, x.data());
  return x;
}

// sum_j a_j * b_j in Z_q[X]/(X^N + 1) where the b_j are already transformed:
// the transform is linear, so the sum is taken on the transformed side.
static Poly inner_product(const Ctx& C, int pi, const std::vector<const Poly*>& a,
                          const std::vector<const Poly*>& b_ntt) {
  const u64 q = C.q[pi];
  Poly acc(C.N, 0), x(C.N);
  for (size_t j = 0; j < a.size(); j++) {
    x = *a[j];
    ntt_fwd(C, pi, x.data());
    const Poly& y = *b_ntt[j];
    for (size_t n = 0; n < C.N; n++) acc[n] = addmod(acc[n], mulmod(x[n], y[n], q), q);
  }
  ntt_inv(C, pi, acc.data());
  return acc;
}

// Galois automorphism phi_k: a(X) -> a(X^k), k odd. Coefficient i moves to
// i*k mod 2N and changes sign when that lands in [N, 2N) (X^N = -1).
void automorph(const u64* a, u64* out, size_t N, u64 k, u64 q) {
  const u64 two_n = 2 * (u64)N;
  for (size_t i = 0; i < N; i++) {
    u64 e = (u64)(((u128)i * k) % two_n);
    if (e < N) out[e] = a[i];
    else out[e - N] = negmod(a[i], q);
  }
}

// Rot(ct, l) rotates slots to the left by l (Sec. II-A, item 6). With slot j
// at root zeta^(5^j), X -> X^(5^l) moves slot j + l to slot j.
u64 galois_elt(const Ctx& C, long step) {
  const long slots = (long)C.N / 2;
  long r = ((step % slots) + slots) % slots;
  return powmod(5, (u64)r, 2 * (u64)C.N);
}

// ---------------------------------------------------------------------------
// Encoding (canonical embedding). Slot j <-> zeta^(5^j mod 2N), zeta =
// exp(i pi / N), j < N/2. For a real slot vector z and scale D:
//   m_k = round(D * (2/N) * Re sum_j z_j zeta^(-5^j k)),  k < N,
// rounding to nearest with ties away from zero. The sum is a length-2N DFT of
// the array holding z_j at index 5^j mod 2N.
// ---------------------------------------------------------------------------
static void fft_inplace(std::vector<std::complex<double>>& a, int sign) {
  const size_t n = a.size();
  int bits = 0;
  while (((size_t)1 << bits) < n) bits++;
  for (size_t i = 0; i < n; i++) {
    size_t j = bitrev(i, bits);
    if (i < j) std::swap(a[i], a[j]);
  }
  // roots exp(sign * 2 pi i k / n), k < n/2, each from cos/sin directly
  std::vector<std::complex<double>> w(n / 2);
  for (size_t k = 0; k < n / 2; k++) {
    double ang = sign * 2.0 * M_PI * (double)k / (double)n;
    w[k] = std::complex<double>(std::cos(ang), std::sin(ang));
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t step = n / len;
    for (size_t i = 0; i < n; i += len) {
      for (size_t j = 0; j < len / 2; j++) {
        std::complex<double> u = a[i + j], v = a[i + j + len / 2] * w[j * step];
        a[i + j] = u + v;
        a[i + j + len / 2] = u - v;
      }
    }
  }
}

static std::vector<size_t> slot_exponents(const Ctx& C) {
  const size_t S = C.N / 2, two_n = 2 * C.N;
  std::vector<size_t> e(S);
  size_t x = 1;
  for (size_t j = 0; j < S; j++) { e[j] = x; x = (x * 5) % two_n; }
  return e;
}

std::vector<i64> encode(const Ctx& C, const double* z, size_t nz, double scale) {
  const size_t N = C.N, S = N / 2;
  if (nz > S) throw std::runtime_error("encode: more values than slots");
  std::vector<std::complex<double>> A(2 * N, 0.0);
  std::vector<size_t> e = slot_exponents(C);
  for (size_t j = 0; j < nz; j++) A[e[j]] = z[j];
  fft_inplace(A, -1);
  std::vector<i64> m(N);
  for (size_t k = 0; k < N; k++) m[k] = std::llround(scale * (2.0 / (double)N) * A[k].real());
  return m;
}

// Inverse of the embedding: z_j = (1/scale) * sum_k m_k zeta^(5^j k) (real part).
static void decode(const Ctx& C, const std::vector<double>& m, double scale, double* z) {
  const size_t N = C.N, S = N / 2;
  std::vector<std::complex<double>> A(2 * N, 0.0);
  for (size_t k = 0; k < N; k++) A[k] = m[k];
  fft_inplace(A, +1);
  std::vector<size_t> e = slot_exponents(C);
  for (size_t j = 0; j < S; j++) z[j] = A[e[j]].real() / scale;
}

// ---------------------------------------------------------------------------
// Big-integer CRT composition (decryption). Little-endian 64-bit words.
// ---------------------------------------------------------------------------
typedef std::vector<u64> Big;

static Big big_mul_small(const Big& a, u64 b) {
  Big r(a.size() + 1, 0);
  u64 carry = 0;
  for (size_t i = 0; i < a.size(); i++) {
    u128 p = (u128)a[i] * b + carry;
    r[i] = (u64)p;
    carry = (u64)(p >> 64);
  }
  r[a.size()] = carry;
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}
static Big big_add(const Big& a, const Big& b) {
  size_t n = std::max(a.size(), b.size());
  Big r(n + 1, 0);
  u64 carry = 0;
  for (size_t i = 0; i < n; i++) {
    u128 s = (u128)(i < a.size() ? a[i] : 0) + (i < b.size() ? b[i] : 0) + carry;
    r[i] = (u64)s;
    carry = (u64)(s >> 64);
  }
  r[n] = carry;
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}
static int big_cmp(const Big& a, const Big& b) {
  size_t n = std::max(a.size(), b.size());
  for (size_t i = n; i-- > 0;) {
    u64 x = i < a.size() ? a[i] : 0, y = i < b.size() ? b[i] : 0;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}
static Big big_sub(const Big& a, const Big& b) {  // a >= b
  Big r(a.size(), 0);
  u64 borrow = 0;
  for (size_t i = 0; i < a.size(); i++) {
    u64 y = i < b.size() ? b[i] : 0;
    u128 d = (u128)a[i] - y - borrow;
    r[i] = (u64)d;
    borrow = (u64)(d >> 64) ? 1 : 0;
  }
  while (r.size() > 1 && r.back() == 0) r.pop_back();
  return r;
}
static double big_to_double(const Big& a) {
  double r = 0.0;
  for (size_t i = a.size(); i-- > 0;) r = r * 18446744073709551616.0 + (double)a[i];
  return r;
}

// Centered CRT lift of residues m[i][n] (i < limbs) to doubles.
static std::vector<double> crt_centered(const Ctx& C, const RnsPoly& m, int limbs) {
  Big Q{1};
  for (int i = 0; i < limbs; i++) Q = big_mul_small(Q, C.q[i]);
  std::vector<Big> Qhat(limbs);
  std::vector<u64> Qhat_inv(limbs);
  for (int i = 0; i < limbs; i++) {
    Big h{1};
    u64 hm = 1;
    for (int j = 0; j < limbs; j++)
      if (j != i) { h = big_mul_small(h, C.q[j]); hm = mulmod(hm, C.q[j] % C.q[i], C.q[i]); }
    Qhat[i] = h;
    Qhat_inv[i] = invmod(hm, C.q[i]);
  }
  Big halfQ = Q;  // floor(Q/2) compared via 2x > Q
  std::vector<double> out(C.N);
  for (size_t n = 0; n < C.N; n++) {
    Big x{0};
    for (int i = 0; i < limbs; i++)
      x = big_add(x, big_mul_small(Qhat[i], mulmod(m[i][n], Qhat_inv[i], C.q[i])));
    while (big_cmp(x, Q) >= 0) x = big_sub(x, Q);
    Big twice = big_add(x, x);
    if (big_cmp(twice, Q) > 0) out[n] = -big_to_double(big_sub(Q, x));
    else out[n] = big_to_double(x);
  }
  (void)halfQ;
  return out;
}

// ---------------------------------------------------------------------------
// Sampling (inputs/he_random.h) into residues.
// ---------------------------------------------------------------------------
static std::vector<i64> sample_ternary(const Ctx& C, u64 tag, u64 obj, u64 sub) {
  u64 st = he_rand_stream(C.seed, tag, obj, sub);
  std::vector<i64> v(C.N);
  for (size_t i = 0; i < C.N; i++) v[i] = he_rand_ternary(st, i);
  return v;
}
static std::vector<i64> sample_gauss(const Ctx& C, u64 tag, u64 obj, u64 sub) {
  u64 st = he_rand_stream(C.seed, tag, obj, sub);
  std::vector<i64> v(C.N);
  for (size_t i = 0; i < C.N; i++) v[i] = he_rand_gauss(st, i, C.cdt, C.cdt_bound);
  return v;
}
static Poly sample_uniform(const Ctx& C, u64 tag, u64 obj, u64 sub, int pi) {
  u64 st = he_rand_stream(C.seed, tag, obj, sub);
  Poly v(C.N);
  for (size_t i = 0; i < C.N; i++) v[i] = he_rand_uniform_mod(st, i, C.q[pi]);
  return v;
}
static Poly to_res(const std::vector<i64>& v, u64 q) {
  Poly r(v.size());
  for (size_t i = 0; i < v.size(); i++) r[i] = reduce_signed(v[i], q);
  return r;
}

// ---------------------------------------------------------------------------
// Keys. s ternary; pk = (-a s + e, a) over Q; a key-switching key from s' to s
// has, per digit j, evk_j = (-a_j s + e_j + P g_j s', a_j) over Q*P, where the
// gadget g_j is 1 modulo the primes of digit j and 0 modulo every other prime
// of Q, so P g_j s' mod q_i = (P mod q_i) s' for q_i in digit j, else 0.
// ---------------------------------------------------------------------------
static void make_ksk(Ctx& C, u64 key_id, const RnsPoly& s_prime /* L1 limbs */) {
  const int np = C.L1 + C.K, beta = C.beta_at(C.L1);
  Ksk key;
  key.d.assign(beta, std::vector<RnsPoly>(2, RnsPoly(np)));
  key.d_ntt = key.d;
  for (int j = 0; j < beta; j++) {
    std::vector<i64> e = sample_gauss(C, HE_TAG_KSK_E, key_id, (u64)j);
    for (int pi = 0; pi < np; pi++) {
      const u64 q = C.q[pi];
      Poly a = sample_uniform(C, HE_TAG_KSK_A, key_id, (u64)j * 256 + (u64)pi, pi);
      Poly as = polymul(C, pi, a, C.s_res[pi]);
      Poly b(C.N);
      u64 pmod = 1;
      for (int k = 0; k < C.K; k++) pmod = mulmod(pmod, C.q[C.L1 + k] % q, q);
      const bool in_digit = pi < C.L1 && pi / C.alpha == j;
      for (size_t n = 0; n < C.N; n++) {
        u64 v = submod(reduce_signed(e[n], q), as[n], q);
        if (in_digit) v = addmod(v, mulmod(pmod, s_prime[pi][n], q), q);
        b[n] = v;
      }
      key.d[j][0][pi] = b;
      key.d[j][1][pi] = a;
      for (int c = 0; c < 2; c++) {
        key.d_ntt[j][c][pi] = key.d[j][c][pi];
        ntt_fwd(C, pi, key.d_ntt[j][c][pi].data());
      }
    }
  }
  C.ksk[key_id] = std::move(key);
}

static void keygen(Ctx& C, const long* steps, int n_steps) {
  const int np = C.L1 + C.K;
  C.s = sample_ternary(C, HE_TAG_SECRET, 0, 0);
  C.s_res.assign(np, Poly());
  for (int pi = 0; pi < np; pi++) C.s_res[pi] = to_res(C.s, C.q[pi]);
  // public key over Q
  std::vector<i64> e = sample_gauss(C, HE_TAG_PK_E, 0, 0);
  C.pk0.assign(C.L1, Poly());
  C.pk1.assign(C.L1, Poly());
  for (int i = 0; i < C.L1; i++) {
    const u64 q = C.q[i];
    Poly a = sample_uniform(C, HE_TAG_PK_A, 0, (u64)i, i);
    Poly as = polymul(C, i, a, C.s_res[i]);
    Poly b(C.N);
    for (size_t n = 0; n < C.N; n++) b[n] = submod(reduce_signed(e[n], q), as[n], q);
    C.pk0[i] = b;
    C.pk1[i] = a;
  }
  // relinearisation key: s' = s^2
  RnsPoly s2(C.L1);
  for (int i = 0; i < C.L1; i++) s2[i] = polymul(C, i, C.s_res[i], C.s_res[i]);
  make_ksk(C, 0, s2);
  // Galois keys: s' = phi_k(s)
  for (int t = 0; t < n_steps; t++) {
    u64 k = galois_elt(C, steps[t]);
    if (k == 1 || C.ksk.count(k)) continue;
    RnsPoly sk(C.L1, Poly(C.N));
    for (int i = 0; i < C.L1; i++) automorph(C.s_res[i].data(), sk[i].data(), C.N, k, C.q[i]);
    make_ksk(C, k, sk);
  }
  C.has_keys = true;
}

// ---------------------------------------------------------------------------
// Enc_pk / Dec_sk (Sec. II-A, items 1-2).
//   Enc: ct = (v pk0 + e0 + m, v pk1 + e1) mod Q_l, v ternary, e0, e1 Gaussian.
//   Dec: m' = c0 + c1 s (+ c2 s^2 for a three-component ciphertext) mod Q_l.
// ---------------------------------------------------------------------------
static Ct encrypt(const Ctx& C, const i64* m, int limbs, u64 ct_id) {
  std::vector<i64> v = sample_ternary(C, HE_TAG_ENC_V, ct_id, 0);
  std::vector<i64> e0 = sample_gauss(C, HE_TAG_ENC_E0, ct_id, 0);
  std::vector<i64> e1 = sample_gauss(C, HE_TAG_ENC_E1, ct_id, 0);
  Ct ct;
  ct.c.assign(2, RnsPoly(limbs));
  for (int i = 0; i < limbs; i++) {
    const u64 q = C.q[i];
    Poly vr = to_res(v, q);
    Poly a0 = polymul(C, i, vr, C.pk0[i]);
    Poly a1 = polymul(C, i, vr, C.pk1[i]);
    for (size_t n = 0; n < C.N; n++) {
      a0[n] = addmod(addmod(a0[n], reduce_signed(e0[n], q), q), reduce_signed(m[n], q), q);
      a1[n] = addmod(a1[n], reduce_signed(e1[n], q), q);
    }
    ct.c[0][i] = a0;
    ct.c[1][i] = a1;
  }
  return ct;
}

static RnsPoly decrypt_res(const Ctx& C, const Ct& ct) {
  const int limbs = ct.limbs();
  RnsPoly m(limbs);
  for (int i = 0; i < limbs; i++) {
    const u64 q = C.q[i];
    Poly acc = ct.c[0][i];
    Poly spow = C.s_res[i];
    for (size_t t = 1; t < ct.c.size(); t++) {
      Poly prod = polymul(C, i, ct.c[t][i], spow);
      for (size_t n = 0; n < C.N; n++) acc[n] = addmod(acc[n], prod[n], q);
      if (t + 1 < ct.c.size()) spow = polymul(C, i, spow, C.s_res[i]);
    }
    m[i] = acc;
  }
  return m;
}

// ---------------------------------------------------------------------------
// Homomorphic operations
// ---------------------------------------------------------------------------
Ct ct_add(const Ctx& C, const Ct& a, const Ct& b) {  // Add (Sec. II-A, item 3)
  Ct r = a;
  const int limbs = a.limbs();
  for (size_t t = 0; t < a.c.size(); t++)
    for (int i = 0; i < limbs; i++)
      for (size_t n = 0; n < C.N; n++) r.c[t][i][n] = addmod(a.c[t][i][n], b.c[t][i][n], C.q[i]);
  return r;
}

// Tensor product, first half of Mul (Sec. II-A, item 4):
// d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.
Ct ct_tensor(Ctx& C, const Ct& a, const Ct& b) {
  const int limbs = a.limbs();
  Ct d;
  d.c.assign(3, RnsPoly(limbs));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < limbs; i++) {
    const u64 q = C.q[i];
    d.c[0][i] = polymul(C, i, a.c[0][i], b.c[0][i]);
    Poly x = polymul(C, i, a.c[0][i], b.c[1][i]);
    Poly y = polymul(C, i, a.c[1][i], b.c[0][i]);
    for (size_t n = 0; n < C.N; n++) x[n] = addmod(x[n], y[n], q);
    d.c[1][i] = x;
    d.c[2][i] = polymul(C, i, a.c[1][i], b.c[1][i]);
  }
  C.cnt.tensors++;
  return d;
}

// ModUp of digit j at level lp: primes I_j = [j alpha, min((j+1) alpha, lp)),
// D_j their product. Limbs of I_j are copied; every other target t of the
// basis {q_0..q_{lp-1}, p_0..p_{K-1}} gets the fast base conversion
//   y_t = sum_{i in I_j} [x_i (D_j/q_i)^{-1}]_{q_i} (D_j/q_i) mod t
// (no correction term, so y_t = x + u D_j mod t for some 0 <= u < |I_j|).
static RnsPoly modup(const Ctx& C, const RnsPoly& x, int lp, int j) {
  const int lo = j * C.alpha, hi = std::min(lo + C.alpha, lp), nb = lp + C.K;
  RnsPoly ext(nb, Poly(C.N));
  std::vector<u64> dhat_inv(hi - lo);
  for (int i = lo; i < hi; i++) {
    u64 h = 1;
    for (int i2 = lo; i2 < hi; i2++)
      if (i2 != i) h = mulmod(h, C.q[i2] % C.q[i], C.q[i]);
    dhat_inv[i - lo] = invmod(h, C.q[i]);
  }
  for (int pos = 0; pos < nb; pos++) {
    const int g = C.gidx(pos, lp);
    const u64 t = C.q[g];
    if (pos >= lo && pos < hi) { ext[pos] = x[pos]; continue; }
    std::vector<u64> dhat_t(hi - lo);  // (D_j / q_i) mod t
    for (int i = lo; i < hi; i++) {
      u64 h = 1;
      for (int i2 = lo; i2 < hi; i2++)
        if (i2 != i) h = mulmod(h, C.q[i2] % t, t);
      dhat_t[i - lo] = h;
    }
    for (size_t n = 0; n < C.N; n++) {
      u64 y = 0;
      for (int i = lo; i < hi; i++)
        y = addmod(y, mulmod(mulmod(x[i][n], dhat_inv[i - lo], C.q[i]) % t, dhat_t[i - lo], t), t);
      ext[pos][n] = y;
    }
  }
  return ext;
}

// ModDown at level lp: out_i = (u_i - BConv_{P->q_i}(u_P)) P^{-1} mod q_i with
// BConv_{P->t}(x) = sum_k [x_k (P/p_k)^{-1}]_{p_k} (P/p_k) mod t.
static RnsPoly moddown(const Ctx& C, const RnsPoly& u, int lp) {
  const int K = C.K;
  std::vector<u64> phat_inv(K);
  for (int k = 0; k < K; k++) {
    const u64 pk = C.q[C.L1 + k];
    u64 h = 1;
    for (int k2 = 0; k2 < K; k2++)
      if (k2 != k) h = mulmod(h, C.q[C.L1 + k2] % pk, pk);
    phat_inv[k] = invmod(h, pk);
  }
  RnsPoly out(lp, Poly(C.N));
  for (int i = 0; i < lp; i++) {
    const u64 q = C.q[i];
    std::vector<u64> phat_q(K);
    u64 pmod = 1;
    for (int k = 0; k < K; k++) {
      u64 h = 1;
      for (int k2 = 0; k2 < K; k2++)
        if (k2 != k) h = mulmod(h, C.q[C.L1 + k2] % q, q);
      phat_q[k] = h;
      pmod = mulmod(pmod, C.q[C.L1 + k] % q, q);
    }
    const u64 pinv = invmod(pmod, q);
    for (size_t n = 0; n < C.N; n++) {
      u64 z = 0;
      for (int k = 0; k < K; k++) {
        const u64 pk = C.q[C.L1 + k];
        z = addmod(z, mulmod(mulmod(u[lp + k][n], phat_inv[k], pk) % q, phat_q[k], q), q);
      }
      out[i][n] = mulmod(submod(u[i][n], z, q), pinv, q);
    }
  }
  return out;
}

// Inner product of the extended digits with a key, then ModDown of both
// components: returns (v0, v1) with v0 + v1 s ~ x s' over Q_l.
static std::vector<RnsPoly> ks_apply(Ctx& C, const std::vector<RnsPoly>& ext, int lp, const Ksk& key) {
  const int nb = lp + C.K, beta = (int)ext.size();
  std::vector<RnsPoly> u(2, RnsPoly(nb));
#pragma omp parallel for schedule(static)
  for (int pos = 0; pos < nb; pos++) {
    const int g = C.gidx(pos, lp);
    for (int c = 0; c < 2; c++) {
      std::vector<const Poly*> a(beta), b(beta);
      for (int j = 0; j < beta; j++) { a[j] = &ext[j][pos]; b[j] = &key.d_ntt[j][c][g]; }
      u[c][pos] = inner_product(C, g, a, b);
    }
  }
  std::vector<RnsPoly> v(2);
  for (int c = 0; c < 2; c++) v[c] = moddown(C, u[c], lp);
  return v;
}

static std::vector<RnsPoly> modup_all(Ctx& C, const RnsPoly& x, int lp) {
  const int beta = C.beta_at(lp);
  std::vector<RnsPoly> ext(beta);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < beta; j++) ext[j] = modup(C, x, lp, j);
  C.cnt.modups++;
  return ext;
}

// Relinearisation, second half of Mul: (d0, d1, d2) -> (d0 + v0, d1 + v1)
// where (v0, v1) is the key switch of d2 from s^2 to s.
Ct ct_relin(Ctx& C, const Ct& d) {
  const int lp = d.limbs();
  std::vector<RnsPoly> ext = modup_all(C, d.c[2], lp);
  std::vector<RnsPoly> v = ks_apply(C, ext, lp, C.ksk.at(0));
  Ct r;
  r.c.assign(2, RnsPoly(lp, Poly(C.N)));
  for (int i = 0; i < lp; i++)
    for (size_t n = 0; n < C.N; n++) {
      r.c[0][i][n] = addmod(d.c[0][i][n], v[0][i][n], C.q[i]);
      r.c[1][i][n] = addmod(d.c[1][i][n], v[1][i][n], C.q[i]);
    }
  C.cnt.relins++;
  return r;
}

// Rot(ct, l) for several l sharing one ModUp (hoisting). Canonical order:
// ModUp(c1) once; per step, phi_k on every extended digit, inner product with
// the Galois key of k, ModDown; result (phi_k(c0) + v0, v1).
std::vector<Ct> ct_rotate_hoisted(Ctx& C, const Ct& ct, const std::vector<long>& steps) {
  const int lp = ct.limbs(), nb = lp + C.K;
  std::vector<Ct> out(steps.size());
  std::vector<RnsPoly> ext;
  bool need = false;
  for (long s : steps) need |= galois_elt(C, s) != 1;
  if (need) ext = modup_all(C, ct.c[1], lp);
  for (size_t t = 0; t < steps.size(); t++) {
    const u64 k = galois_elt(C, steps[t]);
    if (k == 1) { out[t] = ct; continue; }
    std::vector<RnsPoly> ext_k(ext.size(), RnsPoly(nb, Poly(C.N)));
    for (size_t j = 0; j < ext.size(); j++)
      for (int pos = 0; pos < nb; pos++)
        automorph(ext[j][pos].data(), ext_k[j][pos].data(), C.N, k, C.q[C.gidx(pos, lp)]);
    std::vector<RnsPoly> v = ks_apply(C, ext_k, lp, C.ksk.at(k));
    Ct r;
    r.c.assign(2, RnsPoly(lp, Poly(C.N)));
    for (int i = 0; i < lp; i++) {
      automorph(ct.c[0][i].data(), r.c[0][i].data(), C.N, k, C.q[i]);
      for (size_t n = 0; n < C.N; n++) r.c[0][i][n] = addmod(r.c[0][i][n], v[0][i][n], C.q[i]);
      r.c[1][i] = v[1][i];
    }
    out[t] = r;
    C.cnt.rotations++;
  }
  return out;
}

// Rescale by the last prime q_l (round half up):
//   r = (x_l + floor(q_l/2)) mod q_l,  out_i = (x_i + floor(q_l/2) - r) q_l^{-1} mod q_i.
Ct ct_rescale(Ctx& C, const Ct& ct) {
  const int lp = ct.limbs();
  if (lp < 2) throw std::runtime_error("rescale: no level left");
  const u64 ql = C.q[lp - 1], half = ql / 2;
  Ct r;
  r.c.assign(ct.c.size(), RnsPoly(lp - 1, Poly(C.N)));
  for (size_t t = 0; t < ct.c.size(); t++) {
    const Poly& xl = ct.c[t][lp - 1];
    for (int i = 0; i < lp - 1; i++) {
      const u64 q = C.q[i];
      const u64 inv = invmod(ql % q, q), half_q = half % q;
      for (size_t n = 0; n < C.N; n++) {
        const u64 rr = addmod(xl[n], half, ql) % q;
        const u64 v = submod(addmod(ct.c[t][i][n], half_q, q), rr, q);
        r.c[t][i][n] = mulmod(v, inv, q);
      }
    }
  }
  C.cnt.rescales++;
  return r;
}

// cMul by a scalar held as the integer w (a constant polynomial).
Ct ct_mul_scalar(Ctx& C, const Ct& ct, i64 w) {
  Ct r = ct;
  for (size_t t = 0; t < ct.c.size(); t++)
    for (int i = 0; i < ct.limbs(); i++) {
      const u64 q = C.q[i], wq = reduce_signed(w, q);
      for (size_t n = 0; n < C.N; n++) r.c[t][i][n] = mulmod(ct.c[t][i][n], wq, q);
    }
  C.cnt.ct_scalar++;
  return r;
}

// cMul by an encoded plaintext polynomial pt (integer coefficients).
Ct ct_mul_plain(Ctx& C, const Ct& ct, const std::vector<i64>& pt) {
  Ct r = ct;
  for (int i = 0; i < ct.limbs(); i++) {
    Poly p = to_res(pt, C.q[i]);
    for (size_t t = 0; t < ct.c.size(); t++) r.c[t][i] = polymul(C, i, ct.c[t][i], p);
  }
  C.cnt.ct_plain++;
  return r;
}

// Add a constant c (the constant polynomial c) to the message.
Ct ct_add_const(const Ctx& C, const Ct& ct, i64 c) {
  Ct r = ct;
  for (int i = 0; i < ct.limbs(); i++) r.c[0][i][0] = addmod(r.c[0][i][0], reduce_signed(c, C.q[i]), C.q[i]);
  return r;
}

}  // namespace oracle

// ===========================================================================
// C API (host arrays). Ciphertext arrays are [n_polys][limbs][N] uint64,
// coefficient domain, residues in [0, q_i).
// ===========================================================================
using namespace oracle;

namespace oracle {
Ct ct_from(const Ctx& C, const u64* p, int n_polys, int limbs) {
  Ct ct;
  ct.c.assign(n_polys, RnsPoly(limbs, Poly(C.N)));
  for (int t = 0; t < n_polys; t++)
    for (int i = 0; i < limbs; i++)
      std::memcpy(ct.c[t][i].data(), p + ((size_t)t * limbs + i) * C.N, C.N * 8);
  return ct;
}
void ct_to(const Ctx& C, const Ct& ct, u64* p) {
  const int limbs = ct.limbs();
  for (size_t t = 0; t < ct.c.size(); t++)
    for (int i = 0; i < limbs; i++)
      std::memcpy(p + (t * limbs + i) * C.N, ct.c[t][i].data(), C.N * 8);
}
}  // namespace oracle

static thread_local std::string g_err;

#define OC_TRY(...)                    \
  try {                                \
    __VA_ARGS__;                       \
    return 0;                          \
  } catch (const std::exception& e) {  \
    g_err = e.what();                  \
    return -1;                         \
  }

extern "C" {

const char* oc_last_error() { return g_err.c_str(); }

void* oc_create(int log_n, int n_q, const int* q_bits, int n_special, int special_bits, int alpha,
                double sigma, uint64_t seed) {
  try {
    Ctx* C = new Ctx();
    init_params(*C, log_n, n_q, q_bits, n_special, special_bits, alpha, sigma, seed);
    return C;
  } catch (const std::exception& e) {
    g_err = e.what();
    return nullptr;
  }
}
void oc_free(void* h) { delete (Ctx*)h; }

int oc_n_primes(void* h) { Ctx* C = (Ctx*)h; return C->L1 + C->K; }
void oc_primes(void* h, uint64_t* out) { Ctx* C = (Ctx*)h; for (size_t i = 0; i < C->q.size(); i++) out[i] = C->q[i]; }
uint64_t oc_psi(void* h, int pi) { return ((Ctx*)h)->psi[pi]; }

int oc_ntt(void* h, int pi, uint64_t* a, int inverse) {
  OC_TRY(Ctx* C = (Ctx*)h; if (inverse) ntt_inv(*C, pi, a); else ntt_fwd(*C, pi, a));
}
int oc_polymul(void* h, int pi, const uint64_t* a, const uint64_t* b, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; Poly x(a, a + C->N), y(b, b + C->N); Poly r = polymul(*C, pi, x, y);
         std::memcpy(out, r.data(), C->N * 8));
}
int oc_automorph(void* h, int pi, const uint64_t* a, uint64_t k, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; automorph(a, out, C->N, k, C->q[pi]));
}
uint64_t oc_galois_elt(void* h, long step) { return galois_elt(*(Ctx*)h, step); }

// ModUp of digit j: x [lp][N] -> ext [lp+K][N]
int oc_modup(void* h, const uint64_t* x, int lp, int j, uint64_t* ext) {
  OC_TRY(Ctx* C = (Ctx*)h; RnsPoly xx(lp, Poly(C->N));
         for (int i = 0; i < lp; i++) std::memcpy(xx[i].data(), x + (size_t)i * C->N, C->N * 8);
         RnsPoly e = modup(*C, xx, lp, j);
         for (int i = 0; i < lp + C->K; i++) std::memcpy(ext + (size_t)i * C->N, e[i].data(), C->N * 8));
}
// ModDown: u [lp+K][N] -> out [lp][N]
int oc_moddown(void* h, const uint64_t* u, int lp, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; RnsPoly uu(lp + C->K, Poly(C->N));
         for (int i = 0; i < lp + C->K; i++) std::memcpy(uu[i].data(), u + (size_t)i * C->N, C->N * 8);
         RnsPoly o = moddown(*C, uu, lp);
         for (int i = 0; i < lp; i++) std::memcpy(out + (size_t)i * C->N, o[i].data(), C->N * 8));
}

int oc_encode(void* h, const double* z, size_t nz, double scale, int64_t* m) {
  OC_TRY(Ctx* C = (Ctx*)h; std::vector<i64> r = encode(*C, z, nz, scale); std::memcpy(m, r.data(), C->N * 8));
}
int oc_decode(void* h, const double* m, double scale, double* z) {
  OC_TRY(Ctx* C = (Ctx*)h; std::vector<double> mm(m, m + C->N); decode(*C, mm, scale, z));
}

int oc_keygen(void* h, const long* steps, int n_steps) { OC_TRY(keygen(*(Ctx*)h, steps, n_steps)); }
int oc_secret(void* h, int64_t* s) { OC_TRY(Ctx* C = (Ctx*)h; std::memcpy(s, C->s.data(), C->N * 8)); }
// key [beta][2][L1+K][N], coefficient domain
int oc_export_key(void* h, uint64_t key_id, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; const Ksk& k = C->ksk.at(key_id); size_t o = 0;
         for (auto& dj : k.d) for (auto& dc : dj) for (auto& limb : dc) { std::memcpy(out + o, limb.data(), C->N * 8); o += C->N; });
}

int oc_encrypt(void* h, const int64_t* m, int limbs, uint64_t ct_id, uint64_t* ct) {
  OC_TRY(Ctx* C = (Ctx*)h; if (limbs < 1 || limbs > C->L1) throw std::runtime_error("bad level");
         if (C->pk0.size() != (size_t)C->L1) throw std::runtime_error("no public key (call keygen first)");
         Ct r = encrypt(*C, m, limbs, ct_id); ct_to(*C, r, ct));
}
// m' = sum_t c_t s^t, CRT-centred, as doubles [N]
int oc_decrypt_coeffs(void* h, const uint64_t* ct, int n_polys, int limbs, double* out) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct c = ct_from(*C, ct, n_polys, limbs); RnsPoly m = decrypt_res(*C, c);
         std::vector<double> v = crt_centered(*C, m, limbs); std::memcpy(out, v.data(), C->N * 8));
}
int oc_decrypt_slots(void* h, const uint64_t* ct, int n_polys, int limbs, double scale, double* z) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct c = ct_from(*C, ct, n_polys, limbs); RnsPoly m = decrypt_res(*C, c);
         std::vector<double> v = crt_centered(*C, m, limbs); decode(*C, v, scale, z));
}

int oc_add(void* h, const uint64_t* a, const uint64_t* b, int n_polys, int limbs, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct r = ct_add(*C, ct_from(*C, a, n_polys, limbs), ct_from(*C, b, n_polys, limbs)); ct_to(*C, r, out));
}
int oc_tensor(void* h, const uint64_t* a, const uint64_t* b, int limbs, uint64_t* out3) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct r = ct_tensor(*C, ct_from(*C, a, 2, limbs), ct_from(*C, b, 2, limbs)); ct_to(*C, r, out3));
}
int oc_relin(void* h, const uint64_t* d3, int limbs, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct r = ct_relin(*C, ct_from(*C, d3, 3, limbs)); ct_to(*C, r, out));
}
// Key switch of one polynomial x [lp][N] with key `key_id` (0 = relin): out [2][lp][N]
int oc_keyswitch(void* h, const uint64_t* x, int lp, uint64_t key_id, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; RnsPoly xx(lp, Poly(C->N));
         for (int i = 0; i < lp; i++) std::memcpy(xx[i].data(), x + (size_t)i * C->N, C->N * 8);
         std::vector<RnsPoly> ext = modup_all(*C, xx, lp);
         std::vector<RnsPoly> v = ks_apply(*C, ext, lp, C->ksk.at(key_id));
         for (int c = 0; c < 2; c++) for (int i = 0; i < lp; i++)
           std::memcpy(out + ((size_t)c * lp + i) * C->N, v[c][i].data(), C->N * 8));
}
int oc_rotate_hoisted(void* h, const uint64_t* ct, int limbs, const long* steps, int n, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; std::vector<long> st(steps, steps + n);
         std::vector<Ct> r = ct_rotate_hoisted(*C, ct_from(*C, ct, 2, limbs), st);
         for (int t = 0; t < n; t++) ct_to(*C, r[t], out + (size_t)t * 2 * limbs * C->N));
}
int oc_rescale(void* h, const uint64_t* ct, int n_polys, int limbs, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct r = ct_rescale(*C, ct_from(*C, ct, n_polys, limbs)); ct_to(*C, r, out));
}
int oc_mul_scalar(void* h, const uint64_t* ct, int limbs, int64_t w, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; Ct r = ct_mul_scalar(*C, ct_from(*C, ct, 2, limbs), w); ct_to(*C, r, out));
}
int oc_mul_plain(void* h, const uint64_t* ct, int limbs, const int64_t* pt, uint64_t* out) {
  OC_TRY(Ctx* C = (Ctx*)h; std::vector<i64> p(pt, pt + C->N);
         Ct r = ct_mul_plain(*C, ct_from(*C, ct, 2, limbs), p); ct_to(*C, r, out));
}

// counters: rotations, modups, tensors, relins, rescales, ct_scalar, ct_plain
void oc_counters(void* h, long* out) {
  Ctx* C = (Ctx*)h;
  out[0] = C->cnt.rotations; out[1] = C->cnt.modups; out[2] = C->cnt.tensors; out[3] = C->cnt.relins;
  out[4] = C->cnt.rescales; out[5] = C->cnt.ct_scalar; out[6] = C->cnt.ct_plain;
}
void oc_reset_counters(void* h) { ((Ctx*)h)->cnt.reset(); }

}  // extern "C"
