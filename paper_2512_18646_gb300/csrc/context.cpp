// context.cpp - parameters, device tables, key generation, encryption and
// decryption of the GB300 RNS-CKKS engine.
//
// Scheme (Sec. II-A lists Enc_pk, Dec_sk and the evaluation keys the CKKS
// library provides; the RNS form is the standard full-RNS CKKS):
//   secret s ternary; public key (b, a) = (-a s + e, a) over Q;
//   key-switching key from s' to s, digit j of alpha primes:
//     (-a_j s + e_j + P g_j s', a_j) over Q*P, g_j = 1 mod the primes of
//     digit j and 0 mod the other primes of Q;
//   Enc(m) = (v b + e0 + m, v a + e1), v ternary, e0, e1 Gaussian;
//   Dec(c0, c1) = c0 + c1 s.
// Random draws come from the seeded streams of inputs/he_random.h, so that a
// given (seed, ciphertext id) always yields the same ciphertext.
//
// Galois keys are stored pre-permuted: for phi_k the key holds
// phi_{k^-1}(evk) in the NTT domain, so the inner product reads the ModUp
// digits in place and the single permutation is applied to its result
// (sum_j phi_k(d_j) evk_j = phi_k(sum_j d_j phi_{k^-1}(evk_j))).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "../../inputs/he_random.h"
#include "he_internal.h"

namespace he {

typedef unsigned __int128 u128;

void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) throw Error(5, std::string("out of device memory: ") + what);
  throw Error(7, std::string(what) + ": " + cudaGetErrorString(e));
}

// armed by he_debug_fail_allocations: that many of the next allocations fail
std::atomic<int> g_fail_allocs{0};

DevBuf::DevBuf(size_t w, cudaStream_t s) : words(w), st(s) {
  if (w == 0) return;
  if (g_fail_allocs.load() > 0 && g_fail_allocs.fetch_sub(1) > 0) {
    words = 0;
    throw Error(5, "device allocation of " + std::to_string(w * 8) + " bytes failed (injected)");
  }
  void* ptr = nullptr;
  cudaError_t e = cudaMallocAsync(&ptr, w * 8, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(5, "device allocation of " + std::to_string(w * 8) + " bytes failed");
  }
  p = (u64*)ptr;
}
DevBuf::~DevBuf() { reset(); }
void DevBuf::reset() {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
  words = 0;
}
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
  if (this != &o) {
    reset();
    p = o.p; words = o.words; st = o.st;
    o.p = nullptr; o.words = 0;
  }
  return *this;
}

// ---------------------------------------------------------------------------
// host number theory
// ---------------------------------------------------------------------------
static u64 mul_h(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
static u64 pow_h(u64 b, u64 e, u64 m) {
  u64 r = 1;
  b %= m;
  for (; e; e >>= 1, b = mul_h(b, b, m))
    if (e & 1) r = mul_h(r, b, m);
  return r;
}
static u64 inv_h(u64 a, u64 m) { return pow_h(a % m, m - 2, m); }

// Miller-Rabin with the 12 smallest prime bases (exact below 3.3e24).
static bool prime_h(u64 n) {
  const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : small) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  int s = __builtin_ctzll(n - 1);
  const u64 d = (n - 1) >> s;
  for (u64 a : small) {
    u64 x = pow_h(a, d, n);
    if (x == 1 || x == n - 1) continue;
    int r = 1;
    for (; r < s; r++) {
      x = mul_h(x, x, n);
      if (x == n - 1) break;
    }
    if (r == s) return false;
  }
  return true;
}

static u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

static Mod make_mod(u64 q) {
  const u128 mu = (~(u128)0) / q;  // floor(2^128 / q) since q is odd
  return Mod{q, (u64)(mu >> 64), (u64)mu};
}

static u32 brv_h(u32 x, int bits) {
  u32 r = 0;
  for (int i = 0; i < bits; i++, x >>= 1) r = (r << 1) | (x & 1);
  return r;
}

u64 Ctx::galois_elt(long step) const {
  const long slots = (long)N / 2;
  const long r = ((step % slots) + slots) % slots;
  return pow_h(5, (u64)r, 2 * (u64)N);
}

const DevBuf& Ctx::key(u64 k) const {
  auto it = ksk.find(k);
  if (it == ksk.end())
    throw Error(3, k == 1 ? "no relinearisation key (call he_keygen)" : "no rotation key for Galois element " + std::to_string(k));
  return it->second;
}

Staging::~Staging() {
  for (int i = 0; i < kSlots; i++) {
    if (ev[i]) cudaEventSynchronize(ev[i]), cudaEventDestroy(ev[i]);
    if (buf[i]) cudaFreeHost(buf[i]);
  }
}

ImportRing::~ImportRing() {
  if (!copy) return;
  cudaStreamSynchronize(copy);
  for (int k = 0; k < 2; k++) {
    if (pending[k]) cudaEventSynchronize(consumed[k]);
    if (buf[k]) cudaFree(buf[k]);
    cudaEventDestroy(copied[k]);
    cudaEventDestroy(consumed[k]);
  }
  if (bad) cudaFree(bad);
  cudaStreamDestroy(copy);
}

ExportRing::~ExportRing() {
  for (int k = 0; k < kSlots; k++)
    if (done[k]) {
      cudaEventSynchronize(done[k]);
      cudaEventDestroy(done[k]);
    }
}

void upload_async(Ctx& C, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return;
  // A capture of the context's stream, opened by he_graph_begin or by the caller directly (its own
  // cudaStreamBeginCapture or a framework's graph capture), must not record a host-to-device copy:
  // a replay would read a staging slot that later calls reuse, or host memory the call has freed.
  // The call is refused instead (and a he_graph capture marked failed).
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HE_CUDA(cudaStreamIsCapturing(C.stream, &cs));
  if (C.capturing || cs != cudaStreamCaptureStatusNone) {
    C.capture_failed = C.capture_failed || C.capturing;
    throw Error(9 /* HE_E_STATE */, "this call copies host data to the device and cannot run inside a capture of the "
                            "context's stream");
  }
  if (bytes > Staging::kSlotBytes) {
    // pageable source: the call returns once the data is staged
    HE_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, C.stream));
    return;
  }
  Staging& S = C.staging;
  std::lock_guard<std::mutex> lk(S.mu);
  const int i = S.next;
  S.next = (i + 1) % Staging::kSlots;
  if (!S.buf[i]) {
    HE_CUDA(cudaHostAlloc(&S.buf[i], Staging::kSlotBytes, cudaHostAllocDefault));
    HE_CUDA(cudaEventCreateWithFlags(&S.ev[i], cudaEventDisableTiming));
  } else if (S.used[i]) {
    HE_CUDA(cudaEventSynchronize(S.ev[i]));  // the slot's previous copy has run
  }
  std::memcpy(S.buf[i], src, bytes);
  HE_CUDA(cudaMemcpyAsync(dst, S.buf[i], bytes, cudaMemcpyHostToDevice, C.stream));
  HE_CUDA(cudaEventRecord(S.ev[i], C.stream));
  S.used[i] = true;
}

static void upload(const Ctx& C, u64* dst, const void* src, size_t bytes) {
  HE_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, C.stream));
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
void ctx_init(Ctx& C, int log_n, const std::vector<int>& q_bits, int n_special, int special_bits, int alpha,
              double log_scale, double sigma, u64 seed, cudaStream_t st) {
  if (log_n < 4 || log_n > 16) throw Error(1, "log_n must be in [4, 16]");
  if (q_bits.empty() || q_bits.size() > 32) throw Error(1, "n_q must be in [1, 32]");
  if (n_special < 1 || n_special > 8) throw Error(1, "n_special must be in [1, 8]");
  if (alpha < 1 || alpha > 8) throw Error(1, "alpha must be in [1, 8]");
  if (special_bits < 20 || special_bits > 61) throw Error(1, "special_bits must be in [20, 61]");
  for (int b : q_bits)
    if (b < 20 || b > 61) throw Error(1, "prime bit sizes must be in [20, 61]");
  if (!(sigma > 0) || !(log_scale > 0)) throw Error(1, "sigma and log_scale must be positive");
  HE_CUDA(cudaGetDevice(&C.device));
  C.stream = st;
  C.log_n = log_n;
  C.N = (size_t)1 << log_n;
  C.L1 = (int)q_bits.size();
  C.K = n_special;
  C.alpha = alpha;
  C.scale0 = std::ldexp(1.0, 0) * std::pow(2.0, log_scale);
  C.sigma = sigma;
  C.seed = seed;
  C.cdt_bound = he_rand_cdt_init(sigma, C.cdt);
  // keep freed pool memory cached instead of returning it to the driver
  cudaMemPool_t pool;
  HE_CUDA(cudaDeviceGetDefaultMemPool(&pool, C.device));
  uint64_t thr = ~0ull;
  HE_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));

  // prime chain: specials first, then q_0 .. q_L, each the largest unused
  // candidate 2^b - t 2N + 1 of its size
  const u64 two_n = 2 * (u64)C.N;
  std::map<int, u64> cursor;
  auto next_prime = [&](int bits) -> u64 {
    u64& t = cursor[bits];
    for (;;) {
      ++t;
      const u64 top = 1ull << bits;
      if (t * two_n >= top / 2) throw Error(1, "no NTT-friendly prime of " + std::to_string(bits) + " bits left");
      const u64 c = top - t * two_n + 1;
      if (prime_h(c)) return c;
    }
  };
  std::vector<u64> P(n_special);
  for (auto& p : P) p = next_prime(special_bits);
  C.q.clear();
  for (int b : q_bits) C.q.push_back(next_prime(b));
  for (u64 p : P) C.q.push_back(p);
  const int np = C.np();

  // per-prime constants and NTT twiddles
  C.ptab.assign(np, PrimeTab{});
  std::vector<u64> psi_tab((size_t)np * 2 * C.N), ipsi_tab((size_t)np * 2 * C.N);
  std::vector<u64> pw(C.N);
  for (int g = 0; g < np; g++) {
    const u64 q = C.q[g];
    PrimeTab& T = C.ptab[g];
    T.mod = make_mod(q);
    T.ninv = inv_h(C.N % q, q);
    T.ninv_sh = shoup_of(T.ninv, q);
    u64 pm = 1;
    for (u64 p : P) pm = mul_h(pm, p % q, q);
    T.pmod = pm;
    T.one_sh = shoup_of(1, q);
    T.mont_r = (u64)(((u128)1 << 64) % q);
    T.mont_r_sh = shoup_of(T.mont_r, q);
    u64 qi = 1;  // q^{-1} mod 2^64 by Newton iteration (q odd): each step doubles the correct bits
    for (int it = 0; it < 6; it++) qi *= 2 - q * qi;
    T.qinv_neg = (u64)0 - qi;
    int qbits = 0;
    while (qbits < 64 && (q >> qbits)) qbits++;
    T.frd_sh = std::max(0, qbits + 9 - 32);
    T.frd = (float)(std::ldexp(1.0, T.frd_sh) / (double)q);
    // psi = x^((q-1)/2N), x the smallest quadratic non-residue
    u64 x = 2;
    while (pow_h(x, (q - 1) / 2, q) != q - 1) x++;
    const u64 psi = pow_h(x, (q - 1) / two_n, q), ipsi = inv_h(psi, q);
    for (int dir = 0; dir < 2; dir++) {
      const u64 r = dir ? ipsi : psi;
      pw[0] = 1;
      for (size_t e = 1; e < C.N; e++) pw[e] = mul_h(pw[e - 1], r, q);
      u64* tab = (dir ? ipsi_tab.data() : psi_tab.data()) + (size_t)g * 2 * C.N;
      for (size_t k = 0; k < C.N; k++) {  // interleaved (w, w') pairs for 16-byte loads
        const u64 w = pw[brv_h((u32)k, log_n)];
        tab[2 * k] = w;
        tab[2 * k + 1] = shoup_of(w, q);
      }
    }
  }
  C.d_ptab = DevBuf((size_t)np * sizeof(PrimeTab) / 8, st);
  upload(C, C.d_ptab.p, C.ptab.data(), (size_t)np * sizeof(PrimeTab));
  C.d_psi = DevBuf(psi_tab.size(), st);
  upload(C, C.d_psi.p, psi_tab.data(), psi_tab.size() * 8);
  C.d_ipsi = DevBuf(ipsi_tab.size(), st);
  upload(C, C.d_ipsi.p, ipsi_tab.data(), ipsi_tab.size() * 8);

  // ModUp tables per level (`limbs`); digit j covers primes [j alpha, min((j+1) alpha, limbs)):
  //   inv   [L1+1][L1][2]         (D_j/q_i)^{-1} mod q_i, Shoup companion
  //   hat   [L1+1][L1][L1+K][2]   (D_j/q_i) mod t_pos, pos over {q_0..q_{limbs-1}, p_0..}, companion
  //   scale [L1+1][L1][2]         N^{-1} (D_j/q_i)^{-1} mod q_i, companion
  // Each conversion term [x_i (D_j/q_i)^{-1}]_{q_i} (D_j/q_i) is a lazy Shoup product below 2 t.
  const int L1 = C.L1, K = C.K;
  std::vector<u64> up((size_t)(L1 + 1) * L1 * 2 + (size_t)(L1 + 1) * L1 * (L1 + K) * 2 + (size_t)(L1 + 1) * L1 * 2, 0);
  u64* up_inv = up.data();
  u64* up_hat = up.data() + (size_t)(L1 + 1) * L1 * 2;
  // N^{-1} (D_j/q_i)^{-1} mod q_i: the inverse transform before ModUp ends with this one factor
  u64* up_scale = up_hat + (size_t)(L1 + 1) * L1 * (L1 + K) * 2;
  for (int limbs = 1; limbs <= L1; limbs++) {
    for (int i = 0; i < limbs; i++) {
      const int lo = (i / alpha) * alpha, hi = std::min(lo + alpha, limbs);
      u64 h = 1;
      for (int i2 = lo; i2 < hi; i2++)
        if (i2 != i) h = mul_h(h, C.q[i2] % C.q[i], C.q[i]);
      const u64 hinv = inv_h(h, C.q[i]);
      up_inv[((size_t)limbs * L1 + i) * 2] = hinv;
      up_inv[((size_t)limbs * L1 + i) * 2 + 1] = shoup_of(hinv, C.q[i]);
      const u64 sc = mul_h(C.ptab[i].ninv, hinv, C.q[i]);
      up_scale[((size_t)limbs * L1 + i) * 2] = sc;
      up_scale[((size_t)limbs * L1 + i) * 2 + 1] = shoup_of(sc, C.q[i]);
      for (int pos = 0; pos < limbs + K; pos++) {
        const u64 t = C.q[pos < limbs ? pos : L1 + (pos - limbs)];
        u64 ht = 1;
        for (int i2 = lo; i2 < hi; i2++)
          if (i2 != i) ht = mul_h(ht, C.q[i2] % t, t);
        u64* h = up_hat + (((size_t)limbs * L1 + i) * (L1 + K) + pos) * 2;
        h[0] = ht;
        h[1] = shoup_of(ht, t);
      }
    }
  }
  C.d_up = DevBuf(up.size(), st);
  upload(C, C.d_up.p, up.data(), up.size() * 8);

  // ModDown tables: (P/p_k)^{-1} mod p_k, (P/p_k) mod q_i, P^{-1} mod q_i, each with its
  // Shoup companion
  std::vector<u64> down((size_t)2 * K + (size_t)2 * K * L1 + (size_t)2 * L1 + (size_t)2 * K);
  for (int k = 0; k < K; k++) {
    const u64 pk = P[k];
    u64 h = 1;
    for (int k2 = 0; k2 < K; k2++)
      if (k2 != k) h = mul_h(h, P[k2] % pk, pk);
    const u64 hi = inv_h(h, pk);
    down[2 * k] = hi;
    down[2 * k + 1] = shoup_of(hi, pk);
    for (int i = 0; i < L1; i++) {
      u64 hq = 1;
      for (int k2 = 0; k2 < K; k2++)
        if (k2 != k) hq = mul_h(hq, P[k2] % C.q[i], C.q[i]);
      down[2 * K + ((size_t)k * L1 + i) * 2] = hq;
      down[2 * K + ((size_t)k * L1 + i) * 2 + 1] = shoup_of(hq, C.q[i]);
    }
  }
  for (int i = 0; i < L1; i++) {
    const u64 pinv = inv_h(C.ptab[i].pmod, C.q[i]);
    down[2 * K + (size_t)2 * K * L1 + 2 * i] = pinv;
    down[2 * K + (size_t)2 * K * L1 + 2 * i + 1] = shoup_of(pinv, C.q[i]);
  }
  // N^{-1} (P/p_k)^{-1} mod p_k: the inverse transform of the P part ends with this one factor
  for (int k = 0; k < K; k++) {
    const u64 pk = P[k];
    const u64 v = mul_h(C.ptab[L1 + k].ninv, down[2 * k], pk);
    down[2 * K + (size_t)2 * K * L1 + 2 * L1 + 2 * k] = v;
    down[2 * K + (size_t)2 * K * L1 + 2 * L1 + 2 * k + 1] = shoup_of(v, pk);
  }
  C.d_down = DevBuf(down.size(), st);
  upload(C, C.d_down.p, down.data(), down.size() * 8);

  // rescale tables: for `limbs` (before), q_l = q[limbs-1], row i < limbs-1:
  // floor(q_l/2) mod q_i, q_l^{-1} mod q_i, Shoup companion
  std::vector<u64> rs((size_t)(L1 + 1) * L1 * 3, 0);
  for (int limbs = 2; limbs <= L1; limbs++) {
    const u64 ql = C.q[limbs - 1];
    for (int i = 0; i < limbs - 1; i++) {
      const u64 qi = C.q[i];
      const u64 inv = inv_h(ql % qi, qi);
      u64* t = rs.data() + ((size_t)limbs * L1 + i) * 3;
      t[0] = (ql / 2) % qi;
      t[1] = inv;
      t[2] = shoup_of(inv, qi);
    }
  }
  C.d_rs = DevBuf(rs.size(), st);
  upload(C, C.d_rs.p, rs.data(), rs.size() * 8);
  C.d_status = DevBuf(1, st);
  HE_CUDA(cudaMemsetAsync(C.d_status.p, 0, 8, st));

  // host FFT tables for encode / decode (M = N/2 point complex DFT)
  const size_t M = C.N / 2;
  C.fft_root.resize(2 * M);
  C.fft_twist.resize(2 * M);
  C.slot_index.resize(M);
  for (size_t k = 0; k < M; k++) {
    const double a = 2.0 * M_PI * (double)k / (double)M;
    C.fft_root[2 * k] = std::cos(a);
    C.fft_root[2 * k + 1] = std::sin(a);
    const double b = M_PI * (double)k / (double)C.N;
    C.fft_twist[2 * k] = std::cos(b);
    C.fft_twist[2 * k + 1] = std::sin(b);
  }
  u64 e = 1;
  for (size_t j = 0; j < M; j++) {
    C.slot_index[j] = (uint32_t)((e - 1) / 4);
    e = (e * 5) % two_n;
  }
  HE_CUDA(cudaStreamSynchronize(st));
}

std::unique_ptr<CtSet> new_set(Ctx& C, int n, int polys, int limbs, double scale) {
  auto s = std::make_unique<CtSet>();
  s->ctx = &C;
  s->n = n;
  s->polys = polys;
  s->limbs = limbs;
  s->scale = scale;
  s->gen = C.capturing ? C.capture_gen : 0;
  s->buf = DevBuf((size_t)n * polys * limbs * C.N, C.stream);
  return s;
}

// ---------------------------------------------------------------------------
// key generation
// ---------------------------------------------------------------------------
namespace {

// run f(i) for i < n over a few host threads
template <class F>
void parallel_for(size_t n, F f) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 16) nt = 16;
  if (n < 2 || nt == 1) {
    for (size_t i = 0; i < n; i++) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; t++)
    th.emplace_back([&, t] {
      for (size_t i = t; i < n; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

void sample_small(const Ctx& C, int tag, u64 obj, u64 sub, int8_t* out) {
  const u64 st = he_rand_stream(C.seed, (u64)tag, obj, sub);
  if (tag == HE_TAG_SECRET || tag == HE_TAG_ENC_V)
    for (size_t i = 0; i < C.N; i++) out[i] = (int8_t)he_rand_ternary(st, i);
  else
    for (size_t i = 0; i < C.N; i++) out[i] = (int8_t)he_rand_gauss(st, i, C.cdt, C.cdt_bound);
}

// uniform residues for primes g0 .. g0+count-1 with stream sub ids sub0 + g
void sample_uniform(const Ctx& C, int tag, u64 obj, u64 sub0, int count, u64* out) {
  parallel_for((size_t)count, [&](size_t g) {
    const u64 st = he_rand_stream(C.seed, (u64)tag, obj, sub0 + g);
    const u64 q = C.q[g];
    u64* o = out + g * C.N;
    for (size_t i = 0; i < C.N; i++) o[i] = he_rand_uniform_mod(st, i, q);
  });
}

LimbMap all_primes(const Ctx& C) {
  LimbMap m;
  m.lpp = C.np(); m.split = C.np(); m.base0 = 0; m.base1 = 0; m.poly_stride = (size_t)C.np() * C.N;
  return m;
}

// One switching key from s' (NTT domain, np limbs; only Q limbs are used) to s.
DevBuf make_ksk(Ctx& C, u64 key_id, const u64* d_sprime) {
  const int np = C.np(), beta = C.beta_at(C.L1);
  const size_t NPN = (size_t)np * C.N;
  DevBuf key((size_t)beta * 2 * NPN, C.stream);
  std::vector<u64> a_host(NPN);
  std::vector<int8_t> e_host(C.N);
  DevBuf e8(C.N / 8 + 1, C.stream), e_res(NPN, C.stream);
  const LimbMap lm = all_primes(C);
  for (int j = 0; j < beta; j++) {
    sample_uniform(C, HE_TAG_KSK_A, key_id, (u64)j * 256, np, a_host.data());
    sample_small(C, HE_TAG_KSK_E, key_id, (u64)j, e_host.data());
    u64* b = key.p + (size_t)j * 2 * NPN;
    u64* a = b + NPN;
    upload(C, a, a_host.data(), NPN * 8);
    upload(C, e8.p, e_host.data(), C.N);
    HE_CUDA(cudaStreamSynchronize(C.stream));  // host staging buffers are reused
    ntt_forward(C, a, 1, lm);
    k_reduce_small(C, (const int8_t*)e8.p, e_res.p, 1, lm);
    ntt_forward(C, e_res.p, 1, lm);
    k_ksk_combine(C, a, e_res.p, d_sprime, b, j);
  }
  // the inner product reduces its sums by Montgomery reduction, so keys are kept as k 2^64 mod q
  k_mont_form(C, key.p, beta * 2, lm);
  return key;
}

}  // namespace

// Checkpoint of the keys: header [magic, version, log_n, n_q, K, alpha, primes...], the secret
// [L1+K][N] and public key [2][L1][N] (NTT domain), then per switching key its Galois element
// (1: relinearisation), its word count and its words.
static const u64 kKeyMagic = 0x4845474233303031ull;  // "HEGB3001"

size_t keys_export(Ctx& C, u64* out, size_t cap) {
  if (!C.has_keys) throw Error(9, "no keys to export (call he_keygen)");
  const size_t NPN = (size_t)C.np() * C.N, PK = (size_t)2 * C.L1 * C.N;
  size_t need = 6 + C.np() + NPN + PK + 1;
  for (auto& kv : C.ksk) need += 2 + kv.second.words;
  if (!out) return need;
  if (cap < need) throw Error(1, "output too small for the keys (" + std::to_string(need) + " words)");
  size_t o = 0;
  out[o++] = kKeyMagic;
  out[o++] = 1;
  out[o++] = (u64)C.log_n;
  out[o++] = (u64)C.L1;
  out[o++] = (u64)C.K;
  out[o++] = (u64)C.alpha;
  for (int i = 0; i < C.np(); i++) out[o++] = C.q[i];
  HE_CUDA(cudaMemcpyAsync(out + o, C.d_s.p, NPN * 8, cudaMemcpyDeviceToHost, C.stream));
  o += NPN;
  HE_CUDA(cudaMemcpyAsync(out + o, C.d_pk.p, PK * 8, cudaMemcpyDeviceToHost, C.stream));
  o += PK;
  out[o++] = (u64)C.ksk.size();
  for (auto& kv : C.ksk) {
    out[o++] = kv.first;
    out[o++] = (u64)kv.second.words;
    HE_CUDA(cudaMemcpyAsync(out + o, kv.second.p, kv.second.words * 8, cudaMemcpyDeviceToHost, C.stream));
    o += kv.second.words;
  }
  HE_CUDA(cudaStreamSynchronize(C.stream));
  return need;
}

void keys_import(Ctx& C, const u64* in, size_t n) {
  auto need = [&](size_t at, size_t words) {
    if (at + words > n) throw Error(1, "truncated key checkpoint");
  };
  need(0, 6);
  if (in[0] != kKeyMagic || in[1] != 1) throw Error(1, "not a key checkpoint of this library");
  if (in[2] != (u64)C.log_n || in[3] != (u64)C.L1 || in[4] != (u64)C.K || in[5] != (u64)C.alpha)
    throw Error(1, "key checkpoint of other parameters (ring degree, primes or digits)");
  size_t o = 6;
  need(o, C.np());
  for (int i = 0; i < C.np(); i++)
    if (in[o + i] != C.q[i]) throw Error(1, "key checkpoint of another prime chain");
  o += C.np();
  const size_t NPN = (size_t)C.np() * C.N, PK = (size_t)2 * C.L1 * C.N;
  const size_t key_words = (size_t)C.beta_at(C.L1) * 2 * C.np() * C.N;
  need(o, NPN + PK + 1);
  // residues in range: every word below its prime
  for (size_t r = 0; r < (size_t)C.np(); r++)
    for (size_t j = 0; j < C.N; j++)
      if (in[o + r * C.N + j] >= C.q[r]) throw Error(1, "key checkpoint holds a residue out of range");
  DevBuf s(NPN, C.stream), pk(PK, C.stream);
  HE_CUDA(cudaMemcpyAsync(s.p, in + o, NPN * 8, cudaMemcpyHostToDevice, C.stream));
  o += NPN;
  HE_CUDA(cudaMemcpyAsync(pk.p, in + o, PK * 8, cudaMemcpyHostToDevice, C.stream));
  o += PK;
  const u64 nk = in[o++];
  std::map<u64, DevBuf> keys;
  for (u64 t = 0; t < nk; t++) {
    need(o, 2);
    const u64 k = in[o], words = in[o + 1];
    o += 2;
    if (words != key_words || (k != 1 && (k % 2 == 0 || k >= 2 * (u64)C.N)))
      throw Error(1, "key checkpoint holds a malformed switching key");
    need(o, words);
    DevBuf d(words, C.stream);
    HE_CUDA(cudaMemcpyAsync(d.p, in + o, words * 8, cudaMemcpyHostToDevice, C.stream));
    o += words;
    keys[k] = std::move(d);
  }
  HE_CUDA(cudaStreamSynchronize(C.stream));
  C.d_s = std::move(s);
  C.d_pk = std::move(pk);
  C.ksk = std::move(keys);
  C.has_keys = true;
}

void keygen(Ctx& C, const std::vector<long>& steps) {
  const int np = C.np();
  const size_t NPN = (size_t)np * C.N;
  const LimbMap lm = all_primes(C);
  if (!C.has_keys) {
    std::vector<int8_t> s8(C.N);
    sample_small(C, HE_TAG_SECRET, 0, 0, s8.data());
    DevBuf tmp8(C.N / 8 + 1, C.stream);
    upload(C, tmp8.p, s8.data(), C.N);
    C.d_s = DevBuf(NPN, C.stream);
    k_reduce_small(C, (const int8_t*)tmp8.p, C.d_s.p, 1, lm);
    ntt_forward(C, C.d_s.p, 1, lm);
    // public key over Q (computed over all primes, Q limbs kept)
    std::vector<u64> a_host(NPN);
    sample_uniform(C, HE_TAG_PK_A, 0, 0, np, a_host.data());
    std::vector<int8_t> e8(C.N);
    sample_small(C, HE_TAG_PK_E, 0, 0, e8.data());
    DevBuf a(NPN, C.stream), e(NPN, C.stream), b(NPN, C.stream);
    upload(C, a.p, a_host.data(), NPN * 8);
    upload(C, tmp8.p, e8.data(), C.N);
    k_reduce_small(C, (const int8_t*)tmp8.p, e.p, 1, lm);
    ntt_forward(C, a.p, 1, lm);
    ntt_forward(C, e.p, 1, lm);
    k_ksk_combine(C, a.p, e.p, C.d_s.p, b.p, -1);
    C.d_pk = DevBuf((size_t)2 * C.L1 * C.N, C.stream);
    HE_CUDA(cudaMemcpyAsync(C.d_pk.p, b.p, (size_t)C.L1 * C.N * 8, cudaMemcpyDeviceToDevice, C.stream));
    HE_CUDA(cudaMemcpyAsync(C.d_pk.p + (size_t)C.L1 * C.N, a.p, (size_t)C.L1 * C.N * 8, cudaMemcpyDeviceToDevice,
                            C.stream));
    // relinearisation key: s' = s^2
    DevBuf s2(NPN, C.stream);
    k_mul(C, C.d_s.p, C.d_s.p, s2.p, 1, lm);
    C.ksk[1] = make_ksk(C, 0, s2.p);
    HE_CUDA(cudaStreamSynchronize(C.stream));
    C.has_keys = true;
  }
  for (long st : steps) {
    const u64 k = C.galois_elt(st);
    if (k == 1 || C.ksk.count(k)) continue;
    DevBuf sk(NPN, C.stream);
    k_permute(C, C.d_s.p, sk.p, (size_t)np, k);  // phi_k(s)
    DevBuf key = make_ksk(C, k, sk.p);
    // store phi_{k^-1}(key): k^-1 = 5^{-r} mod 2N is the Galois element of step -st
    const u64 kinv = C.galois_elt(-st);
    DevBuf perm(key.words, C.stream);
    k_permute(C, key.p, perm.p, key.words / C.N, kinv);
    C.ksk[k] = std::move(perm);
    HE_CUDA(cudaStreamSynchronize(C.stream));
  }
}

// ---------------------------------------------------------------------------
// encryption / decryption
// ---------------------------------------------------------------------------
std::unique_ptr<CtSet> encrypt_coeffs(Ctx& C, const int64_t* m, int n, int limbs, double scale, u64 id_base) {
  if (!C.has_keys) throw Error(9, "no keys: call he_keygen first");
  if (n < 1 || limbs < 1 || limbs > C.L1) throw Error(1, "bad ciphertext count or level");
  auto out = new_set(C, n, 2, limbs, scale);
  const size_t N = C.N;
  // chunks of at most 32 ciphertexts bound the staging memory
  const int chunk = std::min(n, 32);
  std::vector<int8_t> small((size_t)3 * chunk * N);
  DevBuf d8((size_t)3 * chunk * N / 8 + 1, C.stream), dm((size_t)chunk * N, C.stream);
  DevBuf v((size_t)chunk * limbs * N, C.stream), e0((size_t)chunk * limbs * N, C.stream),
      e1((size_t)chunk * limbs * N, C.stream), mr((size_t)chunk * limbs * N, C.stream);
  const LimbMap lm = limbs_q(limbs, N);
  for (int c0 = 0; c0 < n; c0 += chunk) {
    const int cn = std::min(chunk, n - c0);
    parallel_for((size_t)cn, [&](size_t c) {
      const u64 id = id_base + (u64)(c0 + c);
      sample_small(C, HE_TAG_ENC_V, id, 0, small.data() + c * N);
      sample_small(C, HE_TAG_ENC_E0, id, 0, small.data() + ((size_t)chunk + c) * N);
      sample_small(C, HE_TAG_ENC_E1, id, 0, small.data() + ((size_t)2 * chunk + c) * N);
    });
    upload(C, d8.p, small.data(), (size_t)3 * chunk * N);
    upload(C, dm.p, m + (size_t)c0 * N, (size_t)cn * N * 8);
    const int8_t* p8 = (const int8_t*)d8.p;
    k_reduce_small(C, p8, v.p, cn, lm);
    k_reduce_small(C, p8 + (size_t)chunk * N, e0.p, cn, lm);
    k_reduce_small(C, p8 + (size_t)2 * chunk * N, e1.p, cn, lm);
    k_reduce_signed(C, (const int64_t*)dm.p, mr.p, cn, lm);
    ntt_forward(C, v.p, cn, lm);
    ntt_forward(C, e0.p, cn, lm);
    ntt_forward(C, e1.p, cn, lm);
    ntt_forward(C, mr.p, cn, lm);
    k_encrypt_combine(C, v.p, e0.p, e1.p, mr.p, out->ct(c0), cn, limbs);
    HE_CUDA(cudaStreamSynchronize(C.stream));  // host staging reused by the next chunk
  }
  return out;
}

void decrypt_slots(Ctx& C, const CtSet& s_any, double* out) {
  if (!C.has_keys) throw Error(9, "no secret key in this context");
  std::unique_ptr<CtSet> hold;
  if (s_any.polys == 3) hold = relinearized(C, s_any);  // a relinearised copy
  const CtSet& s = hold ? *hold : s_any;
  if (s.polys != 2) throw Error(1, "decrypt expects two- or three-component ciphertexts");
  const size_t N = C.N, M = N / 2;
  DevBuf m0((size_t)s.n * N, C.stream);
  k_decrypt_limb0(C, s.buf.p, s.limbs, s.n, m0.p);
  LimbMap lm = limbs_q(1, N);
  ntt_inverse(C, m0.p, s.n, lm);
  std::vector<u64> h((size_t)s.n * N);
  HE_CUDA(cudaMemcpyAsync(h.data(), m0.p, h.size() * 8, cudaMemcpyDeviceToHost, C.stream));
  HE_CUDA(cudaStreamSynchronize(C.stream));
  const u64 q0 = C.q[0];
  parallel_for((size_t)s.n, [&](size_t c) {
    std::vector<double> m(N);
    for (size_t j = 0; j < N; j++) {
      const u64 v = h[c * N + j];
      m[j] = v > q0 / 2 ? -(double)(q0 - v) : (double)v;
    }
    decode_real(C, m.data(), s.scale, out + c * M);
  });
}

// After a synchronisation: a kernel whose bounded device-side wait expired has set the status
// word; report it (and clear it) instead of returning its words.
void check_device_status(Ctx& C) {
  u64 st = 0;
  HE_CUDA(cudaMemcpy(&st, C.d_status.p, 8, cudaMemcpyDeviceToHost));
  if (st) {
    HE_CUDA(cudaMemset(C.d_status.p, 0, 8));
    throw Error(6 /* HE_E_TIMEOUT */, "a device-side wait of a tensor-core kernel exceeded its limit");
  }
  if (C.imports.bad) {
    unsigned long long nbad = 0;
    HE_CUDA(cudaMemcpy(&nbad, C.imports.bad, 8, cudaMemcpyDeviceToHost));
    if (nbad) {
      HE_CUDA(cudaMemset(C.imports.bad, 0, 8));
      throw Error(1, std::to_string(nbad) + " residues out of range in an asynchronous import");
    }
  }
}

void export_coeffs(Ctx& C, const CtSet& s, u64* host) {
  DevBuf t(s.buf.words, C.stream);
  HE_CUDA(cudaMemcpyAsync(t.p, s.buf.p, s.buf.words * 8, cudaMemcpyDeviceToDevice, C.stream));
  ntt_inverse(C, t.p, s.n * s.polys, limbs_q(s.limbs, C.N));
  HE_CUDA(cudaMemcpyAsync(host, t.p, s.buf.words * 8, cudaMemcpyDeviceToHost, C.stream));
  HE_CUDA(cudaStreamSynchronize(C.stream));
  check_device_status(C);
}

// copies into host memory cannot be replayed from a graph of the context's stream
static void refuse_under_capture(Ctx& C, const char* what) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HE_CUDA(cudaStreamIsCapturing(C.stream, &cs));
  if (C.capturing || cs != cudaStreamCaptureStatusNone) {
    C.capture_failed = C.capture_failed || C.capturing;
    throw Error(9 /* HE_E_STATE */, std::string(what) + " cannot run inside a capture of the context's stream");
  }
}

uint64_t export_async(Ctx& C, const CtSet& s, u64* host) {
  refuse_under_capture(C, "an export copies to host memory and");
  ExportRing& E = C.exports;
  const uint64_t ticket = E.issued + 1;
  const int k = (int)(ticket % ExportRing::kSlots);
  if (!E.done[k]) HE_CUDA(cudaEventCreateWithFlags(&E.done[k], cudaEventDisableTiming));
  {
    DevBuf t(s.buf.words, C.stream);  // released in stream order after the copy below
    HE_CUDA(cudaMemcpyAsync(t.p, s.buf.p, s.buf.words * 8, cudaMemcpyDeviceToDevice, C.stream));
    ntt_inverse(C, t.p, s.n * s.polys, limbs_q(s.limbs, C.N));
    HE_CUDA(cudaMemcpyAsync(host, t.p, s.buf.words * 8, cudaMemcpyDeviceToHost, C.stream));
  }
  HE_CUDA(cudaEventRecord(E.done[k], C.stream));
  E.seq[k] = ticket;
  E.issued = ticket;
  return ticket;
}

void export_wait(Ctx& C, uint64_t ticket) {
  ExportRing& E = C.exports;
  if (ticket == 0 || ticket > E.issued) throw Error(1, "export ticket not issued by this context");
  if (ticket > E.completed) {
    // the slot holds this ticket or a newer one, which completes after it
    const int k = (int)(ticket % ExportRing::kSlots);
    HE_CUDA(cudaEventSynchronize(E.done[k]));
    E.completed = std::max(E.completed, E.seq[k]);
  }
  check_device_status(C);
}

void export_raw(Ctx& C, const CtSet& s, u64* host) {
  HE_CUDA(cudaMemcpyAsync(host, s.buf.p, s.buf.words * 8, cudaMemcpyDeviceToHost, C.stream));
  HE_CUDA(cudaStreamSynchronize(C.stream));
  check_device_status(C);
}

void export_words(Ctx& C, const CtSet& s, u64* dst, bool on_device) {
  HE_CUDA(cudaMemcpyAsync(dst, s.buf.p, s.buf.words * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          C.stream));
  HE_CUDA(cudaStreamSynchronize(C.stream));
  check_device_status(C);
}

// residues of n_polys polynomials [n_polys][limbs][N] checked against their primes on the device
static void check_residues(Ctx& C, const u64* p, size_t n_polys, int limbs) {
  DevBuf bad(1, C.stream);
  HE_CUDA(cudaMemsetAsync(bad.p, 0, 8, C.stream));
  k_check_range(C, p, n_polys * limbs, limbs, (unsigned long long*)bad.p);
  unsigned long long nbad = 0;
  HE_CUDA(cudaMemcpyAsync(&nbad, bad.p, 8, cudaMemcpyDeviceToHost, C.stream));
  HE_CUDA(cudaStreamSynchronize(C.stream));
  if (nbad) throw Error(1, std::to_string(nbad) + " residues out of range");
}

std::unique_ptr<CtSet> import_coeffs(Ctx& C, const u64* host, int n, int limbs, double scale, bool ntt_domain) {
  if (n < 1 || limbs < 1 || limbs > C.L1) throw Error(1, "bad ciphertext count or level");
  auto s = new_set(C, n, 2, limbs, scale);
  upload(C, s->buf.p, host, s->buf.words * 8);
  // residues are checked on the device before the transform
  check_residues(C, s->buf.p, (size_t)n * 2, limbs);
  if (!ntt_domain) ntt_forward(C, s->buf.p, n * 2, limbs_q(limbs, C.N));
  return s;
}

std::unique_ptr<CtSet> import_async(Ctx& C, const u64* host, int n, int limbs, double scale) {
  if (n < 1 || limbs < 1 || limbs > C.L1) throw Error(1, "bad ciphertext count or level");
  refuse_under_capture(C, "an import copies host data and");
  ImportRing& R = C.imports;
  if (!R.copy) {
    HE_CUDA(cudaStreamCreateWithFlags(&R.copy, cudaStreamNonBlocking));
    for (int k = 0; k < 2; k++) {
      HE_CUDA(cudaEventCreateWithFlags(&R.copied[k], cudaEventDisableTiming));
      HE_CUDA(cudaEventCreateWithFlags(&R.consumed[k], cudaEventDisableTiming));
    }
    HE_CUDA(cudaMalloc(&R.bad, 8));
    HE_CUDA(cudaMemset(R.bad, 0, 8));
  }
  const size_t words = (size_t)n * 2 * limbs * C.N;
  const int k = R.next;
  R.next ^= 1;
  if (R.words[k] < words) {  // grow the buffer once its last reader is done
    if (R.pending[k]) HE_CUDA(cudaEventSynchronize(R.consumed[k]));
    if (R.buf[k]) HE_CUDA(cudaFree(R.buf[k]));
    R.buf[k] = nullptr;
    R.words[k] = 0;
    HE_CUDA(cudaMalloc(&R.buf[k], words * 8));
    R.words[k] = words;
  }
  // the copy waits for the previous reader of the buffer only, not for the context's stream
  if (R.pending[k]) HE_CUDA(cudaStreamWaitEvent(R.copy, R.consumed[k], 0));
  HE_CUDA(cudaMemcpyAsync(R.buf[k], host, words * 8, cudaMemcpyHostToDevice, R.copy));
  HE_CUDA(cudaEventRecord(R.copied[k], R.copy));
  HE_CUDA(cudaStreamWaitEvent(C.stream, R.copied[k], 0));
  auto s = new_set(C, n, 2, limbs, scale);
  k_check_range(C, R.buf[k], (size_t)n * 2 * limbs, limbs, R.bad);  // every limb row
  HE_CUDA(cudaMemcpyAsync(s->buf.p, R.buf[k], words * 8, cudaMemcpyDeviceToDevice, C.stream));
  HE_CUDA(cudaEventRecord(R.consumed[k], C.stream));
  R.pending[k] = true;
  ntt_forward(C, s->buf.p, n * 2, limbs_q(limbs, C.N));
  return s;
}

std::unique_ptr<CtSet> import_words(Ctx& C, const u64* src, bool on_device, int n, int polys, int limbs,
                                    double scale) {
  if (n < 1 || limbs < 1 || limbs > C.L1) throw Error(1, "bad ciphertext count or level");
  if (polys != 2 && polys != 3) throw Error(1, "ciphertexts have two or three components");
  auto s = new_set(C, n, polys, limbs, scale);
  if (on_device)
    HE_CUDA(cudaMemcpyAsync(s->buf.p, src, s->buf.words * 8, cudaMemcpyDeviceToDevice, C.stream));
  else
    upload(C, s->buf.p, src, s->buf.words * 8);
  check_residues(C, s->buf.p, (size_t)n * polys, limbs);
  return s;
}

}  // namespace he
