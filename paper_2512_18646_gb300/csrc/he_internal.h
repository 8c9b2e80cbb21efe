// he_internal.h - internal types of the GB300 RNS-CKKS engine.
//
// Data layout in device memory (all residues uint64 in [0, q), NTT domain
// unless stated):
//   ciphertext set      [n][2][limbs][N]
//   public key          [2][L1][N]
//   switching key       [beta][2][L1 + K][N]   (Q limbs then P limbs)
//   secret              [L1 + K][N]
//   extended digits     [n][beta][limbs + K][N]   (ModUp output)
// A "limb" is the N residues of one polynomial modulo one prime. Limb i of a
// polynomial at level `limbs` uses prime i; extended polynomials append the K
// special primes (global prime indices L1 .. L1+K-1).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "he_arith.cuh"

namespace he {

// Error carried to the C ABI as a status code.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void cuda_check(cudaError_t e, const char* what);
// message returned by he_last_error() on this thread (capi.cpp)
void set_last_error(const std::string& msg);
#define HE_CUDA(x) ::he::cuda_check((x), #x)

struct Ctx;
struct CtSet;

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync on the
// context stream; the pool keeps freed memory for reuse).
struct DevBuf {
  u64* p = nullptr;
  size_t words = 0;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(size_t w, cudaStream_t s);
  ~DevBuf();
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept;
  void reset();
};

// Per-prime constants, one entry per global prime index.
struct PrimeTab {
  Mod mod;
  u64 ninv, ninv_sh;  // N^{-1} mod q and its Shoup companion
  u64 pmod;           // P = p_0 ... p_{K-1} mod q
  u64 one_sh;         // floor(2^64 / q): Shoup companion of 1 (x mod q in [0, 2q) for any word x)
  u64 mont_r, mont_r_sh;  // R = 2^64 mod q (Montgomery radix) and its Shoup companion
  u64 qinv_neg;           // -q^{-1} mod 2^64
  float frd;              // 2^frd_sh / q in fp32: quotient estimates of reduce_fp32
  int frd_sh;             // max(0, bitlen(q) + 9 - 32): the top 32 bits of a value below 2^9 q
};

// Constants of one launch over a batch of limbs. Limb i of each polynomial
// (i < lpp) sits at limb position e = i, or i + gap from position gap_at on
// (a launch that skips limbs gap_at .. gap_at + gap - 1), and uses prime
// base0 + e if e < split, else base1 + e - split.
struct LimbMap {
  int lpp = 1, split = 1, base0 = 0, base1 = 0;
  int gap_at = 1 << 30, gap = 0;
  size_t poly_stride = 0;  // words between consecutive polynomials
  __host__ __device__ int mem(int i) const { return i >= gap_at ? i + gap : i; }
  __host__ __device__ int prime(int i) const {
    const int e = mem(i);
    return e < split ? base0 + e : base1 + (e - split);
  }
};

// Page-locked staging for small host-to-device uploads (weight and constant tables, pointer
// tables): a copy from it returns at once, where a copy from pageable memory can block the host
// until the stream reaches it (and the GPU then idles while the host queues the next launches).
// Slots are reused round-robin once their previous copy's event has completed.
struct Staging {
  static constexpr int kSlots = 16;
  static constexpr size_t kSlotBytes = (size_t)1 << 20;
  void* buf[kSlots] = {};
  cudaEvent_t ev[kSlots] = {};
  bool used[kSlots] = {};
  int next = 0;
  std::mutex mu;
  Staging() = default;
  Staging(const Staging&) = delete;
  Staging& operator=(const Staging&) = delete;
  ~Staging();
};

// Device staging of overlapped imports (he_ctset_import_async): host words are copied into one of
// two device buffers on a copy stream of their own, so that the copy runs while the context's
// stream still computes; the context's stream waits for the copy, checks and takes the words, and
// marks the buffer free for the import after next. Out-of-range residues are counted in `bad` and
// reported at the next synchronisation.
struct ImportRing {
  cudaStream_t copy = nullptr;
  u64* buf[2] = {};
  size_t words[2] = {};
  cudaEvent_t copied[2] = {}, consumed[2] = {};
  bool pending[2] = {};  // consumed[k] recorded since buffer k was last filled
  int next = 0;
  unsigned long long* bad = nullptr;
  ImportRing() = default;
  ImportRing(const ImportRing&) = delete;
  ImportRing& operator=(const ImportRing&) = delete;
  ~ImportRing();
};

// Exports queued by he_ctset_export_async: one event per ticket in a small ring. The context's
// stream runs the exports in order, so a slot re-recorded for a newer ticket still covers the
// older one.
struct ExportRing {
  static constexpr int kSlots = 4;
  cudaEvent_t done[kSlots] = {};
  uint64_t seq[kSlots] = {};  // the ticket last recorded in each slot
  uint64_t issued = 0, completed = 0;
  ExportRing() = default;
  ExportRing(const ExportRing&) = delete;
  ExportRing& operator=(const ExportRing&) = delete;
  ~ExportRing();
};

struct Ctx {
  int device = 0;
  int log_n = 0;
  size_t N = 0;
  int L1 = 0, K = 0, alpha = 1;
  double scale0 = 1.0, sigma = 3.2;
  u64 seed = 0;
  cudaStream_t stream = nullptr;
  std::vector<u64> q;         // host copy, Q then P
  std::vector<PrimeTab> ptab; // host copy
  uint64_t cdt[64];
  int cdt_bound = 0;
  // host FFT tables for encode/decode: e^{2 pi i k / M}, zeta^k (zeta = e^{i pi / N}),
  // and the DFT index t_j = (5^j mod 2N - 1) / 4 of slot j (M = N/2)
  std::vector<double> fft_root, fft_twist;  // interleaved re, im
  std::vector<uint32_t> slot_index;

  // device tables
  DevBuf d_ptab;              // PrimeTab[np] (as words)
  DevBuf d_psi;               // [np][N][2]: psi^{brv(k)} and its Shoup companion
  DevBuf d_ipsi;              // [np][N][2]: psi^{-brv(k)} and its companion
  DevBuf d_up;                // ModUp constants, see modup_table()
  DevBuf d_down;              // ModDown constants
  DevBuf d_rs;                // rescale constants [L1][L1][3]
  DevBuf d_status;            // device status word: nonzero after a bounded device-side wait expired
  bool use_tc = true;         // convolution multiply-accumulate on the tensor cores where it fits
  // bound on the temporaries of one convolution, relinearisation, product or
  // rescale (bytes; 0 = none): larger sets are processed in ciphertext chunks
  // with the same per-ciphertext arithmetic
  size_t work_budget = 0;

  // transform geometry (0: default): column-kernel stages and columns per column block
  int ntt_n1 = 0, ntt_cols = 0;
  // capture of library calls into a CUDA graph (he_graph_begin / he_graph_end): sets made during
  // a capture carry its generation; sets made before it and freed during it are kept here and
  // released after the capture ends (their memory is not the graph's to free)
  bool capturing = false;
  uint64_t capture_gen = 0;
  // a call inside the capture needed a host upload (refused): he_graph_end then fails
  bool capture_failed = false;
  std::vector<std::unique_ptr<CtSet>> deferred;

  Staging staging;
  ImportRing imports;
  ExportRing exports;

  // keys
  bool has_keys = false;
  DevBuf d_s;                 // secret [L1+K][N], NTT domain
  DevBuf d_pk;                // [2][L1][N]
  std::map<u64, DevBuf> ksk;  // Galois element (1 = relinearisation) -> key

  int np() const { return L1 + K; }
  int beta_at(int limbs) const { return (limbs + alpha - 1) / alpha; }
  const PrimeTab* dev_ptab() const { return reinterpret_cast<const PrimeTab*>(d_ptab.p); }
  u64 galois_elt(long step) const;
  const DevBuf& key(u64 k) const;
};

// A set of n ciphertexts (or three-component products) at one level.
struct CtSet {
  Ctx* ctx = nullptr;
  int n = 0, polys = 2, limbs = 0;
  double scale = 1.0;
  uint64_t gen = 0;  // capture generation at creation (0: made outside any capture)
  DevBuf buf;
  size_t ct_words() const { return (size_t)polys * limbs * ctx->N; }
  u64* ct(int i) const { return buf.p + (size_t)i * ct_words(); }
};

// ---- launch accounting (profile.cpp): every kernel launch is bracketed ----
// bytes: the launch's algorithmic traffic (each operand read or written once);
// products: its modular products (64 x 64-bit multiplications followed by a
// reduction or accumulated for one)
void* prof_begin(const char* name, cudaStream_t st, double bytes, double products = 0.0);
void prof_end(void* tok, cudaStream_t st);
// count n kernel launches made by replaying a graph
void prof_add_launches(uint64_t n);

// ---- kernel launchers (kernels.cu / ntt.cu) ----
void ntt_forward(const Ctx& C, u64* data, int n_polys, const LimbMap& lm);
// whether the transform supports n1 column stages (log_n - n1 row stages) with `cols` columns per block
bool ntt_geometry_ok(int log_n, int n1, int cols);
void ntt_inverse(const Ctx& C, u64* data, int n_polys, const LimbMap& lm);
// rescale of `rows` polynomials x [rows][lp][N] whose limb lp - 1 is already in the
// coefficient domain: out [rows][lp - 1][N] = (x_i - NTT_i(expanded last limb)) q_l^{-1};
// with addc [all rows][lp - 1], output row r (row0 + r of the whole set) also gains the
// constant addc[(row0 + r) (lp - 1) + i] in limb i
void ntt_forward_rescale(const Ctx& C, u64* out, u64* x, int rows, int lp, const u64* addc = nullptr,
                         int row0 = 0);
// inverse transform of n_polys polynomials [n_polys][lp][N] over q_0..q_{lp-1}, ending with
// the factor N^{-1} (D_j/q_i)^{-1} mod q_i (the first step of ModUp's base conversion); with
// `src`, polynomial p is read from src + p src_stride (not modified) and the result written to
// data
void ntt_inverse_qscaled(const Ctx& C, u64* data, int n_polys, int lp, const u64* src = nullptr,
                         size_t src_stride = 0);
// ModUp of one digit fused into the forward transform of its extended limbs: polynomial p,
// launch limb i (position lm.mem(i)) gets sum_{t < cnt} yt[p ystride + t N] hat[t hstride +
// lm.mem(i)] and is transformed; lm skips the digit's own limbs
void ntt_forward_modup(const Ctx& C, u64* ext_digit, int n, const LimbMap& lm, const u64* yt, size_t ystride,
                       const u64* hat, int hstride, int cnt);
// inverse transform of n_polys P-part polynomials [n_polys][K][N], ending with the
// factor N^{-1} (P/p_k)^{-1} mod p_k (the first step of ModDown's base conversion)
void ntt_inverse_pscaled(const Ctx& C, u64* data, int n_polys);
// ModDown of the n ciphertexts of one key-switch step, fused into the forward
// transform of z = BConv_{P->Q}(yt): yt [n][2][K][N] from ntt_inverse_pscaled, z
// scratch [n][2][lp][N], u the inner products [n][2][nb][N]; writes
// out[c][comp] = (u_Q[pi_gk] - z) P^{-1} + base term (kmode 0: base[c][comp];
// kmode 1: comp 0 gets base[c][0][pi_gk]), ciphertext c at out + c out_stride
void ntt_forward_moddown(const Ctx& C, u64* z, const u64* yt, int n, int lp, const u64* u, int nb, const u64* base,
                         size_t base_stride, u64* out, size_t out_stride, u64 gk, int kmode);
inline LimbMap limbs_q(int limbs, size_t N) {  // plain polynomials, primes 0..limbs-1
  LimbMap m;
  m.lpp = limbs; m.split = limbs; m.base0 = 0; m.base1 = 0; m.poly_stride = (size_t)limbs * N;
  return m;
}

// int64 coefficients [n][N] (device) -> residues [n][limbs][N] for primes of lm
void k_reduce_signed(const Ctx& C, const int64_t* in, u64* out, int n, const LimbMap& lm);
// small signed coefficients given as int8 [n][N] -> residues
void k_reduce_small(const Ctx& C, const int8_t* in, u64* out, int n, const LimbMap& lm);

// out = (v * pk + e + m) per limb, NTT domain; ct [n][2][limbs][N]
void k_encrypt_combine(const Ctx& C, const u64* v, const u64* e0, const u64* e1, const u64* m, u64* ct, int n,
                       int limbs);
// key digit combine: b = -a s + e + (i in digit ? pmod_i s' : 0) over the QP basis
void k_ksk_combine(const Ctx& C, const u64* a, const u64* e, const u64* sprime, u64* b, int digit);
// out = a * b pointwise (all over QP or Q basis rows with prime map)
void k_mul(const Ctx& C, const u64* a, const u64* b, u64* out, int n_polys, const LimbMap& lm);
// NTT-domain Galois permutation: out[j] = in[pi_k(j)] per limb (rows of N)
void k_permute(const Ctx& C, const u64* in, u64* out, size_t rows, u64 k);
// decrypt q_0 limb: m0 = c0 + c1 s (limb 0), n ciphertexts -> [n][N] (NTT domain)
void k_decrypt_limb0(const Ctx& C, const u64* ct, int limbs, int n, u64* out);
void k_add(const Ctx& C, const u64* a, const u64* b, u64* out, int n_polys, int limbs);
// d[n][3][limbs] = tensor(a[n][2], b[n][2])
void k_tensor(const Ctx& C, const u64* a, const u64* b, u64* d, int n, int limbs);
// key pointers of up to 8 steps for one inner-product launch
struct KeyPtrs {
  const u64* k[8];
};
// u[s][n][2][limbs+K] = sum_j ext[n][j] * key_s[j]  (NTT domain), s < S; digit j's own limbs
// (positions j alpha ..) are read from the input polynomial own + c own_stride instead of ext
void k_ks_inner(const Ctx& C, const u64* ext, const u64* own, size_t own_stride, const KeyPtrs& keys, int S, u64* u,
                int n, int limbs);
// gather P limbs of u (permuted by pi_k) into p [n][2][K][N]
void k_gather_p(const Ctx& C, const u64* u, u64* p, int n, int limbs, u64 k);
// rescale helpers
void k_rescale_expand(const Ctx& C, const u64* last_coeff, u64* r, int rows, int limbs);
void k_rescale_combine(const Ctx& C, const u64* x, const u64* r, u64* out, int rows, int limbs);
// add integer constants to polynomial 0 of each ciphertext (NTT domain);
// c_dev [n / per_group][limbs]: ciphertext c gets row c / per_group
void k_add_const(const Ctx& C, u64* ct, int n, int limbs, const u64* c_dev, int per_group);
// out = in * w mod q_i for rows [rows][limbs][N]; wsh [limbs][2] (residue, Shoup companion)
void k_mul_const(const Ctx& C, const u64* in, u64* out, size_t rows, int limbs, const u64* wsh);
// y[c][comp] += v[c][comp], comp < 2 (y with ypolys components, v with two)
void k_add_comps(const Ctx& C, u64* y, const u64* v, int n, int ypolys, int limbs);
// conv MAC: out[o][j'] = sum_{c,b,a} W * R[c][s j' + b][a]
// the same on the tensor cores (conv_tc.cu) for the limbs of one class (narrow: primes below
// kMac96Prime), reading the rotations column-major ([j][c][a]); conv_mac_tc_all: the context
// allows it, the chunk sums of this shape stay exact in fp32 and the weight tiles fit shared
// memory, for every class of the lp limbs
// one CTA waits on a barrier nothing arrives on for limit_ns, then records the failure in the status word
void k_wait_expires(const Ctx& C, uint64_t limit_ns);
bool conv_mac_tc_all(const Ctx& C, int c_in, int k, int c_out, int lp);
void k_conv_mac_tc(const Ctx& C, const u64* rot, u64* out, const u64* w, int c_in, int w_in, int k, int stride,
                   int c_out, int w_out, int limbs, bool narrow);
void check_device_status(Ctx& C);
extern std::atomic<int> g_fail_allocs;
// colmajor: rot in the tensor-core order [j][c][a] (the tensor cores then run every class of
// limbs), else [c][j][a] for the CUDA-core kernels
void k_conv_mac(const Ctx& C, const u64* rot, u64* out, const u64* w, int c_in, int w_in, int k, int stride,
                int c_out, int w_out, int limbs, bool colmajor);
// conv MAC with encrypted kernels: out[o][j'] (3 components) = sum_{c,b,a} tensor(W[o][c][a][b], R[c][s j' + b][a])
void k_conv_enc_mac(const Ctx& C, const u64* rot, const u64* W, u64* out, int c_in, int w_in, int k, int stride,
                    int c_out, int w_out, int limbs);
// matmul accumulate: d[idx] = sum_k tensor(A_k, R[k][idx]), idx < p; R holds rstride (default p)
// ciphertexts per k
void k_matmul_acc(const Ctx& C, const u64* A, const u64* R, u64* d, int n, int p, int limbs, int rstride = 0);
// up to kSetBlock device ranges passed by value to a kernel (so captured graphs replay them):
// range t starts at p[t] and spans off[t+1] - off[t] words (or ciphertexts, per use)
constexpr int kSetBlock = 128;
struct SetPtrs {
  const u64* p[kSetBlock];
  size_t off[kSetBlock + 1];
};
// T <= kSetBlock products in one launch: d[(t0 + t) p + i0 + idx] = sum_{k < n_t} tensor(A_t[k],
// R[off[t] + k][idx]), idx < ci, n_t = A.off[t+1] - A.off[t] (ciphertexts)
void k_matmul_acc_multi(const Ctx& C, const SetPtrs& A, const u64* R, u64* d, int T, int t0, int p, int i0, int ci,
                        int limbs);
// dir 0: base + off[t] <- p[t]; dir 1: p[t] <- base + off[t] (off in words), T <= kSetBlock ranges, one launch
void k_move_words(const Ctx& C, const SetPtrs& P, u64* base, int T, int dir);
// zero-rotation matmul accumulate: d[g] = sum_k tensor(Ahat[g][k], B[k]), g < G
void k_volley_acc(const Ctx& C, const u64* Ah, const u64* B, u64* d, int n, int G, int limbs);
// fc MAC: out[o] = sum_{cj} pt[o][cj] * X[cj], every one of the `polys` components
// pt: [out_dim][pt_cols][limbs][N]; the n_in input columns are the first n_in of each row of pt
void k_fc_mac(const Ctx& C, const u64* X, const u64* pt, u64* out, int n_in, int pt_cols, int out_dim, int limbs,
              int polys);
// slot-block packing: out[j] = sum_t masks[t] * xs[t][j] ([n_ct][2][limbs][N]); xs is a device array of T pointers
// (ct_stride: words between the ciphertexts of one set, 0 = contiguous)
void k_pack_blocks(const Ctx& C, const u64* const* xs, const u64* masks, int T, int n_ct, int limbs, u64* out,
                   size_t ct_stride = 0);
// data[p][i] *= R mod q (Montgomery form) for the primes of lm
void k_mont_form(const Ctx& C, u64* data, int n_polys, const LimbMap& lm);
// calibration: blocks x threads x 8 chains x iters Shoup products modulo q_0
void k_calib_shoup(const Ctx& C, u64* sink, int blocks, int threads, int iters);
void k_calib_mac96(const Ctx& C, u64* sink, int blocks, int threads, int iters);
// calibration of the forward butterfly of the transforms (narrow: primes below kNarrowPrime)
void k_calib_bfly(const Ctx& C, u64* sink, int blocks, int threads, int iters, bool narrow);
// number of residues >= q_i in rows of limbs (limb = row % limbs), added to *bad
void k_check_range(const Ctx& C, const u64* x, size_t rows, int limbs, unsigned long long* bad);
// copy groups x rows_per_group limbs: row r of group g at src + g src_gs + r N
void k_copy_limbs(const Ctx& C, const u64* src, size_t src_gs, u64* dst, size_t dst_gs, size_t groups,
                  int rows_per_group);

// ---- host-side building blocks (context.cpp / eval.cpp) ----
void ctx_init(Ctx& C, int log_n, const std::vector<int>& q_bits, int n_special, int special_bits, int alpha,
              double log_scale, double sigma, u64 seed, cudaStream_t st);
void keygen(Ctx& C, const std::vector<long>& steps);
// key checkpoint (he_keys_export / he_keys_import); out == nullptr: the size in words
size_t keys_export(Ctx& C, u64* out, size_t cap);
void keys_import(Ctx& C, const u64* in, size_t n);
std::unique_ptr<CtSet> new_set(Ctx& C, int n, int polys, int limbs, double scale);
std::unique_ptr<CtSet> encrypt_coeffs(Ctx& C, const int64_t* m, int n, int limbs, double scale, u64 id_base);
void decrypt_slots(Ctx& C, const CtSet& s, double* out);
void export_coeffs(Ctx& C, const CtSet& s, u64* host);
// export_coeffs without waiting: returns the ticket export_wait takes
uint64_t export_async(Ctx& C, const CtSet& s, u64* host);
// block until the export with this ticket (and every earlier one) has reached the host
void export_wait(Ctx& C, uint64_t ticket);
// device words as held (NTT domain) to host
void export_raw(Ctx& C, const CtSet& s, u64* host);
// the words as held to a host or device buffer (completed on return)
void export_words(Ctx& C, const CtSet& s, u64* dst, bool on_device);
// n ciphertexts of `polys` components from NTT-domain words [n][polys][limbs][N] in a host or device
// buffer, range-checked
std::unique_ptr<CtSet> import_words(Ctx& C, const u64* src, bool on_device, int n, int polys, int limbs,
                                    double scale);
// he_ctset_import without waiting: the copy overlaps the work already queued on the context's
// stream; range errors are reported at the next synchronisation
std::unique_ptr<CtSet> import_async(Ctx& C, const u64* host, int n, int limbs, double scale);
// [n][2][limbs][N] residues, coefficient domain (or already NTT domain), range-checked
std::unique_ptr<CtSet> import_coeffs(Ctx& C, const u64* host, int n, int limbs, double scale,
                                     bool ntt_domain = false);

// ModUp of polynomial 1 of every ciphertext: ext [n][beta][limbs+K][N], NTT domain, except
// each digit's own limbs, which are left unset (they equal the input polynomial's limbs)
DevBuf modup_c1(Ctx& C, const CtSet& in);
// Rot by each step from a ModUp made by modup_c1; out ciphertext (c, s) at
// out + (c * out_cts_per_ct + s) * ct_words
void rotate_from_ext(Ctx& C, const CtSet& in, const DevBuf& ext, const std::vector<long>& steps, u64* out,
                     int out_cts_per_ct);
std::unique_ptr<CtSet> rotate(Ctx& C, const CtSet& in, const std::vector<long>& steps);
// three components -> two (key switch of d2 with the relinearisation key); no rescale
void relinearize(Ctx& C, CtSet& s);
std::unique_ptr<CtSet> relinearized(Ctx& C, const CtSet& s);
// rescale in place; addc [n polys][limbs - 1] (optional): after the rescale, polynomial r of
// the set gains the constant addc[r (limbs - 1) + i] in limb i (e.g. a bias on component 0)
void rescale_inplace(Ctx& C, CtSet& s, const u64* addc = nullptr);
std::unique_ptr<CtSet> conv2d(Ctx& C, const CtSet& in, int c_in, int gap, const double* W, const double* bias,
                              int c_out, int k, int stride);
// convolution with encrypted kernels Wct [c_out][c_in][k][k] (constants at scale q_{limbs-1})
std::unique_ptr<CtSet> conv2d_enc(Ctx& C, const CtSet& in, int c_in, int gap, const CtSet& Wct, const double* bias,
                                  int c_out, int k, int stride);
// diagonals idx in [lo, hi) of the revolver product (hi <= 0: up to p); hi - lo ciphertexts
std::unique_ptr<CtSet> matmul(Ctx& C, const CtSet& A, const CtSet& B, int p, int lo = 0, int hi = 0);
// vRot (Alg. 5) by r inside rows of images of hw slots; masks [2][lp][N] (F1, F2; NTT domain); one level
std::unique_ptr<CtSet> vrot(Ctx& C, const CtSet& in, long r, int hw, const u64* masks);
// Alg. 3 with one ciphertext per operand: E [lp-1][N] column-0 mask, F [p][lp-2][N] (NTT domain); three levels
std::unique_ptr<CtSet> vr_matmul(Ctx& C, const CtSet& A, const CtSet& Bbar, int n, int p, const u64* E, const u64* F);
// Alg. 4 over one-ciphertext image blocks of width Wb: S [k^2] kernel ciphertexts (scale q_{l-1}), bias one
// ciphertext two levels down, masks [k^2][l-1][N] offset masks (NTT domain); two levels
std::unique_ptr<CtSet> vr_conv2d(Ctx& C, const CtSet& in, const CtSet& S, const CtSet& bias, int k, int Wb,
                                 const u64* masks);
// ReForm: rows at gap `gap` (slots b H + gap i, i < h) moved to gap 1; masks [h][limbs][N] (NTT domain,
// 0/1 at slots b H + i, scale q_{limbs-1}); one level
std::unique_ptr<CtSet> reform(Ctx& C, const CtSet& in, int gap, int h, const u64* masks);
// baby-step giant-step revolver with baby-step size g: D [p] as matmul's
std::unique_ptr<CtSet> matmul_bsgs(Ctx& C, const CtSet& A, const CtSet& B, int p, int g);
// zero-rotation matmul: Ahat [G][n] (group-major volley encoding of A), B [n] -> D [G]
std::unique_ptr<CtSet> matmul_volley(Ctx& C, const CtSet& Ahat, const CtSet& B);
// block stride M, positions per ciphertext and groups of the volley layout (throws on misfit)
void volley_geometry(long slots, int m, int p, int& M, int& per, int& G);
std::vector<std::unique_ptr<CtSet>> matmul_batched(Ctx& C, const std::vector<const CtSet*>& As,
                                                   const std::vector<const CtSet*>& Bs, const std::vector<int>& ps);
std::unique_ptr<CtSet> square(Ctx& C, const CtSet& in);
// degree-3 activation c0 + c1 x + c2 x^2 + c3 x^3 (coeffs c[0..3]); two levels, three components out
// host -> device copy on the context stream through the staging slots (pageable copy during a
// capture, which refuses it, or above a slot's size); src may be reused when the call returns
void upload_async(Ctx& C, void* dst, const void* src, size_t bytes);
std::unique_ptr<CtSet> drop_limbs(Ctx& C, const CtSet& x, int limbs);
void add_plain(Ctx& C, CtSet& x, const int64_t* m, int n_vec);
std::unique_ptr<CtSet> poly_act3(Ctx& C, const CtSet& x, const double* c);

std::unique_ptr<CtSet> mul(Ctx& C, const CtSet& a, const CtSet& b);
std::unique_ptr<CtSet> add(Ctx& C, const CtSet& a, const CtSet& b);
std::unique_ptr<CtSet> fc_apply(Ctx& C, const CtSet& in, const u64* pts, int out_dim, int gap, int block_stride,
                                const double* bias);
// the dense layer's sums over input columns [first, first + in.n) of pts [out_dim][pt_cols][limbs][N],
// before the rescale (scale field: the input's; the sums carry the plaintexts' factor q_l)
std::unique_ptr<CtSet> fc_partial(Ctx& C, const CtSet& in, const u64* pts, int out_dim, int pt_cols, int first);
// the rest of the dense layer on full sums, in place: rescale, relinearisation, rotate-and-add, bias
void fc_finish(Ctx& C, CtSet& z, int gap, int block_stride, const double* bias);
DevBuf fc_prepare(Ctx& C, const int64_t* pts_host, int out_dim, int n_in, int limbs);
// rescale(sum_t masks[t] * X_t): T sets of n_ct two-component ciphertexts at `limbs` limbs
// (device pointers xs[t]), masks [T][limbs][N] encoded at scale q_{limbs-1}; result at `scale`
std::unique_ptr<CtSet> pack_blocks(Ctx& C, const std::vector<const u64*>& xs, int n_ct, int limbs, double scale,
                                   const u64* masks);

// f(0) .. f(n-1) on up to 16 host threads (independent items)
template <class F>
void host_parallel(size_t n, F f) {
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

// host encode/decode (encode.cpp): real slot vector -> integer coefficients
void encode_real(const Ctx& C, const double* z, size_t nz, double scale, int64_t* m);
void decode_real(const Ctx& C, const double* m, double scale, double* z);

// Live handles of the C ABI (contexts, ciphertext sets, plaintext sets, graphs, servers): a
// handle registers itself when it is made and leaves the registry when it is freed; every entry
// point checks its handle arguments against the registry before it reads them, so an unknown,
// corrupted or already freed handle is refused with HE_E_ARG instead of being dereferenced.
enum HandleKind { kHCtx = 1, kHSet, kHPts, kHGraph, kHServer };
void handle_add(const void* h, int kind);
void handle_remove(const void* h);
bool handle_is(const void* h, int kind);

}  // namespace he

struct he_ctx {
  he::Ctx c;
  he_ctx() { he::handle_add(this, he::kHCtx); }
  ~he_ctx() { he::handle_remove(this); }
};
struct he_ctset {
  std::unique_ptr<he::CtSet> s;
  he_ctset() { he::handle_add(this, he::kHSet); }
  ~he_ctset() { he::handle_remove(this); }
};
struct he_graph {
  he_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernel nodes, added to the launch counter per replay
  he_graph() { he::handle_add(this, he::kHGraph); }
  ~he_graph() { he::handle_remove(this); }
};
struct he_ptset {
  he::Ctx* ctx = nullptr;
  int out_dim = 0, n_in = 0, limbs = 0, gap = 1, block_stride = 1;
  he::DevBuf buf;  // [out_dim][n_in][limbs][N]
  he_ptset() { he::handle_add(this, he::kHPts); }
  ~he_ptset() { he::handle_remove(this); }
};
struct he_server;
inline bool handle_live(const he_ctx* h) { return he::handle_is(h, he::kHCtx); }
inline bool handle_live(const he_ctset* h) { return he::handle_is(h, he::kHSet); }
inline bool handle_live(const he_graph* h) { return he::handle_is(h, he::kHGraph); }
inline bool handle_live(const he_ptset* h) { return he::handle_is(h, he::kHPts); }
inline bool handle_live(const he_server* h) { return he::handle_is(h, he::kHServer); }
#define HANDLE(p)                                                                                   \
  do {                                                                                              \
    if ((p) && !handle_live(p)) throw he::Error(1 /* HE_E_ARG */, "invalid handle (unknown or freed): " #p); \
  } while (0)
