// eval.cpp - homomorphic operations and the paper's multi-ciphertext layers,
// as sequences of the kernels in kernels.cu / ntt.cu on the context stream.
//
// Canonical schedules (both this library and any checker must follow them for
// bit-identical ciphertexts):
//  - Rot(ct, l) (Sec. II-A): ModUp of c1 once per ciphertext; per step, the
//    automorphism on every extended digit, inner product with the Galois key,
//    ModDown; result (phi_k(c0) + v0, v1).
//  - Mul (Sec. II-A): tensor product, then rescale by the last prime; the
//    three-component result is relinearised (key switch of d2) only when an
//    operation needs two components: a rotation, a convolution input, a
//    matmul operand, the end of a dense layer, decryption.
//  - matmul (Alg. 3 over n ciphertexts per operand, Sec. IV-A): hoisted
//    rotations of every B~_k by idx = 0..p-1 (RowShifter applied idx times
//    equals Rot(., idx) under whole-ring period-p tiling, Sec. III-B); per idx
//    the n tensor products summed as three components (the SumColVec of
//    Alg. 3 becomes ciphertext additions), one rescale, one relinearisation.
//  - conv (Alg. 4 over the column layout, Sec. IV-B): hoisted rotations of
//    every input column by gap*a, a < k; output (o, j') =
//    sum_{c,b,a} round(K[o][c][a][b] q_l) Rot(X_{c, s j' + b}, gap a);
//    rescale; + round(bias_o * scale).
//  - FC: sum_{c,j} pt_{o,c,j} X_{c,j} component by component (two or three
//    components); rescale; relinearise; rotate-and-add over gap, 2 gap, ...,
//    block/2; + round(bias_o * scale).
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "he_internal.h"

namespace he {

static LimbMap ext_map(const Ctx& C, int limbs) {
  LimbMap m;
  m.lpp = limbs + C.K; m.split = limbs; m.base0 = 0; m.base1 = C.L1;
  m.poly_stride = (size_t)(limbs + C.K) * C.N;
  return m;
}

static u64 residue_of(int64_t v, u64 q) {
  const int64_t r = v % (int64_t)q;
  return r < 0 ? (u64)(r + (int64_t)q) : (u64)r;
}

// ModUp of polynomial `poly` of every ciphertext of a set (inverse NTT into a
// scratch buffer, base conversion per digit, forward NTT of the extended limbs).
static DevBuf modup_poly(Ctx& C, const CtSet& in, int poly) {
  const int n = in.n, lp = in.limbs, beta = C.beta_at(lp), nb = lp + C.K;
  const size_t N = C.N;
  // the polynomial to the coefficient domain, each limb times N^{-1} (D_j/q_i)^{-1} (the first
  // pass reads the set, the result goes to x)
  DevBuf x((size_t)n * lp * N, C.stream);
  ntt_inverse_qscaled(C, x.p, n, lp, in.buf.p + (size_t)poly * lp * N, in.ct_words());
  DevBuf ext((size_t)n * beta * nb * N, C.stream);
  const ulonglong2* hat_level = reinterpret_cast<const ulonglong2*>(C.d_up.p + (size_t)(C.L1 + 1) * C.L1 * 2) +
                                (size_t)lp * C.L1 * (C.L1 + C.K);
  for (int j = 0; j < beta; j++) {
    const int lo = j * C.alpha, cnt = std::min(C.alpha, lp - lo);
    // the digit's own limbs are the input itself (the inner product reads them there); the
    // others: base conversion in the load of their forward transform
    LimbMap m = ext_map(C, lp);
    m.lpp = nb - cnt;
    m.gap_at = lo;
    m.gap = cnt;
    m.poly_stride = (size_t)beta * nb * N;
    ntt_forward_modup(C, ext.p + (size_t)j * nb * N, n, m, x.p + (size_t)lo * N, (size_t)lp * N,
                      reinterpret_cast<const u64*>(hat_level + (size_t)lo * (C.L1 + C.K)), C.L1 + C.K, cnt);
  }
  return ext;
}

DevBuf modup_c1(Ctx& C, const CtSet& in) { return modup_poly(C, in, 1); }

// Inner products of the ModUp digits `ext` (of set `in`) with the keys of the
// Galois elements ks[s] (1 = relinearisation key), then ModDown, for all steps
// together: the digits are read once per group of up to 8 keys, and the P-limb
// transforms, base conversions and Q-limb transforms of every step share one
// launch each. mode 0: add the set's first two components (relinearisation of
// d2); mode 1: add phi_k(c0). Output ciphertext c of step s goes to
// outs[s] + c * out_stride.
static void ks_finish(Ctx& C, const CtSet& in, int poly, const DevBuf& ext, const std::vector<u64>& ks, int mode,
                      const std::vector<u64*>& outs, size_t out_stride) {
  const int n = in.n, lp = in.limbs, nb = lp + C.K, S = (int)ks.size();
  if (S == 0) return;
  const size_t N = C.N;
  const size_t ustep = (size_t)n * 2 * nb * N, pstep = (size_t)n * 2 * C.K * N, zstep = (size_t)n * 2 * lp * N;
  DevBuf u((size_t)S * ustep, C.stream);
  for (int s0 = 0; s0 < S; s0 += 8) {
    const int cs = std::min(8, S - s0);
    KeyPtrs kp{};
    for (int t = 0; t < cs; t++) kp.k[t] = C.key(ks[s0 + t]).p;
    k_ks_inner(C, ext.p, in.buf.p + (size_t)poly * lp * N, in.ct_words(), kp, cs, u.p + s0 * ustep, n, lp);
  }
  // ModDown: the P part (permuted by the step's automorphism) to the coefficient domain, scaled
  // for the base conversion; the conversion, forward transform and combine run as one transform
  DevBuf pl((size_t)S * pstep, C.stream);
  for (int s = 0; s < S; s++) k_gather_p(C, u.p + s * ustep, pl.p + s * pstep, n, lp, ks[s]);
  ntt_inverse_pscaled(C, pl.p, S * n * 2);
  DevBuf z(zstep, C.stream);
  for (int s = 0; s < S; s++)
    ntt_forward_moddown(C, z.p, pl.p + s * pstep, n, lp, u.p + s * ustep, nb, in.buf.p, in.ct_words(), outs[s],
                        out_stride, ks[s], mode);
}

void rotate_from_ext(Ctx& C, const CtSet& in, const DevBuf& ext, const std::vector<long>& steps, u64* out,
                     int out_cts_per_ct) {
  const size_t cw = in.ct_words();
  std::vector<u64> ks;
  std::vector<u64*> outs;
  for (size_t s = 0; s < steps.size(); s++) {
    const u64 k = C.galois_elt(steps[s]);
    u64* o = out + s * cw;
    if (k == 1) {
      k_copy_limbs(C, in.buf.p, cw, o, cw * out_cts_per_ct, (size_t)in.n, 2 * in.limbs);
      continue;
    }
    ks.push_back(k);
    outs.push_back(o);
  }
  ks_finish(C, in, 1, ext, ks, 1, outs, cw * out_cts_per_ct);
}

// Ciphertexts [first, first + n) of a set, without owning their memory.
struct SetView {
  CtSet s;
  SetView(const CtSet& src, int first, int n) {
    s.ctx = src.ctx;
    s.n = n;
    s.polys = src.polys;
    s.limbs = src.limbs;
    s.scale = src.scale;
    s.buf.p = src.ct(first);
    s.buf.words = (size_t)n * src.ct_words();
    s.buf.st = src.buf.st;
  }
  ~SetView() {
    s.buf.p = nullptr;
    s.buf.words = 0;
  }
  SetView(const SetView&) = delete;
  SetView& operator=(const SetView&) = delete;
};

// Items per chunk when each item needs `bytes_per_item` of temporaries.
static int chunk_items(const Ctx& C, int n_items, double bytes_per_item) {
  if (C.work_budget == 0 || bytes_per_item <= 0) return std::max(n_items, 1);
  const double k = std::floor((double)C.work_budget / bytes_per_item);
  return (int)std::max(1.0, std::min((double)n_items, k));
}

std::unique_ptr<CtSet> relinearized(Ctx& C, const CtSet& s) {
  if (s.polys != 3) throw Error(1, "relinearisation expects three-component ciphertexts");
  auto out = new_set(C, s.n, 2, s.limbs, s.scale);
  const int lp = s.limbs, nb = lp + C.K, beta = C.beta_at(lp);
  // per ciphertext: the d2 copy, its ModUp digits, the key sums, their P part, the ModDown result
  const double per = 8.0 * C.N * (lp + (double)beta * nb + 2.0 * nb + 2.0 * C.K + 2.0 * lp);
  const int step = chunk_items(C, s.n, per);
  for (int c0 = 0; c0 < s.n; c0 += step) {
    const int cn = std::min(step, s.n - c0);
    SetView v(s, c0, cn);
    DevBuf ext = modup_poly(C, v.s, 2);
    ks_finish(C, v.s, 2, ext, {1}, 0, {out->ct(c0)}, out->ct_words());
  }
  return out;
}

void relinearize(Ctx& C, CtSet& s) {
  if (s.polys == 2) return;
  auto out = relinearized(C, s);
  s.buf = std::move(out->buf);
  s.polys = 2;
}

// A two-component view of `in`: the set itself, or a relinearised copy.
static const CtSet& two_comp(Ctx& C, const CtSet& in, std::unique_ptr<CtSet>& hold) {
  if (in.polys == 2) return in;
  hold = relinearized(C, in);
  return *hold;
}

// Rotations of the input columns of c_in channels (in: [c][j], w_in columns each), stored for the
// tensor-core convolution: the rotation by steps[a] of column j of channel c at ciphertext
// (j c_in + c) k + a, so that the c_in k^2 terms of one output column are consecutive
// ciphertexts. One ModUp for all inputs; the key switches run per channel on views of it.
static std::unique_ptr<CtSet> rotate_colmajor(Ctx& C, const CtSet& in, int c_in, const std::vector<long>& steps) {
  const int w_in = in.n / c_in, k = (int)steps.size();
  for (long s : steps)
    if (C.galois_elt(s) != 1) C.key(C.galois_elt(s));
  auto out = new_set(C, in.n * k, 2, in.limbs, in.scale);
  bool any = false;
  for (long s : steps) any |= C.galois_elt(s) != 1;
  DevBuf ext;
  if (any) ext = modup_c1(C, in);
  const size_t ext_ct = (size_t)C.beta_at(in.limbs) * (in.limbs + C.K) * C.N;
  const size_t cw = in.ct_words();
  for (int c = 0; c < c_in; c++) {
    SetView v(in, c * w_in, w_in);
    DevBuf ev;  // a view of channel c's digits (not owned)
    if (ext.p) {
      ev.p = ext.p + (size_t)c * w_in * ext_ct;
      ev.words = (size_t)w_in * ext_ct;
      ev.st = ext.st;
    }
    rotate_from_ext(C, v.s, ev, steps, out->buf.p + (size_t)c * k * cw, c_in * k);
    ev.p = nullptr;
    ev.words = 0;
  }
  return out;
}

std::unique_ptr<CtSet> rotate(Ctx& C, const CtSet& in_any, const std::vector<long>& steps) {
  std::unique_ptr<CtSet> hold;
  const CtSet& in = two_comp(C, in_any, hold);
  for (long s : steps)
    if (C.galois_elt(s) != 1) C.key(C.galois_elt(s));
  const int S = (int)steps.size();
  auto out = new_set(C, in.n * S, 2, in.limbs, in.scale);
  bool any = false;
  for (long s : steps) any |= C.galois_elt(s) != 1;
  DevBuf ext;
  if (any) ext = modup_c1(C, in);
  rotate_from_ext(C, in, ext, steps, out->buf.p, S);
  return out;
}

// rows polynomials of lp limbs (x) -> rescaled polynomials of lp - 1 limbs (out).
// The last limb of x is transformed in place (x is consumed).
static void rescale_rows(Ctx& C, u64* x, int rows, int lp, u64* out, const u64* addc = nullptr, int row0 = 0) {
  const size_t N = C.N;
  LimbMap lm1;
  lm1.lpp = 1; lm1.split = 1; lm1.base0 = lp - 1; lm1.base1 = 0; lm1.poly_stride = (size_t)lp * N;
  ntt_inverse(C, x + (size_t)(lp - 1) * N, rows, lm1);
  ntt_forward_rescale(C, out, x, rows, lp, addc, row0);
}

void rescale_inplace(Ctx& C, CtSet& s, const u64* addc) {
  const int lp = s.limbs;
  if (lp < 2) throw Error(2, "no level left to rescale");
  const int rows = s.n * s.polys;
  const size_t N = C.N;
  DevBuf out((size_t)rows * (lp - 1) * N, C.stream);
  const int step = chunk_items(C, rows, 8.0 * N * lp);
  for (int r0 = 0; r0 < rows; r0 += step)
    rescale_rows(C, s.buf.p + (size_t)r0 * lp * N, std::min(step, rows - r0), lp, out.p + (size_t)r0 * (lp - 1) * N,
                 addc, r0);
  s.buf = std::move(out);
  s.limbs = lp - 1;
  s.scale = s.scale / (double)C.q[lp - 1];
}


static void check_pair(const CtSet& a, const CtSet& b) {
  if (a.limbs != b.limbs) throw Error(4, "operands at different levels");
  if (a.scale != b.scale) throw Error(4, "operands at different scales");
}

std::unique_ptr<CtSet> mul(Ctx& C, const CtSet& a_any, const CtSet& b_any) {
  if (a_any.n != b_any.n) throw Error(1, "sets of different sizes");
  if (a_any.limbs != b_any.limbs) throw Error(4, "operands at different levels");
  if (a_any.limbs < 2) throw Error(2, "no level left for a product");
  std::unique_ptr<CtSet> ha, hb;
  const CtSet& a = two_comp(C, a_any, ha);
  const CtSet& b = &b_any == &a_any ? a : two_comp(C, b_any, hb);
  const int lp = a.limbs;
  const size_t N = C.N;
  auto out = new_set(C, a.n, 3, lp - 1, (a.scale * b.scale) / (double)C.q[lp - 1]);
  // per ciphertext: the three tensor components and the rescale temporaries
  const int step = chunk_items(C, a.n, 8.0 * N * (3.0 * lp + 3.0 * lp));
  for (int c0 = 0; c0 < a.n; c0 += step) {
    const int cn = std::min(step, a.n - c0);
    DevBuf d((size_t)cn * 3 * lp * N, C.stream);
    k_tensor(C, a.ct(c0), b.ct(c0), d.p, cn, lp);
    rescale_rows(C, d.p, cn * 3, lp, out->ct(c0));
  }
  return out;
}

std::unique_ptr<CtSet> square(Ctx& C, const CtSet& in) { return mul(C, in, in); }

std::unique_ptr<CtSet> add(Ctx& C, const CtSet& a, const CtSet& b) {
  if (a.n != b.n || a.polys != b.polys) throw Error(1, "sets of different sizes or component counts");
  check_pair(a, b);
  auto out = new_set(C, a.n, a.polys, a.limbs, a.scale);
  k_add(C, a.buf.p, b.buf.p, out->buf.p, a.n * a.polys, a.limbs);
  return out;
}

// per-group constants round(v * scale) mod q_i, uploaded as [groups][limbs]
static DevBuf const_table(Ctx& C, const double* v, int groups, int limbs, double scale) {
  std::vector<u64> t((size_t)groups * limbs);
  for (int g = 0; g < groups; g++) {
    const int64_t iv = std::llround(v[g] * scale);
    for (int i = 0; i < limbs; i++) t[(size_t)g * limbs + i] = residue_of(iv, C.q[i]);
  }
  DevBuf d(t.size(), C.stream);
  upload_async(C, d.p, t.data(), t.size() * 8);
  return d;
}

// x times the integer v (every component), a new set at x's level and scale
static std::unique_ptr<CtSet> times_integer(Ctx& C, const CtSet& x, int64_t v) {
  std::vector<u64> t((size_t)2 * x.limbs);
  for (int i = 0; i < x.limbs; i++) {
    const u64 r = residue_of(v, C.q[i]);
    t[2 * i] = r;
    t[2 * i + 1] = (u64)(((unsigned __int128)r << 64) / C.q[i]);
  }
  DevBuf d(t.size(), C.stream);
  upload_async(C, d.p, t.data(), t.size() * 8);
  auto out = new_set(C, x.n, x.polys, x.limbs, x.scale);
  k_mul_const(C, x.buf.p, out->buf.p, (size_t)x.n * x.polys, x.limbs, d.p);
  return out;
}

// the same ciphertexts without their last limb (modulus drop; the scale is unchanged)
// The set modulo q_0 .. q_{limbs-1} only: the residues of the remaining primes, unchanged
// (modulus dropping without division; the scale stays).
std::unique_ptr<CtSet> drop_limbs(Ctx& C, const CtSet& x, int limbs) {
  if (limbs < 1 || limbs > x.limbs) throw Error(1, "the target level must keep 1 .. limbs primes");
  auto out = new_set(C, x.n, x.polys, limbs, x.scale);
  k_copy_limbs(C, x.buf.p, (size_t)x.limbs * C.N, out->buf.p, (size_t)limbs * C.N, (size_t)x.n * x.polys, limbs);
  return out;
}
static std::unique_ptr<CtSet> drop_last_limb(Ctx& C, const CtSet& x) { return drop_limbs(C, x, x.limbs - 1); }

// Plaintext addition: component 0 of ciphertext c gains the encoded integer plaintext m[c]
// (n_vec = set size) or m[0] (n_vec = 1), reduced modulo the set's primes and transformed
// (the plaintext carries the set's scale, so the slots add).
void add_plain(Ctx& C, CtSet& x, const int64_t* m, int n_vec) {
  if (n_vec != 1 && n_vec != x.n) throw Error(1, "one plaintext, or one per ciphertext");
  const int lp = x.limbs;
  const size_t N = C.N;
  DevBuf mi((size_t)n_vec * N, C.stream);
  upload_async(C, mi.p, m, (size_t)n_vec * N * 8);
  DevBuf pt((size_t)n_vec * lp * N, C.stream);
  const LimbMap lm = limbs_q(lp, N);
  k_reduce_signed(C, reinterpret_cast<const int64_t*>(mi.p), pt.p, n_vec, lm);
  ntt_forward(C, pt.p, n_vec, lm);
  for (int c = 0; c < x.n; c++) {
    u64* c0 = x.ct(c);
    k_add(C, c0, pt.p + (size_t)(n_vec == 1 ? 0 : c) * lp * N, c0, 1, lp);
  }
}

// Degree-3 activation (the ACT layers of Table I), depth two, evaluated as
// x^2 (c3 x + c2) + (c1 x + c0); q1, q2 the primes the two rescales drop, D the
// input scale:
//   u = relin(rescale(x (x) x))                  scale s_u = D D / q1
//   t = rescale(x round(c3 q1)) + round(c2 D)    scale D
//   y = rescale(u (x) t)                         scale s_y = s_u D / q2, two levels down
//   v = rescale(x round(c1 s_y q1 / D)) without its last limb, + round(c0 s_y)
//   result y + v with three components (relinearised by the next operation).
std::unique_ptr<CtSet> poly_act3(Ctx& C, const CtSet& x_any, const double* c) {
  std::unique_ptr<CtSet> hx;
  const CtSet& x = two_comp(C, x_any, hx);
  const int lp = x.limbs;
  if (lp < 3) throw Error(2, "a degree-3 activation needs two levels");
  const double D = x.scale;
  const u64 q1 = C.q[lp - 1];
  auto u = mul(C, x, x);
  relinearize(C, *u);
  auto t = times_integer(C, x, std::llround(c[3] * (double)q1));
  rescale_inplace(C, *t);
  t->scale = D;
  {
    DevBuf cb = const_table(C, &c[2], 1, t->limbs, D);
    k_add_const(C, t->buf.p, t->n, t->limbs, cb.p, t->n);
  }
  auto y = mul(C, *u, *t);
  u.reset();
  t.reset();
  const double s_y = y->scale;
  auto v1 = times_integer(C, x, std::llround(c[1] * s_y * (double)q1 / D));
  rescale_inplace(C, *v1);
  auto v = drop_last_limb(C, *v1);
  v1.reset();
  v->scale = s_y;
  {
    DevBuf cb = const_table(C, &c[0], 1, v->limbs, s_y);
    k_add_const(C, v->buf.p, v->n, v->limbs, cb.p, v->n);
  }
  k_add_comps(C, y->buf.p, v->buf.p, y->n, y->polys, y->limbs);
  return y;
}

std::unique_ptr<CtSet> conv2d(Ctx& C, const CtSet& in_any, int c_in, int gap, const double* W, const double* bias,
                              int c_out, int k, int stride) {
  std::unique_ptr<CtSet> hold;
  const CtSet& in = two_comp(C, in_any, hold);
  if (c_in < 1 || c_out < 1 || k < 1 || stride < 1 || gap < 1) throw Error(1, "bad convolution shape");
  if (in.n % c_in) throw Error(1, "input set size is not a multiple of c_in");
  const int w_in = in.n / c_in;
  if (w_in < k) throw Error(1, "image narrower than the kernel");
  const int w_out = (w_in - k) / stride + 1;
  const int lp = in.limbs;
  if (lp < 2) throw Error(2, "no level left for the convolution");
  std::vector<long> steps(k);
  for (int a = 0; a < k; a++) steps[a] = (long)gap * a;
  for (long s : steps)
    if (C.galois_elt(s) != 1) C.key(C.galois_elt(s));
  // integer weights round(K q_l) mod q_i with Shoup companions, [o][c][a][b][limb][2]
  const u64 ql = C.q[lp - 1];
  const size_t nw = (size_t)c_out * c_in * k * k;
  std::vector<u64> wt(nw * lp * 2);
  for (size_t t = 0; t < nw; t++) {
    const int64_t iv = std::llround(W[t] * (double)ql);
    for (int i = 0; i < lp; i++) {
      const u64 r = residue_of(iv, C.q[i]);
      wt[(t * lp + i) * 2] = r;
      wt[(t * lp + i) * 2 + 1] = (u64)(((unsigned __int128)r << 64) / C.q[i]);
    }
  }
  DevBuf dw(wt.size(), C.stream);
  upload_async(C, dw.p, wt.data(), wt.size() * 8);
  auto out = new_set(C, c_out * w_out, 2, lp, in.scale);
  // temporaries per input ciphertext: a gathered copy, its k rotations, its ModUp digits and, per
  // non-trivial step, the key sums, their P part and the ModDown result
  int S = 0;
  for (long s : steps) S += C.galois_elt(s) != 1;
  const int nb = lp + C.K, beta = C.beta_at(lp);
  const double per_ct = 8.0 * C.N * (2.0 * lp + 2.0 * k * lp + (double)beta * nb + S * (2.0 * nb + 2.0 * C.K + 2.0 * lp));
  // output columns per chunk: a chunk of wc columns reads (wc - 1) stride + k input columns per channel
  const int max_span = chunk_items(C, w_in, per_ct * c_in);
  const int wc = max_span >= w_in ? w_out : std::max(1, (max_span - k) / stride + 1);
  // the tensor-core multiply-accumulate reads the rotations column-major ([j][c][a]), the CUDA-core
  // kernels channel-major ([c][j][a])
  const bool tc = conv_mac_tc_all(C, c_in, k, c_out, lp);
  if (wc >= w_out) {
    auto rot = tc ? rotate_colmajor(C, in, c_in, steps) : rotate(C, in, steps);
    k_conv_mac(C, rot->buf.p, out->buf.p, dw.p, c_in, w_in, k, stride, c_out, w_out, lp, tc);
  } else {
    const size_t cw = in.ct_words();
    for (int j0 = 0; j0 < w_out; j0 += wc) {
      const int jn = std::min(wc, w_out - j0), span = (jn - 1) * stride + k, first = j0 * stride;
      auto part = new_set(C, c_in * span, 2, lp, in.scale);
      for (int c = 0; c < c_in; c++)
        HE_CUDA(cudaMemcpyAsync(part->ct(c * span), in.ct(c * w_in + first), (size_t)span * cw * 8,
                                cudaMemcpyDeviceToDevice, C.stream));
      auto rot = tc ? rotate_colmajor(C, *part, c_in, steps) : rotate(C, *part, steps);
      part.reset();
      DevBuf oc((size_t)c_out * jn * cw, C.stream);
      k_conv_mac(C, rot->buf.p, oc.p, dw.p, c_in, span, k, stride, c_out, jn, lp, tc);
      rot.reset();
      for (int o = 0; o < c_out; o++)
        HE_CUDA(cudaMemcpyAsync(out->ct(o * w_out + j0), oc.p + (size_t)o * jn * cw, (size_t)jn * cw * 8,
                                cudaMemcpyDeviceToDevice, C.stream));
    }
  }
  // scalars were encoded at scale q_l, which the rescale removes; the bias round(bias_o D) joins
  // component 0 of every output ciphertext of channel o in the rescale's last pass
  DevBuf cb;
  if (bias) {
    std::vector<u64> t((size_t)out->n * 2 * (lp - 1), 0);
    for (int o = 0; o < c_out; o++) {
      const int64_t iv = std::llround(bias[o] * in.scale);
      for (int j = 0; j < w_out; j++)
        for (int i = 0; i < lp - 1; i++) t[((size_t)(o * w_out + j) * 2) * (lp - 1) + i] = residue_of(iv, C.q[i]);
    }
    cb = DevBuf(t.size(), C.stream);
    upload_async(C, cb.p, t.data(), t.size() * 8);
  }
  rescale_inplace(C, *out, bias ? cb.p : nullptr);
  out->scale = in.scale;
  return out;
}

// Convolution with encrypted kernels (the model provider's kernel ciphertexts,
// Sec. V; Kernelspanner's role, Sec. III-C, in the column layout): Wct[o][c][a][b]
// encrypts the constant K[o][c][a][b] at scale q_l, l the input level. Output (o, j')
// is sum_{c,b,a} Wct[o][c][a][b] (x) Rot(X_{c, s j' + b}, g a) as three components,
// rescaled (scale q_l D / q_l = D), relinearised, plus round(bias_o D). The rotations
// are hoisted per input column as in conv2d; the work budget is not applied.
std::unique_ptr<CtSet> conv2d_enc(Ctx& C, const CtSet& in_any, int c_in, int gap, const CtSet& Wct_any,
                                  const double* bias, int c_out, int k, int stride) {
  std::unique_ptr<CtSet> hold, holdw;
  const CtSet& in = two_comp(C, in_any, hold);
  const CtSet& Wct = two_comp(C, Wct_any, holdw);
  if (c_in < 1 || c_out < 1 || k < 1 || stride < 1 || gap < 1) throw Error(1, "bad convolution shape");
  if (in.n % c_in) throw Error(1, "input set size is not a multiple of c_in");
  if (Wct.n != c_out * c_in * k * k) throw Error(1, "expected c_out c_in k k kernel ciphertexts");
  if (Wct.limbs != in.limbs) throw Error(4, "kernels and input at different levels");
  const int w_in = in.n / c_in;
  if (w_in < k) throw Error(1, "image narrower than the kernel");
  const int w_out = (w_in - k) / stride + 1;
  const int lp = in.limbs;
  if (lp < 2) throw Error(2, "no level left for the convolution");
  std::vector<long> steps(k);
  for (int a = 0; a < k; a++) steps[a] = (long)gap * a;
  for (long s : steps)
    if (C.galois_elt(s) != 1) C.key(C.galois_elt(s));
  auto rot = rotate(C, in, steps);  // [c][j][a]
  auto out = new_set(C, c_out * w_out, 3, lp, in.scale * Wct.scale);
  k_conv_enc_mac(C, rot->buf.p, Wct.buf.p, out->buf.p, c_in, w_in, k, stride, c_out, w_out, lp);
  rot.reset();
  rescale_inplace(C, *out);
  relinearize(C, *out);
  out->scale = in.scale;  // the kernels were encrypted at scale q_l, which the rescale removes
  if (bias) {
    DevBuf cb = const_table(C, bias, c_out, lp - 1, out->scale);
    k_add_const(C, out->buf.p, out->n, lp - 1, cb.p, w_out);
  }
  return out;
}

std::unique_ptr<CtSet> matmul(Ctx& C, const CtSet& A_any, const CtSet& B_any, int p, int lo, int hi) {
  std::unique_ptr<CtSet> ha, hb;
  const CtSet& A = two_comp(C, A_any, ha);
  const CtSet& B = two_comp(C, B_any, hb);
  if (A.n != B.n || A.n < 1) throw Error(1, "A and B must have the same number n of ciphertexts");
  if (p < 1 || (C.N / 2) % (size_t)p) throw Error(1, "p must divide the slot count");
  if (hi <= 0) hi = p;
  if (lo < 0 || lo >= hi || hi > p) throw Error(1, "diagonal range outside [0, p)");
  if (A.limbs != B.limbs) throw Error(4, "operands at different levels");
  if (A.limbs < 2) throw Error(2, "no level left for the product");
  for (int s = std::max(lo, 1); s < hi; s++) C.key(C.galois_elt(s));
  const int n = A.n, lp = A.limbs, nd = hi - lo;
  const size_t cw = (size_t)2 * lp * C.N;
  DevBuf ext;
  if (hi > 1) ext = modup_c1(C, B);
  // rotations by idx in chunks that bound the memory of the rotated operands
  const size_t budget_words = (size_t)1 << 30;  // 8 GiB
  int chunk = (int)std::max<size_t>(1, budget_words / ((size_t)n * cw));
  if (chunk > nd) chunk = nd;
  auto d = new_set(C, nd, 3, lp, A.scale * B.scale);
  DevBuf R((size_t)n * chunk * cw, C.stream);
  for (int i0 = lo; i0 < hi; i0 += chunk) {
    const int ci = std::min(chunk, hi - i0);
    std::vector<long> steps(ci);
    for (int t = 0; t < ci; t++) steps[t] = i0 + t;
    rotate_from_ext(C, B, ext, steps, R.p, ci);
    k_matmul_acc(C, A.buf.p, R.p, d->ct(i0 - lo), n, ci, lp);
  }
  R.reset();
  ext.reset();
  rescale_inplace(C, *d);
  relinearize(C, *d);
  return d;
}

// Alg. 4 on one-ciphertext image blocks (the paper's single-ciphertext convolution
// over virtual ciphertexts, Sec. III-C/D): images row-major in blocks of width Wb;
// S [k^2] the Kernelspanner ciphertexts (scale q_l), bias the encrypted bias block
// (level l - 2, scale D), masks [k^2][l - 1][N] the offset masks (NTT domain, scale
// q_{l-1}). For each offset t = r k + c and each input ciphertext:
//   T = relin(rescale(X (x) S_t)); U = sum_{pos < k} Rot(T, pos);
//   V = U + sum_{1 <= pos < k} Rot(U, pos Wb); acc += rescale(V (x) F_t)
// with hoisted rotations of T and of U (SumForConv, Alg. 1, with its row pass on
// the column sums). Output: n ciphertexts at level l - 2, scale D.
std::unique_ptr<CtSet> vr_conv2d(Ctx& C, const CtSet& in_any, const CtSet& S, const CtSet& bias, int k, int Wb,
                                 const u64* masks) {
  std::unique_ptr<CtSet> hold;
  const CtSet& in = two_comp(C, in_any, hold);
  const int lp = in.limbs;
  if (k < 1 || Wb < 1) throw Error(1, "bad kernel or block width");
  if (lp < 3) throw Error(2, "the single-ciphertext convolution needs two levels");
  if (S.n != k * k || S.limbs != lp || S.polys != 2) throw Error(1, "expected k^2 kernel ciphertexts at the input level");
  if (bias.n != 1 || bias.limbs != lp - 2 || bias.polys != 2) throw Error(1, "expected one bias ciphertext two levels down");
  const double D = in.scale;
  std::vector<long> col(k), row(k);
  for (int pos = 0; pos < k; pos++) {
    col[pos] = pos;
    row[pos] = (long)pos * Wb;
  }
  auto out = new_set(C, in.n, 2, lp - 2, D);
  const size_t mw = (size_t)(lp - 1) * C.N;
  const int kk = k * k;
  // the k^2 offsets of one input ciphertext run side by side as one set (each offset's
  // arithmetic is unchanged); sum_pos R[t][pos] for every offset t: gather R[.][pos] (one
  // launch) and add it to the running sums (one launch)
  auto sum_steps = [&](const CtSet& R, int limbs) {
    const size_t cw = R.ct_words();
    auto U = new_set(C, kk, 2, limbs, R.scale);
    k_copy_limbs(C, R.buf.p, (size_t)k * cw, U->buf.p, cw, (size_t)kk, 2 * limbs);
    if (k > 1) {
      DevBuf g((size_t)kk * cw, C.stream);
      for (int pos = 1; pos < k; pos++) {
        k_copy_limbs(C, R.ct(pos), (size_t)k * cw, g.p, cw, (size_t)kk, 2 * limbs);
        k_add(C, U->buf.p, g.p, U->buf.p, 2 * kk, limbs);
      }
    }
    return U;
  };
  for (int c = 0; c < in.n; c++) {
    // T_t = relin(rescale(X_c (x) S_t)) for every offset t
    auto Xr = new_set(C, kk, 2, lp, in.scale);
    k_copy_limbs(C, in.ct(c), 0, Xr->buf.p, in.ct_words(), (size_t)kk, 2 * lp);
    auto T = mul(C, *Xr, S);
    Xr.reset();
    relinearize(C, *T);
    // SumForConv: the column pass (Rot by pos) then the row pass (Rot by pos Wb)
    auto R = rotate(C, *T, col);  // [t][pos]
    T.reset();
    auto U = sum_steps(*R, lp - 1);
    R.reset();
    auto R2 = rotate(C, *U, row);  // [t][pos]
    U.reset();
    auto V = sum_steps(*R2, lp - 1);
    R2.reset();
    // W_t = rescale(V_t (x) F_t): the masked-sum kernel with one term per offset
    auto W = new_set(C, kk, 2, lp - 1, D);
    {
      std::vector<const u64*> xs(kk);
      for (int t = 0; t < kk; t++) xs[t] = V->ct(t);
      DevBuf dxs((size_t)kk, C.stream);
      upload_async(C, dxs.p, xs.data(), (size_t)kk * 8);
      for (int t = 0; t < kk; t++)
        k_pack_blocks(C, (const u64* const*)dxs.p + t, masks + (size_t)t * mw, 1, 1, lp - 1, W->ct(t));
    }
    V.reset();
    rescale_inplace(C, *W);
    HE_CUDA(cudaMemcpyAsync(out->ct(c), bias.buf.p, bias.buf.words * 8, cudaMemcpyDeviceToDevice, C.stream));
    for (int t = 0; t < kk; t++) k_add(C, out->ct(c), W->ct(t), out->ct(c), 2, lp - 2);
  }
  out->scale = D;  // kernels at scale q_l and masks at q_{l-1}, which the two rescales remove
  return out;
}

// vRot (Alg. 5): virtual ciphertexts are rows of n slots whose first hw slots hold
// an image; every row's image rotates left by r:
//   R = rescale(Rot(X, r) (x) F1 + Rot(X, S - hw + r) (x) F2)
// F1 keeping row positions j < hw - r, F2 positions hw - r <= j < hw (masks [2][lp][N],
// NTT domain, scale q_{lp-1}); the two rotations share one ModUp, the masked terms one
// multiply-accumulate launch and one rescale. One level; the scale is unchanged.
std::unique_ptr<CtSet> vrot(Ctx& C, const CtSet& in_any, long r, int hw, const u64* masks) {
  std::unique_ptr<CtSet> hold;
  const CtSet& in = two_comp(C, in_any, hold);
  if (hw < 1 || r < 0 || r >= hw) throw Error(1, "vRot needs 0 <= r < the image length");
  if (in.limbs < 2) throw Error(2, "no level left for vRot");
  const long S = (long)C.N / 2;
  auto R = rotate(C, in, {r, S - hw + r});  // [ct][2]
  const size_t cw = in.ct_words();
  const u64* xs[2] = {R->buf.p, R->buf.p + cw};
  DevBuf dxs(2, C.stream);
  upload_async(C, dxs.p, xs, 16);
  auto out = new_set(C, in.n, 2, in.limbs, in.scale);
  k_pack_blocks(C, (const u64* const*)dxs.p, masks, 2, in.n, in.limbs, out->buf.p, 2 * cw);
  R.reset();
  rescale_inplace(C, *out);
  out->scale = in.scale;  // the masks were encoded at scale q_l
  return out;
}

// Alg. 3 with one ciphertext per operand (the paper's single-ciphertext matmul): A
// row-major (tau_a), Bbar = tau_b(B) tiled over the whole ring, so RowShifter applied
// idx times is Rot(Bbar, idx n). For idx < p:
//   T = relin(rescale(A (x) Rot(Bbar, idx n)))
//   SumColVec: T += Rot(T, t) (t = 1, 2, .., n/2: row sums in column 0);
//              T = rescale(T (x) E); T += Rot(T, -t) (t = 1, .., n/2: replicated over the row)
//   acc += rescale(T (x) F_idx), F_idx keeping slot i n + ((i + idx) mod p), i < m
// E [lp-1][N] and F [p][lp-2][N] are NTT-domain plaintexts at scales q_{lp-2}, q_{lp-3}.
// C[i][c] ends at slot i n + c; three levels; scale D D / q_{lp-1}.
std::unique_ptr<CtSet> vr_matmul(Ctx& C, const CtSet& A_any, const CtSet& Bbar, int n, int p, const u64* E,
                                 const u64* F) {
  std::unique_ptr<CtSet> hold;
  const CtSet& A = two_comp(C, A_any, hold);
  const int lp = A.limbs;
  if (A.n != 1 || Bbar.n != 1 || Bbar.polys != 2 || Bbar.limbs != lp) throw Error(1, "one ciphertext per operand");
  if (lp < 4) throw Error(2, "the single-ciphertext matmul needs three levels");
  if (n < 1 || (n & (n - 1)) || p < 1) throw Error(1, "n must be a power of two and p positive");
  std::vector<long> shifts(p);
  for (int idx = 0; idx < p; idx++) shifts[idx] = (long)idx * n;
  auto R = rotate(C, Bbar, shifts);  // [p]: RowShifter applied idx times
  // the p revolver positions run side by side as one set of p ciphertexts (each position's
  // arithmetic is unchanged): T_idx = relin(rescale(A (x) R_idx))
  auto Ap = new_set(C, p, 2, lp, A.scale);
  k_copy_limbs(C, A.buf.p, 0, Ap->buf.p, A.ct_words(), (size_t)p, 2 * lp);
  auto T = mul(C, *Ap, *R);
  Ap.reset();
  R.reset();
  relinearize(C, *T);
  const double sc = T->scale;  // (A.scale Bbar.scale) / q_{lp-1}
  // SumColVec, left half: T += Rot(T, t)
  for (int t = 1; t < n; t *= 2) {
    auto r = rotate(C, *T, {(long)t});
    k_add(C, T->buf.p, r->buf.p, T->buf.p, 2 * p, T->limbs);
  }
  // U = rescale(T (x) E) for every position (E at scale q_{lp-2}, so the scale stays)
  auto U = new_set(C, p, 2, T->limbs, sc);
  {
    const u64* x0 = T->buf.p;
    DevBuf dx(1, C.stream);
    upload_async(C, dx.p, &x0, 8);
    k_pack_blocks(C, (const u64* const*)dx.p, E, 1, p, T->limbs, U->buf.p);
  }
  T.reset();
  rescale_inplace(C, *U);
  U->scale = sc;
  // SumColVec, right half: U += Rot(U, -t)
  for (int t = 1; t < n; t *= 2) {
    auto r = rotate(C, *U, {-(long)t});
    k_add(C, U->buf.p, r->buf.p, U->buf.p, 2 * p, U->limbs);
  }
  // D_idx = rescale(U_idx (x) F_idx), then acc = sum over idx
  const size_t fw = (size_t)U->limbs * C.N;
  auto D = new_set(C, p, 2, U->limbs, sc);
  {
    std::vector<const u64*> xs(p);
    for (int idx = 0; idx < p; idx++) xs[idx] = U->ct(idx);
    DevBuf dxs((size_t)p, C.stream);
    upload_async(C, dxs.p, xs.data(), (size_t)p * 8);
    for (int idx = 0; idx < p; idx++)
      k_pack_blocks(C, (const u64* const*)dxs.p + idx, F + (size_t)idx * fw, 1, 1, U->limbs, D->ct(idx));
  }
  U.reset();
  rescale_inplace(C, *D);
  auto acc = new_set(C, 1, 2, lp - 3, sc);
  HE_CUDA(cudaMemcpyAsync(acc->buf.p, D->ct(0), acc->buf.words * 8, cudaMemcpyDeviceToDevice, C.stream));
  for (int idx = 1; idx < p; idx++) k_add(C, acc->buf.p, D->ct(idx), acc->buf.p, 2, lp - 3);
  return acc;
}

// ReForm (Sec. IV-C) in the column layout: a strided layer leaves row i of every
// block at slot b H + g i; a left rotation by (g - 1) i brings it to b H + i, so
// out = rescale(sum_{i < h} mask_i (x) Rot(X, (g - 1) i)) with mask_i the 0/1
// plaintext of slots b H + i at scale q_l: h - 1 hoisted rotations per
// ciphertext, one masked multiply-accumulate launch (k_pack_blocks over the
// rotation steps), one rescale. The scale is unchanged.
std::unique_ptr<CtSet> reform(Ctx& C, const CtSet& in_any, int gap, int h, const u64* masks) {
  std::unique_ptr<CtSet> hold;
  const CtSet& in = two_comp(C, in_any, hold);
  if (gap < 2 || h < 1) throw Error(1, "ReForm needs a row gap of at least 2 and at least one row");
  if (in.limbs < 2) throw Error(2, "no level left for ReForm");
  std::vector<long> steps(h);
  for (int i = 0; i < h; i++) steps[i] = (long)(gap - 1) * i;
  auto R = rotate(C, in, steps);  // [ct][i]
  const size_t cw = in.ct_words();
  std::vector<const u64*> xs(h);
  for (int i = 0; i < h; i++) xs[i] = R->buf.p + (size_t)i * cw;
  DevBuf dxs((size_t)h, C.stream);
  upload_async(C, dxs.p, xs.data(), (size_t)h * 8);
  auto out = new_set(C, in.n, 2, in.limbs, in.scale);
  k_pack_blocks(C, (const u64* const*)dxs.p, masks, h, in.n, in.limbs, out->buf.p, (size_t)h * cw);
  R.reset();
  rescale_inplace(C, *out);
  out->scale = in.scale;  // the masks were encoded at scale q_l
  return out;
}

// Baby-step giant-step form of the revolver: idx = g i + j (j < g). Rotation
// commutes with slotwise products and sums, so
//   D_{g i + j} = Rot( sum_k Rot(A_k, -g i) (x) Rot(B~_k, j), g i ):
// hoisted baby steps j < g of every B~_k, hoisted giant steps -g i of every A_k,
// per giant step one accumulate launch over its g outputs, one rescale and
// relinearisation of all p outputs, then a rotation by g i of the outputs of
// giant step i >= 1: n(g-1) + n(ceil(p/g)-1) + (p - g) rotations instead of n(p-1).
std::unique_ptr<CtSet> matmul_bsgs(Ctx& C, const CtSet& A_any, const CtSet& B_any, int p, int g) {
  std::unique_ptr<CtSet> ha, hb;
  const CtSet& A = two_comp(C, A_any, ha);
  const CtSet& B = two_comp(C, B_any, hb);
  if (A.n != B.n || A.n < 1) throw Error(1, "A and B must have the same number n of ciphertexts");
  const long S = (long)C.N / 2;
  if (p < 1 || S % p) throw Error(1, "p must divide the slot count");
  if (g < 1 || g > p) throw Error(1, "baby-step size out of range");
  if (A.limbs != B.limbs) throw Error(4, "operands at different levels");
  if (A.limbs < 2) throw Error(2, "no level left for the product");
  const int n = A.n, lp = A.limbs, ng = (p + g - 1) / g;
  std::vector<long> baby(g), giant(ng);
  for (int j = 0; j < g; j++) baby[j] = j;
  for (int i = 0; i < ng; i++) giant[i] = i == 0 ? 0 : S - (long)g * i;
  for (long st : baby) C.key(C.galois_elt(st));
  for (int i = 1; i < ng; i++) {
    C.key(C.galois_elt(giant[i]));
    C.key(C.galois_elt((long)g * i));
  }
  const size_t cw = (size_t)2 * lp * C.N;
  auto Rb = rotate(C, B, baby);   // [k][j]
  auto Ra = rotate(C, A, giant);  // [k][i]
  auto d = new_set(C, p, 3, lp, A.scale * B.scale);
  {
    DevBuf Ai((size_t)n * cw, C.stream);
    for (int i = 0; i < ng; i++) {
      const int cnt = std::min(g, p - g * i);
      // the giant step i of every A_k, gathered into n consecutive ciphertexts
      k_copy_limbs(C, Ra->buf.p + (size_t)i * cw, (size_t)ng * cw, Ai.p, cw, (size_t)n, 2 * lp);
      k_matmul_acc(C, Ai.p, Rb->buf.p, d->ct(g * i), n, cnt, lp, g);
    }
  }
  Ra.reset();
  Rb.reset();
  rescale_inplace(C, *d);
  relinearize(C, *d);
  for (int i = 1; i < ng; i++) {
    const int cnt = std::min(g, p - g * i);
    SetView v(*d, g * i, cnt);
    auto r = rotate(C, v.s, {(long)g * i});
    HE_CUDA(cudaMemcpyAsync(d->ct(g * i), r->buf.p, (size_t)cnt * d->ct_words() * 8, cudaMemcpyDeviceToDevice,
                            C.stream));
  }
  return d;
}

// Zero-rotation form of the product. B~_k is tiled with period p, so its slot s
// holds B[k][s mod p]; with A's column k copied to blocks t M + o_g (M = 1 mod p,
// o_g = (g per) mod p) the slotwise product pairs A[i][k] with B[k][(i + g per + t)
// mod p], the revolver's position idx = g per + t, at slot t M + o_g + i. So
// D_g = sum_k Ahat_{g,k} (x) B~_k needs no rotation: G n tensor products summed as
// three components, one rescale and one relinearisation per group.
void volley_geometry(long slots, int m, int p, int& M, int& per, int& G) {
  if (m < 1 || p < 1 || slots % p) throw Error(1, "p must divide the slot count");
  M = p > 1 ? m + (int)(((1 - (long)m) % p + p) % p) : m;
  if ((long)(p - 1) * M + m <= slots) {
    per = p;
    G = 1;
    return;
  }
  const long r = slots - m - (p - 1);
  if (r < 0) throw Error(1, "matrix does not fit the slots");
  per = (int)(r / M) + 1;
  G = (p + per - 1) / per;
}

std::unique_ptr<CtSet> matmul_volley(Ctx& C, const CtSet& Ah_any, const CtSet& B_any) {
  std::unique_ptr<CtSet> ha, hb;
  const CtSet& Ah = two_comp(C, Ah_any, ha);
  const CtSet& B = two_comp(C, B_any, hb);
  if (B.n < 1 || Ah.n % B.n) throw Error(1, "A's volley encoding must hold G groups of n ciphertexts");
  if (Ah.limbs != B.limbs) throw Error(4, "operands at different levels");
  if (Ah.limbs < 2) throw Error(2, "no level left for the product");
  const int n = B.n, G = Ah.n / B.n, lp = B.limbs;
  auto d = new_set(C, G, 3, lp, Ah.scale * B.scale);
  k_volley_acc(C, Ah.buf.p, B.buf.p, d->buf.p, n, G, lp);
  rescale_inplace(C, *d);
  relinearize(C, *d);
  return d;
}

// Independent products A_i B_i evaluated together. Matmuls with the same p, level
// and scale form a group; inside a group, sub-batches of matmuls whose B operands
// fit the working-memory budget are concatenated into one set (one gather launch per
// kSetBlock products), so one ModUp launch and one launch per chunk of rotation
// steps serve all of them (each key tile is read once per launch for every
// ciphertext of the sub-batch). The tensor sums of up to kSetBlock products share a
// launch and write one three-component set, which is rescaled and relinearised
// once and then scattered into the per-product results (one launch per kSetBlock
// products). Every launch takes its pointers as kernel parameters, so the whole
// call can be captured into a CUDA graph. The per-ciphertext arithmetic is that of
// matmul(), so the results are identical to separate calls.
std::vector<std::unique_ptr<CtSet>> matmul_batched(Ctx& C, const std::vector<const CtSet*>& As,
                                                   const std::vector<const CtSet*>& Bs, const std::vector<int>& ps) {
  const int cnt = (int)As.size();
  std::vector<std::unique_ptr<CtSet>> out(cnt);
  std::map<std::tuple<int, int, double>, std::vector<int>> groups;
  for (int i = 0; i < cnt; i++) {
    const CtSet& A = *As[i];
    const CtSet& B = *Bs[i];
    if (A.polys != 2 || B.polys != 2) throw Error(1, "batched matmul operands must have two components");
    if (A.n != B.n || A.n < 1) throw Error(1, "A and B must have the same number n of ciphertexts");
    if (ps[i] < 1 || (C.N / 2) % (size_t)ps[i]) throw Error(1, "p must divide the slot count");
    if (A.limbs != B.limbs || A.scale != B.scale) throw Error(4, "operands at different levels or scales");
    if (A.limbs < 2) throw Error(2, "no level left for the product");
    for (int s = 1; s < ps[i]; s++) C.key(C.galois_elt(s));
    groups[std::make_tuple(ps[i], A.limbs, A.scale)].push_back(i);
  }
  const size_t N = C.N;
  const size_t budget = (size_t)6 << 30;  // words (48 GiB) of digits, rotated operands and key-switch scratch
  for (auto& kv : groups) {
    const int p = std::get<0>(kv.first), lp = std::get<1>(kv.first);
    const double sc = std::get<2>(kv.first);
    const std::vector<int>& members = kv.second;
    const size_t cw = (size_t)2 * lp * N;
    const size_t ext_ct = (size_t)C.beta_at(lp) * (lp + C.K) * N;
    // words per ciphertext per rotation step: rotated operand, inner products, ModDown terms
    const size_t step_ct = cw + (size_t)2 * (lp + C.K) * N + cw;
    size_t m0 = 0;
    while (m0 < members.size()) {
      // sub-batch: as many matmuls as fit with at least 4 steps per chunk
      std::vector<int> sb;
      int ntot = 0;
      for (size_t t = m0; t < members.size(); t++) {
        const int nn = As[members[t]]->n;
        if (!sb.empty() && (size_t)(ntot + nn) * (ext_ct + 4 * step_ct) > budget) break;
        sb.push_back(members[t]);
        ntot += nn;
      }
      m0 += sb.size();
      const int T = (int)sb.size();
      std::vector<size_t> off(T + 1, 0);  // ciphertext offsets of the products in the concatenation
      for (int t = 0; t < T; t++) off[t + 1] = off[t] + (size_t)Bs[sb[t]]->n;
      auto Bcat = new_set(C, ntot, 2, lp, sc);
      for (int t0 = 0; t0 < T; t0 += kSetBlock) {
        const int tn = std::min(kSetBlock, T - t0);
        SetPtrs P;
        for (int t = 0; t <= tn; t++) {
          if (t < tn) P.p[t] = Bs[sb[t0 + t]]->buf.p;
          P.off[t] = (off[t0 + t] - off[t0]) * cw;
        }
        k_move_words(C, P, Bcat->ct((int)off[t0]), tn, 0);
      }
      DevBuf ext;
      if (p > 1) ext = modup_c1(C, *Bcat);
      auto D = new_set(C, T * p, 3, lp, sc * sc);
      const size_t room = budget > (size_t)ntot * ext_ct ? budget - (size_t)ntot * ext_ct : 0;
      int chunk = (int)std::max<size_t>(1, room / ((size_t)ntot * step_ct));
      if (chunk > p) chunk = p;
      DevBuf R((size_t)ntot * chunk * cw, C.stream);
      for (int i0 = 0; i0 < p; i0 += chunk) {
        const int ci = std::min(chunk, p - i0);
        std::vector<long> steps(ci);
        for (int t = 0; t < ci; t++) steps[t] = i0 + t;
        rotate_from_ext(C, *Bcat, ext, steps, R.p, ci);
        for (int t0 = 0; t0 < T; t0 += kSetBlock) {
          const int tn = std::min(kSetBlock, T - t0);
          SetPtrs Ap;
          for (int t = 0; t <= tn; t++) {
            if (t < tn) Ap.p[t] = As[sb[t0 + t]]->buf.p;
            Ap.off[t] = off[t0 + t];
          }
          k_matmul_acc_multi(C, Ap, R.p, D->buf.p, tn, t0, p, i0, ci, lp);
        }
      }
      R.reset();
      ext.reset();
      Bcat.reset();
      rescale_inplace(C, *D);
      relinearize(C, *D);
      const size_t ow = (size_t)p * D->ct_words();
      for (int t = 0; t < T; t++) out[sb[t]] = new_set(C, p, 2, lp - 1, D->scale);
      for (int t0 = 0; t0 < T; t0 += kSetBlock) {
        const int tn = std::min(kSetBlock, T - t0);
        SetPtrs Q;
        for (int t = 0; t <= tn; t++) {
          if (t < tn) Q.p[t] = out[sb[t0 + t]]->buf.p;
          Q.off[t] = (size_t)t * ow;
        }
        k_move_words(C, Q, D->buf.p + (size_t)t0 * ow, tn, 1);
      }
    }
  }
  return out;
}

DevBuf fc_prepare(Ctx& C, const int64_t* pts_host, int out_dim, int n_in, int limbs) {
  const size_t N = C.N, per = (size_t)limbs * N;
  DevBuf pts((size_t)out_dim * n_in * per, C.stream);
  const int chunk = 64;
  DevBuf dm((size_t)chunk * N, C.stream);
  const size_t total = (size_t)out_dim * n_in;
  for (size_t c0 = 0; c0 < total; c0 += chunk) {
    const int cn = (int)std::min<size_t>(chunk, total - c0);
    upload_async(C, dm.p, pts_host + c0 * N, (size_t)cn * N * 8);
    k_reduce_signed(C, (const int64_t*)dm.p, pts.p + c0 * per, cn, limbs_q(limbs, N));
    ntt_forward(C, pts.p + c0 * per, cn, limbs_q(limbs, N));
  }
  HE_CUDA(cudaStreamSynchronize(C.stream));
  return pts;
}

std::unique_ptr<CtSet> fc_partial(Ctx& C, const CtSet& in, const u64* pts, int out_dim, int pt_cols, int first) {
  const int lp = in.limbs;
  if (lp < 2) throw Error(2, "no level left for the dense layer");
  if (first < 0 || first + in.n > pt_cols) throw Error(1, "input columns outside the prepared weights");
  auto z = new_set(C, out_dim, in.polys, lp, in.scale);
  k_fc_mac(C, in.buf.p, pts + (size_t)first * lp * C.N, z->buf.p, in.n, pt_cols, out_dim, lp, in.polys);
  return z;
}

void fc_finish(Ctx& C, CtSet& z, int gap, int block_stride, const double* bias) {
  if (z.limbs < 2) throw Error(2, "no level left for the dense layer");
  for (int t = gap; t < block_stride; t *= 2) C.key(C.galois_elt(t));
  const double scale = z.scale;
  rescale_inplace(C, z);
  z.scale = scale;  // plaintexts were encoded at scale q_l
  relinearize(C, z);
  for (int t = gap; t < block_stride; t *= 2) {
    auto r = rotate(C, z, {(long)t});
    k_add(C, z.buf.p, r->buf.p, z.buf.p, z.n * 2, z.limbs);
  }
  if (bias) {
    DevBuf cb = const_table(C, bias, z.n, z.limbs, z.scale);
    k_add_const(C, z.buf.p, z.n, z.limbs, cb.p, 1);
  }
}

std::unique_ptr<CtSet> fc_apply(Ctx& C, const CtSet& in, const u64* pts, int out_dim, int gap, int block_stride,
                                const double* bias) {
  if (in.limbs < 2) throw Error(2, "no level left for the dense layer");
  for (int t = gap; t < block_stride; t *= 2) C.key(C.galois_elt(t));
  auto z = fc_partial(C, in, pts, out_dim, in.n, 0);
  fc_finish(C, *z, gap, block_stride, bias);
  return z;
}

std::unique_ptr<CtSet> pack_blocks(Ctx& C, const std::vector<const u64*>& xs, int n_ct, int limbs, double scale,
                                   const u64* masks) {
  const int T = (int)xs.size();
  if (T < 1 || n_ct < 1) throw Error(1, "nothing to pack");
  if (limbs < 2) throw Error(2, "packing needs one level");
  DevBuf dxs((size_t)T, C.stream);
  upload_async(C, dxs.p, xs.data(), (size_t)T * 8);
  auto x = new_set(C, n_ct, 2, limbs, scale);
  k_pack_blocks(C, (const u64* const*)dxs.p, masks, T, n_ct, limbs, x->buf.p);
  rescale_inplace(C, *x);
  x->scale = scale;  // the masks were encoded at scale q_l
  return x;
}

}  // namespace he
