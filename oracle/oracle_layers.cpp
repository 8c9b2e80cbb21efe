// oracle_layers.cpp - the paper's multi-ciphertext layer algorithms on the
// CPU oracle: encrypted matrix multiplication (n ciphertexts per operand),
// convolution over the column-wise image layout (w ciphertexts of h pixels),
// square activation and the fully connected layer.
//
// TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
//
// The paper states the multi-ciphertext layouts (abstract; contributions in
// Sec. I-C) and says the single-ciphertext algorithms carry over by
// partitioning and linearity (Sec. IV-A, IV-B); it prints no algorithm for
// them. The readings written out here:
//
// Matmul (Alg. 3 with the operands split into n ciphertexts):
//   A_k holds column k of A at slots i < m; B~_k holds row k of B tiled with
//   period p over all slots (the tiling of tau_b, Sec. III-A, over the whole
//   ring). Because p divides the slot count, RowShifter (Alg. 2) applied idx
//   times is exactly Rot(B~_k, idx) (the m mod p = 0 case, Sec. III-B). Round
//   idx computes D_idx = sum_k A_k (x) Rot(B~_k, idx): the SumColVec of Alg. 3
//   over the n columns becomes n - 1 ciphertext additions, and slot i of
//   D_idx is C[i][(i + idx) mod p]. The rotations of each B~_k share one
//   ModUp; the n products of a round are summed as three-component tensors,
//   rescaled, then relinearised once.
//
// Convolution (Alg. 4 over the column layout, channels summed as in Sec. IV-B):
//   X_{c,j} holds column j of channel c, row r at slot g*r (row gap g) within
//   blocks of H slots, one image per block. Column offsets b of the kernel
//   select ciphertexts; row offsets a are rotations by g*a (the row pass of
//   SumForConv, Alg. 1). Output (o, j') is
//       bias_o + sum_c sum_b sum_a K[o][c][a][b] * Rot(X_{c, s j' + b}, g a),
//   then rescaled; the output row gap is g*s. Scalars are integers
//   round(K * q_l), q_l the prime the following rescale drops, so the scale is
//   unchanged by the layer; the bias is added after the rescale as
//   round(bias * scale).
//
// Fully connected layer: Z_o = sum_{c,j} pt_{o,c,j} (x) X_{c,j}, pt_{o,c,j}
//   holding W[o][c][i][j] at slots b*H + g*i; rescale; sum inside each block by
//   rotate-and-add over g, 2g, ..., H/2 (SumRowVec-style, Sec. II-B); add the
//   bias. The logit o of image b is at slot b*H of Z_o.
//
// Products and relinearisation: Mul (Sec. II-A) is the tensor product
// followed by the rescale; the three-component result is relinearised only
// when an operation needs two components (a rotation, the next product). The
// dense layer is linear in each component, so a squared input enters its sum
// with three components and only the out_dim results are relinearised.
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

#include "oracle_internal.h"

namespace oracle {
Ct ct_from(const Ctx& C, const u64* p, int n_polys, int limbs);
void ct_to(const Ctx& C, const Ct& ct, u64* p);

// Two components: relinearise a three-component ciphertext, pass others on.
static Ct two_comp(Ctx& C, const Ct& x) { return x.c.size() == 3 ? ct_relin(C, x) : x; }

// D_idx, idx < p, from A_k, B~_k (k < n), all at the same level.
static std::vector<Ct> matmul(Ctx& C, const std::vector<Ct>& A, const std::vector<Ct>& B, int p) {
  const int n = (int)A.size();
  std::vector<long> steps(p);
  for (int idx = 0; idx < p; idx++) steps[idx] = idx;
  std::vector<std::vector<Ct>> R(n);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < n; k++) R[k] = ct_rotate_hoisted(C, B[k], steps);
  std::vector<Ct> D(p);
#pragma omp parallel for schedule(dynamic)
  for (int idx = 0; idx < p; idx++) {
    Ct T = ct_tensor(C, A[0], R[0][idx]);
    for (int k = 1; k < n; k++) T = ct_add(C, T, ct_tensor(C, A[k], R[k][idx]));
    D[idx] = ct_relin(C, ct_rescale(C, T));
  }
  return D;
}

// Convolution with encrypted kernels (the model provider's kernel ciphertexts,
// Sec. V; Kernelspanner's role, Sec. III-C, in the column layout): Wct[o][c][a][b]
// encrypts the constant K[o][c][a][b] (every slot) at scale q_l. Output (o, j') is
//     sum_c sum_b sum_a Wct[o][c][a][b] (x) Rot(X_{c, s j' + b}, g a)
// accumulated as three-component tensors (order c, b, a), rescaled,
// relinearised, plus round(bias_o * scale). The rotations are hoisted per input
// column as in the plaintext-weight schedule.
static std::vector<Ct> conv2d_enc(Ctx& C, const std::vector<std::vector<Ct>>& X, int gap, const std::vector<Ct>& Wct,
                                  const double* bias, int c_out, int k, int stride, double scale,
                                  const std::vector<std::pair<int, int>>& sel) {
  const int c_in = (int)X.size();
  std::set<std::pair<int, int>> need;
  for (auto& s : sel)
    for (int c = 0; c < c_in; c++)
      for (int b = 0; b < k; b++) need.insert({c, stride * s.second + b});
  std::vector<std::pair<int, int>> needv(need.begin(), need.end());
  std::vector<long> steps(k);
  for (int a = 0; a < k; a++) steps[a] = (long)gap * a;
  std::vector<std::vector<Ct>> rot(needv.size());
#pragma omp parallel for schedule(dynamic)
  for (size_t t = 0; t < needv.size(); t++)
    rot[t] = ct_rotate_hoisted(C, two_comp(C, X[needv[t].first][needv[t].second]), steps);
  std::map<std::pair<int, int>, size_t> where;
  for (size_t t = 0; t < needv.size(); t++) where[needv[t]] = t;
  std::vector<Ct> out(sel.size());
#pragma omp parallel for schedule(dynamic)
  for (size_t t = 0; t < sel.size(); t++) {
    const int o = sel[t].first, jp = sel[t].second;
    Ct acc;
    bool first = true;
    for (int c = 0; c < c_in; c++)
      for (int b = 0; b < k; b++)
        for (int a = 0; a < k; a++) {
          const Ct& w = Wct[(((size_t)o * c_in + c) * k + a) * k + b];
          Ct term = ct_tensor(C, w, rot[where.at({c, stride * jp + b})][a]);
          acc = first ? term : ct_add(C, acc, term);
          first = false;
        }
    Ct r = ct_relin(C, ct_rescale(C, acc));
    if (bias) r = ct_add_const(C, r, std::llround(bias[o] * scale));
    out[t] = r;
  }
  return out;
}

// Alg. 4 on one ciphertext holding images in row-major blocks of width Wb (the
// paper's single-ciphertext convolution over virtual ciphertexts, Sec. III-C/D).
// For each kernel offset t = r k + c (order t = 0 .. k^2-1):
//   T = relin(rescale(X (x) S_t))                     (S_t the Kernelspanner ciphertext)
//   U = sum_{pos < k} Rot(T, pos)                     (column pass of SumForConv, Alg. 1)
//   V = U + sum_{1 <= pos < k} Rot(U, pos Wb)         (row pass on the column sums)
//   acc += rescale(V (x) F_t)                         (F_t the offset mask)
// starting from acc = the encrypted bias block. Rotations of T and of U are hoisted.
static Ct vr_conv2d(Ctx& C, const Ct& x_any, const std::vector<Ct>& S, const Ct& bias, int k, int Wb,
                    const int64_t* masks) {
  const Ct x = two_comp(C, x_any);
  std::vector<long> col(k), row(k);
  for (int pos = 0; pos < k; pos++) {
    col[pos] = pos;
    row[pos] = (long)pos * Wb;
  }
  Ct acc = bias;
  for (int t = 0; t < k * k; t++) {
    const Ct T = ct_relin(C, ct_rescale(C, ct_tensor(C, x, S[t])));
    std::vector<Ct> rc = ct_rotate_hoisted(C, T, col);
    Ct U = rc[0];
    for (int pos = 1; pos < k; pos++) U = ct_add(C, U, rc[pos]);
    std::vector<Ct> rr = ct_rotate_hoisted(C, U, row);
    Ct V = rr[0];
    for (int pos = 1; pos < k; pos++) V = ct_add(C, V, rr[pos]);
    std::vector<i64> m(masks + (size_t)t * C.N, masks + (size_t)(t + 1) * C.N);
    acc = ct_add(C, acc, ct_rescale(C, ct_mul_plain(C, V, m)));
  }
  return acc;
}

// vRot (Alg. 5): virtual ciphertexts are rows of n slots whose first hw slots hold
// an image; vRot(ct, r) rotates every row's image left by r:
//   R = rescale(Rot(X, r) (x) F1 + Rot(X, S - hw + r) (x) F2)
// with F1 keeping row positions j < hw - r and F2 positions hw - r <= j < hw (the
// rotations hoisted, the two masked terms summed before one rescale). masks [2][N].
static Ct vrot(Ctx& C, const Ct& x_any, long r, int hw, const int64_t* masks) {
  const Ct x = two_comp(C, x_any);
  const long S = (long)C.N / 2;
  std::vector<Ct> R = ct_rotate_hoisted(C, x, {r, S - hw + r});
  std::vector<i64> f1(masks, masks + C.N), f2(masks + C.N, masks + 2 * C.N);
  return ct_rescale(C, ct_add(C, ct_mul_plain(C, R[0], f1), ct_mul_plain(C, R[1], f2)));
}

// Alg. 3 on one ciphertext per operand (the paper's single-ciphertext matmul):
// A row-major (tau_a), Bbar = tau_b(B) tiled over the whole ring. For idx < p:
//   T = relin(rescale(A (x) Rot(Bbar, idx n)))     (RowShifter applied idx times)
//   T = SumColVec(T): T += Rot(T, t) for t = 1, 2, .., n/2 (row sums in column 0);
//       T = rescale(T (x) E) with E the column-0 mask; T += Rot(T, -t) for t = 1, .., n/2
//   acc += rescale(T (x) F_idx), F_idx keeping slot i n + ((i + idx) mod p)
// so C[i][c] ends at slot i n + c. masks [1 + p][N]: E (scale q_{l-2}), then F_idx (q_{l-3}).
static Ct vr_matmul(Ctx& C, const Ct& A_any, const Ct& Bbar, int n, int p, const int64_t* masks) {
  const Ct A = two_comp(C, A_any);
  std::vector<long> shifts(p);
  for (int idx = 0; idx < p; idx++) shifts[idx] = (long)idx * n;
  const std::vector<Ct> R = ct_rotate_hoisted(C, Bbar, shifts);
  auto mask = [&](int t) { return std::vector<i64>(masks + (size_t)t * C.N, masks + (size_t)(t + 1) * C.N); };
  Ct acc;
  for (int idx = 0; idx < p; idx++) {
    Ct T = ct_relin(C, ct_rescale(C, ct_tensor(C, A, R[idx])));
    for (int t = 1; t < n; t *= 2) T = ct_add(C, T, ct_rotate_hoisted(C, T, {(long)t})[0]);
    T = ct_rescale(C, ct_mul_plain(C, T, mask(0)));
    for (int t = 1; t < n; t *= 2) T = ct_add(C, T, ct_rotate_hoisted(C, T, {-(long)t})[0]);
    const Ct D = ct_rescale(C, ct_mul_plain(C, T, mask(1 + idx)));
    acc = idx == 0 ? D : ct_add(C, acc, D);
  }
  return acc;
}

// ReForm (Sec. IV-C) in the column layout: after a strided layer row i of every
// block sits at slot b H + g i; ReForm moves it to b H + i. A left rotation by
// (g - 1) i brings slot b H + g i to b H + i, so
//   out = rescale( sum_{i < h} mask_i (x) Rot(X, (g - 1) i) ),
// mask_i the 0/1 plaintext of slots b H + i encoded at scale q_l (rotations
// hoisted per ciphertext): O(h) rotations, products and additions, as the paper
// counts for its own layout.
static Ct reform(Ctx& C, const Ct& x_any, int gap, int h, const int64_t* masks) {
  const Ct x = two_comp(C, x_any);
  std::vector<long> steps(h);
  for (int i = 0; i < h; i++) steps[i] = (long)(gap - 1) * i;
  std::vector<Ct> r = ct_rotate_hoisted(C, x, steps);
  Ct acc;
  for (int i = 0; i < h; i++) {
    std::vector<i64> m(masks + (size_t)i * C.N, masks + (size_t)(i + 1) * C.N);
    Ct t = ct_mul_plain(C, r[i], m);
    acc = i == 0 ? t : ct_add(C, acc, t);
  }
  return ct_rescale(C, acc);
}

// Baby-step giant-step form of the revolver: idx = g i + j (j < g). Since
// rotation commutes with slotwise products and sums,
//   D_{g i + j} = Rot( sum_k Rot(A_k, -g i) (x) Rot(B~_k, j), g i ):
// the n(p-1) rotations of B~ become n(g-1) baby steps of B~, n(ceil(p/g)-1)
// giant steps of A (hoisted per ciphertext) and one rotation by g i of each
// output with i >= 1, after its rescale and relinearisation.
static std::vector<Ct> matmul_bsgs(Ctx& C, const std::vector<Ct>& A, const std::vector<Ct>& B, int p, int g) {
  const int n = (int)A.size(), ng = (p + g - 1) / g;
  const long S = (long)C.N / 2;
  std::vector<long> baby(g), giant(ng);
  for (int j = 0; j < g; j++) baby[j] = j;
  for (int i = 0; i < ng; i++) giant[i] = i == 0 ? 0 : S - (long)g * i;
  std::vector<std::vector<Ct>> Rb(n), Ra(n);
#pragma omp parallel for schedule(dynamic)
  for (int k = 0; k < n; k++) {
    Rb[k] = ct_rotate_hoisted(C, B[k], baby);
    Ra[k] = ct_rotate_hoisted(C, A[k], giant);
  }
  std::vector<Ct> D(p);
#pragma omp parallel for schedule(dynamic)
  for (int idx = 0; idx < p; idx++) {
    const int i = idx / g, j = idx % g;
    Ct T = ct_tensor(C, Ra[0][i], Rb[0][j]);
    for (int k = 1; k < n; k++) T = ct_add(C, T, ct_tensor(C, Ra[k][i], Rb[k][j]));
    Ct d = ct_relin(C, ct_rescale(C, T));
    D[idx] = i == 0 ? d : ct_rotate_hoisted(C, d, {(long)g * i})[0];
  }
  return D;
}

// Zero-rotation ("volley") form of the same product: group g of A's volley
// encoding holds column k at blocks t*M + o_g (M = 1 mod p), so the slotwise
// product with B~_k (period p) already pairs A[i][k] with B[k][(i + idx) mod p]
// for idx = g*per + t: D_g = sum_k Ahat_{g,k} (x) B~_k, rescaled, then
// relinearised. Ahat is group-major ([G][n]); no rotation is performed.
static std::vector<Ct> matmul_volley(Ctx& C, const std::vector<Ct>& Ahat, const std::vector<Ct>& B) {
  const int n = (int)B.size(), G = (int)Ahat.size() / n;
  std::vector<Ct> D(G);
#pragma omp parallel for schedule(dynamic)
  for (int g = 0; g < G; g++) {
    Ct T = ct_tensor(C, Ahat[(size_t)g * n], B[0]);
    for (int k = 1; k < n; k++) T = ct_add(C, T, ct_tensor(C, Ahat[(size_t)g * n + k], B[k]));
    D[g] = ct_relin(C, ct_rescale(C, T));
  }
  return D;
}

// Degree-3 polynomial activation f(x) = c0 + c1 x + c2 x^2 + c3 x^3 (the ACT
// layers of Table I), depth two, as x^2 (c3 x + c2) + (c1 x + c0). With q1, q2
// the primes the two rescales drop and D the input scale:
//   u = relin(rescale(x (x) x))                      level - 1, scale s_u = D D / q1
//   t = rescale(x round(c3 q1)) + round(c2 D)        level - 1, scale D
//   y = rescale(u (x) t)                             level - 2, scale s_y = s_u D / q2
//   v = rescale(x round(c1 s_y q1 / D)) without its last limb, + round(c0 s_y)
//                                                    level - 2, scale s_y
//   f(x) = y + v, three components (relinearised by the next operation).
// Constants enter component 0 only; a scalar times a ciphertext multiplies every
// component.
static Ct drop_last_limb(const Ct& x) {
  Ct r = x;
  for (auto& comp : r.c) comp.pop_back();
  return r;
}

static Ct poly_act3(Ctx& C, const Ct& x_any, const double* c, double D, double& s_out) {
  const Ct x = two_comp(C, x_any);
  const int lp = x.limbs();
  if (lp < 3) throw std::runtime_error("a degree-3 activation needs two levels");
  const u64 q1 = C.q[lp - 1], q2 = C.q[lp - 2];
  const Ct u = ct_relin(C, ct_rescale(C, ct_tensor(C, x, x)));
  const double s_u = (D * D) / (double)q1;
  const Ct t = ct_add_const(C, ct_rescale(C, ct_mul_scalar(C, x, std::llround(c[3] * (double)q1))),
                            std::llround(c[2] * D));
  Ct y = ct_rescale(C, ct_tensor(C, u, t));
  const double s_y = (s_u * D) / (double)q2;
  const Ct v = ct_add_const(
      C, drop_last_limb(ct_rescale(C, ct_mul_scalar(C, x, std::llround(c[1] * s_y * (double)q1 / D)))),
      std::llround(c[0] * s_y));
  for (int comp = 0; comp < 2; comp++)
    for (int i = 0; i < y.limbs(); i++)
      for (size_t n = 0; n < C.N; n++) y.c[comp][i][n] = addmod(y.c[comp][i][n], v.c[comp][i][n], C.q[i]);
  s_out = s_y;
  return y;
}

static i64 quantise(double w, u64 q) { return std::llround(w * (double)q); }

// Convolution outputs sel = [(o, j')] from inputs X[c][j].
// schedule 0: rotate the inputs, then multiply-accumulate (the canonical one).
// schedule 1: multiply-accumulate per row offset a, then rotate the partial
//             sums by g*a and add (the SumForConv order of Alg. 1 / Alg. 4).
static std::vector<Ct> conv2d(Ctx& C, const std::vector<std::vector<Ct>>& X, int gap, const double* Kw,
                              const double* bias, int c_out, int k, int stride, double scale,
                              const std::vector<std::pair<int, int>>& sel, int schedule) {
  const int c_in = (int)X.size();
  const int lp = X[0][0].limbs();
  const u64 ql = C.q[lp - 1];
  auto kw = [&](int o, int c, int a, int b) { return Kw[((o * c_in + c) * k + a) * k + b]; };
  std::vector<Ct> out(sel.size());
  if (schedule == 0) {
    std::set<std::pair<int, int>> need;
    for (auto& s : sel)
      for (int c = 0; c < c_in; c++)
        for (int b = 0; b < k; b++) need.insert({c, stride * s.second + b});
    std::vector<std::pair<int, int>> needv(need.begin(), need.end());
    std::vector<long> steps(k);
    for (int a = 0; a < k; a++) steps[a] = (long)gap * a;
    std::vector<std::vector<Ct>> rot(needv.size());
#pragma omp parallel for schedule(dynamic)
    for (size_t t = 0; t < needv.size(); t++)
      rot[t] = ct_rotate_hoisted(C, two_comp(C, X[needv[t].first][needv[t].second]), steps);
    std::map<std::pair<int, int>, size_t> where;
    for (size_t t = 0; t < needv.size(); t++) where[needv[t]] = t;
#pragma omp parallel for schedule(dynamic)
    for (size_t t = 0; t < sel.size(); t++) {
      const int o = sel[t].first, jp = sel[t].second;
      Ct acc;
      bool first = true;
      for (int c = 0; c < c_in; c++)
        for (int b = 0; b < k; b++)
          for (int a = 0; a < k; a++) {
            Ct term = ct_mul_scalar(C, rot[where.at({c, stride * jp + b})][a], quantise(kw(o, c, a, b), ql));
            acc = first ? term : ct_add(C, acc, term);
            first = false;
          }
      Ct r = ct_rescale(C, acc);
      if (bias) r = ct_add_const(C, r, std::llround(bias[o] * scale));
      out[t] = r;
    }
  } else {
#pragma omp parallel for schedule(dynamic)
    for (size_t t = 0; t < sel.size(); t++) {
      const int o = sel[t].first, jp = sel[t].second;
      Ct acc;
      for (int a = 0; a < k; a++) {
        Ct part;
        bool first = true;
        for (int c = 0; c < c_in; c++)
          for (int b = 0; b < k; b++) {
            Ct term = ct_mul_scalar(C, two_comp(C, X[c][stride * jp + b]), quantise(kw(o, c, a, b), ql));
            part = first ? term : ct_add(C, part, term);
            first = false;
          }
        Ct rotated = ct_rotate_hoisted(C, part, {(long)gap * a})[0];
        acc = a == 0 ? rotated : ct_add(C, acc, rotated);
      }
      Ct r = ct_rescale(C, acc);
      if (bias) r = ct_add_const(C, r, std::llround(bias[o] * scale));
      out[t] = r;
    }
  }
  return out;
}

// Square activation: tensor, rescale; the result keeps three components.
static Ct square(Ctx& C, const Ct& x) { return ct_rescale(C, ct_tensor(C, x, x)); }

// Plaintext of FC weights for output o, input column (c, j): W[o][c][i][j] at
// slot b*H + g*i for every block b < B and valid row i < hv, zero elsewhere,
// encoded at scale q_l.
static std::vector<i64> fc_plaintext(const Ctx& C, const double* W, int o, int c, int j, int c_in, int hv,
                                     int w_in, int gap, int H, int B, u64 ql) {
  std::vector<double> z(C.N / 2, 0.0);
  const size_t row = (size_t)c_in * hv * w_in;
  for (int b = 0; b < B; b++)
    for (int i = 0; i < hv; i++) z[(size_t)b * H + (size_t)gap * i] = W[(size_t)o * row + ((size_t)c * hv + i) * w_in + j];
  return encode(C, z.data(), z.size(), (double)ql);
}

static Ct fc_output(Ctx& C, const std::vector<std::vector<Ct>>& X, const std::vector<std::vector<i64>>& pts /* [c*w+j] */,
                    int gap, int H, double bias_o, bool has_bias, double scale) {
  const int c_in = (int)X.size(), w_in = (int)X[0].size();
  const int lp = X[0][0].limbs();
  const int P = (int)X[0][0].c.size();
  // sum_{c,j} pt (x) X per component, each product a negacyclic product per limb
  Ct acc;
  acc.c.assign(P, RnsPoly(lp, Poly(C.N, 0)));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < lp; i++) {
    const u64 q = C.q[i];
    for (int t = 0; t < P; t++) {
      Poly sum(C.N, 0), x(C.N), y(C.N);
      for (int c = 0; c < c_in; c++)
        for (int j = 0; j < w_in; j++) {
          const std::vector<i64>& pt = pts[(size_t)c * w_in + j];
          for (size_t n = 0; n < C.N; n++) y[n] = reduce_signed(pt[n], q);
          x = X[c][j].c[t][i];
          ntt_fwd(C, i, x.data());
          ntt_fwd(C, i, y.data());
          for (size_t n = 0; n < C.N; n++) sum[n] = addmod(sum[n], mulmod(x[n], y[n], q), q);
        }
      ntt_inv(C, i, sum.data());
      acc.c[t][i] = sum;
    }
  }
  C.cnt.ct_plain += (long)c_in * w_in;
  Ct z = two_comp(C, ct_rescale(C, acc));
  for (int t = gap; t < H; t *= 2) z = ct_add(C, z, ct_rotate_hoisted(C, z, {(long)t})[0]);
  if (has_bias) z = ct_add_const(C, z, std::llround(bias_o * scale));
  return z;
}

}  // namespace oracle

using namespace oracle;

static thread_local std::string g_lerr;
#define OL_TRY(...)                    \
  try {                                \
    __VA_ARGS__;                       \
    return 0;                          \
  } catch (const std::exception& e) {  \
    g_lerr = e.what();                 \
    return -1;                         \
  }

static std::vector<Ct> cts_from(const Ctx& C, const uint64_t* p, int n, int limbs, int polys = 2) {
  std::vector<Ct> v(n);
  for (int t = 0; t < n; t++) v[t] = ct_from(C, p + (size_t)t * polys * limbs * C.N, polys, limbs);
  return v;
}
static void cts_to(const Ctx& C, const std::vector<Ct>& v, uint64_t* p) {
  size_t off = 0;
  for (size_t t = 0; t < v.size(); t++) {
    ct_to(C, v[t], p + off);
    off += v[t].c.size() * v[t].limbs() * C.N;
  }
}

extern "C" {

const char* ol_last_error() { return g_lerr.c_str(); }

// A [n][2][lp][N], B [n][2][lp][N] -> D [p][2][lp-1][N]
int oc_matmul(void* h, const uint64_t* A, const uint64_t* B, int n, int p, int lp, uint64_t* D) {
  OL_TRY(Ctx* C = (Ctx*)h; std::vector<Ct> d = matmul(*C, cts_from(*C, A, n, lp), cts_from(*C, B, n, lp), p);
         cts_to(*C, d, D));
}

// X [c_in][w_in][polys][lp][N]; Wct [c_out][c_in][k][k][2][lp][N]; bias [c_out] or NULL;
// sel [n_sel][2] = (o, j'); out [n_sel][2][lp-1][N].
int oc_conv2d_enc(void* h, const uint64_t* X, int polys, int lp, int c_in, int w_in, int gap, const uint64_t* Wct,
                  const double* bias, int c_out, int k, int stride, double scale, int n_sel, const int* sel,
                  uint64_t* out) {
  OL_TRY(Ctx* C = (Ctx*)h; std::vector<std::vector<Ct>> x(c_in);
         for (int c = 0; c < c_in; c++) x[c] = cts_from(*C, X + (size_t)c * w_in * polys * lp * C->N, w_in, lp, polys);
         std::vector<Ct> w = cts_from(*C, Wct, c_out * c_in * k * k, lp);
         std::vector<std::pair<int, int>> s(n_sel);
         for (int t = 0; t < n_sel; t++) {
           s[t] = {sel[2 * t], sel[2 * t + 1]};
           if (s[t].first < 0 || s[t].first >= c_out || stride * s[t].second + k > w_in) throw std::runtime_error("bad output index");
         }
         std::vector<Ct> r = conv2d_enc(*C, x, gap, w, bias, c_out, k, stride, scale, s);
         cts_to(*C, r, out));
}

// X [n_ct][polys][lp][N]; masks [2][N] (F1, F2 at scale q_{lp-1}) -> out [n_ct][2][lp-1][N]
int oc_vrot(void* h, const uint64_t* X, int n_ct, int polys, int lp, long r, int hw, const int64_t* masks,
            uint64_t* out) {
  OL_TRY(Ctx* C = (Ctx*)h; if (lp < 2 || r < 0 || r >= hw) throw std::runtime_error("bad vRot arguments");
         std::vector<Ct> x = cts_from(*C, X, n_ct, lp, polys); std::vector<Ct> res(n_ct);
         for (int t = 0; t < n_ct; t++) res[t] = vrot(*C, x[t], r, hw, masks); cts_to(*C, res, out));
}

// A, Bbar [2][lp][N] (one ciphertext each); masks [1 + p][N] -> out [2][lp-3][N]
int oc_vr_matmul(void* h, const uint64_t* A, const uint64_t* Bbar, int lp, int n, int p, const int64_t* masks,
                 uint64_t* out) {
  OL_TRY(Ctx* C = (Ctx*)h; if (lp < 4 || n < 1 || p < 1) throw std::runtime_error("bad single-ciphertext matmul shape");
         const Ct r = vr_matmul(*C, cts_from(*C, A, 1, lp)[0], cts_from(*C, Bbar, 1, lp)[0], n, p, masks);
         cts_to(*C, std::vector<Ct>{r}, out));
}

// X [n][polys][lp][N]; S [k*k][2][lp][N]; bias [2][lp-2][N]; masks [k*k][N] -> out [n][2][lp-2][N]
int oc_vr_conv2d(void* h, const uint64_t* X, int n, int polys, int lp, const uint64_t* S, const uint64_t* bias, int k,
                 int Wb, const int64_t* masks, uint64_t* out) {
  try {
    Ctx* C = (Ctx*)h;
    if (k < 1 || lp < 3) throw std::runtime_error("bad single-ciphertext convolution shape");
    std::vector<Ct> x = cts_from(*C, X, n, lp, polys);
    std::vector<Ct> s = cts_from(*C, S, k * k, lp);
    const Ct b = cts_from(*C, bias, 1, lp - 2)[0];
    std::vector<Ct> r(n);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n; t++) r[t] = vr_conv2d(*C, x[t], s, b, k, Wb, masks);
    cts_to(*C, r, out);
    return 0;
  } catch (const std::exception& e) {
    g_lerr = e.what();
    return -1;
  }
}

// X [n][polys][lp][N] at row gap `gap`, masks [h][N] -> out [n][2][lp-1][N] at gap 1
int oc_reform(void* h, const uint64_t* X, int n, int polys, int lp, int gap, int rows, const int64_t* masks,
              uint64_t* out) {
  try {
    Ctx* C = (Ctx*)h;
    if (gap < 2 || rows < 1) throw std::runtime_error("bad ReForm shape");
    std::vector<Ct> x = cts_from(*C, X, n, lp, polys);
    std::vector<Ct> r(n);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n; t++) r[t] = reform(*C, x[t], gap, rows, masks);
    cts_to(*C, r, out);
    return 0;
  } catch (const std::exception& e) {
    g_lerr = e.what();
    return -1;
  }
}

// A, B [n][2][lp][N] -> D [p][2][lp-1][N], baby-step size g
int oc_matmul_bsgs(void* h, const uint64_t* A, const uint64_t* B, int n, int p, int g, int lp, uint64_t* D) {
  OL_TRY(Ctx* C = (Ctx*)h; if (g < 1 || g > p) throw std::runtime_error("baby-step size out of range");
         std::vector<Ct> d = matmul_bsgs(*C, cts_from(*C, A, n, lp), cts_from(*C, B, n, lp), p, g); cts_to(*C, d, D));
}

// Ahat [G][n][2][lp][N] (volley encoding of A), B [n][2][lp][N] -> D [G][2][lp-1][N]
int oc_matmul_volley(void* h, const uint64_t* Ahat, const uint64_t* B, int n, int G, int lp, uint64_t* D) {
  OL_TRY(Ctx* C = (Ctx*)h; std::vector<Ct> d = matmul_volley(*C, cts_from(*C, Ahat, n * G, lp), cts_from(*C, B, n, lp));
         cts_to(*C, d, D));
}

// X [n][polys][lp][N] (polys 2 or 3), coeffs c0..c3 -> out [n][3][lp-2][N]; *scale_out
int oc_poly_act3(void* h, const uint64_t* X, int n, int polys, int lp, const double* coeffs, double scale,
                 uint64_t* out, double* scale_out) {
  try {
    Ctx* C = (Ctx*)h;
    if (lp < 3) throw std::runtime_error("a degree-3 activation needs two levels");
    std::vector<Ct> x = cts_from(*C, X, n, lp, polys);
    std::vector<Ct> r(n);
    std::vector<double> so(n, scale);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n; t++) r[t] = poly_act3(*C, x[t], coeffs, scale, so[t]);
    *scale_out = so[0];
    cts_to(*C, r, out);
    return 0;
  } catch (const std::exception& e) {
    g_lerr = e.what();
    return -1;
  }
}

// X [c_in][w_in][polys][lp][N] (polys 2, or 3 for unrelinearised products);
// K [c_out][c_in][k][k]; bias [c_out] or NULL;
// sel [n_sel][2] = (o, j'); out [n_sel][2][lp-1][N].
int oc_conv2d(void* h, const uint64_t* X, int polys, int lp, int c_in, int w_in, int gap, const double* K,
              const double* bias, int c_out, int k, int stride, double scale, int n_sel, const int* sel, int schedule,
              uint64_t* out) {
  OL_TRY(Ctx* C = (Ctx*)h; std::vector<std::vector<Ct>> x(c_in);
         for (int c = 0; c < c_in; c++) x[c] = cts_from(*C, X + (size_t)c * w_in * polys * lp * C->N, w_in, lp, polys);
         std::vector<std::pair<int, int>> s(n_sel);
         for (int t = 0; t < n_sel; t++) {
           s[t] = {sel[2 * t], sel[2 * t + 1]};
           if (s[t].first < 0 || s[t].first >= c_out || stride * s[t].second + k > w_in) throw std::runtime_error("bad output index");
         }
         std::vector<Ct> r = conv2d(*C, x, gap, K, bias, c_out, k, stride, scale, s, schedule);
         cts_to(*C, r, out));
}

// x [n][2][lp][N] -> [n][3][lp-1][N]
int oc_square(void* h, const uint64_t* X, int n, int lp, uint64_t* out) {
  try {
    Ctx* C = (Ctx*)h;
    std::vector<Ct> x = cts_from(*C, X, n, lp);
    std::vector<Ct> r(n);
    for (int t = 0; t < n; t++) r[t] = square(*C, x[t]);
    cts_to(*C, r, out);
    return 0;
  } catch (const std::exception& e) {
    g_lerr = e.what();
    return -1;
  }
}

// FC plaintexts for outputs sel_o: pts [n_sel][c_in][w_in][N] (int64 coefficients)
int oc_fc_plaintexts(void* h, int lp, int c_in, int hv, int w_in, int gap, int H, int B, const double* W, int n_sel,
                     const int* sel_o, int64_t* pts) {
  Ctx* C = (Ctx*)h;
  const u64 ql = C->q[lp - 1];
  const long tot = (long)n_sel * c_in * w_in;
#pragma omp parallel for schedule(dynamic)
  for (long t = 0; t < tot; t++) {
    const int s = (int)(t / ((long)c_in * w_in)), rem = (int)(t % ((long)c_in * w_in));
    std::vector<i64> pt = fc_plaintext(*C, W, sel_o[s], rem / w_in, rem % w_in, c_in, hv, w_in, gap, H, B, ql);
    std::memcpy(pts + (size_t)t * C->N, pt.data(), C->N * 8);
  }
  return 0;
}

// X [c_in][w_in][polys][lp][N]; pts [n_sel][c_in][w_in][N] from oc_fc_plaintexts;
// bias [out] or NULL; out [n_sel][2][lp-1][N].
int oc_fc(void* h, const uint64_t* X, int polys, int lp, int c_in, int w_in, int gap, int H, const int64_t* pts,
          const double* bias, double scale, int n_sel, const int* sel_o, uint64_t* out) {
  OL_TRY(Ctx* C = (Ctx*)h; std::vector<std::vector<Ct>> x(c_in);
         for (int c = 0; c < c_in; c++) x[c] = cts_from(*C, X + (size_t)c * w_in * polys * lp * C->N, w_in, lp, polys);
         for (int s = 0; s < n_sel; s++) {
           std::vector<std::vector<i64>> p((size_t)c_in * w_in);
           for (size_t t = 0; t < p.size(); t++) {
             const int64_t* src = pts + ((size_t)s * c_in * w_in + t) * C->N;
             p[t].assign(src, src + C->N);
           }
           Ct z = fc_output(*C, x, p, gap, H, bias ? bias[sel_o[s]] : 0.0, bias != nullptr, scale);
           ct_to(*C, z, out + (size_t)s * 2 * (lp - 1) * C->N);
         });
}

}  // extern "C"
