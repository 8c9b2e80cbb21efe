// kernels.cu - element-wise, base-conversion, key-switching and layer kernels
// of the RNS-CKKS engine. Every kernel works on residues in [0, q) and writes
// residues in [0, q); one thread handles one coefficient position, so global
// reads and writes are coalesced along the N axis of each limb.
//
// Key switching is the hybrid scheme (digits of alpha primes): ModUp by fast
// base conversion without correction, inner product with the key over the
// Q*P basis, ModDown by (u_Q - BConv_P->Q(u_P)) P^{-1}. A Galois automorphism
// phi_k acts on an NTT-domain limb as the permutation
//   pi_k(j) = brv(((2 brv(j) + 1) k mod 2N - 1) / 2)
// (evaluation point psi^(2 brv(j) + 1) goes to psi^((2 brv(j) + 1) k)), which
// the kernels apply as gathers.
#include "he_internal.h"

namespace he {

namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(size_t total) {
  size_t b = (total + kBlock - 1) / kBlock;
  const size_t cap = 152 * 32;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (unsigned)b;
}

#define HE_GRID_LOOP(idx, total) \
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (total); idx += (size_t)gridDim.x * blockDim.x)


__device__ __forceinline__ u64 reduce_i64(int64_t v, const Mod& m) {
  if (v >= 0) return reduce128(0, (u64)v, m);
  const u64 r = reduce128(0, (u64)(-(v + 1)) + 1, m);  // |v| without overflow at INT64_MIN
  return r ? m.q - r : 0;
}

// ---------------------------------------------------------------------------
__global__ void k_reduce_signed_kernel(const int64_t* in, u64* out, int n, LimbMap lm, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n * lm.lpp * N;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1);
    const size_t row = idx >> log_n;
    const int i = (int)(row % lm.lpp), p = (int)(row / lm.lpp);
    out[(size_t)p * lm.poly_stride + (size_t)lm.mem(i) * N + j] = reduce_i64(in[(size_t)p * N + j], pt[lm.prime(i)].mod);
  }
}

__global__ void k_reduce_small_kernel(const int8_t* in, u64* out, int n, LimbMap lm, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n * lm.lpp * N;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1);
    const size_t row = idx >> log_n;
    const int i = (int)(row % lm.lpp), p = (int)(row / lm.lpp);
    const int v = in[(size_t)p * N + j];
    const u64 q = pt[lm.prime(i)].mod.q;
    out[(size_t)p * lm.poly_stride + (size_t)lm.mem(i) * N + j] = v >= 0 ? (u64)v : q - (u64)(-v);
  }
}

// ct0 = v pk0 + e0 + m, ct1 = v pk1 + e1 (inputs [n][limbs][N], pk [2][L1][N])
__global__ void k_encrypt_kernel(const u64* v, const u64* e0, const u64* e1, const u64* m, const u64* pk, u64* ct,
                                 int n, int limbs, int L1, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n * limbs * N;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1);
    const size_t row = idx >> log_n;
    const int i = (int)(row % limbs), c = (int)(row / limbs);
    const Mod md = pt[i].mod;
    const u64 vv = v[idx];
    const u64 p0 = pk[(size_t)i * N + j], p1 = pk[((size_t)L1 + i) * N + j];
    const size_t o = ((size_t)c * 2 * limbs + i) * N + j;
    ct[o] = addmod(addmod(mulmod(vv, p0, md), e0[idx], md.q), m[idx], md.q);
    ct[o + (size_t)limbs * N] = addmod(mulmod(vv, p1, md), e1[idx], md.q);
  }
}

// b = -a s + e + [g in digit] (P mod q_g) s'  over all L1+K primes
__global__ void k_ksk_kernel(const u64* a, const u64* e, const u64* s, const u64* sp, u64* b, int digit, int alpha,
                             int L1, int np, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)np * N;
  HE_GRID_LOOP(idx, total) {
    const int g = (int)(idx >> log_n);
    const PrimeTab P = pt[g];
    const u64 q = P.mod.q;
    u64 r = submod(e[idx], mulmod(a[idx], s[idx], P.mod), q);
    if (g < L1 && g / alpha == digit) r = addmod(r, mulmod(P.pmod, sp[idx], P.mod), q);
    b[idx] = r;
  }
}

__global__ void k_mont_form_kernel(u64* data, int n, LimbMap lm, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n * lm.lpp * N;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1), row = idx >> log_n;
    const int i = (int)(row % lm.lpp), p = (int)(row / lm.lpp);
    const PrimeTab& T = pt[lm.prime(i)];
    u64* x = data + (size_t)p * lm.poly_stride + (size_t)lm.mem(i) * N + j;
    *x = shoup(*x, T.mont_r, T.mont_r_sh, T.mod.q);
  }
}

__global__ void k_mul_kernel(const u64* a, const u64* b, u64* out, int n, LimbMap lm, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n * lm.lpp * N;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1);
    const size_t row = idx >> log_n;
    const int i = (int)(row % lm.lpp), p = (int)(row / lm.lpp);
    const size_t o = (size_t)p * lm.poly_stride + (size_t)lm.mem(i) * N + j;
    out[o] = mulmod(a[o], b[o], pt[lm.prime(i)].mod);
  }
}

__global__ void k_permute_kernel(const u64* in, u64* out, size_t rows, u64 k, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = rows * N;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1), r = idx >> log_n;
    out[idx] = in[r * N + galois_index((u32)j, k, log_n)];
  }
}

__global__ void k_decrypt0_kernel(const u64* ct, const u64* s, int limbs, int n, u64* out, const PrimeTab* pt,
                                  int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n * N;
  const Mod md = pt[0].mod;
  HE_GRID_LOOP(idx, total) {
    const size_t j = idx & (N - 1), c = idx >> log_n;
    const u64* x = ct + c * 2 * limbs * N;
    out[idx] = addmod(x[j], mulmod(x[(size_t)limbs * N + j], s[j], md), md.q);
  }
}

__global__ void k_add_kernel(const u64* a, const u64* b, u64* out, int n_polys, int limbs, const PrimeTab* pt,
                             int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = (size_t)n_polys * limbs * N;
  HE_GRID_LOOP(idx, total) {
    const int i = (int)((idx >> log_n) % limbs);
    out[idx] = addmod(a[idx], b[idx], pt[i].mod.q);
  }
}

// d[c] = (a0 b0, a0 b1 + a1 b0, a1 b1) for ciphertext c = blockIdx.y; a square (a = b)
// takes one cross product, doubled, and reads one operand.
// d = (a0 b0, a0 b1 + a1 b0, a1 b1) per word. Products by Montgomery's reduction (Math. Comp.
// 1985): one operand is first put in Montgomery form by a Shoup product with R = 2^64 mod q, so
// that redc(aR * b) = a b mod q exactly, cheaper than a 128-bit Barrett reduction per product.
__global__ void k_tensor_kernel(const u64* a, const u64* b, u64* d, int n, int limbs, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t c = blockIdx.y;
  const u64* A = a + c * 2 * LN;
  const u64* B = b + c * 2 * LN;
  u64* D = d + c * 3 * LN;
  const bool square = a == b;
  int limb = -1;  // the prime's constants are reloaded only when the stride crosses into another limb
  u64 q = 0, R = 0, Rs = 0, qneg = 0;
  for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < LN; w += (size_t)gridDim.x * blockDim.x) {
    if ((int)(w >> log_n) != limb) {
      limb = (int)(w >> log_n);
      q = pt[limb].mod.q;
      R = pt[limb].mont_r;
      Rs = pt[limb].mont_r_sh;
      qneg = pt[limb].qinv_neg;
    }
    auto mont = [&](u64 xr, u64 y) {  // xr y 2^-64 mod q for xr, y < q
      u64 h, l;
      mul128(xr, y, h, l);
      return redc128(h, l, q, qneg);
    };
    const u64 a0 = A[w], a1 = A[LN + w];
    const u64 a0r = shoup(a0, R, Rs, q), a1r = shoup(a1, R, Rs, q);
    if (square) {
      D[w] = mont(a0r, a0);
      const u64 t = mont(a0r, a1);
      D[LN + w] = addmod(t, t, q);
      D[2 * LN + w] = mont(a1r, a1);
    } else {
      const u64 b0 = B[w], b1 = B[LN + w];
      D[w] = mont(a0r, b0);
      D[LN + w] = addmod(mont(a0r, b1), mont(a1r, b0), q);
      D[2 * LN + w] = mont(a1r, b1);
    }
  }
}


// u[s][c][comp][pos] = sum_j ext[c][j][pos] key_s[j][comp][g(pos)] for the
// steps s of one launch. A block owns one limb position `pos` and a tile of
// KS_TILE coefficients: it reads that tile of every key once into shared
// memory, the two components of a key word side by side (one 16-byte load
// per digit; each thread only touches its own column, so no barrier is
// needed), and then walks all n ciphertexts, loading the next ciphertext's
// digits while the current one is accumulated. Key traffic is one read per
// launch instead of one per ciphertext.
constexpr int KS_TILE = 128;
template <int MAXB>
__global__ void __launch_bounds__(KS_TILE) k_ks_inner_kernel(const u64* __restrict__ ext, const u64* __restrict__ own,
                                                             size_t own_stride, int alpha, KeyPtrs keys, int S,
                                                             u64* __restrict__ u, int n, int limbs, int beta, int L1,
                                                             int K, const PrimeTab* pt, int log_n) {
  extern __shared__ ulonglong2 skey[];  // [S][beta][KS_TILE] (component 0, component 1)
  const size_t N = (size_t)1 << log_n;
  const int nb = limbs + K, npk = L1 + K;
  const int pos = blockIdx.y;
  const int g = pos < limbs ? pos : L1 + (pos - limbs);
  const size_t jn = (size_t)blockIdx.x * KS_TILE + threadIdx.x;
  if (jn >= N) return;
  for (int st = 0; st < S; st++)
    for (int dg = 0; dg < beta; dg++) {
      const u64* kp = keys.k[st] + ((size_t)dg * 2 * npk + g) * N + jn;
      skey[(st * beta + dg) * KS_TILE + threadIdx.x] = make_ulonglong2(__ldg(kp), __ldg(kp + (size_t)npk * N));
    }
  const Mod md = pt[g].mod;
  const u64 qneg = pt[g].qinv_neg;
  const size_t ustep = (size_t)n * 2 * nb * N;
  const size_t cstride = (size_t)beta * nb * N;
  // digit dg at this position: the ModUp output, or for the digit's own primes the input itself
  const u64* Ep = ext + (size_t)pos * N + jn;
  const u64* Op = own + (size_t)pos * N + jn;
  const int own_dg = pos < limbs ? pos / alpha : -1;
  auto digit = [&](int c, int dg) {
    return dg == own_dg ? Op[(size_t)c * own_stride] : Ep[(size_t)c * cstride + (size_t)dg * nb * N];
  };
  u64 e[MAXB];
#pragma unroll
  for (int dg = 0; dg < MAXB; dg++) e[dg] = dg < beta ? digit(0, dg) : 0;
  for (int c = 0; c < n; c++) {
    u64 en[MAXB];
    const int cn = c + 1 < n ? c + 1 : c;
#pragma unroll
    for (int dg = 0; dg < MAXB; dg++) en[dg] = dg < beta ? digit(cn, dg) : 0;
    u64* U = u + (size_t)c * 2 * nb * N + (size_t)pos * N + jn;
    if (md.q < kMac96Prime) {  // uniform across the block: beta products of residues fit 96 bits
      for (int st = 0; st < S; st++) {
        const ulonglong2* kk = skey + (size_t)st * beta * KS_TILE + threadIdx.x;
        Acc96 a0{0, 0, 0}, a1{0, 0, 0};
#pragma unroll
        for (int dg = 0; dg < MAXB; dg++) {
          if (dg < beta) {
            const ulonglong2 kv = kk[dg * KS_TILE];
            mac96(a0, e[dg], kv.x);
            mac96(a1, e[dg], kv.y);
          }
        }
        U[st * ustep] = redc128(a0.w2, ((u64)a0.w1 << 32) | a0.w0, md.q, qneg);
        U[st * ustep + (size_t)nb * N] = redc128(a1.w2, ((u64)a1.w1 << 32) | a1.w0, md.q, qneg);
      }
    } else {
      for (int st = 0; st < S; st++) {
        const ulonglong2* kk = skey + (size_t)st * beta * KS_TILE + threadIdx.x;
        Acc128 a0{0, 0}, a1{0, 0};
#pragma unroll
        for (int dg = 0; dg < MAXB; dg++) {
          if (dg < beta) {
            const ulonglong2 kv = kk[dg * KS_TILE];
            mac128(a0, e[dg], kv.x);
            mac128(a1, e[dg], kv.y);
          }
        }
        // keys are in Montgomery form: the reduction divides the sum by 2^64 (beta q^2 < q 2^64)
        U[st * ustep] = redc128(a0.hi, a0.lo, md.q, qneg);
        U[st * ustep + (size_t)nb * N] = redc128(a1.hi, a1.lo, md.q, qneg);
      }
    }
#pragma unroll
    for (int dg = 0; dg < MAXB; dg++) e[dg] = en[dg];
  }
}

__global__ void k_gather_p_kernel(const u64* u, u64* p, int n, int limbs, int K, u64 k, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const int nb = limbs + K;
  const size_t total = (size_t)n * 2 * K * N;
  HE_GRID_LOOP(idx, total) {
    const size_t jn = idx & (N - 1);
    const size_t r = idx >> log_n;
    const int kk = (int)(r % K);
    const size_t cc = r / K;  // ciphertext * 2 + component
    const u32 src = k == 1 ? (u32)jn : galois_index((u32)jn, k, log_n);
    p[idx] = u[(cc * nb + limbs + kk) * N + src];
  }
}

// Rescale by q_l: out_i = (x_i + h - r) q_l^{-1} with h = floor(q_l/2) added to
// EVERY coefficient and r = (x_l + h) mod q_l. The expansion below forms
// r - h mod q_i per coefficient (coefficient domain) so that, after its
// forward NTT, the combine is out_i = (x_i - NTT(r - h)) q_l^{-1}.
// Rescale constants (words of d_rs): [L1+1][L1][3] = floor(q_l/2) mod q_i, q_l^{-1} mod q_i, Shoup
__global__ void k_rescale_expand_kernel(const u64* last, u64* r, int rows, int limbs, const u64* rs,
                                        const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const int lo = limbs - 1;
  const size_t total = (size_t)rows * N;
  const Mod ml = pt[lo].mod;
  const u64 half = ml.q >> 1;
  HE_GRID_LOOP(idx, total) {
    const size_t jn = idx & (N - 1), row = idx >> log_n;
    const u64 v = addmod(last[idx], half, ml.q);
    for (int i = 0; i < lo; i++)
      r[(row * lo + i) * N + jn] = submod(reduce128(0, v, pt[i].mod), rs[(size_t)i * 3], pt[i].mod.q);
  }
}

__global__ void k_rescale_combine_kernel(const u64* x, const u64* r, u64* out, int rows, int limbs, const u64* rs,
                                         const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const int lo = limbs - 1;
  const size_t total = (size_t)rows * lo * N;
  HE_GRID_LOOP(idx, total) {
    const size_t jn = idx & (N - 1);
    const size_t rr = idx >> log_n;
    const int i = (int)(rr % lo);
    const size_t row = rr / lo;
    const u64 q = pt[i].mod.q;
    const u64* t = rs + (size_t)i * 3;
    const u64 xi = x[(row * limbs + i) * N + jn];
    out[idx] = shoup(submod(xi, r[idx], q), t[1], t[2], q);
  }
}

__global__ void k_add_const_kernel(u64* ct, int n, int limbs, const u64* cdev, int per_group, const PrimeTab* pt,
                                   int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t total = (size_t)n * LN;
  HE_GRID_LOOP(idx, total) {
    const size_t c = idx / LN, w = idx - c * LN;
    const int i = (int)(w >> log_n);
    u64* p = ct + c * 2 * LN + w;
    *p = addmod(*p, cdev[(c / per_group) * limbs + i], pt[i].mod.q);
  }
}

// out = in * w_i mod q_i for rows [rows][limbs][N] (every component of every
// ciphertext); wsh [limbs][2]: the integer's residue mod q_i and its Shoup companion.
__global__ void k_mul_const_kernel(const u64* in, u64* out, size_t rows, int limbs, const u64* wsh,
                                   const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = rows * limbs * N;
  HE_GRID_LOOP(idx, total) {
    const int i = (int)((idx >> log_n) % (size_t)limbs);
    out[idx] = shoup(in[idx], wsh[2 * i], wsh[2 * i + 1], pt[i].mod.q);
  }
}

// y[c][comp] += v[c][comp] for comp < 2: y [n][ypolys][limbs][N], v [n][2][limbs][N]
__global__ void k_add_comps_kernel(u64* y, const u64* v, int n, int ypolys, int limbs, const PrimeTab* pt,
                                   int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t total = (size_t)n * 2 * LN;
  HE_GRID_LOOP(idx, total) {
    const size_t c = idx / (2 * LN), w = idx - c * 2 * LN;
    const int i = (int)((w >> log_n) % (size_t)limbs);
    u64* p = y + c * ypolys * LN + w;
    *p = addmod(*p, v[idx], pt[i].mod.q);
  }
}

// Convolution multiply-accumulate. rot [c_in][w_in][k][2][limbs][N] holds
// Rot(X_{c,j}, gap a) at [c][j][a]; w [c_out][c_in][k][k][limbs][2] holds the
// integer weights mod q_i and Shoup companions ([o][c][a][b]). A block works
// on one (component, limb) and 2 * blockDim.x coefficients; its weights for
// that limb are staged in shared memory (every thread reads the same weight,
// a broadcast). Each thread computes TN adjacent coefficients of OB output
// channels for the output columns jp = blockIdx.z, blockIdx.z + gridDim.z, ...
// NAR (primes below kNarrowPrime): the products take the cheaper quotient
// estimate and lie in [0, 4q); otherwise Shoup's lazy products in [0, 2q).
template <int OB, int TN, bool NAR>
__device__ __forceinline__ void conv_mac_body(const ulonglong2* sw, const u64* rot, u64* out, int c_in, int w_in,
                                              int k, int stride, int c_out, int w_out, size_t LN, size_t off, u64 q,
                                              u64 one_sh) {
  const int T = c_in * k * k;
  // lazy products are below 2q (4q): a word holds `room` of them on top of a reduced sum
  const u64 fit = (~0ull) / ((NAR ? 4 : 2) * q) - 1;
  const int room = fit > (1u << 20) ? (1 << 20) : (int)fit;
  for (int jp = blockIdx.z; jp < w_out; jp += gridDim.z) {
    for (int o0 = 0; o0 < c_out; o0 += OB) {
      u64 acc[OB][TN];
#pragma unroll
      for (int t = 0; t < OB; t++)
#pragma unroll
        for (int v = 0; v < TN; v++) acc[t][v] = 0;
      int pending = 0;
      for (int c = 0; c < c_in; c++)
        for (int b = 0; b < k; b++) {
          const u64* src = rot + ((size_t)(c * w_in + stride * jp + b) * k) * 2 * LN + off;
          for (int a = 0; a < k; a++) {
            u64 x[TN];
            if constexpr (TN == 2) {
              const ulonglong2 xx = *reinterpret_cast<const ulonglong2*>(src + (size_t)a * 2 * LN);
              x[0] = xx.x;
              x[1] = xx.y;
            } else {
#pragma unroll
              for (int v = 0; v < TN; v++) x[v] = src[(size_t)a * 2 * LN + v];
            }
            const ulonglong2* wr = sw + (size_t)o0 * T + (c * k + a) * k + b;
            if (pending == room) {  // uniform across the block
#pragma unroll
              for (int t = 0; t < OB; t++)
#pragma unroll
                for (int v = 0; v < TN; v++) acc[t][v] = shoup_lazy(acc[t][v], 1, one_sh, q);
              pending = 0;
            }
            pending++;
#pragma unroll
            for (int t = 0; t < OB; t++) {
              if (o0 + t < c_out) {
                const ulonglong2 ww = wr[(size_t)t * T];
#pragma unroll
                for (int v = 0; v < TN; v++)
                  acc[t][v] += NAR ? shoup_approx(x[v], ww.x, ww.y, q) : shoup_lazy(x[v], ww.x, ww.y, q);
              }
            }
          }
        }
#pragma unroll
      for (int t = 0; t < OB; t++) {
        if (o0 + t < c_out) {
          u64* dst = out + ((size_t)(o0 + t) * w_out + jp) * 2 * LN + off;
#pragma unroll
          for (int v = 0; v < TN; v++) dst[v] = shoup(acc[t][v], 1, one_sh, q);
        }
      }
    }
  }
}

template <int OB, int TN>
__global__ void k_conv_mac_kernel(const u64* rot, u64* out, const u64* w, int c_in, int w_in, int k, int stride,
                                  int c_out, int w_out, int limbs, const PrimeTab* pt, int log_n) {
  extern __shared__ ulonglong2 sw[];  // [c_out][c_in k k]
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const int i = blockIdx.y % limbs, comp = blockIdx.y / limbs;
  if (pt[i].mod.q < kMac96Prime) return;  // uniform across the block
  const int T = c_in * k * k;
  for (int id = threadIdx.x; id < c_out * T; id += blockDim.x)
    sw[id] = *reinterpret_cast<const ulonglong2*>(w + ((size_t)id * limbs + i) * 2);
  __syncthreads();
  const size_t n0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * TN;
  if (n0 >= N) return;
  const u64 q = pt[i].mod.q, one_sh = pt[i].one_sh;
  if (q < kMac96Prime) return;  // k_conv_mac96_kernel's limbs (uniform across the block)
  const size_t off = (size_t)comp * LN + (size_t)i * N + n0;
  if (q < kNarrowPrime)
    conv_mac_body<OB, TN, true>(sw, rot, out, c_in, w_in, k, stride, c_out, w_out, LN, off, q, one_sh);
  else
    conv_mac_body<OB, TN, false>(sw, rot, out, c_in, w_in, k, stride, c_out, w_out, LN, off, q, one_sh);
}

// The same multiply-accumulate for limbs whose prime is below kMac96Prime: each
// product goes into a 96-bit sum (seven 32-bit multiplies, no per-term reduction;
// Barrett once every `room` terms and at the end). Each thread computes TN
// adjacent coefficients of OB output channels (one shared-memory weight serves TN
// products); the weights (residues only) are staged in shared memory. Blocks of
// other limbs return at once (the Shoup kernel takes them).
template <int OB, int TN>
__global__ void __launch_bounds__(128, 6) k_conv_mac96_kernel(const u64* rot, u64* out, const u64* w, int c_in, int w_in,
                                                           int k, int stride, int c_out, int w_out, int limbs,
                                                           const PrimeTab* pt, int log_n) {
  static_assert(TN == 2 && OB % 2 == 0, "two adjacent coefficients a thread, channels in pairs");
  // weights of this limb in term order (c, b, a), the channels of a term side by side:
  // [T][cp], cp = c_out rounded up to even, so a pair of channels is one 16-byte load
  extern __shared__ ulonglong2 sw128[];
  u64* sw64 = reinterpret_cast<u64*>(sw128);
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const int i = blockIdx.y % limbs, comp = blockIdx.y / limbs;
  const Mod md = pt[i].mod;
  if (md.q >= kMac96Prime) return;  // uniform across the block
  const int kk = k * k, T = c_in * kk, cp = (c_out + 1) & ~1;
  for (int id = threadIdx.x; id < T * cp; id += blockDim.x) {
    const int term = id / cp, o = id - term * cp;
    const int c = term / kk, r = term - c * kk, b = r / k, a = r - b * k;  // term = (c k + b) k + a
    sw64[id] = o < c_out ? w[(((size_t)o * T + (c * k + a) * k + b) * limbs + i) * 2] : 0;
  }
  __syncthreads();
  const size_t n0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * TN;
  if (n0 >= N) return;
  const size_t off = (size_t)comp * LN + (size_t)i * N + n0;
  const int room = mac96_room(md.q);
  // rot [c][j][a][2][LN]: for one channel c the terms (b, a) of output column jp are consecutive
  // blocks of 2 LN words (column j = stride jp + b, rotation a); the next channel starts w_in k
  // blocks further
  const size_t step = 2 * LN, chan = (size_t)w_in * k * 2 * LN;
  for (int jp = blockIdx.z; jp < w_out; jp += gridDim.z) {
    for (int o0 = 0; o0 < c_out; o0 += OB) {
      Acc96 acc[OB][TN];
#pragma unroll
      for (int t = 0; t < OB; t++)
#pragma unroll
        for (int v = 0; v < TN; v++) acc[t][v] = Acc96{0, 0, 0};
      int pending = 0;
      const u64* cbase = rot + (size_t)stride * jp * k * 2 * LN + off;  // channel 0, b = 0, a = 0
      const u64* p = cbase;
      const u64* wr = sw64 + o0;
      ulonglong2 nx = *reinterpret_cast<const ulonglong2*>(p);  // loaded a term ahead
      int r = 0;                                                // (b, a) index inside the channel
      for (int term = 0; term < T; term++) {
        const u64 x0 = nx.x, x1 = nx.y;
        if (++r == kk) {
          r = 0;
          cbase += chan;
          p = cbase;
        } else {
          p += step;
        }
        if (term + 1 < T) nx = *reinterpret_cast<const ulonglong2*>(p);
        if (pending == room) {  // uniform across the block
#pragma unroll
          for (int t = 0; t < OB; t++)
#pragma unroll
            for (int v = 0; v < TN; v++) {
              const u64 rr = reduce96(acc[t][v], md);
              acc[t][v] = Acc96{(u32)rr, (u32)(rr >> 32), 0};
            }
          pending = 0;
        }
        pending++;
#pragma unroll
        for (int t2 = 0; t2 < OB / 2; t2++) {
          // a pair of channels exists in the weight row (cp words, cp even) only if its first
          // channel does: the load stays inside the row, and inside the array at the last term
          if (o0 + 2 * t2 < c_out) {
            const ulonglong2 ww = reinterpret_cast<const ulonglong2*>(wr)[t2];
            mac96(acc[2 * t2][0], x0, ww.x);
            mac96(acc[2 * t2][1], x1, ww.x);
            if (o0 + 2 * t2 + 1 < c_out) {
              mac96(acc[2 * t2 + 1][0], x0, ww.y);
              mac96(acc[2 * t2 + 1][1], x1, ww.y);
            }
          }
        }
        wr += cp;
      }
#pragma unroll
      for (int t = 0; t < OB; t++)
        if (o0 + t < c_out)
#pragma unroll
          for (int v = 0; v < TN; v++) out[((size_t)(o0 + t) * w_out + jp) * 2 * LN + off + v] = reduce96(acc[t][v], md);
    }
  }
}

// Convolution with encrypted kernels: out[o][j'] (3 components) = sum_{c,b,a}
// tensor(W[o][c][a][b], R[c][s j' + b][a]); W [c_out][c_in][k][k][2][limbs][N]
// kernel ciphertexts, R [c_in][w_in][k][2][limbs][N] the hoisted rotations, out
// [c_out][w_out][3][limbs][N]. A thread owns one word position (limb,
// coefficient) and a tile of CO output channels x CJ output columns (blockIdx.y
// enumerates the tiles), so each kernel word is read once per CJ columns and
// each rotated input word once per CO channels. 128-bit sums, reduced every 8
// terms.
template <int CO, int CJ>
__global__ void __launch_bounds__(128) k_conv_enc_mac_kernel(const u64* R, const u64* W, u64* out, int c_in, int w_in, int k, int stride,
                                      int c_out, int w_out, int limbs, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const int tj = (w_out + CJ - 1) / CJ;
  const int o0 = (blockIdx.y / tj) * CO, j0 = (blockIdx.y % tj) * CJ;
  HE_GRID_LOOP(w, LN) {
    const int i = (int)(w >> log_n);
    const Mod md = pt[i].mod;
    Acc128 acc[CO][CJ][3];
#pragma unroll
    for (int t = 0; t < CO; t++)
#pragma unroll
      for (int u = 0; u < CJ; u++)
#pragma unroll
        for (int d = 0; d < 3; d++) acc[t][u][d] = Acc128{0, 0};
    int terms = 0;
    for (int c = 0; c < c_in; c++)
      for (int b = 0; b < k; b++)
        for (int a = 0; a < k; a++) {
          u64 w0[CO], w1[CO], r0[CJ], r1[CJ];
#pragma unroll
          for (int t = 0; t < CO; t++) {
            const int o = o0 + t < c_out ? o0 + t : c_out - 1;
            const u64* wp = W + ((((size_t)o * c_in + c) * k + a) * k + b) * 2 * LN + w;
            w0[t] = wp[0];
            w1[t] = wp[LN];
          }
#pragma unroll
          for (int u = 0; u < CJ; u++) {
            const int jp = j0 + u < w_out ? j0 + u : w_out - 1;
            const u64* rp = R + (((size_t)(c * w_in + stride * jp + b) * k + a) * 2) * LN + w;
            r0[u] = rp[0];
            r1[u] = rp[LN];
          }
#pragma unroll
          for (int t = 0; t < CO; t++)
#pragma unroll
            for (int u = 0; u < CJ; u++) {
              mac128(acc[t][u][0], w0[t], r0[u]);
              mac128(acc[t][u][1], w0[t], r1[u]);
              mac128(acc[t][u][1], w1[t], r0[u]);
              mac128(acc[t][u][2], w1[t], r1[u]);
            }
          if ((++terms & 7) == 0) {
#pragma unroll
            for (int t = 0; t < CO; t++)
#pragma unroll
              for (int u = 0; u < CJ; u++)
#pragma unroll
                for (int d = 0; d < 3; d++) acc[t][u][d] = Acc128{0, reduce128(acc[t][u][d].hi, acc[t][u][d].lo, md)};
          }
        }
#pragma unroll
    for (int t = 0; t < CO; t++)
#pragma unroll
      for (int u = 0; u < CJ; u++) {
        if (o0 + t < c_out && j0 + u < w_out) {
          u64* dst = out + ((size_t)(o0 + t) * w_out + j0 + u) * 3 * LN + w;
#pragma unroll
          for (int d = 0; d < 3; d++) dst[(size_t)d * LN] = reduce128(acc[t][u][d].hi, acc[t][u][d].lo, md);
        }
      }
  }
}

// d[idx] (3 components) = sum_k tensor(A_k, R[k][idx]), idx < p; R [n][rstride][2][limbs][N]
__global__ void k_matmul_acc_kernel(const u64* A, const u64* R, u64* d, int n, int p, int rstride, int limbs,
                                    const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t total = (size_t)p * LN;
  HE_GRID_LOOP(idx, total) {
    const size_t w = idx % LN;
    const int id = (int)(idx / LN);
    const int i = (int)(w >> log_n);
    const Mod md = pt[i].mod;
    Acc128 s0{0, 0}, s1{0, 0}, s2{0, 0};
    for (int kk = 0; kk < n; kk++) {
      const u64* a = A + (size_t)kk * 2 * LN + w;
      const u64* rr = R + ((size_t)kk * rstride + id) * 2 * LN + w;
      const u64 a0 = a[0], a1 = a[LN], r0 = rr[0], r1 = rr[LN];
      mac128(s0, a0, r0);
      mac128(s1, a0, r1);
      mac128(s1, a1, r0);
      mac128(s2, a1, r1);
      if ((kk & 7) == 7) {
        s0 = Acc128{0, reduce128(s0.hi, s0.lo, md)};
        s1 = Acc128{0, reduce128(s1.hi, s1.lo, md)};
        s2 = Acc128{0, reduce128(s2.hi, s2.lo, md)};
      }
    }
    u64* D = d + (size_t)id * 3 * LN + w;
    D[0] = reduce128(s0.hi, s0.lo, md);
    D[LN] = reduce128(s1.hi, s1.lo, md);
    D[2 * LN] = reduce128(s2.hi, s2.lo, md);
  }
}

// Accumulate of up to kSetBlock independent products in one launch (the product
// pointers travel as a kernel parameter, so a captured graph replays them):
// product t (n_t = off[t+1] - off[t] ciphertexts per operand) gets
// d[(t0 + t) p + i0 + idx] = sum_k tensor(A_t[k], R[off[t] + k][idx]), idx < ci, with R
// [sum n][ci][2][limbs][N] the rotations of the concatenated B operands.
__global__ void k_matmul_acc_multi_kernel(SetPtrs A, const u64* R, u64* d, int T, int t0, int p, int i0, int ci,
                                          int limbs, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t total = (size_t)T * ci * LN;
  HE_GRID_LOOP(idx, total) {
    const size_t w = idx % LN;
    const size_t r = idx / LN;
    const int id = (int)(r % ci), t = (int)(r / ci);
    const int i = (int)(w >> log_n);
    const Mod md = pt[i].mod;
    const size_t k0 = A.off[t];
    const int n = (int)(A.off[t + 1] - k0);
    const u64* Ap = A.p[t];
    Acc128 s0{0, 0}, s1{0, 0}, s2{0, 0};
    for (int kk = 0; kk < n; kk++) {
      const u64* a = Ap + (size_t)kk * 2 * LN + w;
      const u64* rr = R + ((k0 + kk) * ci + id) * 2 * LN + w;
      const u64 a0 = a[0], a1 = a[LN], r0 = rr[0], r1 = rr[LN];
      mac128(s0, a0, r0);
      mac128(s1, a0, r1);
      mac128(s1, a1, r0);
      mac128(s2, a1, r1);
      if ((kk & 7) == 7) {
        s0 = Acc128{0, reduce128(s0.hi, s0.lo, md)};
        s1 = Acc128{0, reduce128(s1.hi, s1.lo, md)};
        s2 = Acc128{0, reduce128(s2.hi, s2.lo, md)};
      }
    }
    u64* D = d + ((size_t)(t0 + t) * p + i0 + id) * 3 * LN + w;
    D[0] = reduce128(s0.hi, s0.lo, md);
    D[LN] = reduce128(s1.hi, s1.lo, md);
    D[2 * LN] = reduce128(s2.hi, s2.lo, md);
  }
}

// Gather (dir 0: base + off[t] <- P.p[t]) or scatter (dir 1: P.p[t] <- base + off[t]) of up to
// kSetBlock device ranges of off[t+1] - off[t] words, blockIdx.y = range.
__global__ void k_move_words_kernel(SetPtrs P, u64* base, int T, int dir) {
  const int t = blockIdx.y;
  if (t >= T) return;
  const size_t n = P.off[t + 1] - P.off[t];
  u64* far = const_cast<u64*>(P.p[t]);
  u64* near = base + P.off[t];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (dir == 0) near[i] = far[i];
    else far[i] = near[i];
  }
}

// Zero-rotation matmul accumulate: d[g] (3 components) = sum_k tensor(Ahat[g][k], B[k]);
// Ahat [G][n][2][limbs][N], B [n][2][limbs][N]. Sums of 128-bit products, reduced
// every 8 terms.
__global__ void k_volley_acc_kernel(const u64* Ah, const u64* B, u64* d, int n, int G, int limbs, const PrimeTab* pt,
                                    int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t total = (size_t)G * LN;
  HE_GRID_LOOP(idx, total) {
    const size_t w = idx % LN;
    const int g = (int)(idx / LN);
    const int i = (int)(w >> log_n);
    const Mod md = pt[i].mod;
    Acc128 s0{0, 0}, s1{0, 0}, s2{0, 0};
    for (int kk = 0; kk < n; kk++) {
      const u64* a = Ah + ((size_t)g * n + kk) * 2 * LN + w;
      const u64* b = B + (size_t)kk * 2 * LN + w;
      const u64 a0 = a[0], a1 = a[LN], b0 = b[0], b1 = b[LN];
      mac128(s0, a0, b0);
      mac128(s1, a0, b1);
      mac128(s1, a1, b0);
      mac128(s2, a1, b1);
      if ((kk & 7) == 7) {
        s0 = Acc128{0, reduce128(s0.hi, s0.lo, md)};
        s1 = Acc128{0, reduce128(s1.hi, s1.lo, md)};
        s2 = Acc128{0, reduce128(s2.hi, s2.lo, md)};
      }
    }
    u64* D = d + (size_t)g * 3 * LN + w;
    D[0] = reduce128(s0.hi, s0.lo, md);
    D[LN] = reduce128(s1.hi, s1.lo, md);
    D[2 * LN] = reduce128(s2.hi, s2.lo, md);
  }
}

// out[o] = sum_cj pt[o][cj] X[cj]; X [n_in][P][limbs][N], pt [out_dim][n_in][limbs][N],
// out [out_dim][P][limbs][N], P = 2 or 3 components (products need not be
// relinearised: the sum is linear in each component). One thread per (limb,
// coefficient) handles every component, so each plaintext word is read once.
// The loads of UN input columns are issued before their products so that
// enough reads are in flight to stream the plaintexts at memory speed; sums
// are reduced every 8 columns.
template <int OB, int UN, int P>
__global__ void __launch_bounds__(128) k_fc_mac_kernel(const u64* X, const u64* ptx, u64* out, int n_in, int pt_cols,
                                                       int out_dim, int limbs, const PrimeTab* pt, int log_n) {
  static_assert(8 % UN == 0, "reduction every 8 columns");
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  HE_GRID_LOOP(w, LN) {
    const int i = (int)(w >> log_n);
    const Mod md = pt[i].mod;
    if (md.q < kMac96Prime) continue;  // k_fc_mac96_kernel's limbs (uniform across the block)
    for (int o0 = 0; o0 < out_dim; o0 += OB) {
      Acc128 acc[P][OB];
#pragma unroll
      for (int c = 0; c < P; c++)
#pragma unroll
        for (int t = 0; t < OB; t++) acc[c][t] = Acc128{0, 0};
      for (int cj0 = 0; cj0 < n_in; cj0 += UN) {
        u64 xv[UN][P], pv[UN][OB];
#pragma unroll
        for (int v = 0; v < UN; v++) {
          const int cj = cj0 + v;
          const bool ok = cj < n_in;
#pragma unroll
          for (int c = 0; c < P; c++) xv[v][c] = ok ? X[((size_t)cj * P + c) * LN + w] : 0;
#pragma unroll
          for (int t = 0; t < OB; t++)
            pv[v][t] = (ok && o0 + t < out_dim) ? ptx[((size_t)(o0 + t) * pt_cols + cj) * LN + w] : 0;
        }
#pragma unroll
        for (int v = 0; v < UN; v++)
#pragma unroll
          for (int t = 0; t < OB; t++)
#pragma unroll
            for (int c = 0; c < P; c++) mac128(acc[c][t], xv[v][c], pv[v][t]);
        if (((cj0 + UN) & 7) == 0) {
#pragma unroll
          for (int c = 0; c < P; c++)
#pragma unroll
            for (int t = 0; t < OB; t++) acc[c][t] = Acc128{0, reduce128(acc[c][t].hi, acc[c][t].lo, md)};
        }
      }
#pragma unroll
      for (int t = 0; t < OB; t++)
        if (o0 + t < out_dim)
#pragma unroll
          for (int c = 0; c < P; c++)
            out[((size_t)(o0 + t) * P + c) * LN + w] = reduce128(acc[c][t].hi, acc[c][t].lo, md);
    }
  }
}

// The dense-layer multiply-accumulate for limbs whose prime is below kMac96Prime:
// 96-bit sums (seven 32-bit multiplies a product), reduced once every `room`
// columns and at the end. Same layout and tiling as k_fc_mac_kernel.
template <int OB, int UN, int P>
__global__ void __launch_bounds__(128) k_fc_mac96_kernel(const u64* X, const u64* ptx, u64* out, int n_in,
                                                         int pt_cols, int out_dim, int limbs, const PrimeTab* pt,
                                                         int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  HE_GRID_LOOP(w, LN) {
    const int i = (int)(w >> log_n);
    const Mod md = pt[i].mod;
    if (md.q >= kMac96Prime) continue;  // k_fc_mac_kernel's limbs (uniform across the block)
    const int room = mac96_room(md.q);
    for (int o0 = 0; o0 < out_dim; o0 += OB) {
      Acc96 acc[P][OB];
#pragma unroll
      for (int c = 0; c < P; c++)
#pragma unroll
        for (int t = 0; t < OB; t++) acc[c][t] = Acc96{0, 0, 0};
      int pending = 0;
      for (int cj0 = 0; cj0 < n_in; cj0 += UN) {
        u64 xv[UN][P], pv[UN][OB];
#pragma unroll
        for (int v = 0; v < UN; v++) {
          const int cj = cj0 + v;
          const bool ok = cj < n_in;
#pragma unroll
          for (int c = 0; c < P; c++) xv[v][c] = ok ? X[((size_t)cj * P + c) * LN + w] : 0;
#pragma unroll
          for (int t = 0; t < OB; t++)
            pv[v][t] = (ok && o0 + t < out_dim) ? ptx[((size_t)(o0 + t) * pt_cols + cj) * LN + w] : 0;
        }
        if (pending + UN > room) {  // uniform across the block
#pragma unroll
          for (int c = 0; c < P; c++)
#pragma unroll
            for (int t = 0; t < OB; t++) {
              const u64 r = reduce96(acc[c][t], md);
              acc[c][t] = Acc96{(u32)r, (u32)(r >> 32), 0};
            }
          pending = 0;
        }
        pending += UN;
#pragma unroll
        for (int v = 0; v < UN; v++)
#pragma unroll
          for (int t = 0; t < OB; t++)
#pragma unroll
            for (int c = 0; c < P; c++) mac96(acc[c][t], xv[v][c], pv[v][t]);
      }
#pragma unroll
      for (int t = 0; t < OB; t++)
        if (o0 + t < out_dim)
#pragma unroll
          for (int c = 0; c < P; c++) out[((size_t)(o0 + t) * P + c) * LN + w] = reduce96(acc[c][t], md);
    }
  }
}

// Slot-block packing of T requests: out[j] = sum_t mask_t * X_t[j] for both
// components of column j, where X_t is request t's ciphertext set ([n][2][LN])
// and mask_t (limbs x N, NTT domain) is the plaintext that keeps block t.
// xs is a device array of the T request pointers; every request word and
// every output word is touched once, the masks stay in L2.
__global__ void k_pack_blocks_kernel(const u64* const* xs, const u64* masks, int T, int n_ct, int limbs,
                                     size_t ct_stride, u64* out, const PrimeTab* pt, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const size_t total = (size_t)n_ct * LN;
  HE_GRID_LOOP(idx, total) {
    const size_t w = idx % LN;
    const size_t j = idx / LN;
    const Mod md = pt[(int)(w >> log_n)].mod;
    Acc128 s0{0, 0}, s1{0, 0};
    for (int t = 0; t < T; t++) {
      const u64* x = xs[t] + j * ct_stride + w;
      const u64 m = masks[(size_t)t * LN + w];
      mac128(s0, x[0], m);
      mac128(s1, x[LN], m);
      if ((t & 7) == 7) {
        s0 = Acc128{0, reduce128(s0.hi, s0.lo, md)};
        s1 = Acc128{0, reduce128(s1.hi, s1.lo, md)};
      }
    }
    u64* o = out + j * 2 * LN + w;
    o[0] = reduce128(s0.hi, s0.lo, md);
    o[LN] = reduce128(s1.hi, s1.lo, md);
  }
}

// Integer-arithmetic calibration: 8 independent chains of Shoup products per
// thread (enough instruction-level parallelism to keep the integer pipes
// busy), `iters` products per chain. The xor of the chains is written so the
// work cannot be removed.
__global__ void k_calib_shoup_kernel(u64* sink, u64 q, u64 w, u64 wp, int iters) {
  u64 a[8];
#pragma unroll
  for (int c = 0; c < 8; c++) a[c] = (blockIdx.x * 131ull + threadIdx.x * 7ull + c) % q;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < 8; c++) a[c] = shoup_lazy(a[c], w, wp, q);
  }
  u64 x = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) x ^= a[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// Calibration of the 96-bit multiply-accumulate: eight independent sums per
// thread, each gaining a product of two residues below kMac96Prime per iteration
// (the sums wrap; only the time is used).
__global__ void k_calib_mac96_kernel(u64* sink, u64 q, int iters) {
  Acc96 acc[8];
  u64 a[8];
#pragma unroll
  for (int c = 0; c < 8; c++) {
    a[c] = (blockIdx.x * 131ull + threadIdx.x * 7ull + c) % q;
    acc[c] = Acc96{0, 0, 0};
  }
  const u64 b = q - 3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < 8; c++) mac96(acc[c], a[c], b);
  }
  u64 x = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) x ^= ((u64)acc[c].w2 << 32) ^ acc[c].w1 ^ acc[c].w0;
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// Calibration of the forward transform's butterfly as the transform kernels run it:
// eight independent (X, Y) pairs per thread, each iteration one butterfly per pair
// on its own output. NAR: the growing-range butterfly of primes below kNarrowPrime
// (the cheaper quotient estimate, no reduction: X + T, X - T + 4q); otherwise
// Harvey's (X reduced below 2q, Shoup's lazy product, X + T, X - T + 2q). The
// values wrap; only the time is used.
template <bool NAR>
__global__ void k_calib_bfly_kernel(u64* sink, u64 q, u64 w, u64 wp, int iters) {
  u64 x[8], y[8];
#pragma unroll
  for (int c = 0; c < 8; c++) {
    x[c] = (blockIdx.x * 131ull + threadIdx.x * 7ull + c) % q;
    y[c] = (blockIdx.x * 17ull + threadIdx.x * 29ull + 3 * c) % q;
  }
  const u64 q2 = 2 * q, q4 = 4 * q;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
      if constexpr (NAR) {
        const u64 T = shoup_approx(y[c], w, wp, q);
        const u64 X = x[c];
        x[c] = X + T;
        y[c] = X - T + q4;
      } else {
        u64 X = x[c];
        if (X >= q2) X -= q2;
        const u64 T = shoup_lazy(y[c], w, wp, q);
        x[c] = X + T;
        y[c] = X - T + q2;
      }
    }
  }
  u64 r = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) r ^= x[c] ^ y[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// counts residues >= q_i in [n][limbs][N] rows (limb i of each polynomial)
__global__ void k_check_range_kernel(const u64* x, size_t rows, int limbs, const PrimeTab* pt, int log_n,
                                     unsigned long long* bad) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = rows * N;
  unsigned long long local = 0;
  HE_GRID_LOOP(idx, total) {
    const int i = (int)((idx >> log_n) % limbs);
    local += x[idx] >= pt[i].mod.q;
  }
  if (local) atomicAdd(bad, local);
}

__global__ void k_copy_rows_kernel(const u64* src, size_t src_gs, u64* dst, size_t dst_gs, size_t groups, int rpg,
                                   int log_n) {
  const size_t N = (size_t)1 << log_n;
  const size_t total = groups * rpg * N;
  HE_GRID_LOOP(idx, total) {
    const size_t jn = idx & (N - 1), r = idx >> log_n;
    const size_t g = r / rpg, rr = r - g * rpg;
    dst[g * dst_gs + rr * N + jn] = src[g * src_gs + rr * N + jn];
  }
}

}  // namespace

#define HE_LAUNCH_P(kern, total, bytes, products, ...)                         \
  do {                                                                         \
    const size_t tot_ = (total);                                               \
    if (tot_) {                                                                \
      void* tok_ = prof_begin(#kern, C.stream, (double)(bytes), (double)(products)); \
      kern<<<grid_for(tot_), kBlock, 0, C.stream>>>(__VA_ARGS__);             \
      prof_end(tok_, C.stream);                                                \
    }                                                                          \
    HE_CUDA(cudaGetLastError());                                               \
  } while (0)
#define HE_LAUNCH(kern, total, bytes, ...) HE_LAUNCH_P(kern, total, bytes, 0.0, __VA_ARGS__)

void k_reduce_signed(const Ctx& C, const int64_t* in, u64* out, int n, const LimbMap& lm) {
  HE_LAUNCH(k_reduce_signed_kernel, (size_t)n * lm.lpp * C.N, 8.0 * (double)C.N * n * (1 + lm.lpp), in, out, n, lm, C.dev_ptab(), C.log_n);
}
void k_reduce_small(const Ctx& C, const int8_t* in, u64* out, int n, const LimbMap& lm) {
  HE_LAUNCH(k_reduce_small_kernel, (size_t)n * lm.lpp * C.N, 8.0 * (double)C.N * n * (0.125 + lm.lpp), in, out, n, lm, C.dev_ptab(), C.log_n);
}
void k_encrypt_combine(const Ctx& C, const u64* v, const u64* e0, const u64* e1, const u64* m, u64* ct, int n,
                       int limbs) {
  HE_LAUNCH(k_encrypt_kernel, (size_t)n * limbs * C.N, 8.0 * (double)C.N * limbs * (6.0 * n + 2), v, e0, e1, m, C.d_pk.p, ct, n, limbs, C.L1, C.dev_ptab(),
            C.log_n);
}
void k_ksk_combine(const Ctx& C, const u64* a, const u64* e, const u64* sprime, u64* b, int digit) {
  HE_LAUNCH(k_ksk_kernel, (size_t)C.np() * C.N, 8.0 * (double)C.N * 5 * C.np(), a, e, C.d_s.p, sprime, b, digit, C.alpha, C.L1, C.np(),
            C.dev_ptab(), C.log_n);
}
void k_mul(const Ctx& C, const u64* a, const u64* b, u64* out, int n_polys, const LimbMap& lm) {
  HE_LAUNCH_P(k_mul_kernel, (size_t)n_polys * lm.lpp * C.N, 8.0 * (double)C.N * 3 * n_polys * lm.lpp,
              (double)C.N * n_polys * lm.lpp, a, b, out, n_polys, lm, C.dev_ptab(), C.log_n);
}
void k_mont_form(const Ctx& C, u64* data, int n_polys, const LimbMap& lm) {
  HE_LAUNCH_P(k_mont_form_kernel, (size_t)n_polys * lm.lpp * C.N, 16.0 * (double)C.N * n_polys * lm.lpp,
              (double)C.N * n_polys * lm.lpp, data, n_polys, lm, C.dev_ptab(), C.log_n);
}
void k_permute(const Ctx& C, const u64* in, u64* out, size_t rows, u64 k) {
  HE_LAUNCH(k_permute_kernel, rows * C.N, 8.0 * (double)C.N * 2 * rows, in, out, rows, k, C.log_n);
}
void k_decrypt_limb0(const Ctx& C, const u64* ct, int limbs, int n, u64* out) {
  HE_LAUNCH(k_decrypt0_kernel, (size_t)n * C.N, 8.0 * (double)C.N * (3.0 * n + 1), ct, C.d_s.p, limbs, n, out, C.dev_ptab(), C.log_n);
}
void k_add(const Ctx& C, const u64* a, const u64* b, u64* out, int n_polys, int limbs) {
  HE_LAUNCH(k_add_kernel, (size_t)n_polys * limbs * C.N, 8.0 * (double)C.N * 3 * n_polys * limbs, a, b, out, n_polys, limbs, C.dev_ptab(), C.log_n);
}
void k_tensor(const Ctx& C, const u64* a, const u64* b, u64* d, int n, int limbs) {
  if (n <= 0) return;
  if (n > 65535) throw Error(1, "more than 65535 ciphertexts in one product launch");
  const size_t LN = (size_t)limbs * C.N;
  // a few words a thread, one grid row per ciphertext
  const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>((LN + kBlock - 1) / kBlock,
                                                                     (152 * 32 + (size_t)n - 1) / (size_t)n * 4));
  const double bytes = 8.0 * (double)C.N * limbs * n * (a == b ? 5.0 : 7.0);
  void* tok = prof_begin("k_tensor_kernel", C.stream, bytes, (a == b ? 3.0 : 4.0) * C.N * n * limbs);
  k_tensor_kernel<<<dim3(gx, (unsigned)n), kBlock, 0, C.stream>>>(a, b, d, n, limbs, C.dev_ptab(), C.log_n);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}
void k_ks_inner(const Ctx& C, const u64* ext, const u64* own, size_t own_stride, const KeyPtrs& keys, int S, u64* u,
                int n, int limbs) {
  const int beta = C.beta_at(limbs);
  if (beta > 16) throw Error(8, "more than 16 key-switching digits are not supported");
  if (S < 1 || S > 8) throw Error(1, "1..8 keys per inner-product launch");
  const size_t per_step = (size_t)beta * KS_TILE * 16;
  // steps per launch so that the staged key tiles fit in 96 KiB of shared memory
  const int sc = (int)std::max<size_t>(1, std::min<size_t>((size_t)S, (96 * 1024) / per_step));
  static bool attr = false;
  if (!attr) {
    HE_CUDA(cudaFuncSetAttribute(k_ks_inner_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
    HE_CUDA(cudaFuncSetAttribute(k_ks_inner_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
    attr = true;
  }
  const int nb = limbs + C.K;
  const size_t ustep = (size_t)n * 2 * nb * C.N;
  for (int s0 = 0; s0 < S; s0 += sc) {
    const int cs = std::min(sc, S - s0);
    KeyPtrs kp{};
    for (int t = 0; t < cs; t++) kp.k[t] = keys.k[s0 + t];
    const dim3 grid((unsigned)((C.N + KS_TILE - 1) / KS_TILE), (unsigned)nb);
    const size_t smem = (size_t)cs * per_step;
    const double bytes = 8.0 * (double)C.N * nb * ((double)beta * (n + 2.0 * cs) + 2.0 * n * cs);
    void* tok = prof_begin(beta <= 8 ? "k_ks_inner_kernel<8>" : "k_ks_inner_kernel<16>", C.stream, bytes,
                           2.0 * C.N * nb * beta * (double)n * cs);
    if (beta <= 8)
      k_ks_inner_kernel<8><<<grid, KS_TILE, smem, C.stream>>>(ext, own, own_stride, C.alpha, kp, cs, u + s0 * ustep,
                                                               n, limbs, beta, C.L1, C.K, C.dev_ptab(), C.log_n);
    else
      k_ks_inner_kernel<16><<<grid, KS_TILE, smem, C.stream>>>(ext, own, own_stride, C.alpha, kp, cs, u + s0 * ustep,
                                                                n, limbs, beta, C.L1, C.K, C.dev_ptab(), C.log_n);
    prof_end(tok, C.stream);
    HE_CUDA(cudaGetLastError());
  }
}
void k_gather_p(const Ctx& C, const u64* u, u64* p, int n, int limbs, u64 k) {
  HE_LAUNCH(k_gather_p_kernel, (size_t)n * 2 * C.K * C.N, 8.0 * (double)C.N * 4 * n * C.K, u, p, n, limbs, C.K, k, C.log_n);
}
void k_rescale_expand(const Ctx& C, const u64* last_coeff, u64* r, int rows, int limbs) {
  const u64* tab = C.d_rs.p + (size_t)limbs * C.L1 * 3;
  HE_LAUNCH(k_rescale_expand_kernel, (size_t)rows * C.N, 8.0 * (double)C.N * rows * (double)limbs, last_coeff, r, rows, limbs, tab, C.dev_ptab(), C.log_n);
}
void k_rescale_combine(const Ctx& C, const u64* x, const u64* r, u64* out, int rows, int limbs) {
  const u64* tab = C.d_rs.p + (size_t)limbs * C.L1 * 3;
  HE_LAUNCH(k_rescale_combine_kernel, (size_t)rows * (limbs - 1) * C.N, 8.0 * (double)C.N * 3.0 * rows * (limbs - 1), x, r, out, rows, limbs, tab, C.dev_ptab(),
            C.log_n);
}
void k_mul_const(const Ctx& C, const u64* in, u64* out, size_t rows, int limbs, const u64* wsh) {
  HE_LAUNCH_P(k_mul_const_kernel, rows * limbs * C.N, 16.0 * (double)C.N * rows * limbs, (double)C.N * rows * limbs,
              in, out, rows, limbs, wsh, C.dev_ptab(), C.log_n);
}
void k_add_comps(const Ctx& C, u64* y, const u64* v, int n, int ypolys, int limbs) {
  HE_LAUNCH(k_add_comps_kernel, (size_t)n * 2 * limbs * C.N, 8.0 * (double)C.N * 6.0 * n * limbs, y, v, n, ypolys,
            limbs, C.dev_ptab(), C.log_n);
}
void k_add_const(const Ctx& C, u64* ct, int n, int limbs, const u64* c_dev, int per_group) {
  HE_LAUNCH(k_add_const_kernel, (size_t)n * limbs * C.N, 8.0 * (double)C.N * 2.0 * n * limbs, ct, n, limbs, c_dev, per_group, C.dev_ptab(), C.log_n);
}
void k_conv_mac(const Ctx& C, const u64* rot, u64* out, const u64* w, int c_in, int w_in, int k, int stride,
                int c_out, int w_out, int limbs, bool colmajor) {
  if (colmajor) {  // the tensor cores, every class of limbs (conv_mac_tc_all held)
    k_conv_mac_tc(C, rot, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, false);
    k_conv_mac_tc(C, rot, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, true);
    return;
  }
  constexpr int TN = 2, TH = 128;
  const size_t smem = (size_t)c_out * c_in * k * k * 16;
  if (smem > 200 * 1024) throw Error(8, "convolution weights exceed shared memory");
  // limbs by kernel: 96-bit sums below kMac96Prime, Shoup products above
  int wide = 0;
  for (int i = 0; i < limbs; i++) wide += C.q[i] >= kMac96Prime;
  int narrow = limbs - wide;
  const double T = (double)c_in * k * k;
  auto per_limb_bytes = [&] {
    return 8.0 * (double)C.N * 2.0 * ((double)c_in * (stride * (w_out - 1) + k) * k + (double)c_out * w_out);
  };
  const double prods_limb = 2.0 * C.N * (double)c_out * w_out * T;
  const unsigned gy = (unsigned)(2 * limbs);
  if (wide > 0) {
    const unsigned gx = (unsigned)((C.N / TN + TH - 1) / TH);
    unsigned gz = (unsigned)std::max<size_t>(1, (size_t)152 * 16 / ((size_t)gx * 2 * wide));
    if (gz > (unsigned)w_out) gz = (unsigned)w_out;
    void* tok = prof_begin(c_out <= 8 ? "k_conv_mac_kernel<8>" : "k_conv_mac_kernel<16>", C.stream,
                           per_limb_bytes() * wide, prods_limb * wide);
    if (c_out <= 8) {
      static bool attr8 = false;
      if (!attr8) {
        HE_CUDA(cudaFuncSetAttribute(k_conv_mac_kernel<8, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr8 = true;
      }
      k_conv_mac_kernel<8, TN><<<dim3(gx, gy, gz), TH, smem, C.stream>>>(rot, out, w, c_in, w_in, k, stride, c_out,
                                                                          w_out, limbs, C.dev_ptab(), C.log_n);
    } else {
      static bool attr16 = false;
      if (!attr16) {
        HE_CUDA(cudaFuncSetAttribute(k_conv_mac_kernel<16, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr16 = true;
      }
      k_conv_mac_kernel<16, TN><<<dim3(gx, gy, gz), TH, smem, C.stream>>>(rot, out, w, c_in, w_in, k, stride, c_out,
                                                                           w_out, limbs, C.dev_ptab(), C.log_n);
    }
    prof_end(tok, C.stream);
    HE_CUDA(cudaGetLastError());
  }
  if (narrow > 0) {
    // 8 output channels x 2 coefficients a thread (48 words of sums); 16 channels take two passes
    // over the rotated inputs, which the idle memory bandwidth absorbs
    constexpr int OB96 = 8, TN96 = 2;
    const size_t smem64 = (size_t)((c_out + 1) & ~1) * c_in * k * k * 8;
    const unsigned gx = (unsigned)((C.N / TN96 + TH - 1) / TH);
    unsigned gz = (unsigned)std::max<size_t>(1, (size_t)152 * 16 / ((size_t)gx * 2 * narrow));
    if (gz > (unsigned)w_out) gz = (unsigned)w_out;
    // algorithmic bytes: every rotated input and output word once (the second pass re-reads inputs)
    void* tok = prof_begin("k_conv_mac96_kernel<8, 2>", C.stream, per_limb_bytes() * narrow, prods_limb * narrow);
    static bool attr96 = false;
    if (!attr96) {
      HE_CUDA(cudaFuncSetAttribute(k_conv_mac96_kernel<OB96, TN96>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
      attr96 = true;
    }
    k_conv_mac96_kernel<OB96, TN96><<<dim3(gx, gy, gz), TH, smem64, C.stream>>>(
        rot, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, C.dev_ptab(), C.log_n);
    prof_end(tok, C.stream);
    HE_CUDA(cudaGetLastError());
  }
}
void k_conv_enc_mac(const Ctx& C, const u64* rot, const u64* W, u64* out, int c_in, int w_in, int k, int stride,
                    int c_out, int w_out, int limbs) {
  constexpr int CO = 2, CJ = 2;
  const size_t LN = (size_t)limbs * C.N;
  const unsigned tiles = (unsigned)(((c_out + CO - 1) / CO) * ((w_out + CJ - 1) / CJ));
  constexpr int TH = 128;  // ~160 registers a thread: small blocks keep three per SM
  const unsigned gx = (unsigned)((LN + TH - 1) / TH);
  const double T = (double)c_in * k * k;
  const double bytes = 8.0 * (double)LN * (2.0 * c_out * T + 2.0 * c_in * (stride * (w_out - 1) + k) * k +
                                           3.0 * c_out * w_out);
  void* tok = prof_begin("k_conv_enc_mac_kernel", C.stream, bytes, 4.0 * (double)LN * c_out * w_out * T);
  k_conv_enc_mac_kernel<CO, CJ><<<dim3(gx, tiles), TH, 0, C.stream>>>(rot, W, out, c_in, w_in, k, stride, c_out,
                                                                          w_out, limbs, C.dev_ptab(), C.log_n);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}
void k_matmul_acc(const Ctx& C, const u64* A, const u64* R, u64* d, int n, int p, int limbs, int rstride) {
  HE_LAUNCH_P(k_matmul_acc_kernel, (size_t)p * limbs * C.N, 8.0 * (double)C.N * limbs * (2.0 * n + 2.0 * n * p + 3.0 * p),
              4.0 * C.N * limbs * n * p, A, R, d, n, p, rstride > 0 ? rstride : p, limbs, C.dev_ptab(), C.log_n);
}
void k_matmul_acc_multi(const Ctx& C, const SetPtrs& A, const u64* R, u64* d, int T, int t0, int p, int i0, int ci,
                        int limbs) {
  const double LN = (double)limbs * C.N, n_total = (double)(A.off[T] - A.off[0]);
  HE_LAUNCH_P(k_matmul_acc_multi_kernel, (size_t)T * ci * limbs * C.N,
              8.0 * LN * (2.0 * n_total + 2.0 * n_total * ci + 3.0 * T * ci), 4.0 * LN * n_total * ci, A, R, d, T, t0,
              p, i0, ci, limbs, C.dev_ptab(), C.log_n);
}
void k_move_words(const Ctx& C, const SetPtrs& P, u64* base, int T, int dir) {
  if (T <= 0) return;
  size_t mx = 0;
  for (int t = 0; t < T; t++) mx = std::max(mx, (size_t)(P.off[t + 1] - P.off[t]));
  const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>(64, (mx + 255) / 256));
  void* tok = prof_begin("k_move_words_kernel", C.stream, 16.0 * (double)(P.off[T] - P.off[0]));
  k_move_words_kernel<<<dim3(gx, (unsigned)T), 256, 0, C.stream>>>(P, base, T, dir);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}
void k_volley_acc(const Ctx& C, const u64* Ah, const u64* B, u64* d, int n, int G, int limbs) {
  HE_LAUNCH_P(k_volley_acc_kernel, (size_t)G * limbs * C.N,
              8.0 * (double)C.N * limbs * (2.0 * n * G + 2.0 * n + 3.0 * G), 4.0 * C.N * limbs * n * G, Ah, B, d, n,
              G, limbs, C.dev_ptab(), C.log_n);
}
void k_fc_mac(const Ctx& C, const u64* X, const u64* pt, u64* out, int n_in, int pt_cols, int out_dim, int limbs,
              int polys) {
  if (polys != 2 && polys != 3) throw Error(1, "dense layer inputs have two or three components");
  const size_t total = (size_t)limbs * C.N;
  // 128-thread blocks: at 126-156 registers a thread, three or four blocks fit an SM
  const unsigned grid_fc = (unsigned)std::min<size_t>((total + 127) / 128, (size_t)152 * 64);
  // limbs by kernel: 96-bit sums below kMac96Prime, 128-bit sums above
  int wide = 0;
  for (int i = 0; i < limbs; i++) wide += C.q[i] >= kMac96Prime;
  const int narrow = limbs - wide;
  const double limb_bytes = 8.0 * (double)C.N * ((double)polys * n_in + (double)out_dim * n_in + (double)polys * out_dim);
  const double limb_prods = (double)C.N * polys * (double)n_in * out_dim;
  if (wide > 0) {
    void* tok = prof_begin("k_fc_mac_kernel", C.stream, limb_bytes * wide, limb_prods * wide);
    if (polys == 2)
      k_fc_mac_kernel<5, 2, 2>
          <<<grid_fc, 128, 0, C.stream>>>(X, pt, out, n_in, pt_cols, out_dim, limbs, C.dev_ptab(), C.log_n);
    else
      k_fc_mac_kernel<5, 2, 3>
          <<<grid_fc, 128, 0, C.stream>>>(X, pt, out, n_in, pt_cols, out_dim, limbs, C.dev_ptab(), C.log_n);
    prof_end(tok, C.stream);
    HE_CUDA(cudaGetLastError());
  }
  if (narrow > 0) {
    void* tok = prof_begin("k_fc_mac96_kernel", C.stream, limb_bytes * narrow, limb_prods * narrow);
    if (polys == 2)
      k_fc_mac96_kernel<5, 2, 2>
          <<<grid_fc, 128, 0, C.stream>>>(X, pt, out, n_in, pt_cols, out_dim, limbs, C.dev_ptab(), C.log_n);
    else
      k_fc_mac96_kernel<5, 2, 3>
          <<<grid_fc, 128, 0, C.stream>>>(X, pt, out, n_in, pt_cols, out_dim, limbs, C.dev_ptab(), C.log_n);
    prof_end(tok, C.stream);
    HE_CUDA(cudaGetLastError());
  }
}
void k_pack_blocks(const Ctx& C, const u64* const* xs, const u64* masks, int T, int n_ct, int limbs, u64* out,
                   size_t ct_stride) {
  HE_LAUNCH_P(k_pack_blocks_kernel, (size_t)n_ct * limbs * C.N,
              8.0 * (double)C.N * limbs * (2.0 * n_ct * T + (double)T + 2.0 * n_ct), 2.0 * C.N * limbs * n_ct * T,
              xs, masks, T, n_ct, limbs, ct_stride ? ct_stride : (size_t)2 * limbs * C.N, out, C.dev_ptab(), C.log_n);
}
void k_calib_shoup(const Ctx& C, u64* sink, int blocks, int threads, int iters) {
  const u64 q = C.q[0], w = (q / 3) | 1, wp = (u64)(((unsigned __int128)w << 64) / q);
  void* tok = prof_begin("k_calib_shoup_kernel", C.stream, 0.0, 8.0 * blocks * threads * (double)iters);
  k_calib_shoup_kernel<<<blocks, threads, 0, C.stream>>>(sink, q, w, wp, iters);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}
void k_calib_mac96(const Ctx& C, u64* sink, int blocks, int threads, int iters) {
  u64 q = (1ull << 45) - 55;
  for (int i = 0; i < C.L1; i++)
    if (C.q[i] < kMac96Prime) {
      q = C.q[i];
      break;
    }
  void* tok = prof_begin("k_calib_mac96_kernel", C.stream, 0.0, 8.0 * blocks * threads * (double)iters);
  k_calib_mac96_kernel<<<blocks, threads, 0, C.stream>>>(sink, q, iters);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}
void k_calib_bfly(const Ctx& C, u64* sink, int blocks, int threads, int iters, bool narrow) {
  // a prime of the requested class from the context's chain (Q then P), else a stand-in of that size
  u64 q = narrow ? (1ull << 45) - 55 : (1ull << 60) - 93;
  for (u64 c : C.q)
    if ((c < kNarrowPrime) == narrow) {
      q = c;
      break;
    }
  const u64 w = (q / 3) | 1, wp = (u64)(((unsigned __int128)w << 64) / q);
  void* tok = prof_begin(narrow ? "k_calib_bfly_kernel<narrow>" : "k_calib_bfly_kernel<wide>", C.stream, 0.0,
                         8.0 * blocks * threads * (double)iters);
  if (narrow)
    k_calib_bfly_kernel<true><<<blocks, threads, 0, C.stream>>>(sink, q, w, wp, iters);
  else
    k_calib_bfly_kernel<false><<<blocks, threads, 0, C.stream>>>(sink, q, w, wp, iters);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}
void k_check_range(const Ctx& C, const u64* x, size_t rows, int limbs, unsigned long long* bad) {
  HE_LAUNCH(k_check_range_kernel, rows * C.N, 8.0 * (double)C.N * rows, x, rows, limbs, C.dev_ptab(), C.log_n, bad);
}
void k_copy_limbs(const Ctx& C, const u64* src, size_t src_gs, u64* dst, size_t dst_gs, size_t groups,
                  int rows_per_group) {
  HE_LAUNCH(k_copy_rows_kernel, groups * rows_per_group * C.N, 8.0 * (double)C.N * 2.0 * groups * rows_per_group, src, src_gs, dst, dst_gs, groups, rows_per_group,
            C.log_n);
}

}  // namespace he
