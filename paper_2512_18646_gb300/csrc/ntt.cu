// ntt.cu - batched negacyclic NTT / inverse NTT over 64-bit prime limbs.
//
// Transform (forward): A[j] = sum_i a_i psi^((2 brv(j) + 1) i) mod q, psi a
// primitive 2N-th root; the evaluations of a(X) at the odd powers of psi in
// bit-reversed order, so that a negacyclic product is a pointwise product.
// Forward: Cooley-Tukey butterflies with psi merged into the twiddles
// (stage with m groups, group i: psi^{brv(m + i)}); inverse: Gentleman-Sande
// with psi^{-brv(m + i)}, then a multiply by N^{-1}. Arithmetic: Shoup twiddle
// products and Harvey's lazy ranges ([0, 4q) forward, [0, 2q) inverse).
//
// Decomposition, N = 2^n = 2^{n1} x 2^{n2}, index j = hi 2^{n2} + lo: the first
// n1 forward stages change only `hi` (independent 2^{n1}-point transforms per
// column `lo`), the last n2 only `lo` (2^{n2}-point transforms per run of
// consecutive words). Kernel "cols" takes a tile of C adjacent columns, kernel
// "rows" whole runs; the inverse runs them in the opposite order. grid.y is
// the limb (row of N words), so one launch covers every limb of a batch.
//
// Inside a sub-transform of M = 2^m points each thread holds 2^b elements in
// registers (b = 4 in the column kernels, 3 in the row kernels) and runs up to
// b butterfly stages per round before exchanging through shared memory. In
// round r (stages b r .. b r + b - 1, from the largest distance down) element
// k of thread u is the index with k's bits at the round's distance bit
// positions (plus, in a short last round, the top positions not in the round)
// and u's bits in the remaining positions in order. All index arithmetic is
// compile-time shifts and masks. The column kernels address shared memory by
// element index times the column count plus the column, so the threads of a
// half-warp (adjacent columns) touch adjacent words; the row kernel keeps each
// sub-transform inside one warp and swizzles its shared memory, word x at
// x ^ g(x >> 4) for a GF(2)-linear g, which makes every round's 64-bit
// accesses conflict-free for all M <= 256.
#include "he_internal.h"

namespace he {

namespace {

// Operands of work fused into a transform's load (cols kernel) or store (rows
// kernel), by MODE:
//  1 rescale:  x [rows][lp][N] holds the polynomials being rescaled, limb lp - 1
//              already in the coefficient domain; rs [L1][3] holds floor(q_l/2)
//              mod q_i, q_l^{-1} mod q_i and its Shoup companion for this lp.
//              addc (optional): a constant added after the rescale to polynomial
//              add_row0 + p (of the whole set), limb i: addc[(add_row0 + p) (lp - 1) + i].
//  2 ModDown:  load: yt [polys][K][N] the P part times N^{-1} (P/p_k)^{-1}
//              (coefficient domain), phat [K][L1][2] (P/p_k) mod q_i with Shoup
//              companions; store: out[c][comp][i][j] = (u[c][comp][i][pi(j)] - z)
//              P^{-1} + (mode 0: base[c][comp][i][j]; mode 1, comp 0:
//              base[c][0][i][pi(j)]), pi the Galois index of element gk.
//  3 scaled inverse: the inverse transform ends with the factor iscale[prime -
//              scale_base] (w, Shoup companion) instead of N^{-1}.
//  (inverse rows, any mode) src: when set, polynomial p's limb i is read from
//              src + p src_stride + lm.mem(i) N and the result written to the
//              rows of `data` (an out-of-place first pass).
//  4 ModUp:    load: the target limb at extended position e = lm.mem(i) of digit
//              polynomial pr is sum_{t < K} yt[pr ystride + t N] hat[t hstride + e],
//              yt the digit's source limbs times N^{-1} (D_j/q_i)^{-1} (coefficient
//              domain), hat (D_j/q_i) mod target prime with Shoup companions.
struct Fuse {
  const u64* x = nullptr;
  const u64* rs = nullptr;
  int lp = 0;
  const u64* yt = nullptr;
  const u64* phat = nullptr;
  int K = 0, L1 = 0, nb = 0, kmode = 0;
  const u64* u = nullptr;
  const u64* base = nullptr;
  size_t base_stride = 0, out_stride = 0;
  u64* out = nullptr;
  u64 gk = 1;
  const u64* pinv = nullptr;
  const u64* iscale = nullptr;
  int scale_base = 0;
  size_t ystride = 0;
  int hstride = 0;
  const u64* src = nullptr;
  size_t src_stride = 0;
  const u64* addc = nullptr;
  int add_row0 = 0;
};

// ---------------------------------------------------------------------------
// compile-time round maps
// ---------------------------------------------------------------------------
// Each thread holds 2^KBM elements of a sub-transform and runs up to KBM
// butterfly stages per round between exchanges: KBM = 4 in the column kernels,
// 3 in the row kernels (whose 64-register budget keeps four blocks per SM).
template <int LOGM, int RND, int KBM>
struct RMap {
  static constexpr int KB = LOGM < KBM ? LOGM : KBM;  // k bits (elements per thread = 2^KB)
  static constexpr int E = 1 << KB;
  static constexpr int S0 = KBM * RND;
  static constexpr int NS = (LOGM - S0) < KBM ? (LOGM - S0) : KBM;  // stages in this round
  static constexpr int LO = LOGM - S0 - NS;                         // lowest distance bit of the round
  // bit position of k bit i
  __host__ __device__ static constexpr int kpos(int i) {
    if (i < NS) return LO + i;
    int c = i - NS;
    for (int p = LOGM - 1; p >= 0; p--) {
      if (p >= LO && p < LO + NS) continue;
      if (c == 0) return p;
      c--;
    }
    return 0;
  }
  // i-th smallest k position
  __host__ __device__ static constexpr int sorted_kpos(int i) {
    int v[KBM] = {};
    for (int a = 0; a < KBM; a++) v[a] = a < KB ? kpos(a) : 99;
    for (int a = 0; a < KBM; a++)
      for (int b = a + 1; b < KBM; b++)
        if (v[b] < v[a]) { const int t = v[a]; v[a] = v[b]; v[b] = t; }
    return v[i];
  }
  // u with zero bits inserted at the k positions
  __device__ static __forceinline__ int upart(int u) {
    int x = u;
#pragma unroll
    for (int i = 0; i < KB; i++) {
      const int p = sorted_kpos(i);
      x = ((x >> p) << (p + 1)) | (x & ((1 << p) - 1));
    }
    return x;
  }
  __host__ __device__ static constexpr int kbits(int k) {
    int x = 0;
    for (int i = 0; i < KB; i++) x |= ((k >> i) & 1) << kpos(i);
    return x;
  }
};

template <int LOGM, int KBM>
struct Plan {
  static constexpr int KB = LOGM < KBM ? LOGM : KBM;
  static constexpr int E = 1 << KB;
  static constexpr int T = (1 << LOGM) / E;         // threads per sub-transform
  static constexpr int R = (LOGM + KBM - 1) / KBM;  // rounds
};
constexpr int kColKB = 4, kRowKB = 3;

// bit reversal of the low `bits` bits, for compile-time arguments
__host__ __device__ constexpr u32 brv_const(u32 x, int bits) {
  u32 r = 0;
  for (int b = 0; b < bits; b++) r |= ((x >> b) & 1u) << (bits - 1 - b);
  return r;
}

__device__ __forceinline__ ulonglong2 tw_load(const u64* tw, u64 idx) {
  return __ldg(reinterpret_cast<const ulonglong2*>(tw) + idx);
}

// One forward round: stages S0 .. S0+NS-1 of an M-point sub-transform.
// Twiddle of the butterfly whose lower element is e at local stage s:
//   table[(1 << (soff + s)) + (run << s) + (e >> (LOGM - s))].
// NAR (primes below kNarrowPrime): no reduction of the upper input and the
// cheaper quotient estimate, so each stage raises the bound on the values by
// at most 4q; otherwise Harvey's butterfly keeps them in [0, 4q).
template <int LOGM, int RND, int KBM, bool NAR>
__device__ __forceinline__ void round_fwd(u64 (&a)[Plan<LOGM, KBM>::E], int xu, const u64* tw, int soff, u64 run,
                                          u64 q) {
  using M = RMap<LOGM, RND, KBM>;
  const u64 q2 = 2 * q, q4 = 4 * q;
#pragma unroll
  for (int st = 0; st < M::NS; st++) {
    const int s = M::S0 + st;
    const int ib = M::NS - 1 - st;  // k bit of this stage's distance
    const u64 base = ((u64)1 << (soff + s)) + (run << s);
#pragma unroll
    for (int hi = 0; hi < (M::E >> (ib + 1)); hi++) {
      const int kb = hi << (ib + 1);
      const int e = xu | M::kbits(kb);
      const ulonglong2 w = tw_load(tw, base + (u64)(e >> (LOGM - s)));
#pragma unroll
      for (int lo = 0; lo < (1 << ib); lo++) {
        const int k = kb | lo, k2 = k | (1 << ib);
        u64 X = a[k];
        if constexpr (NAR) {
          const u64 T = shoup_approx(a[k2], w.x, w.y, q);
          a[k] = X + T;
          a[k2] = X - T + q4;
        } else {
          if (X >= q2) X -= q2;
          const u64 T = shoup_lazy(a[k2], w.x, w.y, q);
          a[k] = X + T;
          a[k2] = X - T + q2;
        }
      }
    }
  }
}

// One inverse round (Gentleman-Sande), stages in the opposite order. NAR: the
// sums are not reduced; the inputs of the stage executed t-th (t = LOGM - 1 - s)
// are below 2^(t+1) q, which the difference adds before its product.
template <int LOGM, int RND, int KBM, bool NAR>
__device__ __forceinline__ void round_inv(u64 (&a)[Plan<LOGM, KBM>::E], int xu, const u64* tw, int soff, u64 run,
                                          u64 q) {
  using M = RMap<LOGM, RND, KBM>;
  const u64 q2 = 2 * q;
#pragma unroll
  for (int st = M::NS - 1; st >= 0; st--) {
    const int s = M::S0 + st;
    const int ib = M::NS - 1 - st;
    const u64 base = ((u64)1 << (soff + s)) + (run << s);
    const u64 bt = q << (LOGM - s);
#pragma unroll
    for (int hi = 0; hi < (M::E >> (ib + 1)); hi++) {
      const int kb = hi << (ib + 1);
      const int e = xu | M::kbits(kb);
      const ulonglong2 w = tw_load(tw, base + (u64)(e >> (LOGM - s)));
#pragma unroll
      for (int lo = 0; lo < (1 << ib); lo++) {
        const int k = kb | lo, k2 = k | (1 << ib);
        const u64 X = a[k], Y = a[k2];
        if constexpr (NAR) {
          a[k] = X + Y;
          a[k2] = shoup_approx(X - Y + bt, w.x, w.y, q);
        } else {
          u64 S = X + Y;
          if (S >= q2) S -= q2;
          a[k] = S;
          a[k2] = shoup_lazy(X - Y + q2, w.x, w.y, q);
        }
      }
    }
  }
}

// Rounds RND .. R-1 (forward) with exchanges through shared memory; `addr`
// maps an element index to its shared-memory word.
template <int LOGM, int RND, int KBM, bool NAR, class Sync, class Addr>
__device__ __forceinline__ void rounds_fwd_rest(u64 (&a)[Plan<LOGM, KBM>::E], int u, u64* sm, Addr addr, Sync sync,
                                                const u64* tw, int soff, u64 run, u64 q) {
  if constexpr (RND < Plan<LOGM, KBM>::R) {
    using Mp = RMap<LOGM, RND - 1, KBM>;
    using Mc = RMap<LOGM, RND, KBM>;
    const int xp = Mp::upart(u);
#pragma unroll
    for (int k = 0; k < Plan<LOGM, KBM>::E; k++) sm[addr(xp | Mp::kbits(k))] = a[k];
    sync();
    const int xc = Mc::upart(u);
#pragma unroll
    for (int k = 0; k < Plan<LOGM, KBM>::E; k++) a[k] = sm[addr(xc | Mc::kbits(k))];
    sync();
    round_fwd<LOGM, RND, KBM, NAR>(a, xc, tw, soff, run, q);
    rounds_fwd_rest<LOGM, RND + 1, KBM, NAR>(a, u, sm, addr, sync, tw, soff, run, q);
  }
}

template <int LOGM, int RND, int KBM, bool NAR, class Sync, class Addr>
__device__ __forceinline__ void rounds_inv_rest(u64 (&a)[Plan<LOGM, KBM>::E], int u, u64* sm, Addr addr, Sync sync,
                                                const u64* tw, int soff, u64 run, u64 q) {
  if constexpr (RND >= 0) {
    using Mp = RMap<LOGM, RND + 1, KBM>;
    using Mc = RMap<LOGM, RND, KBM>;
    const int xp = Mp::upart(u);
#pragma unroll
    for (int k = 0; k < Plan<LOGM, KBM>::E; k++) sm[addr(xp | Mp::kbits(k))] = a[k];
    sync();
    const int xc = Mc::upart(u);
#pragma unroll
    for (int k = 0; k < Plan<LOGM, KBM>::E; k++) a[k] = sm[addr(xc | Mc::kbits(k))];
    sync();
    round_inv<LOGM, RND, KBM, NAR>(a, xc, tw, soff, run, q);
    rounds_inv_rest<LOGM, RND - 1, KBM, NAR>(a, u, sm, addr, sync, tw, soff, run, q);
  }
}

__device__ __forceinline__ int swz(int x) {
  // x ^ g(x >> 4), g GF(2)-linear with columns (3, 5, 10, 0) on bits 4..7
  const int y = x >> 4;
  const int g = ((y & 1) ? 3 : 0) ^ ((y & 2) ? 5 : 0) ^ ((y & 4) ? 10 : 0);
  return x ^ g;
}

__device__ __forceinline__ u64* row_ptr(u64* base, const LimbMap& lm, int row, size_t N, int& prime) {
  const int p = row / lm.lpp, i = row - p * lm.lpp;
  prime = lm.prime(i);
  return base + (size_t)p * lm.poly_stride + (size_t)lm.mem(i) * N;
}

constexpr int kRowThreads = 256;

// ---------------------------------------------------------------------------
// rows: last n2 forward stages (sub-size M = 2^LOGM = 2^{n2}), warp-contained
// ---------------------------------------------------------------------------
// Inputs below 4q (wide primes) or below 40q (narrow primes: the column
// kernel's growing range); outputs in [0, q).
template <int LOGM, int MODE, bool NAR>
__device__ __forceinline__ void fwd_rows_body(u64* xr, u64* smw, int rw, int u, const u64* tw, int n, int n1, u64 run,
                                              u64 q, float frd, int frd_sh, const LimbMap& lm, const Fuse& fz) {
  using P = Plan<LOGM, kRowKB>;
  constexpr int M = 1 << LOGM;
  const size_t N = (size_t)1 << n;
  auto addr = [rw](int e) { return swz(rw * M + e); };
  auto sync = [] { __syncwarp(__activemask()); };
  // the transform's result reduced to [0, q) (growing range: the cheaper quotient estimate
  // leaves [0, 4q), as the lazy butterflies do)
  // (growing range: values below 72 q, reduced by an fp32 quotient estimate; Harvey: [0, 4q))
  auto fin = [q, frd, frd_sh](u64 v) { return NAR ? reduce_fp32(v, q, frd, frd_sh) : reduce4q(v, q); };
  // exact products of the fused epilogues, by way of [0, 4q)
  auto mulq = [q](u64 v, u64 w, u64 wp) { return reduce4q(shoup_approx(v, w, wp, q), q); };
  // a multiple of q above every transform output (72q growing range, 4q Harvey), so that
  // x + zq - a is a nonnegative representative of x - a for the fused epilogues, whose exact
  // Shoup product then reduces it
  const u64 zq = (NAR ? 72 : 4) * q;
  u64 a[P::E];
  {
    using M0 = RMap<LOGM, 0, kRowKB>;
    const int x0 = M0::upart(u);
#pragma unroll
    for (int k = 0; k < P::E; k++) a[k] = xr[x0 | M0::kbits(k)];
    round_fwd<LOGM, 0, kRowKB, NAR>(a, x0, tw, n1, run, q);
  }
  rounds_fwd_rest<LOGM, 1, kRowKB, NAR>(a, u, smw, addr, sync, tw, n1, run, q);
  using ML = RMap<LOGM, P::R - 1, kRowKB>;
  const int xl = ML::upart(u);
  if constexpr (MODE == 0) {
#pragma unroll
    for (int k = 0; k < P::E; k++) xr[xl | ML::kbits(k)] = fin(a[k]);
  } else if constexpr (MODE == 1) {
    // rescale: out_i = (x_i - R_i) q_l^{-1} mod q_i, R_i this transform of the expanded last limb
    const int pr = blockIdx.y / lm.lpp, i = blockIdx.y - pr * lm.lpp;
    const u64* xi = fz.x + ((size_t)pr * fz.lp + i) * N + run * M;
    const u64 qi = fz.rs[(size_t)i * 3 + 1], qs = fz.rs[(size_t)i * 3 + 2];
    const u64 cadd = fz.addc ? fz.addc[(size_t)(fz.add_row0 + pr) * lm.lpp + i] : 0;
    if (cadd == 0) {
#pragma unroll
      for (int k = 0; k < P::E; k++) {
        const int e = xl | ML::kbits(k);
        xr[e] = mulq(xi[e] + zq - a[k], qi, qs);
      }
    } else {
#pragma unroll
      for (int k = 0; k < P::E; k++) {
        const int e = xl | ML::kbits(k);
        xr[e] = addmod(mulq(xi[e] + zq - a[k], qi, qs), cadd, q);
      }
    }
  } else {
    // ModDown combine: (u_Q[pi(j)] - z) P^{-1} plus the part the key switch does not touch
    const int pr = blockIdx.y / lm.lpp, i = blockIdx.y - pr * lm.lpp;
    const int comp = pr & 1;
    const size_t c = (size_t)(pr >> 1);
    const size_t LN = (size_t)lm.lpp * N;
    const u64* ui = fz.u + ((size_t)pr * fz.nb + i) * N;
    const u64* bi = fz.base + c * fz.base_stride + (fz.kmode == 0 ? (size_t)comp * LN : 0) + (size_t)i * N;
    u64* oi = fz.out + c * fz.out_stride + (size_t)comp * LN + (size_t)i * N;
    const u64 pv = fz.pinv[2 * i], ps = fz.pinv[2 * i + 1];
    const bool add = fz.kmode == 0 || comp == 0;
    // Galois index of j = run M + e: brv_n(j) = brv_L(e) 2^(n-L) + brv_(n-L)(run), and brv_L(e) is
    // brv_L(xl) | brv_L(kbits(k)) (disjoint bits), so only a constant is or-ed per element
    const u32 hb = (brv_bits((u32)xl, LOGM) << (n - LOGM)) | (n > LOGM ? brv_bits((u32)run, n - LOGM) : 0u);
    const u32 mask = (2u << n) - 1, gk = (u32)fz.gk;
    // (2 (hb | c) + 1) gk = (2 hb + 1) gk + 2 c gk (disjoint bits): one product per thread, and per
    // element the constant 2 c gk, c = brv(kbits(k)) 2^(n-L), as a sum of the products for its bits
    const u32 e0 = (2 * hb + 1) * gk;
    u32 gbit[P::KB];
#pragma unroll
    for (int b = 0; b < P::KB; b++) gbit[b] = (2 * gk * brv_const(ML::kbits(1 << b), LOGM)) << (n - LOGM);
#pragma unroll
    for (int k = 0; k < P::E; k++) {
      const u32 j = (u32)(run * M) + (u32)(xl | ML::kbits(k));
      u32 src = j;
      if (gk != 1) {
        u32 e2 = e0;
#pragma unroll
        for (int b = 0; b < P::KB; b++)
          if ((k >> b) & 1) e2 += gbit[b];
        // brv_n((e2 - 1) / 2) = brev32(e2 - 1) >> (31 - n): e2 is odd, so bit 0 of e2 - 1 is clear
        src = __brev((e2 & mask) - 1) >> (31 - n);
      }
      const u64 v = mulq(ui[src] + zq - a[k], pv, ps);
      oi[j] = add ? addmod(v, bi[fz.kmode == 0 ? j : src], q) : v;
    }
  }
}

template <int LOGM, int MODE>
__global__ void __launch_bounds__(kRowThreads, 4) k_ntt_fwd_rows(u64* data, LimbMap lm, const PrimeTab* pt,
                                                              const u64* tw_all, int n, int n1, Fuse fz) {
  using P = Plan<LOGM, kRowKB>;
  constexpr int M = 1 << LOGM;
  constexpr int RUNS = kRowThreads / P::T;
  __shared__ u64 sm[kRowThreads * P::E];
  const size_t N = (size_t)1 << n;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const u64 q = pt[prime].mod.q;
  const float frd = pt[prime].frd;
  const int frd_sh = pt[prime].frd_sh;
  const u64* tw = tw_all + (size_t)prime * 2 * N;
  const int r_cta = threadIdx.x / P::T, u = threadIdx.x - r_cta * P::T;
  const u64 run = (u64)blockIdx.x * RUNS + r_cta;
  if (run >= ((u64)1 << n1)) return;  // whole runs only, so a warp's active lanes hold whole runs
  u64* xr = x + run * M;
  // shared memory of this thread's warp, runs of the warp side by side
  const int warp = threadIdx.x >> 5;
  const int rw = (threadIdx.x & 31) / P::T;  // run index inside the warp
  u64* smw = sm + warp * 32 * P::E;
  if (q < kNarrowPrime)
    fwd_rows_body<LOGM, MODE, true>(xr, smw, rw, u, tw, n, n1, run, q, frd, frd_sh, lm, fz);
  else
    fwd_rows_body<LOGM, MODE, false>(xr, smw, rw, u, tw, n, n1, run, q, frd, frd_sh, lm, fz);
}

// inverse, first n2 stages (smallest distances) inside runs; inputs below 2q,
// outputs in [0, 2q)
template <int LOGM, bool NAR>
__device__ __forceinline__ void inv_rows_body(const u64* xs, u64* xr, u64* smw, int rw, int u, const u64* tw, int n1,
                                              u64 run, u64 q, float frd, int frd_sh) {
  using P = Plan<LOGM, kRowKB>;
  constexpr int M = 1 << LOGM;
  auto addr = [rw](int e) { return swz(rw * M + e); };
  auto sync = [] { __syncwarp(__activemask()); };
  u64 a[P::E];
  {
    using ML = RMap<LOGM, P::R - 1, kRowKB>;
    const int xl = ML::upart(u);
#pragma unroll
    for (int k = 0; k < P::E; k++) a[k] = xs[xl | ML::kbits(k)];
    round_inv<LOGM, P::R - 1, kRowKB, NAR>(a, xl, tw, n1, run, q);
  }
  rounds_inv_rest<LOGM, P::R - 2, kRowKB, NAR>(a, u, smw, addr, sync, tw, n1, run, q);
  using M0 = RMap<LOGM, 0, kRowKB>;
  const int x0 = M0::upart(u);
#pragma unroll
  // growing range: below 2^9 q after these stages, reduced to [0, q) (within the next kernel's [0, 2q) inputs)
  for (int k = 0; k < P::E; k++) xr[x0 | M0::kbits(k)] = NAR ? reduce_fp32(a[k], q, frd, frd_sh) : a[k];
}

template <int LOGM>
__global__ void __launch_bounds__(kRowThreads, 4) k_ntt_inv_rows(u64* data, LimbMap lm, const PrimeTab* pt,
                                                              const u64* tw_all, int n, int n1, Fuse fz) {
  using P = Plan<LOGM, kRowKB>;
  constexpr int M = 1 << LOGM;
  constexpr int RUNS = kRowThreads / P::T;
  __shared__ u64 sm[kRowThreads * P::E];
  const size_t N = (size_t)1 << n;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const u64 q = pt[prime].mod.q;
  const float frd = pt[prime].frd;
  const int frd_sh = pt[prime].frd_sh;
  const u64* tw = tw_all + (size_t)prime * 2 * N;
  const int r_cta = threadIdx.x / P::T, u = threadIdx.x - r_cta * P::T;
  const u64 run = (u64)blockIdx.x * RUNS + r_cta;
  if (run >= ((u64)1 << n1)) return;
  u64* xr = x + run * M;
  const u64* xs = xr;
  if (fz.src) {
    const int p = blockIdx.y / lm.lpp, i = blockIdx.y - p * lm.lpp;
    xs = fz.src + (size_t)p * fz.src_stride + (size_t)lm.mem(i) * N + run * M;
  }
  const int warp = threadIdx.x >> 5;
  const int rw = (threadIdx.x & 31) / P::T;
  u64* smw = sm + warp * 32 * P::E;
  if (q < kNarrowPrime)
    inv_rows_body<LOGM, true>(xs, xr, smw, rw, u, tw, n1, run, q, frd, frd_sh);
  else
    inv_rows_body<LOGM, false>(xs, xr, smw, rw, u, tw, n1, run, q, frd, frd_sh);
}

// ---------------------------------------------------------------------------
// cols: first n1 forward stages (sub-size 2^LOGM = 2^{n1}) on C adjacent columns
// ---------------------------------------------------------------------------
// Inputs below 4q (8q from a fused two-term base conversion of a narrow prime);
// outputs below 4q (wide primes) or 40q (narrow primes).
template <int LOGM, int MODE, bool NAR>
__device__ __forceinline__ void fwd_cols_body(u64* xc, u64* smc, int u, int C, int lo, const u64* tw, int n, u64 q,
                                              const LimbMap& lm, const PrimeTab* pt, const Fuse& fz) {
  using P = Plan<LOGM, kColKB>;
  const size_t N = (size_t)1 << n;
  const size_t stride = N >> LOGM;
  auto addr = [C, lo](int e) { return e * C + lo; };
  auto sync = [] { __syncthreads(); };
  // fused base conversions: two lazy products per element (below 4q, or 8q with the cheaper
  // estimate of narrow primes), else a running sum kept below 2q
  auto prod = [q](u64 y, ulonglong2 h) { return NAR ? shoup_approx(y, h.x, h.y, q) : shoup_lazy(y, h.x, h.y, q); };
  u64 a[P::E];
  {
    using M0 = RMap<LOGM, 0, kColKB>;
    const int x0 = M0::upart(u);
    if constexpr (MODE == 0) {
#pragma unroll
      for (int k = 0; k < P::E; k++) a[k] = xc[(size_t)(x0 | M0::kbits(k)) * stride];
    } else if constexpr (MODE == 4 || MODE == 2) {
      // ModUp: fast base conversion of the digit, sum_t yt_t (D_j/q_t) mod the target prime;
      // ModDown: of the P part, sum_k yt_k (P/p_k) mod q_i
      const int pr = blockIdx.y / lm.lpp, i = blockIdx.y - pr * lm.lpp;
      const u64* y = MODE == 4 ? fz.yt + (size_t)pr * fz.ystride + (size_t)blockIdx.x * C + lo
                               : fz.yt + (size_t)pr * fz.K * N + (size_t)blockIdx.x * C + lo;
      const ulonglong2* ph = reinterpret_cast<const ulonglong2*>(fz.phat) + (MODE == 4 ? lm.mem(i) : i);
      const size_t hs = MODE == 4 ? (size_t)fz.hstride : (size_t)fz.L1;
      if (fz.K == 2) {
        const ulonglong2 h0 = __ldg(ph), h1 = __ldg(ph + hs);
        u64 y0[P::E], y1[P::E];
#pragma unroll
        for (int k = 0; k < P::E; k++) {
          y0[k] = y[(size_t)(x0 | M0::kbits(k)) * stride];
          y1[k] = y[N + (size_t)(x0 | M0::kbits(k)) * stride];
        }
#pragma unroll
        for (int k = 0; k < P::E; k++) a[k] = prod(y0[k], h0) + prod(y1[k], h1);
      } else {
        const u64 q2 = 2 * q;
#pragma unroll
        for (int k = 0; k < P::E; k++) a[k] = 0;
        for (int t = 0; t < fz.K; t++) {
          const ulonglong2 h = __ldg(ph + (size_t)t * hs);
          const u64* yk = y + (size_t)t * N;
#pragma unroll
          for (int k = 0; k < P::E; k++) {
            u64 v = a[k] + shoup_lazy(yk[(size_t)(x0 | M0::kbits(k)) * stride], h.x, h.y, q);
            a[k] = v >= q2 ? v - q2 : v;
          }
        }
      }
    } else {
      // rescale: the last limb's coefficients r (mod q_l), as (r + floor(q_l/2) mod q_l) - floor(q_l/2) mod q_i
      const int pr = blockIdx.y / lm.lpp, i = blockIdx.y - pr * lm.lpp;
      const u64* src = fz.x + ((size_t)pr * fz.lp + fz.lp - 1) * N + (size_t)blockIdx.x * C + lo;
      const u64 ql = pt[fz.lp - 1].mod.q, one_sh = pt[i].one_sh;
      const u64 half = ql >> 1, q_m_half = q - fz.rs[(size_t)i * 3];
#pragma unroll
      for (int k = 0; k < P::E; k++) {
        const u64 v = addmod(src[(size_t)(x0 | M0::kbits(k)) * stride], half, ql);
        a[k] = shoup_lazy(v, 1, one_sh, q) + q_m_half;  // [0, 3q), within the transform's [0, 4q) inputs
      }
    }
    round_fwd<LOGM, 0, kColKB, NAR>(a, x0, tw, 0, 0, q);
  }
  rounds_fwd_rest<LOGM, 1, kColKB, NAR>(a, u, smc, addr, sync, tw, 0, 0, q);
  using ML = RMap<LOGM, P::R - 1, kColKB>;
  const int xl = ML::upart(u);
#pragma unroll
  for (int k = 0; k < P::E; k++) xc[(size_t)(xl | ML::kbits(k)) * stride] = a[k];
}

template <int LOGM, int MODE>
__global__ void k_ntt_fwd_cols(u64* data, LimbMap lm, const PrimeTab* pt, const u64* tw_all, int n, int C,
                               Fuse fz) {
  extern __shared__ u64 smc[];
  const size_t N = (size_t)1 << n;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const u64 q = pt[prime].mod.q;
  const u64* tw = tw_all + (size_t)prime * 2 * N;
  const int u = threadIdx.x / C, lo = threadIdx.x - u * C;
  u64* xc = x + (size_t)blockIdx.x * C + lo;
  if (q < kNarrowPrime)
    fwd_cols_body<LOGM, MODE, true>(xc, smc, u, C, lo, tw, n, q, lm, pt, fz);
  else
    fwd_cols_body<LOGM, MODE, false>(xc, smc, u, C, lo, tw, n, q, lm, pt, fz);
}

// inverse, last n1 stages (largest distances) on columns, then times N^{-1};
// inputs below 2q, output in [0, q)
template <int LOGM, int MODE, bool NAR>
__device__ __forceinline__ void inv_cols_body(u64* xc, u64* smc, int u, int C, int lo, const u64* tw, int n, u64 q,
                                              u64 sc, u64 scs) {
  using P = Plan<LOGM, kColKB>;
  const size_t N = (size_t)1 << n;
  const size_t stride = N >> LOGM;
  auto addr = [C, lo](int e) { return e * C + lo; };
  auto sync = [] { __syncthreads(); };
  u64 a[P::E];
  {
    using ML = RMap<LOGM, P::R - 1, kColKB>;
    const int xl = ML::upart(u);
#pragma unroll
    for (int k = 0; k < P::E; k++) a[k] = xc[(size_t)(xl | ML::kbits(k)) * stride];
    round_inv<LOGM, P::R - 1, kColKB, NAR>(a, xl, tw, 0, 0, q);
  }
  rounds_inv_rest<LOGM, P::R - 2, kColKB, NAR>(a, u, smc, addr, sync, tw, 0, 0, q);
  using M0 = RMap<LOGM, 0, kColKB>;
  const int x0 = M0::upart(u);
#pragma unroll
  for (int k = 0; k < P::E; k++) xc[(size_t)(x0 | M0::kbits(k)) * stride] = reduce4q(shoup_approx(a[k], sc, scs, q), q);
}

template <int LOGM, int MODE>
__global__ void k_ntt_inv_cols(u64* data, LimbMap lm, const PrimeTab* pt, const u64* tw_all, int n, int C,
                               Fuse fz) {
  extern __shared__ u64 smc[];
  const size_t N = (size_t)1 << n;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const PrimeTab PT = pt[prime];
  const u64 q = PT.mod.q;
  const u64* tw = tw_all + (size_t)prime * 2 * N;
  const int u = threadIdx.x / C, lo = threadIdx.x - u * C;
  u64* xc = x + (size_t)blockIdx.x * C + lo;
  u64 sc = PT.ninv, scs = PT.ninv_sh;
  if constexpr (MODE == 3) {
    sc = fz.iscale[2 * (prime - fz.scale_base)];
    scs = fz.iscale[2 * (prime - fz.scale_base) + 1];
  }
  if (q < kNarrowPrime)
    inv_cols_body<LOGM, MODE, true>(xc, smc, u, C, lo, tw, n, q, sc, scs);
  else
    inv_cols_body<LOGM, MODE, false>(xc, smc, u, C, lo, tw, n, q, sc, scs);
}

struct Geom {
  int n1, n2, C;
};
// The transform's geometry: column stages n1 (the rest, n2, in the row kernels) and the
// columns C of a column block; the context's tuned choice (he_ntt_autotune /
// he_ntt_set_geometry) or the default n1 = log_n / 2, C = min(16, 2^n2).
Geom geom(const Ctx& Cx) {
  Geom g;
  g.n1 = Cx.ntt_n1 > 0 ? Cx.ntt_n1 : Cx.log_n / 2;
  g.n2 = Cx.log_n - g.n1;
  const int S2 = 1 << g.n2;
  g.C = Cx.ntt_cols > 0 ? Cx.ntt_cols : (S2 < 16 ? S2 : 16);
  return g;
}

template <int L, int MODE>
void launch_rows(bool inv, u64* base, const LimbMap& lm, int rows, const Ctx& C, int n1, const u64* tw,
                 const Fuse& fz) {
  constexpr int RUNS = kRowThreads / Plan<L, kRowKB>::T;
  const int runs = 1 << n1;
  const dim3 grid((runs + RUNS - 1) / RUNS, rows);
  // a fused rescale also reads the limbs being rescaled and multiplies by q_l^{-1}
  const bool fused = !inv && (MODE == 1 || MODE == 2);
  const double bytes = (fused ? (MODE == 2 ? 32.0 : 24.0) : 16.0) * rows * (double)C.N;
  // products: the butterflies, plus one Shoup product per element that ends the transform: the
  // fused epilogue's, or else (growing-range path, primes below kNarrowPrime) the reduction of the
  // result to [0, q) (forward) or [0, 2q) (inverse)
  int narrow = 0;
  for (int i = 0; i < lm.lpp; i++) narrow += C.q[lm.prime(i)] < kNarrowPrime;
  const double last = fused ? 1.0 : (double)narrow / lm.lpp;
  const double prods = (double)rows * C.N * ((C.log_n - n1) / 2.0 + last);
  const char* name = inv ? "k_ntt_inv_rows"
                         : MODE == 1 ? "k_ntt_fwd_rows<rescale>" : MODE == 2 ? "k_ntt_fwd_rows<moddown>" : "k_ntt_fwd_rows";
  static_assert(MODE >= 0 && MODE <= 4, "transform modes 0..4");
  void* t = prof_begin(name, C.stream, bytes, prods);
  if (inv) k_ntt_inv_rows<L><<<grid, kRowThreads, 0, C.stream>>>(base, lm, C.dev_ptab(), tw, C.log_n, n1, fz);
  else
    k_ntt_fwd_rows<L, (MODE == 1 || MODE == 2) ? MODE : 0><<<grid, kRowThreads, 0, C.stream>>>(
        base, lm, C.dev_ptab(), tw, C.log_n, n1, fz);
  prof_end(t, C.stream);
}

template <int L, int MODE>
void launch_cols(bool inv, u64* base, const LimbMap& lm, int rows, const Ctx& C, int n2, int Ccols, const u64* tw,
                 const Fuse& fz) {
  const int threads = Ccols * Plan<L, kColKB>::T;
  const size_t smem = (size_t)(1 << L) * Ccols * 8;
  if (smem > 48 * 1024) {  // a wide column tile (autotuner candidate) needs the opt-in shared memory
    static bool attr = false;
    if (!attr) {
      HE_CUDA(cudaFuncSetAttribute(k_ntt_fwd_cols<L, MODE == 3 ? 0 : MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   128 * 1024));
      HE_CUDA(cudaFuncSetAttribute(k_ntt_inv_cols<L, MODE == 3 ? 3 : 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   128 * 1024));
      attr = true;
    }
  }
  const dim3 grid((1 << n2) / Ccols, rows);
  // butterflies, plus N^{-1} (inverse) or the reduction of the expanded limb (fused rescale)
  const double prods = (double)rows * C.N *
                       ((C.log_n - n2) / 2.0 + (inv || MODE == 1 ? 1.0 : MODE == 2 ? 2.0 : MODE == 4 ? 2.0 : 0.0));
  const char* name = inv ? "k_ntt_inv_cols"
                         : MODE == 1   ? "k_ntt_fwd_cols<rescale>"
                         : MODE == 2   ? "k_ntt_fwd_cols<moddown>"
                         : MODE == 4   ? "k_ntt_fwd_cols<modup>"
                                       : "k_ntt_fwd_cols";
  // bytes: every row read and written once; a fused base conversion (ModUp, ModDown) or rescale
  // instead reads its fz.K (resp. one) source limbs per polynomial and writes the rows
  const double src_limbs = MODE == 4 || MODE == 2 ? (double)fz.K : MODE == 1 ? 1.0 : 0.0;
  const double bytes = (!inv && src_limbs > 0) ? 8.0 * (double)C.N * (rows + src_limbs * rows / lm.lpp)
                                               : 16.0 * rows * (double)C.N;
  void* t = prof_begin(name, C.stream, bytes, prods);
  if (inv)
    k_ntt_inv_cols<L, MODE == 3 ? 3 : 0><<<grid, threads, smem, C.stream>>>(base, lm, C.dev_ptab(), tw, C.log_n,
                                                                           Ccols, fz);
  else
    k_ntt_fwd_cols<L, MODE == 3 ? 0 : MODE><<<grid, threads, smem, C.stream>>>(base, lm, C.dev_ptab(), tw, C.log_n,
                                                                              Ccols, fz);
  prof_end(t, C.stream);
}

template <int MODE>
void rows_dispatch(bool inv, u64* base, const LimbMap& lm, int rows, const Ctx& C, const Geom& g, const u64* tw,
                   const Fuse& fz = Fuse{}) {
  switch (g.n2) {
    case 2: launch_rows<2, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    case 3: launch_rows<3, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    case 4: launch_rows<4, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    case 5: launch_rows<5, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    case 6: launch_rows<6, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    case 7: launch_rows<7, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    case 8: launch_rows<8, MODE>(inv, base, lm, rows, C, g.n1, tw, fz); break;
    default: throw Error(1, "unsupported ring degree");
  }
}

template <int MODE>
void cols_dispatch(bool inv, u64* base, const LimbMap& lm, int rows, const Ctx& C, const Geom& g, const u64* tw,
                   const Fuse& fz = Fuse{}) {
  switch (g.n1) {
    case 2: launch_cols<2, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    case 3: launch_cols<3, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    case 4: launch_cols<4, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    case 5: launch_cols<5, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    case 6: launch_cols<6, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    case 7: launch_cols<7, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    case 8: launch_cols<8, MODE>(inv, base, lm, rows, C, g.n2, g.C, tw, fz); break;
    default: throw Error(1, "unsupported ring degree");
  }
}

}  // namespace

void ntt_forward(const Ctx& C, u64* data, int n_polys, const LimbMap& lm) {
  const int rows = n_polys * lm.lpp;
  if (rows == 0) return;
  const Geom g = geom(C);
  // grid.y holds at most 65535 rows; chunks end on polynomial boundaries
  const int step = (65535 / lm.lpp) * lm.lpp;
  for (int r0 = 0; r0 < rows; r0 += step) {
    const int rr = rows - r0 < step ? rows - r0 : step;
    u64* base = data + (size_t)(r0 / lm.lpp) * lm.poly_stride;
    cols_dispatch<0>(false, base, lm, rr, C, g, C.d_psi.p);
    rows_dispatch<0>(false, base, lm, rr, C, g, C.d_psi.p);
  }
  HE_CUDA(cudaGetLastError());
}

void ntt_inverse(const Ctx& C, u64* data, int n_polys, const LimbMap& lm) {
  const int rows = n_polys * lm.lpp;
  if (rows == 0) return;
  const Geom g = geom(C);
  const int step = (65535 / lm.lpp) * lm.lpp;
  for (int r0 = 0; r0 < rows; r0 += step) {
    const int rr = rows - r0 < step ? rows - r0 : step;
    u64* base = data + (size_t)(r0 / lm.lpp) * lm.poly_stride;
    rows_dispatch<0>(true, base, lm, rr, C, g, C.d_ipsi.p);
    cols_dispatch<0>(true, base, lm, rr, C, g, C.d_ipsi.p);
  }
  HE_CUDA(cudaGetLastError());
}

void ntt_inverse_qscaled(const Ctx& C, u64* data, int n_polys, int lp, const u64* src, size_t src_stride) {
  const int rows = n_polys * lp;
  if (rows == 0) return;
  const Geom g = geom(C);
  const LimbMap lm = limbs_q(lp, C.N);
  Fuse fz;
  fz.iscale = C.d_up.p + (size_t)(C.L1 + 1) * C.L1 * 2 + (size_t)(C.L1 + 1) * C.L1 * (C.L1 + C.K) * 2 +
              (size_t)lp * C.L1 * 2;
  fz.scale_base = 0;
  const int step = (65535 / lp) * lp;
  for (int r0 = 0; r0 < rows; r0 += step) {
    const int rr = rows - r0 < step ? rows - r0 : step;
    u64* base = data + (size_t)(r0 / lp) * lm.poly_stride;
    Fuse fr = fz;
    if (src) {
      fr.src = src + (size_t)(r0 / lp) * src_stride;
      fr.src_stride = src_stride;
    }
    rows_dispatch<3>(true, base, lm, rr, C, g, C.d_ipsi.p, fr);
    cols_dispatch<3>(true, base, lm, rr, C, g, C.d_ipsi.p, fz);
  }
  HE_CUDA(cudaGetLastError());
}

void ntt_forward_modup(const Ctx& C, u64* ext_digit, int n, const LimbMap& lm, const u64* yt, size_t ystride,
                       const u64* hat, int hstride, int cnt) {
  const int rows = n * lm.lpp;
  if (rows == 0) return;
  const Geom g = geom(C);
  const int per = 65535 / lm.lpp;  // polynomials per launch (grid.y <= 65535)
  for (int p0 = 0; p0 < n; p0 += per) {
    const int pn = n - p0 < per ? n - p0 : per;
    Fuse fz;
    fz.yt = yt + (size_t)p0 * ystride;
    fz.ystride = ystride;
    fz.phat = hat;
    fz.hstride = hstride;
    fz.K = cnt;
    u64* base = ext_digit + (size_t)p0 * lm.poly_stride;
    cols_dispatch<4>(false, base, lm, pn * lm.lpp, C, g, C.d_psi.p, fz);
    rows_dispatch<4>(false, base, lm, pn * lm.lpp, C, g, C.d_psi.p, fz);
  }
  HE_CUDA(cudaGetLastError());
}

void ntt_inverse_pscaled(const Ctx& C, u64* data, int n_polys) {
  const int lpp = C.K;
  const int rows = n_polys * lpp;
  if (rows == 0) return;
  const Geom g = geom(C);
  LimbMap lm;
  lm.lpp = C.K; lm.split = 0; lm.base0 = 0; lm.base1 = C.L1; lm.poly_stride = (size_t)C.K * C.N;
  Fuse fz;
  fz.iscale = C.d_down.p + 2 * C.K + (size_t)2 * C.K * C.L1 + (size_t)2 * C.L1;
  fz.scale_base = C.L1;
  const int step = (65535 / lpp) * lpp;
  for (int r0 = 0; r0 < rows; r0 += step) {
    const int rr = rows - r0 < step ? rows - r0 : step;
    u64* base = data + (size_t)(r0 / lpp) * lm.poly_stride;
    rows_dispatch<3>(true, base, lm, rr, C, g, C.d_ipsi.p, fz);
    cols_dispatch<3>(true, base, lm, rr, C, g, C.d_ipsi.p, fz);
  }
  HE_CUDA(cudaGetLastError());
}

void ntt_forward_moddown(const Ctx& C, u64* z, const u64* yt, int n, int lp, const u64* u, int nb, const u64* base,
                         size_t base_stride, u64* out, size_t out_stride, u64 gk, int kmode) {
  if (n == 0) return;
  const Geom g = geom(C);
  const LimbMap lm = limbs_q(lp, C.N);
  const int per = 65535 / (2 * lp) * 2;  // polynomials per launch: whole ciphertexts, grid.y <= 65535
  for (int p0 = 0; p0 < 2 * n; p0 += per) {
    const int pn = 2 * n - p0 < per ? 2 * n - p0 : per;
    Fuse fz;
    fz.yt = yt + (size_t)p0 * C.K * C.N;
    fz.phat = C.d_down.p + 2 * C.K;
    fz.K = C.K;
    fz.L1 = C.L1;
    fz.u = u + (size_t)p0 * nb * C.N;
    fz.nb = nb;
    fz.base = base + (size_t)(p0 / 2) * base_stride;
    fz.base_stride = base_stride;
    fz.out = out + (size_t)(p0 / 2) * out_stride;
    fz.out_stride = out_stride;
    fz.gk = gk;
    fz.kmode = kmode;
    fz.pinv = C.d_down.p + 2 * C.K + (size_t)2 * C.K * C.L1;
    u64* zb = z + (size_t)p0 * lp * C.N;
    cols_dispatch<2>(false, zb, lm, pn * lp, C, g, C.d_psi.p, fz);
    rows_dispatch<2>(false, zb, lm, pn * lp, C, g, C.d_psi.p, fz);
  }
  HE_CUDA(cudaGetLastError());
}

bool ntt_geometry_ok(int log_n, int n1, int cols) {
  const int n2 = log_n - n1;
  if (n1 < 2 || n1 > 8 || n2 < 2 || n2 > 8) return false;
  if (cols < 1 || cols > 32 || (cols & (cols - 1)) || cols > (1 << n2)) return false;
  const int kb = n1 < kColKB ? n1 : kColKB;
  const int threads = cols * ((1 << n1) >> kb);
  return threads >= 32 && threads <= 1024 && (size_t)(1 << n1) * cols * 8 <= 128 * 1024;
}

void ntt_forward_rescale(const Ctx& C, u64* out, u64* x, int rows, int lp, const u64* addc, int row0) {
  if (rows == 0) return;
  const Geom g = geom(C);
  const LimbMap lm = limbs_q(lp - 1, C.N);
  const u64* tab = C.d_rs.p + (size_t)lp * C.L1 * 3;
  const int per = 65535 / (lp - 1);  // polynomials per launch (grid.y <= 65535)
  for (int p0 = 0; p0 < rows; p0 += per) {
    const int pn = rows - p0 < per ? rows - p0 : per;
    Fuse fz{x + (size_t)p0 * lp * C.N, tab, lp};
    fz.addc = addc;
    fz.add_row0 = row0 + p0;
    u64* base = out + (size_t)p0 * (lp - 1) * C.N;
    cols_dispatch<1>(false, base, lm, pn * (lp - 1), C, g, C.d_psi.p, fz);
    rows_dispatch<1>(false, base, lm, pn * (lp - 1), C, g, C.d_psi.p, fz);
  }
  HE_CUDA(cudaGetLastError());
}

}  // namespace he
