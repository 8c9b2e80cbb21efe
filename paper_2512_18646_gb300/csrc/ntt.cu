// ntt.cu - batched negacyclic NTT / inverse NTT over 64-bit prime limbs.
//
// Transform (forward): A[j] = sum_i a_i psi^((2 brv(j) + 1) i) mod q, psi a
// primitive 2N-th root; the evaluations of a(X) at the odd powers of psi in
// bit-reversed order, so that a negacyclic product is a pointwise product.
// Forward: Cooley-Tukey butterflies with psi merged into the twiddles
// (psi^{brv(m + i)} at stage m, group i); inverse: Gentleman-Sande with
// psi^{-brv(m + i)} and a final multiply by N^{-1}. Arithmetic: Shoup twiddle
// products and Harvey's lazy ranges ([0, 4q) forward, [0, 2q) inverse).
//
// GPU decomposition, N = 2^n = 2^{n1} x 2^{n2}: write j = hi 2^{n2} + lo.
// The first n1 forward stages pair indices that differ only in `hi`, so for a
// fixed `lo` they form an independent 2^{n1}-point problem: kernel A loads a
// tile of C adjacent `lo` columns (2^{n1} x C words, coalesced rows of C words)
// into shared memory and runs those stages there. The last n2 stages pair
// indices inside one run of 2^{n2} consecutive words: kernel B loads whole
// runs. The inverse runs the same kernels in the opposite order. Each launch
// covers every limb of a batch (grid.y = limb rows), so one launch transforms
// all limbs of many polynomials.
#include "he_internal.h"

namespace he {

namespace {

constexpr int kThreads = 256;
constexpr int kTileWords = 4096;  // 32 KiB of shared memory per block

struct NttGeom {
  int n, n1, n2, C, R;  // C columns per kernel-A tile, R runs per kernel-B tile
};

NttGeom geom(int log_n) {
  NttGeom g;
  g.n = log_n;
  g.n1 = log_n / 2;
  g.n2 = log_n - g.n1;
  const int S2 = 1 << g.n2, R1 = 1 << g.n1;
  g.C = S2 < 16 ? S2 : 16;
  int r = kTileWords / S2;
  if (r < 1) r = 1;
  if (r > R1) r = R1;
  g.R = r;
  return g;
}

__device__ __forceinline__ u64* row_ptr(u64* base, const LimbMap& lm, int row, size_t N, int& prime) {
  const int p = row / lm.lpp, i = row % lm.lpp;
  prime = lm.prime(i);
  return base + (size_t)p * lm.poly_stride + (size_t)i * N;
}

// Forward, first n1 stages (large butterfly distances), columns lo0 .. lo0+C-1.
__global__ void __launch_bounds__(kThreads) k_ntt_fwd_cols(u64* data, LimbMap lm, const PrimeTab* pt,
                                                           const u64* psi_all, int n, int n1, int C) {
  extern __shared__ u64 sm[];
  const size_t N = (size_t)1 << n;
  const int n2 = n - n1, R1 = 1 << n1;
  const size_t stride = (size_t)1 << n2;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const u64 q = pt[prime].mod.q, q2 = 2 * q;
  const u64* W = psi_all + (size_t)prime * 2 * N;
  const u64* Wp = W + N;
  const int lo0 = blockIdx.x * C;
  for (int e = threadIdx.x; e < R1 * C; e += blockDim.x) {
    const int hi = e / C, c = e - hi * C;
    sm[e] = x[hi * stride + lo0 + c];
  }
  __syncthreads();
  for (int s = 0; s < n1; s++) {
    const int m = 1 << s, th = R1 >> (s + 1);
    for (int bf = threadIdx.x; bf < (R1 / 2) * C; bf += blockDim.x) {
      const int k = bf / C, c = bf - k * C;
      const int grp = k / th, pos = k - grp * th;
      const int hi = grp * 2 * th + pos;
      const u64 w = W[m + grp], wp = Wp[m + grp];
      u64 X = sm[hi * C + c];
      const u64 Y = sm[(hi + th) * C + c];
      if (X >= q2) X -= q2;
      const u64 T = shoup_lazy(Y, w, wp, q);
      sm[hi * C + c] = X + T;
      sm[(hi + th) * C + c] = X - T + q2;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < R1 * C; e += blockDim.x) {
    const int hi = e / C, c = e - hi * C;
    x[hi * stride + lo0 + c] = sm[e];
  }
}

// Forward, last n2 stages (distances < 2^{n2}), runs seg0 .. seg0+R-1; output in [0, q).
__global__ void __launch_bounds__(kThreads) k_ntt_fwd_rows(u64* data, LimbMap lm, const PrimeTab* pt,
                                                           const u64* psi_all, int n, int n1, int R) {
  extern __shared__ u64 sm[];
  const size_t N = (size_t)1 << n;
  const int n2 = n - n1, S2 = 1 << n2;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const u64 q = pt[prime].mod.q, q2 = 2 * q;
  const u64* W = psi_all + (size_t)prime * 2 * N;
  const u64* Wp = W + N;
  const size_t base = (size_t)blockIdx.x * R * S2;
  for (int e = threadIdx.x; e < R * S2; e += blockDim.x) sm[e] = x[base + e];
  __syncthreads();
  for (int s = n1; s < n; s++) {
    const int m = 1 << s, t = (int)(N >> (s + 1));
    for (int bf = threadIdx.x; bf < R * (S2 / 2); bf += blockDim.x) {
      const int seg = bf / (S2 / 2), k = bf - seg * (S2 / 2);
      const int g = k / t, pos = k - g * t;
      const int l = seg * S2 + g * 2 * t + pos;
      const size_t i = (base + (size_t)l) / (2 * (size_t)t);
      const u64 w = W[m + i], wp = Wp[m + i];
      u64 X = sm[l];
      const u64 Y = sm[l + t];
      if (X >= q2) X -= q2;
      const u64 T = shoup_lazy(Y, w, wp, q);
      sm[l] = X + T;
      sm[l + t] = X - T + q2;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < R * S2; e += blockDim.x) x[base + e] = reduce4q(sm[e], q);
}

// Inverse, first n2 stages (distances 1 .. 2^{n2-1}) inside runs; output in [0, 2q).
__global__ void __launch_bounds__(kThreads) k_ntt_inv_rows(u64* data, LimbMap lm, const PrimeTab* pt,
                                                           const u64* ipsi_all, int n, int n1, int R) {
  extern __shared__ u64 sm[];
  const size_t N = (size_t)1 << n;
  const int n2 = n - n1, S2 = 1 << n2;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const u64 q = pt[prime].mod.q, q2 = 2 * q;
  const u64* W = ipsi_all + (size_t)prime * 2 * N;
  const u64* Wp = W + N;
  const size_t base = (size_t)blockIdx.x * R * S2;
  for (int e = threadIdx.x; e < R * S2; e += blockDim.x) sm[e] = x[base + e];
  __syncthreads();
  for (int t = 1; t < S2; t <<= 1) {
    const size_t m = N / (2 * (size_t)t);
    for (int bf = threadIdx.x; bf < R * (S2 / 2); bf += blockDim.x) {
      const int seg = bf / (S2 / 2), k = bf - seg * (S2 / 2);
      const int g = k / t, pos = k - g * t;
      const int l = seg * S2 + g * 2 * t + pos;
      const size_t i = (base + (size_t)l) / (2 * (size_t)t);
      const u64 w = W[m + i], wp = Wp[m + i];
      const u64 X = sm[l], Y = sm[l + t];
      u64 S = X + Y;
      if (S >= q2) S -= q2;
      sm[l] = S;
      sm[l + t] = shoup_lazy(X - Y + q2, w, wp, q);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < R * S2; e += blockDim.x) x[base + e] = sm[e];
}

// Inverse, last n1 stages (distances >= 2^{n2}) on columns, then times N^{-1}; output in [0, q).
__global__ void __launch_bounds__(kThreads) k_ntt_inv_cols(u64* data, LimbMap lm, const PrimeTab* pt,
                                                           const u64* ipsi_all, int n, int n1, int C) {
  extern __shared__ u64 sm[];
  const size_t N = (size_t)1 << n;
  const int n2 = n - n1, R1 = 1 << n1;
  const size_t stride = (size_t)1 << n2;
  int prime;
  u64* x = row_ptr(data, lm, blockIdx.y, N, prime);
  const PrimeTab P = pt[prime];
  const u64 q = P.mod.q, q2 = 2 * q;
  const u64* W = ipsi_all + (size_t)prime * 2 * N;
  const u64* Wp = W + N;
  const int lo0 = blockIdx.x * C;
  for (int e = threadIdx.x; e < R1 * C; e += blockDim.x) {
    const int hi = e / C, c = e - hi * C;
    sm[e] = x[hi * stride + lo0 + c];
  }
  __syncthreads();
  for (int th = 1; th < R1; th <<= 1) {
    const int m = R1 / (2 * th);
    for (int bf = threadIdx.x; bf < (R1 / 2) * C; bf += blockDim.x) {
      const int k = bf / C, c = bf - k * C;
      const int grp = k / th, pos = k - grp * th;
      const int hi = grp * 2 * th + pos;
      const u64 w = W[m + grp], wp = Wp[m + grp];
      const u64 X = sm[hi * C + c], Y = sm[(hi + th) * C + c];
      u64 S = X + Y;
      if (S >= q2) S -= q2;
      sm[hi * C + c] = S;
      sm[(hi + th) * C + c] = shoup_lazy(X - Y + q2, w, wp, q);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < R1 * C; e += blockDim.x) {
    const int hi = e / C, c = e - hi * C;
    x[hi * stride + lo0 + c] = shoup(sm[e], P.ninv, P.ninv_sh, q);
  }
}

}  // namespace

void ntt_forward(const Ctx& C, u64* data, int n_polys, const LimbMap& lm) {
  const int rows = n_polys * lm.lpp;
  if (rows == 0) return;
  const NttGeom g = geom(C.log_n);
  const int S2 = 1 << g.n2, R1 = 1 << g.n1;
  // grid.y holds at most 65535 rows; chunks end on polynomial boundaries
  const int step = (65535 / lm.lpp) * lm.lpp;
  for (int r0 = 0; r0 < rows; r0 += step) {
    const int rr = rows - r0 < step ? rows - r0 : step;
    u64* base = data + (size_t)(r0 / lm.lpp) * lm.poly_stride;
    void* t = prof_begin("k_ntt_fwd_cols", C.stream, 16.0 * rr * (double)C.N);
    k_ntt_fwd_cols<<<dim3(S2 / g.C, rr), kThreads, (size_t)R1 * g.C * 8, C.stream>>>(
        base, lm, C.dev_ptab(), C.d_psi.p, g.n, g.n1, g.C);
    prof_end(t, C.stream);
    t = prof_begin("k_ntt_fwd_rows", C.stream, 16.0 * rr * (double)C.N);
    k_ntt_fwd_rows<<<dim3(R1 / g.R, rr), kThreads, (size_t)g.R * S2 * 8, C.stream>>>(
        base, lm, C.dev_ptab(), C.d_psi.p, g.n, g.n1, g.R);
    prof_end(t, C.stream);
  }
  HE_CUDA(cudaGetLastError());
}

void ntt_inverse(const Ctx& C, u64* data, int n_polys, const LimbMap& lm) {
  const int rows = n_polys * lm.lpp;
  if (rows == 0) return;
  const NttGeom g = geom(C.log_n);
  const int S2 = 1 << g.n2, R1 = 1 << g.n1;
  const int step = (65535 / lm.lpp) * lm.lpp;
  for (int r0 = 0; r0 < rows; r0 += step) {
    const int rr = rows - r0 < step ? rows - r0 : step;
    u64* base = data + (size_t)(r0 / lm.lpp) * lm.poly_stride;
    void* t = prof_begin("k_ntt_inv_rows", C.stream, 16.0 * rr * (double)C.N);
    k_ntt_inv_rows<<<dim3(R1 / g.R, rr), kThreads, (size_t)g.R * S2 * 8, C.stream>>>(
        base, lm, C.dev_ptab(), C.d_ipsi.p, g.n, g.n1, g.R);
    prof_end(t, C.stream);
    t = prof_begin("k_ntt_inv_cols", C.stream, 16.0 * rr * (double)C.N);
    k_ntt_inv_cols<<<dim3(S2 / g.C, rr), kThreads, (size_t)R1 * g.C * 8, C.stream>>>(
        base, lm, C.dev_ptab(), C.d_ipsi.p, g.n, g.n1, g.C);
    prof_end(t, C.stream);
  }
  HE_CUDA(cudaGetLastError());
}

}  // namespace he
