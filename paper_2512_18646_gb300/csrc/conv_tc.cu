// conv_tc.cu - the convolution's multiply-accumulate on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory).
//
// The ciphertext-scalar multiply-accumulate of a convolution layer (Alg. 4 in
// the column layout: output (o, j') = sum over (c, b, a) of the weight
// K[o][c][a][b] times Rot(X_{c, s j' + b}, g a)) is, for one limb and one
// component, a matrix product: out[o][n] = sum_t W[o][t] X_t[n] mod q, with
// the c_out channels, T = c_in k^2 terms and the N coefficients of the limb as
// its dimensions. Residues are cut into chunks that fp16 holds exactly and the
// tensor cores sum the chunk products in fp32, which is exact while every sum
// stays below 2^24:
//  - primes below 2^46: NC = 6 bytes; the input chunks are taken signed,
//    x = sum_i (b_i - 128) 256^i + K0 with K0 = 128 (256^6 - 1) / 255, the
//    weight chunks unsigned, so |D_s| <= 6 T 128 255 < 2^24 for T <= 85;
//  - primes below 2^62: NC = 9 chunks of 7 bits, both unsigned,
//    D_s <= 9 T 127^2 < 2^24 for T <= 115;
//   D_s[n][o] = sum_{i + j = s} sum_t x_i[t][n] w_j[o][t], s = 0 .. 2 NC - 2
// (the host takes this path only for such T). Then on the CUDA cores
//   out[o][n] = sum_s D_s[n][o] r^s (+ K0 sum_t W[o][t] for bytes) mod q
// (r = 256 or 128; two 64-bit sums of 32 x 32-bit products, one Barrett
// reduction). The result is the exact residue, the same word the CUDA-core
// kernels compute.
//
// One CTA owns a tile of 128 coefficients of one (component, limb) and runs every output column
// j' of the layer over it, 16 terms (one K step) at a time: the input words of a step arrive by one
// tiled TMA box in a ring of stages; converting warps write their chunks as NC fp16 tiles
// [128 x 16] (K-major, 8 x 16-byte core matrices, no swizzle); one thread issues NC MMAs of
// M = 128, N = NC * OBP, K = 16: MMA i multiplies chunk tile i by the weight tile
// B = [chunk j][channel o] and accumulates at tensor-memory column i * OBP, so that column
// s * OBP + o collects D_s[.][o]; recombining warps, two per lane quarter of the accumulator, turn
// the finished sums of a task into residues while the next task's MMAs run. The roles hand work
// over through mbarriers (see the kernel). Every wait is bounded: past the limit the CTA records
// the failure in the context's status word (read by the host at its next synchronisation), frees
// its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "he_internal.h"

namespace he {

namespace {

constexpr int kTcConvWarps = 8;  // warps converting chunks
constexpr int kTcRecWarps = 8;   // warps recombining the accumulators (a multiple of 4: whole lane quarters)
// + warp 0 (MMA issue) and warp 1 (TMA loads)
constexpr int kTcThreads = 32 * (2 + kTcConvWarps + kTcRecWarps);
constexpr int kZeroBytes = 256 * 16 * 2;  // an all-zero fp16 tile of up to 256 rows x 16 (K-major)
constexpr size_t kTcSmemMax = 227 * 1024;  // dynamic shared memory a CTA may opt in to
constexpr int kTcRows = 128;                         // MMA M: coefficients of one tile
constexpr int kStageBytes = 16 * kTcRows * 8;        // one K step: 16 terms x 128 words
constexpr int kAccCols = 256;                        // tensor-memory columns of one accumulator buffer

template <int NC, int OBP>
struct TcShape {
  static constexpr int NS = 2 * NC - 1;                      // sums s = i + j
  static constexpr int NMMA = (NC * OBP + 15) / 16 * 16;     // MMA N (rows of the weight tile)
  static constexpr int COLS = (NC - 1) * OBP + NMMA;         // accumulator columns the MMAs touch
  static constexpr int ZCOLS = (COLS + 15) / 16 * 16;         // columns the clearing MMA writes
  static constexpr int A_TILE = kTcRows * 16 * 2;            // bytes of a [128 x 16] fp16 tile
  static constexpr int B_TILE = NMMA * 16 * 2;               // bytes of an [NMMA x 16] fp16 tile
  static_assert(ZCOLS <= kAccCols, "accumulators must fit one buffer of 256 columns");
  static_assert(NMMA >= 16 && NMMA <= 256, "MMA N for M = 128");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major tile without swizzle: core matrices of 8 rows x 16
// bytes stored whole; the second core matrix along K (a row's fp16 8..15) 128 bytes after the first
// (leading byte offset), the next group of 8 rows 256 bytes further (stride byte offset); descriptor
// version 1 (bits 46-47), base offset 0, layout type 0 (no swizzle, bits 61-63).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D in f32 (bits 4-5 = 1), A and B fp16 (bits 7-9, 10-12 = 0),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28, dense.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (+)= A B; acc = 0 overwrites D (used with an all-zero A to clear a task's accumulators)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc = 1u) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the completion of the barrier's phase of this parity; false after limit_ns (about two
// seconds unless given), or soon after another role of the CTA has given up (*abort set). Each try
// suspends the thread until the phase completes or 20 us pass (the suspend-time hint), so waiting
// warps do not take issue slots from the working ones.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = 2000000000ull) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 24); it++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(20000u)
        : "memory");
    if (done) return true;
    if (*abort || global_ns() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
  }
  *abort = 1;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


// Two 7-bit chunks (exact small integers) as one f16x2 word, the first in the low half: the fp16
// words 0x6400 | v are 1024 + v exactly (unit spacing in [1024, 2048)), and one f16x2 subtraction of
// 1024 leaves v exactly, without a conversion instruction per chunk.
__device__ __forceinline__ uint32_t chunk_pair(u64 x0, u64 x1, int sh) {
  const uint32_t a = (uint32_t)(x0 >> sh) & 127u, b = (uint32_t)(x1 >> sh) & 127u;
  const uint32_t biased = a | (b << 16) | 0x64006400u;
  __half2 h;
  memcpy(&h, &biased, 4);
  const __half2 r = __hsub2(h, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
  uint32_t out;
  memcpy(&out, &r, 4);
  return out;
}

// Row `row` of chunk tiles C in [LO, HI) (tile C at Ab + C A_TILE) from the 16 input words x of the
// row: chunk indexes and shifts are compile-time, so every extraction is a constant shift and mask.
template <int A_TILE, int C, int HI>
__device__ __forceinline__ void write_chunks(const u64 (&x)[16], unsigned char* Ab) {
  if constexpr (C < HI) {
    constexpr int sh = 7 * C;
    uint4 lo, hi;
    lo.x = chunk_pair(x[0], x[1], sh);
    lo.y = chunk_pair(x[2], x[3], sh);
    lo.z = chunk_pair(x[4], x[5], sh);
    lo.w = chunk_pair(x[6], x[7], sh);
    hi.x = chunk_pair(x[8], x[9], sh);
    hi.y = chunk_pair(x[10], x[11], sh);
    hi.z = chunk_pair(x[12], x[13], sh);
    hi.w = chunk_pair(x[14], x[15], sh);
    *reinterpret_cast<uint4*>(Ab + C * A_TILE) = lo;
    *reinterpret_cast<uint4*>(Ab + C * A_TILE + 128) = hi;
    write_chunks<A_TILE, C + 1, HI>(x, Ab);
  }
}

// Bytes of two words as one f16x2 word of signed values b - 128 (b the byte `bi` of the 32-bit
// halves w0, w1): one byte permutation places the bytes, a mask and the bias 0x6400 make the fp16
// words 1024 + b exactly, and one f16x2 subtraction of 1152 leaves b - 128 exactly.
__device__ __forceinline__ uint32_t byte_pair(uint32_t w0, uint32_t w1, uint32_t sel) {
  const uint32_t biased = (__byte_perm(w0, w1, sel) & 0x00FF00FFu) | 0x64006400u;
  __half2 h;
  memcpy(&h, &biased, 4);
  const __half2 r = __hsub2(h, __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  uint32_t out;
  memcpy(&out, &r, 4);
  return out;
}

// Row `row` of byte tiles C in [C, HI) from the 16 input words (residues below 2^48): tile C holds
// byte C of each word, less 128.
template <int A_TILE, int C, int HI>
__device__ __forceinline__ void write_bytes(const u64 (&x)[16], unsigned char* Ab) {
  if constexpr (C < HI) {
    constexpr int bi = C & 3;
    constexpr uint32_t sel = (uint32_t)bi | ((uint32_t)(4 + bi) << 8);  // result bytes 0, 2: w0.bi, w1.bi
    auto half = [](u64 v) { return C < 4 ? (uint32_t)v : (uint32_t)(v >> 32); };
    uint4 lo, hi;
    lo.x = byte_pair(half(x[0]), half(x[1]), sel);
    lo.y = byte_pair(half(x[2]), half(x[3]), sel);
    lo.z = byte_pair(half(x[4]), half(x[5]), sel);
    lo.w = byte_pair(half(x[6]), half(x[7]), sel);
    hi.x = byte_pair(half(x[8]), half(x[9]), sel);
    hi.y = byte_pair(half(x[10]), half(x[11]), sel);
    hi.z = byte_pair(half(x[12]), half(x[13]), sel);
    hi.w = byte_pair(half(x[14]), half(x[15]), sel);
    *reinterpret_cast<uint4*>(Ab + C * A_TILE) = lo;
    *reinterpret_cast<uint4*>(Ab + C * A_TILE + 128) = hi;
    write_bytes<A_TILE, C + 1, HI>(x, Ab);
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// tiled TMA load of one box of the 2-D tensor map at coordinates (x, y) into this CTA's shared memory
// (box rows one after another); the barrier counts the bytes as they land
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}


__device__ __forceinline__ void tc_ld(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_ld(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tc_ld(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// rot_map: the tensor map of the hoisted rotations stored column-major, [w_in][c_in][k][2][limbs][N]
// (ciphertext (j c_in + c) k + a is the rotation by g a of column j of channel c), so that the terms
// (b, c, a) of output column jp are the consecutive ciphertexts stride jp c_in k + (b c_in + c) k + a;
// w [c_out][c_in][k][k][limbs][2] (residue, Shoup companion),
// out [c_out][w_out][2][limbs][N]. NARROW: the limbs whose prime is below kMac96Prime (7 chunks),
// otherwise the others (9 chunks); blocks of the other class return at once.
//
// A CTA runs every task (channel group og, output column jp) of its tile, K step by K step, with
// its warps in four roles that hand work over through mbarriers (no CTA-wide barrier in the loop):
//  - warp 1, one thread: one tiled TMA box (128 words of 16 consecutive ciphertexts) per step into
//    a ring of ST stages ("full" barriers count the bytes; "xfree" says a stage was read);
//  - warps 2 .. 9: read a stage, convert the words into fp16 chunk tiles in one of AB buffers
//    (two threads a tile row, half of the chunks each; "afull" when written);
//  - warp 0, one thread: per task, one MMA with an all-zero A and accumulation off clears the
//    task's accumulator buffer (two buffers of 256 columns alternate between tasks), then per step
//    NC MMAs, committed to "aempty" (chunk buffer free) and, after the last step, to "accfull";
//  - warps 10 .. 17, two per lane quarter (half of the channels each): read a finished buffer,
//    recombine and store the task's residues, and release the buffer ("accempty") while the next
//    task's MMAs run.
template <int NC, int OBP, bool NARROW, int ST, int AB>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv_mac_tc_kernel(const __grid_constant__ CUtensorMap rot_map, u64* __restrict__ out,
                         const u64* __restrict__ w, int c_in, int w_in, int k, int stride, int c_out, int w_out,
                         int limbs, const PrimeTab* __restrict__ pt, int log_n, u64* status) {
  using S = TcShape<NC, OBP>;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const size_t N = (size_t)1 << log_n;
  const size_t LN = (size_t)limbs * N;
  const int i = blockIdx.y % limbs, comp = blockIdx.y / limbs;
  const Mod md = pt[i].mod;
  if ((md.q < kMac96Prime) != NARROW) return;  // uniform across the block, before any allocation
  const int kk2 = k * k, T = c_in * kk2, n_ks = (T + 15) >> 4;
  const int n_og = (c_out + OBP - 1) / OBP;
  // the CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ... of the limb's N / 128; per tile the
  // tasks (channel group, output column), each n_ks K steps; the pipeline runs across them all
  const int n_tiles = (int)(N / kTcRows);
  const int my_tiles = (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int per_tile = n_og * w_out;
  const int n_tasks = my_tiles * per_tile, G = n_tasks * n_ks;
  const size_t row0 = (size_t)comp * LN + (size_t)i * N;
  auto task_of = [&](int t, int& og, int& jp, size_t& tile) {
    const int m = t / per_tile, r = t - m * per_tile;
    og = r / w_out;
    jp = r - og * w_out;
    tile = row0 + (size_t)((int)blockIdx.x + m * (int)gridDim.x) * kTcRows;  // word of the tile's row 0
  };
  unsigned char* X = tc_smem;                                                 // [ST][16][128] words
  unsigned char* A = X + ST * kStageBytes;                               // [AB][NC][A_TILE]
  unsigned char* B = A + AB * NC * S::A_TILE;                             // [n_og][n_ks][B_TILE]
  unsigned char* Z = B + (size_t)n_og * n_ks * S::B_TILE;                   // kZeroBytes of zeros
  u64* csm = reinterpret_cast<u64*>(Z + kZeroBytes);                         // [NS] 2^(7 s) or 2^(8 s) mod q
  u64* corr = csm + S::NS;                                                    // [n_og OBP] (byte chunks)
  u64* bars = corr + n_og * OBP;
  u64* full = bars;                      // [ST]
  u64* xfree = full + ST;           // [ST]
  u64* afull = xfree + ST;          // [AB]
  u64* aempty = afull + AB;          // [AB]
  u64* accfull = aempty + AB;        // [2]
  u64* accempty = accfull + 2;           // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accempty + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // term t of an output column: (b, c, a) with t = (b c_in + c) k + a, the rotation by g a of input
  // column stride jp + b of channel c, at ciphertext stride jp c_in k + t of the column-major
  // rotations; weight tiles of every channel group: row r = j OBP + o holds chunk j of W[og OBP + o][t]
  const int ck = c_in * k;
  for (int e = tid; e < n_og * n_ks * S::NMMA * 16; e += kTcThreads) {
    const int og = e / (n_ks * S::NMMA * 16), e2 = e - og * (n_ks * S::NMMA * 16);
    const int ks = e2 / (S::NMMA * 16), rem = e2 - ks * (S::NMMA * 16), r = rem >> 4, kk = rem & 15;
    const int t = ks * 16 + kk, j = r / OBP, o = og * OBP + (r - j * OBP);
    uint32_t v = 0;
    if (j < NC && o < c_out && t < T) {
      const int b = t / ck, rr = t - b * ck, c = rr / k, a = rr - c * k;
      const u64 wv = w[(((size_t)o * T + (c * k + a) * k + b) * limbs + i) * 2];
      v = NARROW ? (uint32_t)(wv >> (8 * j)) & 255u : (uint32_t)(wv >> (7 * j)) & 127u;
    }
    __half* dst = reinterpret_cast<__half*>(B + ((size_t)og * n_ks + ks) * S::B_TILE + (r >> 3) * 256 +
                                            (kk >> 3) * 128 + (r & 7) * 16) +
                  (kk & 7);
    *dst = __uint2half_rn(v);
  }
  for (int e = tid; e < kZeroBytes / 16; e += kTcThreads) reinterpret_cast<uint4*>(Z)[e] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    u64 c = 1;
    for (int s = 0; s < S::NS; s++) {
      csm[s] = c;
      c = mulmod(c, NARROW ? 256 : 128, md);
    }
    for (int b = 0; b < ST; b++) {
      mbar_init(smem_u32(&full[b]), 1);
      mbar_init(smem_u32(&xfree[b]), kTcConvWarps);
    }
    for (int b = 0; b < AB; b++) {
      mbar_init(smem_u32(&afull[b]), kTcConvWarps);
      mbar_init(smem_u32(&aempty[b]), 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&accfull[b]), 1);
      mbar_init(smem_u32(&accempty[b]), kTcRecWarps);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (NARROW && tid < n_og * OBP) {
    // byte chunks: x = sum_i (b_i - 128) 256^i + K0, K0 = 128 (256^6 - 1) / 255, so channel o's
    // sum gains K0 sum_t W[o][t]; the recombination adds 2^24 to each signed D_s, so it loses
    // 2^24 sum_s 256^s. corr[o] = K0 sum_t W[o][t] - 2^24 sum_s 256^s mod q (0 past c_out).
    u64 wsum = 0;
    if (tid < c_out)
      for (int t = 0; t < T; t++) wsum = addmod(wsum, w[((size_t)tid * T + t) * limbs * 2 + (size_t)i * 2], md.q);
    u64 c = 1, cs = 0;
    for (int s = 0; s < S::NS; s++) {
      cs = addmod(cs, c, md.q);
      c = mulmod(c, 256, md);
    }
    const u64 k0 = 0x808080808080ull % md.q, two24 = (1ull << 24) % md.q;
    const u64 v = addmod(mulmod(k0, wsum, md), (md.q - mulmod(two24, cs, md)) % md.q, md.q);
    corr[tid] = tid < c_out ? v : 0;
  }
  if (warp == 0) {
    tc_alloc(smem_u32(tslot), 2 * kAccCols);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  fence_async_smem();  // the weight and zero tiles, written by every thread, before the first MMA reads them
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    // ---- MMA issue ----
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc(kTcRows, S::NMMA);
      constexpr uint32_t idesc_zero = tc_idesc(kTcRows, S::ZCOLS);
      const uint64_t zdesc = tc_desc(smem_u32(Z));
      for (int t = 0; t < n_tasks; t++) {
        const int acc = t & 1;
        int og, jp_unused;
        size_t tile_unused;
        task_of(t, og, jp_unused, tile_unused);
        if (t >= 2 && !mbar_wait(smem_u32(&accempty[acc]), ((t >> 1) - 1) & 1, abort)) break;
        tc_fence_after();
        const uint32_t tacc = tmem + acc * kAccCols;
        tc_mma(tacc, zdesc, zdesc, idesc_zero, 0u);  // the buffer's ZCOLS columns := 0
        bool ok = true;
        for (int ks = 0; ks < n_ks; ks++) {
          const int g = t * n_ks + ks, ab = g % AB;
          if (!(ok = mbar_wait(smem_u32(&afull[ab]), (uint32_t)((g / AB) & 1), abort))) break;
          tc_fence_after();
          const uint64_t bdesc = tc_desc(smem_u32(B + ((size_t)og * n_ks + ks) * S::B_TILE));
#pragma unroll
          for (int c = 0; c < NC; c++)
            tc_mma(tacc + c * OBP, tc_desc(smem_u32(A + ((size_t)ab * NC + c) * S::A_TILE)), bdesc, idesc);
          tc_commit(smem_u32(&aempty[ab]));
        }
        if (!ok) break;
        tc_commit(smem_u32(&accfull[acc]));
      }
    }
  } else if (warp == 1) {
    // ---- bulk copies of the input words ----
    if (lane == 0) {
      for (int g = 0; g < G; g++) {
        const int st = g % ST;
        if (g >= ST && !mbar_wait(smem_u32(&xfree[st]), (uint32_t)(((g / ST) - 1) & 1), abort)) break;
        const int t = g / n_ks, ks = g - t * n_ks;
        int og_unused, jp;
        size_t tile;
        task_of(t, og_unused, jp, tile);
        // one box: 128 words of each of the step's 16 consecutive ciphertexts (past the column's
        // last term it reads the next column's, or zeros past the array; those rows go unused)
        const uint32_t bar = smem_u32(&full[st]);
        mbar_expect_tx(bar, (uint32_t)kStageBytes);
        tma_load_2d(smem_u32(X + (size_t)st * kStageBytes), &rot_map, (int)tile,
                    stride * jp * ck + 16 * ks, bar);
      }
    }
  } else if (warp < 2 + kTcConvWarps) {
    // ---- chunk conversion ----
    constexpr int NQ = kTcConvWarps / 4;  // threads a tile row (each converts its share of the chunks)
    const int ci = tid - 64, row = ci & (kTcRows - 1), part = ci >> 7;  // first or second half of the chunks
    const int arow = (row >> 3) * 256 + (row & 7) * 16;
    static_assert(NQ == 2, "two chunk shares");
    for (int g = 0; g < G; g++) {
      const int ks = g % n_ks, st = g % ST, ab = g % AB;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((g / ST) & 1), abort)) break;
      const u64* xs = reinterpret_cast<const u64*>(X + (size_t)st * kStageBytes) + row;
      const int nreal = min(16, T - 16 * ks);
      u64 x[16];
#pragma unroll
      for (int v = 0; v < 16; v++) x[v] = v < nreal ? xs[v * kTcRows] : 0;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&xfree[st]));
      if (g >= AB && !mbar_wait(smem_u32(&aempty[ab]), (uint32_t)(((g / AB) - 1) & 1), abort)) break;
      unsigned char* Ab = A + (size_t)ab * NC * S::A_TILE + arow;
      if constexpr (NARROW) {
        if (part == 0)  // warp-uniform
          write_bytes<S::A_TILE, 0, (NC + 1) / 2>(x, Ab);
        else
          write_bytes<S::A_TILE, (NC + 1) / 2, NC>(x, Ab);
      } else {
        if (part == 0)
          write_chunks<S::A_TILE, 0, (NC + 1) / 2>(x, Ab);
        else
          write_chunks<S::A_TILE, (NC + 1) / 2, NC>(x, Ab);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&afull[ab]));
    }
  } else {
    // ---- recombination: kTcRecWarps / 4 warps per lane quarter, each a share of the channels ----
    // Per channel: sum_s D_s c_s with D_s < 2^24 and c_s = c_hi 2^32 + c_lo, as two independent
    // 64-bit sums of 32 x 32-bit products (below 2^60 for up to 17 sums), joined at the end.
    constexpr int RQ = kTcRecWarps / 4;  // warps per lane quarter
    constexpr int OH = OBP / RQ;         // channels of one warp
    const int rw = warp - 2 - kTcConvWarps, q4 = warp & 3, oh0 = (rw / 4) * OH;
    const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
    const int erow = q4 * 32 + lane;
    constexpr int LB = OH >= 16 ? 2 : OH == 8 ? 4 : 7;  // sums loaded before one wait
    for (int t = 0; t < n_tasks; t++) {
      const int acc = t & 1;
      if (!mbar_wait(smem_u32(&accfull[acc]), (uint32_t)((t >> 1) & 1), abort)) break;
      tc_fence_after();
      const uint32_t tacc = tmem + acc * kAccCols + lanes + oh0;
      u64 slo[OH], shi[OH];
#pragma unroll
      for (int o = 0; o < OH; o++) slo[o] = shi[o] = 0;
#pragma unroll
      for (int s0 = 0; s0 < S::NS; s0 += LB) {
        uint32_t d[LB][OH];
#pragma unroll
        for (int q = 0; q < LB; q++)
          if (s0 + q < S::NS) tc_ld(tacc + (s0 + q) * OBP, d[q]);
        tc_wait_ld();
#pragma unroll
        for (int q = 0; q < LB; q++) {
          if (s0 + q < S::NS) {
            const u64 cs = csm[s0 + q];
            const uint32_t clo = (uint32_t)cs, chi = (uint32_t)(cs >> 32);
#pragma unroll
            for (int o = 0; o < OH; o++) {
              // byte chunks: D_s signed, below 2^24 in magnitude, taken as D_s + 2^24
              const uint32_t dv = NARROW ? (uint32_t)(__float2int_rn(__uint_as_float(d[q][o])) + (1 << 24))
                                         : __float2uint_rn(__uint_as_float(d[q][o]));
              slo[o] += (u64)dv * clo;
              shi[o] += (u64)dv * chi;
            }
          }
        }
      }
      // the buffer is read: the MMAs of the task after next may clear it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&accempty[acc]));
      int og, jp;
      size_t tile;
      task_of(t, og, jp, tile);
      const int o0 = og * OBP + oh0;
      u64* dst = out + ((size_t)o0 * w_out + jp) * 2 * LN + tile + erow;
      const size_t ostep = (size_t)w_out * 2 * LN;
#pragma unroll
      for (int o = 0; o < OH; o++) {
        if (o0 + o >= c_out) continue;
        if constexpr (NARROW) slo[o] += corr[o0 + o];  // below 2^62 with it
        const u64 vlo = slo[o] + (shi[o] << 32);
        const u64 vhi = (shi[o] >> 32) + (vlo < slo[o]);
        dst[o * ostep] = reduce128(vhi, vlo, md);
      }
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, 2 * kAccCols);
  if (*abort && tid == 0) atomicOr(reinterpret_cast<unsigned long long*>(status), 1ull);
}

// A wait that nothing ends, for tests of the failure path: one thread waits on a barrier of its CTA
// that no thread arrives on, gives up after limit_ns, records the failure in the status word (as the
// tensor-core kernels do) and returns; the host reports it at its next synchronisation.
__global__ void k_wait_expires_kernel(u64* status, uint64_t limit_ns) {
  __shared__ __align__(8) u64 bar;
  __shared__ int give_up;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    give_up = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0, &give_up, limit_ns))
    atomicOr(reinterpret_cast<unsigned long long*>(status), 2ull);
}

template <int NC, int OBP, int ST, int AB>
size_t tc_smem_bytes(int T, int c_out) {
  using S = TcShape<NC, OBP>;
  const int n_ks = (T + 15) / 16, n_og = (c_out + OBP - 1) / OBP;
  return (size_t)ST * kStageBytes + (size_t)AB * NC * S::A_TILE + (size_t)n_og * n_ks * S::B_TILE + kZeroBytes +
         S::NS * 8 + (size_t)n_og * OBP * 8 + (2 * ST + 2 * AB + 4) * 8 + 16;
}

// The tensor map of the column-major rotations: dimension 0 the words of a ciphertext (2 limbs N,
// contiguous), dimension 1 the ciphertexts (2 limbs N words apart); boxes of 128 words by 16
// ciphertexts, one K step of one tile. Reads past the last ciphertext fill zeros.
static CUtensorMap rot_tensor_map(const u64* rot, size_t ct_words, size_t n_cts) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    HE_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) throw Error(7, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)ct_words, (cuuint64_t)n_cts};
  const cuuint64_t strides[1] = {(cuuint64_t)ct_words * 8};
  const cuuint32_t box[2] = {(cuuint32_t)kTcRows, 16u};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<u64*>(rot), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(7, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return map;
}

template <int NC, int OBP, bool NARROW, int ST, int AB>
void launch_tc(const Ctx& C, const u64* rot, u64* out, const u64* w, int c_in, int w_in, int k, int stride,
               int c_out, int w_out, int limbs, int n_class, const char* name) {
  const int T = c_in * k * k;
  const size_t smem = tc_smem_bytes<NC, OBP, ST, AB>(T, c_out);
  if (smem > kTcSmemMax) throw Error(8, "convolution too large for the tensor-core multiply-accumulate");
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    HE_CUDA(cudaFuncSetAttribute(k_conv_mac_tc_kernel<NC, OBP, NARROW, ST, AB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax));
    HE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C.device));
    attr = true;
  }
  // one CTA per SM at a time (its shared memory and all tensor memory), one tile of one
  // (component, limb) each
  (void)sms;
  const int gx = (int)(C.N / kTcRows);  // one tile a CTA
  const dim3 grid((unsigned)gx, (unsigned)(2 * limbs), 1);
  const double per_limb_bytes =
      8.0 * (double)C.N * 2.0 * ((double)c_in * (stride * (w_out - 1) + k) * k + (double)c_out * w_out);
  const double prods = 2.0 * C.N * (double)c_out * w_out * T * n_class;
  void* tok = prof_begin(name, C.stream, per_limb_bytes * n_class, prods);
  const size_t ct_words = (size_t)2 * limbs * C.N;
  if ((reinterpret_cast<uintptr_t>(rot) & 15) || ct_words % 2) throw Error(1, "rotations not 16-byte aligned");
  const CUtensorMap map = rot_tensor_map(rot, ct_words, (size_t)w_in * c_in * k);
  k_conv_mac_tc_kernel<NC, OBP, NARROW, ST, AB><<<grid, kTcThreads, smem, C.stream>>>(
      map, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, C.dev_ptab(), C.log_n, C.d_status.p);
  prof_end(tok, C.stream);
  HE_CUDA(cudaGetLastError());
}

}  // namespace

void k_wait_expires(const Ctx& C, uint64_t limit_ns) {
  k_wait_expires_kernel<<<1, 32, 0, C.stream>>>(C.d_status.p, limit_ns);
  HE_CUDA(cudaGetLastError());
}

// shared memory of the launch k_conv_mac_tc makes for a class of limbs
static size_t tc_smem_for(int T, int c_out, bool narrow) {
  if (!narrow) return tc_smem_bytes<9, 8, 6, 2>(T, c_out);
  return c_out <= 8 ? tc_smem_bytes<6, 8, 6, 3>(T, c_out) : tc_smem_bytes<6, 16, 6, 3>(T, c_out);
}

bool conv_mac_tc_all(const Ctx& C, int c_in, int k, int c_out, int lp) {
  if (!C.use_tc || C.log_n < 7) return false;
  const long T = (long)c_in * k * k;
  // below about 128 products per output column and word the CUDA-core kernels are faster: their
  // cost is a few multiplies per product, the tensor path's a conversion per input word and a
  // recombination per output (measured: 4 channels of 9 terms 20.5 ms on the CUDA cores against
  // 22.7 ms here; 8 channels of 25 terms 13.0 against 11.9; 16 of 72, 28.2 against 10.7)
  if (T * c_out < 128) return false;
  bool narrow = false, wide = false;
  for (int i = 0; i < lp; i++) (C.q[i] < kMac96Prime ? narrow : wide) = true;
  // the chunk sums below 2^24: NC T 127^2 (NC = 7 below kMac96Prime, 9 above); every channel
  // group's weight tiles held in shared memory
  const bool ok_n = !narrow || (6 * T * 128 * 255 < (1L << 24) && tc_smem_for((int)T, c_out, true) <= kTcSmemMax);
  const bool ok_w = !wide || (9 * T * 127 * 127 < (1L << 24) && tc_smem_for((int)T, c_out, false) <= kTcSmemMax);
  return ok_n && ok_w;
}

void k_conv_mac_tc(const Ctx& C, const u64* rot, u64* out, const u64* w, int c_in, int w_in, int k, int stride,
                   int c_out, int w_out, int limbs, bool narrow) {
  int n_class = 0;
  for (int i = 0; i < limbs; i++) n_class += (C.q[i] < kMac96Prime) == narrow;
  if (n_class == 0) return;
  if (narrow) {
    if (c_out <= 8)
      launch_tc<6, 8, true, 6, 3>(C, rot, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, n_class,
                                  "k_conv_mac_tc_kernel<6, 8>");
    else
      launch_tc<6, 16, true, 6, 3>(C, rot, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, n_class,
                                   "k_conv_mac_tc_kernel<6, 16>");
  } else {
    launch_tc<9, 8, false, 6, 2>(C, rot, out, w, c_in, w_in, k, stride, c_out, w_out, limbs, n_class,
                                 "k_conv_mac_tc_kernel<9, 8>");
  }
}

}  // namespace he
