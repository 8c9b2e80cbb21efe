// noalloc.cu - he_rescale_noalloc: a rescale that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: a serving loop
// that must keep a fixed memory footprint once it has started, a host
// framework that hands out every device allocation from its own pool and
// forbids others, or a process under a device-memory quota that is already
// used up. For them this entry point takes caller-owned input and output
// buffers and keeps its scratch in one array that the library holds in every
// GPU's memory for the life of the process (file-scope __device__ storage,
// 16 MiB), so the call itself makes no cudaMalloc / cudaFree or any other
// allocating call. The paper has no counterpart; it is an interface for such
// callers.
#include <map>
#include <mutex>

#include "../../include/he_gb300.h"
#include "he_internal.h"

namespace he {

// Scratch of he_rescale_noalloc, shared by every call in this process: 2^21
// words (16 MiB) on each GPU that loads the library.
constexpr size_t kNoAllocWords = (size_t)1 << 21;
static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocWords];

// Device address of the scratch array on the current device. The array's
// name in host code is a host-side stand-in, not a device address, so the
// address is looked up once per device (with that device current) and cached.
static u64* noalloc_scratch(int device) {
  static std::mutex mu;
  static std::map<int, u64*> addr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = addr.find(device);
  if (it != addr.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(HE_E_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") + cudaGetErrorString(e));
  }
  addr[device] = (u64*)p;
  return (u64*)p;
}

}  // namespace he

using namespace he;

extern "C" {

int he_rescale_noalloc(he_ctx* ctx, const uint64_t* in, int n_ct, int limbs, double scale, uint64_t* out,
                       double* out_scale) {
  try {
    if (!ctx || !in || !out) throw Error(HE_E_ARG, "null argument");
    HANDLE(ctx);
    Ctx& C = ctx->c;
    if (n_ct < 1 || limbs < 2 || limbs > C.L1) throw Error(HE_E_ARG, "need n_ct >= 1 and 2 <= limbs <= n_q");
    const size_t N = C.N;
    const size_t rows = (size_t)n_ct * 2;
    const size_t need = rows * (size_t)limbs * N;  // last limb (rows x N) + rounding terms (rows x (limbs-1) x N)
    if (need > kNoAllocWords)
      throw Error(HE_E_ARG, "he_rescale_noalloc: n_ct * 2 * limbs * N = " + std::to_string(need) +
                                " words exceeds the scratch of " + std::to_string(kNoAllocWords) + " words (16 MiB)");
    const uint64_t* in_end = in + rows * limbs * N;
    const uint64_t* out_end = out + rows * (limbs - 1) * N;
    if (in < out_end && out < in_end) throw Error(HE_E_ARG, "input and output overlap");
    int dev = -1;
    HE_CUDA(cudaGetDevice(&dev));
    if (dev != C.device) throw Error(HE_E_ARG, "the context's device must be current");
    u64* last = noalloc_scratch(dev);
    u64* r = last + rows * N;
    // same steps as he_rescale: last limb to the coefficient domain, rounding
    // polynomial per remaining prime, forward NTT, (x_i - r_i) q_l^{-1}
    k_copy_limbs(C, in + (size_t)(limbs - 1) * N, (size_t)limbs * N, last, N, rows, 1);
    LimbMap lm1;
    lm1.lpp = 1; lm1.split = 1; lm1.base0 = limbs - 1; lm1.base1 = 0; lm1.poly_stride = N;
    ntt_inverse(C, last, (int)rows, lm1);
    k_rescale_expand(C, last, r, (int)rows, limbs);
    ntt_forward(C, r, (int)rows, limbs_q(limbs - 1, N));
    k_rescale_combine(C, in, r, out, (int)rows, limbs);
    if (out_scale) *out_scale = scale / (double)C.q[limbs - 1];
    set_last_error("");
    return HE_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return HE_E_CUDA;
  }
}

}  // extern "C"
