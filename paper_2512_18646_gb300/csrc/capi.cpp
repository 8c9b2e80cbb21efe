// capi.cpp - the extern "C" entry points declared in include/he_gb300.h.
// Argument checking, the paper's slot layouts (image columns, matrix
// columns / tiled rows, diagonal matmul output), and translation of internal
// errors into status codes; all arithmetic runs in the kernels.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <thread>
#include <vector>

#include "../../include/he_gb300.h"
#include "he_internal.h"

using namespace he;

static thread_local std::string g_err;

namespace he {
void set_last_error(const std::string& msg) { g_err = msg; }

// the registry is never destroyed, so handles freed during process exit still find it
static std::mutex& reg_mu() {
  static std::mutex* m = new std::mutex;
  return *m;
}
static std::unordered_map<const void*, int>& reg() {
  static auto* r = new std::unordered_map<const void*, int>;
  return *r;
}
void handle_add(const void* h, int kind) {
  std::lock_guard<std::mutex> lk(reg_mu());
  reg()[h] = kind;
}
void handle_remove(const void* h) {
  std::lock_guard<std::mutex> lk(reg_mu());
  reg().erase(h);
}
bool handle_is(const void* h, int kind) {
  std::lock_guard<std::mutex> lk(reg_mu());
  auto it = reg().find(h);
  return it != reg().end() && it->second == kind;
}
}  // namespace he

template <class F>
static int guard(F f) {
  try {
    f();
    g_err.clear();
    return HE_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return HE_E_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return HE_E_CUDA;
  }
}

#define REQUIRE(cond, code, msg) \
  do {                           \
    if (!(cond)) throw Error((code), (msg)); \
  } while (0)

static bool pow2(long x) { return x > 0 && (x & (x - 1)) == 0; }


// Encode slot vectors z [n][M] (host) at scale and encrypt at the top level.
static std::unique_ptr<CtSet> encrypt_slots(Ctx& C, const std::vector<double>& z, int n, u64 id_base) {
  const size_t M = C.N / 2;
  std::vector<int64_t> m((size_t)n * C.N);
  host_parallel((size_t)n, [&](size_t c) { encode_real(C, z.data() + c * M, M, C.scale0, m.data() + c * C.N); });
  return encrypt_coeffs(C, m.data(), n, C.L1, C.scale0, id_base);
}

static he_ctset* wrap(std::unique_ptr<CtSet> s) {
  he_ctset* h = new he_ctset;
  h->s = std::move(s);
  return h;
}

extern "C" {

const char* he_last_error(void) { return g_err.c_str(); }

int he_ctx_create(const he_params_desc* d, uint64_t seed, void* cuda_stream, he_ctx** out) {
  return guard([&] {
    REQUIRE(d && out && d->q_bits, HE_E_ARG, "null argument");
    REQUIRE(d->n_q >= 1 && d->n_q <= 32, HE_E_ARG, "n_q must be in [1, 32]");
    std::vector<int> qb(d->q_bits, d->q_bits + d->n_q);
    auto* h = new he_ctx;
    try {
      ctx_init(h->c, d->log_n, qb, d->n_special, d->special_bits, d->alpha, d->log_scale, d->sigma, seed,
               (cudaStream_t)cuda_stream);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

void he_ctx_destroy(he_ctx* ctx) {
  if (ctx && !handle_live(ctx)) return;
  if (!ctx) return;
  const cudaStream_t st = ctx->c.stream;
  const int dev = ctx->c.device;
  cudaStreamSynchronize(st);
  delete ctx;
  // the buffers were freed in stream order: once the stream has passed the frees, hand the pool's
  // cached memory back (the release threshold set at creation keeps it otherwise)
  cudaStreamSynchronize(st);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  cudaGetLastError();
}

int he_ctx_synchronize(he_ctx* ctx) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null context");
    HE_CUDA(cudaStreamSynchronize(ctx->c.stream));
    check_device_status(ctx->c);
  });
}

int he_ctx_primes(const he_ctx* ctx, uint64_t* out, int n) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && out, HE_E_ARG, "null argument");
    REQUIRE(n >= ctx->c.np(), HE_E_ARG, "output too small");
    for (int i = 0; i < ctx->c.np(); i++) out[i] = ctx->c.q[i];
  });
}

int he_ctx_info(const he_ctx* ctx, int* log_n, int* n_q, int* n_special, int* alpha, double* scale) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null context");
    if (log_n) *log_n = ctx->c.log_n;
    if (n_q) *n_q = ctx->c.L1;
    if (n_special) *n_special = ctx->c.K;
    if (alpha) *alpha = ctx->c.alpha;
    if (scale) *scale = ctx->c.scale0;
  });
}

int he_keygen(he_ctx* ctx, const int32_t* rot_steps, int n_steps) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && n_steps >= 0 && (n_steps == 0 || rot_steps), HE_E_ARG, "bad arguments");
    std::vector<long> st(rot_steps, rot_steps + n_steps);
    keygen(ctx->c, st);
  });
}

int he_keys_export(he_ctx* ctx, uint64_t* words, size_t n_words, size_t* needed) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && (words || needed), HE_E_ARG, "null argument");
    const size_t need = keys_export(ctx->c, nullptr, 0);
    if (needed) *needed = need;
    if (words) keys_export(ctx->c, words, n_words);
  });
}

int he_keys_import(he_ctx* ctx, const uint64_t* words, size_t n_words) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && words, HE_E_ARG, "null argument");
    keys_import(ctx->c, words, n_words);
  });
}

int he_encrypt_image(he_ctx* ctx, const double* px, int batch, int h, int w, int block_stride, uint64_t ct_id_base,
                     he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && px && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long M = (long)C.N / 2;
    REQUIRE(batch >= 1 && h >= 1 && w >= 1, HE_E_ARG, "empty image");
    REQUIRE(pow2(block_stride) && block_stride >= h, HE_E_ARG, "block_stride must be a power of two >= h");
    REQUIRE((long)batch * block_stride <= M, HE_E_ARG, "batch * block_stride exceeds the slot count");
    std::vector<double> z((size_t)w * M, 0.0);
    for (int b = 0; b < batch; b++)
      for (int i = 0; i < h; i++)
        for (int j = 0; j < w; j++) z[(size_t)j * M + (size_t)b * block_stride + i] = px[((size_t)b * h + i) * w + j];
    *out = wrap(encrypt_slots(C, z, w, ct_id_base));
  });
}

int he_encrypt_matrix_a(he_ctx* ctx, const double* A, int m, int n, uint64_t ct_id_base, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && A && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long M = (long)C.N / 2;
    REQUIRE(m >= 1 && n >= 1 && m <= M, HE_E_ARG, "bad matrix shape");
    std::vector<double> z((size_t)n * M, 0.0);
    for (int k = 0; k < n; k++)
      for (int i = 0; i < m; i++) z[(size_t)k * M + i] = A[(size_t)i * n + k];
    *out = wrap(encrypt_slots(C, z, n, ct_id_base));
  });
}

int he_encrypt_matrix_b(he_ctx* ctx, const double* B, int n, int p, uint64_t ct_id_base, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && B && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long M = (long)C.N / 2;
    REQUIRE(n >= 1 && p >= 1 && M % p == 0, HE_E_ARG, "p must divide the slot count");
    std::vector<double> z((size_t)n * M);
    for (int k = 0; k < n; k++)
      for (long s = 0; s < M; s++) z[(size_t)k * M + s] = B[(size_t)k * p + (s % p)];
    *out = wrap(encrypt_slots(C, z, n, ct_id_base));
  });
}

int he_volley_geometry(int slots, int m, int p, int* M, int* per, int* groups) {
  return guard([&] {
    REQUIRE(M && per && groups && slots >= 1, HE_E_ARG, "null argument");
    volley_geometry(slots, m, p, *M, *per, *groups);
  });
}

int he_encrypt_matrix_a_volley(he_ctx* ctx, const double* A, int m, int n, int p, uint64_t ct_id_base,
                               he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && A && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long S = (long)C.N / 2;
    REQUIRE(n >= 1, HE_E_ARG, "bad matrix shape");
    int Mb, per, G;
    volley_geometry(S, m, p, Mb, per, G);
    std::vector<double> z((size_t)G * n * S, 0.0);
    for (int g = 0; g < G; g++) {
      const long o = ((long)g * per) % p;
      for (int t = 0; t < per && g * per + t < p; t++)
        for (int k = 0; k < n; k++)
          for (int i = 0; i < m; i++) z[((size_t)g * n + k) * S + (size_t)t * Mb + o + i] = A[(size_t)i * n + k];
    }
    *out = wrap(encrypt_slots(C, z, G * n, ct_id_base));
  });
}

int he_encrypt_coeffs(he_ctx* ctx, const int64_t* m, int n_ct, int limbs, double scale, uint64_t ct_id_base,
                      he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && m && out, HE_E_ARG, "null argument");
    REQUIRE(scale > 0, HE_E_ARG, "scale must be positive");
    *out = wrap(encrypt_coeffs(ctx->c, m, n_ct, limbs, scale, ct_id_base));
  });
}

int he_matmul(he_ctx* ctx, const he_ctset* A, const he_ctset* B, int m, int p, he_ctset** C_out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(A);
    HANDLE(B);
    REQUIRE(ctx && A && B && C_out, HE_E_ARG, "null argument");
    REQUIRE(m >= 1 && (size_t)m <= ctx->c.N / 2, HE_E_ARG, "bad m");
    REQUIRE(A->s->scale == B->s->scale, HE_E_SCALE, "operands at different scales");
    *C_out = wrap(matmul(ctx->c, *A->s, *B->s, p));
  });
}

int he_matmul_range(he_ctx* ctx, const he_ctset* A, const he_ctset* B, int m, int p, int idx_lo, int idx_hi,
                    he_ctset** C_out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(A);
    HANDLE(B);
    REQUIRE(ctx && A && B && C_out, HE_E_ARG, "null argument");
    REQUIRE(m >= 1 && (size_t)m <= ctx->c.N / 2, HE_E_ARG, "bad m");
    REQUIRE(idx_lo >= 0 && idx_lo < idx_hi && idx_hi <= p, HE_E_ARG, "diagonal range outside [0, p)");
    REQUIRE(A->s->scale == B->s->scale, HE_E_SCALE, "operands at different scales");
    *C_out = wrap(matmul(ctx->c, *A->s, *B->s, p, idx_lo, idx_hi));
  });
}

int he_matmul_bsgs(he_ctx* ctx, const he_ctset* A, const he_ctset* B, int m, int p, int g, he_ctset** C_out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(A);
    HANDLE(B);
    REQUIRE(ctx && A && B && C_out, HE_E_ARG, "null argument");
    REQUIRE(m >= 1 && (size_t)m <= ctx->c.N / 2, HE_E_ARG, "bad m");
    REQUIRE(A->s->scale == B->s->scale, HE_E_SCALE, "operands at different scales");
    REQUIRE(p >= 1 && (long)m + p - 1 <= (long)ctx->c.N / 2, HE_E_ARG, "m + p - 1 exceeds the slot count");
    if (g <= 0) {  // the power of two nearest sqrt(p)
      g = 1;
      while ((long)4 * g * g <= (long)2 * p) g *= 2;
      if (g > p) g = p;
    }
    *C_out = wrap(matmul_bsgs(ctx->c, *A->s, *B->s, p, g));
  });
}

int he_matmul_volley(he_ctx* ctx, const he_ctset* A, const he_ctset* B, he_ctset** C_out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(A);
    HANDLE(B);
    REQUIRE(ctx && A && B && C_out, HE_E_ARG, "null argument");
    REQUIRE(A->s->scale == B->s->scale, HE_E_SCALE, "operands at different scales");
    *C_out = wrap(matmul_volley(ctx->c, *A->s, *B->s));
  });
}

int he_matmul_batched(he_ctx* ctx, int count, const he_ctset* const* A, const he_ctset* const* B, const int* m,
                      const int* p, he_ctset** C_out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && count >= 0 && (count == 0 || (A && B && m && p && C_out)), HE_E_ARG, "null argument");
    std::vector<const CtSet*> As(count), Bs(count);
    std::vector<int> ps(p, p + count);
    for (int i = 0; i < count; i++) {
      REQUIRE(A[i] && B[i], HE_E_ARG, "null operand");
      HANDLE(A[i]);
      HANDLE(B[i]);
      REQUIRE(A[i]->s->scale == B[i]->s->scale, HE_E_SCALE, "operands at different scales");
      REQUIRE(m[i] >= 1 && (size_t)m[i] <= ctx->c.N / 2, HE_E_ARG, "bad m");
      As[i] = A[i]->s.get();
      Bs[i] = B[i]->s.get();
    }
    std::vector<std::unique_ptr<CtSet>> res = matmul_batched(ctx->c, As, Bs, ps);
    for (int i = 0; i < count; i++) C_out[i] = wrap(std::move(res[i]));
  });
}

int he_conv2d(he_ctx* ctx, const he_ctset* in, int c_in, int gap, const double* weights, const double* bias, int c_out,
              int k, int stride, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && weights && out, HE_E_ARG, "null argument");
    *out = wrap(conv2d(ctx->c, *in->s, c_in, gap, weights, bias, c_out, k, stride));
  });
}

int he_encrypt_conv_weights(he_ctx* ctx, const double* W, int c_out, int c_in, int k, int limbs, uint64_t ct_id_base,
                            he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && W && out, HE_E_ARG, "null argument");
    REQUIRE(c_out >= 1 && c_in >= 1 && k >= 1, HE_E_ARG, "bad kernel shape");
    Ctx& C = ctx->c;
    REQUIRE(limbs >= 2 && limbs <= C.L1, HE_E_LEVEL, "bad level");
    const size_t nw = (size_t)c_out * c_in * k * k;
    const double ql = (double)C.q[limbs - 1];
    std::vector<int64_t> m(nw * C.N, 0);
    for (size_t t = 0; t < nw; t++) m[t * C.N] = std::llround(W[t] * ql);  // the constant K q_l
    *out = wrap(encrypt_coeffs(C, m.data(), (int)nw, limbs, ql, ct_id_base));
  });
}

int he_conv2d_enc(he_ctx* ctx, const he_ctset* in, int c_in, int gap, const he_ctset* weights, const double* bias,
                  int c_out, int k, int stride, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    HANDLE(weights);
    REQUIRE(ctx && in && weights && out, HE_E_ARG, "null argument");
    *out = wrap(conv2d_enc(ctx->c, *in->s, c_in, gap, *weights->s, bias, c_out, k, stride));
  });
}

int he_poly_act(he_ctx* ctx, he_ctset* inout, const double* coeffs, int degree) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(inout);
    REQUIRE(ctx && inout && coeffs, HE_E_ARG, "null argument");
    REQUIRE(!ctx->c.capturing || inout->s->gen == ctx->c.capture_gen, HE_E_STATE,
            "in-place operation on a set made before the capture");
    REQUIRE(degree == 2 || degree == 3, HE_E_UNIMPL, "degree 2 or 3 polynomials only");
    if (degree == 2 && coeffs[0] == 0.0 && coeffs[1] == 0.0 && coeffs[2] == 1.0) {
      inout->s = square(ctx->c, *inout->s);  // three components until an operation needs two
      return;
    }
    const double c[4] = {coeffs[0], coeffs[1], coeffs[2], degree == 3 ? coeffs[3] : 0.0};
    inout->s = poly_act3(ctx->c, *inout->s, c);
  });
}

int he_fc_prepare(he_ctx* ctx, const double* W, int out_dim, int c_in, int h_valid, int w_in, int gap,
                  int block_stride, int batch, int limbs, he_ptset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && W && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long M = (long)C.N / 2;
    REQUIRE(out_dim >= 1 && c_in >= 1 && h_valid >= 1 && w_in >= 1 && gap >= 1, HE_E_ARG, "bad shape");
    REQUIRE(pow2(block_stride) && pow2(gap) && (long)gap * (h_valid - 1) < block_stride, HE_E_ARG,
            "rows do not fit the blocks");
    REQUIRE(batch >= 1 && (long)batch * block_stride <= M, HE_E_ARG, "batch * block_stride exceeds the slot count");
    REQUIRE(limbs >= 2 && limbs <= C.L1, HE_E_LEVEL, "bad level");
    const int n_in = c_in * w_in;
    const double ql = (double)C.q[limbs - 1];
    std::vector<int64_t> pts((size_t)out_dim * n_in * C.N);
    const size_t row = (size_t)c_in * h_valid * w_in;
    host_parallel((size_t)out_dim * n_in, [&](size_t t) {
      const int o = (int)(t / n_in), cj = (int)(t % n_in), c = cj / w_in, j = cj % w_in;
      std::vector<double> z(M, 0.0);
      for (int b = 0; b < batch; b++)
        for (int i = 0; i < h_valid; i++)
          z[(size_t)b * block_stride + (size_t)gap * i] = W[(size_t)o * row + ((size_t)c * h_valid + i) * w_in + j];
      encode_real(C, z.data(), M, ql, pts.data() + t * C.N);
    });
    auto* h = new he_ptset;
    h->ctx = &C;
    h->out_dim = out_dim; h->n_in = n_in; h->limbs = limbs; h->gap = gap; h->block_stride = block_stride;
    try {
      h->buf = fc_prepare(C, pts.data(), out_dim, n_in, limbs);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

int he_fc_prepare_coeffs(he_ctx* ctx, const int64_t* pts, int out_dim, int c_in, int w_in, int gap, int block_stride,
                         int limbs, he_ptset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && pts && out, HE_E_ARG, "null argument");
    REQUIRE(out_dim >= 1 && c_in >= 1 && w_in >= 1, HE_E_ARG, "bad shape");
    REQUIRE(pow2(block_stride) && pow2(gap), HE_E_ARG, "gap and block_stride must be powers of two");
    REQUIRE(limbs >= 2 && limbs <= ctx->c.L1, HE_E_LEVEL, "bad level");
    auto* h = new he_ptset;
    h->ctx = &ctx->c;
    h->out_dim = out_dim; h->n_in = c_in * w_in; h->limbs = limbs; h->gap = gap; h->block_stride = block_stride;
    try {
      h->buf = fc_prepare(ctx->c, pts, out_dim, c_in * w_in, limbs);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

void he_ptset_free(he_ptset* pts) {
  if (pts && !handle_live(pts)) return;
  delete pts;
}

int he_fc_apply(he_ctx* ctx, const he_ctset* in, const he_ptset* pts, const double* bias, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    HANDLE(pts);
    REQUIRE(ctx && in && pts && out, HE_E_ARG, "null argument");
    REQUIRE(in->s->n == pts->n_in, HE_E_ARG, "input size does not match the prepared weights");
    REQUIRE(in->s->limbs == pts->limbs, HE_E_LEVEL, "input level does not match the prepared weights");
    *out = wrap(fc_apply(ctx->c, *in->s, pts->buf.p, pts->out_dim, pts->gap, pts->block_stride, bias));
  });
}

int he_fc_partial(he_ctx* ctx, const he_ctset* in, const he_ptset* pts, int first, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    HANDLE(pts);
    REQUIRE(ctx && in && pts && out, HE_E_ARG, "null argument");
    REQUIRE(first >= 0 && first + in->s->n <= pts->n_in, HE_E_ARG, "input columns outside the prepared weights");
    REQUIRE(in->s->limbs == pts->limbs, HE_E_LEVEL, "input level does not match the prepared weights");
    *out = wrap(fc_partial(ctx->c, *in->s, pts->buf.p, pts->out_dim, pts->n_in, first));
  });
}

int he_fc_finish(he_ctx* ctx, const he_ctset* sums, const he_ptset* pts, const double* bias, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(sums);
    HANDLE(pts);
    REQUIRE(ctx && sums && pts && out, HE_E_ARG, "null argument");
    const CtSet& z = *sums->s;
    REQUIRE(z.n == pts->out_dim, HE_E_ARG, "one sum per output expected");
    REQUIRE(z.limbs == pts->limbs, HE_E_LEVEL, "sums at a level other than the prepared weights'");
    auto r = new_set(ctx->c, z.n, z.polys, z.limbs, z.scale);
    HE_CUDA(cudaMemcpyAsync(r->buf.p, z.buf.p, z.buf.words * 8, cudaMemcpyDeviceToDevice, ctx->c.stream));
    fc_finish(ctx->c, *r, pts->gap, pts->block_stride, bias);
    *out = wrap(std::move(r));
  });
}

int he_fc(he_ctx* ctx, const he_ctset* in, const double* W, const double* b, int out_dim, int c_in, int h_valid,
          int w_in, int gap, int block_stride, int batch, he_ctset** out) {
  he_ptset* pts = nullptr;
  if ((ctx && !handle_live(ctx)) || (in && !handle_live(in))) {
    set_last_error("invalid handle (unknown or freed)");
    return HE_E_ARG;
  }
  int rc = he_fc_prepare(ctx, W, out_dim, c_in, h_valid, w_in, gap, block_stride, batch, in ? in->s->limbs : 0, &pts);
  if (rc != HE_OK) return rc;
  rc = he_fc_apply(ctx, in, pts, b, out);
  he_ptset_free(pts);
  return rc;
}

// ---- the paper's single-ciphertext layout (virtual ciphertexts, Sec. III-C/D) ----
// an h x w matrix (row-major, doubles) replicated into every Hb x Wb block of a slot vector
static void vr_blocks(const std::vector<double>& mat, int h, int w, int Hb, int Wb, long S, double* z) {
  for (long b = 0; b < S / ((long)Hb * Wb); b++)
    for (int r = 0; r < h; r++)
      for (int c = 0; c < w; c++) z[b * Hb * Wb + (long)r * Wb + c] = mat[(size_t)r * w + c];
}

static void vr_check(const Ctx& C, int h, int w, int k, int Hb, int Wb) {
  const long S = (long)C.N / 2;
  if (h < 1 || w < 1 || k < 1 || k > h || k > w || Hb < h || Wb < w || (long)Hb * Wb > S)
    throw Error(HE_E_ARG, "image, kernel or block sizes do not fit");
}

int he_vr_encrypt_images(he_ctx* ctx, const double* px, int batch, int h, int w, int block_h, int block_w,
                         uint64_t ct_id_base, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && px && out && batch >= 1, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    vr_check(C, h, w, 1, block_h, block_w);
    const long S = (long)C.N / 2, per = S / ((long)block_h * block_w);
    const int n_ct = (int)((batch + per - 1) / per);
    std::vector<double> z((size_t)n_ct * S, 0.0);
    for (int b = 0; b < batch; b++) {
      const long base = (b / per) * S + (b % per) * block_h * block_w;
      for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) z[base + (long)r * block_w + c] = px[((size_t)b * h + r) * w + c];
    }
    *out = wrap(encrypt_slots(C, z, n_ct, ct_id_base));
  });
}

int he_vr_encrypt_kernels(he_ctx* ctx, const double* K, int k, double k0, int h, int w, int block_h, int block_w,
                          int limbs, uint64_t ct_id_base, he_ctset** kernels, he_ctset** bias) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && K && kernels && bias, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    vr_check(C, h, w, k, block_h, block_w);
    REQUIRE(limbs >= 3 && limbs <= C.L1, HE_E_LEVEL, "bad level");
    const long S = (long)C.N / 2;
    const int T = k * k;
    // Kernelspanner (Sec. III-C): for offset (r, c) the kernel tiled from (r, c) wherever a copy fits
    std::vector<double> z((size_t)T * S, 0.0);
    for (int r = 0; r < k; r++)
      for (int c = 0; c < k; c++) {
        std::vector<double> P((size_t)h * w, 0.0);
        for (int top = r; top + k <= h; top += k)
          for (int left = c; left + k <= w; left += k)
            for (int a = 0; a < k; a++)
              for (int b = 0; b < k; b++) P[(size_t)(top + a) * w + left + b] = K[a * k + b];
        vr_blocks(P, h, w, block_h, block_w, S, z.data() + (size_t)(r * k + c) * S);
      }
    const double ql = (double)C.q[limbs - 1];
    std::vector<int64_t> m((size_t)T * C.N);
    host_parallel((size_t)T, [&](size_t t) { encode_real(C, z.data() + t * S, (size_t)S, ql, m.data() + t * C.N); });
    auto ks = encrypt_coeffs(C, m.data(), T, limbs, ql, ct_id_base);
    // the initial accumulator of Alg. 4: k0 at every valid output position
    std::vector<double> B((size_t)h * w, 0.0), zb(S, 0.0);
    for (int r = 0; r + k <= h; r++)
      for (int c = 0; c + k <= w; c++) B[(size_t)r * w + c] = k0;
    vr_blocks(B, h, w, block_h, block_w, S, zb.data());
    std::vector<int64_t> mb(C.N);
    encode_real(C, zb.data(), (size_t)S, C.scale0, mb.data());
    auto bs = encrypt_coeffs(C, mb.data(), 1, limbs - 2, C.scale0, ct_id_base + (uint64_t)T);
    *kernels = wrap(std::move(ks));
    *bias = wrap(std::move(bs));
  });
}

int he_vr_conv2d_coeffs(he_ctx* ctx, const he_ctset* in, const he_ctset* kernels, const he_ctset* bias, int k,
                        int block_w, const int64_t* masks, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    HANDLE(kernels);
    HANDLE(bias);
    REQUIRE(ctx && in && kernels && bias && masks && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const int lp = in->s->limbs;
    REQUIRE(lp >= 3, HE_E_LEVEL, "the single-ciphertext convolution needs two levels");
    DevBuf m = fc_prepare(C, masks, 1, k * k, lp - 1);
    *out = wrap(vr_conv2d(C, *in->s, *kernels->s, *bias->s, k, block_w, m.p));
  });
}

int he_vr_conv2d(he_ctx* ctx, const he_ctset* in, const he_ctset* kernels, const he_ctset* bias, int h, int w, int k,
                 int block_h, int block_w, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    HANDLE(kernels);
    HANDLE(bias);
    REQUIRE(ctx && in && kernels && bias && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    vr_check(C, h, w, k, block_h, block_w);
    const int lp = in->s->limbs;
    REQUIRE(lp >= 3, HE_E_LEVEL, "the single-ciphertext convolution needs two levels");
    const long S = (long)C.N / 2;
    const int T = k * k;
    // Alg. 4's offset masks: (hth - r) mod k = 0, (wth - c) mod k = 0, hth + k <= h, wth + k <= w
    std::vector<double> z((size_t)T * S, 0.0);
    for (int r = 0; r < k; r++)
      for (int c = 0; c < k; c++) {
        std::vector<double> F((size_t)h * w, 0.0);
        for (int hth = r; hth + k <= h; hth += k)
          for (int wth = c; wth + k <= w; wth += k) F[(size_t)hth * w + wth] = 1.0;
        vr_blocks(F, h, w, block_h, block_w, S, z.data() + (size_t)(r * k + c) * S);
      }
    const double ql = (double)C.q[lp - 2];
    std::vector<int64_t> m((size_t)T * C.N);
    host_parallel((size_t)T, [&](size_t t) { encode_real(C, z.data() + t * S, (size_t)S, ql, m.data() + t * C.N); });
    DevBuf dm = fc_prepare(C, m.data(), 1, T, lp - 1);
    *out = wrap(vr_conv2d(C, *in->s, *kernels->s, *bias->s, k, block_w, dm.p));
  });
}

int he_vrot_coeffs(he_ctx* ctx, const he_ctset* in, int r, int img_len, const int64_t* masks, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && masks && out, HE_E_ARG, "null argument");
    const int lp = in->s->limbs;
    REQUIRE(lp >= 2, HE_E_LEVEL, "no level left for vRot");
    DevBuf m = fc_prepare(ctx->c, masks, 1, 2, lp);
    *out = wrap(vrot(ctx->c, *in->s, r, img_len, m.p));
  });
}

int he_vrot(he_ctx* ctx, const he_ctset* in, int r, int row_len, int img_len, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long S = (long)C.N / 2;
    REQUIRE(row_len >= 1 && S % row_len == 0 && img_len >= 1 && img_len <= row_len && r >= 0 && r < img_len,
            HE_E_ARG, "rows must tile the slots, images fit the rows and 0 <= r < img_len");
    const int lp = in->s->limbs;
    REQUIRE(lp >= 2, HE_E_LEVEL, "no level left for vRot");
    std::vector<double> z((size_t)2 * S, 0.0);
    for (long row = 0; row < S / row_len; row++)
      for (int j = 0; j < img_len; j++) z[(size_t)(j < img_len - r ? 0 : 1) * S + row * row_len + j] = 1.0;
    std::vector<int64_t> m((size_t)2 * C.N);
    for (int t = 0; t < 2; t++) encode_real(C, z.data() + (size_t)t * S, (size_t)S, (double)C.q[lp - 1], m.data() + t * C.N);
    DevBuf dm = fc_prepare(C, m.data(), 1, 2, lp);
    *out = wrap(vrot(C, *in->s, r, img_len, dm.p));
  });
}

int he_vr_encrypt_matrix_a(he_ctx* ctx, const double* A, int m, int n, uint64_t ct_id_base, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && A && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long S = (long)C.N / 2;
    REQUIRE(m >= 1 && n >= 1 && (long)m * n <= S, HE_E_ARG, "A does not fit one ciphertext");
    std::vector<double> z(S, 0.0);
    for (long t = 0; t < (long)m * n; t++) z[t] = A[t];  // tau_a: row-major
    *out = wrap(encrypt_slots(C, z, 1, ct_id_base));
  });
}

int he_vr_encrypt_matrix_b(he_ctx* ctx, const double* B, int n, int p, uint64_t ct_id_base, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && B && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long S = (long)C.N / 2;
    REQUIRE(n >= 1 && p >= 1 && S % n == 0 && (S / n) % p == 0, HE_E_ARG,
            "n must divide the slot count and p the number of rows");
    std::vector<double> z(S);
    for (long s = 0; s < S; s++) z[s] = B[(size_t)(s % n) * p + (s / n) % p];  // tau_b tiled over the ring
    *out = wrap(encrypt_slots(C, z, 1, ct_id_base));
  });
}

static std::unique_ptr<CtSet> vr_matmul_from_host(Ctx& C, const CtSet& A, const CtSet& Bb, int n, int p,
                                                  const int64_t* masks) {
  const int lp = A.limbs;
  if (lp < 4) throw Error(HE_E_LEVEL, "the single-ciphertext matmul needs three levels");
  DevBuf E = fc_prepare(C, masks, 1, 1, lp - 1);
  DevBuf F = fc_prepare(C, masks + C.N, 1, p, lp - 2);
  return vr_matmul(C, A, Bb, n, p, E.p, F.p);
}

int he_vr_matmul_coeffs(he_ctx* ctx, const he_ctset* A, const he_ctset* Bbar, int m, int n, int p, const int64_t* masks,
                        he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(A);
    HANDLE(Bbar);
    REQUIRE(ctx && A && Bbar && masks && out, HE_E_ARG, "null argument");
    REQUIRE(m >= 1 && (long)m * n <= (long)ctx->c.N / 2, HE_E_ARG, "bad shape");
    *out = wrap(vr_matmul_from_host(ctx->c, *A->s, *Bbar->s, n, p, masks));
  });
}

int he_vr_matmul(he_ctx* ctx, const he_ctset* A, const he_ctset* Bbar, int m, int n, int p, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(A);
    HANDLE(Bbar);
    REQUIRE(ctx && A && Bbar && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long S = (long)C.N / 2;
    REQUIRE(m >= 1 && (long)m * n <= S && p >= 1 && p <= n, HE_E_ARG, "bad shape");
    const int lp = A->s->limbs;
    REQUIRE(lp >= 4, HE_E_LEVEL, "the single-ciphertext matmul needs three levels");
    std::vector<double> z((size_t)(1 + p) * S, 0.0);
    for (int i = 0; i < m; i++) z[(size_t)i * n] = 1.0;  // SumColVec's column-0 mask
    for (int idx = 0; idx < p; idx++)
      for (int i = 0; i < m; i++) z[(size_t)(1 + idx) * S + (size_t)i * n + (i + idx) % p] = 1.0;  // Alg. 3's F
    std::vector<int64_t> m_((size_t)(1 + p) * C.N);
    host_parallel((size_t)(1 + p), [&](size_t t) {
      encode_real(C, z.data() + t * S, (size_t)S, (double)C.q[t == 0 ? lp - 2 : lp - 3], m_.data() + t * C.N);
    });
    *out = wrap(vr_matmul_from_host(C, *A->s, *Bbar->s, n, p, m_.data()));
  });
}

int he_reform_coeffs(he_ctx* ctx, const he_ctset* in, int gap, int h_valid, const int64_t* masks, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && masks && out, HE_E_ARG, "null argument");
    REQUIRE(gap >= 2 && h_valid >= 1, HE_E_ARG, "bad ReForm shape");
    Ctx& C = ctx->c;
    const int lp = in->s->limbs;
    REQUIRE(lp >= 2, HE_E_LEVEL, "no level left for ReForm");
    DevBuf m = fc_prepare(C, masks, 1, h_valid, lp);
    *out = wrap(reform(C, *in->s, gap, h_valid, m.p));
  });
}

int he_reform(he_ctx* ctx, const he_ctset* in, int gap, int h_valid, int block_stride, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    const long S = (long)C.N / 2;
    REQUIRE(gap >= 2 && h_valid >= 1 && pow2(block_stride) && block_stride <= S &&
                (long)gap * (h_valid - 1) < block_stride,
            HE_E_ARG, "rows do not fit the blocks");
    const int lp = in->s->limbs;
    REQUIRE(lp >= 2, HE_E_LEVEL, "no level left for ReForm");
    const double ql = (double)C.q[lp - 1];
    std::vector<int64_t> m((size_t)h_valid * C.N);
    host_parallel((size_t)h_valid, [&](size_t i) {
      std::vector<double> z(S, 0.0);
      for (long b = 0; b < S / block_stride; b++) z[b * block_stride + (long)i] = 1.0;
      encode_real(C, z.data(), (size_t)S, ql, m.data() + i * C.N);
    });
    DevBuf dm = fc_prepare(C, m.data(), 1, h_valid, lp);
    *out = wrap(reform(C, *in->s, gap, h_valid, dm.p));
  });
}

int he_pack_blocks(he_ctx* ctx, const he_ctset* const* sets, int n_sets, const he_ptset* masks, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(masks);
    REQUIRE(ctx && sets && masks && out && n_sets >= 1, HE_E_ARG, "null argument");
    for (int t = 0; t < n_sets; t++) HANDLE(sets[t]);
    REQUIRE(sets[0], HE_E_ARG, "null set");
    const CtSet& s0 = *sets[0]->s;
    std::vector<const u64*> xs;
    for (int t = 0; t < n_sets; t++) {
      REQUIRE(sets[t], HE_E_ARG, "null set");
      const CtSet& s = *sets[t]->s;
      REQUIRE(s.n == s0.n && s.polys == 2, HE_E_ARG, "sets of different sizes or three-component sets");
      REQUIRE(s.limbs == s0.limbs && s.scale == s0.scale, HE_E_SCALE, "sets at different levels or scales");
      xs.push_back(s.buf.p);
    }
    REQUIRE(masks->n_in == 1 && masks->out_dim >= n_sets && masks->limbs == s0.limbs, HE_E_ARG,
            "masks must be prepared as [n_sets][1] plaintexts at the sets' level");
    *out = wrap(pack_blocks(ctx->c, xs, s0.n, s0.limbs, s0.scale, masks->buf.p));
  });
}

int he_rotate(he_ctx* ctx, const he_ctset* in, const int32_t* steps, int n_steps, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && steps && out && n_steps >= 1, HE_E_ARG, "bad arguments");
    std::vector<long> st(steps, steps + n_steps);
    *out = wrap(rotate(ctx->c, *in->s, st));
  });
}

int he_mul(he_ctx* ctx, const he_ctset* a, const he_ctset* b, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(a);
    HANDLE(b);
    REQUIRE(ctx && a && b && out, HE_E_ARG, "null argument");
    *out = wrap(mul(ctx->c, *a->s, *b->s));
  });
}

int he_rescale(he_ctx* ctx, he_ctset* inout) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(inout);
    REQUIRE(ctx && inout, HE_E_ARG, "null argument");
    REQUIRE(!ctx->c.capturing || inout->s->gen == ctx->c.capture_gen, HE_E_STATE,
            "in-place operation on a set made before the capture");
    rescale_inplace(ctx->c, *inout->s);
  });
}

int he_add(he_ctx* ctx, const he_ctset* a, const he_ctset* b, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(a);
    HANDLE(b);
    REQUIRE(ctx && a && b && out, HE_E_ARG, "null argument");
    *out = wrap(add(ctx->c, *a->s, *b->s));
  });
}

int he_decrypt_slots(he_ctx* ctx, const he_ctset* in, double* out, size_t out_len) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && out, HE_E_ARG, "null argument");
    REQUIRE(out_len >= (size_t)in->s->n * (ctx->c.N / 2), HE_E_ARG, "output too small");
    decrypt_slots(ctx->c, *in->s, out);
  });
}

int he_decrypt_matrix(he_ctx* ctx, const he_ctset* Cs, int m, int p, double* C_out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(Cs);
    REQUIRE(ctx && Cs && C_out, HE_E_ARG, "null argument");
    REQUIRE(Cs->s->n == p && m >= 1 && (size_t)m <= ctx->c.N / 2, HE_E_ARG, "shape does not match");
    const size_t M = ctx->c.N / 2;
    std::vector<double> z((size_t)p * M);
    decrypt_slots(ctx->c, *Cs->s, z.data());
    for (int idx = 0; idx < p; idx++)
      for (int i = 0; i < m; i++) C_out[(size_t)i * p + (i + idx) % p] = z[(size_t)idx * M + i];
  });
}

int he_decrypt_matrix_volley(he_ctx* ctx, const he_ctset* Cs, int m, int p, double* C_out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(Cs);
    REQUIRE(ctx && Cs && C_out, HE_E_ARG, "null argument");
    const long S = (long)ctx->c.N / 2;
    int Mb, per, G;
    volley_geometry(S, m, p, Mb, per, G);
    REQUIRE(Cs->s->n == G, HE_E_ARG, "shape does not match");
    std::vector<double> z((size_t)G * S);
    decrypt_slots(ctx->c, *Cs->s, z.data());
    for (int g = 0; g < G; g++) {
      const long o = ((long)g * per) % p;
      for (int t = 0; t < per && g * per + t < p; t++) {
        const int idx = g * per + t;
        for (int i = 0; i < m; i++) C_out[(size_t)i * p + (i + idx) % p] = z[(size_t)g * S + (size_t)t * Mb + o + i];
      }
    }
  });
}

int he_decrypt_image(he_ctx* ctx, const he_ctset* in, int batch, int block_stride, int gap, int h_valid, double* out,
                     size_t out_len) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && out, HE_E_ARG, "null argument");
    const size_t M = ctx->c.N / 2;
    const int n = in->s->n;
    REQUIRE(batch >= 1 && h_valid >= 1 && gap >= 1 && (size_t)batch * block_stride <= M &&
                (long)gap * (h_valid - 1) < block_stride,
            HE_E_ARG, "layout does not fit");
    REQUIRE(out_len >= (size_t)batch * n * h_valid, HE_E_ARG, "output too small");
    std::vector<double> z((size_t)n * M);
    decrypt_slots(ctx->c, *in->s, z.data());
    for (int b = 0; b < batch; b++)
      for (int c = 0; c < n; c++)
        for (int i = 0; i < h_valid; i++)
          out[((size_t)b * n + c) * h_valid + i] = z[(size_t)c * M + (size_t)b * block_stride + (size_t)gap * i];
  });
}

int he_ctset_export(const he_ctset* set, uint64_t* host, size_t n_words) {
  return guard([&] {
    HANDLE(set);
    REQUIRE(set && host, HE_E_ARG, "null argument");
    REQUIRE(n_words >= set->s->buf.words, HE_E_ARG, "output too small");
    export_coeffs(*set->s->ctx, *set->s, host);
  });
}

int he_ctset_export_async(const he_ctset* set, uint64_t* host, size_t n_words, uint64_t* ticket) {
  return guard([&] {
    HANDLE(set);
    REQUIRE(set && host && ticket, HE_E_ARG, "null argument");
    REQUIRE(n_words >= set->s->buf.words, HE_E_ARG, "output too small");
    *ticket = export_async(*set->s->ctx, *set->s, host);
  });
}

int he_ctset_export_wait(he_ctx* ctx, uint64_t ticket) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null context");
    export_wait(ctx->c, ticket);
  });
}

int he_ctset_import(he_ctx* ctx, const uint64_t* host, int n, int limbs, double scale, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && host && out, HE_E_ARG, "null argument");
    *out = wrap(import_coeffs(ctx->c, host, n, limbs, scale));
  });
}

int he_debug_wait_timeout(he_ctx* ctx, int limit_us) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null context");
    REQUIRE(limit_us >= 1 && limit_us <= 2000000, HE_E_ARG, "limit outside 1 .. 2,000,000 us");
    k_wait_expires(ctx->c, (uint64_t)limit_us * 1000);
  });
}

int he_debug_fail_allocations(int n) {
  return guard([&] {
    REQUIRE(n >= 0, HE_E_ARG, "n must be >= 0");
    g_fail_allocs.store(n);
  });
}

int he_ctx_set_tensor_cores(he_ctx* ctx, int on) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null context");
    ctx->c.use_tc = on != 0;
  });
}

int he_ctx_set_work_budget(he_ctx* ctx, size_t bytes) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null context");
    ctx->c.work_budget = bytes;
  });
}

int he_ctset_import_async(he_ctx* ctx, const uint64_t* host, int n, int limbs, double scale, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && host && out, HE_E_ARG, "null argument");
    REQUIRE(scale > 0, HE_E_ARG, "scale must be positive");
    *out = wrap(import_async(ctx->c, host, n, limbs, scale));
  });
}

int he_ctset_export_raw(const he_ctset* set, uint64_t* host, size_t n_words) {
  return guard([&] {
    HANDLE(set);
    REQUIRE(set && host, HE_E_ARG, "null argument");
    REQUIRE(n_words >= set->s->buf.words, HE_E_ARG, "output too small");
    export_raw(*set->s->ctx, *set->s, host);
  });
}

int he_ctset_import_raw(he_ctx* ctx, const uint64_t* host, int n, int limbs, double scale, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && host && out, HE_E_ARG, "null argument");
    *out = wrap(import_coeffs(ctx->c, host, n, limbs, scale, true));
  });
}

int he_ctset_export_words(const he_ctset* set, uint64_t* dst, int dst_on_device, size_t n_words) {
  return guard([&] {
    HANDLE(set);
    REQUIRE(set && dst, HE_E_ARG, "null argument");
    REQUIRE(n_words >= set->s->buf.words, HE_E_ARG, "output too small");
    export_words(*set->s->ctx, *set->s, dst, dst_on_device != 0);
  });
}

int he_ctset_import_words(he_ctx* ctx, const uint64_t* src, int src_on_device, int n, int polys, int limbs,
                          double scale, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && src && out, HE_E_ARG, "null argument");
    REQUIRE(scale > 0, HE_E_ARG, "scale must be positive");
    *out = wrap(import_words(ctx->c, src, src_on_device != 0, n, polys, limbs, scale));
  });
}

int he_ctset_info(const he_ctset* set, int* n_ct, int* limbs, double* scale, int* polys) {
  return guard([&] {
    HANDLE(set);
    REQUIRE(set, HE_E_ARG, "null set");
    if (n_ct) *n_ct = set->s->n;
    if (limbs) *limbs = set->s->limbs;
    if (scale) *scale = set->s->scale;
    if (polys) *polys = set->s->polys;
  });
}

int he_ctset_drop_levels(he_ctx* ctx, const he_ctset* in, int limbs, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(in);
    REQUIRE(ctx && in && out, HE_E_ARG, "null argument");
    REQUIRE(limbs >= 1 && limbs <= in->s->limbs, HE_E_LEVEL, "the target level must keep 1 .. limbs primes");
    *out = wrap(drop_limbs(ctx->c, *in->s, limbs));
  });
}

int he_add_plain_coeffs(he_ctx* ctx, he_ctset* inout, const int64_t* m, int n_vec) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(inout);
    REQUIRE(ctx && inout && m, HE_E_ARG, "null argument");
    REQUIRE(n_vec == 1 || n_vec == inout->s->n, HE_E_ARG, "one plaintext, or one per ciphertext");
    REQUIRE(!ctx->c.capturing || inout->s->gen == ctx->c.capture_gen, HE_E_STATE,
            "in-place operation on a set made before the capture");
    add_plain(ctx->c, *inout->s, m, n_vec);
  });
}

int he_add_slots(he_ctx* ctx, he_ctset* inout, const double* v, int n_vec) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(inout);
    REQUIRE(ctx && inout && v, HE_E_ARG, "null argument");
    REQUIRE(n_vec == 1 || n_vec == inout->s->n, HE_E_ARG, "one slot vector, or one per ciphertext");
    REQUIRE(!ctx->c.capturing || inout->s->gen == ctx->c.capture_gen, HE_E_STATE,
            "in-place operation on a set made before the capture");
    Ctx& C = ctx->c;
    const size_t M = C.N / 2;
    std::vector<int64_t> m((size_t)n_vec * C.N);
    for (int k = 0; k < n_vec; k++) encode_real(C, v + (size_t)k * M, M, inout->s->scale, m.data() + (size_t)k * C.N);
    add_plain(C, *inout->s, m.data(), n_vec);
  });
}

int he_relinearize(he_ctx* ctx, he_ctset* inout) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(inout);
    REQUIRE(ctx && inout, HE_E_ARG, "null argument");
    REQUIRE(!ctx->c.capturing || inout->s->gen == ctx->c.capture_gen, HE_E_STATE,
            "in-place operation on a set made before the capture");
    relinearize(ctx->c, *inout->s);
  });
}

int he_ctset_device_ptr(const he_ctset* set, uint64_t** dptr) {
  return guard([&] {
    HANDLE(set);
    REQUIRE(set && dptr, HE_E_ARG, "null argument");
    *dptr = set->s->buf.p;
  });
}

int he_ctset_slice(he_ctx* ctx, const he_ctset* set, int first, int n, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(set);
    REQUIRE(ctx && set && out, HE_E_ARG, "null argument");
    const CtSet& s = *set->s;
    REQUIRE(first >= 0 && n >= 1 && first + n <= s.n, HE_E_ARG, "slice out of range");
    auto r = new_set(ctx->c, n, s.polys, s.limbs, s.scale);
    HE_CUDA(cudaMemcpyAsync(r->buf.p, s.ct(first), (size_t)n * s.ct_words() * 8, cudaMemcpyDeviceToDevice,
                            ctx->c.stream));  // any component count
    *out = wrap(std::move(r));
  });
}

int he_ctset_concat(he_ctx* ctx, const he_ctset* const* sets, int n_sets, he_ctset** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && sets && out && n_sets >= 1, HE_E_ARG, "null argument");
    for (int i = 0; i < n_sets; i++) HANDLE(sets[i]);
    REQUIRE(sets[0], HE_E_ARG, "null set");
    int total = 0;
    for (int i = 0; i < n_sets; i++) {
      REQUIRE(sets[i], HE_E_ARG, "null set");
      REQUIRE(sets[i]->s->limbs == sets[0]->s->limbs && sets[i]->s->polys == sets[0]->s->polys, HE_E_LEVEL,
              "sets at different levels");
      REQUIRE(sets[i]->s->scale == sets[0]->s->scale, HE_E_SCALE, "sets at different scales");
      total += sets[i]->s->n;
    }
    const CtSet& s0 = *sets[0]->s;
    auto r = new_set(ctx->c, total, s0.polys, s0.limbs, s0.scale);
    size_t off = 0;
    for (int i = 0; i < n_sets; i++) {
      const size_t w = sets[i]->s->buf.words;
      HE_CUDA(cudaMemcpyAsync(r->buf.p + off, sets[i]->s->buf.p, w * 8, cudaMemcpyDeviceToDevice, ctx->c.stream));
      off += w;
    }
    *out = wrap(std::move(r));
  });
}

void he_ctset_free(he_ctset* set) {
  if (set && !handle_live(set)) return;
  if (!set) return;
  Ctx* C = set->s ? set->s->ctx : nullptr;
  if (C && C->capturing && set->s->gen != C->capture_gen) {
    // made before the capture: its memory is not the graph's to free; release it after the capture
    C->deferred.push_back(std::move(set->s));
  }
  delete set;
}

int he_graph_begin(he_ctx* ctx) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    REQUIRE(!C.capturing, HE_E_STATE, "a capture is already open on this context");
    REQUIRE(C.stream != nullptr, HE_E_STATE, "graphs need a non-default context stream");
    HE_CUDA(cudaStreamSynchronize(C.stream));
    HE_CUDA(cudaStreamBeginCapture(C.stream, cudaStreamCaptureModeThreadLocal));
    C.capturing = true;
    C.capture_failed = false;
    C.capture_gen++;
  });
}

int he_graph_end(he_ctx* ctx, he_graph** out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && out, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    REQUIRE(C.capturing, HE_E_STATE, "no capture is open on this context");
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(C.stream, &g);
    C.capturing = false;
    C.deferred.clear();  // sets made before the capture and freed during it
    if (e == cudaSuccess && C.capture_failed) {
      if (g) cudaGraphDestroy(g);
      throw Error(HE_E_CUDA, "capture failed: a call inside it copies host data to the device");
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      throw Error(HE_E_CUDA, std::string("capture failed (a call inside it is not capturable): ") +
                                 cudaGetErrorString(e));
    }
    auto* h = new he_graph;
    h->ctx = ctx;
    h->graph = g;
    const cudaError_t ei = cudaGraphInstantiateWithFlags(&h->exec, g, cudaGraphInstantiateFlagAutoFreeOnLaunch);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      delete h;
      throw Error(HE_E_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ei));
    }
    size_t nn = 0;
    HE_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) HE_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      HE_CUDA(cudaGraphNodeGetType(nd, &t));
      h->kernels += t == cudaGraphNodeTypeKernel;
    }
    *out = h;
  });
}

int he_graph_launch(he_graph* g) {
  return guard([&] {
    HANDLE(g);
    REQUIRE(g && g->exec, HE_E_ARG, "null graph");
    Ctx& C = g->ctx->c;
    REQUIRE(!C.capturing, HE_E_STATE, "a capture is open on this context");
    HE_CUDA(cudaGraphLaunch(g->exec, C.stream));
    prof_add_launches(g->kernels);
  });
}

int he_graph_info(const he_graph* g, uint64_t* kernel_nodes) {
  return guard([&] {
    HANDLE(g);
    REQUIRE(g && kernel_nodes, HE_E_ARG, "null argument");
    *kernel_nodes = g->kernels;
  });
}

void he_graph_destroy(he_graph* g) {
  if (g && !handle_live(g)) return;
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

int he_ctset_assign(he_ctx* ctx, he_ctset* dst, const he_ctset* src) {
  return guard([&] {
    HANDLE(ctx);
    HANDLE(dst);
    HANDLE(src);
    REQUIRE(ctx && dst && src, HE_E_ARG, "null argument");
    const CtSet& a = *src->s;
    CtSet& b = *dst->s;
    REQUIRE(a.n == b.n && a.polys == b.polys && a.limbs == b.limbs, HE_E_ARG, "sets of different shapes");
    REQUIRE(!ctx->c.capturing || b.gen == ctx->c.capture_gen, HE_E_STATE,
            "a set made before the capture cannot be overwritten inside it");
    HE_CUDA(cudaMemcpyAsync(b.buf.p, a.buf.p, a.buf.words * 8, cudaMemcpyDeviceToDevice, ctx->c.stream));
    b.scale = a.scale;
  });
}

int he_calibrate_modmul(he_ctx* ctx, double* modmul_per_s) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && modmul_per_s, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    int sms = 0;
    HE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C.device));
    const int threads = 256, blocks = sms * 8, iters = 4096;
    DevBuf sink((size_t)blocks * threads, C.stream);
    k_calib_shoup(C, sink.p, blocks, threads, 64);  // warm-up
    cudaEvent_t a, b;
    HE_CUDA(cudaEventCreate(&a));
    HE_CUDA(cudaEventCreate(&b));
    HE_CUDA(cudaEventRecord(a, C.stream));
    k_calib_shoup(C, sink.p, blocks, threads, iters);
    HE_CUDA(cudaEventRecord(b, C.stream));
    HE_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    HE_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *modmul_per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
  });
}

int he_calibrate_mac96(he_ctx* ctx, double* mac_per_s) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && mac_per_s, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    int sms = 0;
    HE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C.device));
    const int threads = 256, blocks = sms * 8, iters = 4096;
    DevBuf sink((size_t)blocks * threads, C.stream);
    k_calib_mac96(C, sink.p, blocks, threads, 64);  // warm-up
    cudaEvent_t a, b;
    HE_CUDA(cudaEventCreate(&a));
    HE_CUDA(cudaEventCreate(&b));
    HE_CUDA(cudaEventRecord(a, C.stream));
    k_calib_mac96(C, sink.p, blocks, threads, iters);
    HE_CUDA(cudaEventRecord(b, C.stream));
    HE_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    HE_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *mac_per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
  });
}

int he_calibrate_butterfly(he_ctx* ctx, int narrow, double* bfly_per_s) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && bfly_per_s, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    int sms = 0;
    HE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C.device));
    const int threads = 256, blocks = sms * 8, iters = 4096;
    DevBuf sink((size_t)blocks * threads, C.stream);
    k_calib_bfly(C, sink.p, blocks, threads, 64, narrow != 0);  // warm-up
    cudaEvent_t a, b;
    HE_CUDA(cudaEventCreate(&a));
    HE_CUDA(cudaEventCreate(&b));
    HE_CUDA(cudaEventRecord(a, C.stream));
    k_calib_bfly(C, sink.p, blocks, threads, iters, narrow != 0);
    HE_CUDA(cudaEventRecord(b, C.stream));
    HE_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    HE_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *bfly_per_s = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
  });
}

int he_ntt_set_geometry(he_ctx* ctx, int n1, int cols) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx, HE_E_ARG, "null argument");
    Ctx& C = ctx->c;
    if (n1 == 0 && cols == 0) {
      C.ntt_n1 = C.ntt_cols = 0;
      return;
    }
    REQUIRE(ntt_geometry_ok(C.log_n, n1, cols), HE_E_ARG, "unsupported transform geometry");
    C.ntt_n1 = n1;
    C.ntt_cols = cols;
  });
}

int he_ntt_autotune(he_ctx* ctx, int rows, int* n1_out, int* cols_out, double* us_out) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && rows >= 1, HE_E_ARG, "bad arguments");
    Ctx& C = ctx->c;
    REQUIRE(!C.capturing, HE_E_STATE, "a capture is open on this context");
    const int lp = C.L1;
    const int polys = (rows + lp - 1) / lp;
    DevBuf d((size_t)polys * lp * C.N, C.stream);
    HE_CUDA(cudaMemsetAsync(d.p, 0, d.words * 8, C.stream));
    const LimbMap lm = limbs_q(lp, C.N);
    cudaEvent_t e0, e1;
    HE_CUDA(cudaEventCreate(&e0));
    HE_CUDA(cudaEventCreate(&e1));
    const int saved_n1 = C.ntt_n1, saved_cols = C.ntt_cols;
    double best = 1e30;
    int bn1 = 0, bc = 0;
    try {
      for (int n1 = 2; n1 <= 8; n1++)
        for (int cols = 4; cols <= 32; cols *= 2) {
          if (!ntt_geometry_ok(C.log_n, n1, cols)) continue;
          C.ntt_n1 = n1;
          C.ntt_cols = cols;
          ntt_forward(C, d.p, polys, lm);  // warm-up (and the one-time shared-memory opt-in)
          ntt_inverse(C, d.p, polys, lm);
          constexpr int reps = 3;
          HE_CUDA(cudaEventRecord(e0, C.stream));
          for (int r = 0; r < reps; r++) {
            ntt_forward(C, d.p, polys, lm);
            ntt_inverse(C, d.p, polys, lm);
          }
          HE_CUDA(cudaEventRecord(e1, C.stream));
          HE_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          HE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          const double us = 1e3 * ms / reps;
          if (us < best) {
            best = us;
            bn1 = n1;
            bc = cols;
          }
        }
    } catch (...) {
      C.ntt_n1 = saved_n1;
      C.ntt_cols = saved_cols;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    REQUIRE(bn1 > 0, HE_E_UNIMPL, "no transform geometry for this ring degree");
    C.ntt_n1 = bn1;
    C.ntt_cols = bc;
    if (n1_out) *n1_out = bn1;
    if (cols_out) *cols_out = bc;
    if (us_out) *us_out = best;
  });
}

int he_ntt(he_ctx* ctx, uint64_t* host, int n_polys, int limbs, int first_prime, int inverse) {
  return guard([&] {
    HANDLE(ctx);
    REQUIRE(ctx && host && n_polys >= 1 && limbs >= 1, HE_E_ARG, "bad arguments");
    Ctx& C = ctx->c;
    REQUIRE(first_prime >= 0 && first_prime + limbs <= C.np(), HE_E_ARG, "prime range out of bounds");
    const size_t words = (size_t)n_polys * limbs * C.N;
    for (size_t idx = 0; idx < words; idx++)
      REQUIRE(host[idx] < C.q[first_prime + (int)((idx / C.N) % limbs)], HE_E_ARG, "residue out of range");
    DevBuf d(words, C.stream);
    HE_CUDA(cudaMemcpyAsync(d.p, host, words * 8, cudaMemcpyHostToDevice, C.stream));
    LimbMap lm;
    lm.lpp = limbs; lm.split = limbs; lm.base0 = first_prime; lm.base1 = 0; lm.poly_stride = (size_t)limbs * C.N;
    if (inverse) ntt_inverse(C, d.p, n_polys, lm);
    else ntt_forward(C, d.p, n_polys, lm);
    HE_CUDA(cudaMemcpyAsync(host, d.p, words * 8, cudaMemcpyDeviceToHost, C.stream));
    HE_CUDA(cudaStreamSynchronize(C.stream));
  });
}

}  // extern "C"
