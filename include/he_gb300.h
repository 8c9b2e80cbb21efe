/*
 * he_gb300.h - C ABI of the GB300 (sm_103a) RNS-CKKS engine for encrypted
 * matrix multiplication and convolution over the multi-ciphertext layouts of
 * "Volley Revolver: A Novel Matrix-Encoding Method for Privacy-Preserving
 * Deep Learning (Inference++)" (arXiv 2512.18646).
 *
 * The paper (Sec. II-A) uses the CKKS primitives Enc, Dec, Add, Mul, cMul and
 * Rot, and (abstract, Sec. I-C) encrypts an m x n by n x p matrix product as n
 * ciphertexts per operand and an h x w image as w ciphertexts of h column
 * pixels. This library evaluates those layouts with RNS-CKKS on the GPU:
 * negacyclic NTTs over word-size primes, hybrid key switching with keys
 * resident in device memory, and rescaling after every multiplication.
 *
 * Conventions for every entry point:
 *  - Return value: HE_OK (0) or one of the HE_E_* codes below. On error the
 *    outputs are left unset (no partially built handle is returned) and
 *    he_last_error() gives a message for the calling thread.
 *  - Handles (he_ctx, he_ctset, he_ptset) are created and owned by
 *    the library; release them with the matching *_free / *_destroy call.
 *    Destroying a context invalidates every handle made from it.
 *  - Pointer arguments without further note are HOST pointers, borrowed for
 *    the duration of the call. Arrays are C-contiguous, row-major.
 *  - Work is enqueued on the context's CUDA stream. Calls that return host
 *    data (decrypt, export, info that needs device state) synchronise that
 *    stream; the others may return before the GPU finishes.
 *  - A ciphertext set (he_ctset) is n ciphertexts at one level (number of Q
 *    limbs) and one scale, held in device memory in the NTT domain as
 *    [n][2][limbs][N] 64-bit residues.
 *  - Rotation steps follow Rot(ct, l) of Sec. II-A: a left rotation of the
 *    N/2 slots by l.
 */
#ifndef HE_GB300_H
#define HE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HE_OK 0
#define HE_E_ARG 1      /* invalid argument (size, shape, null pointer)        */
#define HE_E_LEVEL 2    /* not enough levels left for the operation            */
#define HE_E_NOKEY 3    /* a needed rotation key was not generated             */
#define HE_E_SCALE 4    /* operands at different scales or levels              */
#define HE_E_OOM 5      /* device allocation failed                            */
#define HE_E_TIMEOUT 6  /* a bounded wait expired                              */
#define HE_E_CUDA 7     /* a CUDA call failed                                  */
#define HE_E_UNIMPL 8   /* operation not supported for these arguments         */
#define HE_E_STATE 9    /* handle in the wrong state (e.g. no keys yet)        */

typedef struct he_ctx he_ctx;       /* parameters, NTT tables, keys, stream      */
typedef struct he_ctset he_ctset;   /* n ciphertexts at one level and scale      */
typedef struct he_ptset he_ptset;   /* encoded plaintexts prepared on the device */
typedef struct he_graph he_graph;   /* a captured sequence of library calls       */

/*
 * Scheme parameters. Primes: the n_special primes of P take the largest
 * special_bits-bit values of the form 2^b - t 2N + 1 (t = 1, 2, ...) that are
 * prime; then q_0, q_1, ..., q_L take, in order, the largest unused such
 * prime of q_bits[i] bits. Key switching uses digits of `alpha` consecutive
 * Q primes (dnum = ceil(n_q / alpha) digits at the top level).
 */
typedef struct {
  int log_n;           /* ring degree N = 2^log_n, 4 <= log_n <= 16           */
  int n_q;             /* number of Q primes (levels + 1), 1..32             */
  const int* q_bits;   /* n_q bit sizes, each in [20, 61]                     */
  int n_special;       /* K special primes, 1..8                              */
  int special_bits;    /* bit size of each special prime, in [20, 61]         */
  int alpha;           /* primes per key-switching digit, 1..8                */
  double log_scale;    /* encoding scale = 2^log_scale                        */
  double sigma;        /* Gaussian error parameter (3.2)                      */
} he_params_desc;

/*
 * he_ctx_create: build the prime chain, the NTT tables and the constants of
 * base conversion and rescaling, on the GPU that is current for the calling
 * thread. `seed` names every random stream keygen and encryption draw
 * (inputs/he_random.h). `cuda_stream` is a cudaStream_t or NULL for the
 * default stream. Errors: HE_E_ARG on invalid parameters, HE_E_CUDA /
 * HE_E_OOM on device failures.
 */
int he_ctx_create(const he_params_desc* desc, uint64_t seed, void* cuda_stream, he_ctx** out);
/*
 * he_ctx_destroy: wait for the context's stream, free its keys, tables and
 * staging buffers, then return the unused part of the device's default memory
 * pool to the driver (a context keeps freed pool memory cached while it lives;
 * memory still held by other contexts' ciphertexts is not touched). A null or
 * already destroyed handle is ignored.
 */
void he_ctx_destroy(he_ctx* ctx);

/* Block until all work enqueued on the context's stream has finished. */
int he_ctx_synchronize(he_ctx* ctx);

/* The n_q + n_special primes, Q then P, into out[n] (n >= their count). */
int he_ctx_primes(const he_ctx* ctx, uint64_t* out, int n);

/* Ring degree exponent, prime counts, digit size, scale. Any pointer may be NULL. */
int he_ctx_info(const he_ctx* ctx, int* log_n, int* n_q, int* n_special, int* alpha, double* scale);

/* Bound, in bytes, on the device temporaries of one convolution,
 * relinearisation, ciphertext product or rescale: larger sets are processed
 * in chunks of ciphertexts (convolutions: of output columns, with the input
 * columns each chunk needs) with the same per-ciphertext arithmetic, so the
 * results do not change. 0 (the default) means no bound. */
int he_ctx_set_work_budget(he_ctx* ctx, size_t bytes);

/*
 * Whether the convolution's ciphertext-scalar multiply-accumulate (Alg. 4's
 * sum over channels and kernel offsets, he_conv2d) runs on the tensor cores
 * (on != 0, the default) or on the CUDA cores. The tensor-core form splits
 * the residues into chunks (bytes for primes below 2^46, 7 bits above) whose
 * products the tensor cores sum exactly in fp32 and recombines the sums modulo
 * q; it is taken where those sums stay below 2^24 (c_in k^2 up to 85 terms
 * below 2^46, 115 above), the weight tiles fit shared memory, the layer has
 * at least 128 products per output column and coefficient (c_in k^2 c_out; the
 * CUDA cores are faster below) and N >= 128. Both forms compute the same
 * words. Errors: HE_E_ARG.
 */
int he_ctx_set_tensor_cores(he_ctx* ctx, int on);

/*
 * he_keygen: draw the ternary secret s, the public key (-a s + e, a) over Q,
 * the relinearisation key (s^2 -> s) and one Galois key per rotation step
 * (phi_{5^l}(s) -> s), as hybrid key-switching keys over Q*P (Sec. II-A says
 * the library provides these keys). All keys stay in device memory. The
 * secret is kept in the context for decryption (the context is the key
 * owner's). Steps are reduced mod N/2; 0 is ignored. May be called again to
 * add rotation keys. Errors: HE_E_ARG, HE_E_OOM, HE_E_CUDA.
 */
int he_keygen(he_ctx* ctx, const int32_t* rot_steps, int n_steps);

/*
 * he_keys_export: a checkpoint of the context's keys in n_words 64-bit words
 * (host memory, caller-owned): a header with the ring degree, the prime chain
 * and the digit size, then the secret and public keys and every switching key
 * (relinearisation and Galois keys), coefficient words in the NTT domain.
 * *needed (may be NULL) gets the size; words == NULL only asks for it.
 * A client keeps its secret: strip it before handing keys to a server. The
 * paper has no counterpart (it assumes the keys exist, Sec. II-A).
 * Errors: HE_E_STATE (no keys), HE_E_ARG (output too small).
 *
 * he_keys_import: load such a checkpoint into a context made with the same
 * parameters (ring degree, primes, special primes, digits), replacing its
 * keys; ciphertexts of the exporting context then decrypt and rotate here.
 * The words are checked (header, primes, sizes, residues below their
 * primes). Errors: HE_E_ARG (other parameters, malformed or truncated).
 */
int he_keys_export(he_ctx* ctx, uint64_t* words, size_t n_words, size_t* needed);
int he_keys_import(he_ctx* ctx, const uint64_t* words, size_t n_words);

/* ---- encryption into the paper's layouts (Enc_pk, Sec. II-A) ---- */

/*
 * he_encrypt_image: column-wise image layout (abstract; Sec. I-C). px is
 * [batch][h][w] doubles. Output: w ciphertexts at the top level and scale
 * 2^log_scale; ciphertext j holds column j, image b's row i at slot
 * b * block_stride + i. block_stride is a power of two >= h with
 * batch * block_stride <= N/2 (one image per block, the virtual ciphertexts
 * of Sec. III-D). Ciphertext ids (the randomness streams) are ct_id_base + j.
 */
int he_encrypt_image(he_ctx* ctx, const double* px, int batch, int h, int w, int block_stride,
                     uint64_t ct_id_base, he_ctset** out);

/* A [m][n] -> n ciphertexts; ciphertext k holds column k of A at slots i < m
 * (abstract; Sec. I-C: n ciphertexts per operand). Ids ct_id_base + k. */
int he_encrypt_matrix_a(he_ctx* ctx, const double* A, int m, int n, uint64_t ct_id_base, he_ctset** out);

/* B [n][p] -> n ciphertexts; ciphertext k holds row k of B tiled with period p
 * over every slot (the tiling of tau_b, Sec. III-A). p must divide N/2. */
int he_encrypt_matrix_b(he_ctx* ctx, const double* B, int n, int p, uint64_t ct_id_base, he_ctset** out);

/*
 * he_volley_geometry: the zero-rotation ("volley") layout of an m x n by n x p
 * product on `slots` slots. B stays as he_encrypt_matrix_b encodes it (row k
 * tiled with period p, so slot s holds B[k][s mod p]); A's column k is copied to
 * blocks starting at t * M + o_g, with M >= m and M = 1 (mod p), so slot
 * t * M + o_g + i pairs A[i][k] with B[k][(i + g * per + t) mod p]: position
 * idx = g * per + t of the revolver of Alg. 3 (Sec. III-B), without rotating.
 * Outputs: *M the block stride, *per the positions one ciphertext holds
 * (t < per), *groups = ceil(p / per) ciphertexts per column of A; group g
 * starts at block offset o_g = (g * per) mod p. Host-only arithmetic.
 * Errors: HE_E_ARG if p does not divide `slots` or m + p - 1 > slots.
 */
int he_volley_geometry(int slots, int m, int p, int* M, int* per, int* groups);

/*
 * he_encrypt_matrix_a_volley: A [m][n] -> groups * n ciphertexts, group-major
 * ([g][k]), in the layout of he_volley_geometry for this p (slots = N/2): group
 * g, column k holds A[i][k] at slots t * M + o_g + i for t < min(per, p - g *
 * per), i < m, zero elsewhere. Ids ct_id_base + g * n + k.
 */
int he_encrypt_matrix_a_volley(he_ctx* ctx, const double* A, int m, int n, int p, uint64_t ct_id_base,
                               he_ctset** out);

/*
 * he_encrypt_coeffs: encrypt already-encoded plaintexts. m is [n_ct][N]
 * signed integer coefficients; the result has `limbs` Q limbs and the given
 * scale. Ciphertext i uses randomness id ct_id_base + i. Used to start two
 * implementations from the same integer plaintexts.
 */
int he_encrypt_coeffs(he_ctx* ctx, const int64_t* m, int n_ct, int limbs, double scale, uint64_t ct_id_base,
                      he_ctset** out);

/* ---- evaluation (all operands in device memory) ---- */

/*
 * he_matmul: encrypted C = A B (Alg. 3 over n ciphertexts per operand, Sec.
 * IV-A). A from he_encrypt_matrix_a (m x n), B from he_encrypt_matrix_b
 * (n x p), same level and scale. Result: p ciphertexts at one level lower;
 * ciphertext idx holds C[i][(i + idx) mod p] at slot i < m (decode with
 * he_decrypt_matrix). Needs rotation keys for steps 1..p-1.
 * Errors: HE_E_ARG (shape), HE_E_SCALE, HE_E_LEVEL, HE_E_NOKEY.
 */
int he_matmul(he_ctx* ctx, const he_ctset* A, const he_ctset* B, int m, int p, he_ctset** C);

/*
 * he_matmul_range: the diagonals idx_lo <= idx < idx_hi of he_matmul's result
 * (idx_hi - idx_lo ciphertexts, ciphertext t equal to he_matmul's ciphertext
 * idx_lo + t, word for word). Sec. IV-A splits the product across the columns
 * of B, one diagonal per worker; this is one worker's share, so that a matmul
 * can be sharded over GPUs by diagonal index with A and B replicated and no
 * exchange. Needs rotation keys for the steps of the range (step 0 needs none).
 * Errors: as he_matmul; HE_E_ARG if the range is empty or outside [0, p).
 */
int he_matmul_range(he_ctx* ctx, const he_ctset* A, const he_ctset* B, int m, int p, int idx_lo, int idx_hi,
                    he_ctset** C);

/*
 * he_matmul_bsgs: he_matmul's result (same operands, same p diagonal
 * ciphertexts, decoded by he_decrypt_matrix) with the rotations of Alg. 3 split
 * into baby and giant steps: idx = g i + j, j < g, and
 * D_{g i + j} = Rot(sum_k Rot(A_k, -g i) (x) Rot(B~_k, j), g i), which needs
 * n(g-1) + n(ceil(p/g)-1) + (p - g) rotations instead of n(p-1). g <= 0 picks
 * the power of two nearest sqrt(p). Needs rotation keys for steps 1..g-1,
 * N/2 - g i and g i (i = 1..ceil(p/g)-1), and m + p - 1 <= N/2.
 * Errors: HE_E_ARG, HE_E_SCALE, HE_E_LEVEL, HE_E_NOKEY.
 */
int he_matmul_bsgs(he_ctx* ctx, const he_ctset* A, const he_ctset* B, int m, int p, int g, he_ctset** C);

/*
 * he_matmul_volley: encrypted C = A B without rotations. A from
 * he_encrypt_matrix_a_volley (groups * n ciphertexts), B from
 * he_encrypt_matrix_b (n ciphertexts), same level and scale. Result: `groups`
 * ciphertexts at one level lower, D_g = relin(rescale(sum_k Ahat_{g,k} (x)
 * B~_k)); slot t * M + o_g + i of D_g holds C[i][(i + g * per + t) mod p]
 * (decode with he_decrypt_matrix_volley). Needs only the relinearisation key.
 * Errors: HE_E_ARG (counts), HE_E_SCALE, HE_E_LEVEL.
 */
int he_matmul_volley(he_ctx* ctx, const he_ctset* A, const he_ctset* B, he_ctset** C);

/*
 * he_matmul_batched: `count` independent products A[i] B[i] (each as in
 * he_matmul, shapes m[i], p[i]; two-component operands) evaluated together;
 * C[i] receives each result, identical to he_matmul's. Products with the same
 * p, level and scale share their ModUp and rotation launches (the B operands of
 * a group are concatenated within a 48 GiB working-memory budget), so each key
 * is read once per launch for all of them; their tensor sums share launches
 * (128 products each), one rescale and one relinearisation. Every launch takes
 * its pointers as kernel parameters, so the call can be captured into a CUDA
 * graph (he_graph_begin) and replayed on new operand contents.
 */
int he_matmul_batched(he_ctx* ctx, int count, const he_ctset* const* A, const he_ctset* const* B, const int* m,
                      const int* p, he_ctset** C);

/*
 * he_conv2d: valid 2-D convolution (cross-correlation, no kernel flip) over
 * the column layout (Alg. 4 with channels summed as in Sec. IV-B). `in` holds
 * c_in * w_in ciphertexts, channel-major ([c][j]), rows at gap `gap` (1 for an
 * input image). weights [c_out][c_in][k][k], bias [c_out] or NULL. Output:
 * c_out * w_out ciphertexts ([o][j']), w_out = (w_in - k) / stride + 1, row
 * gap gap * stride, one level lower, same scale. Needs rotation keys for
 * steps gap * a, a = 1..k-1.
 */
int he_conv2d(he_ctx* ctx, const he_ctset* in, int c_in, int gap, const double* weights, const double* bias,
              int c_out, int k, int stride, he_ctset** out);

/* ---- the paper's single-ciphertext method (Sec. III-C/D): images in one ciphertext ----
 *
 * Layout (virtual ciphertexts, Sec. III-D): image b of a batch is row-major
 * inside a block of block_h x block_w slots starting at slot (b mod per)
 * block_h block_w of ciphertext b / per, per = (N/2) / (block_h block_w);
 * row r at + r block_w. Rot by pos and by pos block_w move one column / row in
 * every block at once.
 *
 * he_vr_encrypt_images: px [batch][h][w] -> ceil(batch / per) ciphertexts.
 *
 * he_vr_encrypt_kernels: the model provider's Kernelspanner (Sec. III-C) for a
 * k x k kernel K (row-major) and bias k0 on h x w images: k^2 ciphertexts at
 * `limbs` limbs, offset (r, c) at index r k + c, holding K tiled from (r, c) at
 * every position where a whole copy fits (scale q_{limbs-1}); and one bias
 * ciphertext at limbs - 2 limbs holding k0 at every valid output position
 * (scale of the context). Ids ct_id_base + t, bias ct_id_base + k^2.
 *
 * he_vr_conv2d: Alg. 4 over every input ciphertext: for each offset t,
 * T = relin(rescale(X (x) S_t)), U = sum_{pos < k} Rot(T, pos), V = U + sum_{1
 * <= pos < k} Rot(U, pos block_w) (SumForConv, Alg. 1, its row pass on the
 * column sums), acc += rescale(V (x) F_t) with F_t Alg. 4's offset mask
 * ((hth - r) mod k = 0, (wth - c) mod k = 0, hth + k <= h, wth + k <= w, at
 * scale q_{l-1}), acc starting from the bias ciphertext. Output: valid
 * convolution (no kernel flip) at positions hth <= h - k, wth <= w - k of each
 * block, two levels down, the input's scale. Needs rotation keys for steps
 * 1..k-1 and block_w .. (k-1) block_w. he_vr_conv2d_coeffs takes the k^2 masks
 * as encoded integer plaintexts [k^2][N] at scale q_{l-1} instead.
 */
/*
 * he_vrot: vRot (Alg. 5). Virtual ciphertexts are rows of row_len slots (row_len
 * divides N/2) whose first img_len slots hold an image; every row's image is
 * rotated left by r (0 <= r < img_len): R = rescale(Rot(X, r) (x) F1 +
 * Rot(X, N/2 - img_len + r) (x) F2), F1 keeping row positions j < img_len - r and
 * F2 positions img_len - r <= j < img_len of every row (Alg. 5 applies F2 to the
 * last row only, a misprint: every row needs its wrapped part), masks at scale
 * q_l; slots past img_len become 0. One level, the scale unchanged. Needs
 * rotation keys for steps r and N/2 - img_len + r. he_vrot_coeffs takes F1, F2
 * as encoded integer plaintexts [2][N].
 */
int he_vrot(he_ctx* ctx, const he_ctset* in, int r, int row_len, int img_len, he_ctset** out);
int he_vrot_coeffs(he_ctx* ctx, const he_ctset* in, int r, int img_len, const int64_t* masks, he_ctset** out);

/*
 * Alg. 3 with one ciphertext per operand (the paper's single-ciphertext matmul).
 * he_vr_encrypt_matrix_a: tau_a, A [m][n] row-major at slots i n + j (m n <= N/2).
 * he_vr_encrypt_matrix_b: tau_b tiled over the whole ring, slot i n + j holds
 * B[j][i mod p] for every row i < N/(2n) (n | N/2, p | N/(2n)); then
 * RowShifter applied idx times is Rot(., idx n) (the m mod p = 0 case, Sec. III-B).
 * he_vr_matmul: for idx < p, T = relin(rescale(A (x) Rot(Bbar, idx n))),
 * SumColVec (T += Rot(T, t), t = 1, 2, .., n/2; rescale(T (x) E) with E the
 * column-0 mask at scale q_{l-2}; T += Rot(T, -t)), acc += rescale(T (x) F_idx)
 * with F_idx keeping slot i n + ((i + idx) mod p), i < m, at scale q_{l-3}.
 * C[i][c] ends at slot i n + c (c < p <= n), three levels down, scale
 * D D / q_{l-1}. n must be a power of two. Keys: steps idx n (idx < p) and
 * +-1, +-2, .., +-n/2. he_vr_matmul_coeffs takes the plaintexts as encoded
 * integers [1 + p][N] (E, then F_idx).
 */
int he_vr_encrypt_matrix_a(he_ctx* ctx, const double* A, int m, int n, uint64_t ct_id_base, he_ctset** out);
int he_vr_encrypt_matrix_b(he_ctx* ctx, const double* B, int n, int p, uint64_t ct_id_base, he_ctset** out);
int he_vr_matmul(he_ctx* ctx, const he_ctset* A, const he_ctset* Bbar, int m, int n, int p, he_ctset** out);
int he_vr_matmul_coeffs(he_ctx* ctx, const he_ctset* A, const he_ctset* Bbar, int m, int n, int p, const int64_t* masks,
                        he_ctset** out);

int he_vr_encrypt_images(he_ctx* ctx, const double* px, int batch, int h, int w, int block_h, int block_w,
                         uint64_t ct_id_base, he_ctset** out);
int he_vr_encrypt_kernels(he_ctx* ctx, const double* K, int k, double k0, int h, int w, int block_h, int block_w,
                          int limbs, uint64_t ct_id_base, he_ctset** kernels, he_ctset** bias);
int he_vr_conv2d(he_ctx* ctx, const he_ctset* in, const he_ctset* kernels, const he_ctset* bias, int h, int w, int k,
                 int block_h, int block_w, he_ctset** out);
int he_vr_conv2d_coeffs(he_ctx* ctx, const he_ctset* in, const he_ctset* kernels, const he_ctset* bias, int k,
                        int block_w, const int64_t* masks, he_ctset** out);

/*
 * he_reform: ReForm (Sec. IV-C) in the column layout. After a strided layer
 * row i of image block b sits at slot b * block_stride + gap * i; ReForm moves
 * it to b * block_stride + i (row gap 1), every other slot becoming 0:
 * out = rescale(sum_{i < h_valid} mask_i (x) Rot(X, (gap - 1) i)), mask_i the
 * 0/1 plaintext of slots b * block_stride + i encoded at scale q_l. h_valid - 1
 * rotations per ciphertext (one hoisted ModUp), one level, scale unchanged.
 * Needs rotation keys for steps (gap - 1) i, i = 1..h_valid-1. Errors:
 * HE_E_ARG (shape), HE_E_LEVEL, HE_E_NOKEY.
 */
int he_reform(he_ctx* ctx, const he_ctset* in, int gap, int h_valid, int block_stride, he_ctset** out);

/* he_reform_coeffs: he_reform with the masks given as encoded integer
 * plaintexts masks [h_valid][N] (signed coefficients at scale q_l), so two
 * implementations can start from the same plaintexts. */
int he_reform_coeffs(he_ctx* ctx, const he_ctset* in, int gap, int h_valid, const int64_t* masks, he_ctset** out);

/*
 * he_encrypt_conv_weights: the model provider's kernel ciphertexts (Sec. V:
 * kernels are encrypted before they reach the server; Kernelspanner's role,
 * Sec. III-C, in the column layout). W [c_out][c_in][k][k] -> c_out * c_in * k
 * * k ciphertexts in that order, each encrypting the constant polynomial
 * round(W q_{limbs-1}) (the weight at every slot, at scale q_{limbs-1}) with
 * `limbs` limbs. Ids ct_id_base + index. Errors: HE_E_ARG, HE_E_LEVEL.
 */
int he_encrypt_conv_weights(he_ctx* ctx, const double* W, int c_out, int c_in, int k, int limbs, uint64_t ct_id_base,
                            he_ctset** out);

/*
 * he_conv2d_enc: he_conv2d with encrypted kernels (from
 * he_encrypt_conv_weights at the input's level). Output (o, j') = sum_{c,b,a}
 * W[o][c][a][b] (x) Rot(X_{c, s j' + b}, gap a), summed as three-component
 * tensor products, rescaled, relinearised, plus round(bias_o scale); layout,
 * scale, level and keys as he_conv2d (plus the relinearisation key). All
 * rotations of the input are held at once (the work budget is not applied).
 */
int he_conv2d_enc(he_ctx* ctx, const he_ctset* in, int c_in, int gap, const he_ctset* weights, const double* bias,
                  int c_out, int k, int stride, he_ctset** out);

/*
 * he_poly_act: polynomial activation in place, coeffs[0..degree] the
 * coefficients c0, c1, ... of f(x) = sum_d c_d x^d.
 *  - degree 2 with coeffs {0, 0, 1} (x -> x^2): tensor product, rescale; one
 *    level.
 *  - degree 3 (the ACT layers of Table I, e.g. ACT-1 = -0.00015120704 +
 *    0.4610149 x + 2.0225089 x^2 - 1.4511951 x^3), and any other degree-2
 *    polynomial (as c3 = 0): depth two, as x^2 (c3 x + c2) + (c1 x + c0):
 *    u = relin(rescale(x (x) x)), t = rescale(x round(c3 q1)) + round(c2 D),
 *    y = rescale(u (x) t), v = rescale(x round(c1 s_y q1 / D)) with its last
 *    limb dropped, + round(c0 s_y); f(x) = y + v. q1, q2 are the primes the
 *    two rescales drop, D the input scale, s_y = ((D D / q1) D) / q2 the
 *    output scale (computed in that order in double precision). Needs the
 *    relinearisation key and two levels (HE_E_LEVEL otherwise).
 * The result keeps three components (d0, d1, d2) and is relinearised by the
 * next operation that needs two (rotation, convolution, matmul, the end of a
 * dense layer, decryption) or by he_relinearize; a dense layer consumes it
 * directly. Other degrees return HE_E_UNIMPL.
 */
int he_poly_act(he_ctx* ctx, he_ctset* inout, const double* coeffs, int degree);

/*
 * he_fc_prepare: encode dense-layer weights for inputs in the column layout:
 * W [out_dim][c_in * h_valid * w_in] in (channel, row, column) order; for
 * output o and input column (c, j) a plaintext with W[o][c][i][j] at slot
 * b * block_stride + gap * i for every block b < batch. Plaintexts are
 * encoded at scale q_l (the prime dropped after the product) at `limbs`
 * limbs, and kept on the device.
 */
int he_fc_prepare(he_ctx* ctx, const double* W, int out_dim, int c_in, int h_valid, int w_in, int gap,
                  int block_stride, int batch, int limbs, he_ptset** out);

/* Same, from integer coefficients pts [out_dim][c_in][w_in][N] encoded elsewhere. */
int he_fc_prepare_coeffs(he_ctx* ctx, const int64_t* pts, int out_dim, int c_in, int w_in, int gap,
                         int block_stride, int limbs, he_ptset** out);
void he_ptset_free(he_ptset* pts);

/*
 * he_fc_apply: Z_o = sum_{c,j} pt_{o,c,j} (x) in_{c,j}, rescale, then sum
 * inside each block by rotate-and-add over gap, 2 gap, ..., block_stride / 2,
 * then add bias[o] (NULL for none). Logit o of image b is at slot
 * b * block_stride of output o (he_decrypt_slots). Needs rotation keys for
 * those steps. Three-component inputs are summed component by component and
 * the out_dim results relinearised.
 */
int he_fc_apply(he_ctx* ctx, const he_ctset* in, const he_ptset* pts, const double* bias, he_ctset** out);

/*
 * he_fc_partial / he_fc_finish: he_fc_apply in two halves, so that a dense
 * layer can be sharded over its input columns (Sec. IV-B: the products of
 * different channels and columns are independent and meet only in a sum).
 * he_fc_partial: `in` holds the n input ciphertexts of columns first ..
 * first + n - 1 of the layout `pts` was prepared for (two or three
 * components); out receives out_dim ciphertexts, the sums
 * sum_{first <= cj < first + n} pt_{o,cj} (x) in_cj mod q, before the rescale
 * (same components as the input; the scale field is the input's while the
 * sums still carry the plaintexts' factor q_l). Partial sums of disjoint
 * column ranges add (he_add, mod q) to the full sums exactly.
 * he_fc_finish: from the full sums (out_dim ciphertexts at the prepared level):
 * rescale, relinearisation, rotate-and-add inside blocks, bias; the result
 * equals he_fc_apply's word for word. `sums` is not modified.
 * Errors: HE_E_ARG (columns outside the prepared range, count), HE_E_LEVEL,
 * HE_E_NOKEY (finish).
 */
int he_fc_partial(he_ctx* ctx, const he_ctset* in, const he_ptset* pts, int first, he_ctset** out);
int he_fc_finish(he_ctx* ctx, const he_ctset* sums, const he_ptset* pts, const double* bias, he_ctset** out);

/* he_fc: he_fc_prepare + he_fc_apply + he_ptset_free. Inputs may have two or
 * three components; the outputs are relinearised before the rotations. */
int he_fc(he_ctx* ctx, const he_ctset* in, const double* W, const double* b, int out_dim, int c_in, int h_valid,
          int w_in, int gap, int block_stride, int batch, he_ctset** out);

/* ---- primitives (Sec. II-A), for composition and testing ---- */

/* Rot(ct, l) for every ciphertext of `in` and every step: one ModUp per
 * ciphertext shared by its steps (hoisting). out has n * n_steps
 * ciphertexts, [ct][step]. */
int he_rotate(he_ctx* ctx, const he_ctset* in, const int32_t* steps, int n_steps, he_ctset** out);

/* Mul(a_i, b_i) pairwise: tensor product and rescale; the result keeps three
 * components until relinearised (see he_poly_act). */
int he_mul(he_ctx* ctx, const he_ctset* a, const he_ctset* b, he_ctset** out);

/* Three components -> two: key switch of d2 with the relinearisation key
 * (no-op for two-component sets). */
int he_relinearize(he_ctx* ctx, he_ctset* inout);

/* Drop the last prime: round(x / q_l) in every limb; scale /= q_l. */
int he_rescale(he_ctx* ctx, he_ctset* inout);

/* Add(a_i, b_i) pairwise (same level and scale). */
int he_add(he_ctx* ctx, const he_ctset* a, const he_ctset* b, he_ctset** out);

/* Add with a plaintext operand (Sec. II-A's Add; Alg. 3 starts its accumulator
 * from such a constant, e.g. a dense layer's bias), in place on component 0:
 * he_add_slots encodes the real slot vectors v (n_vec = 1: one vector of N/2
 * values for every ciphertext; n_vec = the set size: one per ciphertext) at the
 * set's own scale, reduces them modulo the set's primes and adds them;
 * he_add_plain_coeffs takes the encoded integer plaintexts m [n_vec][N]
 * instead. HE_E_ARG for another n_vec; refused (HE_E_STATE) on a set made
 * before an open capture. */
int he_add_slots(he_ctx* ctx, he_ctset* inout, const double* v, int n_vec);
int he_add_plain_coeffs(he_ctx* ctx, he_ctset* inout, const int64_t* m, int n_vec);

/* Modulus dropping: a new set holding every polynomial's residues modulo
 * q_0 .. q_{limbs-1} only (the same ciphertexts modulo a smaller Q, no
 * division, the scale unchanged), e.g. to bring an operand encrypted at the
 * top level down to its partner's level before a product. HE_E_LEVEL unless
 * 1 <= limbs <= the set's limbs. The caller frees *out. */
int he_ctset_drop_levels(he_ctx* ctx, const he_ctset* in, int limbs, he_ctset** out);

/* ---- decryption (Dec_sk, Sec. II-A) ---- */

/*
 * he_decrypt_slots: out [n][N/2] real slot values. Decryption computes
 * c0 + c1 s on the device and reads the q_0 limb: valid while |message +
 * noise| < q_0 / 2, which the parameter sets keep (q_0 is the large base
 * prime).
 */
int he_decrypt_slots(he_ctx* ctx, const he_ctset* in, double* out, size_t out_len);

/* he_decrypt_matrix: C [m][p] from he_matmul's p diagonal ciphertexts. */
int he_decrypt_matrix(he_ctx* ctx, const he_ctset* C, int m, int p, double* C_out);

/* he_decrypt_matrix_volley: C [m][p] from he_matmul_volley's ciphertexts. */
int he_decrypt_matrix_volley(he_ctx* ctx, const he_ctset* C, int m, int p, double* C_out);

/* he_decrypt_image: [batch][n_ct][h_valid] column values, row i of image b
 * read at slot b * block_stride + gap * i of each ciphertext. */
int he_decrypt_image(he_ctx* ctx, const he_ctset* in, int batch, int block_stride, int gap, int h_valid,
                     double* out, size_t out_len);

/* ---- ciphertext sets ---- */

/* Copy out as coefficient-domain limbs [n][polys][limbs][N] (inverse NTT on
 * the device; polys from he_ctset_info). n_words must be at least
 * n * polys * limbs * N. Synchronises. */
int he_ctset_export(const he_ctset* set, uint64_t* host, size_t n_words);

/*
 * he_ctset_export_async: he_ctset_export that does not wait, so that a caller
 * streaming results can queue the next batch while this one is still on the
 * GPU. The inverse transform and the copy into `host` ([n][polys][limbs][N],
 * coefficient domain, n_words as for he_ctset_export) are queued on the
 * context's stream after the work already there; *ticket receives a number
 * above 0 that grows with every export of the context. The words may be read
 * once he_ctset_export_wait has returned for that ticket (or the context has
 * been synchronised). The set may be freed right after the call: its release
 * is ordered after the copy. Page-locked host memory lets the call return at
 * once; with pageable memory the copy completes before the call returns.
 * Refused (HE_E_STATE) inside a capture of the context's stream. The paper
 * has no counterpart (an interface for streaming callers).
 */
int he_ctset_export_async(const he_ctset* set, uint64_t* host, size_t n_words, uint64_t* ticket);

/*
 * he_ctset_export_wait: block until the export with this ticket, and every
 * earlier export of the context, has reached host memory; a device error
 * raised meanwhile is reported as by he_ctx_synchronize. HE_E_ARG for 0 or a
 * ticket the context has not issued.
 */
int he_ctset_export_wait(he_ctx* ctx, uint64_t ticket);

/* Build a set from coefficient-domain limbs [n][2][limbs][N] (residues < q_i). */
int he_ctset_import(he_ctx* ctx, const uint64_t* host, int n, int limbs, double scale, he_ctset** out);

/*
 * he_ctset_import_async: he_ctset_import that does not wait for the copy, so
 * that a caller streaming inputs can upload the next batch while the GPU still
 * computes the current one. The host words [n][2][limbs][N] (coefficient
 * domain) are copied on a copy stream of the context into one of two device
 * staging buffers the context keeps (allocated on first use and grown to the
 * largest import, freed with the context); the context's stream waits for the
 * copy, range-checks the residues, takes them into the new set and transforms
 * them. The host words must stay unchanged until the copy has completed, which
 * is certain once the context has been synchronised (he_ctx_synchronize, an
 * export, a decryption); page-locked host memory lets the copy overlap the
 * computation. Out-of-range residues are reported as HE_E_ARG by that
 * synchronisation. Refused (HE_E_STATE) inside a capture of the context's
 * stream. The paper has no counterpart (an interface for streaming callers).
 */
int he_ctset_import_async(he_ctx* ctx, const uint64_t* host, int n, int limbs, double scale, he_ctset** out);

/* Copy out the device words as held, [n][polys][limbs][N] in the NTT domain
 * (no transform). n_words must be at least n * polys * limbs * N.
 * Synchronises. */
int he_ctset_export_raw(const he_ctset* set, uint64_t* host, size_t n_words);

/* Build a set of two-component ciphertexts from NTT-domain words
 * [n][2][limbs][N] as he_ctset_export_raw writes them; every residue is
 * checked to be below its prime (HE_E_ARG otherwise). */
int he_ctset_import_raw(he_ctx* ctx, const uint64_t* host, int n, int limbs, double scale, he_ctset** out);

/*
 * Word exchange between processes (a sharded layer's all-gather or halo
 * exchange): he_ctset_export_words copies the words as held, [n][polys][limbs][N]
 * in the NTT domain, into dst -- HOST memory (dst_on_device = 0) or DEVICE
 * memory of the context's GPU (dst_on_device = 1, e.g. a communication
 * library's buffer) -- and returns when the copy is complete. n_words must be
 * at least n * polys * limbs * N. he_ctset_import_words builds a set of n
 * ciphertexts of `polys` (2 or 3) components at `limbs` limbs and the given
 * scale from such words in host or device memory (src_on_device); the source
 * is read on the context's stream, so device writes to it must be complete (or
 * ordered before the call on that stream) when the call is made, and it may be
 * reused when the call returns. Every residue is checked against its prime
 * (HE_E_ARG otherwise).
 */
int he_ctset_export_words(const he_ctset* set, uint64_t* dst, int dst_on_device, size_t n_words);
int he_ctset_import_words(he_ctx* ctx, const uint64_t* src, int src_on_device, int n, int polys, int limbs,
                          double scale, he_ctset** out);

/* Number of ciphertexts, limbs (level + 1), scale, components per ciphertext
 * (2, or 3 for an unrelinearised product). Any pointer may be NULL. */
int he_ctset_info(const he_ctset* set, int* n_ct, int* limbs, double* scale, int* polys);

/* Device address of the residues, [n][2][limbs][N] uint64 in the NTT domain. */
int he_ctset_device_ptr(const he_ctset* set, uint64_t** dptr);

/* A set of n ciphertexts taken from `set` starting at ciphertext `first`
 * (a copy). */
int he_ctset_slice(he_ctx* ctx, const he_ctset* set, int first, int n, he_ctset** out);

/* Concatenate sets of equal level and scale (a copy). */
int he_ctset_concat(he_ctx* ctx, const he_ctset* const* sets, int n_sets, he_ctset** out);

void he_ctset_free(he_ctset* set);

/*
 * he_rescale_noalloc: he_rescale for callers that cannot allocate device
 * memory during the call -- a serving loop that must keep a fixed memory
 * footprint once started, a framework that hands out every device
 * allocation from its own pool, or a process whose device-memory quota is
 * used up. The paper has no counterpart; this is an interface for such
 * callers. It makes no cudaMalloc, cudaFree or other allocating call.
 *
 * in:  DEVICE pointer, n_ct ciphertexts [n_ct][2][limbs][N] in the NTT domain
 *      (the layout of he_ctset_device_ptr), at the given scale.
 * out: DEVICE pointer, caller-owned, [n_ct][2][limbs-1][N]; must not overlap in.
 * out_scale (host, may be NULL) receives scale / q_{limbs-1}.
 * The result equals he_rescale's. Work is enqueued on the context's stream.
 *
 * Scratch: one array of 2^21 64-bit words (16 MiB) that the library keeps in
 * every GPU that loads it, until the process exits. Sizes with
 * n_ct * 2 * limbs * N > 2^21 are rejected with HE_E_ARG (e.g. at N = 2^16 one
 * ciphertext of up to 16 limbs per call). The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture. The context's
 * device must be current. Every call shares the array and it keeps the last
 * call's contents (no step reads scratch it has not written in the same
 * call), so calls whose GPU work overlaps -- on different streams or from
 * different threads -- race on it.
 */
int he_rescale_noalloc(he_ctx* ctx, const uint64_t* in, int n_ct, int limbs, double scale, uint64_t* out,
                       double* out_scale);

/*
 * he_pack_blocks: several images per ciphertext set (Sec. III-D): out =
 * rescale(sum_t masks_t * sets_t), ciphertext by ciphertext. Each set holds n
 * two-component ciphertexts at the same level and scale; masks is a plaintext
 * set prepared by he_fc_prepare_coeffs with out_dim >= n_sets, c_in = w_in = 1
 * and limbs = the sets' level, mask t encoded at scale q_{limbs-1} (1 on the
 * slots set t keeps, 0 elsewhere). The result is at one level lower and the
 * sets' scale. Errors: HE_E_ARG (shapes), HE_E_SCALE, HE_E_LEVEL.
 */
int he_pack_blocks(he_ctx* ctx, const he_ctset* const* sets, int n_sets, const he_ptset* masks, he_ctset** out);

/* ---- serving: continuous batching of encrypted CNN requests ---- */

/*
 * A server answers encrypted inference requests for the three-layer CNN of
 * the evaluation (conv 8x5x5 stride 2 -> x^2 -> conv 16x3x3 stride 2 -> x^2
 * -> dense 10; Sec. IV-C uses the same conv / square / dense structure) on
 * square images of the sides it was created for, all on one context (one
 * GPU, one key set kept in device memory).
 *
 * Request layout: a side x side image as `side` ciphertexts (column j holds
 * the column's pixels, Sec. I-C), fresh at the top level and the context's
 * scale, with the image repeated in every slot block of stride `side`
 * (he_encrypt_image with batch = (N/2)/side copies of the image and
 * block_stride = side), exported as the device words [side][2][n_q][N]
 * (he_ctset_export_raw). Requests are batched by slot blocks, the paper's
 * several images per ciphertext (Sec. III-D): request t of a batch is kept in
 * block t by a 0/1 plaintext mask, the masked requests are summed into one
 * set, rescaled once (one level: a request uses 6 of the n_q - 1 levels), and
 * the network runs once for the whole batch.
 *
 * Scheduling (one worker thread per server): requests are admitted to device
 * memory in submission order while the bytes of admitted requests and
 * unclaimed results plus a reserve for one running batch stay within
 * hbm_budget_bytes; the oldest waiting request blocks later ones. When the
 * GPU is free the next batch takes the image side of the oldest admitted
 * request and up to max_blocks admitted requests of that side, oldest first.
 * Requests that arrive while a batch runs are admitted (memory permitting)
 * and copied to the device on the server's own stream, overlapping the
 * batch, and join the next batch. The reserve is measured at creation by
 * running one batch per side on an all-zero request (the stream-ordered
 * allocator's high-water mark), plus 1/16.
 *
 * Results: logit o of a request is slot block*side of ciphertext o of its
 * result set (10 ciphertexts; decrypt with he_decrypt_slots). Decrypted
 * results are the same alone and in any mix, up to CKKS noise.
 */
/* ---- CUDA graphs of library calls (no counterpart in the paper) ----
 *
 * he_graph_begin starts capturing the calls made on ctx's stream (which must
 * be a non-default stream) into a CUDA graph; he_graph_end stops, instantiates
 * it and returns the graph; he_graph_launch replays it on ctx's stream. A
 * replay reads the current contents of the sets made before the capture and
 * rewrites the sets made during it: their handles stay valid and hold the
 * results of the latest replay once the stream has reached it (the graph's
 * memory is re-allocated at the same addresses on each replay). Inside a
 * capture:
 *  - calls that only read their input sets and return new sets (products,
 *    rotations, matmuls, dense layers, ...) are captured;
 *  - in-place calls (he_rescale, he_relinearize, he_poly_act) and
 *    he_ctset_assign into sets made before the capture return HE_E_STATE;
 *  - calls that upload host data (encryption, convolution weights, biases,
 *    plaintext preparation) cannot be captured: they return HE_E_STATE (or
 *    fail inside CUDA) and he_graph_end returns HE_E_CUDA;
 *  - he_ctset_free of a set made before the capture is deferred to he_graph_end.
 * Free the sets made during a capture after the graph's last replay. Kernel
 * launches of a replay are added to he_kernel_launches. A capture that the
 * caller opens on the context's stream itself (cudaStreamBeginCapture, a
 * framework's graph capture) refuses the calls that upload host data the
 * same way: they return HE_E_STATE without recording the copy.
 */
int he_graph_begin(he_ctx* ctx);
int he_graph_end(he_ctx* ctx, he_graph** out);
int he_graph_launch(he_graph* g);
/* number of kernel nodes in the graph */
int he_graph_info(const he_graph* g, uint64_t* kernel_nodes);
void he_graph_destroy(he_graph* g);

/* Copy src's ciphertexts into dst (same count, components and level; device to
 * device on ctx's stream): new inputs for a graph's next replay. */
int he_ctset_assign(he_ctx* ctx, he_ctset* dst, const he_ctset* src);

typedef struct he_server he_server;

#define HE_REQ_WAITING 0   /* in host memory, not admitted yet  */
#define HE_REQ_ADMITTED 1  /* copied (or being copied) to the device */
#define HE_REQ_RUNNING 2   /* in the batch on the GPU           */
#define HE_REQ_DONE 3      /* result ready for he_server_take   */
#define HE_REQ_FAILED 4    /* he_server_take reports the error  */
#define HE_REQ_CANCELLED 5 /* withdrawn by he_server_cancel      */

typedef struct {
  const double* conv1_w;         /* [8][1][5][5]                               */
  const double* conv1_b;         /* [8]                                        */
  const double* conv2_w;         /* [16][8][3][3]                              */
  const double* conv2_b;         /* [16]                                       */
  int n_sides;                   /* number of image sides served               */
  const int* sides;              /* [n_sides], powers of two in [16, N/2]      */
  const double* const* fc_w;     /* per side: [10][16 h2 h2], h2 the spatial
                                    size after both convs, (c, i, j) order     */
  const double* const* fc_b;     /* per side: [10]                             */
  size_t hbm_budget_bytes;       /* device bytes for requests, results and the
                                    running batch (keys and tables excluded)  */
  int max_blocks;                /* requests per batch (1 = one at a time)     */
  int start_paused;              /* nonzero: no batch starts before
                                    he_server_pause(srv, 0)                    */
} he_server_desc;

/*
 * he_server_create: build the masks and dense-layer plaintexts of every side,
 * add the rotation keys the network needs (he_keygen semantics), measure the
 * batch reserve, and start the worker. The weights are copied. Needs n_q >= 7.
 * Lowers the context's work budget (he_ctx_set_work_budget) to at most
 * 16 GiB, so that batches leave room for requests.
 * Errors: HE_E_ARG (sides, null weights), HE_E_LEVEL, HE_E_OOM, HE_E_CUDA.
 * While a server runs, do not call he_keygen on its context or destroy the
 * context; other calls on the context may come from any thread, and their
 * GPU work queues on the context stream with the server's batches.
 */
int he_server_create(he_ctx* ctx, const he_server_desc* desc, he_server** out);

/* Words of one request of this side: side * 2 * n_q * N. */
int he_server_request_words(const he_server* srv, int side, size_t* n_words);

/*
 * he_server_submit: queue a request (layout above). host_words is borrowed
 * until the request is DONE or FAILED and should be page-locked so its upload
 * overlaps the running batch. Host work only (the server's uploader thread
 * copies admitted requests); returns at once with the request id.
 * Errors: HE_E_ARG (side not served, wrong size), HE_E_OOM (the request alone
 * exceeds the budget).
 */
int he_server_submit(he_server* srv, const uint64_t* host_words, size_t n_words, int side, uint64_t* req_id);

/* Current HE_REQ_* state of a request not yet taken. */
int he_server_poll(he_server* srv, uint64_t req_id, int* state);

/* Wait up to timeout_ms for a request to be DONE, FAILED or CANCELLED
 * (*state gets its state). HE_E_TIMEOUT if it is not. */
int he_server_wait(he_server* srv, uint64_t req_id, int timeout_ms, int* state);

/*
 * he_server_take: claim a DONE request's result, a copy of its batch's 10
 * logit ciphertexts (free with he_ctset_free), and forget the request. The
 * copy runs on the server's result stream.
 * block: its slot block. times_ms (may be NULL): [submit, admit, start of its
 * batch, end of its batch] in milliseconds of the host's monotonic clock
 * (CLOCK_MONOTONIC). HE_E_STATE if not done; HE_E_CUDA (with the message)
 * for a failed request, which is forgotten too.
 */
int he_server_take(he_server* srv, uint64_t req_id, he_ctset** logits, int* block, double* times_ms);

/* Words of one result: the 10 logit ciphertexts, 10 * 2 * (n_q - 6) * N. */
int he_server_result_words(const he_server* srv, size_t* n_words);

/*
 * he_server_take_host: he_server_take into host memory: the result's device
 * words as held ([10][2][n_q - 6][N], NTT domain; he_ctset_import_raw at
 * n_q - 6 limbs and the context's scale rebuilds the set). The copy runs on
 * the server's result stream, so it does not wait for the running batch;
 * page-locked memory makes it a direct transfer. n_words >= the result words.
 */
int he_server_take_host(he_server* srv, uint64_t req_id, uint64_t* host, size_t n_words, int* block,
                        double* times_ms);

/* Hold (paused != 0) or resume starting batches; a running batch finishes. */
int he_server_pause(he_server* srv, int paused);

/*
 * he_server_cancel: withdraw a request. Not yet in a batch: it leaves the
 * queue at once and its device memory and budget are released (requests
 * behind it may be admitted). In a running batch: the batch finishes and the
 * request's share of the result is dropped. Done: its share of the result is
 * released. The request then reads HE_REQ_CANCELLED; he_server_take returns
 * HE_E_STATE for it and forgets it. Errors: HE_E_ARG (unknown request).
 */
int he_server_cancel(he_server* srv, uint64_t req_id);

/*
 * counts[7]: submitted, waiting (host), admitted (on the device, not
 * running), done, failed, batches started, cancelled. bytes[4]: budgeted bytes held now,
 * the most ever held, the batch reserve, the allocator's high-water mark
 * (including keys and tables). Either may be NULL.
 */
int he_server_stats(he_server* srv, uint64_t* counts, size_t* bytes);

/* Stop the worker after its running batch and free everything the server
 * holds; result sets already taken stay valid. */
void he_server_destroy(he_server* srv);

/*
 * he_sched_simulate: the server's scheduler on a simulated GPU (no device
 * work), for checking the policy. Request i arrives at arrival_ms[i]
 * (ascending) with image side[i] and bytes[i]; a batch of T requests of
 * side sides[s] takes base_ms[s] + per_request_ms[s] * T; a batch's result
 * (out_bytes) is claimed when the batch ends. Outputs per request: batch
 * number (-1 if it can never fit the budget), slot block, and the admit /
 * start / done times (-1 if rejected); *max_held the most budgeted bytes ever
 * held (may be NULL).
 */
int he_sched_simulate(int n, const double* arrival_ms, const int* side, const size_t* bytes, int n_sides,
                      const int* sides, const double* base_ms, const double* per_request_ms, size_t budget,
                      size_t reserve, int max_blocks, size_t out_bytes, int64_t* batch, int* block,
                      double* admit_ms, double* start_ms, double* done_ms, size_t* max_held);

/* ---- transforms (testing) ---- */

/*
 * he_ntt: negacyclic NTT of host data [n_polys][limbs][N] in place, limb i
 * modulo q_i (prime index `first_prime` + i). Forward: out[j] =
 * sum_i a_i psi^((2 brv(j) + 1) i) mod q with psi = x^((q-1)/2N) for the
 * smallest quadratic non-residue x of q; inverse undoes it.
 */
int he_ntt(he_ctx* ctx, uint64_t* host, int n_polys, int limbs, int first_prime, int inverse);

/*
 * Transform geometry (no counterpart in the paper, which describes no number-
 * theoretic transform). The negacyclic transform of a limb runs as n1 stages in
 * column kernels (blocks of `cols` adjacent columns) and log_n - n1 stages in
 * row kernels; every geometry computes the same transform, so results do not
 * depend on it. he_ntt_set_geometry(ctx, 0, 0) restores the default (n1 =
 * log_n / 2, 16 columns); unsupported choices return HE_E_ARG.
 * he_ntt_autotune times a forward and an inverse transform of `rows` limbs
 * (rounded up to whole polynomials) for every supported (n1, cols) with cols
 * in {4, 8, 16, 32} (CUDA events on the context stream, 3 repetitions after a
 * warm-up), keeps the fastest for the context and returns it with its time
 * in microseconds (any output pointer may be NULL).
 */
int he_ntt_set_geometry(he_ctx* ctx, int n1, int cols);
int he_ntt_autotune(he_ctx* ctx, int rows, int* n1, int* cols, double* us);

/* ---- instrumentation ---- */

/* Measured peak of 64-bit Shoup modular products (x w mod q with a
 * precomputed companion of w, the NTT butterfly's product) per second on the
 * context's GPU: independent chains in registers on every SM, timed with
 * CUDA events. Used as the integer-arithmetic roofline. */
int he_calibrate_modmul(he_ctx* ctx, double* modmul_per_s);

/* Measured peak of 96-bit multiply-accumulates (acc += a b for residues a, b
 * below 2^46, seven 32-bit multiplies by PTX carry chains, the product of the
 * convolution kernels for such primes) per second on the context's GPU,
 * measured like he_calibrate_modmul. */
int he_calibrate_mac96(he_ctx* ctx, double* mac_per_s);

/* Measured peak of forward-transform butterflies per second on the context's
 * GPU, in the form the transform kernels run them (the negacyclic NTT's
 * Cooley-Tukey butterfly with the twiddle product of Shoup's method): narrow
 * != 0 for primes below 2^54 (growing-range butterfly: the cheaper quotient
 * estimate, no reduction between stages), 0 for the wider primes (Harvey's
 * lazy butterfly). Independent chains in registers on every SM, timed like
 * he_calibrate_modmul; the roofline of the transform kernels.
 * Errors: HE_E_ARG (null pointers), HE_E_CUDA. */
int he_calibrate_butterfly(he_ctx* ctx, int narrow, double* bfly_per_s);

/* Fault injection on the host, for tests of the error paths: the next n
 * device allocations of the library (any context, any thread) fail as if the
 * device were out of memory (HE_E_OOM); n = 0 disarms it. No GPU fault is
 * involved. The paper has no counterpart. */
int he_debug_fail_allocations(int n);

/* Device-side fault path, for tests: enqueue on the context's stream one
 * thread that waits on a barrier nothing arrives on, gives up after limit_us
 * microseconds (1 .. 2,000,000) and records the failure in the context's
 * status word -- the path every bounded wait of the tensor-core kernels takes.
 * The next he_ctx_synchronize (or export) returns HE_E_TIMEOUT once and clears
 * the word; the context stays usable. No GPU fault is involved. The paper has
 * no counterpart. Errors: HE_E_ARG. */
int he_debug_wait_timeout(he_ctx* ctx, int limit_us);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t he_kernel_launches(void);

/* Per-kernel timing: when on, every launch is bracketed by CUDA events on its
 * stream. Off by default. */
int he_profile_enable(int on);

/* Synchronise the recorded events and report, per kernel name, the summed
 * device time (ms), launch count, algorithmic bytes (each operand of a
 * launch read or written once) and modular products (64-bit multiplications
 * that are reduced or accumulated: NTT butterflies, multiply-accumulate
 * terms, base-conversion terms) since the last read; clears the record.
 * names receives the kernel names separated by '\n' (truncated to names_len);
 * ms, counts, bytes and products (each may be NULL) receive the first
 * max_kernels entries; *n_kernels the number of distinct kernels. */
int he_profile_read(char* names, size_t names_len, double* ms, uint64_t* counts, double* bytes, double* products,
                    int max_kernels, int* n_kernels);

/* Message of the last failed call on this thread ("" if none). */
const char* he_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HE_GB300_H */
