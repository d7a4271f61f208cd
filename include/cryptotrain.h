/*
 * cryptotrain.h -- C ABI of the GB300 library for the homomorphic linear
 * layers of CryptoTrain (arXiv 2409.16675): RLWE/BFV ciphertext x plaintext
 * polynomial convolution (CPMul + CCAdd) in the conventional row-major and the
 * correlated polynomial encodings, the offline CCMul-Precompute path
 * (ciphertext x ciphertext tensor product, exact rescaling,
 * relinearisation), PPMul, encryption and decryption.
 *
 * Conventions shared by every entry point
 *  - Return value: HE_OK (0) or a negative HE_ERR_* code.  A failing call
 *    leaves a message retrievable with he_last_error().  No call aborts the
 *    process.
 *  - Handles (he_ctx, he_keys, he_plan) are owned by the library and freed by
 *    the matching *_destroy call.
 *  - Data buffers are caller-owned DEVICE pointers (cudaMalloc / PyTorch
 *    tensors) unless a parameter says "host"; the library never frees them.
 *    All are dense, C-contiguous, 8-byte aligned.
 *  - Every compute call is asynchronous on the given cudaStream_t (NULL = the
 *    legacy default stream).  A context owns one scratch workspace: calls on
 *    one context must be issued from one host thread and, if they use
 *    different streams, be ordered by the caller.  Workspace growth
 *    synchronises the device, so make one warm-up call before capturing a
 *    CUDA graph.
 *  - Layouts (coefficient form, the only form that crosses this boundary):
 *      ciphertext  uint64 [2][L][N], limb i in [0, q_i)
 *      plaintext   uint64 [N] in [0, t)
 *      secret key  int64  [N] in {-1, 0, 1}
 *      public key  uint64 [2][L][N] = (b, a), b = -(a s + e)
 *      relin key   uint64 [ell][2][L][N], rlk_j = (-(a_j s + e_j) + 2^(base*j) s^2, a_j)
 *  - Keys are bound to the parameters (he_ctx_fingerprint) of the context
 *    that made them, and a plan to its ring degree N: a call given keys of
 *    a context with other parameters, or a plan of another N, fails with
 *    HE_ERR_INVALID_ARG before any device work.
 *  - All arithmetic is exact integer arithmetic; results are bit-identical
 *    to the CPU oracle for the same seeds.
 */
#ifndef CRYPTOTRAIN_H
#define CRYPTOTRAIN_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HE_OK 0
#define HE_ERR_INVALID_ARG -1
#define HE_ERR_UNSUPPORTED_PARAMS -2
#define HE_ERR_PLAN_DOES_NOT_FIT -3
#define HE_ERR_OOM -4
#define HE_ERR_BUDGET_EXCEEDED -5
#define HE_ERR_TIMEOUT -6
#define HE_ERR_CUDA -7

#define HE_MAX_LIMBS 16

/* encodings (Section 3.3) */
#define HE_ENC_CONVENTIONAL 0 /* row-major packing of the zero-padded input (left half of Fig. 7) */
#define HE_ENC_CORRELATED 1   /* Eq. 1 and Eq. 2: x^[iO+j] = x[i,j], w^[(h-i-1)O+(h-j-1)] = w[i,j] */
/* OR-ed into the encoding of he_conv_plan / he_plan_search: a depthwise layer
 * (M = C, output channel m reads input channel m only: weights diagonal in
 * the channel indices, e.g. the gamma of a batch norm).  The plan keeps the
 * output channels of a kernel polynomial in one channel group and every
 * product call skips the (kernel polynomial, channel group) pairs whose
 * weights are all zero: MG * T products per image instead of MG * G * T. */
#define HE_PLAN_DEPTHWISE 16

/* roles of a tensor in an encoding */
#define HE_ROLE_INPUT 0  /* activations x [batch][C][H][W] */
#define HE_ROLE_KERNEL 1 /* weights     w [M][C][h][h]     */

/* tensor element types */
#define HE_DTYPE_U8 0
#define HE_DTYPE_I8 1
#define HE_DTYPE_I64 2

/* key export selectors */
#define HE_KEY_SK 0
#define HE_KEY_PK 1
#define HE_KEY_RLK 2

/*
 * Ring parameters.  Section 2 (Notations) fixes the ring A_{N,p} =
 * Z_p[x]/(x^N+1) with N a power of two; the paper states no values, so the
 * caller chooses them.
 *   N            ring degree, a power of two in [1024, 16384]
 *   L            number of RNS limbs of q, 1..HE_MAX_LIMBS
 *   q[]          explicit limb primes (each prime, = 1 mod 2N, < 2^61,
 *                distinct); if q[0] == 0 they are generated from prime_bits
 *   prime_bits[] per-limb bit size b in [20, 61]: the largest unused prime
 *                below 2^b that is = 1 mod 2N, limbs in the given order
 *   t            plaintext modulus, 2 <= t < 2^61, coprime to every q_i.
 *                PPMul needs t prime and t = 1 mod 2N.
 *   base_log2    relinearisation digit size in bits, 1..32 (0 -> 16)
 *   eta          centred-binomial error parameter, 1..32 (0 -> 21)
 *   max_ccmul_group  largest number of tensor products summed into one CCMul
 *                output (sizes the auxiliary basis; 0 -> 64)
 *   device       CUDA device ordinal
 */
typedef struct he_params {
    int32_t N;
    int32_t L;
    int32_t prime_bits[HE_MAX_LIMBS];
    uint64_t q[HE_MAX_LIMBS];
    uint64_t t;
    int32_t base_log2;
    int32_t eta;
    int32_t max_ccmul_group;
    int32_t device;
    double max_ccmul_scratch_bytes;  /* per-call CCMul scratch; larger calls run in chunks of
                                        outputs (0: 4 GiB) */
    double max_table_cache_bytes;    /* device copies of term tables kept between calls (they
                                        are reused by calls of the same shape); once above this,
                                        the next call synchronises the device and frees them
                                        (0: 256 MiB) */
} he_params;

/* Read-only description of a context (filled by he_ctx_query). */
typedef struct he_ctx_info {
    int32_t N, L;
    uint64_t q[HE_MAX_LIMBS];
    uint64_t t;
    int32_t ell;         /* relinearisation digits = ceil(bitlen(q) / base_log2) */
    int32_t n_aux;       /* auxiliary primes of the CCMul basis */
    uint64_t aux[24];
    int32_t ppmul_ok;    /* 1 if t supports he_ppmul_* */
    int32_t ks_primes;   /* small primes (< 2^30) of the relinearisation key switch, 0 when it
                            runs over the limbs of q instead (see he_ccmul_precompute) */
} he_ctx_info;

/* Convolution shape (stride 1, square kernel, zero padding pad <= h-1). */
typedef struct he_conv_shape {
    int32_t C, H, W; /* input channels and spatial size */
    int32_t M;       /* output channels */
    int32_t h;       /* kernel size */
    int32_t pad;     /* zero padding on each side */
} he_conv_shape;

/* Plan summary (filled by he_plan_query). */
typedef struct he_plan_info {
    int32_t encoding;
    int32_t Cn, G;      /* channels per polynomial, channel groups */
    int32_t th, tw;     /* output tile size */
    int32_t Th, Tw, T;  /* tiles per image (T = Th * Tw) */
    int32_t Hn, Wn, Ooff; /* conventional window and kernel offset */
    int32_t O, S;       /* correlated row stride and channel stride */
    int32_t Ho, Wo;
    int32_t Mn, Sout;   /* output channels per kernel polynomial and their stride */
    int32_t MG;         /* kernel polynomials per channel group: ceil(M / Mn) */
    int32_t depthwise;  /* 1: only pair (mg, g = mg * Mn / Cn) is multiplied */
} he_plan_info;

typedef struct he_ctx he_ctx;
typedef struct he_keys he_keys;
typedef struct he_plan he_plan;

/* he_setup: validate params, search the primes, build NTT / CRT tables on
 * `device`, and return a new context in *ctx.  Errors: INVALID_ARG,
 * UNSUPPORTED_PARAMS (no such primes, N out of range), CUDA, OOM. */
int he_setup(const he_params *params, he_ctx **ctx);
int he_ctx_destroy(he_ctx *ctx);
int he_ctx_query(const he_ctx *ctx, he_ctx_info *info);
/* Copy the last error message of ctx (NULL ctx: of the last he_setup) into
 * buf (host, len bytes, always NUL-terminated). */
int he_last_error(const he_ctx *ctx, char *buf, int len);

/* he_keygen (Section 2, HE; the relinearisation key is what CCMul needs,
 * Fig. 3(b)): ternary s, pk = (-(a s + e), a), and if with_relin the ell
 * relinearisation keys, all drawn from the ChaCha20 streams of `seed`.  Keys
 * stay resident on the device. */
int he_keygen(he_ctx *ctx, uint64_t seed, int with_relin, he_keys **keys, cudaStream_t stream);
int he_keys_destroy(he_keys *keys);
/* Copy a key in coefficient form into device buffer dst (layouts above). */
int he_keys_export(he_ctx *ctx, const he_keys *keys, int which, void *dst, cudaStream_t stream);
/* Keys from their coefficient forms (device buffers in the layouts above, as
 * written by he_keys_export; rlk may be NULL for keys without relinearisation)
 * -- the resume half of a checkpoint of a serving process.  The NTT forms are
 * recomputed on the device.  INVALID_ARG when sk is not ternary or a residue
 * of pk / rlk is not below its limb modulus (checked on the device; the call
 * synchronises the stream). */
int he_keys_import(he_ctx *ctx, const int64_t *sk, const uint64_t *pk, const uint64_t *rlk, he_keys **keys,
                   cudaStream_t stream);
/* 64-bit fingerprint (FNV-1a) of the parameters that fix a context's
 * arithmetic (N, L, primes, t, digit base, eta, ell, auxiliary primes), to
 * check that a checkpoint is resumed on an identical context. */
int he_ctx_fingerprint(const he_ctx *ctx, uint64_t *fingerprint);

/* he_encrypt, eps(p, pk) of Section 2: pt [n][N] in [0,t) -> ct [n][2][L][N];
 * ct_k = (b u + e1 + Delta m, a u + e2), Delta = floor(q/t), u ternary and
 * e1, e2 CBD drawn from the streams (seed, k).  Values of pt >= t are
 * reduced mod t. */
int he_encrypt(he_ctx *ctx, const he_keys *keys, const uint64_t *pt, int n, uint64_t seed, uint64_t *ct,
               cudaStream_t stream);
/* he_encrypt_many: he_encrypt of n_groups (1 to 4) independent groups in
 * one call, group g encrypting pts[g] [counts[g]][N] with seed seeds[g] into
 * cts[g] [counts[g]][2][L][N] -- bit-identical to n_groups he_encrypt calls,
 * with all groups' transforms sharing the same kernel launches (the client
 * side of a CryptoTrain-P layer encrypts x, w, r^x and r^w, Section 3.2).
 * No paper counterpart beyond eps(p, pk).  INVALID_ARG for n_groups outside
 * [1, 4], a negative count or a missing pointer of a non-empty group. */
int he_encrypt_many(he_ctx *ctx, const he_keys *keys, int n_groups, const uint64_t *const *pts, const int *counts,
                    const uint64_t *seeds, uint64_t *const *cts, cudaStream_t stream);
/* Seed-compressed secret-key encryption (the client of Section 3 holds the
 * secret key; no paper counterpart beyond eps).  he_encrypt_symmetric:
 * pt [n][N] in [0,t) -> c0 [n][L][N] with c0_k = -(a_k s + e_k) + Delta m_k,
 * a_k uniform mod q from the streams (seed, 10, k, limb) and e_k CBD from
 * (seed, 11, k); the ciphertext is (c0_k, a_k), of which only c0 and the
 * 8-byte seed travel (half the bytes of a full ciphertext).
 * he_expand_symmetric: (seed, c0 [n][L][N]) -> ct [n][2][L][N], regenerating
 * a_k on the device.  Both INVALID_ARG for n < 0 or missing buffers. */
int he_encrypt_symmetric(he_ctx *ctx, const he_keys *keys, const uint64_t *pt, int n, uint64_t seed, uint64_t *c0,
                         cudaStream_t stream);
int he_expand_symmetric(he_ctx *ctx, uint64_t seed, int n, const uint64_t *c0, uint64_t *ct, cudaStream_t stream);
/* he_decrypt, sigma(c, sk) of Section 2: m = floor((t [c0 + c1 s]_q +
 * floor(q/2)) / q) mod t, exactly.  ct [n][2][L][N] -> pt [n][N]. */
int he_decrypt(he_ctx *ctx, const he_keys *keys, const uint64_t *ct, int n, uint64_t *pt, cudaStream_t stream);
/* Uniform masks mod t (Section 3.2, preprocessing: r^x, r^w): out [n][N],
 * polynomial k from stream (seed, k). */
int he_sample_masks(he_ctx *ctx, uint64_t seed, int n, uint64_t *out, cudaStream_t stream);
/* Elementwise (a - b) mod t over n values (the shares x - r^x, w - r^w). */
int he_pt_sub(he_ctx *ctx, const uint64_t *a, const uint64_t *b, int64_t n, uint64_t *out, cudaStream_t stream);

/* he_conv_plan: window search of Section 3.3 for `encoding`; fails with
 * PLAN_DOES_NOT_FIT when no window fits the ring.  Besides the input window
 * and channel packing, a plan packs Mn output channels into one kernel
 * polynomial (as the fully connected protocol the paper builds on packs
 * matrix rows), so a layer has MG = ceil(M / Mn) kernel polynomials per
 * channel group; the plan minimises the products MG * G * T per image. */
int he_conv_plan(he_ctx *ctx, const he_conv_shape *shape, int encoding, he_plan **plan);
/* he_plan_search: the same window and output-packing search for ring degree
 * N without a context (host only, no device memory): fills *info exactly as
 * he_plan_query would for the plan he_conv_plan builds.  Used to count
 * polynomial products per image (MG * G * T, Section 3.3 and Fig. 8) for any
 * shape.  Errors as he_conv_plan; INVALID_ARG also for N not a power of two. */
int he_plan_search(int N, const he_conv_shape *shape, int encoding, he_plan_info *info);
/* he_ks_primes: the small primes of the relinearisation key switch that a
 * context with these parameters uses (host only, no device memory; Section 2,
 * CCMul and Fig. 3(b)): the largest primes p < 2^30 with p = 1 mod 2N, as
 * many (2 to 4) as make their product exceed 4 ell N (2^base_log2 - 1)
 * (max q_i - 1), four times the largest |sum_j D_j rlk_{j,i}|.  *np = 0 when
 * a limb is below 2^31 (the key switch then runs over the limbs).  primes:
 * caller array of at least 4 entries.  Errors as he_setup for N, L,
 * prime_bits, q and base_log2. */
int he_ks_primes(const he_params *params, uint64_t *primes, int32_t *np);
int he_plan_destroy(he_plan *plan);
int he_plan_query(const he_plan *plan, he_plan_info *info);

/* Encoders (Section 3.3).  role INPUT: tensor [batch][C][H][W] -> polys
 * [batch][T][G][N]; role KERNEL: tensor [M][C][h][h] -> polys [MG][G][N]
 * (batch ignored).  Values are reduced into [0, t).  The plan's encoding
 * must match the entry point. */
int he_encode_conventional(he_ctx *ctx, const he_plan *plan, int role, const void *tensor, int dtype, int batch,
                           uint64_t *polys, cudaStream_t stream);
int he_encode_correlated(he_ctx *ctx, const he_plan *plan, int role, const void *tensor, int dtype, int batch,
                         uint64_t *polys, cudaStream_t stream);

/* he_cpmul_conv: CPMul + CCAdd over a plan (Fig. 3(c); Section 3.2 online),
 * for each kernel polynomial mg < MG:
 *   out[b][mg][t] = sum_g ct_x[b][t][g] * pt_w[mg][g]
 *                 + sum_g ct_w[mg][g]    * pt_x[b][t][g]
 *                 + ct_add[b][mg][t]
 * Each family is skipped when its ciphertext pointer is NULL (at least one
 * must be given); ct_add may be NULL or equal to ct_out (in place; any other
 * overlap between inputs and ct_out is undefined).  Plaintexts in [0,t) are
 * centre-lifted.  In a depthwise plan (HE_PLAN_DEPTHWISE) only the pairs
 * g = mg * Mn / Cn enter the sums.
 * Shapes: ct_x [batch][T][G][2][L][N], pt_w [MG][G][N], ct_w [MG][G][2][L][N],
 * pt_x [batch][T][G][N], ct_add / ct_out [batch][MG][T][2][L][N].
 * Runs as one batched forward NTT and one fused MAC -> inverse NTT -> add. */
int he_cpmul_conv(he_ctx *ctx, const he_plan *plan, int batch, const uint64_t *ct_x, const uint64_t *pt_w,
                  const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add, uint64_t *ct_out,
                  cudaStream_t stream);

/* he_cpmul_conv_noalloc: the same computation and argument layout as
 * he_cpmul_conv, bit-identical results, but the call allocates no device
 * memory at all: no cudaMalloc, cudaFree or allocating library routine.  It
 * is meant for callers that cannot allocate at call time: serving processes
 * whose device memory is fully reserved up front by another allocator (a
 * framework's caching pool, an inference engine's arena), so that a
 * cudaMalloc inside the library would fail or evict their cache, and
 * latency-critical loops that must not hit the device-wide synchronisation
 * that cudaMalloc/cudaFree imply.  The paper has no counterpart; this is a
 * deployment variant of the CPMul convolution.
 *  - Scratch: a fixed 32 MiB static device array inside the library (held on
 *    every GPU that loads the library until the process exits).  A call whose
 *    NTT-form operands and term table need more returns
 *    HE_ERR_BUDGET_EXCEEDED and does nothing; the online 3x32x32 -> 16 layer
 *    of one image (N = 8192, L = 4, 9 input ciphertexts, 8 output
 *    polynomials after output packing) needs about 7 MiB.
 *  - The term table is written on the device by a kernel from scalar
 *    arguments; the call leaves no host buffer for the stream to read.
 *  - The first call on a device looks up the array's device address once
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - Every call on a device shares the one array and overwrites it (each byte
 *    read is written earlier in the same call, so no state carries over).
 *    Calls whose executions overlap on the GPU (different streams, or
 *    different contexts on the same device) race on it: order them. */
int he_cpmul_conv_noalloc(he_ctx *ctx, const he_plan *plan, int batch, const uint64_t *ct_x, const uint64_t *pt_w,
                          const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add, uint64_t *ct_out,
                          cudaStream_t stream);

/* he_ccmul_precompute: CCMul with relinearisation (Section 2, Motivation;
 * Section 3.2 preprocessing).  Output o sums the tensor products of pairs
 * [o*group, (o+1)*group): d0 = sum a0 b0, d1 = sum a0 b1 + a1 b0, d2 = sum
 * a1 b1 of the centred lifts (exact integers), d_j <- floor((t d_j +
 * floor(q/2)) / q) mod q, (c0, c1) = (d0, d1) + sum_j D_j rlk_j with D_j the
 * base-2^base_log2 digits of d2.  ct_a [n_a][2][L][N], ct_b [n_b][2][L][N];
 * pair_a, pair_b: HOST int32 [n_pairs] indices; out [n_pairs/group][2][L][N].
 * Needs keys made with_relin.  group <= max_ccmul_group.  Outputs run in
 * chunks whose device scratch fits max_ccmul_scratch_bytes (he_params).
 * The sums sum_j D_j rlk_j are exact: where he_ctx_info.ks_primes > 0 they
 * are taken modulo that many primes below 2^30 whose product exceeds four
 * times their largest magnitude and brought to each limb by a CRT, otherwise
 * modulo the limbs themselves; the output bits are the same either way. */
int he_ccmul_precompute(he_ctx *ctx, const he_keys *keys, const uint64_t *ct_a, int n_a, const uint64_t *ct_b,
                        int n_b, const int32_t *pair_a, const int32_t *pair_b, int n_pairs, int group,
                        uint64_t *ct_out, cudaStream_t stream);
/* The same over a plan: out[b][mg][t] = sum_g [r^x][b][t][g] (x) [r^w][mg][g]
 * (the precomputed [r^x r^w] of Section 3.2; also the online [x][w] of the
 * CryptoTrain-B layer, Section 3.1).  ct_rx [batch][T][G][2][L][N],
 * ct_rw [MG][G][2][L][N], out [batch][MG][T][2][L][N].  In a depthwise plan
 * only the pair g = mg * Mn / Cn enters each sum. */
int he_ccmul_conv_precompute(he_ctx *ctx, const he_keys *keys, const he_plan *plan, int batch,
                             const uint64_t *ct_rx, const uint64_t *ct_rw, uint64_t *ct_out, cudaStream_t stream);

/* he_ppmul_conv: PPMul of Section 3.2, p[b][mg][t] = sum_g pt_x[b][t][g] *
 * pt_w[mg][g] in Z_t[x]/(x^N+1).  pt_x [batch][T][G][N], pt_w [MG][G][N],
 * out [batch][MG][T][N].  UNSUPPORTED_PARAMS if t is not an NTT prime. */
int he_ppmul_conv(he_ctx *ctx, const he_plan *plan, int batch, const uint64_t *pt_x, const uint64_t *pt_w,
                  uint64_t *out, cudaStream_t stream);

/* he_decode (Section 3.3, output positions of each encoding): out[b][m][a][c]
 * = centred((pt - sub)[b][m / Mn][tile(a,c)][coef(a,c) + (m mod Mn) Sout]
 * mod t) as int64, centred means v > (t-1)/2 -> v - t.  pt, sub
 * [batch][MG][T][N] (sub may be NULL); out [batch][M][Ho][Wo]. */
int he_decode(he_ctx *ctx, const he_plan *plan, int batch, const uint64_t *pt, const uint64_t *sub, int64_t *out,
              cudaStream_t stream);

/* he_encode_output: the inverse of he_decode's gather (Section 3.3 output
 * positions): polys [batch][MG][T][N] = 0 except
 * polys[b][m / Mn][tile(a,c)][coef(a,c) + (m mod Mn) Sout] = values[b][m][a][c]
 * mod t (values int64 [batch][M][Ho][Wo], negative values as t - |v| mod t).
 * Places a per-output plaintext -- a bias, the beta of a batch-norm layer --
 * where the layer's products land, so that its encryption can be added to
 * the layer's ciphertexts (he_ct_add). */
int he_encode_output(he_ctx *ctx, const he_plan *plan, int batch, const int64_t *values, uint64_t *polys,
                     cudaStream_t stream);
/* he_ct_add (CCAdd, Section 3.2): out = a + b mod q_i over n ciphertexts
 * [n][2][L][N]; out may alias a or b. */
int he_ct_add(he_ctx *ctx, const uint64_t *a, const uint64_t *b, int n, uint64_t *out, cudaStream_t stream);

/* ------------------------------------------------------------------
 * Batched execution of many heterogeneous CPMul convolutions (an execution
 * form of he_cpmul_conv; the paper has no counterpart).  Jobs may use
 * different contexts (ring degree, limbs, primes) and plans on one device.
 *   plain       one he_cpmul_conv call per job (three launches per job);
 *   persistent  per ring degree present, one forward-NTT launch and one
 *               multiply-accumulate/inverse-NTT launch over device work lists
 *               (one limb polynomial per item, the heaviest first): either
 *               persistent CTAs that pull items from a device counter, or one
 *               CTA per item in list order, as he_batch_autotune measures best
 *               (default: persistent, 2 CTAs per SM);
 *   fused       one persistent launch for the whole batch: both phases of
 *               every job and both ring degrees (one degree, or two of which
 *               one is half the other, up to 2^13).  CTAs of the larger
 *               degree's tile take work units from one device counter: all
 *               forward units first (an item of the larger degree, or two of
 *               the smaller, one per half of the CTA), then the
 *               multiply-accumulate units, heaviest first; each of those waits
 *               until its job's forward items are counted done.  Every wait
 *               is bounded (he_batch_set_wait_limit): a unit that runs out
 *               writes HE_ERR_TIMEOUT to the batch's status word, skips its
 *               work, and every CTA stops at its next claim;
 *   graph       the faster of the persistent and the fused forms (as
 *               he_batch_autotune measured; he_batch_set_fused overrides)
 *               captured once in a CUDA graph and replayed (needs a
 *               non-default stream).
 * Results are bit-identical in every form and to a job run alone.  The batch
 * owns one device allocation (made by he_batch_prepare) holding every job's
 * NTT-form operands, term tables and work lists; input and output pointers
 * stay caller-owned and must stay valid while the batch is used.
 * ------------------------------------------------------------------ */
#define HE_BATCH_PLAIN 0
#define HE_BATCH_PERSISTENT 1
#define HE_BATCH_GRAPH 2
#define HE_BATCH_FUSED 3

typedef struct he_batch he_batch;
/* launch configuration chosen by he_batch_autotune for one ring degree */
typedef struct he_batch_tuning {
    int32_t logN;
    int32_t regs_ctas_per_sm;  /* register budget: resident CTAs per SM the kernels are compiled for */
    int32_t grid_ctas_per_sm;  /* persistent CTAs launched per SM; 0: one CTA per work item instead */
    float ms;                  /* best time of the ring degree's two launches */
    int32_t fwd_items, mac_items;
} he_batch_tuning;

int he_batch_create(int device, he_batch **batch);
int he_batch_destroy(he_batch *batch);
int he_batch_last_error(const he_batch *batch, char *buf, int len);
/* Register one job with the arguments of he_cpmul_conv (the ciphertext-input
 * family: ct_x [batch][T][G][2][L][N], pt_w [MG][G][N], ct_add nullable,
 * ct_out [batch][MG][T][2][L][N]).  Returns the job index (>= 0). */
int he_batch_add_cpmul(he_batch *batch, he_ctx *ctx, const he_plan *plan, int n_images, const uint64_t *ct_x,
                       const uint64_t *pt_w, const uint64_t *ct_add, uint64_t *ct_out);
/* The same with both operand families of he_cpmul_conv (the CryptoTrain-P
 * online layer: ct_x * pt_w + ct_w * pt_x + ct_add); either family may be
 * NULL but not both. */
int he_batch_add_cpmul2(he_batch *batch, he_ctx *ctx, const he_plan *plan, int n_images, const uint64_t *ct_x,
                        const uint64_t *pt_w, const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add,
                        uint64_t *ct_out);
/* Freeze the job list: one device allocation for the batch, work lists built
 * and uploaded (synchronous). */
int he_batch_prepare(he_batch *batch);
/* Run the batch in `mode` on `stream` (asynchronous). */
int he_batch_run(he_batch *batch, int mode, cudaStream_t stream);
/* Time every candidate launch configuration of each ring degree on the
 * prepared batch (register budget 1 or 2 CTAs per SM; 1..4 persistent CTAs
 * per SM or one CTA per item; three runs each, best kept), keep the fastest,
 * and report it in
 * out[0 .. min(max_out, n)) with n = number of ring degrees.  Overwrites the
 * jobs' outputs; synchronises; invalidates a captured graph. */
int he_batch_autotune(he_batch *batch, cudaStream_t stream, he_batch_tuning *out, int max_out, int *n);
/* Set the launch configuration of the listed ring degrees (logN,
 * regs_ctas_per_sm 1..2 -- 1 only for logN >= 14 --, grid_ctas_per_sm 0..16;
 * ms and the item counts are ignored), e.g. to reuse an earlier tuning.
 * INVALID_ARG for a value out of range or a degree with no job; invalidates
 * a captured graph. */
int he_batch_set_tuning(he_batch *batch, const he_batch_tuning *tuning, int n);

/* The one-launch (fused) form: whether the batch's degrees allow it, whether
 * the graph form uses it, its register budget (resident CTAs per SM: 1 or 2)
 * and unit count, and the times he_batch_autotune measured for it and for the
 * per-degree launches (0 before autotuning). */
typedef struct he_batch_info {
    int32_t fused_supported, graph_fused, fused_regs_ctas_per_sm, n_units;
    float fused_ms, per_degree_ms;
} he_batch_info;
int he_batch_query(const he_batch *batch, he_batch_info *info);
/* Make the graph form use the fused launch (graph_fused = 1) or the
 * per-degree launches (0), and set the fused register budget (1 or 2; 0
 * keeps it).  UNSUPPORTED_PARAMS if the degrees allow no fused form;
 * invalidates a captured graph. */
int he_batch_set_fused(he_batch *batch, int graph_fused, int regs_ctas_per_sm);
/* Synchronise `stream` and read the status word of the fused form: HE_OK, or
 * HE_ERR_TIMEOUT (message: the unit that gave up) if a unit of a fused run
 * on it ran out of its wait limit; clears the word.  While the word holds a
 * timeout every fused run stops at its first claim and does no work, so
 * check it after fused or graph runs before trusting their outputs. */
int he_batch_status(he_batch *batch, cudaStream_t stream);
/* Polls (each followed by a sleep of at least 256 ns) of a job's counter
 * before a multiply-accumulate unit of the fused form gives up (default
 * 2^22, about a second or more); invalidates a captured graph. */
int he_batch_set_wait_limit(he_batch *batch, long long polls);
/* Test hook of the bounded wait: with hold = 1 the fused form waits for one
 * more forward item of `job` than it has, so that job's multiply-accumulate
 * units run out of their limit (the wait's failure path, made on the host
 * without any fault); hold = 0 restores the count. */
int he_batch_test_hold_job(he_batch *batch, int job, int hold);

/* ------------------------------------------------------------------
 * Continuous-batching request server for CPMul convolution layers (the
 * online phase of the CryptoTrain-P linear layer; a serving form, the paper
 * has no counterpart).  At creation the server reserves hbm_budget_bytes of
 * device memory as its arena and starts a worker thread.  A submitted
 * request (the arguments of he_cpmul_conv, whose keys, precomputed products
 * and operands stay resident in caller memory) waits until its scratch fits
 * in the arena and fewer than max_inflight launch groups are running; the
 * worker then launches up to max_group admitted requests together as
 * work-list kernels (one CTA per item) on the next of n_streams streams, so requests
 * arriving while others run join the next group and groups overlap on the
 * device.  Each result is bit-identical to he_cpmul_conv on the same
 * arguments.  Latency is measured from submission to the worker observing
 * completion (polling every poll_us).
 * ------------------------------------------------------------------ */
typedef struct he_server he_server;
typedef struct he_server_config {
    int32_t device;
    double hbm_budget_bytes;  /* arena size (admission cap) */
    int32_t max_group;        /* requests per launch group */
    int32_t max_inflight;     /* launch groups on the device at once */
    int32_t n_streams;
    int32_t poll_us;          /* completion polling interval (0 -> 20) */
} he_server_config;
typedef struct he_server_report {
    int64_t submitted, completed, images, groups;
    double p50_us, p99_us, mean_us, max_us;
    double span_s;            /* first submission to last completion */
    double arena_peak_bytes, arena_bytes;
} he_server_report;
int he_server_create(const he_server_config *cfg, he_server **server);
/* Queue one request; returns at once.  BUDGET_EXCEEDED if it could never fit
 * the arena.  Buffers must stay valid until the request is done. */
int he_server_submit(he_server *server, he_ctx *ctx, const he_plan *plan, int n_images, const uint64_t *ct_x,
                     const uint64_t *pt_w, const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add,
                     uint64_t *ct_out, int64_t *request_id);
/* *done = 1 once the request completed or was cancelled; latency_us is the
 * submission-to-completion time of a completed request, else -1. */
int he_server_poll(he_server *server, int64_t request_id, int *done, double *latency_us);
/* Withdraw a request that is still waiting for admission (*cancelled = 1; its
 * buffers are never touched); an admitted or finished request is not affected
 * (*cancelled = 0). */
int he_server_cancel(he_server *server, int64_t request_id, int *cancelled);
/* Arena bytes one request would reserve (its scratch plus its share of the
 * work lists), for admission planning; has_x / has_w select the families. */
int he_server_request_bytes(const he_ctx *ctx, const he_plan *plan, int n_images, int has_x, int has_w,
                            double *bytes);
/* Block until every submitted request is done (TIMEOUT after timeout_s). */
int he_server_wait_all(he_server *server, double timeout_s);
/* Statistics over the requests submitted since the last reset. */
int he_server_stats(he_server *server, he_server_report *stats);
int he_server_reset_stats(he_server *server);
/* Drain the queue, stop the worker, release the arena. */
int he_server_destroy(he_server *server);

/* Launch tracing (profiling aid, not part of the paper's method).  While
 * enabled, every kernel launch of the context is bracketed by two CUDA events
 * on its stream and tagged with the kernel family name and its algorithmic
 * bytes (each distinct input polynomial read once, each output written
 * once) and 64-bit modular products.  he_trace_read synchronises the device,
 * folds the recorded launches into one entry per kernel family and call
 * site, named "family.role" (for example mac_intt.relin, ntt_fwd.relin_digits,
 * mac_intt.cpmul), and clears the record.  Tracing adds two event records per
 * launch. */
typedef struct he_trace_entry {
    char name[32];
    int64_t launches;
    double total_ms;     /* sum of event-measured launch durations */
    double bytes;        /* algorithmic bytes, summed over launches */
    double modmuls;      /* 64-bit modular products, summed over launches */
} he_trace_entry;
int he_trace_enable(he_ctx *ctx, int on);
int he_trace_read(he_ctx *ctx, he_trace_entry *out, int max_entries, int *n_entries);

/* ------------------------------------------------------------------
 * Bounds-checked debug build (a sanitizer stand-in; the paper has no
 * counterpart).  libcryptotrain_checks.so is the same library compiled with
 * every kernel's global loads and stores checked against the device ranges
 * the call may touch: the library's own allocations and the allocations that
 * hold the call's device pointers.  An access outside them is skipped (a load
 * yields zero, a store does nothing; nothing traps), and the entry point
 * returns HE_ERR_INVALID_ARG after synchronising the device.  Kernels run
 * several times slower; the request server's asynchronous launches are
 * reported by the next call.
 *   he_checks_enabled      1 in the checks build, 0 otherwise.
 *   he_checks_last_error   the first violation of the last failing call:
 *                          source file and line, address.
 *   he_checks_test_exclude (test hook) leave [ptr, ptr + bytes) out of the
 *                          ranges, so that accesses to that valid memory are
 *                          reported and skipped; ptr = NULL clears it.
 *                          UNSUPPORTED_PARAMS outside the checks build.
 * ------------------------------------------------------------------ */
int he_checks_enabled(void);
int he_checks_last_error(char *buf, int len);
int he_checks_test_exclude(const void *ptr, long long bytes);

#ifdef __cplusplus
}
#endif
#endif
