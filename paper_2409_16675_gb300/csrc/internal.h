// internal.h -- structures shared by the host code and the kernels of the
// GB300 homomorphic linear-layer library.
#pragma once
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <unordered_map>
#include <cuda_runtime.h>

#include "../../include/cryptotrain.h"

typedef uint64_t u64;

namespace he {

constexpr int MAX_MODS = 48;   // Q limbs + aux limbs + t
constexpr int MAXP = 24;       // primes of one CRT basis
constexpr int MAXW = 18;       // 64-bit words of a CRT sum (< n * M)

// Register tile of the NTT kernels: every thread holds 2^kNttTileBits
// coefficients, and passes of up to kNttTileBits stages run in registers.
// The forward factor table's order (below) follows the same pass structure.
constexpr int kNttTileBits = 4;

// One NTT-friendly modulus: constants for Shoup products and its tables.
//   fw[2^s + i]  forward factor of group i at stage s of the merged-twist
//                negacyclic transform, psi^bitrev(2^s + i), stored within its
//                stage at the position the forward pass reads it from:
//                group i = h 2^gb + g (g < 2^gb, gb = the register bits of the
//                stage above the butterfly bit) sits at 2^s + g 2^(s-gb) + h,
//                so that a warp's loads of one g are contiguous
//   iw[2^s + k]  inverse (decimation-in-time, bit-reversed input) factor for
//                offset k at stage s: omega^-(k 2^(n-1-s)), omega = psi^2
//   z[e]         untwist and scale: psi^-e N^-1
// each with its Shoup companion, stored as interleaved (value, companion)
// pairs so one 16-byte load fetches both.
struct ModDev {
    u64 q, twoq;
    u64 nq;            // 2^64 - q
    u64 r64, r64s;     // 2^64 mod q, Shoup companion
    u64 one_s;         // floor(2^64 / q): Shoup companion of 1
    u64 ninv, ninvs;   // N^-1 mod q
    const ulonglong2 *fw, *iw, *z;
    float qf;          // 2^qsh / q in single precision, rounded down
    int qsh;           // max(0, bitlen(q) + 6 - 32): x >> qsh fits 32 bits for x < 64 q
    u64 qinv;          // q^-1 mod 2^64 (Montgomery reduction of the accumulated products)
    int fold;          // products summed between exact folds: min(15, floor((2^64-1)/q) + 1)
};

// A CRT basis {m_i}: M = prod m_i, hat_i = M / m_i, inv_i = hat_i^-1 mod m_i.
struct CrtDev {
    int n, W;                 // primes, words used by sums
    int Wh;                   // words of the largest hat_i = M / m_i (<= W)
    u64 m[MAXP];
    u64 inv[MAXP], invs[MAXP];
    u64 hat[MAXP][MAXW];
    u64 M[MAXW];
    u64 Mhalf[MAXW];          // floor(M / 2)
};

// Overflow estimate of a CRT sum: with m_i' = m_i << sh_i in [2^63, 2^64) and
// c_i = floor(2^127 / m_i'), mulhi(y_i << sh_i, c_i) >> 5 underestimates
// y_i / m_i * 2^58 by less than 1.07.
struct ConvDev {
    u64 sh[MAXP];
    u64 c[MAXP];
};

// Relinearisation over small primes.  The key-switch sum of limb i,
// E_i = sum_j D_j rlk_{j,i} (a product in Z[x]/(x^N + 1) of the digits
// D_j < 2^base and the key residues rlk_{j,i} < q_i), has |E_i| below
// ell N (2^base - 1)(q_i - 1).  It is computed exactly modulo np primes
// p_k < 2^30 with P = prod p_k > 4 max|E_i|, in 32-bit arithmetic, and mapped
// to q_i by a mixed-radix (Garner) CRT: y_0 = r_0, y_k = (((r_k - y_0)
// p_0^-1 - y_1) p_1^-1 - ... - y_{k-1}) p_{k-1}^-1 mod p_k, E' = y_0 + p_0
// (y_1 + p_1 (y_2 + ...)) in [0, P), and E = E' - P when y_{np-1} >
// p_{np-1} / 2 (E' >= 3P/4 exactly when E < 0).
constexpr int kKsMaxPrimes = 4;
struct Mod32Dev {
    uint32_t p, twop;
    uint32_t pinv;               // -p^-1 mod 2^32 (Montgomery reduction of the 64-bit sums)
    uint32_t ones;               // floor(2^32 / p): Shoup companion of 1
    uint32_t r32;                // 2^32 mod p
    uint32_t pad_;
    const uint2 *fw, *iw, *z;    // as in ModDev, (value, floor(value 2^32 / p)) pairs;
                                 // z_e = psi^-e N^-1 2^32 (undoes the Montgomery 2^-32)
};
struct KsDev {
    int np;                      // primes in use (0: the 64-bit path is used)
    int fold;                    // products added to a 64-bit sum between exact folds
    Mod32Dev m[kKsMaxPrimes];
    uint32_t ginv[kKsMaxPrimes][kKsMaxPrimes], ginvs[kKsMaxPrimes][kKsMaxPrimes];  // p_m^-1 mod p_k (m < k)
    uint32_t half_top;           // p_{np-1} / 2
    int pad_;
    u64 pq_s[HE_MAX_LIMBS][kKsMaxPrimes];  // floor(p_m 2^64 / q_i): Shoup companion of p_m (< q_i) mod q_i
    u64 P_q[HE_MAX_LIMBS], P_qs[HE_MAX_LIMBS];  // P mod q_i and companion
};

// Everything the exact kernels need in one device block.
struct ExactDev {
    CrtDev Q;                 // coefficient modulus basis
    CrtDev B;                 // auxiliary basis for the tensor product
    ConvDev Qc, Bc;           // overflow estimates over Q and over B
    // base-conversion tables with Shoup companions:
    // QhatB[j][i] = (Q / q_i) mod b_j, BhatQ[i][j] = (B / b_j) mod q_i, Qhat_t[i] = (Q / q_i) mod t;
    // the ...m tables hold the same values times 2^64 (Montgomery form, for
    // sums of products ended by one Montgomery reduction)
    u64 QhatB[MAXP][MAXP], QhatBm[MAXP][MAXP];
    u64 BhatQ[MAXP][MAXP], BhatQm[MAXP][MAXP];
    u64 Qhat_t[MAXP], Qhat_ts[MAXP];
    u64 Q_bs[MAXP], B_qs[MAXP];  // Shoup companions of Q mod b_j and B mod q_i
    u64 Q_t, Q_ts;               // Q mod t
    // per aux prime b_j: Q mod b_j, floor(Q/2) mod b_j, Q^-1 mod b_j (+Shoup), t mod b_j (+Shoup)
    u64 Q_b[MAXP], Qhalf_b[MAXP], Qinv_b[MAXP], Qinv_bs[MAXP], t_b[MAXP], t_bs[MAXP];
    // per q_i: B mod q_i, floor(Q/2) mod q_i, t mod q_i (+Shoup), Delta mod q_i (+Shoup)
    u64 B_q[MAXP], Qhalf_q[MAXP], t_q[MAXP], t_qs[MAXP], delta_q[MAXP], delta_qs[MAXP];
    // decryption: floor(Q/2) mod t, Q^-1 mod t (+Shoup w.r.t. t), 2^64 mod t (+Shoup), floor(2^64/t)
    u64 t, Qhalf_t, Qinv_t, Qinv_ts, r64_t, r64_ts, one_ts;
    // Folded constants of the rescaling (each a product of the constants
    // above, so one modular product replaces two or three).  With
    // inv_i = (Q/q_i)^-1 mod q_i and c_j = Q^-1 (B/b_j)^-1 mod b_j:
    //   tq[i] = t inv_i, hq[i] = floor(Q/2) inv_i                 (mod q_i)
    //   tb[j] = t c_j, hb[j] = floor(Q/2) c_j, cb[j] = c_j,
    //   QhatBc[j][i] = (Q/q_i) c_j, Q_bc[j] = Q c_j               (mod b_j)
    //   BhatQi[i][j] = (B/b_j) inv_i, B_qi[i] = B inv_i           (mod q_i)
    u64 f_tq[MAXP], f_tqs[MAXP], f_hq[MAXP];
    u64 f_tb[MAXP], f_tbs[MAXP], f_hb[MAXP], f_cb[MAXP], f_cbs[MAXP];
    u64 QhatBc[MAXP][MAXP], QhatBcm[MAXP][MAXP], Q_bc[MAXP], Q_bcs[MAXP];
    u64 BhatQi[MAXP][MAXP], BhatQim[MAXP][MAXP], B_qi[MAXP], B_qis[MAXP];
};

}  // namespace he

struct he_ctx {
    he_params P;
    uint64_t fp = 0;                      // parameter fingerprint (he_ctx_fingerprint)
    int N = 0, logN = 0, L = 0, K = 0;   // K auxiliary primes
    int n_mods = 0;                       // L + K (+1 if the t modulus is available)
    int t_mod = -1;                       // index of the t modulus in the table, -1 if PPMul unsupported
    int ell = 0;
    std::vector<u64> q, aux;
    // device tables
    he::ModDev *d_mods = nullptr;       // [n_mods]
    he::ExactDev *d_exact = nullptr;
    std::vector<void *> allocs;          // twiddle tables etc.
    // host copies
    std::vector<he::ModDev> h_mods;
    he::ExactDev h_exact;
    he::KsDev h_ks;                       // relinearisation over small primes (h_ks.np == 0: not used);
                                          // passed to its kernels by value
    // workspace
    void *ws = nullptr;
    size_t ws_size = 0;
    // small host->device tables cached by content
    std::unordered_map<std::string, void *> table_cache;
    size_t table_cache_bytes = 0;
    std::string err;
    // launch tracing
    bool trace = false;
    struct TraceRec { const char *name, *role; cudaEvent_t a, b; double bytes, modmuls; };
    std::vector<TraceRec> trace_recs;
};

struct he_keys {
    int L = 0, ell = 0, N = 0;
    int device = 0;
    uint64_t fp = 0;         // fingerprint of the parameters the keys were made for
    u64 *sk = nullptr;       // int64 [N] (stored in u64 words)
    u64 *s_ntt = nullptr;    // [L][N] NTT form
    u64 *pk = nullptr;       // [2][L][N] coefficient form
    u64 *pk_ntt = nullptr;   // [2][L][N]
    u64 *rlk = nullptr;      // [ell][2][L][N] coefficient form (or null)
    u64 *rlk_ntt = nullptr;  // [ell][2][L][N]
    uint32_t *rlk32 = nullptr;  // [ell][2][L][np][N] NTT form mod the small primes (contexts with np > 0)
};

struct he_plan {
    he_conv_shape s;
    he_plan_info info;
    int N = 0;
    // tiles: a0,a1,b0,b1,r0,r1,s0,s1 per tile
    std::vector<int> tiles;
    // device index maps
    int32_t *in_map = nullptr;   // [T*G][N] -> index into one image [C][H][W], -1 = zero
    int32_t *ker_map = nullptr;  // [MG][G][N] -> index into w [M][C][h][h], -1 = zero
    int32_t *out_map = nullptr;  // [M][Ho*Wo] -> (mg*T + t)*N + coefficient
    // host copies for tests of the plan
    std::vector<int32_t> h_in_map, h_ker_map, h_out_map;
};
// Whether product pair (kernel polynomial group mg, channel group g) of a plan
// is multiplied: always, except in a depthwise plan, where only the channel
// group holding the Mn outputs of mg is.
inline bool plan_pair(const he_plan *p, int mg, int g) {
    return !p->info.depthwise || g == (mg * p->info.Mn) / p->info.Cn;
}


namespace he {

// Device allocations of the library.  In the bounds-checked build (HE_CHECKS)
// each allocation's range is registered for the kernels' address checks and
// unregistered when freed; otherwise these are cudaMalloc / cudaFree.
#ifdef HE_CHECKS
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
void checks_register(const void *p, size_t bytes);  // a range that is not a cudaMalloc (a __device__ array)
#else
inline cudaError_t dev_alloc(void **p, size_t bytes) { return cudaMalloc(p, bytes); }
inline void dev_free(void *p) { cudaFree(p); }
inline void checks_register(const void *, size_t) {}
#endif

// The role of the launches a call site issues (a string literal, or null);
// the trace reports each launch as "family.role".
extern thread_local const char *g_trace_role;
struct TraceRole {
    const char *prev;
    explicit TraceRole(const char *r) : prev(g_trace_role) { g_trace_role = r; }
    ~TraceRole() { g_trace_role = prev; }
};

// launch tracing: bracket a launch with events when the context traces
struct TraceScope {
    he_ctx *c;
    cudaStream_t st;
    int idx = -1;
    TraceScope(he_ctx *c, cudaStream_t st, const char *name, double bytes, double modmuls);
    ~TraceScope();
};

// host helpers (capi.cu / params.cpp / plan.cpp)
int fail(he_ctx *c, int code, const std::string &msg);
int cuda_check(he_ctx *c, cudaError_t e, const char *what);
int build_tables(he_ctx *c, std::string &err);
int build_plan(he_ctx *c, const he_conv_shape &s, int encoding, he_plan *p, std::string &err);

// ---------------------------------------------------------------- launchers
// Forward NTT of n_polys polynomials over n_limbs consecutive moduli starting
// at mod_base.  Source kinds:
enum SrcKind {
    SRC_RNS = 0,     // u64 residues: src + p*src_stride + limb*N (limbs < split), src2 for limbs >= split
    SRC_T_LIFT = 1,  // u64 values in [0,t) (>= t reduced), centred lift: src + p*src_stride
    SRC_I8 = 2,      // int8 small signed values: src + p*src_stride
    SRC_U32 = 3,     // uint32 small unsigned values (< every modulus): src + p*src_stride
    SRC_T_RAW = 4,   // u64 values taken mod the modulus (used for the t modulus)
};
struct FwdJob {
    const void *src;
    const void *src2;       // second source for limbs >= split (SRC_RNS only)
    long long src_stride;   // elements between polynomials
    long long src2_stride;
    int split;              // limbs < split read from src
    int kind;
    u64 t;                  // for SRC_T_LIFT
    u64 *dst;               // NTT form [p][n_limbs][N] with dst_stride elements between polys
    long long dst_stride;
    int n_polys, n_limbs, mod_base;
};
int launch_fwd(he_ctx *c, const FwdJob &j, cudaStream_t st);
// Several forward jobs over the same moduli (n_limbs, mod_base) in one grid,
// so that small transforms of one call fill the GPU together.
constexpr int kMaxFwdJobs = 4;
struct FwdJobs {
    FwdJob j[kMaxFwdJobs];
    int start[kMaxFwdJobs];
    int n;
};
int launch_fwd_multi(he_ctx *c, const FwdJob *jobs, int n, cudaStream_t st);

// Fused multiply-accumulate in the NTT domain followed by the inverse NTT and
// an epilogue.  Output o, limb l:
//   v = INTT( sum_{k in [ptr[o], ptr[o+1])} A[(ta[k]+l)*N ...] * B[(tb[k]+l)*N ...] )
// Epilogue (natural order, coefficient x):
//   r = v (+ add[o*add_stride + l*N + x]) (+ err8[o*err_stride + x])
//       (+ delta_l * msg[o*msg_stride + x] mod t) (+ g_l * s2[l*N + x]),
//   negated first if `negate` (r = -(v + err) + ...).
struct MacJob {
    const u64 *A, *B;
    const int32_t *ptr, *ta, *tb;
    u64 *out;
    long long out_stride;
    const u64 *add;
    long long add_stride;
    const int8_t *err;          // small error added (after negation rule)
    long long err_stride;
    const u64 *msg;             // plaintext, Delta * msg added to outputs o with o % msg_div == 0
    long long msg_stride;       // message index o / msg_div
    int msg_div;
    const ExactDev *E;          // Delta and t for msg
    const u64 *s2;              // s^2 coefficient form [L][N] times gmul (relin keys)
    const u64 *gmul;            // [n_limbs] multipliers for s2 (device)
    int negate;
    int n_out, n_limbs, mod_base;
    // for tracing: distinct A and B polynomials referenced, total terms
    int n_dist_a, n_dist_b, n_terms;
};
int launch_mac_intt(he_ctx *c, const MacJob &j, cudaStream_t st);
// Several multiply-accumulate jobs over the same moduli in one grid.
constexpr int kMaxMacJobs = 8;
struct MacJobs {
    MacJob j[kMaxMacJobs];
    int start[kMaxMacJobs];
    int n;
};
int launch_mac_multi(he_ctx *c, const MacJob *jobs, int n, cudaStream_t st);

// Work items of the persistent queue kernels (batched execution).
struct FwdItem {            // forward NTT of one limb polynomial
    const void *src;        // this limb's source (kind as in FwdJob)
    u64 *dst;               // this limb's NTT-form output
    const ModDev *mod;      // its modulus (device pointer)
    u64 t;                  // plaintext modulus for SRC_T_LIFT
    int kind;
    int pad_;
};
struct MacItem {            // multiply-accumulate + inverse NTT + add of one output limb
    const u64 *A, *B;       // NTT-form bases (limb 0) of the operands
    const int32_t *ta, *tb; // term tables
    int t0, t1;             // term range
    int limb;
    int pad_;
    u64 *out;               // this limb's output (coefficient form)
    const u64 *add;         // this limb's addend or null
    const ModDev *mod;
};
// The batched form as one persistent launch (fused.cu): a unit is one work
// item of the larger ring degree of the batch (the whole CTA) or up to two
// items of the degree half its size (one per half of the CTA).  Forward
// units come first; a multiply-accumulate unit starts once every forward item
// of its job has been counted in fwd_done.
struct FusedUnit {
    int32_t mac;      // 0: forward items, 1: multiply-accumulate items
    int32_t big;      // 1: one item of the larger degree; 0: up to two of the smaller
    int32_t item[2];  // indices into that degree's forward or MAC item list (-1: none)
    int32_t job[2];   // job of each item
};
struct FusedArgs {
    const FwdItem *fwd_big, *fwd_small;
    const MacItem *mac_big, *mac_small;
    const FusedUnit *units;
    int n_units;
    int *counter;          // next unit (zero at launch)
    int *fwd_done;         // per job: forward items finished (zero at launch)
    const int *fwd_need;   // per job: forward items to wait for
    int *status;           // [0]: 0 or HE_ERR_TIMEOUT, [1]: the unit that gave up
    long long wait_limit;  // polls of a job's counter before a unit gives up
};
// Launch the fused kernel whose larger degree is 2^logN_big (12 or 13),
// compiled for minb (1 or 2) resident CTAs per SM, with `grid` CTAs.
int launch_fused(int logN_big, int minb, const FusedArgs &a, int grid, cudaStream_t st);
// Set the fused kernel's per-device attributes (done by its first launch;
// called before a stream capture so that nothing but the launch is captured).
int fused_set_attributes(int logN_big, int minb);

// One CPMul convolution job (he_cpmul_conv arguments) for the work-list forms.
struct JobDesc {
    he_ctx *c;
    const he_plan *p;
    int batch;
    const u64 *ct_x, *pt_w, *ct_w, *pt_x, *ct_add;
    u64 *out;
};
struct JobLayout {
    size_t a_bytes, b_bytes, t_bytes;  // device scratch: ct NTT forms, pt NTT forms, term table (256-aligned)
    size_t n_fwd, n_mac;               // work items the job adds
};
JobLayout job_layout(const JobDesc &J);
// Work items of a job whose scratch starts at device address dev; terms gets
// the host image of its term table (to be copied to dev + a_bytes + b_bytes).
void job_items(const JobDesc &J, char *dev, std::vector<int32_t> &terms, std::vector<FwdItem> &F,
               std::vector<MacItem> &M);

// A contiguous array of work items and the launch-wide index of its first item.
struct ItemSeg {
    const void *items;
    int begin;
    int pad_;
};
// Persistent kernel over `total` items (fwd: FwdItem, else MacItem) held in
// nseg segments sorted by begin (device table), ring degree 2^logN; minb
// selects the register budget (resident CTAs per SM the kernel is compiled
// for); lazy only when every item's modulus is below 2^57; grid > 0: that
// many persistent CTAs pulling items from *counter (which must be 0);
// grid <= 0: one CTA per item, in list order (counter unused).
int launch_queue(int logN, int minb, bool fwd, bool lazy, const ItemSeg *segs, int nseg, int total, int *counter,
                 int grid, cudaStream_t st);
// true when every limb modulus of the context is below 2^57
bool ctx_lazy(const he_ctx *c);

// sampling (ChaCha20 streams): kinds
enum SampleKind { SAMPLE_TERNARY = 0, SAMPLE_CBD = 1, SAMPLE_UNIFORM_Q = 2, SAMPLE_UNIFORM_T = 3 };
// n_obj objects, object k uses stream (seed, tag, idx0 + k, limb); for
// SAMPLE_UNIFORM_Q every object has n_limbs limbs (limb field = limb index),
// output u64 [k][limb][N]; ternary / CBD output int8 [k][N]; uniform t u64 [k][N].
int launch_encode_output(he_ctx *c, const int32_t *map, int HW, int M, int polys, int batch, const int64_t *values,
                         u64 *out, cudaStream_t st);
int launch_ct_add(he_ctx *c, const u64 *a, const u64 *b, long long n_polys, u64 *out, cudaStream_t st);
int launch_import_sk(he_ctx *c, const int64_t *sk, int8_t *s8, int *bad, cudaStream_t st);
int launch_check_residues(he_ctx *c, const u64 *a, long long n_polys, int *bad, cudaStream_t st);
int launch_sample(he_ctx *c, int kind, uint64_t seed, uint32_t tag, uint32_t idx0, int n_obj, int n_limbs,
                  void *out, cudaStream_t st);
// several sample jobs (each as for launch_sample) in one launch
struct SampleJob {
    int kind;
    uint32_t tag, idx0;
    int n_obj, n_limbs;
    uint64_t seed;
    void *out;
};
constexpr int kMaxSampleJobs = 12;
int launch_sample_multi(he_ctx *c, const SampleJob *jobs, int n, cudaStream_t st);

int launch_base_extend(he_ctx *c, const u64 *src, long long n_polys, u64 *dst_aux, cudaStream_t st);
int launch_scale_round(he_ctx *c, const u64 *d, int n_out, u64 *dq, uint32_t *digits, cudaStream_t st);
// Key switch over the small primes (keyswitch.cu, contexts with h_ks.np > 0).
// Forward: n_polys sources (u32 digits < 2^base at src + p*N, or u64 residues
// of limb p % L at src + p*N when u64_src) to NTT form mod every small
// prime: dst + (p*np + k)*N.
int launch_ks_fwd(he_ctx *c, const void *src, bool u64_src, int n_polys, uint32_t *dst, cudaStream_t st);
// Multiply-accumulate: for output o < n_out, component comp and limb i,
// out[(o*2 + comp)*L*N + i*N + x] = add[same] + E_i[x] mod q_i with
// E_i = sum_j D_{o,j} rlk_{j,comp,i}, D in NTT form at dig + (o*ell + j)*np*N.
// park: device scratch of n_out*L*2*(np-1)*N words.
int launch_ks_mac(he_ctx *c, const uint32_t *dig, const uint32_t *rlk32, const u64 *add, int n_out, u64 *out,
                  uint32_t *park, cudaStream_t st);
// Choose the small primes for a context (params.cpp; np = 0 when the sums do
// not fit four of them or the kernel's shared memory) and upload their tables.
int build_ks(he_ctx *c, std::string &err);
int launch_decrypt_exact(he_ctx *c, const u64 *x, int n, u64 *m, cudaStream_t st);
int launch_encode(he_ctx *c, const int32_t *map, int n_polys, int map_polys, const void *tensor, int dtype,
                  long long tensor_stride, int batch, long long out_batch_polys, u64 *out, cudaStream_t st);
int launch_encode_kernel(he_ctx *c, const int32_t *map, int G, int M, const void *tensor, int dtype,
                         long long per_m, u64 *out, cudaStream_t st);
int launch_decode(he_ctx *c, const int32_t *map, int HW, int M, int polys, int batch, const u64 *pt, const u64 *sub,
                  int64_t *out, cudaStream_t st);
int launch_pt_sub(he_ctx *c, const u64 *a, const u64 *b, long long n, u64 *out, cudaStream_t st);
int launch_copy_sk(he_ctx *c, const int8_t *s8, u64 *sk, cudaStream_t st);

}  // namespace he
