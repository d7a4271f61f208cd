// capi.cu -- the extern "C" entry points declared in include/cryptotrain.h.
// Host logic only: argument checks, workspace carving, term tables, and the
// kernel launch sequence of each operation.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <map>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace he {

static std::string g_setup_err;
static std::mutex g_setup_mu;

std::vector<u64> relin_multipliers(const he_ctx *c);

int fail(he_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_check(he_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HE_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? HE_ERR_OOM : HE_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

// Scratch memory of a context.  Growing it synchronises the device (the old
// buffer may still be read by queued kernels).
static int ws_reserve(he_ctx *c, size_t bytes) {
    if (bytes <= c->ws_size) return HE_OK;
    size_t want = bytes + bytes / 4 + (1 << 20);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_check(c, e, "sync before workspace growth");
    if (c->ws) he::dev_free(c->ws);
    c->ws = nullptr;
    c->ws_size = 0;
    e = he::dev_alloc((void **)&c->ws, want);
    if (e != cudaSuccess) return cuda_check(c, e, "workspace cudaMalloc");
    c->ws_size = want;
    return HE_OK;
}

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <class T> T *take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base + off);
        off += n * sizeof(T);
        return p;
    }
    static size_t round(size_t n) { return (n + 255) & ~(size_t)255; }
};

// device copy of a small host table, cached by content for the context's life
static const void *cached_table(he_ctx *c, const void *data, size_t bytes, int *rc) {
    std::string key((const char *)data, bytes);
    auto it = c->table_cache.find(key);
    if (it != c->table_cache.end()) { *rc = HE_OK; return it->second; }
    void *d = nullptr;
    cudaError_t e = he::dev_alloc((void **)&d, bytes ? bytes : 8);
    if (e != cudaSuccess) { *rc = cuda_check(c, e, "table cudaMalloc"); return nullptr; }
    e = cudaMemcpy(d, data, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { he::dev_free(d); *rc = cuda_check(c, e, "table upload"); return nullptr; }
    c->table_cache.emplace(std::move(key), d);
    c->table_cache_bytes += bytes;
    *rc = HE_OK;
    return d;
}

// CSR term table: ptr[n_out+1], then ta, tb, uploaded as one int32 block
struct Terms {
    std::vector<int32_t> ptr{0}, ta, tb;
    void add(int a, int b) { ta.push_back(a); tb.push_back(b); }
    void close() { ptr.push_back((int32_t)ta.size()); }
    int n_out() const { return (int)ptr.size() - 1; }
};
static int upload_terms_raw(he_ctx *c, const Terms &T, const int32_t **dptr, const int32_t **dta, const int32_t **dtb) {
    std::vector<int32_t> blob;
    blob.push_back((int32_t)T.ptr.size());
    blob.push_back((int32_t)T.ta.size());
    blob.insert(blob.end(), T.ptr.begin(), T.ptr.end());
    blob.insert(blob.end(), T.ta.begin(), T.ta.end());
    blob.insert(blob.end(), T.tb.begin(), T.tb.end());
    int rc;
    const int32_t *d = (const int32_t *)cached_table(c, blob.data(), blob.size() * 4, &rc);
    if (rc) return rc;
    *dptr = d + 2;
    *dta = *dptr + T.ptr.size();
    *dtb = *dta + T.ta.size();
    return HE_OK;
}

static int count_distinct(std::vector<int32_t> v) {
    std::sort(v.begin(), v.end());
    return (int)(std::unique(v.begin(), v.end()) - v.begin());
}
static int upload_terms(he_ctx *c, const Terms &T, MacJob &m) {
    m.n_dist_a = count_distinct(T.ta);
    m.n_dist_b = count_distinct(T.tb);
    m.n_terms = (int)T.ta.size();
    return upload_terms_raw(c, T, &m.ptr, &m.ta, &m.tb);
}

thread_local const char *g_trace_role = nullptr;

// Every traced launch is also an NVTX range (host side, around the enqueue),
// so profilers can select the library's stages by name.
TraceScope::TraceScope(he_ctx *c_, cudaStream_t st_, const char *name, double bytes, double modmuls) : c(c_), st(st_) {
    nvtxRangePushA(name);
    if (!c || !c->trace) return;
    he_ctx::TraceRec r{name, g_trace_role, nullptr, nullptr, bytes, modmuls};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
    cudaEventRecord(r.a, st);
    c->trace_recs.push_back(r);
    idx = (int)c->trace_recs.size() - 1;
}
TraceScope::~TraceScope() {
    if (idx >= 0) cudaEventRecord(c->trace_recs[idx].b, st);
    nvtxRangePop();
}

static MacJob mac_job() {
    MacJob j;
    memset(&j, 0, sizeof j);
    j.msg_div = 1;
    return j;
}
static FwdJob fwd_job() {
    FwdJob j;
    memset(&j, 0, sizeof j);
    j.split = 1 << 30;
    return j;
}

#define TRY(x)                        \
    do {                              \
        int _rc = (x);                \
        if (_rc != HE_OK) return _rc; \
    } while (0)

// Start of a call: select the context's device, and drop the cached term
// tables once they exceed their budget.  No call holds a cached pointer from
// an earlier call, and the synchronisation waits for the kernels that read
// them.
// 64-bit FNV-1a over every parameter that fixes the arithmetic of a context
static uint64_t params_fingerprint(const he_ctx *c) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; i++) { h ^= (v >> (8 * i)) & 0xff; h *= 1099511628211ull; }
    };
    mix((uint64_t)c->N); mix((uint64_t)c->L); mix(c->P.t); mix((uint64_t)c->P.base_log2); mix((uint64_t)c->P.eta);
    mix((uint64_t)c->ell); mix((uint64_t)c->K);
    for (u64 q : c->q) mix(q);
    for (u64 b : c->aux) mix(b);
    return h;
}

// Keys and plans carry the parameters they were made for; a call refuses
// those of another ring (their buffers have other sizes) or other primes.
static int check_keys(he_ctx *c, const he_keys *k) {
    if (k->fp != c->fp || k->N != c->N || k->L != c->L)
        return fail(c, HE_ERR_INVALID_ARG, "keys were made for a context with other parameters");
    return HE_OK;
}
static int check_plan(he_ctx *c, const he_plan *p) {
    if (p->N != c->N) return fail(c, HE_ERR_INVALID_ARG, "plan of another ring degree");
    return HE_OK;
}

static int set_device(he_ctx *c) {
    int rc = cuda_check(c, cudaSetDevice(c->P.device), "cudaSetDevice");
    if (rc) return rc;
    const size_t cap = c->P.max_table_cache_bytes > 0 ? (size_t)c->P.max_table_cache_bytes : (size_t)256 << 20;
    if (c->table_cache_bytes > cap) {
        rc = cuda_check(c, cudaDeviceSynchronize(), "sync before dropping cached tables");
        if (rc) return rc;
        for (auto &kv : c->table_cache) he::dev_free(kv.second);
        c->table_cache.clear();
        c->table_cache_bytes = 0;
    }
    return HE_OK;
}

}  // namespace he

using namespace he;

extern "C" {

int he_setup(const he_params *params, he_ctx **ctx) {
    if (!params || !ctx) return HE_ERR_INVALID_ARG;
    *ctx = nullptr;
    he_ctx *c = new he_ctx();
    c->P = *params;
    std::string err;
    int rc = cuda_check(c, cudaSetDevice(params->device), "cudaSetDevice");
    if (rc == HE_OK) {
        rc = build_tables(c, err);
        if (rc != HE_OK && c->err.empty()) c->err = err;
    }
    if (rc == HE_OK) c->fp = params_fingerprint(c);
    if (rc != HE_OK) {
        std::lock_guard<std::mutex> g(g_setup_mu);
        g_setup_err = c->err;
        he_ctx_destroy(c);
        return rc;
    }
    *ctx = c;
    return HE_OK;
}

int he_ctx_destroy(he_ctx *c) {
    if (!c) return HE_OK;
    cudaSetDevice(c->P.device);
    cudaDeviceSynchronize();
    for (void *p : c->allocs) he::dev_free(p);
    for (auto &kv : c->table_cache) he::dev_free(kv.second);
    if (c->d_mods) he::dev_free(c->d_mods);
    if (c->d_exact) he::dev_free(c->d_exact);
    if (c->ws) he::dev_free(c->ws);
    delete c;
    return HE_OK;
}

int he_ctx_query(const he_ctx *c, he_ctx_info *info) {
    if (!c || !info) return HE_ERR_INVALID_ARG;
    memset(info, 0, sizeof *info);
    info->N = c->N;
    info->L = c->L;
    for (int i = 0; i < c->L; i++) info->q[i] = c->q[i];
    info->t = c->P.t;
    info->ell = c->ell;
    info->n_aux = c->K;
    for (int j = 0; j < c->K && j < 24; j++) info->aux[j] = c->aux[j];
    info->ppmul_ok = c->t_mod >= 0;
    info->ks_primes = c->h_ks.np;
    return HE_OK;
}

int he_last_error(const he_ctx *c, char *buf, int len) {
    if (!buf || len <= 0) return HE_ERR_INVALID_ARG;
    std::string s;
    if (c) s = c->err;
    else {
        std::lock_guard<std::mutex> g(g_setup_mu);
        s = g_setup_err;
    }
    snprintf(buf, (size_t)len, "%s", s.c_str());
    return HE_OK;
}

// ------------------------------------------------------------------ keys
// The relinearisation key in NTT form modulo the context's small primes (for
// the key switch over them), from its coefficient form.
static int ks_key(he_ctx *c, he_keys *k, cudaStream_t st) {
    const int np = c->h_ks.np;
    if (!k->ell || np < 2) return HE_OK;
    const size_t n = (size_t)k->ell * 2 * c->L * np * c->N;
    if (he::dev_alloc((void **)&k->rlk32, n * 4) != cudaSuccess) return fail(c, HE_ERR_OOM, "key allocation");
    return launch_ks_fwd(c, k->rlk, true, k->ell * 2 * c->L, k->rlk32, st);
}

int he_keygen(he_ctx *c, uint64_t seed, int with_relin, he_keys **out, cudaStream_t st) {
    if (!c || !out) return HE_ERR_INVALID_ARG;
    *out = nullptr;
    TraceRole tr_("keygen");
    TRY(set_device(c));
    const int N = c->N, L = c->L, ell = with_relin ? c->ell : 0;
    const size_t LN = (size_t)L * N;
    he_keys *k = new he_keys();
    k->L = L; k->N = N; k->ell = ell; k->device = c->P.device; k->fp = c->fp;
    auto alloc = [&](u64 **p, size_t n) { return he::dev_alloc((void **)p, n * 8) == cudaSuccess; };
    if (!alloc(&k->sk, N) || !alloc(&k->s_ntt, LN) || !alloc(&k->pk, 2 * LN) || !alloc(&k->pk_ntt, 2 * LN) ||
        (ell && (!alloc(&k->rlk, (size_t)ell * 2 * LN) || !alloc(&k->rlk_ntt, (size_t)ell * 2 * LN)))) {
        he_keys_destroy(k);
        return fail(c, HE_ERR_OOM, "key allocation");
    }
    size_t need = Carver::round(N) + Carver::round((size_t)(1 + ell) * N) + Carver::round(LN * 8) + 4096;
    int rc = ws_reserve(c, need);
    if (rc) { he_keys_destroy(k); return rc; }
    Carver cv(c->ws);
    int8_t *s8 = cv.take<int8_t>(N);
    int8_t *e8 = cv.take<int8_t>((size_t)(1 + ell) * N);
    u64 *s2 = cv.take<u64>(LN);
    auto run = [&]() -> int {
        TRY(launch_sample(c, SAMPLE_TERNARY, seed, 1, 0, 1, 1, s8, st));
        TRY(launch_copy_sk(c, s8, k->sk, st));
        FwdJob f = fwd_job();
        f.src = s8; f.kind = SRC_I8; f.src_stride = N; f.dst = k->s_ntt; f.dst_stride = LN;
        f.n_polys = 1; f.n_limbs = L;
        TRY(launch_fwd(c, f, st));
        // pk: a (uniform), e (CBD), b = -(a s + e)
        TRY(launch_sample(c, SAMPLE_UNIFORM_Q, seed, 2, 0, 1, L, k->pk + LN, st));
        TRY(launch_sample(c, SAMPLE_CBD, seed, 3, 0, 1, 1, e8, st));
        f = fwd_job();
        f.src = k->pk + LN; f.kind = SRC_RNS; f.src_stride = LN; f.dst = k->pk_ntt + LN; f.dst_stride = LN;
        f.n_polys = 1; f.n_limbs = L;
        TRY(launch_fwd(c, f, st));
        Terms T1; T1.add(L, 0); T1.close();
        MacJob m = mac_job();
        TRY(upload_terms(c, T1, m));
        m.A = k->pk_ntt; m.B = k->s_ntt; m.out = k->pk; m.out_stride = LN; m.err = e8; m.err_stride = N;
        m.negate = 1; m.n_out = 1; m.n_limbs = L;
        TRY(launch_mac_intt(c, m, st));
        f = fwd_job();
        f.src = k->pk; f.kind = SRC_RNS; f.src_stride = LN; f.dst = k->pk_ntt; f.dst_stride = LN;
        f.n_polys = 1; f.n_limbs = L;
        TRY(launch_fwd(c, f, st));
        if (!ell) return HE_OK;
        // s^2
        MacJob sq = mac_job();
        Terms T0; T0.add(0, 0); T0.close();
        TRY(upload_terms(c, T0, sq));
        sq.A = k->s_ntt; sq.B = k->s_ntt; sq.out = s2; sq.out_stride = LN; sq.n_out = 1; sq.n_limbs = L;
        TRY(launch_mac_intt(c, sq, st));
        // rlk_j = (-(a_j s + e_j) + 2^(base j) s^2, a_j)
        for (int j = 0; j < ell; j++)
            TRY(launch_sample(c, SAMPLE_UNIFORM_Q, seed, 7, (uint32_t)j, 1, L, k->rlk + (2 * (size_t)j + 1) * LN, st));
        TRY(launch_sample(c, SAMPLE_CBD, seed, 8, 0, ell, 1, e8 + N, st));
        f = fwd_job();
        f.src = k->rlk + LN; f.kind = SRC_RNS; f.src_stride = 2 * LN; f.dst = k->rlk_ntt + LN; f.dst_stride = 2 * LN;
        f.n_polys = ell; f.n_limbs = L;
        TRY(launch_fwd(c, f, st));
        Terms TR;
        for (int j = 0; j < ell; j++) { TR.add((2 * j + 1) * L, 0); TR.close(); }
        std::vector<u64> g = relin_multipliers(c);
        int rc2;
        const u64 *dg = (const u64 *)cached_table(c, g.data(), g.size() * 8, &rc2);
        if (rc2) return rc2;
        MacJob r = mac_job();
        TRY(upload_terms(c, TR, r));
        r.A = k->rlk_ntt; r.B = k->s_ntt; r.out = k->rlk; r.out_stride = 2 * LN; r.err = e8 + N; r.err_stride = N;
        r.negate = 1; r.s2 = s2; r.gmul = dg; r.n_out = ell; r.n_limbs = L;
        TRY(launch_mac_intt(c, r, st));
        f = fwd_job();
        f.src = k->rlk; f.kind = SRC_RNS; f.src_stride = 2 * LN; f.dst = k->rlk_ntt; f.dst_stride = 2 * LN;
        f.n_polys = ell; f.n_limbs = L;
        TRY(launch_fwd(c, f, st));
        return ks_key(c, k, st);
    };
    rc = run();
    if (rc) { he_keys_destroy(k); return rc; }
    *out = k;
    return HE_OK;
}

// Keys from their coefficient forms (e.g. a checkpoint written with
// he_keys_export): the NTT forms are recomputed on the device.
int he_keys_import(he_ctx *c, const int64_t *sk, const uint64_t *pk, const uint64_t *rlk, he_keys **out,
                   cudaStream_t st) {
    if (!c || !sk || !pk || !out) return HE_ERR_INVALID_ARG;
    *out = nullptr;
    TRY(set_device(c));
    const int N = c->N, L = c->L, ell = rlk ? c->ell : 0;
    const size_t LN = (size_t)L * N;
    he_keys *k = new he_keys();
    k->L = L; k->N = N; k->ell = ell; k->device = c->P.device; k->fp = c->fp;
    auto alloc = [&](u64 **p, size_t n) { return he::dev_alloc((void **)p, n * 8) == cudaSuccess; };
    if (!alloc(&k->sk, N) || !alloc(&k->s_ntt, LN) || !alloc(&k->pk, 2 * LN) || !alloc(&k->pk_ntt, 2 * LN) ||
        (ell && (!alloc(&k->rlk, (size_t)ell * 2 * LN) || !alloc(&k->rlk_ntt, (size_t)ell * 2 * LN)))) {
        he_keys_destroy(k);
        return fail(c, HE_ERR_OOM, "key allocation");
    }
    int rc = ws_reserve(c, Carver::round(N) + Carver::round(8) + 4096);
    if (rc) { he_keys_destroy(k); return rc; }
    Carver cv(c->ws);
    int8_t *s8 = cv.take<int8_t>(N);
    int *bad = cv.take<int>(2);
    auto run = [&]() -> int {
        TRY(cuda_check(c, cudaMemsetAsync(bad, 0, sizeof(int), st), "import flag"));
        TRY(cuda_check(c, cudaMemcpyAsync(k->sk, sk, (size_t)N * 8, cudaMemcpyDeviceToDevice, st), "sk copy"));
        TRY(cuda_check(c, cudaMemcpyAsync(k->pk, pk, 2 * LN * 8, cudaMemcpyDeviceToDevice, st), "pk copy"));
        if (ell)
            TRY(cuda_check(c, cudaMemcpyAsync(k->rlk, rlk, (size_t)ell * 2 * LN * 8, cudaMemcpyDeviceToDevice, st),
                           "rlk copy"));
        TRY(launch_import_sk(c, (const int64_t *)k->sk, s8, bad, st));
        TRY(launch_check_residues(c, k->pk, 2, bad, st));
        if (ell) TRY(launch_check_residues(c, k->rlk, 2LL * ell, bad, st));
        int h_bad = 0;
        TRY(cuda_check(c, cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "import flag read"));
        TRY(cuda_check(c, cudaStreamSynchronize(st), "import sync"));
        if (h_bad & 1) return fail(c, HE_ERR_INVALID_ARG, "secret key is not ternary");
        if (h_bad & 2) return fail(c, HE_ERR_INVALID_ARG, "key residue not below its limb modulus");
        FwdJob fj[3];
        int nf = 0;
        FwdJob f = fwd_job();
        f.src = s8; f.kind = SRC_I8; f.src_stride = N; f.dst = k->s_ntt; f.dst_stride = LN; f.n_polys = 1; f.n_limbs = L;
        fj[nf++] = f;
        f = fwd_job();
        f.src = k->pk; f.kind = SRC_RNS; f.src_stride = LN; f.dst = k->pk_ntt; f.dst_stride = LN; f.n_polys = 2;
        f.n_limbs = L;
        fj[nf++] = f;
        if (ell) {
            f.src = k->rlk; f.dst = k->rlk_ntt; f.n_polys = 2 * ell;
            fj[nf++] = f;
        }
        TRY(launch_fwd_multi(c, fj, nf, st));
        return ks_key(c, k, st);
    };
    rc = run();
    if (rc) { he_keys_destroy(k); return rc; }
    *out = k;
    return HE_OK;
}

int he_ctx_fingerprint(const he_ctx *c, uint64_t *fp) {
    if (!c || !fp) return HE_ERR_INVALID_ARG;
    *fp = c->fp;
    return HE_OK;
}

int he_keys_destroy(he_keys *k) {
    if (!k) return HE_OK;
    cudaSetDevice(k->device);
    cudaDeviceSynchronize();
    u64 *ps[] = {k->sk, k->s_ntt, k->pk, k->pk_ntt, k->rlk, k->rlk_ntt};
    for (u64 *p : ps)
        if (p) he::dev_free(p);
    if (k->rlk32) he::dev_free(k->rlk32);
    delete k;
    return HE_OK;
}

int he_keys_export(he_ctx *c, const he_keys *k, int which, void *dst, cudaStream_t st) {
    if (!c || !k || !dst) return HE_ERR_INVALID_ARG;
    TRY(check_keys(c, k));
    TRY(set_device(c));
    const size_t LN = (size_t)c->L * c->N;
    const void *src;
    size_t bytes;
    if (which == HE_KEY_SK) { src = k->sk; bytes = (size_t)c->N * 8; }
    else if (which == HE_KEY_PK) { src = k->pk; bytes = 2 * LN * 8; }
    else if (which == HE_KEY_RLK) {
        if (!k->rlk) return fail(c, HE_ERR_INVALID_ARG, "keys have no relinearisation key");
        src = k->rlk; bytes = (size_t)k->ell * 2 * LN * 8;
    } else return fail(c, HE_ERR_INVALID_ARG, "bad key selector");
    return cuda_check(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st), "key export");
}

// ------------------------------------------------------------------ encrypt / decrypt
// Encryption of n_groups groups (each its own plaintexts, count and seed) in
// one forward launch (the u of every ciphertext) and one multiply-accumulate
// launch (both components of every ciphertext: u pk_comp + e (+ Delta m)).
static int encrypt_groups(he_ctx *c, const he_keys *k, int n_groups, const uint64_t *const *pts, const int *counts,
                          const uint64_t *seeds, uint64_t *const *cts, cudaStream_t st) {
    if (!c || !k || n_groups < 1 || n_groups > 4 || !pts || !counts || !seeds || !cts) return HE_ERR_INVALID_ARG;
    TRY(check_keys(c, k));
    TraceRole tr_("enc");
    int n = 0;
    for (int g = 0; g < n_groups; g++) {
        if (counts[g] < 0 || (counts[g] && (!pts[g] || !cts[g]))) return HE_ERR_INVALID_ARG;
        n += counts[g];
    }
    if (!n) return HE_OK;
    TRY(set_device(c));
    const int N = c->N, L = c->L;
    const size_t LN = (size_t)L * N;
    TRY(ws_reserve(c, Carver::round((size_t)n * N) + Carver::round((size_t)n * 2 * N) +
                          Carver::round((size_t)n * LN * 8) + 4096));
    Carver cv(c->ws);
    int8_t *u8 = cv.take<int8_t>((size_t)n * N);
    int8_t *e8 = cv.take<int8_t>((size_t)n * 2 * N);  // per group: e1 of its ciphertexts, then e2
    u64 *un = cv.take<u64>((size_t)n * LN);
    FwdJob fj[4];
    MacJob mj[8];
    SampleJob sj[3 * 4];
    int nf = 0, nm = 0, ns = 0;
    size_t off = 0;
    for (int g = 0; g < n_groups; g++) {
        const int m = counts[g];
        if (!m) continue;
        int8_t *ug = u8 + off * N, *eg = e8 + off * 2 * N;
        u64 *ung = un + off * LN;
        // u (ternary), e1 and e2 (CBD) of every ciphertext of the group
        sj[ns++] = SampleJob{SAMPLE_TERNARY, 4, 0, m, 1, seeds[g], ug};
        sj[ns++] = SampleJob{SAMPLE_CBD, 5, 0, m, 1, seeds[g], eg};
        sj[ns++] = SampleJob{SAMPLE_CBD, 6, 0, m, 1, seeds[g], eg + (size_t)m * N};
        FwdJob f = fwd_job();
        f.src = ug; f.kind = SRC_I8; f.src_stride = N; f.dst = ung; f.dst_stride = LN; f.n_polys = m; f.n_limbs = L;
        fj[nf++] = f;
        // component comp of ciphertext i: u_i pk_comp + e_comp,i (+ Delta m_i for comp 0)
        for (int comp = 0; comp < 2; comp++) {
            Terms T;
            for (int i = 0; i < m; i++) { T.add((int)((off + i) * L), comp * L); T.close(); }
            MacJob mk = mac_job();
            TRY(upload_terms(c, T, mk));
            mk.A = un; mk.B = k->pk_ntt; mk.out = cts[g] + comp * LN; mk.out_stride = 2 * LN;
            mk.err = eg + (size_t)comp * m * N; mk.err_stride = N;
            if (comp == 0) { mk.msg = pts[g]; mk.msg_stride = N; mk.msg_div = 1; mk.E = c->d_exact; }
            mk.n_out = m; mk.n_limbs = L;
            mj[nm++] = mk;
        }
        off += m;
    }
    TRY(launch_sample_multi(c, sj, ns, st));
    TRY(launch_fwd_multi(c, fj, nf, st));
    return launch_mac_multi(c, mj, nm, st);
}

int he_encrypt(he_ctx *c, const he_keys *k, const uint64_t *pt, int n, uint64_t seed, uint64_t *ct,
               cudaStream_t st) {
    if (!c || !k || n < 0 || (n && (!pt || !ct))) return HE_ERR_INVALID_ARG;
    if (!n) return HE_OK;
    return encrypt_groups(c, k, 1, &pt, &n, &seed, &ct, st);
}

int he_encrypt_many(he_ctx *c, const he_keys *k, int n_groups, const uint64_t *const *pts, const int *counts,
                    const uint64_t *seeds, uint64_t *const *cts, cudaStream_t st) {
    return encrypt_groups(c, k, n_groups, pts, counts, seeds, cts, st);
}

// ------------------------------------------------------------------ seed-compressed symmetric encryption
// ct_k = (c0, c1) = (-(a_k s + e_k) + Delta m_k, a_k) with a_k uniform mod q
// from the stream (seed, 10, k, limb) and e_k CBD from (seed, 11, k): the
// client keeps the secret key, sends c0 and the seed, and the receiver
// regenerates c1 = a_k from the seed -- half the bytes of a full ciphertext.
int he_encrypt_symmetric(he_ctx *c, const he_keys *k, const uint64_t *pt, int n, uint64_t seed, uint64_t *c0,
                         cudaStream_t st) {
    if (!c || !k || n < 0 || (n && (!pt || !c0))) return HE_ERR_INVALID_ARG;
    TRY(check_keys(c, k));
    TraceRole tr_("enc_sym");
    if (!n) return HE_OK;
    TRY(set_device(c));
    const int N = c->N, L = c->L;
    const size_t LN = (size_t)L * N;
    TRY(ws_reserve(c, 2 * Carver::round((size_t)n * LN * 8) + Carver::round((size_t)n * N) + 4096));
    Carver cv(c->ws);
    u64 *a = cv.take<u64>((size_t)n * LN);
    u64 *an = cv.take<u64>((size_t)n * LN);
    int8_t *e8 = cv.take<int8_t>((size_t)n * N);
    TRY(launch_sample(c, SAMPLE_UNIFORM_Q, seed, 10, 0, n, L, a, st));
    TRY(launch_sample(c, SAMPLE_CBD, seed, 11, 0, n, 1, e8, st));
    FwdJob f = fwd_job();
    f.src = a; f.kind = SRC_RNS; f.src_stride = LN; f.dst = an; f.dst_stride = LN; f.n_polys = n; f.n_limbs = L;
    TRY(launch_fwd(c, f, st));
    Terms T;
    for (int i = 0; i < n; i++) { T.add(i * L, 0); T.close(); }
    MacJob m = mac_job();
    TRY(upload_terms(c, T, m));
    m.A = an; m.B = k->s_ntt; m.out = c0; m.out_stride = LN;
    m.err = e8; m.err_stride = N; m.negate = 1;
    m.msg = pt; m.msg_stride = N; m.msg_div = 1; m.E = c->d_exact;
    m.n_out = n; m.n_limbs = L;
    return launch_mac_intt(c, m, st);
}

int he_expand_symmetric(he_ctx *c, uint64_t seed, int n, const uint64_t *c0, uint64_t *ct, cudaStream_t st) {
    if (!c || n < 0 || (n && (!c0 || !ct))) return HE_ERR_INVALID_ARG;
    if (!n) return HE_OK;
    TraceRole tr_("expand_sym");
    TRY(set_device(c));
    const int N = c->N, L = c->L;
    const size_t LN = (size_t)L * N;
    TRY(ws_reserve(c, Carver::round((size_t)n * LN * 8) + 4096));
    Carver cv(c->ws);
    u64 *a = cv.take<u64>((size_t)n * LN);
    TRY(launch_sample(c, SAMPLE_UNIFORM_Q, seed, 10, 0, n, L, a, st));
    // ct[k] = (c0[k], a[k]): two strided copies into the [n][2][L][N] layout
    TRY(cuda_check(c, cudaMemcpy2DAsync(ct, 2 * LN * 8, c0, LN * 8, LN * 8, n, cudaMemcpyDeviceToDevice, st),
                   "c0 copy"));
    return cuda_check(c, cudaMemcpy2DAsync(ct + LN, 2 * LN * 8, a, LN * 8, LN * 8, n, cudaMemcpyDeviceToDevice, st),
                      "c1 copy");
}

int he_decrypt(he_ctx *c, const he_keys *k, const uint64_t *ct, int n, uint64_t *pt, cudaStream_t st) {
    if (!c || !k || n < 0 || (n && (!pt || !ct))) return HE_ERR_INVALID_ARG;
    TRY(check_keys(c, k));
    TraceRole tr_("dec");
    if (!n) return HE_OK;
    TRY(set_device(c));
    const int N = c->N, L = c->L;
    const size_t LN = (size_t)L * N;
    TRY(ws_reserve(c, 2 * Carver::round((size_t)n * LN * 8) + 4096));
    Carver cv(c->ws);
    u64 *c1n = cv.take<u64>((size_t)n * LN);
    u64 *x = cv.take<u64>((size_t)n * LN);
    FwdJob f = fwd_job();
    f.src = ct + LN; f.kind = SRC_RNS; f.src_stride = 2 * LN; f.dst = c1n; f.dst_stride = LN; f.n_polys = n; f.n_limbs = L;
    TRY(launch_fwd(c, f, st));
    Terms T;
    for (int i = 0; i < n; i++) { T.add(i * L, 0); T.close(); }
    MacJob m = mac_job();
    TRY(upload_terms(c, T, m));
    m.A = c1n; m.B = k->s_ntt; m.out = x; m.out_stride = LN; m.add = ct; m.add_stride = 2 * LN; m.n_out = n; m.n_limbs = L;
    TRY(launch_mac_intt(c, m, st));
    return launch_decrypt_exact(c, x, n, pt, st);
}

int he_sample_masks(he_ctx *c, uint64_t seed, int n, uint64_t *out, cudaStream_t st) {
    if (!c || n < 0 || (n && !out)) return HE_ERR_INVALID_ARG;
    TRY(set_device(c));
    return launch_sample(c, SAMPLE_UNIFORM_T, seed, 9, 0, n, 1, out, st);
}

int he_pt_sub(he_ctx *c, const uint64_t *a, const uint64_t *b, int64_t n, uint64_t *out, cudaStream_t st) {
    if (!c || n < 0 || (n && (!a || !b || !out))) return HE_ERR_INVALID_ARG;
    TRY(set_device(c));
    return launch_pt_sub(c, a, b, n, out, st);
}

// ------------------------------------------------------------------ plans / encoding
int he_conv_plan(he_ctx *c, const he_conv_shape *s, int encoding, he_plan **out) {
    if (!c || !s || !out) return HE_ERR_INVALID_ARG;
    *out = nullptr;
    TRY(set_device(c));
    he_plan *p = new he_plan();
    std::string err;
    int rc = build_plan(c, *s, encoding, p, err);
    if (rc) { he_plan_destroy(p); return fail(c, rc, err); }
    *out = p;
    return HE_OK;
}

int he_plan_destroy(he_plan *p) {
    if (!p) return HE_OK;
    if (p->in_map) he::dev_free(p->in_map);
    if (p->ker_map) he::dev_free(p->ker_map);
    if (p->out_map) he::dev_free(p->out_map);
    delete p;
    return HE_OK;
}

int he_plan_query(const he_plan *p, he_plan_info *info) {
    if (!p || !info) return HE_ERR_INVALID_ARG;
    *info = p->info;
    return HE_OK;
}

static int encode_common(he_ctx *c, const he_plan *p, int enc, int role, const void *tensor, int dtype, int batch,
                         uint64_t *polys, cudaStream_t st) {
    if (!c || !p || !tensor || !polys) return HE_ERR_INVALID_ARG;
    TRY(check_plan(c, p));
    if (p->info.encoding != enc) return fail(c, HE_ERR_INVALID_ARG, "plan encoding does not match the encoder");
    if (dtype != HE_DTYPE_U8 && dtype != HE_DTYPE_I8 && dtype != HE_DTYPE_I64) return fail(c, HE_ERR_INVALID_ARG, "bad dtype");
    TRY(set_device(c));
    const he_conv_shape &s = p->s;
    if (role == HE_ROLE_INPUT) {
        if (batch < 0) return HE_ERR_INVALID_ARG;
        const int TG = p->info.T * p->info.G;
        return launch_encode(c, p->in_map, TG, TG, tensor, dtype, (long long)s.C * s.H * s.W, batch, TG, polys, st);
    }
    if (role == HE_ROLE_KERNEL)
        return launch_encode_kernel(c, p->ker_map, p->info.G, p->info.MG, tensor, dtype, 0, polys, st);
    return fail(c, HE_ERR_INVALID_ARG, "bad role");
}

int he_encode_conventional(he_ctx *c, const he_plan *p, int role, const void *tensor, int dtype, int batch,
                           uint64_t *polys, cudaStream_t st) {
    return encode_common(c, p, HE_ENC_CONVENTIONAL, role, tensor, dtype, batch, polys, st);
}
int he_encode_correlated(he_ctx *c, const he_plan *p, int role, const void *tensor, int dtype, int batch,
                         uint64_t *polys, cudaStream_t st) {
    return encode_common(c, p, HE_ENC_CORRELATED, role, tensor, dtype, batch, polys, st);
}

// ------------------------------------------------------------------ CPMul conv
int he_cpmul_conv(he_ctx *c, const he_plan *p, int batch, const uint64_t *ct_x, const uint64_t *pt_w,
                  const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add, uint64_t *ct_out,
                  cudaStream_t st) {
    if (!c || !p || batch < 0 || !ct_out || (!ct_x && !ct_w)) return HE_ERR_INVALID_ARG;
    TRY(check_plan(c, p));
    TraceRole tr_("cpmul");
    if ((ct_x && !pt_w) || (ct_w && !pt_x)) return fail(c, HE_ERR_INVALID_ARG, "missing plaintext operand");
    if (!batch) return HE_OK;
    TRY(set_device(c));
    const int N = c->N, L = c->L, T = p->info.T, G = p->info.G, M = p->info.MG;
    const size_t LN = (size_t)L * N;
    const long long nX = ct_x ? (long long)batch * T * G * 2 : 0;   // ct polys (components)
    const long long nW = ct_w ? (long long)M * G * 2 : 0;
    const long long nWp = ct_x ? (long long)M * G : 0;              // pt polys
    const long long nXp = ct_w ? (long long)batch * T * G : 0;
    TRY(ws_reserve(c, Carver::round((nX + nW) * LN * 8) + Carver::round((nWp + nXp) * LN * 8) + 4096));
    Carver cv(c->ws);
    u64 *An = cv.take<u64>((nX + nW) * LN);
    u64 *Bn = cv.take<u64>((nWp + nXp) * LN);
    // every operand to the NTT domain in one launch
    FwdJob fj[4];
    int nf = 0;
    auto add_fwd = [&](const void *src, int kind, long long src_stride, u64 *dst, long long n_polys) {
        FwdJob f = fwd_job();
        f.n_limbs = L; f.src = src; f.kind = kind; f.t = c->P.t; f.src_stride = src_stride;
        f.dst = dst; f.dst_stride = LN; f.n_polys = (int)n_polys;
        fj[nf++] = f;
    };
    if (ct_x) {
        add_fwd(ct_x, SRC_RNS, LN, An, nX);
        add_fwd(pt_w, SRC_T_LIFT, N, Bn, nWp);
    }
    if (ct_w) {
        add_fwd(ct_w, SRC_RNS, LN, An + nX * LN, nW);
        add_fwd(pt_x, SRC_T_LIFT, N, Bn + nWp * LN, nXp);
    }
    TRY(launch_fwd_multi(c, fj, nf, st));
    Terms Tm;
    for (int b = 0; b < batch; b++)
        for (int m = 0; m < M; m++)
            for (int t = 0; t < T; t++)
                for (int comp = 0; comp < 2; comp++) {
                    for (int g = 0; g < G; g++) {
                        if (!plan_pair(p, m, g)) continue;
                        if (ct_x) Tm.add((int)((((long long)(b * T + t) * G + g) * 2 + comp) * L), (m * G + g) * L);
                        if (ct_w) Tm.add((int)((nX + (long long)(m * G + g) * 2 + comp) * L),
                                         (int)((nWp + (long long)(b * T + t) * G + g) * L));
                    }
                    Tm.close();
                }
    MacJob mj = mac_job();
    TRY(upload_terms(c, Tm, mj));
    mj.A = An; mj.B = Bn; mj.out = ct_out; mj.out_stride = LN;
    if (ct_add) { mj.add = ct_add; mj.add_stride = LN; }
    mj.n_out = Tm.n_out(); mj.n_limbs = L;
    return launch_mac_intt(c, mj, st);
}

// ------------------------------------------------------------------ CCMul precompute
int he_ccmul_precompute(he_ctx *c, const he_keys *k, const uint64_t *ct_a, int n_a, const uint64_t *ct_b, int n_b,
                        const int32_t *pair_a, const int32_t *pair_b, int n_pairs, int group, uint64_t *ct_out,
                        cudaStream_t st) {
    if (!c || !k || !ct_a || !ct_b || !pair_a || !pair_b || !ct_out || n_a < 1 || n_b < 1 || n_pairs < 0 ||
        group < 1 || n_pairs % group)
        return HE_ERR_INVALID_ARG;
    TRY(check_keys(c, k));
    if (!k->rlk_ntt) return fail(c, HE_ERR_INVALID_ARG, "keys have no relinearisation key");
    if (group > c->P.max_ccmul_group) return fail(c, HE_ERR_INVALID_ARG, "group exceeds max_ccmul_group");
    for (int i = 0; i < n_pairs; i++)
        if (pair_a[i] < 0 || pair_a[i] >= n_a || pair_b[i] < 0 || pair_b[i] >= n_b)
            return fail(c, HE_ERR_INVALID_ARG, "pair index out of range");
    if (!n_pairs) return HE_OK;
    TRY(set_device(c));
    const int N = c->N, L = c->L, K = c->K, LK = L + K, ell = c->ell;
    const size_t LN = (size_t)L * N, KN = (size_t)K * N, LKN = (size_t)LK * N;
    const int n_out = n_pairs / group;
    // the key switch over the small primes when the context has them (and the
    // keys their form of the relinearisation key), else over the limbs
    const int np = c->h_ks.np;
    const bool ks32 = np >= 2 && k->rlk32;
    // per-output scratch: tensor d (3 polys over Q u B), rescaled d0, d1, digits, digit NTTs
    const size_t dign_words = ks32 ? ((size_t)ell * np * N + 1) / 2 : (size_t)ell * LN;
    const size_t park_words = ks32 ? ((size_t)2 * L * (np - 1) * N + 1) / 2 : 0;  // key switch's parked residues
    const size_t per_out = 3 * LKN * 8 + 2 * LN * 8 + (size_t)ell * N * 4 + dign_words * 8 + park_words * 8;
    // outputs are processed in chunks whose scratch fits the context's budget (default 4 GiB)
    const size_t chunk_budget =
        c->P.max_ccmul_scratch_bytes > 0 ? (size_t)c->P.max_ccmul_scratch_bytes : (size_t)4 << 30;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_out, chunk_budget / per_out));
    size_t need = Carver::round((size_t)(n_a + n_b) * 2 * KN * 8) + Carver::round((size_t)(n_a + n_b) * 2 * LKN * 8) +
                  Carver::round((size_t)chunk * 3 * LKN * 8) + Carver::round((size_t)chunk * 2 * LN * 8) +
                  Carver::round((size_t)chunk * ell * N * 4) + Carver::round((size_t)chunk * dign_words * 8) +
                  Carver::round((size_t)chunk * park_words * 8) + 8192;
    TRY(ws_reserve(c, need));
    Carver cv(c->ws);
    u64 *aux_a = cv.take<u64>((size_t)n_a * 2 * KN);
    u64 *aux_b = cv.take<u64>((size_t)n_b * 2 * KN);
    u64 *An = cv.take<u64>((size_t)n_a * 2 * LKN);
    u64 *Bn = cv.take<u64>((size_t)n_b * 2 * LKN);
    u64 *d = cv.take<u64>((size_t)chunk * 3 * LKN);
    u64 *dq = cv.take<u64>((size_t)chunk * 2 * LN);
    uint32_t *dig = cv.take<uint32_t>((size_t)chunk * ell * N);
    u64 *dign = cv.take<u64>((size_t)chunk * dign_words);
    u64 *park = cv.take<u64>((size_t)chunk * park_words);
    TraceRole tr_("ccmul_in");
    // 1. exact base extension Q -> B of both operands
    TRY(launch_base_extend(c, ct_a, (long long)n_a * 2, aux_a, st));
    TRY(launch_base_extend(c, ct_b, (long long)n_b * 2, aux_b, st));
    // 2. forward NTT over Q u B (both operand sets in one launch)
    FwdJob fab[2];
    FwdJob f = fwd_job();
    f.kind = SRC_RNS; f.split = L; f.n_limbs = LK; f.dst_stride = LKN;
    f.src = ct_a; f.src_stride = LN; f.src2 = aux_a; f.src2_stride = KN; f.dst = An; f.n_polys = n_a * 2;
    fab[0] = f;
    f.src = ct_b; f.src2 = aux_b; f.dst = Bn; f.n_polys = n_b * 2;
    fab[1] = f;
    TRY(launch_fwd_multi(c, fab, 2, st));
    for (int o0 = 0; o0 < n_out; o0 += chunk) {
        const int nc = std::min(chunk, n_out - o0);
        g_trace_role = "tensor";
        // 3. tensor product (summed over the group) + inverse NTT, output o*3 + j
        Terms Tt;
        for (int o = o0; o < o0 + nc; o++)
            for (int j = 0; j < 3; j++) {
                for (int pi = o * group; pi < (o + 1) * group; pi++) {
                    const int a0 = pair_a[pi] * 2 * LK, a1 = a0 + LK, b0 = pair_b[pi] * 2 * LK, b1 = b0 + LK;
                    if (j == 0) Tt.add(a0, b0);
                    else if (j == 1) { Tt.add(a0, b1); Tt.add(a1, b0); }
                    else Tt.add(a1, b1);
                }
                Tt.close();
            }
        MacJob mt = mac_job();
        TRY(upload_terms(c, Tt, mt));
        mt.A = An; mt.B = Bn; mt.out = d; mt.out_stride = LKN; mt.n_out = nc * 3; mt.n_limbs = L;
        // two launches with the same term table: the limbs of Q, whose moduli
        // may allow the lazy transform, and the auxiliary limbs of B (61-bit,
        // never lazy), whose operand and output bases start L limbs on
        TRY(launch_mac_intt(c, mt, st));
        MacJob mb = mt;
        mb.A = An + LN; mb.B = Bn + LN; mb.out = d + LN; mb.n_limbs = K; mb.mod_base = L;
        TRY(launch_mac_intt(c, mb, st));
        g_trace_role = "rescale";
        // 4. exact rescaling by t/q and digits of d2
        TRY(launch_scale_round(c, d, nc, dq, dig, st));
        if (ks32) {
            // 5-6. key switch over the small primes: digits to the NTT domain
            // mod each p_k, then per (output, limb, component) the sums, the
            // inverse transforms and the CRT to q_i, added to (d0, d1)
            g_trace_role = "relin_digits";
            TRY(launch_ks_fwd(c, dig, false, nc * ell, (uint32_t *)dign, st));
            g_trace_role = "relin";
            TRY(launch_ks_mac(c, (const uint32_t *)dign, k->rlk32, dq, nc, ct_out + (size_t)o0 * 2 * LN,
                              (uint32_t *)park, st));
            continue;
        }
        g_trace_role = "relin_digits";
        // 5. digits to the NTT domain over Q
        f = fwd_job();
        f.kind = SRC_U32; f.src = dig; f.src_stride = N; f.dst = dign; f.dst_stride = LN; f.n_polys = nc * ell;
        f.n_limbs = L;
        TRY(launch_fwd(c, f, st));
        g_trace_role = "relin";
        // 6. key switch: (c0, c1) = (d0, d1) + sum_j D_j rlk_j
        Terms Tk;
        for (int o = 0; o < nc; o++)
            for (int comp = 0; comp < 2; comp++) {
                for (int j = 0; j < ell; j++) Tk.add((o * ell + j) * L, (j * 2 + comp) * L);
                Tk.close();
            }
        MacJob mk = mac_job();
        TRY(upload_terms(c, Tk, mk));
        mk.A = dign; mk.B = k->rlk_ntt; mk.out = ct_out + (size_t)o0 * 2 * LN; mk.out_stride = LN; mk.add = dq;
        mk.add_stride = LN; mk.n_out = nc * 2; mk.n_limbs = L;
        TRY(launch_mac_intt(c, mk, st));
    }
    return HE_OK;
}

int he_ccmul_conv_precompute(he_ctx *c, const he_keys *k, const he_plan *p, int batch, const uint64_t *ct_rx,
                             const uint64_t *ct_rw, uint64_t *ct_out, cudaStream_t st) {
    if (!c || !p || !k || batch < 0) return HE_ERR_INVALID_ARG;
    TRY(check_plan(c, p));
    TRY(check_keys(c, k));
    if (!batch) return HE_OK;
    const int T = p->info.T, G = p->info.G, M = p->info.MG;
    std::vector<int32_t> pa, pb;
    for (int b = 0; b < batch; b++)
        for (int m = 0; m < M; m++)
            for (int t = 0; t < T; t++)
                for (int g = 0; g < G; g++)
                    if (plan_pair(p, m, g)) { pa.push_back((b * T + t) * G + g); pb.push_back(m * G + g); }
    // pairs per output: G, or one in a depthwise plan
    return he_ccmul_precompute(c, k, ct_rx, batch * T * G, ct_rw, M * G, pa.data(), pb.data(), (int)pa.size(),
                               p->info.depthwise ? 1 : G, ct_out, st);
}

// ------------------------------------------------------------------ PPMul / decode
int he_ppmul_conv(he_ctx *c, const he_plan *p, int batch, const uint64_t *pt_x, const uint64_t *pt_w, uint64_t *out,
                  cudaStream_t st) {
    if (!c || !p || batch < 0 || (batch && (!pt_x || !pt_w || !out))) return HE_ERR_INVALID_ARG;
    TRY(check_plan(c, p));
    if (c->t_mod < 0) return fail(c, HE_ERR_UNSUPPORTED_PARAMS, "t is not an NTT prime for this N");
    if (!batch) return HE_OK;
    TRY(set_device(c));
    TraceRole tr_("ppmul");
    const int N = c->N, T = p->info.T, G = p->info.G, M = p->info.MG;
    const long long nX = (long long)batch * T * G, nW = (long long)M * G;
    TRY(ws_reserve(c, Carver::round((nX + nW) * N * 8) + 4096));
    Carver cv(c->ws);
    u64 *Xn = cv.take<u64>(nX * N);
    u64 *Wn = cv.take<u64>(nW * N);
    FwdJob fxw[2];
    FwdJob f = fwd_job();
    f.kind = SRC_T_RAW; f.n_limbs = 1; f.mod_base = c->t_mod; f.dst_stride = N; f.src_stride = N;
    f.src = pt_x; f.dst = Xn; f.n_polys = (int)nX;
    fxw[0] = f;
    f.src = pt_w; f.dst = Wn; f.n_polys = (int)nW;
    fxw[1] = f;
    TRY(launch_fwd_multi(c, fxw, 2, st));
    Terms Tm;
    for (int b = 0; b < batch; b++)
        for (int m = 0; m < M; m++)
            for (int t = 0; t < T; t++) {
                for (int g = 0; g < G; g++)
                    if (plan_pair(p, m, g)) Tm.add((b * T + t) * G + g, m * G + g);
                Tm.close();
            }
    MacJob mj = mac_job();
    TRY(upload_terms(c, Tm, mj));
    mj.A = Xn; mj.B = Wn; mj.out = out; mj.out_stride = N; mj.n_out = Tm.n_out(); mj.n_limbs = 1; mj.mod_base = c->t_mod;
    return launch_mac_intt(c, mj, st);
}

int he_decode(he_ctx *c, const he_plan *p, int batch, const uint64_t *pt, const uint64_t *sub, int64_t *out,
              cudaStream_t st) {
    if (!c || !p || batch < 0 || (batch && (!pt || !out))) return HE_ERR_INVALID_ARG;
    TRY(check_plan(c, p));
    TRY(set_device(c));
    return launch_decode(c, p->out_map, p->info.Ho * p->info.Wo, p->s.M, p->info.MG * p->info.T, batch, pt, sub, out,
                         st);
}

int he_encode_output(he_ctx *c, const he_plan *p, int batch, const int64_t *values, uint64_t *polys,
                     cudaStream_t st) {
    if (!c || !p || batch < 0 || (batch && (!values || !polys))) return HE_ERR_INVALID_ARG;
    TRY(check_plan(c, p));
    TRY(set_device(c));
    return launch_encode_output(c, p->out_map, p->info.Ho * p->info.Wo, p->s.M, p->info.MG * p->info.T, batch, values,
                                polys, st);
}

int he_ct_add(he_ctx *c, const uint64_t *a, const uint64_t *b, int n, uint64_t *out, cudaStream_t st) {
    if (!c || n < 0 || (n && (!a || !b || !out))) return HE_ERR_INVALID_ARG;
    TRY(set_device(c));
    return launch_ct_add(c, a, b, (long long)n * 2, out, st);
}

#ifndef HE_CHECKS
// the bounds-checked build's calls (checks.cpp); this build has no checks
int he_checks_enabled(void) { return 0; }
int he_checks_last_error(char *buf, int len) {
    if (!buf || len <= 0) return HE_ERR_INVALID_ARG;
    buf[0] = 0;
    return HE_OK;
}
int he_checks_test_exclude(const void *, long long) { return HE_ERR_UNSUPPORTED_PARAMS; }
#endif

int he_trace_enable(he_ctx *c, int on) {
    if (!c) return HE_ERR_INVALID_ARG;
    c->trace = on != 0;
    return HE_OK;
}

int he_trace_read(he_ctx *c, he_trace_entry *out, int max_entries, int *n_entries) {
    if (!c || !n_entries || (max_entries > 0 && !out)) return HE_ERR_INVALID_ARG;
    TRY(set_device(c));
    TRY(cuda_check(c, cudaDeviceSynchronize(), "trace sync"));
    std::map<std::string, he_trace_entry> acc;
    for (auto &r : c->trace_recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        const std::string key = r.role ? std::string(r.name) + "." + r.role : std::string(r.name);
        he_trace_entry &e = acc[key];
        snprintf(e.name, sizeof e.name, "%s", key.c_str());
        e.launches++;
        e.total_ms += ms;
        e.bytes += r.bytes;
        e.modmuls += r.modmuls;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->trace_recs.clear();
    int n = 0;
    for (auto &kv : acc) {
        if (n < max_entries) out[n] = kv.second;
        n++;
    }
    *n_entries = n;
    return HE_OK;
}

}  // extern "C"
