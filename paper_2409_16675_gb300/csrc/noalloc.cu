// noalloc.cu -- he_cpmul_conv_noalloc: the CPMul + CCAdd convolution of
// he_cpmul_conv with its scratch memory in a fixed, statically sized device
// array instead of the context's growable workspace, so the call itself
// never allocates device memory.
//
// The scratch holds the NTT forms of the input ciphertexts and plaintexts and
// the term table of the fused multiply-accumulate; a small kernel writes the
// table from scalar arguments, so the stream's work reads no host memory.
// The array's device address is looked up once per device with
// cudaGetSymbolAddress (its name in host code is only a host-side stand-in,
// not a device address).
#include <cstring>
#include <mutex>

#include "internal.h"
#include "checks.cuh"

namespace {

// Maximum scratch of one call: 32 MiB, resident on every GPU that loads the
// library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 256;
void *g_noalloc_addr[kMaxDevices] = {};

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

// Scalars from which k_noalloc_terms writes the term table of one call.
struct NoAllocTermArgs {
    int32_t *ptr, *ta, *tb;
    long long n_out, per_out, nX, nWp;
    int M, T, G, L, Mn, Cn;
    int has_x, has_w, depthwise;
};

// Thread o writes ptr[o] and, for o < n_out, the terms of output o =
// ((b M + m) T + t) 2 + comp: for each channel group g paired with m, the
// input-family term (A = [x] polynomial (b, t, g, comp), B = pt_w (m, g)) and
// then the weight-family term (A = [w] polynomial (m, g, comp), B = pt_x
// (b, t, g)), offsets in limb polynomials.
__global__ void k_noalloc_terms(const NoAllocTermArgs a) {
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o > a.n_out) return;
    HE_ST(a.ptr + o, (int32_t)(o * a.per_out));
    if (o == a.n_out) return;
    const int comp = (int)(o & 1);
    long long r = o >> 1;
    const int t = (int)(r % a.T);
    r /= a.T;
    const int m = (int)(r % a.M);
    const long long b = r / a.M;
    long long k = o * a.per_out;
    for (int g = 0; g < a.G; g++) {
        if (a.depthwise && g != (m * a.Mn) / a.Cn) continue;
        if (a.has_x) {
            HE_ST(a.ta + k, (int32_t)((((b * a.T + t) * a.G + g) * 2 + comp) * a.L));
            HE_ST(a.tb + k, (int32_t)(((long long)m * a.G + g) * a.L));
            k++;
        }
        if (a.has_w) {
            HE_ST(a.ta + k, (int32_t)((a.nX + ((long long)m * a.G + g) * 2 + comp) * a.L));
            HE_ST(a.tb + k, (int32_t)((a.nWp + (b * a.T + t) * a.G + g) * a.L));
            k++;
        }
    }
}

}  // namespace

using namespace he;

extern "C" int he_cpmul_conv_noalloc(he_ctx *c, const he_plan *p, int batch, const uint64_t *ct_x,
                                     const uint64_t *pt_w, const uint64_t *ct_w, const uint64_t *pt_x,
                                     const uint64_t *ct_add, uint64_t *ct_out, cudaStream_t st) {
    if (!c || !p || batch < 0 || !ct_out || (!ct_x && !ct_w)) return HE_ERR_INVALID_ARG;
    if (p->N != c->N) return fail(c, HE_ERR_INVALID_ARG, "plan of another ring degree");
    if ((ct_x && !pt_w) || (ct_w && !pt_x)) return fail(c, HE_ERR_INVALID_ARG, "missing plaintext operand");
    if (!batch) return HE_OK;
    const int dev = c->P.device;
    if (dev < 0 || dev >= kMaxDevices) return fail(c, HE_ERR_INVALID_ARG, "device ordinal out of range");
    int rc = cuda_check(c, cudaSetDevice(dev), "cudaSetDevice");
    if (rc) return rc;
    TraceRole tr_("cpmul_noalloc");
    const int N = c->N, L = c->L, T = p->info.T, G = p->info.G, M = p->info.MG;
    const size_t LN = (size_t)L * N;
    const long long nX = ct_x ? (long long)batch * T * G * 2 : 0;
    const long long nW = ct_w ? (long long)M * G * 2 : 0;
    const long long nWp = ct_x ? (long long)M * G : 0;
    const long long nXp = ct_w ? (long long)batch * T * G : 0;
    // The term table (ptr[n_out + 1], ta[n_terms], tb[n_terms]) is written on
    // the device by k_noalloc_terms from the scalars below; no host buffer is
    // read by the stream's work after this call returns.  Outputs run over
    // (b, m, t, comp); each takes the same number of (m, g) pairs: every g in a
    // dense plan, the one channel group g = m Mn / Cn in a depthwise plan.
    const int per_m = p->info.depthwise ? 1 : G;
    int n_pairs = 0, n_gx = 0;
    for (int m = 0; m < M; m++) {
        int cnt = 0;
        for (int g = 0; g < G; g++) cnt += plan_pair(p, m, g) ? 1 : 0;
        if (cnt != per_m) return fail(c, HE_ERR_INVALID_ARG, "plan with an uneven number of product pairs");
        n_pairs += cnt;
    }
    for (int g = 0; g < G; g++) {
        bool used = false;
        for (int m = 0; m < M && !used; m++) used = plan_pair(p, m, g);
        n_gx += used ? 1 : 0;
    }
    const int n_fam = (ct_x ? 1 : 0) + (ct_w ? 1 : 0);
    const long long n_out = (long long)batch * M * T * 2;
    const long long per_out = (long long)per_m * n_fam;
    const long long n_terms = n_out * per_out;
    const size_t bytesA = round256((size_t)(nX + nW) * LN * 8), bytesB = round256((size_t)(nWp + nXp) * LN * 8);
    const size_t bytesT = round256((size_t)(n_out + 1 + 2 * n_terms) * 4);
    if (bytesA + bytesB + bytesT > kNoAllocScratchBytes)
        return fail(c, HE_ERR_BUDGET_EXCEEDED,
                    "he_cpmul_conv_noalloc: this call needs " + std::to_string(bytesA + bytesB + bytesT) +
                        " bytes of scratch, more than the fixed 32 MiB (33554432 bytes); use he_cpmul_conv or a smaller batch");
    // within the cap every polynomial offset and term index is below 2^22, so
    // the table's int32 entries cannot overflow
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *a = nullptr;
            rc = cuda_check(c, cudaGetSymbolAddress(&a, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)");
            if (rc) return rc;
            checks_register(a, kNoAllocScratchBytes);  // (bounds-checked build only)
            g_noalloc_addr[dev] = a;
        }
        base = g_noalloc_addr[dev];
    }
    char *s = (char *)base;
    u64 *An = (u64 *)s;
    u64 *Bn = (u64 *)(s + bytesA);
    int32_t *dterms = (int32_t *)(s + bytesA + bytesB);
    // every scratch byte that is read below is written first in this call, so
    // the previous call's contents never leak into the result
    {
        NoAllocTermArgs a;
        a.ptr = dterms;
        a.ta = dterms + n_out + 1;
        a.tb = a.ta + n_terms;
        a.n_out = n_out; a.per_out = per_out;
        a.M = M; a.T = T; a.G = G; a.L = L;
        a.nX = nX; a.nWp = nWp;
        a.has_x = ct_x != nullptr; a.has_w = ct_w != nullptr;
        a.depthwise = p->info.depthwise; a.Mn = p->info.Mn; a.Cn = p->info.Cn;
        const long long threads = n_out + 1;
        k_noalloc_terms<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(a);
        rc = cuda_check(c, cudaGetLastError(), "k_noalloc_terms");
        if (rc) return rc;
    }
    FwdJob fj[4];
    int nf = 0;
    auto add_fwd = [&](const void *src, int kind, long long src_stride, u64 *dst, long long n_polys) {
        FwdJob f;
        memset(&f, 0, sizeof f);
        f.split = 1 << 30;
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
    if ((rc = launch_fwd_multi(c, fj, nf, st))) return rc;
    MacJob mj;
    memset(&mj, 0, sizeof mj);
    mj.msg_div = 1;
    mj.ptr = dterms;
    mj.ta = dterms + n_out + 1;
    mj.tb = mj.ta + n_terms;
    mj.A = An; mj.B = Bn; mj.out = ct_out; mj.out_stride = LN;
    if (ct_add) { mj.add = ct_add; mj.add_stride = LN; }
    mj.n_out = (int)n_out;
    mj.n_limbs = L;
    // distinct operand polynomials (launch tracing only): the two families'
    // index ranges are disjoint
    mj.n_dist_a = (int)((ct_x ? (long long)batch * T * 2 * n_gx : 0) + (ct_w ? 2ll * n_pairs : 0));
    mj.n_dist_b = (int)((ct_x ? (long long)n_pairs : 0) + (ct_w ? (long long)batch * T * n_gx : 0));
    mj.n_terms = (int)n_terms;
    return launch_mac_intt(c, mj, st);
}

HE_CHECKS_UNIT(noalloc)
