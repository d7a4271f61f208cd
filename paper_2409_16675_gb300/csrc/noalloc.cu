// noalloc.cu -- he_cpmul_conv_noalloc: the CPMul + CCAdd convolution of
// he_cpmul_conv with its scratch memory in a fixed, statically sized device
// array instead of the context's growable workspace, so the call itself
// never allocates device memory.
//
// The scratch holds the NTT forms of the input ciphertexts and plaintexts and
// the term table of the fused multiply-accumulate.  Its host-visible address
// is looked up once per device with cudaGetSymbolAddress (the array's name in
// host code is only a host-side stand-in, not a device address).
#include <cstring>
#include <mutex>
#include <vector>
#include <algorithm>

#include "internal.h"

namespace {

// Maximum scratch of one call: 32 MiB, resident on every GPU that loads the
// library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 256;
void *g_noalloc_addr[kMaxDevices] = {};

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

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
    const int N = c->N, L = c->L, T = p->info.T, G = p->info.G, M = p->info.MG;
    const size_t LN = (size_t)L * N;
    const long long nX = ct_x ? (long long)batch * T * G * 2 : 0;
    const long long nW = ct_w ? (long long)M * G * 2 : 0;
    const long long nWp = ct_x ? (long long)M * G : 0;
    const long long nXp = ct_w ? (long long)batch * T * G : 0;
    // term table: ptr[n_out + 1], ta[n_terms], tb[n_terms]
    std::vector<int32_t> ptr(1, 0), ta, tb;
    for (int b = 0; b < batch; b++)
        for (int m = 0; m < M; m++)
            for (int t = 0; t < T; t++)
                for (int comp = 0; comp < 2; comp++) {
                    for (int g = 0; g < G; g++) {
                        if (!plan_pair(p, m, g)) continue;
                        if (ct_x) {
                            ta.push_back((int32_t)((((long long)(b * T + t) * G + g) * 2 + comp) * L));
                            tb.push_back((m * G + g) * L);
                        }
                        if (ct_w) {
                            ta.push_back((int32_t)((nX + (long long)(m * G + g) * 2 + comp) * L));
                            tb.push_back((int32_t)((nWp + (long long)(b * T + t) * G + g) * L));
                        }
                    }
                    ptr.push_back((int32_t)ta.size());
                }
    const size_t bytesA = round256((size_t)(nX + nW) * LN * 8), bytesB = round256((size_t)(nWp + nXp) * LN * 8);
    const size_t bytesT = round256((ptr.size() + 2 * ta.size()) * 4);
    if (bytesA + bytesB + bytesT > kNoAllocScratchBytes)
        return fail(c, HE_ERR_BUDGET_EXCEEDED,
                    "he_cpmul_conv_noalloc: this call needs " + std::to_string(bytesA + bytesB + bytesT) +
                        " bytes of scratch, more than the fixed 32 MiB (33554432 bytes); use he_cpmul_conv or a smaller batch");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *a = nullptr;
            rc = cuda_check(c, cudaGetSymbolAddress(&a, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)");
            if (rc) return rc;
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
    std::vector<int32_t> blob(ptr);
    blob.insert(blob.end(), ta.begin(), ta.end());
    blob.insert(blob.end(), tb.begin(), tb.end());
    rc = cuda_check(c, cudaMemcpyAsync(dterms, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice, st),
                    "term table copy");
    if (rc) return rc;
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
    mj.ta = dterms + ptr.size();
    mj.tb = mj.ta + ta.size();
    mj.A = An; mj.B = Bn; mj.out = ct_out; mj.out_stride = LN;
    if (ct_add) { mj.add = ct_add; mj.add_stride = LN; }
    mj.n_out = (int)ptr.size() - 1;
    mj.n_limbs = L;
    {
        std::vector<int32_t> da(ta), db(tb);
        std::sort(da.begin(), da.end());
        std::sort(db.begin(), db.end());
        mj.n_dist_a = (int)(std::unique(da.begin(), da.end()) - da.begin());
        mj.n_dist_b = (int)(std::unique(db.begin(), db.end()) - db.begin());
        mj.n_terms = (int)ta.size();
    }
    return launch_mac_intt(c, mj, st);
}
