// checks.cpp -- host side of the bounds-checked debug build (-DHE_CHECKS only).
//
// Keeps the ranges the kernels may touch: every device allocation the library
// makes (registered by dev_alloc, removed by dev_free) and the allocation
// that holds each device pointer passed to an entry point (found with the
// driver's address-range query).  Before each checked call the merged,
// sorted table is copied to every translation unit's device copy; after the
// call the device is synchronised and the units' error words are read: any
// violation makes the call return HE_ERR_INVALID_ARG with the first bad
// address and source line in he_checks_last_error.
#ifdef HE_CHECKS
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "checks.cuh"
#include "internal.h"

// each unit's table and error word (HE_CHECKS_UNIT in ntt.cu, fused.cu,
// exact.cu, noalloc.cu, keyswitch.cu)
int checks_put_ntt(const he::CheckTable *);
int checks_take_ntt(he::CheckError *);
int checks_put_fused(const he::CheckTable *);
int checks_take_fused(he::CheckError *);
int checks_put_exact(const he::CheckTable *);
int checks_take_exact(he::CheckError *);
int checks_put_noalloc(const he::CheckTable *);
int checks_take_noalloc(he::CheckError *);
int checks_put_keyswitch(const he::CheckTable *);
int checks_take_keyswitch(he::CheckError *);

namespace he {
namespace {

std::mutex g_mu;
std::map<unsigned long long, unsigned long long> g_lib;     // library allocations: lo -> hi
std::map<unsigned long long, unsigned long long> g_caller;  // allocations holding caller buffers
unsigned long long g_hole_lo = 0, g_hole_hi = 0;            // test hook: a range left out of the table
std::string g_last;

typedef CUresult (*AddrRangeFn)(CUdeviceptr *, size_t *, CUdeviceptr);
AddrRangeFn addr_range() {
    static AddrRangeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuMemGetAddressRange", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (AddrRangeFn)p;
    }
    return fn;
}

// the sorted, merged table of every registered range, with the test hook's
// hole [g_hole_lo, g_hole_hi) cut out
void build_table(CheckTable *t) {
    std::vector<std::pair<unsigned long long, unsigned long long>> v, m;
    for (auto &kv : g_lib) v.push_back(kv);
    for (auto &kv : g_caller) v.push_back(kv);
    std::sort(v.begin(), v.end());
    for (auto &r : v) {
        if (r.second <= r.first) continue;
        if (!m.empty() && r.first <= m.back().second) m.back().second = std::max(m.back().second, r.second);
        else m.push_back(r);
    }
    t->n = 0;
    auto add = [&](unsigned long long lo, unsigned long long hi) {
        if (hi > lo && t->n < kCheckRanges) { t->lo[t->n] = lo; t->hi[t->n] = hi; t->n++; }
    };
    for (auto &r : m) {
        if (g_hole_hi > g_hole_lo && g_hole_lo < r.second && g_hole_hi > r.first) {
            add(r.first, std::max(r.first, g_hole_lo));
            add(std::min(r.second, g_hole_hi), r.second);
        } else {
            add(r.first, r.second);
        }
    }
}

int put_all(const CheckTable *t) {
    return checks_put_ntt(t) | checks_put_fused(t) | checks_put_exact(t) | checks_put_noalloc(t) |
           checks_put_keyswitch(t);
}

// read (and clear) every unit's error word; the first violation's text
unsigned take_all(std::string &text) {
    struct U { const char *name; int (*take)(CheckError *); } units[] = {
        {"ntt.cu / ntt_core.cuh", checks_take_ntt}, {"fused.cu", checks_take_fused},
        {"exact.cu", checks_take_exact}, {"noalloc.cu", checks_take_noalloc},
        {"keyswitch.cu", checks_take_keyswitch}};
    unsigned total = 0;
    for (auto &u : units) {
        CheckError e = {0, 0, 0};
        if (u.take(&e)) continue;
        if (e.count && !total) {
            char buf[160];
            snprintf(buf, sizeof buf, "out-of-range device access in %s line %u at address 0x%llx", u.name, e.line,
                     e.addr);
            text = buf;
        }
        total += e.count;
    }
    return total;
}

}  // namespace

// An allocation made inside a call (keys, a grown workspace, a term table)
// must reach the device table before that call's kernels run: register it,
// let earlier work finish, and upload the table again.
void republish() {
    static CheckTable t;  // 64 KiB: kept off the stack
    cudaDeviceSynchronize();
    build_table(&t);
    put_all(&t);
}

cudaError_t dev_alloc(void **p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> g(g_mu);
        g_lib[(unsigned long long)*p] = (unsigned long long)*p + bytes;
        republish();
    }
    return e;
}

void dev_free(void *p) {
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_lib.erase((unsigned long long)p);
    }
    cudaFree(p);
}

void checks_register(const void *p, size_t bytes) {
    std::lock_guard<std::mutex> g(g_mu);
    g_lib[(unsigned long long)p] = (unsigned long long)p + bytes;
    republish();
}

// One checked entry-point call: registers the allocations holding its
// pointer arguments, uploads the table, and after the call synchronises and
// reads the error words.
struct CheckCall {
    int pre = 0;
    std::string pre_text;
    CheckCall() {
        // violations of earlier asynchronous work (the request server's
        // worker) are reported by the next call
        cudaDeviceSynchronize();
        std::lock_guard<std::mutex> g(g_mu);
        if (take_all(pre_text)) pre = 1;
    }
    void arg(const void *p) {
        if (!p || !addr_range()) return;
        CUdeviceptr base = 0;
        size_t size = 0;
        if (addr_range()(&base, &size, (CUdeviceptr)p) != CUDA_SUCCESS) {
            cudaGetLastError();  // a host pointer
            return;
        }
        std::lock_guard<std::mutex> g(g_mu);
        g_caller[(unsigned long long)base] = (unsigned long long)base + size;
    }
    void finish_setup() {
        std::lock_guard<std::mutex> g(g_mu);
        republish();
    }
    int finish(int rc) {
        cudaDeviceSynchronize();
        std::string text;
        unsigned n;
        {
            std::lock_guard<std::mutex> g(g_mu);
            n = take_all(text);
            if (pre && !n) text = pre_text + " (in work launched before this call)";
            if (n || pre) g_last = text;
        }
        return (n || pre) ? HE_ERR_INVALID_ARG : rc;
    }
};

}  // namespace he

// used by the generated wrappers (checks_api.cpp)
void *he_checks_call_begin() { return new he::CheckCall(); }
void he_checks_call_arg(void *cc, const void *p) { ((he::CheckCall *)cc)->arg(p); }
void he_checks_call_ready(void *cc) { ((he::CheckCall *)cc)->finish_setup(); }
int he_checks_call_end(void *cc, int rc) {
    const int r = ((he::CheckCall *)cc)->finish(rc);
    delete (he::CheckCall *)cc;
    return r;
}

extern "C" {

int he_checks_enabled(void) { return 1; }

int he_checks_last_error(char *buf, int len) {
    if (!buf || len <= 0) return HE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(he::g_mu);
    snprintf(buf, (size_t)len, "%s", he::g_last.c_str());
    return HE_OK;
}

int he_checks_test_exclude(const void *ptr, long long bytes) {
    if (bytes < 0) return HE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(he::g_mu);
    he::g_hole_lo = (unsigned long long)ptr;
    he::g_hole_hi = ptr ? (unsigned long long)ptr + (unsigned long long)bytes : 0;
    return HE_OK;
}

}  // extern "C"
#endif  // HE_CHECKS
