// batch.cu -- batched execution of many heterogeneous CPMul convolution jobs.
//
// Each job is one he_cpmul_conv over its own context and plan (any ring
// degree, limb count and primes).  he_batch_prepare lays out every job's
// NTT-form scratch in one device allocation and turns the whole batch into
// two device work lists per ring degree: the limb polynomials to forward
// transform, and the output limb polynomials to multiply-accumulate, inverse
// transform and add.  The persistent form runs each list with one persistent
// kernel whose CTAs pull items from an atomic counter (heaviest items first);
// the graph form replays that launch sequence from a captured CUDA graph.
// The plain form calls he_cpmul_conv once per job, for comparison.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

struct he_batch {
    int device = 0;
    int n_sms = 0;
    struct Job {
        he_ctx *c;
        const he_plan *p;
        int batch;
        const u64 *ct_x, *pt_w, *ct_add;
        u64 *out;
    };
    std::vector<Job> jobs;
    bool prepared = false;
    void *mem = nullptr;
    struct Class {
        int logN;
        const he::FwdItem *fi;
        int nf;
        const he::MacItem *mi;
        int nm;
        int minb = 2;
        int grid_mult = 2;
        float best_ms = 0;
    };
    std::vector<Class> classes;
    int *counters = nullptr;  // two per class
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    std::string err;
};

namespace {

int bfail(he_batch *b, int code, const std::string &m) {
    b->err = m;
    return code;
}

size_t al(size_t n) { return (n + 255) & ~size_t(255); }

int run_persistent(he_batch *b, cudaStream_t st) {
    if (cudaMemsetAsync(b->counters, 0, sizeof(int) * 2 * b->classes.size(), st) != cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "counter reset");
    for (size_t i = 0; i < b->classes.size(); i++) {
        const auto &k = b->classes[i];
        int rc = he::launch_queue(k.logN, k.minb, k.fi, k.nf, nullptr, 0, b->counters + 2 * i, b->n_sms * k.grid_mult, st);
        if (rc) return bfail(b, rc, "forward queue launch");
    }
    for (size_t i = 0; i < b->classes.size(); i++) {
        const auto &k = b->classes[i];
        int rc = he::launch_queue(k.logN, k.minb, nullptr, 0, k.mi, k.nm, b->counters + 2 * i + 1,
                                  b->n_sms * k.grid_mult, st);
        if (rc) return bfail(b, rc, "multiply-accumulate queue launch");
    }
    return HE_OK;
}

void drop_graph(he_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" {

int he_batch_create(int device, he_batch **out) {
    if (!out) return HE_ERR_INVALID_ARG;
    *out = nullptr;
    he_batch *b = new he_batch();
    b->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete b;
        return HE_ERR_CUDA;
    }
    *out = b;
    return HE_OK;
}

int he_batch_destroy(he_batch *b) {
    if (!b) return HE_OK;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->mem) cudaFree(b->mem);
    delete b;
    return HE_OK;
}

int he_batch_last_error(const he_batch *b, char *buf, int len) {
    if (!b || !buf || len <= 0) return HE_ERR_INVALID_ARG;
    snprintf(buf, (size_t)len, "%s", b->err.c_str());
    return HE_OK;
}

int he_batch_add_cpmul(he_batch *b, he_ctx *c, const he_plan *p, int batch, const uint64_t *ct_x,
                       const uint64_t *pt_w, const uint64_t *ct_add, uint64_t *ct_out) {
    if (!b || !c || !p || batch < 1 || !ct_x || !pt_w || !ct_out) return HE_ERR_INVALID_ARG;
    if (b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "batch already prepared");
    if (c->P.device != b->device) return bfail(b, HE_ERR_INVALID_ARG, "context on another device");
    if (p->N != c->N) return bfail(b, HE_ERR_INVALID_ARG, "plan of another ring");
    b->jobs.push_back({c, p, batch, ct_x, pt_w, ct_add, ct_out});
    return (int)b->jobs.size() - 1;
}

int he_batch_prepare(he_batch *b) {
    if (!b) return HE_ERR_INVALID_ARG;
    if (b->prepared) return HE_OK;
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "cudaSetDevice");
    // scratch layout and term tables
    struct JL { size_t a_off, b_off, t_off; std::vector<int32_t> ta, tb; int G; };
    std::vector<JL> lay(b->jobs.size());
    size_t off = 0;
    for (size_t j = 0; j < b->jobs.size(); j++) {
        const auto &J = b->jobs[j];
        const int L = J.c->L, N = J.c->N, T = J.p->info.T, G = J.p->info.G, MG = J.p->info.MG;
        const size_t LN = (size_t)L * N;
        const long long nX = (long long)J.batch * T * G * 2, nW = (long long)MG * G;
        JL &l = lay[j];
        l.G = G;
        for (int bb = 0; bb < J.batch; bb++)
            for (int m = 0; m < MG; m++)
                for (int t = 0; t < T; t++)
                    for (int comp = 0; comp < 2; comp++)
                        for (int g = 0; g < G; g++) {
                            l.ta.push_back((int32_t)((((long long)(bb * T + t) * G + g) * 2 + comp) * L));
                            l.tb.push_back((m * G + g) * L);
                        }
        l.a_off = off;
        off += al((size_t)nX * LN * 8);
        l.b_off = off;
        off += al((size_t)nW * LN * 8);
        l.t_off = off;
        off += al(l.ta.size() * 8);
    }
    // items, grouped by ring degree
    std::vector<int> degrees;
    for (const auto &J : b->jobs)
        if (std::find(degrees.begin(), degrees.end(), J.c->logN) == degrees.end()) degrees.push_back(J.c->logN);
    std::sort(degrees.begin(), degrees.end());
    std::vector<std::vector<he::FwdItem>> F(degrees.size());
    std::vector<std::vector<he::MacItem>> Mi(degrees.size());
    char *base = nullptr;  // device base, known after allocation: build items with offsets first
    // first pass: compute total sizes of the item arrays
    size_t items_off = off;
    size_t nf_total = 0, nm_total = 0;
    for (const auto &J : b->jobs) {
        const long long L = J.c->L, T = J.p->info.T, G = J.p->info.G, MG = J.p->info.MG;
        nf_total += (size_t)(J.batch * T * G * 2 + MG * G) * L;
        nm_total += (size_t)(J.batch * MG * T * 2) * L;
    }
    off += al(nf_total * sizeof(he::FwdItem));
    size_t mitems_off = off;
    off += al(nm_total * sizeof(he::MacItem));
    size_t cnt_off = off;
    off += al(2 * degrees.size() * sizeof(int));
    if (cudaMalloc(&b->mem, off) != cudaSuccess) return bfail(b, HE_ERR_OOM, "batch scratch allocation");
    base = (char *)b->mem;
    for (size_t j = 0; j < b->jobs.size(); j++) {
        const auto &J = b->jobs[j];
        const JL &l = lay[j];
        const int ci = (int)(std::find(degrees.begin(), degrees.end(), J.c->logN) - degrees.begin());
        const int L = J.c->L, N = J.c->N, T = J.p->info.T, G = J.p->info.G, MG = J.p->info.MG;
        const size_t LN = (size_t)L * N;
        u64 *A = (u64 *)(base + l.a_off), *B = (u64 *)(base + l.b_off);
        const int32_t *ta = (const int32_t *)(base + l.t_off), *tb = ta + l.ta.size();
        const long long nX = (long long)J.batch * T * G * 2, nW = (long long)MG * G;
        for (long long p = 0; p < nX; p++)
            for (int li = 0; li < L; li++)
                F[ci].push_back({J.ct_x + p * LN + (size_t)li * N, A + p * LN + (size_t)li * N, J.c->d_mods + li, 0,
                                 he::SRC_RNS, 0});
        for (long long p = 0; p < nW; p++)
            for (int li = 0; li < L; li++)
                F[ci].push_back({J.pt_w + p * N, B + p * LN + (size_t)li * N, J.c->d_mods + li, J.c->P.t,
                                 he::SRC_T_LIFT, 0});
        const long long n_out = (long long)J.batch * MG * T * 2;
        for (long long o = 0; o < n_out; o++)
            for (int li = 0; li < L; li++)
                Mi[ci].push_back({A, B, ta, tb, (int)(o * G), (int)((o + 1) * G), li, 0,
                                  J.out + o * LN + (size_t)li * N,
                                  J.ct_add ? J.ct_add + o * LN + (size_t)li * N : nullptr, J.c->d_mods + li});
    }
    // heaviest multiply-accumulate items first
    for (auto &v : Mi)
        std::stable_sort(v.begin(), v.end(), [](const he::MacItem &x, const he::MacItem &y) {
            return (x.t1 - x.t0) > (y.t1 - y.t0);
        });
    // stage everything on the host and upload once
    std::vector<char> host(off, 0);
    for (size_t j = 0; j < b->jobs.size(); j++) {
        const JL &l = lay[j];
        memcpy(host.data() + l.t_off, l.ta.data(), l.ta.size() * 4);
        memcpy(host.data() + l.t_off + l.ta.size() * 4, l.tb.data(), l.tb.size() * 4);
    }
    size_t fo = items_off, mo = mitems_off;
    b->classes.clear();
    for (size_t ci = 0; ci < degrees.size(); ci++) {
        he_batch::Class k;
        k.logN = degrees[ci];
        memcpy(host.data() + fo, F[ci].data(), F[ci].size() * sizeof(he::FwdItem));
        memcpy(host.data() + mo, Mi[ci].data(), Mi[ci].size() * sizeof(he::MacItem));
        k.fi = (const he::FwdItem *)(base + fo);
        k.nf = (int)F[ci].size();
        k.mi = (const he::MacItem *)(base + mo);
        k.nm = (int)Mi[ci].size();
        k.minb = k.logN >= 14 ? 1 : 2;
        k.grid_mult = k.minb;
        fo += F[ci].size() * sizeof(he::FwdItem);
        mo += Mi[ci].size() * sizeof(he::MacItem);
        b->classes.push_back(k);
    }
    b->counters = (int *)(base + cnt_off);
    // only the term tables and the items need initial contents (counters are
    // reset before every run)
    for (size_t j = 0; j < b->jobs.size(); j++) {
        const JL &l = lay[j];
        if (cudaMemcpy(base + l.t_off, host.data() + l.t_off, l.ta.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, HE_ERR_CUDA, "term upload");
    }
    if (cudaMemcpy(base + items_off, host.data() + items_off, off - items_off, cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "item upload");
    b->prepared = true;
    return HE_OK;
}

int he_batch_run(he_batch *b, int mode, cudaStream_t st) {
    if (!b) return HE_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "cudaSetDevice");
    if (mode == HE_BATCH_PLAIN) {
        for (const auto &J : b->jobs) {
            int rc = he_cpmul_conv(J.c, J.p, J.batch, J.ct_x, J.pt_w, nullptr, nullptr, J.ct_add, J.out, st);
            if (rc) return bfail(b, rc, "plain job: " + J.c->err);
        }
        return HE_OK;
    }
    if (!b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "he_batch_prepare first");
    if (mode == HE_BATCH_PERSISTENT) return run_persistent(b, st);
    if (mode != HE_BATCH_GRAPH) return bfail(b, HE_ERR_INVALID_ARG, "bad mode");
    if (!b->exec || b->graph_stream != st) {
        drop_graph(b);
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(b, HE_ERR_CUDA, "stream capture (a non-default stream is needed)");
        int rc = run_persistent(b, st);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, rc ? rc : HE_ERR_CUDA, "graph capture failed");
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            drop_graph(b);
            return bfail(b, HE_ERR_CUDA, "graph instantiate");
        }
        b->graph_stream = st;
    }
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "graph launch");
    return HE_OK;
}

int he_batch_autotune(he_batch *b, cudaStream_t st, he_batch_tuning *out, int max_out, int *n_out) {
    if (!b || !st) return HE_ERR_INVALID_ARG;
    if (!b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "he_batch_prepare first");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "cudaSetDevice");
    drop_graph(b);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (size_t i = 0; i < b->classes.size(); i++) {
        auto &k = b->classes[i];
        const int minbs[2] = {1, 2};
        float best = 1e30f;
        int bm = k.minb, bg = k.grid_mult;
        for (int mb : minbs) {
            if (k.logN >= 14 && mb == 2) continue;
            for (int gm = 1; gm <= 4; gm++) {
                float tmin = 1e30f;
                for (int rep = 0; rep < 3; rep++) {
                    cudaMemsetAsync(b->counters + 2 * i, 0, 2 * sizeof(int), st);
                    cudaEventRecord(e0, st);
                    int rc = he::launch_queue(k.logN, mb, k.fi, k.nf, nullptr, 0, b->counters + 2 * i, b->n_sms * gm, st);
                    if (!rc) rc = he::launch_queue(k.logN, mb, nullptr, 0, k.mi, k.nm, b->counters + 2 * i + 1,
                                                   b->n_sms * gm, st);
                    cudaEventRecord(e1, st);
                    if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return bfail(b, HE_ERR_CUDA, "autotune launch");
                    }
                    float ms;
                    cudaEventElapsedTime(&ms, e0, e1);
                    tmin = std::min(tmin, ms);
                }
                if (tmin < best) { best = tmin; bm = mb; bg = gm; }
            }
        }
        k.minb = bm;
        k.grid_mult = bg;
        k.best_ms = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_out) *n_out = (int)b->classes.size();
    for (size_t i = 0; i < b->classes.size() && (int)i < max_out && out; i++) {
        out[i].logN = b->classes[i].logN;
        out[i].regs_ctas_per_sm = b->classes[i].minb;
        out[i].grid_ctas_per_sm = b->classes[i].grid_mult;
        out[i].ms = b->classes[i].best_ms;
        out[i].fwd_items = b->classes[i].nf;
        out[i].mac_items = b->classes[i].nm;
    }
    return HE_OK;
}

}  // extern "C"
