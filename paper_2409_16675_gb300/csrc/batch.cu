// batch.cu -- batched execution of many heterogeneous CPMul convolution jobs.
//
// Each job is one he_cpmul_conv over its own context and plan (any ring
// degree, limb count and primes).  he_batch_prepare lays out every job's
// NTT-form scratch in one device allocation and turns the whole batch into
// two device work lists per ring degree: the limb polynomials to forward
// transform, and the output limb polynomials to multiply-accumulate, inverse
// transform and add.  The persistent form runs each list with one launch:
// persistent CTAs pulling items from an atomic counter (heaviest items
// first), or one CTA per item in list order, whichever the autotuner
// measures faster.  The one-launch form (fused.cu) runs every degree's
// forward and multiply-accumulate items in a single persistent launch; the
// graph form replays whichever of the two the autotuner measured faster.
// The plain form calls he_cpmul_conv once per job, for comparison.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace he {

JobLayout job_layout(const JobDesc &J) {
    const int L = J.c->L, N = J.c->N, T = J.p->info.T, G = J.p->info.G, MG = J.p->info.MG;
    const size_t LN = (size_t)L * N;
    const long long nX = J.ct_x ? (long long)J.batch * T * G * 2 : 0, nW = J.ct_w ? (long long)MG * G * 2 : 0;
    const long long nWp = J.ct_x ? (long long)MG * G : 0, nXp = J.ct_w ? (long long)J.batch * T * G : 0;
    const long long n_out = (long long)J.batch * MG * T * 2;
    const long long n_terms = n_out * G * ((J.ct_x ? 1 : 0) + (J.ct_w ? 1 : 0));
    auto al = [](size_t n) { return (n + 255) & ~size_t(255); };
    JobLayout l;
    l.a_bytes = al((size_t)(nX + nW) * LN * 8);
    l.b_bytes = al((size_t)(nWp + nXp) * LN * 8);
    l.t_bytes = al((size_t)(n_out + 1 + 2 * n_terms) * 4);
    l.n_fwd = (size_t)(nX + nW + nWp + nXp) * L;
    l.n_mac = (size_t)n_out * L;
    return l;
}

void job_items(const JobDesc &J, char *dev, std::vector<int32_t> &terms, std::vector<FwdItem> &F,
               std::vector<MacItem> &Mi) {
    const int L = J.c->L, N = J.c->N, T = J.p->info.T, G = J.p->info.G, MG = J.p->info.MG;
    const size_t LN = (size_t)L * N;
    const JobLayout l = job_layout(J);
    const long long nX = J.ct_x ? (long long)J.batch * T * G * 2 : 0, nW = J.ct_w ? (long long)MG * G * 2 : 0;
    const long long nWp = J.ct_x ? (long long)MG * G : 0, nXp = J.ct_w ? (long long)J.batch * T * G : 0;
    u64 *A = (u64 *)dev, *B = (u64 *)(dev + l.a_bytes);
    // term table: ta then tb
    std::vector<int32_t> ta, tb;
    std::vector<int> t0;
    for (int bb = 0; bb < J.batch; bb++)
        for (int m = 0; m < MG; m++)
            for (int t = 0; t < T; t++)
                for (int comp = 0; comp < 2; comp++) {
                    t0.push_back((int)ta.size());
                    for (int g = 0; g < G; g++) {
                        if (!plan_pair(J.p, m, g)) continue;
                        const long long xi = (long long)(bb * T + t) * G + g;
                        if (J.ct_x) {
                            ta.push_back((int32_t)((xi * 2 + comp) * L));
                            tb.push_back((int32_t)((long long)(m * G + g) * L));
                        }
                        if (J.ct_w) {
                            ta.push_back((int32_t)((nX + (long long)(m * G + g) * 2 + comp) * L));
                            tb.push_back((int32_t)((nWp + xi) * L));
                        }
                    }
                }
    t0.push_back((int)ta.size());
    terms.assign(l.t_bytes / 4, 0);
    std::copy(ta.begin(), ta.end(), terms.begin());
    std::copy(tb.begin(), tb.end(), terms.begin() + ta.size());
    const int32_t *dta = (const int32_t *)(dev + l.a_bytes + l.b_bytes), *dtb = dta + ta.size();
    auto fwd = [&](const u64 *src, int kind, u64 *dst, long long n, long long stride) {
        for (long long p = 0; p < n; p++)
            for (int li = 0; li < L; li++)
                F.push_back({kind == SRC_RNS ? (const void *)(src + p * LN + (size_t)li * N) : (const void *)(src + p * stride),
                             dst + p * LN + (size_t)li * N, J.c->d_mods + li, J.c->P.t, kind, 0});
    };
    if (J.ct_x) { fwd(J.ct_x, SRC_RNS, A, nX, 0); fwd(J.pt_w, SRC_T_LIFT, B, nWp, N); }
    if (J.ct_w) { fwd(J.ct_w, SRC_RNS, A + nX * LN, nW, 0); fwd(J.pt_x, SRC_T_LIFT, B + nWp * LN, nXp, N); }
    const long long n_out = (long long)J.batch * MG * T * 2;
    for (long long o = 0; o < n_out; o++)
        for (int li = 0; li < L; li++)
            Mi.push_back({A, B, dta, dtb, t0[o], t0[o + 1], li, 0, J.out + o * LN + (size_t)li * N,
                          J.ct_add ? J.ct_add + o * LN + (size_t)li * N : nullptr, J.c->d_mods + li});
}

}  // namespace he

struct he_batch {
    int device = 0;
    int n_sms = 0;
    std::vector<he::JobDesc> jobs;
    bool prepared = false;
    void *mem = nullptr;
    struct Class {
        int logN;
        const he::FwdItem *fi;
        int nf;
        const he::MacItem *mi;
        int nm;
        const he::ItemSeg *fseg, *mseg;  // one-segment tables (device)
        bool lazy = true;                // every job's moduli below 2^57
        int minb = 2;
        int grid_mult = 2;
        float best_ms = 0;
    };
    std::vector<Class> classes;
    int *counters = nullptr;  // two per class
    // the one-launch form (fused.cu): possible when the batch has one ring
    // degree, or two of which one is half the other, and the larger is 2^12
    // or 2^13
    bool fused_ok = false;
    int fused_big = 0;        // logN of the larger degree
    int fused_minb = 2;       // register budget: resident CTAs per SM
    bool graph_fused = false; // the graph and persistent forms use the one-launch form
    he::FusedUnit *units = nullptr;
    int n_units = 0;
    int *fused_counter = nullptr;  // [1 + jobs]: unit counter, then each job's finished forward items
    int *fwd_need = nullptr;       // per job: its forward items
    int *status = nullptr;         // [2]
    std::vector<int> need_host;
    long long wait_limit = 1ll << 22;  // polls of 256 ns or more: a second or longer
    float fused_ms = 0, per_degree_ms = 0;
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
        int rc = he::launch_queue(k.logN, k.minb, true, k.lazy, k.fseg, 1, k.nf, b->counters + 2 * i, b->n_sms * k.grid_mult, st);
        if (rc) return bfail(b, rc, "forward queue launch");
    }
    for (size_t i = 0; i < b->classes.size(); i++) {
        const auto &k = b->classes[i];
        int rc = he::launch_queue(k.logN, k.minb, false, k.lazy, k.mseg, 1, k.nm, b->counters + 2 * i + 1,
                                  b->n_sms * k.grid_mult, st);
        if (rc) return bfail(b, rc, "multiply-accumulate queue launch");
    }
    return HE_OK;
}

he::FusedArgs fused_args(const he_batch *b) {
    he::FusedArgs a;
    memset(&a, 0, sizeof a);
    for (const auto &k : b->classes) {
        if (k.logN == b->fused_big) { a.fwd_big = k.fi; a.mac_big = k.mi; }
        else { a.fwd_small = k.fi; a.mac_small = k.mi; }
    }
    a.units = b->units;
    a.n_units = b->n_units;
    a.counter = b->fused_counter;
    a.fwd_done = b->fused_counter + 1;
    a.fwd_need = b->fwd_need;
    a.status = b->status;
    a.wait_limit = b->wait_limit;
    return a;
}

int run_fused(he_batch *b, cudaStream_t st, int minb) {
    if (!b->fused_ok)
        return bfail(b, HE_ERR_UNSUPPORTED_PARAMS,
                     "one-launch form needs one ring degree, or two of which one is half the other, up to 2^13");
    if (cudaMemsetAsync(b->fused_counter, 0, sizeof(int) * (1 + b->jobs.size()), st) != cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "counter reset");
    const int rc = he::launch_fused(b->fused_big, minb, fused_args(b), b->n_sms * minb, st);
    return rc ? bfail(b, rc, "fused launch") : HE_OK;
}

int run_batch_form(he_batch *b, cudaStream_t st) {
    return b->graph_fused ? run_fused(b, st, b->fused_minb) : run_persistent(b, st);
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
    if (b->mem) he::dev_free(b->mem);
    delete b;
    return HE_OK;
}

int he_batch_last_error(const he_batch *b, char *buf, int len) {
    if (!b || !buf || len <= 0) return HE_ERR_INVALID_ARG;
    snprintf(buf, (size_t)len, "%s", b->err.c_str());
    return HE_OK;
}

int he_batch_add_cpmul2(he_batch *b, he_ctx *c, const he_plan *p, int batch, const uint64_t *ct_x,
                        const uint64_t *pt_w, const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add,
                        uint64_t *ct_out) {
    if (!b || !c || !p || batch < 1 || !ct_out || (!ct_x && !ct_w) || (ct_x && !pt_w) || (ct_w && !pt_x))
        return HE_ERR_INVALID_ARG;
    if (b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "batch already prepared");
    if (c->P.device != b->device) return bfail(b, HE_ERR_INVALID_ARG, "context on another device");
    if (p->N != c->N) return bfail(b, HE_ERR_INVALID_ARG, "plan of another ring");
    b->jobs.push_back({c, p, batch, ct_x, pt_w, ct_w, pt_x, ct_add, ct_out});
    return (int)b->jobs.size() - 1;
}

int he_batch_add_cpmul(he_batch *b, he_ctx *c, const he_plan *p, int batch, const uint64_t *ct_x,
                       const uint64_t *pt_w, const uint64_t *ct_add, uint64_t *ct_out) {
    if (!ct_x || !pt_w) return HE_ERR_INVALID_ARG;
    return he_batch_add_cpmul2(b, c, p, batch, ct_x, pt_w, nullptr, nullptr, ct_add, ct_out);
}

int he_batch_prepare(he_batch *b) {
    if (!b) return HE_ERR_INVALID_ARG;
    if (b->prepared) return HE_OK;
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "cudaSetDevice");
    std::vector<int> degrees;
    for (const auto &J : b->jobs)
        if (std::find(degrees.begin(), degrees.end(), J.c->logN) == degrees.end()) degrees.push_back(J.c->logN);
    std::sort(degrees.begin(), degrees.end());
    // layout: per job [A][B][terms], then all forward items, all MAC items, counters
    std::vector<size_t> job_off(b->jobs.size());
    size_t off = 0, nf_total = 0, nm_total = 0;
    for (size_t j = 0; j < b->jobs.size(); j++) {
        const he::JobLayout l = he::job_layout(b->jobs[j]);
        job_off[j] = off;
        off += l.a_bytes + l.b_bytes + l.t_bytes;
        nf_total += l.n_fwd;
        nm_total += l.n_mac;
    }
    const size_t items_off = off;
    off += al(nf_total * sizeof(he::FwdItem));
    const size_t mitems_off = off;
    off += al(nm_total * sizeof(he::MacItem));
    const size_t seg_off = off;
    off += al(2 * degrees.size() * sizeof(he::ItemSeg));
    const size_t cnt_off = off;
    off += al(2 * degrees.size() * sizeof(int));
    // one-launch form: units, [counter][fwd_done per job], fwd_need per job, status
    b->fused_ok = (degrees.size() == 1 && (degrees[0] == 12 || degrees[0] == 13)) ||
                  (degrees.size() == 2 && degrees[1] == degrees[0] + 1 && (degrees[1] == 12 || degrees[1] == 13));
    b->fused_big = degrees.empty() ? 0 : degrees.back();
    const size_t units_off = off;
    off += al((nf_total + nm_total) * sizeof(he::FusedUnit));
    const size_t fcnt_off = off;
    off += al((1 + b->jobs.size()) * sizeof(int));
    const size_t need_off = off;
    off += al(b->jobs.size() * sizeof(int));
    const size_t status_off = off;
    off += al(2 * sizeof(int));
    if (he::dev_alloc((void **)&b->mem, off) != cudaSuccess) return bfail(b, HE_ERR_OOM, "batch scratch allocation");
    char *base = (char *)b->mem;
    std::vector<std::vector<he::FwdItem>> F(degrees.size());
    std::vector<std::vector<he::MacItem>> Mi(degrees.size());
    std::vector<std::vector<int>> Fjob(degrees.size()), Mjob(degrees.size());  // the job of each item
    std::vector<int32_t> terms;
    b->need_host.assign(b->jobs.size(), 0);
    for (size_t j = 0; j < b->jobs.size(); j++) {
        const auto &J = b->jobs[j];
        const int ci = (int)(std::find(degrees.begin(), degrees.end(), J.c->logN) - degrees.begin());
        const he::JobLayout l = he::job_layout(J);
        const size_t f0 = F[ci].size(), m0 = Mi[ci].size();
        he::job_items(J, base + job_off[j], terms, F[ci], Mi[ci]);
        Fjob[ci].resize(F[ci].size(), (int)j);
        Mjob[ci].resize(Mi[ci].size(), (int)j);
        b->need_host[j] = (int)(F[ci].size() - f0);
        (void)m0;
        if (cudaMemcpy(base + job_off[j] + l.a_bytes + l.b_bytes, terms.data(), terms.size() * 4,
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, HE_ERR_CUDA, "term upload");
    }
    // heaviest multiply-accumulate items first (the job of each item follows it)
    for (size_t ci = 0; ci < degrees.size(); ci++) {
        std::vector<size_t> perm(Mi[ci].size());
        for (size_t i = 0; i < perm.size(); i++) perm[i] = i;
        const auto &v = Mi[ci];
        std::stable_sort(perm.begin(), perm.end(),
                         [&](size_t x, size_t y) { return (v[x].t1 - v[x].t0) > (v[y].t1 - v[y].t0); });
        std::vector<he::MacItem> sorted(v.size());
        std::vector<int> sj(v.size());
        for (size_t i = 0; i < perm.size(); i++) { sorted[i] = v[perm[i]]; sj[i] = Mjob[ci][perm[i]]; }
        Mi[ci].swap(sorted);
        Mjob[ci].swap(sj);
    }
    // one-launch units: every forward unit (an item of the larger degree, or
    // two of the smaller), then the multiply-accumulate units, heaviest first
    if (b->fused_ok) {
        std::vector<he::FusedUnit> U;
        const int cb = (int)degrees.size() - 1, cs = degrees.size() == 2 ? 0 : -1;
        auto pairs = [&](int ci, int mac, std::vector<he::FusedUnit> &out) {
            const size_t n = mac ? Mi[ci].size() : F[ci].size();
            const std::vector<int> &jb = mac ? Mjob[ci] : Fjob[ci];
            for (size_t i = 0; i < n; i += 2) {
                he::FusedUnit u{mac, 0, {(int32_t)i, -1}, {jb[i], 0}};
                if (i + 1 < n) { u.item[1] = (int32_t)(i + 1); u.job[1] = jb[i + 1]; }
                out.push_back(u);
            }
        };
        for (size_t i = 0; i < F[cb].size(); i++) U.push_back({0, 1, {(int32_t)i, -1}, {Fjob[cb][i], 0}});
        if (cs >= 0) pairs(cs, 0, U);
        std::vector<he::FusedUnit> small_mac;
        if (cs >= 0) pairs(cs, 1, small_mac);
        auto weight = [&](const he::FusedUnit &u) {
            const auto &v = Mi[u.big ? cb : cs];
            return v[u.item[0]].t1 - v[u.item[0]].t0;  // the first item of a pair is the heavier
        };
        size_t ib = 0, is = 0;
        while (ib < Mi[cb].size() || is < small_mac.size()) {
            const he::FusedUnit ub{1, 1, {(int32_t)ib, -1}, {ib < Mi[cb].size() ? Mjob[cb][ib] : 0, 0}};
            if (is >= small_mac.size() || (ib < Mi[cb].size() && weight(ub) >= weight(small_mac[is]))) {
                U.push_back(ub);
                ib++;
            } else {
                U.push_back(small_mac[is++]);
            }
        }
        b->n_units = (int)U.size();
        b->units = (he::FusedUnit *)(base + units_off);
        b->fused_counter = (int *)(base + fcnt_off);
        b->fwd_need = (int *)(base + need_off);
        b->status = (int *)(base + status_off);
        if (cudaMemcpy(b->units, U.data(), U.size() * sizeof(he::FusedUnit), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->fwd_need, b->need_host.data(), b->need_host.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemset(b->status, 0, 2 * sizeof(int)) != cudaSuccess)
            return bfail(b, HE_ERR_CUDA, "unit upload");
    }
    size_t fo = items_off, mo = mitems_off;
    std::vector<he::ItemSeg> segs;
    b->classes.clear();
    for (size_t ci = 0; ci < degrees.size(); ci++) {
        he_batch::Class k;
        k.logN = degrees[ci];
        if (cudaMemcpy(base + fo, F[ci].data(), F[ci].size() * sizeof(he::FwdItem), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(base + mo, Mi[ci].data(), Mi[ci].size() * sizeof(he::MacItem), cudaMemcpyHostToDevice) != cudaSuccess)
            return bfail(b, HE_ERR_CUDA, "item upload");
        k.fi = (const he::FwdItem *)(base + fo);
        k.nf = (int)F[ci].size();
        k.mi = (const he::MacItem *)(base + mo);
        k.nm = (int)Mi[ci].size();
        k.fseg = (const he::ItemSeg *)(base + seg_off) + 2 * ci;
        k.mseg = k.fseg + 1;
        segs.push_back({k.fi, 0, 0});
        segs.push_back({k.mi, 0, 0});
        for (const auto &J : b->jobs)
            if (J.c->logN == k.logN && !he::ctx_lazy(J.c)) k.lazy = false;
        k.minb = k.logN >= 14 ? 1 : 2;
        k.grid_mult = k.minb;
        fo += F[ci].size() * sizeof(he::FwdItem);
        mo += Mi[ci].size() * sizeof(he::MacItem);
        b->classes.push_back(k);
    }
    if (cudaMemcpy(base + seg_off, segs.data(), segs.size() * sizeof(he::ItemSeg), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "segment upload");
    b->counters = (int *)(base + cnt_off);
    b->prepared = true;
    return HE_OK;
}

int he_batch_run(he_batch *b, int mode, cudaStream_t st) {
    if (!b) return HE_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "cudaSetDevice");
    if (mode == HE_BATCH_PLAIN) {
        for (const auto &J : b->jobs) {
            int rc = he_cpmul_conv(J.c, J.p, J.batch, J.ct_x, J.pt_w, J.ct_w, J.pt_x, J.ct_add, J.out, st);
            if (rc) return bfail(b, rc, "plain job: " + J.c->err);
        }
        return HE_OK;
    }
    if (!b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "he_batch_prepare first");
    if (mode == HE_BATCH_PERSISTENT) return run_persistent(b, st);
    if (mode == HE_BATCH_FUSED) return run_fused(b, st, b->fused_minb);
    if (mode != HE_BATCH_GRAPH) return bfail(b, HE_ERR_INVALID_ARG, "bad mode");
    if (!b->exec || b->graph_stream != st) {
        drop_graph(b);
        if (b->graph_fused && he::fused_set_attributes(b->fused_big, b->fused_minb))
            return bfail(b, HE_ERR_CUDA, "fused kernel attributes");
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(b, HE_ERR_CUDA, "stream capture (a non-default stream is needed)");
        int rc = run_batch_form(b, st);
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

int he_batch_set_tuning(he_batch *b, const he_batch_tuning *t, int n) {
    if (!b || (n > 0 && !t) || n < 0) return HE_ERR_INVALID_ARG;
    if (!b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "he_batch_prepare first");
    for (int i = 0; i < n; i++) {
        if (t[i].regs_ctas_per_sm < 1 || t[i].regs_ctas_per_sm > 2 || t[i].grid_ctas_per_sm < 0 ||
            t[i].grid_ctas_per_sm > 16)
            return bfail(b, HE_ERR_INVALID_ARG, "tuning out of range (regs 1..2, grid 0..16)");
        if (t[i].logN >= 14 && t[i].regs_ctas_per_sm == 2)
            return bfail(b, HE_ERR_INVALID_ARG, "ring degrees >= 2^14 run one CTA per SM");
        bool found = false;
        for (auto &k : b->classes)
            if (k.logN == t[i].logN) {
                k.minb = t[i].regs_ctas_per_sm;
                k.grid_mult = t[i].grid_ctas_per_sm;
                found = true;
            }
        if (!found) return bfail(b, HE_ERR_INVALID_ARG, "no job of that ring degree");
    }
    drop_graph(b);
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
            for (int gm = 0; gm <= 4; gm++) {  // 0: one CTA per item; else persistent CTAs per SM
                float tmin = 1e30f;
                for (int rep = 0; rep < 3; rep++) {
                    cudaMemsetAsync(b->counters + 2 * i, 0, 2 * sizeof(int), st);
                    cudaEventRecord(e0, st);
                    int rc = he::launch_queue(k.logN, mb, true, k.lazy, k.fseg, 1, k.nf, b->counters + 2 * i, b->n_sms * gm, st);
                    if (!rc) rc = he::launch_queue(k.logN, mb, false, k.lazy, k.mseg, 1, k.nm, b->counters + 2 * i + 1,
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
    b->per_degree_ms = 0;
    for (const auto &k : b->classes) b->per_degree_ms += k.best_ms;
    // the one-launch form at both register budgets, three runs each
    b->fused_ms = 0;
    if (b->fused_ok) {
        float best = 1e30f;
        int bm = b->fused_minb;
        for (int mb = 1; mb <= 2; mb++) {
            float tmin = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                cudaEventRecord(e0, st);
                int rc = run_fused(b, st, mb);
                cudaEventRecord(e1, st);
                if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return bfail(b, rc ? rc : HE_ERR_CUDA, "autotune of the one-launch form");
                }
                float ms;
                cudaEventElapsedTime(&ms, e0, e1);
                tmin = std::min(tmin, ms);
            }
            if (tmin < best) { best = tmin; bm = mb; }
        }
        int st_h[2] = {0, 0};
        if (cudaMemcpy(st_h, b->status, sizeof st_h, cudaMemcpyDeviceToHost) != cudaSuccess || st_h[0]) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return bfail(b, st_h[0] ? st_h[0] : HE_ERR_CUDA, "one-launch form gave up waiting during autotuning");
        }
        b->fused_minb = bm;
        b->fused_ms = best;
        b->graph_fused = best < b->per_degree_ms;
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

int he_batch_query(const he_batch *b, he_batch_info *info) {
    if (!b || !info) return HE_ERR_INVALID_ARG;
    memset(info, 0, sizeof *info);
    info->fused_supported = b->fused_ok;
    info->graph_fused = b->graph_fused;
    info->fused_regs_ctas_per_sm = b->fused_minb;
    info->n_units = b->n_units;
    info->fused_ms = b->fused_ms;
    info->per_degree_ms = b->per_degree_ms;
    return HE_OK;
}

int he_batch_set_fused(he_batch *b, int graph_fused, int regs_ctas_per_sm) {
    if (!b || regs_ctas_per_sm < 0 || regs_ctas_per_sm > 2) return HE_ERR_INVALID_ARG;
    if (!b->prepared) return bfail(b, HE_ERR_INVALID_ARG, "he_batch_prepare first");
    if (graph_fused && !b->fused_ok) return bfail(b, HE_ERR_UNSUPPORTED_PARAMS, "no one-launch form for these degrees");
    b->graph_fused = graph_fused != 0;
    if (regs_ctas_per_sm) b->fused_minb = regs_ctas_per_sm;
    drop_graph(b);
    return HE_OK;
}

int he_batch_status(he_batch *b, cudaStream_t st) {
    if (!b) return HE_ERR_INVALID_ARG;
    if (!b->prepared || !b->status) return HE_OK;
    if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "stream synchronisation");
    int h[2] = {0, 0};
    if (cudaMemcpy(h, b->status, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(b->status, 0, sizeof h) != cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "status read");
    if (h[0])
        return bfail(b, h[0], "one-launch form: work unit " + std::to_string(h[1]) +
                                  " gave up waiting for its job's forward transforms");
    return HE_OK;
}

int he_batch_set_wait_limit(he_batch *b, long long polls) {
    if (!b || polls < 1) return HE_ERR_INVALID_ARG;
    b->wait_limit = polls;
    drop_graph(b);
    return HE_OK;
}

int he_batch_test_hold_job(he_batch *b, int job, int hold) {
    if (!b || job < 0 || job >= (int)b->jobs.size()) return HE_ERR_INVALID_ARG;
    if (!b->prepared || !b->fused_ok) return bfail(b, HE_ERR_INVALID_ARG, "prepared one-launch batch needed");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HE_ERR_CUDA, "cudaSetDevice");
    const int need = b->need_host[job] + (hold ? 1 : 0);
    if (cudaMemcpy(b->fwd_need + job, &need, sizeof need, cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(b, HE_ERR_CUDA, "hold");
    return HE_OK;
}

}  // extern "C"
