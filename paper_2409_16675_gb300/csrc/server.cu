// server.cu -- continuous-batching request server for CPMul convolution
// layers (the online phase of the CryptoTrain-P linear layer, Section 3.2).
//
// The server reserves one device arena of the configured HBM budget at start.
// Submitting a request only queues it.  A worker thread loops:
//   1. retires launch groups whose completion event has fired, stamping their
//      requests done and returning their arena blocks;
//   2. admits waiting requests in arrival order while their scratch (NTT-form
//      operands and term table) fits in the arena and the number of groups in
//      flight is below the limit -- requests that arrived while others run on
//      the GPU join as soon as memory and a slot free up;
//   3. launches the admitted group as work-list kernels (one forward and one
//      multiply-accumulate/inverse launch per ring degree, each over a table
//      of the requests' item arrays, one CTA per item) on the next of several
//      streams, so consecutive groups overlap on the device.
// A request's arena block holds its operands, term table and work items, so
// admission is the only point where memory can run short: a launch never
// waits for memory, and the oldest waiting request always fits once the
// groups ahead of it have retired.
// Every request's result is bit-identical to he_cpmul_conv on its arguments
// alone: the work items of a request never read another request's data.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t al(size_t n) { return (n + 255) & ~size_t(255); }

// first-fit allocator over [0, size) with coalescing frees
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> length
    size_t used = 0, peak = 0;
    void init(size_t size) { free_.clear(); free_[0] = size; }
    bool alloc(size_t n, size_t &off) {
        n = al(n);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used += n;
                peak = std::max(peak, used);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        n = al(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace

struct he_server {
    he_server_config cfg;
    int n_sms = 0;
    char *arena_base = nullptr;
    size_t arena_size = 0;
    Arena arena;
    // Per-group control blocks (counters and segment tables), one per
    // in-flight slot, carved from the arena at creation so that launching an
    // admitted group never needs more arena space.
    static constexpr int kMaxDegrees = 8;  // ring degrees 2^10 .. 2^17
    size_t slot_bytes = 0, slots_off = 0;
    std::vector<int> free_slots;
    struct Req {
        he::JobDesc J;
        size_t bytes = 0, off = 0;  // [A][B][terms][forward items][MAC items]
        double t_submit = 0, t_admit = 0, t_done = 0;
        int state = 0;  // 0 queued, 1 admitted, 2 done, 3 cancelled while queued
    };
    std::vector<Req> reqs;
    std::deque<int64_t> pending;
    struct Flight {
        cudaEvent_t ev = nullptr;
        std::vector<int64_t> ids;
        int slot = -1;
        char *host = nullptr;    // pinned staging of items and terms, reused after completion
        size_t host_size = 0;
    };
    std::vector<std::pair<char *, size_t>> pinned_free;  // idle pinned staging buffers
    std::deque<Flight> inflight;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    int64_t groups = 0, stat_from = 0;
    std::string err;
    int worker_rc = HE_OK;
};

namespace {

// arena bytes of one request: NTT-form operands, term table and its own items
size_t request_bytes(const he::JobLayout &l) {
    return l.a_bytes + l.b_bytes + l.t_bytes + al(l.n_fwd * sizeof(he::FwdItem)) + al(l.n_mac * sizeof(he::MacItem));
}

size_t slot_bytes(int max_group) {
    return al(2 * he_server::kMaxDegrees * sizeof(int)) +
           al((size_t)2 * he_server::kMaxDegrees * max_group * sizeof(he::ItemSeg));
}

// Launch one admitted group (its requests' arena blocks are reserved and
// f.slot is a free control slot); called with the lock held.  Each request's
// term table and item lists are staged in pinned memory and copied into its
// own block with one asynchronous copy; the group's control block (zeroed
// counters, then per degree a forward and a MAC segment table listing the
// requests' item arrays) follows with one more.
int launch_group(he_server *s, std::vector<int64_t> &ids, he_server::Flight &f) {
    std::vector<int> degrees;
    for (int64_t id : ids) {
        const int d = s->reqs[id].J.c->logN;
        if (std::find(degrees.begin(), degrees.end(), d) == degrees.end()) degrees.push_back(d);
    }
    std::sort(degrees.begin(), degrees.end());
    if ((int)degrees.size() > he_server::kMaxDegrees) return HE_ERR_INVALID_ARG;
    size_t need = s->slot_bytes;
    for (int64_t id : ids) {
        const auto &r = s->reqs[id];
        const he::JobLayout l = he::job_layout(r.J);
        need += r.bytes - l.a_bytes - l.b_bytes;
    }
    for (size_t i = 0; i < s->pinned_free.size(); i++)
        if (s->pinned_free[i].second >= need) {
            f.host = s->pinned_free[i].first;
            f.host_size = s->pinned_free[i].second;
            s->pinned_free.erase(s->pinned_free.begin() + i);
            break;
        }
    if (!f.host) {
        f.host_size = std::max(need, (size_t)16 << 20);
        if (cudaHostAlloc((void **)&f.host, f.host_size, cudaHostAllocDefault) != cudaSuccess) {
            f.host = nullptr;
            return HE_ERR_OOM;
        }
    }
    cudaStream_t st = s->streams[s->next_stream];
    s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
    char *h = f.host;
    // control block: counters, then forward/MAC segment tables per degree
    const size_t seg_base = al(2 * he_server::kMaxDegrees * sizeof(int));
    const size_t per_table = (size_t)s->cfg.max_group * sizeof(he::ItemSeg);
    memset(h, 0, s->slot_bytes);
    std::vector<int> nseg(2 * degrees.size(), 0), total(2 * degrees.size(), 0);
    size_t ho = s->slot_bytes;
    std::vector<int32_t> terms;
    std::vector<he::FwdItem> F;
    std::vector<he::MacItem> Mi;
    for (int64_t id : ids) {
        auto &r = s->reqs[id];
        const int ci = (int)(std::find(degrees.begin(), degrees.end(), r.J.c->logN) - degrees.begin());
        const he::JobLayout l = he::job_layout(r.J);
        F.clear();
        Mi.clear();
        he::job_items(r.J, s->arena_base + r.off, terms, F, Mi);
        std::stable_sort(Mi.begin(), Mi.end(), [](const he::MacItem &x, const he::MacItem &y) {
            return (x.t1 - x.t0) > (y.t1 - y.t0);
        });
        // [terms][forward items][MAC items] contiguous, as in the arena block
        const size_t meta = r.bytes - l.a_bytes - l.b_bytes;
        char *hm = h + ho;
        memcpy(hm, terms.data(), terms.size() * 4);
        memcpy(hm + l.t_bytes, F.data(), F.size() * sizeof(he::FwdItem));
        memcpy(hm + l.t_bytes + al(F.size() * sizeof(he::FwdItem)), Mi.data(), Mi.size() * sizeof(he::MacItem));
        char *dm = s->arena_base + r.off + l.a_bytes + l.b_bytes;
        if (cudaMemcpyAsync(dm, hm, meta, cudaMemcpyHostToDevice, st) != cudaSuccess) return HE_ERR_CUDA;
        ho += meta;
        he::ItemSeg *fs = (he::ItemSeg *)(h + seg_base + (2 * ci) * per_table);
        he::ItemSeg *ms = (he::ItemSeg *)(h + seg_base + (2 * ci + 1) * per_table);
        fs[nseg[2 * ci]++] = {dm + l.t_bytes, total[2 * ci], 0};
        ms[nseg[2 * ci + 1]++] = {dm + l.t_bytes + al(F.size() * sizeof(he::FwdItem)), total[2 * ci + 1], 0};
        total[2 * ci] += (int)F.size();
        total[2 * ci + 1] += (int)Mi.size();
    }
    char *ctl = s->arena_base + s->slots_off + (size_t)f.slot * s->slot_bytes;
    if (cudaMemcpyAsync(ctl, h, s->slot_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return HE_ERR_CUDA;
    int *counters = (int *)ctl;
    std::vector<char> lazy(degrees.size(), 1);
    for (int64_t id : ids) {
        const he_ctx *c = s->reqs[id].J.c;
        if (!he::ctx_lazy(c)) lazy[std::find(degrees.begin(), degrees.end(), c->logN) - degrees.begin()] = 0;
    }
    for (int pass = 0; pass < 2; pass++)
        for (size_t i = 0; i < degrees.size(); i++) {
            const int k = 2 * (int)i + pass;
            const int mb = degrees[i] >= 14 ? 1 : 2;
            const he::ItemSeg *segs = (const he::ItemSeg *)(ctl + seg_base + k * per_table);
            // one CTA per item, heaviest first within each request (the form the
            // batch autotuner measures fastest on these kernels)
            int rc = he::launch_queue(degrees[i], mb, pass == 0, lazy[i] != 0, segs, nseg[k], total[k], counters + k,
                                      0, st);
            if (rc) return rc;
        }
    if (cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming) != cudaSuccess) return HE_ERR_CUDA;
    if (cudaEventRecord(f.ev, st) != cudaSuccess) return HE_ERR_CUDA;
    f.ids = ids;
    return HE_OK;
}

void worker_loop(he_server *s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        // 1. retire finished groups (in any order)
        for (auto it = s->inflight.begin(); it != s->inflight.end();) {
            const cudaError_t e = cudaEventQuery(it->ev);
            if (e == cudaErrorNotReady) { ++it; continue; }
            const double t = now_us();
            for (int64_t id : it->ids) {
                auto &r = s->reqs[id];
                r.t_done = t;
                r.state = 2;
                s->arena.release(r.off, r.bytes);
            }
            s->free_slots.push_back(it->slot);
            s->pinned_free.emplace_back(it->host, it->host_size);
            cudaEventDestroy(it->ev);
            if (e != cudaSuccess && s->worker_rc == HE_OK) {
                s->worker_rc = HE_ERR_CUDA;
                s->err = std::string("device error: ") + cudaGetErrorString(e);
            }
            it = s->inflight.erase(it);
            progress = true;
        }
        // 2. admit in arrival order while memory and a slot are free
        std::vector<int64_t> group;
        while (!s->pending.empty() && (int)group.size() < s->cfg.max_group &&
               (int)s->inflight.size() < s->cfg.max_inflight) {
            auto &r = s->reqs[s->pending.front()];
            size_t off;
            if (!s->arena.alloc(r.bytes, off)) break;
            r.off = off;
            r.state = 1;
            r.t_admit = now_us();
            group.push_back(s->pending.front());
            s->pending.pop_front();
        }
        if (!group.empty()) {
            he_server::Flight f;
            f.slot = s->free_slots.back();
            s->free_slots.pop_back();
            const int rc = launch_group(s, group, f);
            if (rc != HE_OK) {
                // nothing of the group is known to be in flight: wait for the
                // device, then fail its requests and every later one
                for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
                if (f.ev) cudaEventDestroy(f.ev);
                if (f.host) s->pinned_free.emplace_back(f.host, f.host_size);
                s->free_slots.push_back(f.slot);
                if (s->worker_rc == HE_OK) {
                    s->worker_rc = rc;
                    s->err = "group launch failed";
                }
                for (int64_t id : group) {
                    auto &r = s->reqs[id];
                    s->arena.release(r.off, r.bytes);
                    r.state = 2;
                    r.t_done = now_us();
                }
            } else {
                s->inflight.push_back(std::move(f));
                s->groups++;
            }
            progress = true;
        }
        if (s->stop && s->pending.empty() && s->inflight.empty()) break;
        if (!progress) {
            s->cv.notify_all();
            s->cv.wait_for(lk, std::chrono::microseconds(s->cfg.poll_us));
        } else {
            s->cv.notify_all();
        }
    }
    s->cv.notify_all();
}

}  // namespace

extern "C" {

int he_server_create(const he_server_config *cfg, he_server **out) {
    if (!cfg || !out || cfg->max_group < 1 || cfg->max_inflight < 1 || cfg->n_streams < 1 || cfg->hbm_budget_bytes <= 0)
        return HE_ERR_INVALID_ARG;
    *out = nullptr;
    he_server *s = new he_server();
    s->cfg = *cfg;
    if (s->cfg.poll_us <= 0) s->cfg.poll_us = 20;
    if (cudaSetDevice(cfg->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->n_sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess) {
        delete s;
        return HE_ERR_CUDA;
    }
    s->arena_size = al((size_t)cfg->hbm_budget_bytes);
    if (he::dev_alloc((void **)&s->arena_base, s->arena_size) != cudaSuccess) {
        delete s;
        return HE_ERR_OOM;
    }
    s->arena.init(s->arena_size);
    s->slot_bytes = slot_bytes(cfg->max_group);
    if (!s->arena.alloc(s->slot_bytes * cfg->max_inflight, s->slots_off)) {
        he::dev_free(s->arena_base);
        delete s;
        return HE_ERR_BUDGET_EXCEEDED;
    }
    for (int i = cfg->max_inflight - 1; i >= 0; i--) s->free_slots.push_back(i);
    for (int i = 0; i < cfg->n_streams; i++) {
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return HE_OK;
}

int he_server_submit(he_server *s, he_ctx *c, const he_plan *p, int n_images, const uint64_t *ct_x,
                     const uint64_t *pt_w, const uint64_t *ct_w, const uint64_t *pt_x, const uint64_t *ct_add,
                     uint64_t *ct_out, int64_t *request_id) {
    if (!s || !c || !p || n_images < 1 || !ct_out || !request_id || (!ct_x && !ct_w) || (ct_x && !pt_w) ||
        (ct_w && !pt_x))
        return HE_ERR_INVALID_ARG;
    if (c->P.device != s->cfg.device || p->N != c->N) return HE_ERR_INVALID_ARG;
    he::JobDesc J{c, p, n_images, ct_x, pt_w, ct_w, pt_x, ct_add, ct_out};
    const size_t bytes = request_bytes(he::job_layout(J));
    // a request larger than the arena less the control slots could never be admitted
    if (bytes > s->arena_size - s->slot_bytes * s->cfg.max_inflight) return HE_ERR_BUDGET_EXCEEDED;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return HE_ERR_INVALID_ARG;
    he_server::Req r;
    r.J = J;
    r.bytes = bytes;
    r.t_submit = now_us();
    s->reqs.push_back(r);
    *request_id = (int64_t)s->reqs.size() - 1;
    s->pending.push_back(*request_id);
    s->cv.notify_all();
    return HE_OK;
}

int he_server_request_bytes(const he_ctx *c, const he_plan *p, int n_images, int has_x, int has_w, double *bytes) {
    if (!c || !p || n_images < 1 || !bytes || (!has_x && !has_w)) return HE_ERR_INVALID_ARG;
    static const u64 dummy = 0;
    he::JobDesc J{const_cast<he_ctx *>(c), p, n_images, has_x ? &dummy : nullptr, has_x ? &dummy : nullptr,
                  has_w ? &dummy : nullptr, has_w ? &dummy : nullptr, nullptr, nullptr};
    *bytes = (double)request_bytes(he::job_layout(J));
    return HE_OK;
}

int he_server_poll(he_server *s, int64_t id, int *done, double *latency_us) {
    if (!s || !done) return HE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (id < 0 || id >= (int64_t)s->reqs.size()) return HE_ERR_INVALID_ARG;
    const auto &r = s->reqs[id];
    *done = r.state >= 2;
    if (latency_us) *latency_us = r.state == 2 ? r.t_done - r.t_submit : -1.0;
    return s->worker_rc;
}

int he_server_cancel(he_server *s, int64_t id, int *cancelled) {
    if (!s || !cancelled) return HE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (id < 0 || id >= (int64_t)s->reqs.size()) return HE_ERR_INVALID_ARG;
    auto &r = s->reqs[id];
    *cancelled = 0;
    if (r.state != 0) return HE_OK;  // admitted requests run to completion
    auto it = std::find(s->pending.begin(), s->pending.end(), id);
    if (it != s->pending.end()) s->pending.erase(it);
    r.state = 3;
    r.t_done = now_us();
    *cancelled = 1;
    s->cv.notify_all();
    return HE_OK;
}

int he_server_wait_all(he_server *s, double timeout_s) {
    if (!s) return HE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (!(s->pending.empty() && s->inflight.empty())) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) return HE_ERR_TIMEOUT;
    }
    return s->worker_rc;
}

int he_server_stats(he_server *s, he_server_report *out) {
    if (!s || !out) return HE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    memset(out, 0, sizeof *out);
    std::vector<double> lat;
    double t0 = 1e300, t1 = 0;
    for (size_t i = (size_t)s->stat_from; i < s->reqs.size(); i++) {
        const auto &r = s->reqs[i];
        if (r.state != 2) continue;
        lat.push_back(r.t_done - r.t_submit);
        t0 = std::min(t0, r.t_submit);
        t1 = std::max(t1, r.t_done);
        out->images += r.J.batch;
    }
    out->completed = (int64_t)lat.size();
    out->submitted = (int64_t)s->reqs.size() - s->stat_from;
    out->groups = s->groups;
    out->arena_peak_bytes = (double)s->arena.peak;
    out->arena_bytes = (double)s->arena_size;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) { return lat[std::min(lat.size() - 1, (size_t)(p * (lat.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = lat.back();
        double sum = 0;
        for (double v : lat) sum += v;
        out->mean_us = sum / lat.size();
        out->span_s = (t1 - t0) * 1e-6;
    }
    return s->worker_rc;
}

int he_server_reset_stats(he_server *s) {
    if (!s) return HE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    s->stat_from = (int64_t)s->reqs.size();
    s->groups = 0;
    s->arena.peak = s->arena.used;
    return HE_OK;
}

int he_server_destroy(he_server *s) {
    if (!s) return HE_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->cfg.device);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (auto &p : s->pinned_free) cudaFreeHost(p.first);
    if (s->arena_base) he::dev_free(s->arena_base);
    delete s;
    return HE_OK;
}

}  // extern "C"
