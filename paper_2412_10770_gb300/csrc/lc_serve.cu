// lc_serve.cu -- serving runtime: continuous batching of access, lower_bound
// and range-decode requests over device-resident columns (lc_server_* in
// include/lc.h).
//
// One scheduler thread owns the GPU side.  Its loop: (1) retire batches whose
// completion event has fired (results to the callers' buffers, memory back to
// the budget, slot free); (2) while a slot is free, pack the oldest waiting
// requests that fit in the free HBM budget into one batch and launch it on the
// slot's stream: one host-to-device copy of the packed descriptors and
// queries, one fused query launch, one persistent decode launch, the copies
// back, an event; (3) sleep briefly when there is nothing to do.  No GPU-side
// waits: completion is observed with cudaEventQuery.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lc_internal.h"

namespace lcx {
namespace {

using Clock = std::chrono::steady_clock;

constexpr uint64_t kMaxBatchQueries = 1ull << 21;
constexpr uint32_t kMaxBatchDecodes = 512;
constexpr uint32_t kMaxBatchRequests = 4096;

struct Pending {
    lc_request r;
    uint64_t ticket;
    Clock::time_point t0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<Pending> reqs;
    std::vector<uint64_t> qoff;  // per request: first query (access / lower_bound)
    uint8_t* h_stage = nullptr;  // pinned: descriptors and queries in, query results out
    size_t h_cap = 0;
    uint8_t* d_buf = nullptr;
    uint64_t charged = 0;
    size_t out_off = 0;  // where the query results land in h_stage
};

}  // namespace
}  // namespace lcx

struct lc_server {
    std::vector<lc_column*> cols;
    int device = 0;
    int kb = 8;
    lcx::ColView* d_views = nullptr;
    uint32_t max_tile_segs = 1;
    uint64_t budget = 0, used = 0, peak_used = 0;
    std::vector<lcx::Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<lcx::Pending> pending;
    std::deque<lc_completion> done;
    std::condition_variable cv_done;
    std::thread th;
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, batches = 0;
    uint32_t inflight = 0, peak_inflight = 0;
    cudaMemPool_t pool = nullptr;  // the batches' device memory; never trimmed while the server lives
    double launch_us_max = 0, launch_us_total = 0;
    uint64_t staging_regrows = 0;
};

namespace lcx {
namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Page-locked staging a batch of nqreq query requests (nq queries) and ndreq
// decodes needs: descriptors, work offsets and queries in, query results out
// (the layout launch_batch writes).
size_t staging_bytes(size_t nqreq, size_t ndreq, size_t nq) {
    const size_t o_d = al256(sizeof(SrvReq) * nqreq);
    const size_t o_w = al256(o_d + sizeof(SrvReq) * ndreq);
    const size_t o_in = al256(o_w + 8 * (ndreq + 1));
    const size_t o_out = al256(o_in + 8 * nq);
    return o_out + 8 * nq;
}

uint64_t device_need(const lc_server* s, const lc_request& r) {
    if (r.op == LC_OP_DECODE) return al256(r.count * s->kb);
    return 16 * r.count;  // one 8-byte query in and one 8-byte result out
}

// A request that is wrong on its face completes at once with an error.
int precheck(const lc_server* s, const lc_request& r) {
    if (r.column >= s->cols.size() || (r.count && !r.output)) return LC_ERR_INVALID_ARG;
    const lc_column* c = s->cols[r.column];
    switch (r.op) {
        case LC_OP_ACCESS: {
            if (r.count && !r.input) return LC_ERR_INVALID_ARG;
            const uint64_t* in = (const uint64_t*)r.input;
            for (uint64_t q = 0; q < r.count; ++q)
                if (in[q] >= c->N) return LC_ERR_OUT_OF_RANGE;
            return LC_OK;
        }
        case LC_OP_LOWER_BOUND:
            if (r.count && !r.input) return LC_ERR_INVALID_ARG;
            return c->list_mode ? LC_ERR_UNSUPPORTED : LC_OK;
        case LC_OP_DECODE:
            return (r.begin > c->N || r.count > c->N - r.begin) ? LC_ERR_OUT_OF_RANGE : LC_OK;
        default:
            return LC_ERR_INVALID_ARG;
    }
}

void complete(lc_server* s, const Pending& p, int status, uint32_t batch) {
    lc_completion c;
    c.ticket = p.ticket;
    c.user = p.r.user;
    c.status = status;
    c.batch_size = batch;
    c.latency_us = std::chrono::duration<double, std::micro>(Clock::now() - p.t0).count();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->done.push_back(c);
        ++s->completed;
    }
    s->cv_done.notify_all();
}

// Pack the batch, copy it in, launch, copy results back, record the event.
int launch_batch(lc_server* s, Slot& sl) {
    const uint32_t nreq = (uint32_t)sl.reqs.size();
    std::vector<SrvReq> qr, dr;
    std::vector<uint64_t> work_off(1, 0);
    sl.qoff.assign(nreq, 0);
    uint64_t nq = 0, dec_bytes = 0;
    for (uint32_t i = 0; i < nreq; ++i) {
        const lc_request& r = sl.reqs[i].r;
        SrvReq d{};
        d.col = r.column;
        d.op = r.op;
        d.count = r.count;
        if (r.op == LC_OP_DECODE) {
            if (r.count == 0) continue;
            const lc_column* c = s->cols[r.column];
            d.begin = r.begin;
            d.first_tile = tile_of_key(c, r.begin);
            const uint64_t nt = tile_of_key(c, r.begin + r.count - 1) - d.first_tile + 1;
            d.out = dec_bytes;  // offset for now, device address below
            dec_bytes += al256(r.count * s->kb);
            work_off.push_back(work_off.back() + nt);
            dr.push_back(d);
        } else {
            if (r.count == 0) continue;
            d.qoff = nq;
            sl.qoff[i] = nq;
            nq += r.count;
            qr.push_back(d);
        }
    }
    // device layout: descriptors | work offsets | queries in | results out | decode outputs
    const size_t o_q = 0, o_d = al256(o_q + sizeof(SrvReq) * qr.size());
    const size_t o_w = al256(o_d + sizeof(SrvReq) * dr.size());
    const size_t o_in = al256(o_w + 8 * work_off.size());
    const size_t o_out = al256(o_in + 8 * nq);
    const size_t o_dec = al256(o_out + 8 * nq);
    const size_t total = o_dec + dec_bytes;
    const size_t stage_in = o_out;  // bytes copied in
    const size_t need_h = o_out + 8 * nq;
    if (sl.h_cap < need_h) {  // grow by doubling: page-locking is slow and synchronises the device
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        size_t cap = std::max(sl.h_cap, (size_t)1 << 20);
        while (cap < need_h) cap *= 2;
        sl.h_cap = cap;
        ++s->staging_regrows;
        if (cudaMallocHost((void**)&sl.h_stage, sl.h_cap) != cudaSuccess) {
            sl.h_stage = nullptr;
            sl.h_cap = 0;
            return LC_ERR_NOMEM;
        }
    }
    if (cudaMallocFromPoolAsync((void**)&sl.d_buf, std::max<size_t>(total, 256), s->pool, sl.st) != cudaSuccess)
        return LC_ERR_NOMEM;
    const uint64_t dbase = (uint64_t)(uintptr_t)(sl.d_buf + o_dec);
    for (SrvReq& d : dr) d.out += dbase;
    uint8_t* h = sl.h_stage;
    if (!qr.empty()) memcpy(h + o_q, qr.data(), sizeof(SrvReq) * qr.size());
    if (!dr.empty()) memcpy(h + o_d, dr.data(), sizeof(SrvReq) * dr.size());
    memcpy(h + o_w, work_off.data(), 8 * work_off.size());
    uint64_t* hin = (uint64_t*)(h + o_in);
    for (uint32_t i = 0; i < nreq; ++i) {
        const lc_request& r = sl.reqs[i].r;
        if (r.op == LC_OP_DECODE || r.count == 0) continue;
        uint64_t* dst = hin + sl.qoff[i];
        if (r.op == LC_OP_LOWER_BOUND && s->kb == 4) {
            const uint32_t* src = (const uint32_t*)r.input;
            for (uint64_t q = 0; q < r.count; ++q) dst[q] = src[q];
        } else {
            memcpy(dst, r.input, 8 * r.count);
        }
    }
    int rc = cuda_status(cudaMemcpyAsync(sl.d_buf, h, stage_in, cudaMemcpyHostToDevice, sl.st));
    if (!rc)
        rc = serve_launch(s->d_views, s->kb, (const SrvReq*)(sl.d_buf + o_q), (uint32_t)qr.size(), nq,
                          (const uint64_t*)(sl.d_buf + o_in), (uint64_t*)(sl.d_buf + o_out),
                          (const SrvReq*)(sl.d_buf + o_d), (uint32_t)dr.size(), (const uint64_t*)(sl.d_buf + o_w),
                          work_off.back(), s->max_tile_segs, s->cols[0]->status, sl.st);
    if (!rc && nq) rc = cuda_status(cudaMemcpyAsync(h + o_out, sl.d_buf + o_out, 8 * nq, cudaMemcpyDeviceToHost, sl.st));
    size_t k = 0;
    for (uint32_t i = 0; !rc && i < nreq; ++i) {
        const lc_request& r = sl.reqs[i].r;
        if (r.op != LC_OP_DECODE || r.count == 0) continue;
        rc = cuda_status(cudaMemcpyAsync(r.output, (const void*)(uintptr_t)dr[k].out, r.count * s->kb,
                                         cudaMemcpyDeviceToHost, sl.st));
        ++k;
    }
    if (!rc) rc = cuda_status(cudaEventRecord(sl.ev, sl.st));
    cudaFreeAsync(sl.d_buf, sl.st);
    sl.d_buf = nullptr;
    sl.out_off = o_out;
    return rc;
}

void retire_batch(lc_server* s, Slot& sl, int status) {
    const uint32_t nreq = (uint32_t)sl.reqs.size();
    const uint64_t* hout = (const uint64_t*)(sl.h_stage + sl.out_off);
    for (uint32_t i = 0; i < nreq; ++i) {
        const lc_request& r = sl.reqs[i].r;
        if (!status && r.count && r.op != LC_OP_DECODE) {
            const uint64_t* src = hout + sl.qoff[i];
            if (r.op == LC_OP_ACCESS && s->kb == 4) {
                uint32_t* dst = (uint32_t*)r.output;
                for (uint64_t q = 0; q < r.count; ++q) dst[q] = (uint32_t)src[q];
            } else {
                memcpy(r.output, src, 8 * r.count);
            }
        }
        complete(s, sl.reqs[i], status, nreq);
    }
    sl.reqs.clear();
    sl.busy = false;
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= sl.charged;
    sl.charged = 0;
    --s->inflight;
}

void scheduler(lc_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool active = false;
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            active = true;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            retire_batch(s, sl, q == cudaSuccess ? LC_OK : LC_ERR_CUDA);
        }
        // admit waiting requests into free slots
        for (Slot& sl : s->slots) {
            if (sl.busy) continue;
            std::vector<Pending> take;
            uint64_t charge = 0, nq = 0;
            uint32_t nd = 0;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                while (!s->pending.empty() && take.size() < kMaxBatchRequests) {
                    const Pending& p = s->pending.front();
                    const uint64_t need = device_need(s, p.r);
                    const bool dec = p.r.op == LC_OP_DECODE;
                    if (need > s->budget) {  // can never fit: fail it
                        Pending bad = p;
                        s->pending.pop_front();
                        s->mu.unlock();
                        complete(s, bad, LC_ERR_NOMEM, 1);
                        s->mu.lock();
                        continue;
                    }
                    if (s->used + charge + need > s->budget) break;
                    if (!dec && nq + p.r.count > kMaxBatchQueries && !take.empty()) break;
                    if (dec && nd + 1 > kMaxBatchDecodes) break;
                    charge += need;
                    if (dec) ++nd;
                    else nq += p.r.count;
                    take.push_back(p);
                    s->pending.pop_front();
                }
                if (!take.empty()) {
                    s->used += charge;
                    s->peak_used = std::max(s->peak_used, s->used);
                    ++s->inflight;
                    s->peak_inflight = std::max(s->peak_inflight, s->inflight);
                    ++s->batches;
                }
            }
            if (take.empty()) break;
            sl.reqs = std::move(take);
            sl.charged = charge;
            sl.busy = true;
            active = true;
            const auto tl = Clock::now();
            const int rc = launch_batch(s, sl);
            const double us = std::chrono::duration<double, std::micro>(Clock::now() - tl).count();
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->launch_us_total += us;
                s->launch_us_max = std::max(s->launch_us_max, us);
            }
            if (rc) {
                cudaStreamSynchronize(sl.st);
                retire_batch(s, sl, rc);
            }
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop.load() && s->pending.empty() && s->inflight == 0) break;
            if (!active && s->pending.empty()) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (active) std::this_thread::yield();
    }
}

}  // namespace
}  // namespace lcx

using namespace lcx;

extern "C" {

int lc_server_create(lc_column* const* cols, int ncols, uint64_t hbm_budget, int slots, lc_server** out) {
    if (!cols || !out || ncols < 1 || slots < 1 || slots > 64 || hbm_budget == 0) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    lc_server* s = new (std::nothrow) lc_server;
    if (!s) return LC_ERR_NOMEM;
    cudaGetDevice(&s->device);
    s->kb = (int)cols[0]->key_bytes;
    for (int i = 0; i < ncols; ++i) {
        if (!cols[i] || (int)cols[i]->key_bytes != s->kb || cols[i]->device != s->device) {
            delete s;
            return LC_ERR_INVALID_ARG;
        }
        s->cols.push_back(cols[i]);
        s->max_tile_segs = std::max(s->max_tile_segs, cols[i]->view.max_tile_segs);
    }
    s->budget = hbm_budget;
    std::vector<ColView> views;
    for (lc_column* c : s->cols) views.push_back(c->view);
    if (cudaMalloc((void**)&s->d_views, sizeof(ColView) * views.size()) != cudaSuccess ||
        cudaMemcpy(s->d_views, views.data(), sizeof(ColView) * views.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        if (s->d_views) cudaFree(s->d_views);
        delete s;
        return LC_ERR_NOMEM;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    uint64_t keep = ~0ull;  // keep what the batches freed: re-mapping device memory costs milliseconds
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        if (s->pool) cudaMemPoolDestroy(s->pool);
        cudaFree(s->d_views);
        delete s;
        return LC_ERR_CUDA;
    }
    s->slots.resize(slots);
    // every slot's staging sized for the largest batch the admission rules let
    // through (a single request above the query cap still grows it): growing
    // it while serving page-locks memory and synchronises the device
    const size_t stage = staging_bytes(kMaxBatchRequests, kMaxBatchDecodes, kMaxBatchQueries);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            lc_server_destroy(s);
            return LC_ERR_CUDA;
        }
        if (cudaMallocHost((void**)&sl.h_stage, stage) != cudaSuccess) {
            sl.h_stage = nullptr;
            lc_server_destroy(s);
            return LC_ERR_NOMEM;
        }
        sl.h_cap = stage;
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return LC_OK;
}

int lc_server_submit(lc_server* s, const lc_request* req, uint64_t* ticket) {
    if (!s || !req) return LC_ERR_INVALID_ARG;
    Pending p;
    p.r = *req;
    p.t0 = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop.load()) return LC_ERR_INVALID_ARG;
        p.ticket = s->next_ticket++;
        ++s->submitted;
    }
    if (ticket) *ticket = p.ticket;
    const int pre = precheck(s, p.r);
    if (pre) {
        complete(s, p, pre, 1);
        return LC_OK;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->pending.push_back(p);
    }
    s->cv.notify_one();
    return LC_OK;
}

int lc_server_poll(lc_server* s, lc_completion* out, int max, int* got) {
    if (!s || !got || (max > 0 && !out)) return LC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *got = n;
    return LC_OK;
}

int lc_server_wait(lc_server* s, lc_completion* out, int max, int* got, uint64_t timeout_us) {
    if (!s || !got || (max > 0 && !out)) return LC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->done.empty(); });
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *got = n;
    return n ? LC_OK : LC_ERR_TIMEOUT;
}

int lc_server_stats(lc_server* s, lc_server_stats_t* st) {
    if (!s || !st) return LC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->batches = s->batches;
    st->peak_hbm_bytes = s->peak_used;
    st->peak_inflight = s->peak_inflight;
    st->slots = (uint32_t)s->slots.size();
    st->launch_us_max = s->launch_us_max;
    st->launch_us_total = s->launch_us_total;
    st->staging_regrows = s->staging_regrows;
    return LC_OK;
}

int lc_server_destroy(lc_server* s) {
    if (!s) return LC_ERR_INVALID_ARG;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (Slot& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
    }
    if (s->d_views) cudaFree(s->d_views);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return LC_OK;
}

int lc_serve_sync(lc_column* const* cols, int ncols, const lc_request* req, void* stream, lc_completion* out) {
    if (!cols || !req || !out || req->column >= (uint32_t)ncols) return LC_ERR_INVALID_ARG;
    const auto t0 = Clock::now();
    const lc_column* c = cols[req->column];
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t n = req->count;
    const int kb = (int)c->key_bytes;
    int rc = LC_OK;
    uint8_t* d = nullptr;
    if (n) {
        const size_t in_b = req->op == LC_OP_DECODE ? 0 : al256(8 * n);
        const size_t out_b = 8 * n;
        if (cudaMallocAsync((void**)&d, in_b + out_b, st) != cudaSuccess) return LC_ERR_NOMEM;
        switch (req->op) {
            case LC_OP_ACCESS:
                rc = cuda_status(cudaMemcpyAsync(d, req->input, 8 * n, cudaMemcpyHostToDevice, st));
                if (!rc) rc = lc_access(c, (const uint64_t*)d, n, d + in_b, st);
                if (!rc) rc = cuda_status(cudaMemcpyAsync(req->output, d + in_b, (size_t)kb * n, cudaMemcpyDeviceToHost, st));
                break;
            case LC_OP_LOWER_BOUND:
                rc = cuda_status(cudaMemcpyAsync(d, req->input, (size_t)kb * n, cudaMemcpyHostToDevice, st));
                if (!rc) rc = lc_lower_bound(c, d, n, (uint64_t*)(d + in_b), st);
                if (!rc) rc = cuda_status(cudaMemcpyAsync(req->output, d + in_b, 8 * n, cudaMemcpyDeviceToHost, st));
                break;
            case LC_OP_DECODE:
                rc = lc_decode(c, req->begin, n, d, st);
                if (!rc) rc = cuda_status(cudaMemcpyAsync(req->output, d, (size_t)kb * n, cudaMemcpyDeviceToHost, st));
                break;
            default:
                rc = LC_ERR_INVALID_ARG;
        }
        cudaFreeAsync(d, st);
        const int rs = cuda_status(cudaStreamSynchronize(st));
        if (!rc) rc = rs;
    }
    if (!rc && req->op == LC_OP_ACCESS) rc = lc_status(c, st);
    out->ticket = 0;
    out->user = req->user;
    out->status = rc;
    out->batch_size = 1;
    out->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    return LC_OK;
}

}  // extern "C"
