// Serving: continuous batching of motif-count requests on one GPU.
//
// Requests (host edge lists, copied at submit into a page-locked staging arena when it has room)
// wait in a FIFO.  Two builder threads admit them in order while the device memory held by admitted
// requests stays within the HBM budget and a slot is free, copy each edge list to the device and
// build its CSR, each on its own copy stream.  Built requests go to one of two lanes by size: small
// requests (at most small_edges input pairs) and the rest.  Each lane has an executor thread that
// takes every built request of its lane as the next batch and counts it with the batched pipeline
// (the disjoint union of the batch, one launch per kernel) on the lane's compute stream; the small
// lane's stream has the higher priority, so when a large batch's kernel finishes its blocks the small
// batch's kernels are scheduled first and a small request does not wait for a whole large batch.
// With a batching window an executor first waits, up to the window, while requests are still queued
// for admission or being built.  Requests that arrive while batches are on the GPU are admitted,
// copied and built meanwhile (their copies and CSR builds overlap the running counts) and form their
// lane's next batch as soon as its current one finishes; results are retired per ticket.
// A request whose own footprint exceeds the budget is counted by the halo-partitioned path with the
// canonical anchor-owner rule (harp_count4_partitioned) under the same budget.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "harp_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum class ReqState { Pending, Built, Running, Done };

// First-fit allocator over one page-locked host block (caller holds the server lock).
struct StagingArena {
    unsigned char* base = nullptr;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;  // offset -> size, coalesced

    void init(void* p, size_t n) {
        base = static_cast<unsigned char*>(p);
        bytes = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    void* alloc(size_t n) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            return base + off;
        }
        return nullptr;
    }
    void release(void* p, size_t n) {
        if (!p) return;
        n = (n + 255) & ~(size_t)255;
        size_t off = static_cast<unsigned char*>(p) - base;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                n += prev->second;
                free_.erase(prev);
            }
        }
        free_[off] = n;
    }
};

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0, m_in = 0;
    std::vector<int32_t> src, dst;    // pageable copy (when the staging arena had no room)
    int32_t* staged = nullptr;        // [2 * m_in] in the staging arena: src then dst
    const int32_t* hsrc = nullptr;    // the edge list the builder reads
    const int32_t* hdst = nullptr;
    ReqState state = ReqState::Pending;
    harp_status status = HARP_OK;
    uint64_t counts[6] = {0, 0, 0, 0, 0, 0};
    size_t need = 0;  // device bytes this request holds from admission to completion
    harp_csr* csr = nullptr;
    bool partitioned = false;
    Clock::time_point t_submit, t_done;
};

// Device bytes one request holds while resident: its CSR, its share of the batch's union copy and
// counting workspace (estimated with the input pair count as an upper bound of the edge count).
size_t footprint(int64_t n, int64_t m_in) {
    harp::Workspace probe;
    const size_t ws = harp::ws_layout(probe, nullptr, n, m_in);
    const size_t csr = sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * 2 * (size_t)m_in;
    const size_t batch_share = csr + sizeof(int32_t) * 2 * (size_t)n + 16 * sizeof(uint64_t) * 2;
    const size_t build_tmp = sizeof(uint64_t) * 2 * 2 * (size_t)m_in + sizeof(int64_t) * (2 * (size_t)m_in + 1) +
                             sizeof(int32_t) * 4 * (size_t)m_in;
    const size_t steady = csr + batch_share + ws;
    return steady > build_tmp + csr ? steady : build_tmp + csr;
}

}  // namespace

struct harp_server {
    int device = 0;
    harp_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_build;   // builder: pending work or room freed
    std::condition_variable cv_exec;    // executor: built requests available
    std::condition_variable cv_done;    // waiters: a request finished
    std::deque<uint64_t> pending;       // tickets in arrival order
    static constexpr int kLanes = 2;    // 0: large requests, 1: small requests (higher priority)
    std::deque<uint64_t> built[kLanes]; // tickets with a CSR, waiting for a batch of their lane
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1;
    size_t resident = 0;
    size_t peak_resident = 0;
    int64_t inflight = 0;
    int64_t building = 0;               // requests between admission and a built CSR
    bool stop = false;
    static constexpr int kBuilders = 2;
    cudaStream_t copy_stream[kBuilders] = {nullptr, nullptr};
    cudaStream_t compute_stream[kLanes] = {nullptr, nullptr};
    std::thread builder[kBuilders], executor[kLanes];
    StagingArena staging;
    // statistics
    uint64_t completed = 0, batches = 0, partitioned = 0, batched_requests = 0, max_batch_seen = 0;
    std::vector<double> latencies_ms;   // ring of the last kLatencyRing completions
    size_t latency_next = 0;
};

namespace {

constexpr size_t kLatencyRing = 65536;

void finish(harp_server* s, Request* r, harp_status st) {
    r->status = st;
    r->state = ReqState::Done;
    r->t_done = Clock::now();
    const double ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (s->latencies_ms.size() < kLatencyRing) s->latencies_ms.push_back(ms);
    else s->latencies_ms[s->latency_next] = ms;
    s->latency_next = (s->latency_next + 1) % kLatencyRing;
    s->completed++;
}

// The head of the queue can be admitted now (caller holds the lock): a free slot, and room in the
// budget.  An oversize request runs alone under the whole budget; others must fit beside the
// resident set.
bool can_admit(const harp_server* s) {
    if (s->pending.empty()) return false;
    const Request* r = s->reqs.at(s->pending.front());
    const bool slot = s->opts.max_inflight == 0 || s->inflight < (int64_t)s->opts.max_inflight;
    const bool oversize = r->need > s->opts.hbm_budget_bytes;
    return slot && (oversize ? s->resident == 0 : s->resident + r->need <= s->opts.hbm_budget_bytes);
}

// Lane of a request: 1 (small, the higher-priority stream) for at most small_edges input pairs.
int lane_of(const harp_server* s, const Request* r) {
    const uint64_t small = s->opts.small_edges ? s->opts.small_edges : 65536u;
    return (uint64_t)r->m_in <= small ? 1 : 0;
}

void drop_host_copy(harp_server* s, Request* r) {  // caller holds the lock
    if (r->staged) s->staging.release(r->staged, sizeof(int32_t) * 2 * (size_t)r->m_in);
    r->staged = nullptr;
    r->hsrc = r->hdst = nullptr;
    std::vector<int32_t>().swap(r->src);
    std::vector<int32_t>().swap(r->dst);
}

void builder_loop(harp_server* s, int which) {
    cudaSetDevice(s->device);
    cudaStream_t stream = s->copy_stream[which];
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_build.wait(lk, [&] { return s->stop || can_admit(s); });
        if (s->stop) return;
        Request* r = s->reqs[s->pending.front()];
        s->pending.pop_front();
        const bool oversize = r->need > s->opts.hbm_budget_bytes;
        const size_t charge = oversize ? s->opts.hbm_budget_bytes : r->need;
        s->resident += charge;
        if (s->resident > s->peak_resident) s->peak_resident = s->resident;
        s->inflight++;
        harp_status st;
        if (oversize) {
            lk.unlock();
            // halo-partitioned path with the owner rule, within the budget; counted right here
            st = harp_count4_partitioned(r->n, r->m_in, r->hsrc, r->hdst, s->opts.hbm_budget_bytes, 0, r->counts,
                                         nullptr);
            lk.lock();
            drop_host_copy(s, r);
            r->partitioned = true;
            s->partitioned++;
            s->resident -= charge;
            s->inflight--;
            finish(s, r, st);
            s->cv_done.notify_all();
            s->cv_build.notify_all();
            continue;
        }
        s->building++;
        lk.unlock();
        st = harp_build_csr(r->n, r->m_in, r->hsrc, r->hdst, HARP_PTR_HOST, stream, &r->csr);
        lk.lock();
        s->building--;
        drop_host_copy(s, r);  // the build has copied and synchronised
        if (st != HARP_OK) {
            s->resident -= charge;
            s->inflight--;
            finish(s, r, st);
            s->cv_done.notify_all();
            s->cv_exec.notify_all();  // a waiting batch need not wait for this one
            continue;
        }
        r->state = ReqState::Built;
        s->built[lane_of(s, r)].push_back(r->ticket);
        s->cv_exec.notify_all();
    }
}

void executor_loop(harp_server* s, int lane) {
    cudaSetDevice(s->device);
    std::deque<uint64_t>& built = s->built[lane];
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_exec.wait(lk, [&] { return s->stop || !built.empty(); });
        if (s->stop) return;
        const size_t cap = s->opts.max_batch ? s->opts.max_batch : 4096;
        if (s->opts.batch_window_us) {
            // gather: wait, up to the window, while more requests are on their way (being built, or
            // admissible now); requests held back by the budget cannot join before this batch ends
            s->cv_exec.wait_for(lk, std::chrono::microseconds(s->opts.batch_window_us), [&] {
                return s->stop || built.size() >= cap || (s->building == 0 && !can_admit(s));
            });
            if (s->stop) return;
        }
        std::vector<Request*> batch;
        while (!built.empty() && batch.size() < cap) {
            Request* r = s->reqs[built.front()];
            built.pop_front();
            r->state = ReqState::Running;
            batch.push_back(r);
        }
        lk.unlock();
        std::vector<const harp_csr*> hs(batch.size());
        for (size_t k = 0; k < batch.size(); ++k) hs[k] = batch[k]->csr;
        std::vector<uint64_t> counts(6 * batch.size());
        harp_batch* b = nullptr;
        harp_status st = harp_batch_create(hs.data(), (int64_t)hs.size(), &b);
        if (st == HARP_OK) {
            harp_plan p;
            std::memset(&p, 0, sizeof(p));
            p.version = HARP_ABI_VERSION;
            p.flags = HARP_PLAN_NO_GRAPH;  // every batch has a different shape
            st = harp_batch_count(b, &p, reinterpret_cast<uint64_t(*)[6]>(counts.data()), nullptr,
                                  s->compute_stream[lane]);
            harp_batch_free(b);
        }
        for (Request* r : batch) {
            harp_csr_free(r->csr);
            r->csr = nullptr;
        }
        lk.lock();
        s->batches++;
        s->batched_requests += batch.size();
        if (batch.size() > s->max_batch_seen) s->max_batch_seen = batch.size();
        for (size_t k = 0; k < batch.size(); ++k) {
            Request* r = batch[k];
            if (st == HARP_OK) std::memcpy(r->counts, &counts[6 * k], sizeof(r->counts));
            s->resident -= r->need;
            s->inflight--;
            finish(s, r, st);
        }
        s->cv_done.notify_all();
        s->cv_build.notify_all();
    }
}

}  // namespace

extern "C" {

harp_status harp_server_create(const harp_server_opts* opts, harp_server** out) {
    if (!out) return HARP_EINVAL;
    harp_server* s = new (std::nothrow) harp_server();
    if (!s) return HARP_ENOMEM;
    if (opts) s->opts = *opts;
    if (s->opts.hbm_budget_bytes == 0) s->opts.hbm_budget_bytes = (uint64_t)64 << 30;
    if (s->opts.staging_mib == 0) s->opts.staging_mib = 512;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return HARP_ECUDA;
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < harp_server::kBuilders && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithFlags(&s->copy_stream[k], cudaStreamNonBlocking);
    // lane 1 (small requests) gets the greatest priority the device offers, lane 0 the least
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&s->compute_stream[0], cudaStreamNonBlocking, prio_least);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&s->compute_stream[1], cudaStreamNonBlocking, prio_greatest);
    void* arena = nullptr;
    const size_t arena_bytes = (size_t)s->opts.staging_mib << 20;
    if (e == cudaSuccess) e = cudaMallocHost(&arena, arena_bytes);
    if (e != cudaSuccess) {
        harp::record_cuda_error(e);
        for (cudaStream_t c : s->copy_stream)
            if (c) cudaStreamDestroy(c);
        for (cudaStream_t c : s->compute_stream)
            if (c) cudaStreamDestroy(c);
        delete s;
        return e == cudaErrorMemoryAllocation ? HARP_ENOMEM : HARP_ECUDA;
    }
    s->staging.init(arena, arena_bytes);
    for (int k = 0; k < harp_server::kBuilders; ++k) s->builder[k] = std::thread(builder_loop, s, k);
    for (int k = 0; k < harp_server::kLanes; ++k) s->executor[k] = std::thread(executor_loop, s, k);
    *out = s;
    return HARP_OK;
}

harp_status harp_submit(harp_server* s, int64_t n, int64_t m_in, const int32_t* src, const int32_t* dst,
                        uint64_t* ticket) {
    if (!s || !ticket || n < 0 || m_in < 0 || (m_in > 0 && (!src || !dst))) return HARP_EINVAL;
    if (n > 2147483647LL || m_in > 2147483647LL) return HARP_EOVERFLOW;
    Request* r = new (std::nothrow) Request();
    if (!r) return HARP_ENOMEM;
    r->n = n;
    r->m_in = m_in;
    r->need = footprint(n, m_in);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (m_in > 0) r->staged = static_cast<int32_t*>(s->staging.alloc(sizeof(int32_t) * 2 * (size_t)m_in));
    }
    if (r->staged) {
        std::memcpy(r->staged, src, sizeof(int32_t) * (size_t)m_in);
        std::memcpy(r->staged + m_in, dst, sizeof(int32_t) * (size_t)m_in);
        r->hsrc = r->staged;
        r->hdst = r->staged + m_in;
    } else if (m_in > 0) {
        try {
            r->src.assign(src, src + m_in);
            r->dst.assign(dst, dst + m_in);
        } catch (...) {
            delete r;
            return HARP_ENOMEM;
        }
        r->hsrc = r->src.data();
        r->hdst = r->dst.data();
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        drop_host_copy(s, r);
        delete r;
        return HARP_EINVAL;
    }
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->pending.push_back(r->ticket);
    *ticket = r->ticket;
    s->cv_build.notify_one();
    return HARP_OK;
}

harp_status harp_poll(harp_server* s, uint64_t ticket, uint64_t counts_out[6], int* done) {
    if (!s || !done) return HARP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HARP_ENOTFOUND;
    Request* r = it->second;
    if (r->state != ReqState::Done) {
        *done = 0;
        return HARP_OK;
    }
    *done = 1;
    const harp_status st = r->status;
    if (st == HARP_OK && counts_out) std::memcpy(counts_out, r->counts, sizeof(r->counts));
    s->reqs.erase(it);
    delete r;
    return st;
}

harp_status harp_wait(harp_server* s, uint64_t ticket, uint64_t counts_out[6], double timeout_ms) {
    if (!s) return HARP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HARP_ENOTFOUND;
    Request* r = it->second;
    const auto pred = [&] { return r->state == ReqState::Done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) {
        return HARP_ETIMEOUT;
    }
    const harp_status st = r->status;
    if (st == HARP_OK && counts_out) std::memcpy(counts_out, r->counts, sizeof(r->counts));
    s->reqs.erase(ticket);
    delete r;
    return st;
}

harp_status harp_server_get_stats(harp_server* s, harp_server_stats* out) {
    if (!s || !out) return HARP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->completed = s->completed;
    out->batches = s->batches;
    out->batched_requests = s->batched_requests;
    out->partitioned = s->partitioned;
    out->max_batch = s->max_batch_seen;
    out->pending = s->pending.size() + s->built[0].size() + s->built[1].size();
    out->resident_bytes = s->resident;
    out->peak_resident_bytes = s->peak_resident;
    out->latency_p50_us = out->latency_p99_us = 0;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v(s->latencies_ms);
        auto q = [&](double f) {
            const size_t k = (size_t)(f * (double)(v.size() - 1) + 0.5);
            std::nth_element(v.begin(), v.begin() + (long)k, v.end());
            return (uint64_t)(v[k] * 1000.0 + 0.5);
        };
        out->latency_p50_us = q(0.50);
        out->latency_p99_us = q(0.99);
    }
    return HARP_OK;
}

void harp_server_destroy(harp_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_build.notify_all();
    s->cv_exec.notify_all();
    for (auto& b : s->builder)
        if (b.joinable()) b.join();
    for (auto& x : s->executor)
        if (x.joinable()) x.join();
    cudaSetDevice(s->device);
    for (auto& kv : s->reqs) {
        if (kv.second->csr) harp_csr_free(kv.second->csr);
        delete kv.second;
    }
    for (cudaStream_t c : s->copy_stream) {
        cudaStreamSynchronize(c);
        cudaStreamDestroy(c);
    }
    for (cudaStream_t c : s->compute_stream) {
        cudaStreamSynchronize(c);
        cudaStreamDestroy(c);
    }
    cudaFreeHost(s->staging.base);
    delete s;
}

}  // extern "C"
