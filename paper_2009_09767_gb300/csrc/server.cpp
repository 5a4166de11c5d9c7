// server.cpp -- continuous-batching SVD service on one GPU (include/ranky.h,
// svd_server_*).
//
// A scheduler thread owns the device: it admits submitted requests in arrival
// order whenever a stream slot is free and the request fits in what is left
// of the device-memory budget, places its plan workspace, CSC and outputs in
// one allocation from a first-fit pool over a single budget-sized device
// buffer, and enqueues host->device copies, the SVD and device->host copies
// on the slot's stream.  Consecutive small requests waiting together are
// admitted into one slot as a group and run as ONE batched pass (the slot's
// reusable batch: all their block eigensolves in one persistent launch, all
// their merge eigensolves in another); a large request, or one arriving
// alone, runs by itself.  Requests that arrive while others are running are
// admitted as slots and memory free up, so their kernels overlap on the GPU.
// Completion is detected by polling one CUDA event per admitted group; the
// requests' pool memory and plans are released at once and their latency
// stamped.
//
// Fault injection for the tests is host-side only: a chosen ticket can be
// made to fail its pool allocation (SVD_INJECT_ALLOC) or to have its CSC
// treated as malformed (SVD_INJECT_BAD_CSC).  Nothing here makes the GPU
// fault or wait forever.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ranky.h"
#include "batch_engine.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) with 256-byte granules.
class Pool {
public:
    explicit Pool(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align256(std::max<size_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align256(std::max<size_t>(bytes, 1));
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

enum State { kPending = 0, kRunning = 1, kDone = 2 };

// Grouping: requests of at most kSmallM rows and kSmallBlocks blocks batch
// together, up to kMaxGroup per pass and kEngineItems eigensolves.
constexpr int kSmallM = 256;
constexpr int kSmallBlocks = 16;
constexpr int kMaxGroup = 64;
constexpr size_t kEngineItems = kMaxGroup * (kSmallBlocks + 1);

struct Request {
    uint64_t ticket = 0;
    svd_desc desc{};
    std::vector<int64_t> bounds;
    svd_request io{};
    State state = kPending;
    svd_status result = SVD_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t plan_bytes = 0, total_bytes = 0, off = 0;
    svd_plan_t plan = nullptr;
    int slot = -1;
    cudaEvent_t done_ev = nullptr;
    bool inject_alloc = false, inject_bad_csc = false;
    void* direct_v = nullptr;   // device address of a page-locked h_V (written in place)
    char* base_at = nullptr;    // the request's pool allocation
};

struct Layout {
    size_t plan, col_ptr, row_idx, vals, sigma, U, V, rank, total;
};

Layout layout(const svd_desc& d, size_t plan_bytes, bool v_buffer) {
    const int64_t k = d.k > 0 ? d.k : std::min<int64_t>(d.M, d.N);
    const size_t sv = d.value_type == SVD_VALUE_F32 ? 4 : 8;
    const size_t sV = d.precision == SVD_PREC_MIXED ? 4 : 8;
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += align256(std::max<size_t>(bytes, 1)); return at; };
    L.plan = take(plan_bytes);
    L.col_ptr = take(sizeof(int64_t) * (size_t)(d.N + 1));
    L.row_idx = take(sizeof(int32_t) * (size_t)d.nnz);
    L.vals = take(sv * (size_t)d.nnz);
    L.sigma = take(sizeof(double) * (size_t)k);
    L.U = take(sizeof(double) * (size_t)d.M * (size_t)k);
    L.V = take((d.flags & SVD_FLAG_SKIP_V) || !v_buffer ? 1 : sV * (size_t)d.N * (size_t)k);
    L.rank = take(sizeof(int32_t));
    L.total = off;
    return L;
}

}  // namespace

struct svd_server_s {
    int device = 0;
    size_t budget = 0;
    char* base = nullptr;
    Pool* pool = nullptr;
    int max_inflight = 1;
    std::vector<cudaStream_t> streams;
    std::vector<int> slot_busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<std::vector<Request*>> running;   // admitted groups (event of the first)
    std::vector<svd_batch_t> engines;             // one reusable batch per slot
    std::unordered_map<uint64_t, Request*> all;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_rejected = 0;
    std::unordered_map<uint64_t, int> injections;
};

namespace {

void finish(svd_server_s* s, Request* r, svd_status st) {
    r->result = st;
    r->state = kDone;
    r->t_done = now_s();
    if (st == SVD_OK) ++s->n_completed; else ++s->n_failed;
}

// Device addresses of one placed request.
struct Placed {
    int64_t* cp;
    int32_t* ri;
    void* va;
    double* sg;
    double* U;
    void* V;
    int32_t* rk;
    bool want_v;
};

// Place one admitted request's plan and copy its inputs on stream st
// (scheduler thread, lock NOT held: copies from pageable host memory can
// block this thread).
svd_status setup(Request* r, cudaStream_t st, Placed& P) {
    char* at = r->base_at;
    const Layout L = layout(r->desc, r->plan_bytes, r->direct_v == nullptr);
    svd_status res = svd_plan_ws(&r->desc, at + L.plan, r->plan_bytes, &r->plan);
    if (res != SVD_OK) return res;
    const svd_desc& d = r->desc;
    const size_t sv = d.value_type == SVD_VALUE_F32 ? 4 : 8;
    P.want_v = r->io.h_V && !(d.flags & SVD_FLAG_SKIP_V);
    P.cp = reinterpret_cast<int64_t*>(at + L.col_ptr);
    P.ri = reinterpret_cast<int32_t*>(at + L.row_idx);
    P.va = at + L.vals;
    P.sg = reinterpret_cast<double*>(at + L.sigma);
    P.U = reinterpret_cast<double*>(at + L.U);
    P.V = r->direct_v ? r->direct_v : at + L.V;
    P.rk = reinterpret_cast<int32_t*>(at + L.rank);
    bool ok = cudaMemcpyAsync(P.cp, r->io.h_col_ptr, sizeof(int64_t) * (d.N + 1),
                              cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (d.nnz > 0) {
        ok = ok && cudaMemcpyAsync(P.ri, r->io.h_row_idx, sizeof(int32_t) * d.nnz,
                                   cudaMemcpyHostToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(P.va, r->io.h_vals, sv * d.nnz, cudaMemcpyHostToDevice, st) ==
                       cudaSuccess;
    }
    if (!ok) { cudaGetLastError(); return SVD_ERR_CUDA; }
    if (r->inject_bad_csc) {
        // the host-side stand-in for a malformed request: a column pointer
        // that does not end at nnz, which the CSC check rejects
        int64_t bad = d.nnz + 1;
        cudaMemcpyAsync(P.cp + d.N, &bad, sizeof(bad), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    if (d.flags & SVD_FLAG_CHECK_CSC) {
        res = svd_check_csc(d.M, d.N, d.nnz, P.cp, P.ri, st);
        if (res != SVD_OK) return res;
    }
    return SVD_OK;
}

// Results back to the request's host buffers on stream st.
svd_status copy_back(Request* r, const Placed& P, cudaStream_t st) {
    const svd_desc& d = r->desc;
    const int64_t k = d.k > 0 ? d.k : std::min<int64_t>(d.M, d.N);
    const size_t sV = d.precision == SVD_PREC_MIXED ? 4 : 8;
    bool ok = cudaMemcpyAsync(r->io.h_sigma, P.sg, sizeof(double) * k, cudaMemcpyDeviceToHost, st) ==
              cudaSuccess;
    ok = ok && cudaMemcpyAsync(r->io.h_U, P.U, sizeof(double) * d.M * k, cudaMemcpyDeviceToHost,
                               st) == cudaSuccess;
    if (P.want_v && !r->direct_v)
        ok = ok && cudaMemcpyAsync(r->io.h_V, P.V, sV * (size_t)d.N * k, cudaMemcpyDeviceToHost,
                                   st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(r->io.h_rank, P.rk, sizeof(int32_t), cudaMemcpyDeviceToHost, st) ==
                   cudaSuccess;
    if (!ok) { cudaGetLastError(); return SVD_ERR_CUDA; }
    return SVD_OK;
}

// Start one admitted group on its slot (lock NOT held): place every request,
// run the group (one request: svd_run; several: one batched pass on the
// slot's batch) and queue the copies back; the group's event is recorded on
// the slot stream after all of it.  res[i] is request i's status; the
// requests with SVD_OK form the running group (event: the first one's).
void start_group(svd_server_s* s, const std::vector<Request*>& g, std::vector<svd_status>& res) {
    const int slot = g[0]->slot;
    cudaStream_t st = s->streams[slot];
    res.assign(g.size(), SVD_OK);
    std::vector<Placed> P(g.size());
    std::vector<size_t> live;
    for (size_t i = 0; i < g.size(); ++i) {
        res[i] = setup(g[i], st, P[i]);
        if (res[i] == SVD_OK) live.push_back(i);
    }
    svd_status run = SVD_OK;
    if (live.size() == 1) {
        const size_t i = live[0];
        run = svd_run(g[i]->plan, P[i].cp, P[i].ri, P[i].va, P[i].sg, P[i].U, P[i].want_v ? P[i].V : nullptr,
                      P[i].rk, nullptr, nullptr, st);
    } else if (live.size() > 1) {
        std::vector<svd_plan_t> plans;
        std::vector<svd_io> ios;
        for (size_t i : live) {
            plans.push_back(g[i]->plan);
            ios.push_back(svd_io{P[i].cp, P[i].ri, P[i].va, P[i].sg, P[i].U,
                                 P[i].want_v ? P[i].V : nullptr, P[i].rk, nullptr, nullptr});
        }
        run = batch_engine_assign(s->engines[slot], (int)plans.size(), plans.data(), st);
        if (run == SVD_OK) run = svd_batch_run(s->engines[slot], ios.data(), st);
    }
    for (size_t i : live) {
        res[i] = run;
        if (res[i] == SVD_OK) res[i] = copy_back(g[i], P[i], st);
    }
    // the event of the first running request marks the whole group
    for (size_t i : live)
        if (res[i] == SVD_OK) {
            if (cudaEventRecord(g[i]->done_ev, st) != cudaSuccess) {
                cudaGetLastError();
                for (size_t j : live) res[j] = SVD_ERR_CUDA;
            }
            break;
        }
}

void release(svd_server_s* s, Request* r) {
    if (r->plan) { svd_free(r->plan); r->plan = nullptr; }
    if (r->total_bytes) { s->pool->release(r->off, r->total_bytes); r->total_bytes = 0; }
    r->slot = -1;
}

bool small_request(const Request* r) {
    return r->desc.M <= kSmallM && r->desc.num_blocks <= kSmallBlocks && !r->inject_alloc &&
           !r->inject_bad_csc && r->desc.merge_arity <= 1;
}

void scheduler(svd_server_s* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        // completions: one event per running group
        for (size_t i = 0; i < s->running.size();) {
            std::vector<Request*>& g = s->running[i];
            const cudaError_t q = cudaEventQuery(g[0]->done_ev);
            if (q == cudaErrorNotReady) { ++i; continue; }
            if (q != cudaSuccess) cudaGetLastError();
            const int slot = g[0]->slot;
            std::vector<svd_status> sts(g.size());
            for (size_t j = 0; j < g.size(); ++j)
                sts[j] = q == cudaSuccess ? svd_sync(g[j]->plan) : SVD_ERR_CUDA;
            // a batched group's plans leave the slot's batch before they are freed
            if (g.size() > 1) batch_engine_detach(s->engines[slot]);
            for (size_t j = 0; j < g.size(); ++j) {
                release(s, g[j]);
                finish(s, g[j], sts[j]);
            }
            s->slot_busy[slot] = 0;
            s->running.erase(s->running.begin() + i);
            progressed = true;
        }
        // admissions, in arrival order: reserve a slot and pool memory; a small
        // request takes the small ones queued right behind it into its group
        std::vector<std::vector<Request*>> admitted;
        while (!s->pending.empty()) {
            int slot = -1;
            for (int i = 0; i < s->max_inflight; ++i)
                if (!s->slot_busy[i]) { slot = i; break; }
            if (slot < 0) break;
            Request* r = s->pending.front();
            if (r->inject_alloc) {
                s->pending.pop_front();
                finish(s, r, SVD_ERR_OOM);
                progressed = true;
                continue;
            }
            std::vector<Request*> g;
            size_t items = 0;
            while (!s->pending.empty()) {
                Request* q = s->pending.front();
                if (!g.empty() && (!small_request(g[0]) || !small_request(q) ||
                                   (int)g.size() >= kMaxGroup ||
                                   items + q->desc.num_blocks + 1 > kEngineItems))
                    break;
                size_t off = 0;
                if (!s->pool->alloc(q->total_bytes, &off)) break;   // wait for memory
                s->pending.pop_front();
                q->off = off;
                q->base_at = s->base + off;
                q->slot = slot;
                q->t_admit = now_s();
                q->state = kRunning;
                items += q->desc.num_blocks + 1;
                g.push_back(q);
            }
            if (g.empty()) break;
            s->slot_busy[slot] = 1;
            admitted.push_back(std::move(g));
        }
        if (!admitted.empty()) {
            // enqueue their work without holding the lock
            lk.unlock();
            std::vector<std::vector<svd_status>> res(admitted.size());
            for (size_t i = 0; i < admitted.size(); ++i) {
                start_group(s, admitted[i], res[i]);
                // a request that failed part-way may still have copies in flight
                // on the slot's stream: let them land before its memory is reused
                for (svd_status st : res[i])
                    if (st != SVD_OK) { cudaStreamSynchronize(s->streams[admitted[i][0]->slot]); break; }
            }
            lk.lock();
            for (size_t i = 0; i < admitted.size(); ++i) {
                std::vector<Request*> run;
                const int slot = admitted[i][0]->slot;
                // a failed request's plan must leave the batch before it is freed.
                // The slot's stream was synchronised above whenever a member
                // failed, so the batched pass of the survivors has finished
                // (batch_engine_detach's precondition); their completion only
                // waits on the group's event and frees them afterwards.
                for (size_t j = 0; j < admitted[i].size(); ++j)
                    if (res[i][j] != SVD_OK) {
                        batch_engine_detach(s->engines[slot]);
                        break;
                    }
                for (size_t j = 0; j < admitted[i].size(); ++j) {
                    Request* r = admitted[i][j];
                    if (res[i][j] == SVD_OK) {
                        run.push_back(r);
                    } else {
                        release(s, r);
                        finish(s, r, res[i][j]);
                    }
                }
                if (run.empty()) s->slot_busy[slot] = 0;
                else s->running.push_back(std::move(run));
            }
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        if (s->stop && s->running.empty() && s->pending.empty()) break;
        if (!progressed) {
            if (s->running.empty() && !s->stop)
                s->cv_work.wait(lk);
            else
                s->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace

extern "C" {

svd_status svd_server_create(size_t budget_bytes, int32_t max_inflight, svd_server_t* out) {
    if (!out || budget_bytes < 4096 || max_inflight < 1 || max_inflight > 256)
        return SVD_ERR_INVALID_ARG;
    *out = nullptr;
    svd_server_s* s = new (std::nothrow) svd_server_s();
    if (!s) return SVD_ERR_OOM;
    cudaGetDevice(&s->device);
    s->budget = budget_bytes & ~(size_t)255;
    if (cudaMalloc(&s->base, s->budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return SVD_ERR_OOM;
    }
    s->pool = new Pool(s->budget);
    s->max_inflight = max_inflight;
    s->streams.resize(max_inflight);
    s->slot_busy.assign(max_inflight, 0);
    for (auto& st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->engines.assign(max_inflight, nullptr);
    for (auto& e : s->engines) {
        if (batch_engine_create(4, kEngineItems, &e) != SVD_OK) {
            for (auto& f : s->engines)
                if (f) svd_batch_free(f);
            for (auto& st : s->streams) cudaStreamDestroy(st);
            cudaFree(s->base);
            delete s->pool;
            delete s;
            return SVD_ERR_OOM;
        }
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return SVD_OK;
}

svd_status svd_server_submit(svd_server_t s, const svd_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || !req->h_col_ptr || !req->h_sigma || !req->h_U || !req->h_rank)
        return SVD_ERR_INVALID_ARG;
    if (req->desc.flags & SVD_FLAG_TALL) return SVD_ERR_UNSUPPORTED;
    size_t plan_bytes = 0;
    svd_status st = svd_plan_bytes(&req->desc, &plan_bytes);
    if (st != SVD_OK) return st;
    Request* r = new (std::nothrow) Request();
    if (!r) return SVD_ERR_OOM;
    r->desc = req->desc;
    if (req->desc.block_col_bounds) {
        r->bounds.assign(req->desc.block_col_bounds,
                         req->desc.block_col_bounds + req->desc.num_blocks + 1);
        r->desc.block_col_bounds = r->bounds.data();
    }
    r->io = *req;
    if (!req->h_V) r->desc.flags |= SVD_FLAG_SKIP_V;   // no V wanted: none computed
    r->plan_bytes = plan_bytes;
    // a page-locked V buffer is written in place by the device (no staging
    // buffer in the pool, no copy); not with rank-fix insertions, whose V
    // correction uses atomic adds
    if (req->h_V && !(r->desc.flags & SVD_FLAG_SKIP_V) && r->desc.rank_fix == SVD_RANKFIX_TRUNCATE) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, req->h_V) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer)
            r->direct_v = at.devicePointer;
        cudaGetLastError();
    }
    r->total_bytes = layout(r->desc, plan_bytes, r->direct_v == nullptr).total;
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->total_bytes > s->budget) {
        ++s->n_rejected;
        delete r;
        return SVD_ERR_BUDGET;
    }
    if (cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return SVD_ERR_CUDA;
    }
    r->ticket = s->next_ticket++;
    auto inj = s->injections.find(r->ticket);
    if (inj != s->injections.end()) {
        r->inject_alloc = inj->second == SVD_INJECT_ALLOC;
        r->inject_bad_csc = inj->second == SVD_INJECT_BAD_CSC;
        if (r->inject_bad_csc) r->desc.flags |= SVD_FLAG_CHECK_CSC;
        s->injections.erase(inj);
    }
    r->t_submit = now_s();
    s->pending.push_back(r);
    s->all[r->ticket] = r;
    ++s->n_submitted;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return SVD_OK;
}

svd_status svd_server_poll(svd_server_t s, uint64_t ticket, int32_t* done, svd_status* result) {
    if (!s || !done) return SVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SVD_ERR_INVALID_ARG;
    *done = it->second->state == kDone;
    if (result) *result = it->second->result;
    return SVD_OK;
}

svd_status svd_server_wait(svd_server_t s, uint64_t ticket, double timeout_s, svd_status* result) {
    if (!s) return SVD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SVD_ERR_INVALID_ARG;
    Request* r = it->second;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(std::max(timeout_s, 0.0)));
    while (r->state != kDone) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != kDone)
            return SVD_ERR_TIMEOUT;
    }
    if (result) *result = r->result;
    return SVD_OK;
}

svd_status svd_server_cancel(svd_server_t s, uint64_t ticket) {
    if (!s) return SVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SVD_ERR_INVALID_ARG;
    Request* r = it->second;
    if (r->state != kPending) return SVD_ERR_INVALID_ARG;   // only queued requests
    s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), r), s->pending.end());
    r->state = kDone;
    r->result = SVD_ERR_INVALID_ARG;
    r->t_done = now_s();
    ++s->n_failed;
    s->cv_done.notify_all();
    return SVD_OK;
}

svd_status svd_server_times(svd_server_t s, uint64_t ticket, double* t_submit, double* t_admit,
                            double* t_done) {
    if (!s) return SVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SVD_ERR_INVALID_ARG;
    if (t_submit) *t_submit = it->second->t_submit;
    if (t_admit) *t_admit = it->second->t_admit;
    if (t_done) *t_done = it->second->t_done;
    return SVD_OK;
}

svd_status svd_server_release(svd_server_t s, uint64_t ticket) {
    if (!s) return SVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end() || it->second->state != kDone) return SVD_ERR_INVALID_ARG;
    if (it->second->done_ev) cudaEventDestroy(it->second->done_ev);
    delete it->second;
    s->all.erase(it);
    return SVD_OK;
}

svd_status svd_server_inject(svd_server_t s, int32_t what, uint64_t ticket) {
    if (!s || (what != SVD_INJECT_ALLOC && what != SVD_INJECT_BAD_CSC)) return SVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->injections[ticket] = what;
    return SVD_OK;
}

svd_status svd_server_stats(svd_server_t s, int64_t* out8) {
    if (!s || !out8) return SVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out8[0] = s->n_submitted;
    out8[1] = s->n_completed;
    out8[2] = s->n_failed;
    out8[3] = s->n_rejected;
    int64_t nrun = 0;
    for (const auto& g : s->running) nrun += (int64_t)g.size();
    out8[4] = nrun;
    out8[5] = (int64_t)s->pending.size();
    out8[6] = (int64_t)s->pool->used();
    out8[7] = (int64_t)s->pool->peak();
    return SVD_OK;
}

void svd_server_destroy(svd_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued requests are dropped; running ones finish first
        for (Request* r : s->pending) {
            r->state = kDone;
            r->result = SVD_ERR_INVALID_ARG;
        }
        s->pending.clear();
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->all) {
        if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
        delete kv.second;
    }
    for (auto& e : s->engines)
        if (e) svd_batch_free(e);
    for (auto& st : s->streams) cudaStreamDestroy(st);
    cudaFree(s->base);
    delete s->pool;
    delete s;
}

}  // extern "C"
