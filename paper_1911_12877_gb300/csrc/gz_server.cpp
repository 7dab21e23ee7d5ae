// gz_server.cpp - continuous-batching request loop (no paper counterpart; the
// paper motivates just-in-time queries, Sec. 1 and Sec. 7.3).
//
// A worker thread owns max_inflight_launches CUDA streams ("slots"). Requests
// fall in two classes by the service time the loop has observed for their
// (plan, graph) pair; a pair not yet seen counts as slow:
//  - fast requests are admitted in arrival order, as many as fit a launch and
//    the scratch budget, and run as one batched launch on a free slot;
//  - slow requests run one at a time, each as one launch. While fast work is
//    waiting or running and no other slow request queues behind it, a slow
//    launch's grids take only the share slow_share of the resident CTAs. Every
//    kernel here is persistent (its CTAs stay until its work queue is empty),
//    so the SM capacity it leaves free is there at once for the fast batches on
//    the other slots: a fast request does not wait for the slow one to end.
//    Otherwise (nothing else to run, or slow requests backed up) it takes the
//    whole device.
// Completions are detected by polling each slot's event, so arrivals are
// admitted while earlier launches run and their work overlaps on the device.
// A whole-device mode (the FIFO baseline of gz_server_replay) runs every
// request as one full launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "gz_internal.h"

namespace gz {
gz_status prepare_query(const gz_plan* p, const gz_graph* g, int use_orientation, int64_t root_lo,
                        int64_t root_hi, cudaStream_t s, Query& q);
}

using namespace gz;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
    int64_t ticket;
    const gz_plan* plan;
    const gz_graph* graph;
    int ori;
    Clock::time_point t_submit, t_done;
    uint64_t count = 0;
    uint64_t scratch = 0;
    gz_status status = GZ_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    unsigned long long* h_counts = nullptr;  // pinned
    int cap = 0;
    std::vector<Req*> batch;
    uint64_t scratch = 0;
    bool busy = false;
    bool slow = false;          // runs one slow request on part of the device
    Clock::time_point t_launch;
};

// Observed service time of a (plan, graph) pair.
struct CostKey {
    const gz_plan* p;
    const gz_graph* g;
    bool operator<(const CostKey& o) const { return p != o.p ? p < o.p : g < o.g; }
};

}  // namespace

struct gz_server {
    gz_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;   // arrived, not yet launched
    std::map<int64_t, Req*> reqs;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    bool whole = false;         // whole-device mode (FIFO baseline)
    int64_t next_ticket = 1;
    uint64_t inflight_scratch = 0;
    int64_t launches = 0;
    int64_t max_queue = 0;
    int device = 0;
    std::map<CostKey, double> cost_ms;  // moving average per (plan, graph)
};

namespace {

const LaunchCfg kCfg = [] {
    LaunchCfg c;
    c.block_warps = 8;
    c.chunk = 4;
    return c;
}();

uint64_t req_scratch(const Req* r) {
    const GzView* v = r->ori ? &r->graph->ori : &r->graph->orig;
    return (uint64_t)resident_warps(kCfg) * scratch_words_per_warp(r->plan->prog, *r->graph, *v) * 4 + 256;
}

// Launches the slot's requests as one batch on the slot's stream and queues the
// read-back of their counts; the lock is released.
gz_status launch_batch(Slot& sl, double grid_frac) {
    GZ_RANGE("gz_server_launch");
    const int nq = (int)sl.batch.size();
    std::vector<Query> qs(nq);
    for (int i = 0; i < nq; ++i) {
        Req* r = sl.batch[i];
        gz_status st = prepare_query(r->plan, r->graph, r->ori, 0, -1, sl.stream, qs[i]);
        if (st != GZ_OK) return st;
    }
    LaunchCfg cfg = kCfg;
    cfg.grid_frac = grid_frac;
    const uint64_t meta = (mixed_meta_bytes(qs.data(), nq) + 255) & ~255ull;
    const uint64_t need = meta + mixed_scratch_bytes(qs.data(), nq, cfg) + 256;
    // counts [nq], status, clique work counters [kCliqueWork nq]
    const size_t words = (size_t)nq + 1 + kCliqueWork * (size_t)nq;
    void* scratch = nullptr;
    unsigned long long* d = nullptr;
    cudaError_t e = gz_malloc_async(&scratch, need, sl.stream);
    if (e == cudaSuccess) e = gz_malloc_async(&d, sizeof(unsigned long long) * words, sl.stream);
    if (e != cudaSuccess) {
        if (scratch) cudaFreeAsync(scratch, sl.stream);
        return cuda_fail(e, "server: scratch");
    }
    e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * words, sl.stream);
    gz_status st = e == cudaSuccess ? GZ_OK : cuda_fail(e, "server: memset");
    if (st == GZ_OK)
        st = launch_mixed(qs.data(), nq, cfg, sl.stream, d, reinterpret_cast<int*>(d + nq), d + nq + 1,
                          reinterpret_cast<char*>(scratch) + meta, need - meta, scratch, meta, false);
    if (st == GZ_OK) {
        e = cudaMemcpyAsync(sl.h_counts, d, sizeof(unsigned long long) * (nq + 1), cudaMemcpyDeviceToHost, sl.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "server: copy back");
    }
    cudaFreeAsync(scratch, sl.stream);
    cudaFreeAsync(d, sl.stream);
    if (st == GZ_OK) {
        e = cudaEventRecord(sl.done_ev, sl.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "server: event");
    }
    return st;
}

void finish(gz_server* s, Req* r, gz_status st, Clock::time_point now) {
    r->status = st;
    r->t_done = now;
    r->done = true;
    s->cv_done.notify_all();
}

void worker_main(gz_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    const double heavy_ms = s->opts.heavy_ms > 0 ? s->opts.heavy_ms : 20.0;
    const double share = s->opts.slow_share > 0 && s->opts.slow_share <= 1 ? s->opts.slow_share : 0.75;
    auto slow = [&](const Req* r) {
        if (s->whole || s->opts.heavy_ms < 0) return false;  // whole device / class-blind
        auto it = s->cost_ms.find(CostKey{r->plan, r->graph});
        return it == s->cost_ms.end() || it->second > heavy_ms;
    };
    while (!s->stop) {
        bool progress = false;
        // 1. completions
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done_ev);
            if (q == cudaErrorNotReady) continue;
            auto now = Clock::now();
            const double ms = std::chrono::duration<double, std::milli>(now - sl.t_launch).count();
            if (q != cudaSuccess) cudaGetLastError();
            const int nq = (int)sl.batch.size();
            const int bad = *reinterpret_cast<int*>(&sl.h_counts[nq]);
            for (int i = 0; i < nq; ++i) {
                sl.batch[i]->count = sl.h_counts[i];
                finish(s, sl.batch[i], q != cudaSuccess ? GZ_ECUDA : (bad ? GZ_EOVERFLOW : GZ_OK), now);
            }
            if (nq == 1 && q == cudaSuccess) {  // service time of the pair, alone in its launch
                double& c = s->cost_ms[CostKey{sl.batch[0]->plan, sl.batch[0]->graph}];
                c = c > 0 ? 0.7 * c + 0.3 * ms : ms;
            }
            s->inflight_scratch -= sl.scratch;
            sl.batch.clear();
            sl.busy = false;
            sl.slow = false;
            progress = true;
        }
        // 2. admission into free slots: fast requests batched in arrival order;
        //    a slow request alone, on part of the device, one at a time
        const uint64_t budget = s->opts.scratch_budget;
        for (Slot& sl : s->slots) {
            if (sl.busy || s->pending.empty()) continue;
            bool slow_busy = false;
            for (const Slot& o : s->slots) slow_busy = slow_busy || (o.busy && o.slow);
            uint64_t used = 0;
            for (auto it = s->pending.begin(); it != s->pending.end() && (int)sl.batch.size() < sl.cap;) {
                Req* r = *it;
                const bool rs = slow(r);
                if (rs && (slow_busy || !sl.batch.empty())) { ++it; continue; }
                const uint64_t need = std::max(used, r->scratch);  // a batch needs its largest query's scratch
                if (s->inflight_scratch + need > budget && (s->inflight_scratch > 0 || !sl.batch.empty())) break;
                used = need;
                sl.batch.push_back(r);
                it = s->pending.erase(it);
                if (rs) {
                    sl.slow = true;
                    break;
                }
            }
            if (sl.batch.empty()) continue;
            // a slow launch leaves room only when fast work needs it now, and
            // not when slow requests queue behind it (then they are the
            // bottleneck and take the whole device)
            double frac = 1.0;
            if (sl.slow) {
                bool fast_work = false, slow_waiting = false;
                for (const Req* r : s->pending) {
                    const bool rs = slow(r);
                    fast_work = fast_work || !rs;
                    slow_waiting = slow_waiting || rs;
                }
                for (const Slot& o : s->slots) fast_work = fast_work || (o.busy && !o.slow);
                if (fast_work && !slow_waiting) frac = share;
            }
            sl.scratch = used;
            s->inflight_scratch += used;
            sl.busy = true;
            sl.t_launch = Clock::now();
            s->launches++;
            lk.unlock();
            gz_status st = launch_batch(sl, frac);
            lk.lock();
            if (st != GZ_OK) {
                auto now = Clock::now();
                for (Req* r : sl.batch) finish(s, r, st, now);
                s->inflight_scratch -= sl.scratch;
                sl.batch.clear();
                sl.busy = false;
                sl.slow = false;
            }
            progress = true;
        }
        if (!progress) {
            bool any_busy = false;
            for (Slot& sl : s->slots) any_busy = any_busy || sl.busy;
            // poll completions every 20 us while launches run; otherwise sleep until a submit
            if (any_busy) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

extern "C" {

gz_status gz_server_create(const gz_server_opts* opts, gz_server** out) {
    if (!out) { set_error("gz_server_create: out is NULL"); return GZ_EINVAL; }
    *out = nullptr;
    gz_server* s = new (std::nothrow) gz_server;
    if (!s) { set_error("gz_server_create: out of host memory"); return GZ_ENOMEM; }
    if (opts) s->opts = *opts;
    if (s->opts.max_inflight_launches <= 0) s->opts.max_inflight_launches = 4;
    if (s->opts.max_batch <= 0) s->opts.max_batch = 64;
    if (s->opts.scratch_budget == 0) s->opts.scratch_budget = 4ull << 30;
    cudaGetDevice(&s->device);
    s->slots.resize(s->opts.max_inflight_launches);
    for (Slot& sl : s->slots) {
        sl.cap = s->opts.max_batch;
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = gz_malloc_host(&sl.h_counts, sizeof(unsigned long long) * (sl.cap + 1));
        if (e != cudaSuccess) {
            gz_status st = cuda_fail(e, "gz_server_create");
            gz_server_destroy(s);
            return st;
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GZ_OK;
}

gz_status gz_server_submit(gz_server* s, const gz_plan* p, const gz_graph* g, int use_orientation,
                           int64_t* ticket) {
    if (!s || !p || !g || !ticket) { set_error("gz_server_submit: NULL argument"); return GZ_EINVAL; }
    if (use_orientation && !g->oriented) { set_error("gz_server_submit: graph not oriented"); return GZ_EINVAL; }
    Req* r = new (std::nothrow) Req;
    if (!r) { set_error("gz_server_submit: out of host memory"); return GZ_ENOMEM; }
    r->plan = p;
    r->graph = g;
    r->ori = use_orientation ? 1 : 0;
    // the out-list view must exist before scratch can be estimated
    {
        gz_graph* gg = const_cast<gz_graph*>(g);
        GzView* v = r->ori ? &gg->ori : &gg->orig;
        if (!v->has_dag || (!p->prog.unit_dag && !v->src)) {
            std::lock_guard<std::mutex> lk(s->mu);
            gz_status st = build_dag(gg, v, 0);
            if (st == GZ_OK && !p->prog.unit_dag) st = build_src(gg, v, 0);
            cudaStreamSynchronize(0);
            if (st != GZ_OK) { delete r; return st; }
        }
    }
    r->scratch = req_scratch(r);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->pending.push_back(r);
        s->max_queue = std::max<int64_t>(s->max_queue, (int64_t)s->pending.size());
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return GZ_OK;
}

gz_status gz_server_wait(gz_server* s, int64_t ticket, int64_t timeout_ms, uint64_t* count,
                         int64_t* latency_ns) {
    if (!s) { set_error("gz_server_wait: server is NULL"); return GZ_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("gz_server_wait: unknown ticket %lld", (long long)ticket); return GZ_EINVAL; }
    Req* r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_error("gz_server_wait: ticket %lld not done", (long long)ticket);
        return GZ_ETIMEOUT;
    }
    gz_status st = r->status;
    if (count) *count = r->count;
    if (latency_ns)
        *latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done - r->t_submit).count();
    s->reqs.erase(it);
    delete r;
    if (st != GZ_OK) set_error("gz_server_wait: request failed with status %d", st);
    return st;
}

gz_status gz_server_replay(gz_server* s, const gz_plan* const* plans, const gz_graph* const* graphs,
                           const int* use_orientation, int64_t nreq, const int64_t* arrival_ns,
                           const int32_t* plan_idx, const int32_t* graph_idx, int fifo,
                           uint64_t* counts, int64_t* latency_ns, double* stats_out) {
    if (!s || nreq < 0 || (nreq > 0 && (!plans || !graphs || !arrival_ns || !plan_idx || !graph_idx ||
                                         !counts || !latency_ns))) {
        set_error("gz_server_replay: bad arguments");
        return GZ_EINVAL;
    }
    int64_t launches0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        launches0 = s->launches;
        s->max_queue = 0;
    }
    std::vector<int64_t> tickets(nreq, 0);
    std::vector<Clock::time_point> arrive(nreq);
    auto t0 = Clock::now();
    gz_status st = GZ_OK;
    if (fifo) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->whole = true;
        }
        // plain baseline: one query per launch, strictly one at a time, in arrival order
        for (int64_t i = 0; i < nreq && st == GZ_OK; ++i) {
            arrive[i] = t0 + std::chrono::nanoseconds(arrival_ns[i]);
            std::this_thread::sleep_until(arrive[i]);
            int64_t t;
            int ori = use_orientation ? use_orientation[i] : 0;
            st = gz_server_submit(s, plans[plan_idx[i]], graphs[graph_idx[i]], ori, &t);
            if (st != GZ_OK) break;
            int64_t lat;
            st = gz_server_wait(s, t, -1, &counts[i], &lat);
            latency_ns[i] = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - arrive[i]).count();
        }
        // requests that arrived while earlier ones were served waited in the queue;
        // latency above is measured from each request's own arrival time
        std::lock_guard<std::mutex> lk(s->mu);
        s->whole = false;
    } else {
        std::thread sub([&] {
            for (int64_t i = 0; i < nreq; ++i) {
                arrive[i] = t0 + std::chrono::nanoseconds(arrival_ns[i]);
                std::this_thread::sleep_until(arrive[i]);
                int ori = use_orientation ? use_orientation[i] : 0;
                gz_server_submit(s, plans[plan_idx[i]], graphs[graph_idx[i]], ori, &tickets[i]);
            }
        });
        sub.join();
        for (int64_t i = 0; i < nreq; ++i) {
            if (tickets[i] == 0) { st = GZ_EINVAL; continue; }
            int64_t lat;
            gz_status r = gz_server_wait(s, tickets[i], -1, &counts[i], &lat);
            latency_ns[i] = lat;  // submission happens at the arrival time
            if (r != GZ_OK && st == GZ_OK) st = r;
        }
    }
    double wall = std::chrono::duration<double>(Clock::now() - t0).count();
    if (stats_out) {
        std::lock_guard<std::mutex> lk(s->mu);  // the worker updates both counters
        stats_out[0] = wall > 0 ? (double)nreq / wall : 0.0;
        stats_out[1] = (double)s->max_queue;
        stats_out[2] = (double)(s->launches - launches0);
        stats_out[3] = wall;
    }
    return st;
}

void gz_server_destroy(gz_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done_ev) cudaEventDestroy(sl.done_ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_counts) cudaFreeHost(sl.h_counts);
    }
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
