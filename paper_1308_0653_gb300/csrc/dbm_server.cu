// Serving runtime: continuous batching of simulations over one batch.
//
// A scheduler thread owns a CUDA stream for the batched steps and a second
// stream for per-request I/O (initial-state upload, moments download).  Each
// round it
//   1. admits queued requests while a slot and pool memory are free (carve a
//      block from the pool, create the simulation, upload and initialise its
//      state on the I/O stream, attach it), overlapping the quantum in flight;
//   2. waits for the quantum in flight, then detaches every simulation that
//      has finished or was cancelled, so the next quantum's tables omit it;
//   3. enqueues the next quantum of batched steps on the compute stream
//      (after the I/O stream's uploads);
//   4. retires the detached simulations while that quantum runs (no launch
//      touches their buffers): moments and totals to host memory, destroy,
//      free the pool block.
// Requests that arrive while others run join at the next quantum boundary,
// and the steps of all resident simulations share each launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dbm.h"

namespace {

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over [0, size) with 256-byte granularity.
struct Pool {
    std::map<size_t, size_t> free_;  // offset -> size
    size_t total = 0;
    void init(size_t off, size_t size)
    {
        free_.clear();
        total = size;
        if (size) free_[off] = size;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t roff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = align256(bytes);
        auto it = free_.emplace(off, bytes).first;
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
    size_t largest() const
    {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
};

enum ReqState { QUEUED, RUNNING, DONE };

struct Request {
    uint64_t ticket;
    dbm_params p;
    int64_t nsteps;
    std::vector<double> init;    // 5 * N doubles, copied at submit
    ReqState state = QUEUED;
    bool cancel = false;
    int slot = -1;
    size_t off = 0, bytes = 0;
    dbm_t *h = nullptr;
    int64_t end_step = 0;        // batch step at which its last step is done
    bool leaving = false;        // detached, waiting to be retired
    dbm_result res;
    int bypassed = 0;            // times a later request was admitted ahead of it
};

}  // namespace

struct dbm_server_s {
    dbm_server_config cfg;
    unsigned char *pool_base;
    size_t pool_bytes;
    Pool pool;
    dbm_batch_t *batch = nullptr;
    int device = 0;
    cudaStream_t compute = nullptr, io = nullptr;
    std::vector<Request *> slots;
    std::deque<Request *> queue;
    std::map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread th;
    std::chrono::steady_clock::time_point t0;
    dbm_server_stats stats;
    int fatal = DBM_OK;          // first error of a batched step; ends the server's work
    int64_t fail_quantum = -1;   // fault injection: this quantum fails with DBM_ECUDA
};

namespace {

void finish(dbm_server_t *S, Request *r, int status)
{
    // caller holds S->mu
    r->res.status = status;
    r->res.t_end = now_s(S->t0);
    r->state = DONE;
    if (status == DBM_OK) {
        S->stats.completed += 1;
        S->stats.updates += (double)r->p.nr * r->p.ntheta * DBM_NV * (double)r->nsteps;
    } else if (status == DBM_ECANCELLED) {
        S->stats.cancelled += 1;
    } else {
        S->stats.failed += 1;
    }
    S->cv_done.notify_all();
}

double *alloc_fields(size_t N)
{
    return static_cast<double *>(std::malloc(sizeof(double) * 5 * N));
}

// Retire a request whose slot was already detached and whose buffers no
// launch touches any more: moments to host (status DBM_OK), or no result
// (DBM_ECANCELLED, or the server's fatal error), destroy, free its pool
// block.  Scheduler thread, lock not held.
void retire(dbm_server_t *S, Request *r, int status)
{
    if (status == DBM_OK) {
        const size_t N = (size_t)r->p.nr * r->p.ntheta;
        double *host = alloc_fields(N);
        if (!host) {
            status = DBM_ENOMEM;
        } else {
            status = dbm_moments(r->h, host, host + N, host + 2 * N, host + 3 * N, host + 4 * N,
                                 r->res.totals, S->io);
            if (status == DBM_OK || status == DBM_ENONFINITE) {
                r->res.rho = host;
                r->res.ur = host + N;
                r->res.uth = host + 2 * N;
                r->res.T = host + 3 * N;
                r->res.lam = host + 4 * N;
            } else {
                std::free(host);
            }
        }
    }
    r->res.steps = dbm_steps_done(r->h);
    dbm_destroy(r->h);
    r->h = nullptr;
    std::lock_guard<std::mutex> lock(S->mu);
    S->pool.release(r->off, r->bytes);
    S->slots[r->slot] = nullptr;
    S->stats.running -= 1;
    finish(S, r, status);
}

// Admit one request into a slot and pool block (scheduler thread, lock not
// held): create the simulation, upload and initialise its state on the I/O
// stream, attach it to the batch from the batch's current step on.
void admit(dbm_server_t *S, Request *r, int slot, size_t off, size_t bytes)
{
    r->slot = slot;
    r->off = off;
    r->bytes = bytes;
    int rc = dbm_create(&r->p, S->pool_base + off, bytes, &r->h);
    if (rc == DBM_OK) {
        const size_t N = (size_t)r->p.nr * r->p.ntheta;
        const double *f = r->init.data();
        rc = dbm_init_state(r->h, f, f + N, f + 2 * N, f + 3 * N, f + 4 * N, S->io);
    }
    if (rc == DBM_OK) {
        r->end_step = dbm_batch_time(S->batch) + r->nsteps;
        rc = dbm_batch_attach(S->batch, slot, r->h, r->nsteps);
    }
    if (rc != DBM_OK) {
        if (r->h) dbm_destroy(r->h);
        r->h = nullptr;
        std::lock_guard<std::mutex> lock(S->mu);
        S->pool.release(off, bytes);
        S->slots[slot] = nullptr;
        S->stats.running -= 1;
        finish(S, r, rc);
        return;
    }
    std::vector<double>().swap(r->init);  // the copy is on the device now
}

// The scheduler keeps up to two quanta in flight on the compute stream: it
// enqueues quantum n, then waits for quantum n-1 while n runs, so the host
// work between quanta (admission, table updates, retirement) overlaps the
// GPU.  Which attached simulations advance in a step is decided on the device
// from the batch step counter, so a simulation that ends inside a quantum
// needs no table change to stop; it is detached once found finished and
// retired (moments, destroy, free) as soon as no launch in flight can touch
// its buffers: at once if it ended before the running quantum starts, else
// once that quantum is done.  A cancelled simulation is active in the running
// quantum and waits for it the same way.  If a batched step fails (a CUDA
// error, a device self-check), the scheduler enqueues nothing more, waits for
// the quanta in flight and ends every queued and resident request with that
// error; later submissions are refused with it.
void scheduler(dbm_server_t *S)
{
    cudaSetDevice(S->device);
    cudaEvent_t qdone[2], io_done;
    cudaEventCreateWithFlags(&qdone[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&qdone[1], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&io_done, cudaEventDisableTiming);
    bool pend[2] = {false, false};
    int64_t pend_seq[2] = {0, 0}, pend_start[2] = {0, 0};
    int64_t qseq = 0;      // quanta enqueued so far
    int64_t done_q = -1;   // every quantum up to this one is complete
    struct Deferred {
        Request *r;
        int status;        // DBM_OK, DBM_ECANCELLED or the fatal error
        int64_t wait_q;    // retire once this quantum is complete
    };
    std::vector<Deferred> deferred;
    auto wait_slot = [&](int k) {
        if (!pend[k]) return;
        cudaEventSynchronize(qdone[k]);
        pend[k] = false;
        done_q = std::max(done_q, pend_seq[k]);
    };
    for (;;) {
        // ---- 1. admission (overlaps the quanta in flight) ---------------------
        std::vector<std::pair<Request *, int>> to_admit;
        std::vector<std::pair<size_t, size_t>> blocks;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            for (;;) {
                const bool any_running = S->stats.running > 0;
                if (S->stop && S->queue.empty() && !any_running) {
                    lock.unlock();
                    wait_slot(0);
                    wait_slot(1);
                    cudaEventDestroy(qdone[0]);
                    cudaEventDestroy(qdone[1]);
                    cudaEventDestroy(io_done);
                    return;
                }
                if (!S->queue.empty() || any_running) break;
                S->cv_work.wait_for(lock, std::chrono::milliseconds(50));
            }
            for (auto it = S->queue.begin(); it != S->queue.end();) {  // cancelled while queued
                if ((*it)->cancel || S->fatal != DBM_OK) {
                    S->stats.queued -= 1;
                    finish(S, *it, (*it)->cancel ? DBM_ECANCELLED : S->fatal);
                    it = S->queue.erase(it);
                } else {
                    ++it;
                }
            }
            // first fit in arrival order; a request passed over max_bypass
            // times blocks the later ones until it is admitted
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                Request *r = *it;
                int slot = -1;
                for (int k = 0; k < S->cfg.max_slots; ++k)
                    if (!S->slots[k]) {
                        slot = k;
                        break;
                    }
                if (slot < 0) break;
                const size_t bytes = dbm_state_bytes(&r->p);
                size_t off = 0;
                if (S->pool.alloc(bytes, &off)) {
                    S->slots[slot] = r;
                    r->state = RUNNING;
                    r->res.t_start = now_s(S->t0);
                    S->stats.running += 1;
                    S->stats.queued -= 1;
                    to_admit.push_back({r, slot});
                    blocks.push_back({off, bytes});
                    it = S->queue.erase(it);
                } else {
                    if (r->bypassed >= S->cfg.max_bypass) break;
                    r->bypassed += 1;
                    ++it;
                }
            }
        }
        for (size_t k = 0; k < to_admit.size(); ++k)
            admit(S, to_admit[k].first, to_admit[k].second, blocks[k].first, blocks[k].second);
        if (!to_admit.empty()) {
            // the next quantum must see the uploaded initial states
            cudaEventRecord(io_done, S->io);
            cudaStreamWaitEvent(S->compute, io_done, 0);
        }

        // ---- 2. enqueue quantum n if anything is active ------------------------
        // A quantum ends no later than the first active simulation does: the
        // work items are balanced over the CTAs for the active set, and one
        // that finishes early would leave its CTAs idle for the rest.
        const int64_t t_now = dbm_batch_time(S->batch);
        bool any_active = false;
        int64_t steps = S->cfg.quantum;
        int fatal = DBM_OK;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            fatal = S->fatal;
            for (int k = 0; k < S->cfg.max_slots && fatal == DBM_OK; ++k) {
                Request *r = S->slots[k];
                if (!r || !r->h || r->state != RUNNING || r->leaving || r->cancel) continue;
                const int64_t left = dbm_batch_remaining(S->batch, k);
                if (left > 0) {
                    any_active = true;
                    steps = std::min(steps, left);
                }
            }
        }
        double work = 0.0;  // site-velocity updates this quantum will execute
        if (any_active) {
            std::lock_guard<std::mutex> lock(S->mu);
            for (int k = 0; k < S->cfg.max_slots; ++k) {
                Request *r = S->slots[k];
                if (!r || !r->h || r->state != RUNNING || r->leaving || r->cancel) continue;
                if (dbm_batch_remaining(S->batch, k) > 0)
                    work += (double)r->p.nr * r->p.ntheta * DBM_NV * (double)steps;
            }
        }
        bool enqueued = false;
        if (any_active) {
            const int k = (int)(qseq & 1);
            wait_slot(k);  // quantum n-2: at most two in flight
            const int rc = S->fail_quantum == qseq ? DBM_ECUDA  // host-side fault injection
                                                   : dbm_batch_step(S->batch, steps, S->compute);
            std::lock_guard<std::mutex> lock(S->mu);
            if (rc == DBM_OK) {
                cudaEventRecord(qdone[k], S->compute);
                pend[k] = true;
                pend_seq[k] = qseq;
                pend_start[k] = t_now;
                ++qseq;
                enqueued = true;
                S->stats.executed += work;
                S->stats.batch_time = (double)dbm_batch_time(S->batch);  // read under the lock by stats
            } else {
                S->fatal = fatal = rc;
            }
        }

        // ---- 3. wait for quantum n-1 (or the last one, if none was enqueued) ---
        for (int k = 0; k < 2; ++k)
            if (pend[k] && (!enqueued || pend_seq[k] < qseq - 1)) wait_slot(k);
        int64_t running_q = -1, running_from = INT64_MAX;  // the quantum still in flight
        for (int k = 0; k < 2; ++k)
            if (pend[k]) {
                running_q = pend_seq[k];
                running_from = pend_start[k];
            }

        // ---- 4. retire what no launch in flight touches ------------------------
        std::vector<std::pair<Request *, int>> now;
        {
            std::vector<Deferred> keep;
            for (const Deferred &d : deferred) {
                if (d.wait_q <= done_q)
                    now.push_back({d.r, d.status});  // its steps ran before any failure
                else
                    keep.push_back(d);
            }
            deferred.swap(keep);
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            for (int k = 0; k < S->cfg.max_slots; ++k) {
                Request *r = S->slots[k];
                if (!r || !r->h || r->state != RUNNING || r->leaving) continue;
                const bool finished = dbm_batch_remaining(S->batch, k) == 0;
                if (!r->cancel && !finished && fatal == DBM_OK) continue;
                const int status = r->cancel ? DBM_ECANCELLED : finished ? DBM_OK : fatal;
                r->leaving = true;
                dbm_batch_detach(S->batch, k);  // out of the next quantum's tables
                if (running_q < 0 || (!r->cancel && r->end_step <= running_from))
                    now.push_back({r, status});
                else
                    deferred.push_back({r, status, running_q});
            }
        }
        for (auto &lr : now) retire(S, lr.first, lr.second);
    }
}

}  // namespace

extern "C" {

size_t dbm_server_min_bytes(const dbm_server_config *cfg)
{
    if (!cfg) return 0;
    return dbm_batch_bytes(cfg->max_slots, cfg->max_items, cfg->precision) + 256;
}

int dbm_server_create(const dbm_server_config *cfg, void *dev_pool, size_t pool_bytes,
                      dbm_server_t **out)
{
    if (!cfg || !dev_pool || !out || cfg->max_slots < 1 || cfg->max_queue < 1 || cfg->quantum < 1 ||
        cfg->max_items < 1 || cfg->max_bypass < 0 ||
        (cfg->precision != DBM_FP32 && cfg->precision != DBM_FP64))
        return DBM_EINVAL;
    *out = nullptr;
    if (((uintptr_t)dev_pool & 255) != 0) return DBM_EINVAL;
    const size_t bb = dbm_batch_bytes(cfg->max_slots, cfg->max_items, cfg->precision);
    if (pool_bytes < bb + 256) return DBM_ENOMEM;
    dbm_server_t *S = new (std::nothrow) dbm_server_t();
    if (!S) return DBM_ENOMEM;
    S->cfg = *cfg;
    S->pool_base = static_cast<unsigned char *>(dev_pool);
    S->pool_bytes = pool_bytes;
    std::memset(&S->stats, 0, sizeof(S->stats));
    S->slots.assign(cfg->max_slots, nullptr);
    S->t0 = std::chrono::steady_clock::now();
    // Host-side fault injection for tests of the failure path: quantum n
    // (counted from 0) reports DBM_ECUDA instead of launching.
    if (const char *env = std::getenv("DBM_SERVER_FAIL_QUANTUM")) S->fail_quantum = std::atoll(env);
    int rc = DBM_OK;
    if (cudaGetDevice(&S->device) != cudaSuccess) rc = DBM_ECUDA;
    if (rc == DBM_OK && cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking) != cudaSuccess)
        rc = DBM_ECUDA;
    if (rc == DBM_OK && cudaStreamCreateWithFlags(&S->io, cudaStreamNonBlocking) != cudaSuccess)
        rc = DBM_ECUDA;
    if (rc == DBM_OK)
        rc = dbm_batch_create(cfg->max_slots, cfg->max_items, cfg->precision, cfg->rows_per_item,
                              dev_pool, bb, &S->batch);
    if (rc != DBM_OK) {
        if (S->compute) cudaStreamDestroy(S->compute);
        if (S->io) cudaStreamDestroy(S->io);
        delete S;
        return rc;
    }
    S->pool.init(align256(bb), pool_bytes - align256(bb));
    S->th = std::thread(scheduler, S);
    *out = S;
    return DBM_OK;
}

int dbm_submit(dbm_server_t *S, const dbm_params *p, const dbm_fields *init, int64_t nsteps,
               uint64_t *ticket)
{
    if (!S || !p || !init || !ticket || nsteps < 0) return DBM_EINVAL;
    if (!init->rho || !init->ur || !init->uth || !init->T || !init->lam) return DBM_EINVAL;
    if (p->precision != S->cfg.precision) return DBM_EINVAL;
    int rc = dbm_check(p, nullptr);
    if (rc != DBM_OK) return rc;
    const size_t bytes = dbm_state_bytes(p);
    if (align256(bytes) > S->pool.total) return DBM_ENOMEM;  // can never fit
    Request *r = new (std::nothrow) Request();
    if (!r) return DBM_ENOMEM;
    const size_t N = (size_t)p->nr * p->ntheta;
    try {
        r->init.resize(5 * N);
    } catch (...) {
        delete r;
        return DBM_ENOMEM;
    }
    const double *src[5] = {init->rho, init->ur, init->uth, init->T, init->lam};
    for (int c = 0; c < 5; ++c) std::memcpy(r->init.data() + c * N, src[c], N * sizeof(double));
    r->p = *p;
    r->nsteps = nsteps;
    std::memset(&r->res, 0, sizeof(r->res));
    r->res.nr = p->nr;
    r->res.ntheta = p->ntheta;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) {
            delete r;
            return DBM_EINVAL;
        }
        if (S->fatal != DBM_OK) {
            delete r;
            return S->fatal;
        }
        if ((int64_t)S->queue.size() >= S->cfg.max_queue) {
            delete r;
            return DBM_EBUSY;
        }
        r->ticket = S->next_ticket++;
        r->res.t_submit = now_s(S->t0);
        S->queue.push_back(r);
        S->reqs[r->ticket] = r;
        S->stats.submitted += 1;
        S->stats.queued += 1;
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();
    return DBM_OK;
}

int dbm_poll(dbm_server_t *S, uint64_t ticket, dbm_result *out, int64_t timeout_us)
{
    if (!S || !out) return DBM_EINVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return DBM_ENOTFOUND;
    Request *r = it->second;
    if (r->state != DONE) {
        if (timeout_us == 0) return DBM_ENOTREADY;
        auto pred = [&] { return r->state == DONE; };
        if (timeout_us < 0)
            S->cv_done.wait(lock, pred);
        else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred))
            return DBM_ETIMEOUT;
    }
    *out = r->res;
    S->reqs.erase(it);
    delete r;
    return DBM_OK;
}

int dbm_result_free(dbm_result *res)
{
    if (!res) return DBM_EINVAL;
    std::free(res->rho);  // one block holds all five fields
    res->rho = res->ur = res->uth = res->T = res->lam = nullptr;
    return DBM_OK;
}

int dbm_cancel(dbm_server_t *S, uint64_t ticket)
{
    if (!S) return DBM_EINVAL;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return DBM_ENOTFOUND;
        if (it->second->state == DONE) return DBM_OK;
        it->second->cancel = true;
    }
    S->cv_work.notify_all();
    return DBM_OK;
}

int dbm_server_stats_get(dbm_server_t *S, dbm_server_stats *out)
{
    if (!S || !out) return DBM_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    *out = S->stats;
    out->pool_free_largest = (double)S->pool.largest();
    out->status = S->fatal;  // batch_time: kept in S->stats by the scheduler thread
    return DBM_OK;
}

int dbm_server_destroy(dbm_server_t *S)
{
    if (!S) return DBM_EINVAL;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        for (auto &kv : S->reqs)
            if (kv.second->state != DONE) kv.second->cancel = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaStreamSynchronize(S->compute);
    cudaStreamSynchronize(S->io);
    for (auto &kv : S->reqs) {
        dbm_result_free(&kv.second->res);
        delete kv.second;
    }
    dbm_batch_destroy(S->batch);
    cudaStreamDestroy(S->compute);
    cudaStreamDestroy(S->io);
    delete S;
    return DBM_OK;
}

}  // extern "C"
