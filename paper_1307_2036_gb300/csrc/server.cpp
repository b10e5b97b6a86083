// Continuous-batching request server.
//
// Submitted solves wait in a FIFO queue.  Between refinement steps a worker
// thread admits queued requests while a slot is free and their device
// footprint fits the HBM budget, retires finished ones, and advances every
// admitted request by one refinement step (FP64 residual, FP32 V-cycle, FP64
// update) with one launch per kernel and level over all of them.  A request
// that arrives while others are on the GPU therefore joins at the next step,
// and its own arithmetic is the same as when it is solved alone.  Problems
// (hierarchy vectors) are pooled per grid shape and the grid geometry is shared
// through the library's geometry cache, so repeated shapes stay resident.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ellsolve.h"
#include "solver.hpp"

using namespace ells;

namespace {

using Clock = std::chrono::steady_clock;

struct ShapeKey {
    int kind, n, nz, mapping;
    double side;
    bool operator<(const ShapeKey &o) const {
        return std::tie(kind, n, nz, mapping, side) < std::tie(o.kind, o.n, o.nz, o.mapping, o.side);
    }
};

ShapeKey shape_of(const ellsolve_grid &g) {
    return ShapeKey{g.kind, g.n, g.nz, g.kind == 1 ? g.mapping : 0, g.kind == 0 ? g.box_side : 0.0};
}

struct Request {
    uint64_t ticket = 0;
    ellsolve_grid grid{};
    double omega2 = 0, lambda2 = 0;
    std::vector<double> r;
    size_t footprint = 0;
    enum State { kQueued, kActive, kDone } state = kQueued;
    ellsolve_status status = ELLSOLVE_PENDING;
    ellsolve_result result{};
    Clock::time_point t_submit;
    std::unique_ptr<ellsolve_s> prob;
    MemberRun run;
};

}  // namespace

struct ellsolve_server_s {
    size_t budget = 0;
    int max_slots = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    ellsolve_opts opts{};

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t in_use = 0;

    // worker-only state
    std::vector<Request *> active;
    std::multimap<ShapeKey, std::unique_ptr<ellsolve_s>> pool;
    size_t pool_bytes = 0;
    std::unique_ptr<Plan> plan;
    std::thread worker;

    void run_worker();
    std::unique_ptr<ellsolve_s> acquire(const Request &q);
    void release(std::unique_ptr<ellsolve_s> p);
    void finish(Request *q, ellsolve_status st);
};

std::unique_ptr<ellsolve_s> ellsolve_server_s::acquire(const Request &q) {
    auto it = pool.find(shape_of(q.grid));
    std::unique_ptr<ellsolve_s> p;
    if (it != pool.end()) {
        p = std::move(it->second);
        pool_bytes -= p->footprint_bytes();
        pool.erase(it);
        p->rebind(q.omega2, q.lambda2, q.r.data());
    } else {
        // keep idle pooled problems within what the budget leaves
        while (!pool.empty() && in_use + pool_bytes > budget) {
            auto victim = pool.begin();
            pool_bytes -= victim->second->footprint_bytes();
            pool.erase(victim);
        }
        p = std::make_unique<ellsolve_s>();
        p->build(q.grid, q.omega2, q.lambda2, q.r.data(), opts, stream);
    }
    return p;
}

void ellsolve_server_s::release(std::unique_ptr<ellsolve_s> p) {
    if (!p) return;
    p->plan.reset();
    pool_bytes += p->footprint_bytes();
    ShapeKey k = shape_of(p->grid);
    pool.emplace(k, std::move(p));
}

void ellsolve_server_s::finish(Request *q, ellsolve_status st) {
    // caller holds mu
    q->status = st;
    q->state = Request::kDone;
    q->result.seconds = std::chrono::duration<double>(Clock::now() - q->t_submit).count();
    in_use -= q->footprint;
    cv_done.notify_all();
}

void ellsolve_server_s::run_worker() {
    cudaSetDevice(device);
    bool changed = false;
    std::vector<Request *> joined;
    for (;;) {
        joined.clear();
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait(lock, [&] { return stop || !queue.empty() || !active.empty(); });
            if (stop && queue.empty() && active.empty()) break;
            // admission: FIFO while a slot is free and the footprint fits
            while (!queue.empty() && int(active.size() + joined.size()) < max_slots) {
                Request *q = queue.front();
                if (in_use + q->footprint > budget) break;
                queue.pop_front();
                in_use += q->footprint;
                q->state = Request::kActive;
                joined.push_back(q);
            }
        }
        try {
            for (Request *q : joined) {
                q->prob = acquire(*q);
                active.push_back(q);
                changed = true;
            }
            if (active.empty()) continue;
            if (changed) {
                // the batch changed: one plan over every admitted request, the
                // new ones (at the end) start their refinement
                std::vector<Problem *> mem;
                std::vector<MemberRun *> run;
                for (Request *q : active) {
                    mem.push_back(q->prob.get());
                    run.push_back(&q->run);
                }
                if (!plan) plan = std::make_unique<Plan>();
                plan->build(mem, 1);
                ir_bind(*plan, run);
                const int m0 = int(active.size() - joined.size());
                ir_start(*plan, run, m0, int(active.size()), false);
                changed = false;
            }
            std::vector<MemberRun *> run;
            for (Request *q : active) run.push_back(&q->run);
            bool any = false;
            for (MemberRun *r : run) any = any || r->active;
            if (any) ir_advance(*plan, run, false);
            // retire finished requests (a request that stopped before any update
            // gets its x = 0 written first)
            if (ir_zero_unwritten(*plan, run))
                check_cuda(cudaStreamSynchronize(plan->mem[0]->stream), "retire sync");
            std::vector<Request *> keep;
            std::lock_guard<std::mutex> lock(mu);
            for (Request *q : active) {
                if (q->run.active) {
                    keep.push_back(q);
                    continue;
                }
                const ellsolve_status st = run_result(q->run, 0.0, &q->result);
                release(std::move(q->prob));
                finish(q, st);
                changed = true;
            }
            active.swap(keep);
        } catch (const Error &e) {
            std::lock_guard<std::mutex> lock(mu);
            set_last_error(e.what());
            for (Request *q : active) {
                q->prob.reset();
                finish(q, e.status);
            }
            for (Request *q : joined)
                if (q->state != Request::kDone) {
                    q->prob.reset();
                    finish(q, e.status);
                }
            active.clear();
            plan.reset();
            changed = true;
        }
    }
    plan.reset();
    pool.clear();
}

extern "C" {

ellsolve_status ellsolve_server_create(size_t hbm_budget_bytes, int max_slots, void *stream,
                                       ellsolve_server_t *out) {
    try {
        if (!out || max_slots < 1 || hbm_budget_bytes == 0)
            throw Error(ELLSOLVE_ERR_ARG, "server: need out, max_slots >= 1 and a budget");
        *out = nullptr;
        auto s = std::make_unique<ellsolve_server_s>();
        s->budget = hbm_budget_bytes;
        s->max_slots = max_slots;
        s->stream = static_cast<cudaStream_t>(stream);
        check_cuda(cudaGetDevice(&s->device), "cudaGetDevice");
        ellsolve_default_opts(&s->opts);
        s->opts.precision = 1;
        s->opts.use_graph = 0;
        ellsolve_server_s *raw = s.get();
        s->worker = std::thread([raw] { raw->run_worker(); });
        *out = s.release();
        return ELLSOLVE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return ELLSOLVE_ERR_ARG;
    }
}

ellsolve_status ellsolve_submit(ellsolve_server_t s, const ellsolve_grid *grid, double omega2,
                                double lambda2, const double *r_levels, const void *rhs_dev,
                                void *x_dev, double rtol, int maxit, uint64_t *ticket) {
    try {
        if (!s || !grid || !r_levels || !rhs_dev || !x_dev || !ticket)
            throw Error(ELLSOLVE_ERR_ARG, "submit: null argument");
        if (grid->kind != 0 && grid->kind != 1) throw Error(ELLSOLVE_ERR_ARG, "submit: bad kind");
        if (grid->n < 1 || grid->nz < 1) throw Error(ELLSOLVE_ERR_ARG, "submit: bad size");
        if (!(omega2 > 0) || !(lambda2 > 0)) throw Error(ELLSOLVE_ERR_ARG, "submit: bad omega2/lambda2");
        if (maxit < 1 || !(rtol >= 0)) throw Error(ELLSOLVE_ERR_ARG, "submit: bad rtol/maxit");
        for (int k = 0; k < grid->nz; ++k)
            if (!(r_levels[k + 1] > r_levels[k]))
                throw Error(ELLSOLVE_ERR_ARG, "submit: r_levels not increasing");
        auto q = std::make_unique<Request>();
        q->grid = *grid;
        q->omega2 = omega2;
        q->lambda2 = lambda2;
        q->r.assign(r_levels, r_levels + grid->nz + 1);
        q->run.f = static_cast<const double *>(rhs_dev);
        q->run.x = static_cast<double *>(x_dev);
        q->run.rtol = rtol;
        q->run.maxit = maxit;
        q->footprint = problem_vector_bytes(*grid, s->opts) + geometry_bytes(*grid, s->opts);
        if (q->footprint > s->budget)
            throw Error(ELLSOLVE_ERR_CAPACITY, "submit: request needs " +
                                                   std::to_string(q->footprint) +
                                                   " bytes, more than the server's budget");
        q->t_submit = Clock::now();
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) throw Error(ELLSOLVE_ERR_ARG, "submit: server is shutting down");
        q->ticket = s->next_ticket++;
        *ticket = q->ticket;
        s->queue.push_back(q.get());
        s->reqs.emplace(q->ticket, std::move(q));
        s->cv_work.notify_one();
        return ELLSOLVE_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return ELLSOLVE_ERR_ARG;
    }
}

ellsolve_status ellsolve_poll(ellsolve_server_t s, uint64_t ticket, int timeout_us,
                              ellsolve_result *res) {
    if (!s) {
        set_last_error("poll: null server");
        return ELLSOLVE_ERR_ARG;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_last_error("poll: unknown ticket");
        return ELLSOLVE_ERR_ARG;
    }
    Request *q = it->second.get();
    auto done = [&] { return q->state == Request::kDone; };
    if (!done()) {
        if (timeout_us == 0) return ELLSOLVE_PENDING;
        if (timeout_us < 0) s->cv_done.wait(lock, done);
        else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), done))
            return ELLSOLVE_PENDING;
    }
    if (res) *res = q->result;
    const ellsolve_status st = q->status;
    s->reqs.erase(it);
    return st;
}

void ellsolve_server_destroy(ellsolve_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

}  // extern "C"
