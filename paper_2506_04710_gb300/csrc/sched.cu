// Serving scheduler: continuous batching of array solves with admission by
// device-memory footprint and resident plans (the FFT'd generating blocks, B
// and C stay on the device under a caller-chosen key).
//
// Worker threads each own a CUDA stream.  A request is admitted when a worker
// is free and   bytes reserved by running requests + idle resident plans +
// ztoep_footprint(request) <= budget;   idle plans are evicted least-recently
// used to make room.  Admitted requests run concurrently on their streams, so
// the kernels of different requests overlap on the device; a request that
// arrives while others run starts as soon as a worker and memory free up.
// The queue is FIFO (only its head is considered, so large requests are not
// starved).  Every request runs exactly the ztoep_solve it would run alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    int64_t id = 0;
    ztoep_request_t r{};
    size_t fp = 0;          // reserved bytes while running
    int state = 0;          // 0 queued, 1 running, 2 done
    int status = 0;
    int reused = 0;
    int consumed = 0;        // the plan exists: T, B, C no longer read
    bool holds_ref = false;  // holds a reference on the resident plan of its key
    Clock::time_point t_submit, t_start, t_done;
};

struct CachedPlan {
    ztoep_plan_t plan = nullptr;
    size_t bytes = 0;
    int refs = 0;
    uint64_t last_use = 0;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct ztoep_sched_s {
    ztoep_sched_opts_t o{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
    std::unordered_map<uint64_t, CachedPlan> plans;
    std::vector<std::thread> threads;
    bool stop = false;
    int64_t next_id = 1, submitted = 0, completed = 0, in_flight = 0, max_in_flight = 0;
    size_t bytes_work = 0, peak = 0;
    int64_t built = 0, reused = 0, evicted = 0, groups = 0;
    uint64_t tick = 0;
    int nsm = 152;  // SM count of the device (chunk shapes of the grouped solve)
    // Plans evicted under mu, destroyed by a worker after it releases mu:
    // ztoep_plan_destroy frees device memory, and cudaFree can wait for the
    // whole device, which must not block the other workers' bookkeeping.
    std::vector<ztoep_plan_t> doomed;

    size_t idle_plan_bytes() const {
        size_t s = 0;
        for (const auto &kv : plans)
            if (kv.second.refs == 0) s += kv.second.bytes;
        return s;
    }
    size_t plan_bytes() const {
        size_t s = 0;
        for (const auto &kv : plans) s += kv.second.bytes;
        return s;
    }

    // Under mu: reserve the head request's bytes, evicting idle plans if needed.
    bool try_admit(Req *q) {
        for (;;) {
            const size_t held = bytes_work + idle_plan_bytes();
            if (held + q->fp <= o.hbm_budget) {
                bytes_work += q->fp;
                peak = std::max(peak, bytes_work + idle_plan_bytes());
                return true;
            }
            // evict the least recently used idle plan (never the one this request reuses)
            auto victim = plans.end();
            for (auto it = plans.begin(); it != plans.end(); ++it)
                if (it->second.refs == 0 && it->first != q->r.plan_key &&
                    (victim == plans.end() || it->second.last_use < victim->second.last_use))
                    victim = it;
            if (victim == plans.end()) return false;
            if (!o.fake_backend) doomed.push_back(victim->second.plan);
            plans.erase(victim);
            ++evicted;
        }
    }

    // Plan of a request: the resident one of its key, or a new build from its
    // inputs (device inputs directly, host inputs through stream-ordered
    // staging).  Sets q->consumed once T, B and C are no longer read.
    ztoep_status_t acquire(Req *q, cudaStream_t s, ztoep_plan_t *out, bool *from_cache) {
        ztoep_request_t &r = q->r;
        ztoep_plan_t plan = nullptr;
        *from_cache = false;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (r.plan_key) {
                auto it = plans.find(r.plan_key);
                if (it != plans.end()) {
                    plan = it->second.plan;
                    *from_cache = true;
                    it->second.refs++;  // not evictable while this request uses it
                    q->holds_ref = true;
                    q->consumed = 1;
                }
            }
        }
        ztoep_status_t st = ZTOEP_OK;
        if (!plan) {
            if (r.inputs_on_device) {
                st = ztoep_plan(&r.desc, r.T, r.B, r.C, s, &plan);
                // ztoep_plan is stream-ordered: the blocks are read once the stream passes it
                if (st == ZTOEP_OK) cudaStreamSynchronize(s);
            } else {  // stage the host blocks on the device for the plan build
                const int64_t nt = (int64_t)r.desc.nx * r.desc.ny * r.desc.b, e = r.desc.n_edge;
                const size_t tb = sizeof(double2) * (size_t)(2 * r.desc.ny - 1) * (2 * r.desc.nx - 1) * r.desc.b * r.desc.b;
                const size_t bb = sizeof(double2) * (size_t)e * nt, cb = sizeof(double2) * (size_t)e * e;
                void *dT = nullptr, *dB = nullptr, *dC = nullptr;
                // stream-ordered staging (counted in the request's reserved bytes)
                bool ok = cudaMallocAsync(&dT, tb, s) == cudaSuccess;
                if (ok && e > 0) ok = cudaMallocAsync(&dB, bb, s) == cudaSuccess && cudaMallocAsync(&dC, cb, s) == cudaSuccess;
                if (ok) {
                    cudaMemcpyAsync(dT, r.T, tb, cudaMemcpyHostToDevice, s);
                    if (e > 0) {
                        cudaMemcpyAsync(dB, r.B, bb, cudaMemcpyHostToDevice, s);
                        cudaMemcpyAsync(dC, r.C, cb, cudaMemcpyHostToDevice, s);
                    }
                    st = ztoep_plan(&r.desc, dT, dB, dC, s, &plan);
                } else {
                    cudaGetLastError();
                    st = ZTOEP_ERR_NOMEM;
                }
                if (dT) cudaFreeAsync(dT, s);
                if (dB) cudaFreeAsync(dB, s);
                if (dC) cudaFreeAsync(dC, s);
                cudaStreamSynchronize(s);
            }
            std::lock_guard<std::mutex> lk(mu);
            q->consumed = 1;
        }
        *out = plan;
        return st;
    }

    // After the solve: a new plan joins the resident set under its key (or is
    // destroyed); statistics.
    void release(Req *q, ztoep_plan_t plan, bool from_cache) {
        q->reused = from_cache ? 1 : 0;
        std::lock_guard<std::mutex> lk(mu);
        if (from_cache) {
            ++reused;
        } else if (plan) {
            ++built;
            if (q->r.plan_key && plans.find(q->r.plan_key) == plans.end()) {
                ztoep_plan_info_t pi{};
                ztoep_plan_get_info(plan, &pi);
                CachedPlan cp;
                cp.plan = plan;
                cp.bytes = pi.resident_bytes;
                cp.refs = 1;  // released when the request completes
                plans.emplace(q->r.plan_key, cp);
                q->holds_ref = true;
            } else {
                ztoep_plan_destroy(plan);
            }
        }
    }

    // Host logic only: no device work, plans are bookkeeping entries.
    void run_fake(const std::vector<Req *> &grp) {
        std::this_thread::sleep_for(std::chrono::microseconds(o.fake_us));
        std::lock_guard<std::mutex> lk(mu);
        for (Req *q : grp) {
            ztoep_request_t &r = q->r;
            q->status = ZTOEP_OK;
            q->consumed = 1;
            if (!r.plan_key) continue;
            auto it = plans.find(r.plan_key);
            if (it != plans.end()) {
                ++reused;
                q->reused = 1;
            } else {
                ++built;
                CachedPlan cp;
                cp.bytes = q->fp / 2;
                plans.emplace(r.plan_key, cp);
                it = plans.find(r.plan_key);
            }
            it->second.refs++;
            q->holds_ref = true;
        }
    }

    // One request alone (ztoep_solve / ztoep_solve_host), or several device-
    // input requests as one grouped solve (ztoep_solve_group: one launch per
    // step for all of them, each with exactly its solve-alone arithmetic).
    void run(const std::vector<Req *> &grp, cudaStream_t s) {
        if (o.fake_backend) {
            run_fake(grp);
            return;
        }
        cudaSetDevice(o.device);
        const int n = (int)grp.size();
        std::vector<ztoep_plan_t> pl(n, nullptr);
        std::vector<char> cached(n, 0);
        std::vector<ztoep_status_t> ast(n, ZTOEP_OK);
        for (int i = 0; i < n; ++i) {
            bool fc = false;
            ast[i] = acquire(grp[i], s, &pl[i], &fc);
            cached[i] = fc;
        }
        ztoep_solve_opts_t so = grp[0]->r.opts;
        so.flags |= ZTOEP_FLAG_ZERO_GUESS;
        if (n == 1) {
            ztoep_request_t &r = grp[0]->r;
            ztoep_status_t st = ast[0];
            if (st == ZTOEP_OK) {
                st = r.inputs_on_device ? ztoep_solve(pl[0], &so, r.nrhs, r.V, r.X, r.info, s)
                                        : ztoep_solve_host(pl[0], &so, r.nrhs, r.V, r.X, r.info, s);
                cudaStreamSynchronize(s);
            }
            grp[0]->status = st;
        } else {
            // members whose plan failed are solved by nobody and report that error
            std::vector<ztoep_plan_t> gp;
            std::vector<int32_t> gr;
            std::vector<const void *> gv;
            std::vector<void *> gx;
            std::vector<std::vector<ztoep_solve_info_t>> tmp(n);
            std::vector<ztoep_solve_info_t *> gi;
            std::vector<int> idx;
            for (int i = 0; i < n; ++i) {
                if (ast[i] != ZTOEP_OK) continue;
                ztoep_request_t &r = grp[i]->r;
                tmp[i].assign(r.nrhs, ztoep_solve_info_t{});
                gp.push_back(pl[i]);
                gr.push_back(r.nrhs);
                gv.push_back(r.V);
                gx.push_back(r.X);
                gi.push_back(tmp[i].data());
                idx.push_back(i);
            }
            ztoep_status_t gst = ZTOEP_OK;
            if (!gp.empty()) {
                gst = ztoep_solve_group((int32_t)gp.size(), gp.data(), &so, gr.data(), gv.data(), gx.data(),
                                        gi.data(), s);
                cudaStreamSynchronize(s);
            }
            for (int i = 0; i < n; ++i) grp[i]->status = ast[i];
            for (int k = 0; k < (int)idx.size(); ++k) {
                Req *q = grp[idx[k]];
                ztoep_status_t st = ZTOEP_OK;
                if (gst == ZTOEP_ERR_ARG || gst == ZTOEP_ERR_CUDA || gst == ZTOEP_ERR_NOMEM ||
                    gst == ZTOEP_ERR_UNSUPPORTED) {
                    st = gst;
                } else {
                    for (const ztoep_solve_info_t &in : tmp[idx[k]])
                        if (in.status != ZTOEP_OK && (st == ZTOEP_OK || in.status == ZTOEP_ERR_NONFINITE ||
                                                      in.status == ZTOEP_ERR_TIMEOUT))
                            st = (ztoep_status_t)in.status;
                }
                q->status = st;
                if (q->r.info) std::memcpy(q->r.info, tmp[idx[k]].data(), sizeof(ztoep_solve_info_t) * q->r.nrhs);
            }
        }
        for (int i = 0; i < n; ++i) release(grp[i], pl[i], cached[i] != 0);
    }

    // Can request c join the group grp (in one grouped solve)?  Device
    // inputs, the same options, a plan of its own, the same chunk shape of
    // the solver's kernels, and a size within a factor 4 of the first one's
    // (the group runs until its slowest member converges).
    bool groupable(const std::vector<Req *> &grp, const Req *c) const {
        const ztoep_request_t &a = grp[0]->r, &b = c->r;
        if (!o.fake_backend && (!a.inputs_on_device || !b.inputs_on_device)) return false;
        if (a.opts.tol != b.opts.tol || a.opts.restart != b.opts.restart || a.opts.max_iter != b.opts.max_iter ||
            a.opts.max_outer != b.opts.max_outer || a.opts.prec != b.opts.prec ||
            a.opts.inner_tol != b.opts.inner_tol || a.opts.timeout_ns != b.opts.timeout_ns ||
            a.opts.flags != b.opts.flags)
            return false;
        for (const Req *g : grp)
            if (b.plan_key && g->r.plan_key == b.plan_key) return false;
        auto n_of = [](const ztoep_request_t &r) {
            return (double)r.desc.nx * r.desc.ny * r.desc.b + r.desc.n_edge;
        };
        auto big = [&](const ztoep_request_t &r) { return (n_of(r) + 255) / 256 >= 8.0 * nsm; };
        if (big(a) != big(b)) return false;
        const double ca = n_of(a) * a.nrhs, cb = n_of(b) * b.nrhs;
        return cb <= 4 * ca && ca <= 4 * cb;
    }

    void worker() {
        cudaStream_t s = nullptr;
        if (!o.fake_backend) {
            cudaSetDevice(o.device);
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        }
        const size_t gmax = (size_t)std::max(1, std::min(o.group_max, 8));
        for (;;) {
            std::vector<Req *> grp;
            std::vector<ztoep_plan_t> victims;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return (stop && queue.empty()) || (!queue.empty() && try_admit(queue.front())); });
                if (queue.empty()) {
                    victims.swap(doomed);
                    lk.unlock();
                    for (ztoep_plan_t v : victims) ztoep_plan_destroy(v);
                    break;
                }
                grp.push_back(queue.front());
                queue.pop_front();
                // the next requests in arrival order join while they fit
                while (grp.size() < gmax && !queue.empty() && groupable(grp, queue.front()) &&
                       try_admit(queue.front())) {
                    grp.push_back(queue.front());
                    queue.pop_front();
                }
                victims.swap(doomed);
                for (Req *q : grp) {
                    q->state = 1;
                    q->t_start = Clock::now();
                    ++in_flight;
                }
                max_in_flight = std::max(max_in_flight, in_flight);
                if (grp.size() > 1) ++groups;
            }
            for (ztoep_plan_t v : victims) ztoep_plan_destroy(v);  // outside mu
            run(grp, s);
            {
                std::lock_guard<std::mutex> lk(mu);
                for (Req *q : grp) {
                    bytes_work -= q->fp;
                    if (q->holds_ref) {
                        auto it = plans.find(q->r.plan_key);
                        if (it != plans.end()) {
                            it->second.refs--;
                            it->second.last_use = ++tick;
                        }
                    }
                    --in_flight;
                    ++completed;
                    q->t_done = Clock::now();
                    q->state = 2;
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        if (s) cudaStreamDestroy(s);
    }
};

extern "C" {

ztoep_status_t ztoep_sched_create(const ztoep_sched_opts_t *o, ztoep_sched_t *out) {
    if (!o || !out || o->workers < 1 || o->workers > 64 || o->hbm_budget == 0 || o->fake_us < 0 || o->group_max < 0 ||
        o->group_max > 8)
        return ZTOEP_ERR_ARG;
    *out = nullptr;
    auto *s = new (std::nothrow) ztoep_sched_s();
    if (!s) return ZTOEP_ERR_NOMEM;
    s->o = *o;
    if (!o->fake_backend && cudaSetDevice(o->device) != cudaSuccess) {
        delete s;
        return ZTOEP_ERR_CUDA;
    }
    if (!o->fake_backend) cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, o->device);
    for (int i = 0; i < o->workers; ++i) s->threads.emplace_back([s] { s->worker(); });
    *out = s;
    return ZTOEP_OK;
}

ztoep_status_t ztoep_sched_submit(ztoep_sched_t s, const ztoep_request_t *r, int64_t *id) {
    if (!s || !r || !id || r->nrhs < 1 || !r->T || !r->V || !r->X) return ZTOEP_ERR_ARG;
    if (r->desc.n_edge > 0 && (!r->B || !r->C)) return ZTOEP_ERR_ARG;
    size_t fp = ztoep_footprint(&r->desc, r->nrhs, r->opts.restart > 0 ? r->opts.restart : 30);
    if (fp == 0) return ZTOEP_ERR_ARG;
    if (!r->inputs_on_device) {  // device staging copies of T, B and C for the plan build
        const size_t nt = (size_t)r->desc.nx * r->desc.ny * r->desc.b, e = (size_t)r->desc.n_edge;
        fp += sizeof(double) * 2 *
              ((size_t)(2 * r->desc.ny - 1) * (2 * r->desc.nx - 1) * r->desc.b * r->desc.b + e * nt + e * e);
    }
    if (fp > s->o.hbm_budget) return ZTOEP_ERR_NOMEM;
    auto q = std::make_unique<Req>();
    q->r = *r;
    q->fp = fp;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return ZTOEP_ERR_ARG;
        q->id = s->next_id++;
        *id = q->id;
        s->queue.push_back(q.get());
        s->reqs.emplace(q->id, std::move(q));
        ++s->submitted;
    }
    s->cv_work.notify_one();
    return ZTOEP_OK;
}

static void fill_state(const Req *q, ztoep_request_state_t *st) {
    st->state = q->state;
    st->status = q->state == 2 ? q->status : 0;
    st->plan_reused = q->reused;
    st->inputs_consumed = q->consumed || q->state == 2;
    st->queue_ms = q->state >= 1 ? ms_between(q->t_submit, q->t_start) : 0.0;
    st->latency_ms = q->state == 2 ? ms_between(q->t_submit, q->t_done) : 0.0;
}

ztoep_status_t ztoep_sched_poll(ztoep_sched_t s, int64_t id, ztoep_request_state_t *st) {
    if (!s || !st) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ZTOEP_ERR_ARG;
    fill_state(it->second.get(), st);
    return ZTOEP_OK;
}

ztoep_status_t ztoep_sched_wait(ztoep_sched_t s, int64_t id, int64_t timeout_ms, ztoep_request_state_t *st) {
    if (!s || !st) return ZTOEP_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return ZTOEP_ERR_ARG;
    Req *q = it->second.get();
    auto done = [&] { return q->state == 2; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        fill_state(q, st);
        return ZTOEP_ERR_TIMEOUT;
    }
    fill_state(q, st);
    return ZTOEP_OK;
}

ztoep_status_t ztoep_sched_get_stats(ztoep_sched_t s, ztoep_sched_stats_t *st) {
    if (!s || !st) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->max_in_flight = s->max_in_flight;
    st->bytes_in_use = s->bytes_work + s->idle_plan_bytes();
    st->peak_bytes = s->peak;
    st->resident_plan_bytes = s->plan_bytes();
    st->plans_built = s->built;
    st->plans_reused = s->reused;
    st->plans_evicted = s->evicted;
    st->groups = s->groups;
    return ZTOEP_OK;
}

void ztoep_sched_destroy(ztoep_sched_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) t.join();
    if (!s->o.fake_backend) {
        cudaSetDevice(s->o.device);
        for (auto &kv : s->plans) ztoep_plan_destroy(kv.second.plan);
        for (ztoep_plan_t v : s->doomed) ztoep_plan_destroy(v);
    }
    delete s;
}

}  // extern "C"
