// Serving loop: continuous batching of time-stepping requests.
//
// Requests (a grid, a quadrature shape, an RK scheme, a number of steps and
// a step size) are queued by wke_server_submit from any thread.  One worker
// thread owns every CUDA call.  It admits requests in arrival order as soon
// as a slot is free and the request's device footprint fits the budget
// (plans of the same shape left by finished requests are reused, and idle
// plans are evicted least recently used first to make room); a request that
// has to wait for memory may be overtaken by at most kMaxBypass later
// requests that fit, after which nothing is admitted until it fits.  An
// admitted request's initial data is copied through pinned staging, all of
// its steps are enqueued on its own stream and a completion event is
// recorded, so work of different requests overlaps on the device; a request
// admitted while others run starts immediately.  Completion is detected by
// polling the events.  The server mutex guards only the request records
// (queue, status, times): plan creation, allocation, copies and launches
// run without it, so submit, cancel and wait never wait behind them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wke_internal.h"
#include "wke_nvtx.h"

using wke::fail;

namespace {

struct PlanKey {
    int d, N, n_r, n_s, n_sig, precision, rk_stages;
    double L;
    bool operator==(const PlanKey &o) const {
        return d == o.d && N == o.N && n_r == o.n_r && n_s == o.n_s && n_sig == o.n_sig &&
               precision == o.precision && L == o.L;
    }
};

struct PlanInst {
    PlanKey key;
    wke_plan *plan = nullptr;
    void *f_dev = nullptr;
    void *pin_in = nullptr, *pin_out = nullptr;
    size_t grid_bytes = 0, dev_bytes = 0;
    bool busy = false;
    unsigned long long last_used = 0;
};

struct Req {
    long long id = 0;
    wke_request r{};
    int status = 1;                 // 1 pending, 2 active, 0 done, < 0 error (guarded by the mutex)
    double t_submit = 0, t_admit = 0, t_done = 0;
    PlanInst *inst = nullptr;       // worker only
    cudaStream_t stream = nullptr;  // worker only
    cudaEvent_t done = nullptr;     // worker only
    bool cancelled = false;         // guarded by the mutex
    int bypassed = 0;               // worker only: later requests admitted while this one waited
    size_t need = 0;                // worker only: device bytes of a new plan instance (0: unknown)
};

// A request waiting for memory is overtaken by at most this many later requests.
constexpr int kMaxBypass = 8;

size_t grid_bytes_of(const wke_request &r) {
    size_t nd = 1;
    for (int a = 0; a < r.d; ++a) nd *= (size_t)r.N;
    return nd * (r.precision == WKE_FP64 ? 8 : 4);
}

}  // namespace

struct wke_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::vector<Req *> active;
    std::unordered_map<long long, std::unique_ptr<Req>> reqs;
    std::vector<std::unique_ptr<PlanInst>> pool;
    std::vector<cudaStream_t> free_streams;
    size_t budget = 0, used = 0;
    int max_active = 1;
    int device = 0;
    bool stop = false;
    long long next_id = 1;
    unsigned long long tick = 0;
    std::chrono::steady_clock::time_point t0;
    std::thread worker;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // ------------------------------------------------------------ worker side
    // pool, used, free_streams, active and the worker-only request fields are
    // touched by the worker thread alone; request status and times are
    // written under the mutex.
    void free_inst(PlanInst *p) {
        if (p->plan) wke_plan_destroy(p->plan);
        if (p->f_dev) cudaFree(p->f_dev);
        if (p->pin_in) cudaFreeHost(p->pin_in);
        if (p->pin_out) cudaFreeHost(p->pin_out);
        used -= p->dev_bytes;
    }

    void drop_inst(PlanInst *p) {
        for (size_t i = 0; i < pool.size(); ++i)
            if (pool[i].get() == p) {
                free_inst(p);
                pool.erase(pool.begin() + i);
                return;
            }
    }

    bool evict_one_idle() {
        int victim = -1;
        for (int i = 0; i < (int)pool.size(); ++i)
            if (!pool[i]->busy && (victim < 0 || pool[i]->last_used < pool[victim]->last_used)) victim = i;
        if (victim < 0) return false;
        free_inst(pool[victim].get());
        pool.erase(pool.begin() + victim);
        return true;
    }

    static PlanKey key_of(const wke_request &r) {
        return PlanKey{r.d, r.N, r.n_r, r.n_s, r.n_sig, r.precision, r.rk_stages, r.L};
    }
    static wke_quadrature quad_of(const wke_request &r) {
        wke_quadrature q;
        wke_quadrature_default(&q);
        q.n_r = r.n_r;
        q.n_s = r.n_s;
        q.n_sig = r.n_sig;
        q.precision = r.precision;
        return q;
    }
    PlanInst *idle_instance(const PlanKey &k) {
        for (auto &p : pool)
            if (!p->busy && p->key == k) return p.get();
        return nullptr;
    }
    size_t idle_bytes() const {
        size_t b = 0;
        for (const auto &p : pool)
            if (!p->busy) b += p->dev_bytes;
        return b;
    }

    // Whether q can be admitted now (an idle instance of its shape, or room
    // for a new one once idle instances are evicted); *err is set when it can
    // never run (invalid shape, or larger than the whole budget).
    bool fits(Req *q, int *err) {
        if (idle_instance(key_of(q->r))) return true;
        if (!q->need) {
            const wke_quadrature qd = quad_of(q->r);
            size_t fp = 0;
            int rc = wke_plan_footprint_bytes(q->r.d, q->r.N, q->r.L, q->r.n_r * q->r.n_s * q->r.n_sig, &qd, &fp);
            if (rc) {
                *err = rc;
                return false;
            }
            q->need = fp + grid_bytes_of(q->r);
            if (q->need > budget) {
                *err = fail(WKE_ERR_OOM, "request needs " + std::to_string(q->need) + " device bytes, budget is " +
                                             std::to_string(budget));
                return false;
            }
        }
        return used - idle_bytes() + q->need <= budget;
    }

    // The instance for an admitted request (fits() was true): an idle one of
    // its shape, or a new one after evicting idle instances.
    PlanInst *instance_for(Req *q, int *err) {
        const wke_request &r = q->r;
        if (PlanInst *p = idle_instance(key_of(r))) return p;
        while (used + q->need > budget && evict_one_idle()) {
        }
        auto inst = std::make_unique<PlanInst>();
        inst->key = key_of(r);
        inst->grid_bytes = grid_bytes_of(r);
        const wke_quadrature qd = quad_of(r);
        int rc = wke_plan_create(r.d, r.N, r.L, r.n_r * r.n_s * r.n_sig, &qd, &inst->plan);
        if (rc == WKE_OK && cudaMalloc(&inst->f_dev, inst->grid_bytes) != cudaSuccess) rc = WKE_ERR_OOM;
        if (rc == WKE_OK && cudaMallocHost(&inst->pin_in, inst->grid_bytes) != cudaSuccess) rc = WKE_ERR_OOM;
        if (rc == WKE_OK && cudaMallocHost(&inst->pin_out, inst->grid_bytes) != cudaSuccess) rc = WKE_ERR_OOM;
        if (rc) {
            cudaGetLastError();
            inst->dev_bytes = 0;
            free_inst(inst.get());
            *err = rc == WKE_ERR_OOM ? fail(WKE_ERR_OOM, "device allocation for a request failed") : rc;
            return nullptr;
        }
        wke_plan_info info;
        wke_plan_get_info(inst->plan, &info);
        inst->dev_bytes = info.device_bytes + inst->grid_bytes;
        used += inst->dev_bytes;
        pool.push_back(std::move(inst));
        return pool.back().get();
    }

    // Copies and all steps of q on its own stream; returns WKE_OK or an error
    // code, in which case the stream has been drained.
    int launch(Req *q) {
        PlanInst *p = q->inst;
        const wke_request &r = q->r;
        if (free_streams.empty()) {
            cudaStream_t s;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return fail(WKE_ERR_CUDA, "stream creation failed");
            }
            free_streams.push_back(s);
        }
        q->stream = free_streams.back();
        free_streams.pop_back();
        int rc = (int)cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming);
        if (!rc) {
            std::memcpy(p->pin_in, r.f_host, p->grid_bytes);
            rc = (int)cudaMemcpyAsync(p->f_dev, p->pin_in, p->grid_bytes, cudaMemcpyHostToDevice, q->stream);
        }
        if (!rc) rc = wke_plan_set_stream(p->plan, q->stream);
        for (int s = 0; s < r.steps && !rc; ++s) rc = wke_step(p->plan, p->f_dev, r.dt, r.rk_stages);
        if (!rc) rc = (int)cudaMemcpyAsync(p->pin_out, p->f_dev, p->grid_bytes, cudaMemcpyDeviceToHost, q->stream);
        if (!rc) rc = (int)cudaEventRecord(q->done, q->stream);
        if (rc) {
            // work already queued on the stream must end before its buffers are reused
            cudaStreamSynchronize(q->stream);
            cudaGetLastError();
            return rc > 0 ? WKE_ERR_CUDA : rc;
        }
        return WKE_OK;
    }

    // Publish q's final status (and its result, status 0); release its
    // stream and instance.  An instance whose launch failed is destroyed,
    // since its plan may hold a partial evaluation.
    void finish(Req *q, int status) {
        if (status == 0 && q->inst) std::memcpy(q->r.out_host, q->inst->pin_out, q->inst->grid_bytes);
        if (q->inst) {
            if (status == 0) {
                q->inst->busy = false;
                q->inst->last_used = ++tick;
            } else {
                drop_inst(q->inst);
            }
            q->inst = nullptr;
        }
        if (q->stream) free_streams.push_back(q->stream);
        if (q->done) cudaEventDestroy(q->done);
        q->stream = nullptr;
        q->done = nullptr;
        std::lock_guard<std::mutex> lk(mu);
        q->t_done = now();
        q->status = status;
    }

    void run() {
        cudaSetDevice(device);
        std::deque<Req *> queue;       // arrival order, not yet admitted
        while (true) {
            bool progress = false;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (queue.empty() && active.empty() && pending.empty()) {
                    if (stop) break;
                    cv_work.wait(lk, [&] { return stop || !pending.empty(); });
                }
                while (!pending.empty()) {
                    queue.push_back(pending.front());
                    pending.pop_front();
                }
                for (auto it = queue.begin(); it != queue.end();) {
                    if ((*it)->cancelled) {
                        (*it)->t_done = now();
                        (*it)->status = WKE_CANCELLED;
                        it = queue.erase(it);
                        progress = true;
                    } else {
                        ++it;
                    }
                }
            }
            if (progress) cv_done.notify_all();
            // admissions in arrival order; a request waiting for memory is
            // overtaken by at most kMaxBypass later ones
            for (size_t i = 0; i < queue.size() && (int)active.size() < max_active;) {
                Req *q = queue[i];
                int err = 0;
                const bool ok = fits(q, &err);
                if (err) {                                  // can never run
                    queue.erase(queue.begin() + i);
                    finish(q, err);
                    progress = true;
                    continue;
                }
                if (!ok) {
                    if (q->bypassed >= kMaxBypass) break;   // nothing more goes past it
                    ++i;
                    continue;
                }
                {
                    std::lock_guard<std::mutex> lk(mu);
                    if (q->cancelled) {
                        q->t_done = now();
                        q->status = WKE_CANCELLED;
                    } else {
                        q->status = 2;
                        q->t_admit = now();
                    }
                }
                queue.erase(queue.begin() + i);
                progress = true;
                if (q->status == WKE_CANCELLED) continue;
                wke::NvtxRange nvtx_range("wke_server admission");
                for (size_t k = 0; k < i; ++k) ++queue[k]->bypassed;
                q->inst = instance_for(q, &err);
                if (!q->inst) {
                    finish(q, err ? err : WKE_ERR_OOM);
                    continue;
                }
                q->inst->busy = true;
                const int rc = launch(q);
                if (rc) finish(q, rc);
                else active.push_back(q);
            }
            // completions
            for (size_t i = 0; i < active.size();) {
                Req *q = active[i];
                cudaError_t e = cudaEventQuery(q->done);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                active.erase(active.begin() + i);
                finish(q, e == cudaSuccess ? 0 : WKE_ERR_CUDA);
                progress = true;
            }
            if (progress) {
                cv_done.notify_all();
            } else {
                std::unique_lock<std::mutex> lk(mu);
                if (pending.empty()) cv_work.wait_for(lk, std::chrono::microseconds(50));
            }
        }
        for (cudaStream_t s : free_streams) cudaStreamDestroy(s);
        free_streams.clear();
        for (auto &p : pool) free_inst(p.get());
        pool.clear();
    }
};

extern "C" {

int wke_server_create(size_t device_budget_bytes, int max_active, wke_server **out) {
    if (!out || max_active < 1 || device_budget_bytes == 0)
        return fail(WKE_ERR_INVALID, "need an output pointer, max_active >= 1 and a nonzero budget");
    *out = nullptr;
    auto *s = new (std::nothrow) wke_server();
    if (!s) return fail(WKE_ERR_OOM, "host allocation failed");
    s->budget = device_budget_bytes;
    s->max_active = max_active;
    cudaGetDevice(&s->device);
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return WKE_OK;
}

int wke_server_submit(wke_server *s, const wke_request *r, long long *id) {
    if (!s || !r || !id) return fail(WKE_ERR_INVALID, "server, request and id must be non-NULL");
    if (!r->f_host || !r->out_host) return fail(WKE_ERR_INVALID, "request needs f_host and out_host");
    if (r->steps < 0 || !(r->dt == r->dt) || (r->rk_stages != 1 && r->rk_stages != 2 && r->rk_stages != 4))
        return fail(WKE_ERR_INVALID, "steps >= 0, finite dt and rk_stages in {1, 2, 4} are required");
    auto q = std::make_unique<Req>();
    q->r = *r;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(WKE_ERR_INVALID, "server is shutting down");
    q->id = s->next_id++;
    q->t_submit = s->now();
    *id = q->id;
    s->pending.push_back(q.get());
    s->reqs[q->id] = std::move(q);
    s->cv_work.notify_one();
    return WKE_OK;
}

int wke_server_cancel(wke_server *s, long long id) {
    if (!s) return fail(WKE_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(WKE_ERR_INVALID, "unknown request id");
    if (it->second->status != 1) return fail(WKE_ERR_INVALID, "request is no longer pending");
    it->second->cancelled = true;
    s->cv_work.notify_one();
    return WKE_OK;
}

int wke_server_wait(wke_server *s, long long id, double timeout_s, wke_request_stats *st) {
    if (!s || !st) return fail(WKE_ERR_INVALID, "server and stats must be non-NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(WKE_ERR_INVALID, "unknown request id");
    Req *q = it->second.get();
    auto pred = [&] { return q->status <= 0; };
    if (timeout_s < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return fail(WKE_ERR_INVALID, "timed out waiting for the request");
    st->id = q->id;
    st->status = q->status;
    st->t_submit = q->t_submit;
    st->t_admit = q->t_admit;
    st->t_done = q->t_done;
    return WKE_OK;
}

int wke_server_destroy(wke_server *s) {
    if (!s) return WKE_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return WKE_OK;
}

}  // extern "C"
