// Serving loop: continuous batching of time-stepping requests.
//
// Requests (a grid, a quadrature shape, an RK scheme, a number of steps and
// a step size) are queued by wke_server_submit from any thread.  One worker
// thread owns every CUDA call.  It admits the oldest pending request as soon
// as a slot is free and the request's device footprint fits the budget
// (plans of the same shape left by finished requests are reused, and idle
// plans are evicted least recently used first to make room), copies the
// initial data through pinned staging, enqueues all steps on the request's
// own stream, and records a completion event.  Work of different requests
// therefore overlaps on the device; a request admitted while others run
// starts immediately.  Completion is detected by polling the events.
#include <cuda_runtime.h>

#include <algorithm>
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
    int status = 1;                 // 1 pending, 2 active, 0 done, < 0 error
    double t_submit = 0, t_admit = 0, t_done = 0;
    PlanInst *inst = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool cancelled = false;
};

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
    void free_inst(PlanInst *p) {
        if (p->plan) wke_plan_destroy(p->plan);
        if (p->f_dev) cudaFree(p->f_dev);
        if (p->pin_in) cudaFreeHost(p->pin_in);
        if (p->pin_out) cudaFreeHost(p->pin_out);
        used -= p->dev_bytes;
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

    // Returns an idle instance for the key, a new one, nullptr when it must
    // wait for memory, or sets *err when the request can never fit.
    PlanInst *acquire(const wke_request &r, int *err) {
        PlanKey key{r.d, r.N, r.n_r, r.n_s, r.n_sig, r.precision, r.rk_stages, r.L};
        for (auto &p : pool)
            if (!p->busy && p->key == key) return p.get();
        wke_quadrature q;
        wke_quadrature_default(&q);
        q.n_r = r.n_r;
        q.n_s = r.n_s;
        q.n_sig = r.n_sig;
        q.precision = r.precision;
        size_t fp = 0;
        int rc = wke_plan_footprint_bytes(r.d, r.N, r.L, r.n_r * r.n_s * r.n_sig, &q, &fp);
        if (rc) {
            *err = rc;
            return nullptr;
        }
        const size_t need = fp + grid_bytes_of(r);
        if (need > budget) {
            *err = fail(WKE_ERR_OOM, "request needs " + std::to_string(need) + " device bytes, budget is " +
                                         std::to_string(budget));
            return nullptr;
        }
        while (used + need > budget && evict_one_idle()) {
        }
        if (used + need > budget) return nullptr;   // wait for active requests
        auto inst = std::make_unique<PlanInst>();
        inst->key = key;
        inst->grid_bytes = grid_bytes_of(r);
        rc = wke_plan_create(r.d, r.N, r.L, r.n_r * r.n_s * r.n_sig, &q, &inst->plan);
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

    void launch(Req *q) {
        PlanInst *p = q->inst;
        const wke_request &r = q->r;
        if (free_streams.empty()) {
            cudaStream_t s;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            free_streams.push_back(s);
        }
        q->stream = free_streams.back();
        free_streams.pop_back();
        cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming);
        std::memcpy(p->pin_in, r.f_host, p->grid_bytes);
        int rc = (int)cudaMemcpyAsync(p->f_dev, p->pin_in, p->grid_bytes, cudaMemcpyHostToDevice, q->stream);
        if (!rc) rc = wke_plan_set_stream(p->plan, q->stream);
        for (int s = 0; s < r.steps && !rc; ++s) rc = wke_step(p->plan, p->f_dev, r.dt, r.rk_stages);
        if (!rc) rc = (int)cudaMemcpyAsync(p->pin_out, p->f_dev, p->grid_bytes, cudaMemcpyDeviceToHost, q->stream);
        if (!rc) rc = (int)cudaEventRecord(q->done, q->stream);
        q->status = rc ? (rc > 0 ? WKE_ERR_CUDA : rc) : 2;
    }

    void finish(Req *q, int status) {
        q->t_done = now();
        if (status == 0 && q->inst) std::memcpy(q->r.out_host, q->inst->pin_out, q->inst->grid_bytes);
        q->status = status;
        if (q->inst) {
            q->inst->busy = false;
            q->inst->last_used = ++tick;
        }
        if (q->stream) free_streams.push_back(q->stream);
        if (q->done) cudaEventDestroy(q->done);
        q->stream = nullptr;
        q->done = nullptr;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progress = false;
            // admissions, oldest first
            while (!pending.empty() && (int)active.size() < max_active) {
                Req *q = pending.front();
                if (q->cancelled) {
                    pending.pop_front();
                    q->t_done = now();
                    q->status = WKE_CANCELLED;
                    progress = true;
                    continue;
                }
                int err = 0;
                PlanInst *p = acquire(q->r, &err);
                if (!p && err) {                         // can never run
                    pending.pop_front();
                    q->t_done = now();
                    q->status = err;
                    progress = true;
                    continue;
                }
                if (!p) break;                           // wait for memory
                pending.pop_front();
                p->busy = true;
                q->inst = p;
                q->t_admit = now();
                launch(q);
                if (q->status != 2) finish(q, q->status);
                else active.push_back(q);
                progress = true;
            }
            // completions
            for (size_t i = 0; i < active.size();) {
                Req *q = active[i];
                cudaError_t e = cudaEventQuery(q->done);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                finish(q, e == cudaSuccess ? 0 : WKE_ERR_CUDA);
                active.erase(active.begin() + i);
                progress = true;
            }
            if (progress) cv_done.notify_all();
            if (stop && pending.empty() && active.empty()) break;
            if (!progress) {
                if (active.empty() && pending.empty()) cv_work.wait(lk, [&] { return stop || !pending.empty(); });
                else cv_work.wait_for(lk, std::chrono::microseconds(50));
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
