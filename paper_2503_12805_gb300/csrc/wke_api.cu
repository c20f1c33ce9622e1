// C ABI of the library (declared in include/wke.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include "wke_check.cuh"
#include "wke_internal.h"
#include "wke_nvtx.h"

namespace wke {
const char *last_error();

template <typename T> int forward_T(const HostPlan &, const DevicePtrs &, cudaStream_t);
template <typename T> int pass1_T(const HostPlan &, const DevicePtrs &, int, cudaStream_t);
template <typename T> int nyquist_T(const HostPlan &, const DevicePtrs &, int, cudaStream_t);
template <typename T> int pass2_T(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);
template <typename T> int finalize_T(const HostPlan &, const DevicePtrs &, void *, void *, cudaStream_t);
template <typename T> int spectrum_T(const HostPlan &, const DevicePtrs &, const void *, void *, cudaStream_t);
template <typename T> int moments_T(const HostPlan &, const void *, double *, double *, cudaStream_t);
template <typename T>
int rk_stage_T(const HostPlan &, const void *, const void *, double *, void *, double, double, int, cudaStream_t);
template <typename T> int rk_final_T(const HostPlan &, void *, const double *, double, cudaStream_t);
template <typename T> int dealias_prepare_T(const HostPlan &, const DevicePtrs &, cudaStream_t);
template <typename T> int axis0_T(const HostPlan &, const DevicePtrs &, int, cudaStream_t);
template <typename T> int products_T(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);
template <typename T> int sep_planes_T(const HostPlan &, const DevicePtrs &, int, cudaStream_t);
template <typename T> int fused_T(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);
template <typename T> int dealias_finish_T(const HostPlan &, const DevicePtrs &, void *, void *, cudaStream_t);

int moments_partials_count(const HostPlan &) { return 256; }

static int cuda_fail(cudaError_t e, const char *what) {
    return fail(WKE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The bounds-check word of each device (checked builds write it; see
// wke_check.cuh).  Allocated and zeroed on first use.
static std::mutex g_check_mutex;
static unsigned *g_check_word[64] = {nullptr};

unsigned *check_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_check_mutex);
    if (!g_check_word[dev]) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned)) != cudaSuccess || cudaMemset(p, 0, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            if (p) cudaFree(p);
            return nullptr;
        }
        g_check_word[dev] = static_cast<unsigned *>(p);
    }
    return g_check_word[dev];
}
}  // namespace wke

using namespace wke;

// An instantiated graph of one evaluation for a given (f, Q, Qim).
struct GraphEntry {
    const void *f;
    void *Q;
    void *Qim;
    cudaGraphExec_t exec;
    unsigned long long used;
};

// An instantiated graph of one Runge-Kutta step for a given (f, dt, stages).
struct StepGraph {
    void *f;
    double dt;
    int stages;
    cudaGraphExec_t exec;
    unsigned long long used;
};

struct wke_plan {
    HostPlan hp;
    DevicePtrs dp{};
    void *Hbuf[2] = {nullptr, nullptr};   // double-buffered chunk intermediates
    void *Vbuf[2] = {nullptr, nullptr};   // double-buffered chunk Nyquist tables
    void *Sbuf[2] = {nullptr, nullptr};   // double-buffered pair planes (separable plans)
    // pass 1 of chunk c+1 runs on s1 while pass 2 of chunk c runs on s2; the
    // Nyquist tables of each chunk are built on s3
    cudaStream_t s1 = nullptr, s2 = nullptr, s3 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fwd = nullptr;
    cudaEvent_t ev_p1[2] = {nullptr, nullptr}, ev_p2[2] = {nullptr, nullptr}, ev_nq[2] = {nullptr, nullptr};
    bool use_graphs = true;
    std::vector<GraphEntry> graphs;
    std::vector<StepGraph> step_graphs;
    unsigned long long tick = 0;
    std::vector<void *> allocs;
    void *f_stage = nullptr, *Q_stage = nullptr;   // wke_collision_host buffers
    void *rk_y = nullptr, *rk_k = nullptr;
    double *rk_acc = nullptr;
    double *mom_partials = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t bytes = 0;
    bool dirty = false;   // accumulators may hold a partial sum after a failure
    // kernel timing (wke_plan_profile): recorded (class, start, stop) events
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_class;       // class of each recorded interval
};

namespace {

size_t grid_elems(const HostPlan &hp) { return hp.d == 2 ? (size_t)hp.N * hp.N : (size_t)hp.N * hp.N * hp.N; }
// points of the caller's grids (f, Q): N_in^d
size_t grid_in_elems(const HostPlan &hp) {
    return hp.d == 2 ? (size_t)hp.N_in * hp.N_in : (size_t)hp.N_in * hp.N_in * hp.N_in;
}

int dev_alloc(wke_plan *p, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? WKE_ERR_OOM : WKE_ERR_CUDA,
                    std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                        cudaGetErrorString(e));
    }
    p->allocs.push_back(*ptr);
    p->bytes += bytes;
    return WKE_OK;
}

// Free the unit buffers (a fused separable plan runs without them).  The
// caller ensures no queued work uses them.
void release_unit_buffers(wke_plan *p) {
    for (void *&h : p->Hbuf) {
        if (!h) continue;
        for (size_t i = 0; i < p->allocs.size(); ++i)
            if (p->allocs[i] == h) {
                p->allocs.erase(p->allocs.begin() + i);
                break;
            }
        cudaFree(h);
        p->bytes -= chunk_unit_bytes(p->hp);
        h = nullptr;
    }
}

void free_graphs(wke_plan *p) {
    for (GraphEntry &g : p->graphs) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
    for (StepGraph &g : p->step_graphs) cudaGraphExecDestroy(g.exec);
    p->step_graphs.clear();
}

void free_plan(wke_plan *p) {
    free_graphs(p);
    for (cudaEvent_t e : {p->ev_fork, p->ev_join, p->ev_fwd, p->ev_p1[0], p->ev_p1[1], p->ev_p2[0], p->ev_p2[1],
                          p->ev_nq[0], p->ev_nq[1]})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {p->s1, p->s2, p->s3})
        if (st) cudaStreamDestroy(st);
    p->s1 = p->s2 = p->s3 = nullptr;
    for (void *ptr : p->allocs) cudaFree(ptr);
    p->allocs.clear();
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    p->ev_pool.clear();
    p->ev_used = 0;
    p->ev_class.clear();
}

// Record one event of a timed interval (profiling only); returns false when
// an event could not be created, in which case timing is silently skipped.
bool prof_event(wke_plan *p, cudaStream_t s) {
    if (p->ev_used == p->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        p->ev_pool.push_back(e);
    }
    cudaEventRecord(p->ev_pool[p->ev_used++], s);
    return true;
}

struct ProfScope {
    wke_plan *p;
    cudaStream_t s;
    bool on;
    ProfScope(wke_plan *p_, cudaStream_t s_, int cls) : p(p_), s(s_), on(p_->profiling) {
        if (on) {
            on = prof_event(p, s);
            if (on) p->ev_class.push_back(cls);
        }
    }
    ~ProfScope() {
        if (on && !prof_event(p, s)) {
            // keep the pool consistent: drop the unmatched start
            --p->ev_used;
            p->ev_class.pop_back();
        }
    }
};

template <typename T> int upload_tables(wke_plan *p) {
    const HostPlan &hp = p->hp;
    typedef typename std::conditional<sizeof(T) == 4, float2, double2>::type C;
    const int nf = hp.n_fields_total;
    std::vector<C> phase((size_t)nf * hp.d * hp.N);
    std::vector<double> row(2 * hp.N);
    for (int f = 0; f < nf; ++f)
        for (int a = 0; a < hp.d; ++a) {
            phase_row(hp.N, hp.L, hp.field_shift[(size_t)f * hp.d + a], row.data());
            for (int k = 0; k < hp.N; ++k) {
                C c;
                c.x = (T)row[2 * k];
                c.y = (T)row[2 * k + 1];
                phase[((size_t)f * hp.d + a) * hp.N + k] = c;
            }
        }
    std::vector<C> tw(hp.N);
    std::vector<double2> tw64(hp.N_in);
    const double two_pi = 6.28318530717958647692528676655900577;
    for (int k = 0; k < hp.N; ++k) {
        const double th = two_pi * k / hp.N;
        tw[k].x = (T)std::cos(th);
        tw[k].y = (T)std::sin(th);
    }
    for (int k = 0; k < hp.N_in; ++k) {
        const double th = two_pi * k / hp.N_in;
        tw64[k] = make_double2(std::cos(th), std::sin(th));
    }
    std::vector<int> pl(2 * hp.prod_fa.size());
    for (size_t i = 0; i < hp.prod_fa.size(); ++i) {
        pl[2 * i] = hp.prod_fa[i];
        pl[2 * i + 1] = hp.prod_fb[i];
    }
    cudaError_t e;
    if ((e = cudaMemcpy(const_cast<void *>(p->dp.phase), phase.data(), phase.size() * sizeof(C),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "phase table upload");
    if ((e = cudaMemcpy(const_cast<void *>(p->dp.tw), tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "twiddle upload");
    if ((e = cudaMemcpy(const_cast<double *>(p->dp.tw64), tw64.data(), tw64.size() * sizeof(double2),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "twiddle upload");
    if ((e = cudaMemcpy(const_cast<int *>(p->dp.prod_local), pl.data(), pl.size() * sizeof(int),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "product table upload");
    if ((e = cudaMemcpy(const_cast<double *>(p->dp.prod_W), hp.prod_W.data(), hp.prod_W.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "weight upload");
    if (hp.separable && hp.can_fuse) {
        // each unit's axis-0 phase rows (fields a, b), interleaved per j1
        std::vector<float> ue((size_t)total_units(hp) * hp.N * 4, 0.0f);
        std::vector<double> ra(2 * hp.N), rb(2 * hp.N);
        for (int c = 0; c < hp.n_chunks; ++c) {
            const int f0 = hp.chunk_f0[c], K = hp.chunk_f0[c + 1] - f0;
            for (int u = 0; u < (K + 1) / 2; ++u) {
                const int fa = f0 + 2 * u;
                phase_row(hp.N, hp.L, hp.field_shift[(size_t)fa * hp.d], ra.data());
                const bool pair = 2 * u + 1 < K;
                if (pair) phase_row(hp.N, hp.L, hp.field_shift[(size_t)(fa + 1) * hp.d], rb.data());
                float *row = &ue[(size_t)(hp.chunk_u0[c] + u) * hp.N * 4];
                for (int j = 0; j < hp.N; ++j) {
                    row[4 * j] = (float)ra[2 * j];
                    row[4 * j + 1] = (float)ra[2 * j + 1];
                    row[4 * j + 2] = pair ? (float)rb[2 * j] : 0.0f;
                    row[4 * j + 3] = pair ? (float)rb[2 * j + 1] : 0.0f;
                }
            }
        }
        if ((e = cudaMemcpy(const_cast<void *>(p->dp.unit_e0), ue.data(), ue.size() * sizeof(float),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "unit phase upload");
    }
    if (hp.separable) {
        const std::pair<const std::vector<int> *, const int *> tabs[3] = {
            {&hp.sep_v, p->dp.sep_v}, {&hp.sep_p, p->dp.sep_p}, {&hp.field_pair, p->dp.field_pair}};
        for (const auto &tb : tabs)
            if ((e = cudaMemcpy(const_cast<int *>(tb.second), tb.first->data(), tb.first->size() * sizeof(int),
                                cudaMemcpyHostToDevice)) != cudaSuccess)
                return cuda_fail(e, "separable table upload");
    }
    if (hp.shared) {
        std::vector<int> gc(hp.group_cfield);
        if ((e = cudaMemcpy(const_cast<int *>(p->dp.group_cfield), gc.data(), gc.size() * sizeof(int),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "group table upload");
    }
    if (hp.dealias) {
        // Per-axis maps between the N_in grid k_i = -L + i 2L/N_in and the 2N
        // grid k'_i = -L + i 2L/N of the same domain, through the modes
        // j in [-N_in/2, N_in/2-1] of Eq. (3.1):
        //   interpolation (N x N_in): f_N(k'_a) = sum_b Kint[a][b] f(k_b), with
        //     Kint[a][b] = (1/N_in) sum_j exp(i pi j (k'_a - k_b) / L) over the
        //     modes without j = -N_in/2 (the plan zeroes them);
        //   projection (N_in x N): Q(k_a) = sum_b Kproj[a][b] Q2(k'_b), with
        //     Kproj[a][b] = (1/N) sum_j exp(i pi j (k_a - k'_b) / L) over all
        //     of [-N_in/2, N_in/2-1] (Q keeps its -N_in/2 modes).
        const int n = hp.N, m = hp.N_in;
        const double pi = 3.14159265358979323846264338327950288;
        std::vector<double2> Ki((size_t)n * m), Kp((size_t)m * n);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < m; ++b) {
                const double dk = (-hp.L + a * 2.0 * hp.L / n) - (-hp.L + b * 2.0 * hp.L / m);
                double re = 0.0, im = 0.0, rp = 0.0, ip = 0.0;
                for (int j = -m / 2; j < m / 2; ++j) {
                    const double c = std::cos(pi * j * dk / hp.L), sn = std::sin(pi * j * dk / hp.L);
                    if (j != -m / 2) {
                        re += c;
                        im += sn;
                    }
                    rp += c;      // projection term of (k_b - k'_a) = -dk: conjugate phase
                    ip -= sn;
                }
                Ki[(size_t)a * m + b] = make_double2(re / m, im / m);
                Kp[(size_t)b * n + a] = make_double2(rp / n, ip / n);
            }
        if ((e = cudaMemcpy(const_cast<void *>(p->dp.Kint), Ki.data(), Ki.size() * sizeof(double2),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "interpolation map upload");
        if ((e = cudaMemcpy(const_cast<void *>(p->dp.Kproj), Kp.data(), Kp.size() * sizeof(double2),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "projection map upload");
    }
    return WKE_OK;
}

int clear_accumulators(wke_plan *p, cudaStream_t s) {
    const size_t acc = (size_t)n_accumulators(p->hp) * grid_elems(p->hp) * sizeof(double);
    cudaError_t e = cudaMemsetAsync(p->dp.Qacc, 0, acc, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->dp.Qacc_im, 0, acc, s);
    if (e != cudaSuccess) return cuda_fail(e, "accumulator reset");
    p->dirty = false;
    return WKE_OK;
}

// Enqueue one evaluation: fork from `origin` to the plan's two streams, the
// forward transform and pass 1 of each chunk on s1, pass 2 of each chunk on
// s2 (chunk c uses intermediate buffer c % 2), finalize on s2, join back.
template <typename T> int enqueue_T(wke_plan *p, const void *f, void *Q, void *Qim, cudaStream_t origin) {
    HostPlan &hp = p->hp;
    DevicePtrs dp = p->dp;
    dp.f = f;
    dp.H = p->Hbuf[0];
    dp.S = p->Sbuf[0];
    // while profiling, both passes share one stream so that each launch's
    // interval measures that kernel alone
    cudaStream_t s1 = p->s1, s2 = p->profiling ? p->s1 : p->s2, s3 = p->profiling ? p->s1 : p->s3;
    const bool nyq = hp.nyquist == WKE_NYQ_KEEP;
    int e = (int)cudaEventRecord(p->ev_fork, origin);
    if (!e) e = (int)cudaStreamWaitEvent(s1, p->ev_fork, 0);
    if (!e) e = (int)cudaStreamWaitEvent(s2, p->ev_fork, 0);
    if (!e) {
        ProfScope ps(p, s1, 0);
        e = forward_T<T>(hp, dp, s1);
        if (!e && hp.dealias) e = dealias_prepare_T<T>(hp, dp, s1);   // coefficients and f on the 2N grid
    }
    if (hp.dealias) dp.f = dp.ffine;     // the products take F = f_N on the 2N grid
    // s3 joins only when it has work (a forked stream must be joined back)
    if (nyq && !e) e = (int)cudaEventRecord(p->ev_fwd, s1);
    if (nyq && !e) e = (int)cudaStreamWaitEvent(s3, p->ev_fwd, 0);
    const bool im = Qim != nullptr && !hp.dealias;
    for (int c = 0; c < hp.n_chunks && !e; ++c) {
        const int buf = c & 1;
        dp.H = p->Hbuf[buf];
        dp.V = p->Vbuf[buf];
        dp.S = p->Sbuf[buf];
        if (nyq) {
            // tables of chunk c on s3, once pass 2 of chunk c-2 has read the buffer
            if (c >= 2 && !e) e = (int)cudaStreamWaitEvent(s3, p->ev_p2[buf], 0);
            if (!e) {
                ProfScope ps(p, s3, 4);
                e = nyquist_T<T>(hp, dp, c, s3);
            }
            if (!e) e = (int)cudaEventRecord(p->ev_nq[buf], s3);
        }
        if (c >= 2 && !e) e = (int)cudaStreamWaitEvent(s1, p->ev_p2[buf], 0);
        if (!e) {
            ProfScope ps(p, s1, 1);
            e = hp.separable ? sep_planes_T<T>(hp, dp, c, s1) : pass1_T<T>(hp, dp, c, s1);
        }
        if (hp.shared && !hp.fused && !e) {   // shared-field layout: axis 0 into H, then the product pass
            ProfScope ps(p, s1, 5);
            e = axis0_T<T>(hp, dp, c, s1);
        }
        if (!e) e = (int)cudaEventRecord(p->ev_p1[buf], s1);
        if (!e) e = (int)cudaStreamWaitEvent(s2, p->ev_p1[buf], 0);
        if (!e && nyq) e = (int)cudaStreamWaitEvent(s2, p->ev_nq[buf], 0);
        // a fused plan (not de-aliased) writes Q in its last chunk's product kernel
        const bool write_q = hp.fused && !hp.dealias && c == hp.n_chunks - 1;
        dp.Qout = write_q ? Q : nullptr;
        dp.Qiout = write_q ? Qim : nullptr;
        dp.scale_out = hp.scale;
        if (!e) {
            ProfScope ps(p, s2, 2);
            e = hp.fused ? fused_T<T>(hp, dp, c, im, s2)
                : hp.shared ? products_T<T>(hp, dp, c, im, s2) : pass2_T<T>(hp, dp, c, im, s2);
        }
        if (!e) e = (int)cudaEventRecord(p->ev_p2[buf], s2);
    }
    if (!e && !(hp.fused && !hp.dealias)) {
        ProfScope ps(p, s2, 3);
        e = hp.dealias ? dealias_finish_T<T>(hp, dp, Q, Qim, s2) : finalize_T<T>(hp, dp, Q, Qim, s2);
    }
    if (!e) e = (int)cudaEventRecord(p->ev_join, s2);
    if (!e) e = (int)cudaStreamWaitEvent(origin, p->ev_join, 0);
    return e;
}

int enqueue(wke_plan *p, const void *f, void *Q, void *Qim, cudaStream_t origin) {
    return p->hp.precision == WKE_FP32 ? enqueue_T<float>(p, f, Q, Qim, origin)
                                       : enqueue_T<double>(p, f, Q, Qim, origin);
}

// The instantiated graph for (f, Q, Qim), captured on first use.  At most 8
// are kept per plan (least recently used evicted).
int graph_for(wke_plan *p, const void *f, void *Q, void *Qim, cudaGraphExec_t *out) {
    for (GraphEntry &g : p->graphs)
        if (g.f == f && g.Q == Q && g.Qim == Qim) {
            g.used = ++p->tick;
            *out = g.exec;
            return WKE_OK;
        }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(p->s1, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph capture start");
    int e = enqueue(p, f, Q, Qim, p->s1);
    ce = cudaStreamEndCapture(p->s1, &graph);
    if (e || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return cuda_fail(e ? (cudaError_t)e : ce, "graph capture");
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiation");
    if (p->graphs.size() >= 8) {
        size_t lru = 0;
        for (size_t i = 1; i < p->graphs.size(); ++i)
            if (p->graphs[i].used < p->graphs[lru].used) lru = i;
        cudaGraphExecDestroy(p->graphs[lru].exec);
        p->graphs.erase(p->graphs.begin() + lru);
    }
    p->graphs.push_back({f, Q, Qim, exec, ++p->tick});
    *out = exec;
    return WKE_OK;
}

int collision(wke_plan *p, const void *f, void *Q, void *Qim, cudaStream_t s) {
    int rc;
    if (p->dirty && (rc = clear_accumulators(p, s))) return rc;
    int e;
    if (p->use_graphs && !p->profiling) {
        cudaGraphExec_t exec;
        if ((rc = graph_for(p, f, Q, Qim, &exec))) {
            p->dirty = true;
            return rc;
        }
        e = (int)cudaGraphLaunch(exec, s);
    } else {
        e = enqueue(p, f, Q, Qim, s);
    }
    if (e) {
        p->dirty = true;
        return cuda_fail((cudaError_t)e, "collision launch");
    }
    return WKE_OK;
}

}  // namespace

extern "C" {

int wke_quadrature_default(wke_quadrature *q) {
    if (!q) return fail(WKE_ERR_INVALID, "quadrature descriptor is NULL");
    std::memset(q, 0, sizeof(*q));
    q->sphere_rule = -1;
    q->sphere_rule_sig = -1;
    q->R = 0.0;
    q->precision = WKE_FP64;
    q->nyquist = WKE_NYQ_KEEP;
    q->dispersion = WKE_OMEGA_HALF_K2;
    q->pair_antipodal = 1;
    q->chunk_bytes = 0;
    return WKE_OK;
}

int wke_plan_footprint_bytes(int d, int N, double L, int M, const wke_quadrature *quad, size_t *bytes) {
    if (!bytes) return fail(WKE_ERR_INVALID, "bytes is NULL");
    HostPlan hp;
    int rc = build_host_plan(d, N, L, M, quad, hp);
    if (rc) return rc;
    *bytes = plan_device_bytes(hp);
    return WKE_OK;
}

int wke_plan_create(int d, int N, double L, int M, const wke_quadrature *quad, wke_plan **out) {
    NvtxRange nvtx_range("wke_plan_create");
    if (!out) return fail(WKE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    wke_plan *p = new (std::nothrow) wke_plan();
    if (!p) return fail(WKE_ERR_OOM, "host allocation failed");
    int rc = build_host_plan(d, N, L, M, quad, p->hp);
    if (rc) {
        delete p;
        return rc;
    }
    cudaGetDevice(&p->device);
    {
        // checked builds: every kernel unit's check word, before any capture
        const int brc = check_bind_kernels_f32() | check_bind_kernels_f64() | check_bind_fused64_f32() |
                        check_bind_fused_f32();
        if (brc) {
            cudaGetLastError();
            delete p;
            return fail(WKE_ERR_CUDA, "binding the bounds-check word failed");
        }
    }
    const HostPlan &hp = p->hp;
    const size_t nd = grid_elems(hp);
    const size_t tb = hp.precision == WKE_FP64 ? 8 : 4, cxb = 2 * tb;
    const size_t nf = (size_t)hp.n_fields_total;
    void *ptr;
#define ALLOC(field, bytes)                                  \
    do {                                                     \
        if ((rc = dev_alloc(p, &ptr, (bytes)))) goto error;  \
        field = static_cast<decltype(field)>(ptr);           \
    } while (0)
    ALLOC(p->dp.ghat, nd * cxb);
    ALLOC(p->dp.nslice, (size_t)hp.d * (nd / hp.N) * cxb);
    if (needs_unit_buffers(hp)) {
        ALLOC(p->Hbuf[0], chunk_unit_bytes(hp));
        ALLOC(p->Hbuf[1], chunk_unit_bytes(hp));
    }
    if (hp.separable) {                   // S[0] also serves as the forward scratch (N^d complex double)
        ALLOC(p->Sbuf[0], std::max(chunk_s_bytes(hp), nd * 16));
        ALLOC(p->Sbuf[1], std::max(chunk_s_bytes(hp), nd * 16));
        ALLOC(p->dp.sep_v, hp.sep_v.size() * sizeof(int));
        ALLOC(p->dp.sep_p, hp.sep_p.size() * sizeof(int));
        ALLOC(p->dp.field_pair, hp.field_pair.size() * sizeof(int));
        if (hp.can_fuse) ALLOC(p->dp.unit_e0, (size_t)total_units(hp) * hp.N * 16);
    }
    if (hp.nyquist == WKE_NYQ_KEEP) {
        ALLOC(p->Vbuf[0], chunk_v_bytes(hp));
        ALLOC(p->Vbuf[1], chunk_v_bytes(hp));
    }
    p->dp.H = p->Hbuf[0];
    p->dp.S = p->Sbuf[0];
    p->dp.fwd_tmp = needs_unit_buffers(hp) ? p->Hbuf[0] : p->Sbuf[0];
    ALLOC(p->dp.Qacc, (size_t)n_accumulators(hp) * nd * 8);
    ALLOC(p->dp.Qacc_im, (size_t)n_accumulators(hp) * nd * 8);
    ALLOC(p->dp.group_cfield, (size_t)hp.n_groups * sizeof(int));
    ALLOC(p->dp.phase, nf * hp.d * hp.N * cxb);
    ALLOC(p->dp.tw, hp.N * cxb);
    ALLOC(p->dp.tw64, hp.N_in * 16);
    if (hp.dealias) {
        ALLOC(p->dp.ghat_in, grid_in_elems(hp) * cxb);
        ALLOC(p->dp.ffine, nd * tb);
        ALLOC(p->dp.map0, nd * 16);
        ALLOC(p->dp.map1, nd * 16);
        ALLOC(p->dp.Kint, (size_t)hp.N * hp.N_in * 16);
        ALLOC(p->dp.Kproj, (size_t)hp.N * hp.N_in * 16);
    }
    ALLOC(p->dp.prod_local, hp.prod_fa.size() * 2 * sizeof(int));
    ALLOC(p->dp.prod_W, (size_t)hp.n_groups * hp.products_per_group * 8);
    ALLOC(p->f_stage, grid_in_elems(hp) * tb);
    ALLOC(p->Q_stage, grid_in_elems(hp) * tb);
    ALLOC(p->rk_y, grid_in_elems(hp) * tb);
    ALLOC(p->rk_k, grid_in_elems(hp) * tb);
    ALLOC(p->rk_acc, grid_in_elems(hp) * 8);
    ALLOC(p->mom_partials, (size_t)moments_partials_count(hp) * (hp.d + 2) * 8);
#undef ALLOC
    rc = hp.precision == WKE_FP32 ? upload_tables<float>(p) : upload_tables<double>(p);
    if (rc) goto error;
    {
        cudaError_t e = cudaStreamCreateWithFlags(&p->s1, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s3, cudaStreamNonBlocking);
        for (cudaEvent_t *ev : {&p->ev_fork, &p->ev_join, &p->ev_fwd, &p->ev_p1[0], &p->ev_p1[1], &p->ev_p2[0],
                                &p->ev_p2[1], &p->ev_nq[0], &p->ev_nq[1]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "stream and event creation");
            goto error;
        }
    }
    if ((rc = clear_accumulators(p, nullptr))) goto error;
    {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "plan set-up");
            goto error;
        }
    }
    *out = p;
    return WKE_OK;
error:
    free_plan(p);
    delete p;
    return rc;
}

int wke_plan_destroy(wke_plan *plan) {
    if (!plan) return WKE_OK;
    free_plan(plan);
    delete plan;
    return WKE_OK;
}

// Counts of a plan layout (shared by wke_plan_get_info and wke_plan_describe).
static void fill_info(const HostPlan &hp, wke_plan_info *info) {
    info->d = hp.d;
    info->N = hp.N_in;
    info->N_compute = hp.N;
    info->shared_fields = hp.shared ? 1 : 0;
    info->units_per_collision = (int)total_units(hp);
    info->M = hp.M;
    info->precision = hp.split ? WKE_SPLIT : hp.precision;
    info->n_groups = hp.n_groups;
    info->fields_per_group = hp.fields_per_group;
    info->products_per_group = hp.products_per_group;
    info->groups_per_chunk = hp.groups_per_chunk;
    info->n_chunks = hp.n_chunks;
    info->launches_per_collision = launches_per_collision(hp);
    info->separable = hp.separable ? 1 : 0;
    info->pair_planes_per_collision = hp.separable ? hp.chunk_p0.back() : 0;
    info->fused_products = hp.fused ? 1 : 0;
    info->row_values_per_collision = hp.separable ? hp.chunk_v0.back() : 0;
    info->rule_products_available = hp.cube.empty() ? 0 : 1;
    info->flops_per_collision = plan_flops(hp);
    info->l2_bytes_per_collision = plan_l2_bytes(hp);
}

int wke_plan_get_info(const wke_plan *plan, wke_plan_info *info) {
    if (!plan || !info) return fail(WKE_ERR_INVALID, "plan or info is NULL");
    fill_info(plan->hp, info);
    info->device_bytes = plan->bytes;
    return WKE_OK;
}

int wke_plan_describe(int d, int N, double L, int M, const wke_quadrature *quad, wke_plan_info *info) {
    if (!info) return fail(WKE_ERR_INVALID, "info is NULL");
    HostPlan hp;
    int rc = build_host_plan(d, N, L, M, quad, hp);
    if (rc) return rc;
    fill_info(hp, info);
    info->device_bytes = plan_device_bytes(hp);
    return WKE_OK;
}

int wke_plan_node_table(const wke_plan *plan, double *out) {
    if (!plan || !out) return fail(WKE_ERR_INVALID, "plan or output is NULL");
    const HostPlan &hp = plan->hp;
    const int d = hp.d;
    for (int p = 0; p < hp.M; ++p) {
        double *row = out + (size_t)p * (1 + 3 * d);
        row[0] = hp.W[p];
        for (int a = 0; a < d; ++a) {
            row[1 + a] = hp.q[(size_t)p * d + a];
            row[1 + d + a] = hp.a[(size_t)p * d + a];
            row[1 + 2 * d + a] = hp.b[(size_t)p * d + a];
        }
    }
    return WKE_OK;
}

int wke_collision_ex(wke_plan *plan, const void *f, void *Q, void *Qim, void *stream) {
    NvtxRange nvtx_range("wke_collision_ex");
    if (!plan || !f || !Q) return fail(WKE_ERR_INVALID, "plan, f and Q must be non-NULL");
    if (f == Q || (Qim && (Qim == Q || Qim == f))) return fail(WKE_ERR_INVALID, "f, Q and Qim must not alias");
    return collision(plan, f, Q, Qim, static_cast<cudaStream_t>(stream));
}

int wke_collision(wke_plan *plan, const void *f, void *Q, void *stream) {
    NvtxRange nvtx_range("wke_collision");
    return wke_collision_ex(plan, f, Q, nullptr, stream);
}

int wke_collision_spectrum(wke_plan *plan, const void *f, void *Q, void *Qhat, void *stream) {
    NvtxRange nvtx_range("wke_collision_spectrum");
    if (!plan || !f || !Q || !Qhat) return fail(WKE_ERR_INVALID, "plan, f, Q and Qhat must be non-NULL");
    const size_t es = plan->hp.precision == WKE_FP64 ? 8 : 4, n = grid_in_elems(plan->hp);
    auto overlap = [](const void *a, size_t na, const void *b, size_t nb) {
        const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
        return x < y + nb && y < x + na;
    };
    if (overlap(f, n * es, Q, n * es) || overlap(f, n * es, Qhat, 2 * n * es) || overlap(Q, n * es, Qhat, 2 * n * es))
        return fail(WKE_ERR_INVALID, "f, Q and Qhat must not overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = collision(plan, f, Q, nullptr, s);
    if (rc) return rc;
    // ordered after the evaluation on `s`, whose forward scratch it reuses
    rc = plan->hp.precision == WKE_FP64 ? spectrum_T<double>(plan->hp, plan->dp, Q, Qhat, s)
                                        : spectrum_T<float>(plan->hp, plan->dp, Q, Qhat, s);
    if (rc) return cuda_fail(static_cast<cudaError_t>(rc), "Q-hat transform");
    return WKE_OK;
}

int wke_collision_host(wke_plan *plan, const void *f_host, void *Q_host) {
    NvtxRange nvtx_range("wke_collision_host");
    if (!plan || !f_host || !Q_host) return fail(WKE_ERR_INVALID, "plan, f_host and Q_host must be non-NULL");
    const size_t bytes = grid_in_elems(plan->hp) * (plan->hp.precision == WKE_FP64 ? 8 : 4);
    cudaStream_t s = plan->stream;
    cudaError_t e = cudaMemcpyAsync(plan->f_stage, f_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    int rc = collision(plan, plan->f_stage, plan->Q_stage, nullptr, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(Q_host, plan->Q_stage, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    return WKE_OK;
}

int wke_plan_set_stream(wke_plan *plan, void *stream) {
    if (!plan) return fail(WKE_ERR_INVALID, "plan is NULL");
    plan->stream = static_cast<cudaStream_t>(stream);
    return WKE_OK;
}

// Butcher tableaux: b (weights) and c (node of the next stage) for forward
// Euler, Heun and classical RK4.
static bool rk_tableau(int stages, const double **b, const double **c) {
    static const double b1[1] = {1.0}, c1[1] = {0.0};
    static const double b2[2] = {0.5, 0.5}, c2[2] = {1.0, 0.0};
    static const double b4[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}, c4[4] = {0.5, 0.5, 1.0, 0.0};
    if (stages == 1) *b = b1, *c = c1;
    else if (stages == 2) *b = b2, *c = c2;
    else if (stages == 4) *b = b4, *c = c4;
    else return false;
    return true;
}

// Enqueue one step on stream s: every stage's evaluation launched directly
// (no nested graph) followed by its stage kernel, then the update.
static int enqueue_step(wke_plan *plan, void *f, double dt, int stages, cudaStream_t s) {
    const double *b, *c;
    rk_tableau(stages, &b, &c);
    const HostPlan &hp = plan->hp;
    const bool f32 = hp.precision == WKE_FP32;
    for (int st = 0; st < stages; ++st) {
        const void *y = st == 0 ? f : plan->rk_y;
        int e = enqueue(plan, y, plan->rk_k, nullptr, s);
        if (e) return e;
        void *ynext = st == stages - 1 ? nullptr : plan->rk_y;
        e = f32 ? rk_stage_T<float>(hp, f, plan->rk_k, plan->rk_acc, ynext, b[st], c[st] * dt, st == 0, s)
                : rk_stage_T<double>(hp, f, plan->rk_k, plan->rk_acc, ynext, b[st], c[st] * dt, st == 0, s);
        if (e) return e;
    }
    return f32 ? rk_final_T<float>(hp, f, plan->rk_acc, dt, s) : rk_final_T<double>(hp, f, plan->rk_acc, dt, s);
}

// The instantiated graph of a whole step for (f, dt, stages), captured on
// first use (at most 8 per plan, least recently used evicted).
static int step_graph_for(wke_plan *p, void *f, double dt, int stages, cudaGraphExec_t *out) {
    for (StepGraph &g : p->step_graphs)
        if (g.f == f && g.dt == dt && g.stages == stages) {
            g.used = ++p->tick;
            *out = g.exec;
            return WKE_OK;
        }
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(p->s1, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail(ce, "step graph capture start");
    int e = enqueue_step(p, f, dt, stages, p->s1);
    ce = cudaStreamEndCapture(p->s1, &graph);
    if (e || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return cuda_fail(e ? (cudaError_t)e : ce, "step graph capture");
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "step graph instantiation");
    if (p->step_graphs.size() >= 8) {
        size_t lru = 0;
        for (size_t i = 1; i < p->step_graphs.size(); ++i)
            if (p->step_graphs[i].used < p->step_graphs[lru].used) lru = i;
        cudaGraphExecDestroy(p->step_graphs[lru].exec);
        p->step_graphs.erase(p->step_graphs.begin() + lru);
    }
    p->step_graphs.push_back({f, dt, stages, exec, ++p->tick});
    *out = exec;
    return WKE_OK;
}

int wke_step(wke_plan *plan, void *f, double dt, int rk_stages) {
    NvtxRange nvtx_range("wke_step");
    if (!plan || !f) return fail(WKE_ERR_INVALID, "plan and f must be non-NULL");
    if (!std::isfinite(dt)) return fail(WKE_ERR_INVALID, "dt must be finite");
    const double *b, *c;
    if (!rk_tableau(rk_stages, &b, &c)) return fail(WKE_ERR_INVALID, "rk_stages must be 1, 2 or 4");
    cudaStream_t s = plan->stream;
    int rc;
    if (plan->dirty && (rc = clear_accumulators(plan, s))) return rc;
    int e;
    if (plan->use_graphs && !plan->profiling) {
        cudaGraphExec_t exec;
        if ((rc = step_graph_for(plan, f, dt, rk_stages, &exec))) {
            plan->dirty = true;
            return rc;
        }
        e = (int)cudaGraphLaunch(exec, s);
    } else {
        e = enqueue_step(plan, f, dt, rk_stages, s);
    }
    if (e) {
        plan->dirty = true;
        return cuda_fail((cudaError_t)e, "Runge-Kutta step");
    }
    return WKE_OK;
}

int wke_moments(wke_plan *plan, const void *g, double *out, void *stream) {
    if (!plan || !g || !out) return fail(WKE_ERR_INVALID, "plan, g and out must be non-NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int e = plan->hp.precision == WKE_FP32 ? moments_T<float>(plan->hp, g, plan->mom_partials, out, s)
                                           : moments_T<double>(plan->hp, g, plan->mom_partials, out, s);
    if (e) return cuda_fail((cudaError_t)e, "moments");
    return WKE_OK;
}

// Pass-2 points per thread the kernels actually use: lengths 3 * 2^a always
// take 12, N >= 128 always 8, otherwise the tuned value.
static int effective_p2(const HostPlan &hp) { return hp.N % 3 == 0 ? 12 : hp.N >= 128 ? 8 : hp.tune_p2_points; }

int wke_plan_get_tuning(const wke_plan *plan, wke_tuning *out) {
    if (!plan || !out) return fail(WKE_ERR_INVALID, "plan and out must be non-NULL");
    out->pass2_points_per_thread = effective_p2(plan->hp);
    out->pass1_units_per_block = plan->hp.tune_p1_units_per_block;
    out->fuse_products = plan->hp.fused ? 1 : 0;
    out->forward_fp32 = plan->hp.tune_forward_fp32 ? 1 : 0;
    out->rule_products = plan->hp.fused && !plan->hp.cube.empty() && plan->hp.tune_rule_products ? 1 : 0;
    return WKE_OK;
}

int wke_plan_set_tuning(wke_plan *plan, const wke_tuning *t) {
    if (!plan || !t) return fail(WKE_ERR_INVALID, "plan and tuning must be non-NULL");
    if (t->pass2_points_per_thread != 4 && t->pass2_points_per_thread != 8 &&
        !(t->pass2_points_per_thread == 12 && plan->hp.N % 3 == 0))
        return fail(WKE_ERR_INVALID, "pass2_points_per_thread must be 4 or 8 (or 12 for N = 3 * 2^a)");
    if (t->pass1_units_per_block < 0 || t->pass1_units_per_block > max_chunk_units(plan->hp))
        return fail(WKE_ERR_INVALID, "pass1_units_per_block must be 0..units per chunk");
    if (t->fuse_products != 0 && t->fuse_products != 1)
        return fail(WKE_ERR_INVALID, "fuse_products must be 0 or 1");
    if (t->forward_fp32 != 0 && t->forward_fp32 != 1)
        return fail(WKE_ERR_INVALID, "forward_fp32 must be 0 or 1");
    if (t->forward_fp32 && (plan->hp.precision != WKE_FP32 || plan->hp.dealias))
        return fail(WKE_ERR_INVALID, "forward_fp32 needs a WKE_FP32 plan that is not de-aliased");
    if (t->rule_products != 0 && t->rule_products != 1)
        return fail(WKE_ERR_INVALID, "rule_products must be 0 or 1");
    if (t->rule_products && (!t->fuse_products || plan->hp.cube.empty()))
        return fail(WKE_ERR_INVALID, "rule_products needs fuse_products and a plan of the cube rule");
    if (t->fuse_products && !plan->hp.can_fuse)
        return fail(WKE_ERR_INVALID, "this plan has no fused axis-0 + product kernel (3D FP32 shared layouts only)");
    if (!t->fuse_products && !plan->Hbuf[0]) {
        // the separate axis-0 pass needs the unit buffers the fused plan went without
        plan->hp.fused = false;
        int rc = dev_alloc(plan, &plan->Hbuf[0], chunk_unit_bytes(plan->hp));
        if (!rc) rc = dev_alloc(plan, &plan->Hbuf[1], chunk_unit_bytes(plan->hp));
        if (rc) {
            plan->hp.fused = true;
            release_unit_buffers(plan);
            return rc;
        }
    }
    plan->hp.fused = t->fuse_products == 1;
    plan->hp.tune_forward_fp32 = t->forward_fp32 == 1;
    if (t->fuse_products) plan->hp.tune_rule_products = t->rule_products == 1;
    plan->hp.tune_p2_points = t->pass2_points_per_thread == 12 ? 8 : t->pass2_points_per_thread;
    plan->hp.tune_p1_units_per_block = t->pass1_units_per_block;
    free_graphs(plan);
    return WKE_OK;
}

int wke_plan_autotune(wke_plan *plan, const void *f, void *Q, int reps, wke_tuning *chosen, double *best_ms) {
    if (!plan || !f || !Q || reps < 1) return fail(WKE_ERR_INVALID, "plan, f, Q and reps >= 1 are required");
    const HostPlan &hp = plan->hp;
    std::vector<wke_tuning> cands;
    const int p2s[2] = {4, 8};
    const int upc = max_chunk_units(hp);
    const int p1s[4] = {0, 1, 2, 3};
    const bool p2_choice = hp.N <= 64 && hp.N % 3 != 0;
    // the axis-0 layout matters only where a separate axis-0 pass runs, and
    // pass 1's units per block only where pass 1 transforms units
    const bool had_units = plan->Hbuf[0] != nullptr;
    for (int fz = hp.can_fuse ? 1 : 0; fz >= 0; --fz)
        for (int a = 0; a < (p2_choice && !fz ? 2 : 1); ++a)
            for (int b = 0; b < (hp.d == 3 && !hp.separable ? 4 : 1); ++b)
                for (int rp = fz && !hp.cube.empty() ? 1 : 0; rp >= 0; --rp)
                    if (p1s[b] <= upc)
                        cands.push_back(wke_tuning{p2_choice ? p2s[a] : effective_p2(hp), p1s[b], fz,
                                                   hp.tune_forward_fp32 ? 1 : 0, rp});
    cudaStream_t s = plan->stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "autotune events");
    wke_tuning best = cands[0];
    double best_t = 1e300;
    int rc = WKE_OK;
    for (const wke_tuning &c : cands) {
        if ((rc = wke_plan_set_tuning(plan, &c))) break;
        if ((rc = collision(plan, f, Q, nullptr, s))) break;      // warm-up (and graph capture)
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !rc; ++r) rc = collision(plan, f, Q, nullptr, s);
        cudaEventRecord(e1, s);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (rc) break;
        if (ce != cudaSuccess) {
            rc = cuda_fail(ce, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < best_t) {
            best_t = ms / reps;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = wke_plan_set_tuning(plan, &best))) return rc;
    if (best.fuse_products && !had_units) {   // the unit buffers were only needed while tuning
        const cudaError_t ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune");
        release_unit_buffers(plan);
    }
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return WKE_OK;
}

int wke_plan_create_autotuned(int d, int N, double L, int M, const wke_quadrature *quad, const void *f, void *Q,
                              void *stream, int reps, wke_plan **out, int *layout_out, double *best_ms) {
    if (!out) return fail(WKE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!quad || !f || !Q || reps < 1) return fail(WKE_ERR_INVALID, "quad, f, Q and reps >= 1 are required");
    // pencil layouts: which axes each shifted field is transformed along on
    // its own (per-group and shared: all of them; separable: axis 0 only)
    std::vector<int> layouts;
    if (quad->layout != WKE_LAYOUT_AUTO) {
        layouts.push_back(quad->layout);
    } else {
        if (d == 3 && quad->precision != WKE_SPLIT) layouts.push_back(WKE_LAYOUT_SEPARABLE);
        layouts.push_back(WKE_LAYOUT_SHARED);
        if (quad->precision != WKE_SPLIT) layouts.push_back(WKE_LAYOUT_PER_GROUP);
    }
    wke_plan *best = nullptr;
    double best_t = 1e300;
    int best_layout = -1, last_rc = WKE_ERR_INVALID;
    std::string last_msg = "no layout applies";
    for (int lay : layouts) {
        wke_quadrature q = *quad;
        q.layout = lay;
        wke_plan *p = nullptr;
        int rc = wke_plan_create(d, N, L, M, &q, &p);
        if (rc) {   // this layout does not apply to the rule (or does not fit): try the next
            last_rc = rc;
            last_msg = wke_last_error_string();
            continue;
        }
        if (stream) rc = wke_plan_set_stream(p, stream);
        double ms = 0.0;
        if (!rc) rc = wke_plan_autotune(p, f, Q, reps, nullptr, &ms);
        if (rc) {
            const std::string msg = wke_last_error_string();
            wke_plan_destroy(p);
            if (best) wke_plan_destroy(best);
            return fail(rc, "autotuning layout " + std::to_string(lay) + ": " + msg);
        }
        if (ms < best_t) {
            if (best) wke_plan_destroy(best);
            best = p;
            best_t = ms;
            best_layout = lay;
        } else {
            wke_plan_destroy(p);
        }
    }
    if (!best) return fail(last_rc, last_msg);
    *out = best;
    if (layout_out) *layout_out = best_layout;
    if (best_ms) *best_ms = best_t;
    return WKE_OK;
}

int wke_plan_use_graphs(wke_plan *plan, int enable) {
    if (!plan) return fail(WKE_ERR_INVALID, "plan is NULL");
    plan->use_graphs = enable != 0;
    if (!plan->use_graphs) free_graphs(plan);
    return WKE_OK;
}

int wke_plan_profile(wke_plan *plan, int enable) {
    if (!plan) return fail(WKE_ERR_INVALID, "plan is NULL");
    plan->profiling = enable != 0;
    plan->ev_used = 0;
    plan->ev_class.clear();
    return WKE_OK;
}

int wke_plan_profile_read(wke_plan *plan, double *out) {
    if (!plan || !out) return fail(WKE_ERR_INVALID, "plan and out must be non-NULL");
    for (int k = 0; k < 2 * WKE_PROF_CLASSES; ++k) out[k] = 0.0;
    for (size_t i = 0; i < plan->ev_class.size(); ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, plan->ev_pool[2 * i], plan->ev_pool[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "reading kernel timings (is the stream idle?)");
        out[2 * plan->ev_class[i]] += ms;
        out[2 * plan->ev_class[i] + 1] += 1.0;
    }
    plan->ev_used = 0;
    plan->ev_class.clear();
    return WKE_OK;
}

const char *wke_last_error_string(void) { return wke::last_error(); }

#ifdef WKE_CHECK
const char *wke_version(void) { return "wke-gb300 0.2 (sm_103a, bounds-checked)"; }
#else
const char *wke_version(void) { return "wke-gb300 0.2 (sm_103a)"; }
#endif

int wke_check_status(unsigned *flags) {
    if (!flags) return fail(WKE_ERR_INVALID, "flags is NULL");
    *flags = 0;
#ifdef WKE_CHECK
    unsigned *w = check_word();
    if (!w) return fail(WKE_ERR_CUDA, "check word unavailable");
    cudaError_t e = cudaMemcpy(flags, w, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "reading the check word");
    if (*flags) {
        char buf[96];
        std::snprintf(buf, sizeof(buf), "bounds check failed at sites 0x%x", *flags);
        return fail(WKE_ERR_CUDA, buf);
    }
#endif
    return WKE_OK;
}

}  // extern "C"
