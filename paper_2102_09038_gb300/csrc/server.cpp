// Continuous-batching solve server (not part of the paper's method): admits
// Richardson solves (Algorithm 3) of different problems into worker slots as
// slots and an HBM budget free up.  Each slot owns a CUDA stream; a request
// runs setup, right-hand side, solve and copy-back on its slot's stream, so
// the device work of concurrent requests overlaps while every solve keeps its
// iterate and residual on the device.  Requests are admitted in arrival
// order (no request overtakes an earlier one that does not fit yet).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/rte.h"
#include "rte_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    int m = 0, levels = 0, nrhs = 1;
    double g = 0.0, tol = 1e-6;
    std::vector<double> sigma_t, sigma_s, q_nodal, u;
    std::string key;          // the operator: mesh, sphere, g and sigma fields
    rte_handle* cached = nullptr;   // an idle handle of the same operator, if one was taken
    size_t bytes = 0;
    int status = RTE_OK;
    std::string error;
    rte_stats stats{};
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
};

// A set-up handle kept after its request for the next request with the same
// operator (the solve needs only a new right-hand side).
struct Idle {
    std::string key;
    rte_handle* h = nullptr;
    size_t bytes = 0;
    int cap_rhs = 0;
};

// The operator of a request as bytes: mesh, sphere level, g and the sigma
// fields (the options are the server's, the same for every request).
std::string operator_key(const rte_problem& p) {
    const size_t nc = 2 * (size_t)p.mesh_m * p.mesh_m;
    std::string k(sizeof(int) * 2 + sizeof(double) * (1 + 2 * nc), '\0');
    char* o = &k[0];
    std::memcpy(o, &p.mesh_m, sizeof(int));
    std::memcpy(o + sizeof(int), &p.sphere_levels, sizeof(int));
    std::memcpy(o + 2 * sizeof(int), &p.g, sizeof(double));
    std::memcpy(o + 2 * sizeof(int) + sizeof(double), p.sigma_t, nc * sizeof(double));
    std::memcpy(o + 2 * sizeof(int) + sizeof(double) * (1 + nc), p.sigma_s, nc * sizeof(double));
    return k;
}

}  // namespace

struct rte_server {
    rte_options opt{};
    size_t budget = 0;
    int slots = 1, device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::map<long long, std::shared_ptr<Request>> requests;
    size_t in_use = 0;
    // idle handles, most recently used first; their bytes count against the
    // budget until they are taken again or evicted
    std::list<Idle> idle;
    size_t idle_bytes = 0;
    long long hits = 0, misses = 0;
    long long next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

// Runs one request on the slot's stream: set-up (unless an idle handle of
// the same operator was taken), right-hand side, solve, copy-back.  Returns
// the handle for the idle set, or nullptr when it was destroyed.
rte_handle* run_request(rte_server* sv, cudaStream_t stream, Request& r) {
    rte_problem p{r.m, r.levels, r.sigma_t.data(), r.sigma_s.data(), r.g};
    rte_options o = sv->opt;
    o.max_rhs = r.nrhs;
    rte_handle* h = r.cached;
    if (h) {
        rte_set_stream(h, stream);
    } else {
        r.status = rte_setup(&p, &o, stream, &h);
        if (r.status != RTE_OK) {
            r.error = rte_last_error();
            return nullptr;
        }
    }
    int nRp = 0, nSp = 0;
    rte_sizes(h, &nRp, nullptr, &nSp, nullptr, nullptr, nullptr);
    const size_t ne = (size_t)r.nrhs * nRp * nSp;
    double *qn = nullptr, *q = nullptr, *u = nullptr;
    if (cudaMallocAsync(&qn, sizeof(double) * r.nrhs * nRp, stream) != cudaSuccess ||
        cudaMallocAsync(&q, sizeof(double) * ne, stream) != cudaSuccess ||
        cudaMallocAsync(&u, sizeof(double) * ne, stream) != cudaSuccess) {
        r.status = RTE_ERR_NOMEM;
        r.error = "request buffers";
    }
    if (r.status == RTE_OK) {
        cudaMemcpyAsync(qn, r.q_nodal.data(), sizeof(double) * r.nrhs * nRp,
                        cudaMemcpyHostToDevice, stream);
        cudaMemsetAsync(u, 0, sizeof(double) * ne, stream);
        r.status = rte_rhs(h, qn, q, r.nrhs);
    }
    if (r.status == RTE_OK) {
        r.stats = rte_stats{};
        r.status = rte_solve(h, q, u, r.nrhs, r.tol, &r.stats);
        if (r.status != RTE_OK) r.error = rte_last_error();
        r.u.resize(ne);
        cudaMemcpyAsync(r.u.data(), u, sizeof(double) * ne, cudaMemcpyDeviceToHost, stream);
    }
    cudaFreeAsync(qn, stream);
    cudaFreeAsync(q, stream);
    cudaFreeAsync(u, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess && r.status == RTE_OK) {
        r.status = RTE_ERR_CUDA;
        r.error = "stream synchronisation";
    }
    if (r.status != RTE_OK) {   // a handle that failed a request is not kept
        rte_destroy(h);
        return nullptr;
    }
    return h;
}

// An idle handle for the front request, if one of its operator with enough
// right-hand sides is kept (caller holds the lock).
std::list<Idle>::iterator find_idle(rte_server* sv, const Request& r) {
    for (auto it = sv->idle.begin(); it != sv->idle.end(); ++it)
        if (it->cap_rhs >= r.nrhs && it->key == r.key) return it;
    return sv->idle.end();
}

void destroy_on(cudaStream_t stream, rte_handle* h) {
    // an idle handle has no work queued; its memory is freed in the order of
    // this slot's stream
    rte_set_stream(h, stream);
    rte_destroy(h);
}

void worker(rte_server* sv) {
    cudaSetDevice(sv->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    while (true) {
        std::shared_ptr<Request> r;
        std::vector<rte_handle*> evict;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // admit the front request when its operator has an idle handle
            // (no new memory), or when its estimate fits the budget beside
            // the running requests once idle handles are evicted (oldest
            // first); a request larger than the budget runs alone
            sv->cv_work.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->pending.empty()) return false;
                const Request& f = *sv->pending.front();
                if (find_idle(sv, f) != sv->idle.end()) return true;
                return sv->in_use == 0 || sv->in_use + f.bytes <= sv->budget;
            });
            if (sv->stop) break;
            r = sv->pending.front();
            sv->pending.pop_front();
            auto it = find_idle(sv, *r);
            if (it != sv->idle.end()) {
                r->cached = it->h;
                r->bytes = it->bytes;
                sv->idle_bytes -= it->bytes;
                sv->idle.erase(it);
                ++sv->hits;
            } else {
                ++sv->misses;
                while (!sv->idle.empty() && sv->in_use + sv->idle_bytes + r->bytes > sv->budget) {
                    evict.push_back(sv->idle.back().h);
                    sv->idle_bytes -= sv->idle.back().bytes;
                    sv->idle.pop_back();
                }
            }
            sv->in_use += r->bytes;
            r->t_start = Clock::now();
        }
        for (rte_handle* h : evict) destroy_on(stream, h);
        rte_handle* keep = run_request(sv, stream, *r);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->t_done = Clock::now();
            r->done = true;
            sv->in_use -= r->bytes;
            if (keep) {
                sv->idle.push_front(Idle{r->key, keep, r->bytes, r->nrhs});
                sv->idle_bytes += r->bytes;
            }
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
    cudaStreamDestroy(stream);
}

double secs(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

}  // namespace

extern "C" {

size_t rte_estimate_bytes(const rte_problem* p, const rte_options* o, int nrhs) {
    if (!p) return 0;
    const size_t m = p->mesh_m, nRp = (m + 1) * (m + 1), nRm = 2 * m * m;
    const size_t nSp = (size_t)4 << (2 * p->sphere_levels), nSm = 3 * nSp;
    const size_t r = nrhs > 0 ? nrhs : 1;
    const int dP = o && o->n_plus >= 0 ? (o->n_plus + 1) * (o->n_plus + 2) / 2 : 15;
    size_t b = 0;
    b += r * nRm * nSm * 8 * 5;                // odd work arrays and slices
    b += r * nRp * nSp * 8 * 10;               // even work arrays
    if (!(o ? (o->e0_route == RTE_E0_DIRECT || (o->e0_route == RTE_E0_AUTO && m <= 156))
            : m <= 156))
        b += r * nRp * nSp * (8 * 3 + 4);      // E_0 CG vectors and FP32 iterate
    const bool p1_pcg = o && (o->p1_route == RTE_P1_PCG ||
                              (o->p1_route == RTE_P1_AUTO && o->precision != RTE_FP64));
    if (p1_pcg) b += r * nRp * nSp * 8 * 2;    // the P_1 PCG's r and p
    b += nSm * nSm * 8 * 5 + nSp * nSp * 8 * 3;   // dense angular factors, slices
    const bool split = o && (o->dgemm == RTE_DGEMM_SPLIT ||
                             (o->dgemm == RTE_DGEMM_AUTO && o->precision != RTE_FP64));
    if (split && o->mk_route != RTE_MK_PCG)
        b += nRm * nSm * 8;                    // the split GEMM's reciprocal table
    b += 7 * nRp * nSp * 8;                    // E_0 stencil coefficients
    const bool direct = o ? (o->e0_route == RTE_E0_DIRECT ||
                             (o->e0_route == RTE_E0_AUTO && m <= 156))
                          : m <= 156;
    if (direct) {
        // the factor (FP64 in FP64 mode, FP32 otherwise) and its setup scratch
        const size_t ld = (m + 1 + 3) & ~(size_t)3;
        const bool fp64 = !o || o->precision == RTE_FP64;
        b += nSp * (m + 1) * ld * ld * (fp64 ? 8 : 4) + nSp * nRp * 8;
    } else {
        b += 7 * nRp * nSp * 4;                // FP64 kernel's FP32 copy
        b += 7 * nRp * nSp * 4 * 4 / 3;        // multigrid coefficients
        b += r * nRp * nSp * 4 * 3 * 4 / 3;    // multigrid vectors
    }
    b += 7 * nRp * (size_t)dP * dP * 8;       // E_c blocks (FP64 level 0)
    const bool ec_direct = dP > 0 && o && o->coarse_route == RTE_EC_DIRECT;
    if (ec_direct) {
        // the coarse factor and its set-up scratch (three FP64 row blocks)
        const size_t Bd = (m + 1) * (size_t)dP, ld = (Bd + 3) & ~(size_t)3;
        const bool fp64 = !o || o->precision == RTE_FP64;
        b += (m + 1) * Bd * ld * (fp64 ? 8 : 4) + 3 * Bd * Bd * 8;
    } else {
        b += 7 * nRp * (size_t)dP * dP * 4 * 4 / 3;   // multigrid blocks
    }
    b += r * nRp * dP * 8 * 10;                // coarse vectors
    b += 64ull << 20;                          // small arrays, allocator slack
    return b;
}

int rte_server_create(size_t hbm_budget_bytes, int slots, const rte_options* opts,
                      rte_server** out) {
    if (!out || slots < 1 || slots > 64) return rte::fail(RTE_ERR_ARG, "bad server arguments");
    auto* sv = new rte_server();
    if (opts) sv->opt = *opts; else rte_default_options(&sv->opt);
    sv->budget = hbm_budget_bytes;
    sv->slots = slots;
    cudaGetDevice(&sv->device);
    for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv);
    *out = sv;
    return RTE_OK;
}

int rte_server_submit(rte_server* sv, const rte_problem* p, const double* q_nodal, int nrhs,
                      double tol, long long* id) {
    if (!sv || !p || !q_nodal || nrhs < 1 || !id || !p->sigma_t || !p->sigma_s)
        return rte::fail(RTE_ERR_ARG, "bad submit arguments");
    auto r = std::make_shared<Request>();
    r->m = p->mesh_m;
    r->levels = p->sphere_levels;
    r->g = p->g;
    r->nrhs = nrhs;
    r->tol = tol;
    const size_t nc = 2 * (size_t)p->mesh_m * p->mesh_m;
    const size_t nn = (size_t)(p->mesh_m + 1) * (p->mesh_m + 1);
    r->sigma_t.assign(p->sigma_t, p->sigma_t + nc);
    r->sigma_s.assign(p->sigma_s, p->sigma_s + nc);
    r->q_nodal.assign(q_nodal, q_nodal + nn * nrhs);
    r->bytes = rte_estimate_bytes(p, &sv->opt, nrhs);
    r->key = operator_key(*p);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next_id++;
        sv->requests[r->id] = r;
        sv->pending.push_back(r);
        *id = r->id;
    }
    sv->cv_work.notify_all();
    return RTE_OK;
}

int rte_server_wait(rte_server* sv, long long id, double timeout_s, double* u, size_t u_len,
                    rte_stats* stats, double* latency_s, double* queue_s) {
    if (!sv) return rte::fail(RTE_ERR_ARG, "NULL server");
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        auto it = sv->requests.find(id);
        if (it == sv->requests.end()) return rte::fail(RTE_ERR_ARG, "unknown request id");
        r = it->second;
        const auto pred = [&] { return r->done; };
        if (timeout_s >= 0) {
            if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
                return rte::fail(RTE_ERR_TIMEOUT, "request still running");
        } else {
            sv->cv_done.wait(lk, pred);
        }
        sv->requests.erase(it);
    }
    if (u) {
        if (u_len < r->u.size()) return rte::fail(RTE_ERR_ARG, "result buffer too small");
        std::copy(r->u.begin(), r->u.end(), u);
    }
    if (stats) {
        double* hist = stats->history;
        const int cap = stats->history_cap;
        *stats = r->stats;
        stats->history = hist;
        stats->history_cap = cap;
    }
    if (latency_s) *latency_s = secs(r->t_submit, r->t_done);
    if (queue_s) *queue_s = secs(r->t_submit, r->t_start);
    if (r->status != RTE_OK) return rte::fail(r->status, r->error);
    return RTE_OK;
}

void rte_server_destroy(rte_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    // the idle handles' streams belonged to the workers, which destroyed
    // them on exit: free the handles in the order of a stream that exists
    cudaSetDevice(sv->device);
    for (auto& e : sv->idle) {
        rte_set_stream(e.h, nullptr);
        rte_destroy(e.h);
    }
    delete sv;
}

int rte_server_cache_stats(rte_server* sv, long long* hits, long long* misses,
                           size_t* idle_bytes) {
    if (!sv) return rte::fail(RTE_ERR_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (hits) *hits = sv->hits;
    if (misses) *misses = sv->misses;
    if (idle_bytes) *idle_bytes = sv->idle_bytes;
    return RTE_OK;
}

int rte_solve_batch(const rte_problem* probs, const double* const* q_nodal, const int* nrhs,
                    double* const* u, int count, double tol, const rte_options* opts,
                    size_t hbm_budget_bytes, int slots, rte_stats* stats) {
    if (!probs || !q_nodal || !nrhs || !u || count < 0)
        return rte::fail(RTE_ERR_ARG, "bad batch arguments");
    rte_server* sv = nullptr;
    RTE_TRY(rte_server_create(hbm_budget_bytes, slots, opts, &sv));
    std::vector<long long> ids(count);
    int rc = RTE_OK;
    for (int i = 0; i < count && rc == RTE_OK; ++i)
        rc = rte_server_submit(sv, &probs[i], q_nodal[i], nrhs[i], tol, &ids[i]);
    for (int i = 0; i < count; ++i) {
        if (rc != RTE_OK && ids[i] == 0) continue;
        const size_t n = (size_t)nrhs[i] * (probs[i].mesh_m + 1) * (probs[i].mesh_m + 1) *
                         ((size_t)4 << (2 * probs[i].sphere_levels));
        const int r = rte_server_wait(sv, ids[i], -1.0, u[i], n, stats ? &stats[i] : nullptr,
                                      nullptr, nullptr);
        if (r != RTE_OK && rc == RTE_OK) rc = r;
    }
    rte_server_destroy(sv);
    return rc;
}

}  // extern "C"
