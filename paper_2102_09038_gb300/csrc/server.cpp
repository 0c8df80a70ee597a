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
#include <deque>
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
    size_t bytes = 0;
    int status = RTE_OK;
    std::string error;
    rte_stats stats{};
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
};

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
    long long next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

void run_request(rte_server* sv, cudaStream_t stream, Request& r) {
    rte_problem p{r.m, r.levels, r.sigma_t.data(), r.sigma_s.data(), r.g};
    rte_options o = sv->opt;
    o.max_rhs = r.nrhs;
    rte_handle* h = nullptr;
    r.status = rte_setup(&p, &o, stream, &h);
    if (r.status != RTE_OK) {
        r.error = rte_last_error();
        return;
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
    rte_destroy(h);
}

void worker(rte_server* sv) {
    cudaSetDevice(sv->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    while (true) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                return sv->stop ||
                       (!sv->pending.empty() &&
                        (sv->in_use == 0 || sv->in_use + sv->pending.front()->bytes <= sv->budget));
            });
            if (sv->stop) break;
            r = sv->pending.front();
            sv->pending.pop_front();
            sv->in_use += r->bytes;
            r->t_start = Clock::now();
        }
        run_request(sv, stream, *r);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->t_done = Clock::now();
            r->done = true;
            sv->in_use -= r->bytes;
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
    b += r * nRp * nSp * 8 * 13;               // even work arrays, E_0 CG vectors
    b += r * nRp * nSp * 4;                    // E_0 FP32 iterate
    const bool p1_pcg = o && (o->p1_route == RTE_P1_PCG ||
                              (o->p1_route == RTE_P1_AUTO && o->precision != RTE_FP64));
    if (p1_pcg) b += r * nRp * nSp * 8 * 2;    // the P_1 PCG's r and p
    b += nSm * nSm * 8 * 5 + nSp * nSp * 8 * 3;   // dense angular factors, slices
    b += 7 * nRp * nSp * 12;                   // E_0 stencil coefficients
    b += 7 * nRp * nSp * 4 * 4 / 3;            // multigrid coefficients
    b += r * nRp * nSp * 4 * 3 * 4 / 3;        // multigrid vectors
    b += 7 * nRp * (size_t)dP * dP * 12 * 4 / 3;   // E_c blocks
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
    delete sv;
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
