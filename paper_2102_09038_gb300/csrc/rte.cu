// C ABI of the library: setup (Section 4 assembly, Section 5.1/5.4 eigenpairs
// and coarse matrix), the operator applies of Algorithm 1, the preconditioner
// of Algorithm 2 / eq. (product_pre) and the Richardson loop of Algorithm 3.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "device.h"
#include "mg_host.h"
#include "rte_internal.h"
#include "tc_gemm.h"
#include "h2.h"
#include "tune.h"

namespace rte {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

}  // namespace rte

using namespace rte;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct TimerRec {
    int name;
    cudaEvent_t a, b;
};

struct rte_handle {
    rte_options opt;
    cudaStream_t stream = nullptr;
    DevSystem d{};
    std::vector<void*> allocs;
    // host copies kept for rte_export
    std::vector<double> h_Sp, h_Sm, h_m, h_MSm, h_A1, h_A2, h_omx, h_omy, h_lamP,
        h_lamM, h_WpN, h_ec;
    // E_c = sum_q S_q (x) G_q: Q scalar stencils [Q][nnz] and Q angular
    // d x d blocks (Q = 0: no Kronecker form, the explicit blocks are used)
    int ec_Q = 0;
    std::vector<double> h_ecS, h_ecG;
    // workspace
    int cap_rhs = 0;
    double *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *z4 = nullptr;   // odd
    double *z5 = nullptr, *z6 = nullptr, *z7 = nullptr, *zsk = nullptr;  // PCG route
    void* slices = nullptr;                                             // split GEMM operand
    double *e1 = nullptr, *e2 = nullptr, *e3 = nullptr, *e4 = nullptr, *e5 = nullptr,
           *e6 = nullptr, *e7 = nullptr, *e8 = nullptr;                     // even
    double *e9 = nullptr, *e10 = nullptr;   // even, RTE_P1_PCG only
    double *c1 = nullptr, *c2 = nullptr;                                    // coarse
    // mixed precision: FP32 even vectors, low-precision odd GEMM operands
    bool mixed = false;
    float *f1 = nullptr, *f2 = nullptr, *f3 = nullptr;
    void *zl1 = nullptr, *zl2 = nullptr, *xl = nullptr;
    float* zf = nullptr;
    double *partial = nullptr, *sc = nullptr;                               // reductions
    void* e0work = nullptr;
    size_t e0bytes = 0;
    void* cowork = nullptr;
    size_t cobytes = 0;
    SolveStatus* status = nullptr;
    unsigned long long* trace = nullptr;   // phase trace buffer (profiling)
    // digit slices the split GEMMs of the current solve use (<= d.split_S,
    // from the solve's tolerance; d.split_S outside rte_solve)
    int split_now = 0;
    // autotuned tile widths of the low-precision GEMMs (0: by N)
    int bn_mk1 = 0, bn_mk2 = 0, bn_kplus = 0;
    // Algorithm 1's PCG loop as a CUDA graph whose while node repeats one
    // iteration until a device-side check ends it (one executable graph per
    // right-hand-side count), captured on a private stream; mk_state: [0]
    // iterations of the last solve, [1] converged, [2] non-finite residual,
    // [3] iterations since set-up (device, and a pinned host copy)
    cudaStream_t cap_stream = nullptr;
    std::map<int, cudaGraphExec_t> mk_graph;   // by 16 nrhs + slices
    int* mk_state = nullptr;
    int* mk_state_host = nullptr;
    int mk_total_seen = 0;
    long long mk_body_launches = 0;
    bool mk_pending = false;
    bool capturing = false;
    // statistics of the last inner solves
    int e0_iters = 0, co_iters = 0, mk_iters = 0;
    // E_0^{-1} work of the current solve: launches, V-cycles, and V-cycles
    // weighted by the fraction of quads (direction columns) still active
    int e0_launches = 0;
    double e0_vcycles = 0.0, e0_active_vcycles = 0.0;
    // timing
    bool timing = false;
    std::vector<std::string> tnames;
    std::vector<TimerRec> trecs;
    std::vector<double> tms;
    // wall-clock stages of rte_setup
    std::vector<std::string> setup_names;
    std::vector<double> setup_ms;
    std::vector<long long> tcount;
};

namespace {

// Device memory of a handle is stream-ordered (cudaMallocAsync on the
// handle's stream, freed the same way by rte_destroy): unlike cudaMalloc and
// cudaFree, neither waits for the work of other streams, so the server's
// slots set up and tear down solves while the others compute.  The device's
// default pool keeps up to kPoolKeep bytes of freed memory for reuse.
constexpr uint64_t kPoolKeep = 8ull << 30;

void keep_pool_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t cur = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur);
    if (cur < kPoolKeep) {
        uint64_t v = kPoolKeep;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &v);
    }
}

// Refuses, before any allocation, a problem whose estimated device memory
// (rte_estimate_bytes) exceeds what the device can still give: its free
// memory plus what the default pool holds unused.
int check_device_memory(const rte_problem& p, const rte_options& o) {
    if (p.mesh_m < 1 || p.sphere_levels < 0 || p.sphere_levels > 5) return RTE_OK;   // refused later
    const size_t need = rte_estimate_bytes(&p, &o, o.max_rhs);
    size_t free_b = 0, total_b = 0;
    RTE_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    int dev = 0;
    RTE_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    uint64_t reserved = 0, used = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    }
    const size_t avail = free_b + (size_t)(reserved > used ? reserved - used : 0);
    if (need > avail)
        return fail(RTE_ERR_NOMEM, "the problem needs about " + std::to_string(need >> 20) +
                                       " MiB of device memory; " + std::to_string(avail >> 20) +
                                       " MiB are available");
    return RTE_OK;
}

template <typename T>
int dalloc(rte_handle* h, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMallocAsync((void**)p, n * sizeof(T), h->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(RTE_ERR_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back((void*)*p);
    return RTE_OK;
}

// One cuSOLVER handle per host thread, kept for the thread's life (creating
// and destroying one per call allocates and frees device memory each time).
struct SolverHandle {
    cusolverDnHandle_t h = nullptr;
    ~SolverHandle() {
        if (h) cusolverDnDestroy(h);
    }
};

int solver_handle(cudaStream_t s, cusolverDnHandle_t* out) {
    thread_local SolverHandle sh;
    if (!sh.h && cusolverDnCreate(&sh.h) != CUSOLVER_STATUS_SUCCESS) {
        sh.h = nullptr;
        return fail(RTE_ERR_CUDA, "cusolverDnCreate failed");
    }
    cusolverDnSetStream(sh.h, s);
    *out = sh.h;
    return RTE_OK;
}

template <typename T>
int upload(rte_handle* h, const T** dst, const std::vector<T>& src) {
    T* p = nullptr;
    RTE_TRY(dalloc(h, &p, src.size()));
    if (!src.empty())
        RTE_CUDA_TRY(cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T),
                                     cudaMemcpyHostToDevice, h->stream));
    *dst = p;
    return RTE_OK;
}

// ------------------------------------------------------------- timing
// Wall-clock stages of rte_setup: mark() waits for the stream (so a stage's
// device work is charged to it) and records the time since the last mark.
struct SetupClock {
    rte_handle* h;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void mark(const char* name) {
        if (h) cudaStreamSynchronize(h->stream);
        const auto now = std::chrono::steady_clock::now();
        if (h) {
            h->setup_names.push_back(name);
            h->setup_ms.push_back(std::chrono::duration<double, std::milli>(now - t).count());
        }
        t = now;
    }
};

struct Scope {
    rte_handle* h;
    int idx = -1;
    cudaEvent_t b{};
    Scope(rte_handle* hh, const char* name) : h(hh) {
        if (!h->timing || h->capturing) return;
        for (size_t i = 0; i < h->tnames.size(); ++i)
            if (h->tnames[i] == name) idx = (int)i;
        if (idx < 0) {
            idx = (int)h->tnames.size();
            h->tnames.push_back(name);
            h->tms.push_back(0.0);
            h->tcount.push_back(0);
        }
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, h->stream);
        h->trecs.push_back({idx, a, b});
    }
    ~Scope() {
        if (idx >= 0) cudaEventRecord(b, h->stream);
    }
};

void flush_timers(rte_handle* h) {
    if (h->trecs.empty()) return;
    cudaStreamSynchronize(h->stream);
    for (auto& t : h->trecs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            h->tms[t.name] += ms;
            h->tcount[t.name] += 1;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    h->trecs.clear();
}

// ---------------------------------------------------------- eigenpairs
// Symmetric eigen-decomposition of an n x n matrix on the device
// (cusolverDnDsyevd, setup only).  On return C holds the eigenvectors as
// rows (row-major view of the column-major output) and w the ascending
// eigenvalues.
int sym_eig(rte_handle* h, std::vector<double>& C, std::vector<double>& w, int n) {
    cusolverDnHandle_t cs = nullptr;
    RTE_TRY(solver_handle(h->stream, &cs));
    const cudaStream_t st = h->stream;
    double *dA = nullptr, *dW = nullptr, *dWork = nullptr;
    int* dInfo = nullptr;
    int rc = RTE_OK;
    int lwork = 0;
    if (cudaMallocAsync(&dA, sizeof(double) * (size_t)n * n, st) != cudaSuccess ||
        cudaMallocAsync(&dW, sizeof(double) * n, st) != cudaSuccess ||
        cudaMallocAsync(&dInfo, sizeof(int), st) != cudaSuccess) {
        rc = fail(RTE_ERR_NOMEM, "eigensolver allocation failed");
    }
    if (rc == RTE_OK) {
        cudaMemcpyAsync(dA, C.data(), sizeof(double) * (size_t)n * n,
                        cudaMemcpyHostToDevice, h->stream);
        if (cusolverDnDsyevd_bufferSize(cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                        n, dA, n, dW, &lwork) != CUSOLVER_STATUS_SUCCESS)
            rc = fail(RTE_ERR_CUDA, "syevd_bufferSize failed");
    }
    if (rc == RTE_OK && cudaMallocAsync(&dWork, sizeof(double) * (size_t)std::max(lwork, 1), st) != cudaSuccess)
        rc = fail(RTE_ERR_NOMEM, "eigensolver workspace allocation failed");
    if (rc == RTE_OK &&
        cusolverDnDsyevd(cs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW,
                         dWork, lwork, dInfo) != CUSOLVER_STATUS_SUCCESS)
        rc = fail(RTE_ERR_CUDA, "syevd failed");
    if (rc == RTE_OK) {
        int info = 0;
        w.resize(n);
        cudaMemcpyAsync(C.data(), dA, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost,
                        h->stream);
        cudaMemcpyAsync(w.data(), dW, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
        cudaMemcpyAsync(&info, dInfo, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess)
            rc = fail(RTE_ERR_CUDA, "eigensolver synchronisation failed");
        else if (info != 0)
            rc = fail(RTE_ERR_CUDA, "syevd did not converge");
    }
    if (dA) cudaFreeAsync(dA, st);
    if (dW) cudaFreeAsync(dW, st);
    if (dWork) cudaFreeAsync(dWork, st);
    if (dInfo) cudaFreeAsync(dInfo, st);
    return rc;
}

// Inverses of `count` SPD n x n matrices (row-major, consecutive in A) by
// Cholesky on the device (cusolverDnDpotrf / potrs against the identity,
// setup only); written to inv as FP32.
int spd_inverse_batch(rte_handle* h, int n, int count, const std::vector<double>& A,
                      std::vector<float>& inv) {
    cusolverDnHandle_t cs = nullptr;
    RTE_TRY(solver_handle(h->stream, &cs));
    const cudaStream_t st = h->stream;
    const size_t nn = (size_t)n * n;
    double *dA = nullptr, *dB = nullptr, *dWork = nullptr;
    int* dInfo = nullptr;
    int rc = RTE_OK, lwork = 0;
    std::vector<double> I(nn, 0.0), out(nn);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    inv.resize(nn * count);
    if (cudaMallocAsync(&dA, nn * 8, st) != cudaSuccess || cudaMallocAsync(&dB, nn * 8, st) != cudaSuccess ||
        cudaMallocAsync(&dInfo, sizeof(int), st) != cudaSuccess)
        rc = fail(RTE_ERR_NOMEM, "coarse inverse allocation failed");
    if (rc == RTE_OK &&
        cusolverDnDpotrf_bufferSize(cs, CUBLAS_FILL_MODE_LOWER, n, dA, n, &lwork) !=
            CUSOLVER_STATUS_SUCCESS)
        rc = fail(RTE_ERR_CUDA, "potrf_bufferSize failed");
    if (rc == RTE_OK && cudaMallocAsync(&dWork, sizeof(double) * std::max(lwork, 1), st) != cudaSuccess)
        rc = fail(RTE_ERR_NOMEM, "coarse inverse workspace allocation failed");
    for (int b = 0; b < count && rc == RTE_OK; ++b) {
        // symmetric: the row-major matrix is its own column-major transpose
        cudaMemcpyAsync(dA, A.data() + nn * b, nn * 8, cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(dB, I.data(), nn * 8, cudaMemcpyHostToDevice, h->stream);
        int info = 0;
        if (cusolverDnDpotrf(cs, CUBLAS_FILL_MODE_LOWER, n, dA, n, dWork, lwork, dInfo) !=
                CUSOLVER_STATUS_SUCCESS ||
            cudaMemcpyAsync(&info, dInfo, sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess || info != 0) {
            rc = fail(RTE_ERR_ARG, "coarsest multigrid matrix is not positive definite");
            break;
        }
        if (cusolverDnDpotrs(cs, CUBLAS_FILL_MODE_LOWER, n, n, dA, n, dB, n, dInfo) !=
            CUSOLVER_STATUS_SUCCESS) {
            rc = fail(RTE_ERR_CUDA, "potrs failed");
            break;
        }
        cudaMemcpyAsync(out.data(), dB, nn * 8, cudaMemcpyDeviceToHost, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            rc = fail(RTE_ERR_CUDA, "coarse inverse synchronisation failed");
            break;
        }
        for (size_t t = 0; t < nn; ++t) inv[nn * b + t] = (float)out[t];
    }
    if (dA) cudaFreeAsync(dA, st);
    if (dB) cudaFreeAsync(dB, st);
    if (dWork) cudaFreeAsync(dWork, st);
    if (dInfo) cudaFreeAsync(dInfo, st);
    return rc;
}

bool chol_inv_sym(int d, const double* A, double* Ainv) {
    // Gauss-Jordan inverse with partial pivoting of a small d x d matrix
    std::vector<double> M(A, A + d * d), I(d * d, 0.0);
    for (int i = 0; i < d; ++i) I[i * d + i] = 1.0;
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (std::fabs(M[r * d + c]) > std::fabs(M[piv * d + c])) piv = r;
        if (!(std::fabs(M[piv * d + c]) > 0)) return false;
        if (piv != c)
            for (int k = 0; k < d; ++k) {
                std::swap(M[c * d + k], M[piv * d + k]);
                std::swap(I[c * d + k], I[piv * d + k]);
            }
        const double inv = 1.0 / M[c * d + c];
        for (int k = 0; k < d; ++k) {
            M[c * d + k] *= inv;
            I[c * d + k] *= inv;
        }
        for (int r = 0; r < d; ++r) {
            if (r == c) continue;
            const double f = M[r * d + c];
            if (f == 0.0) continue;
            for (int k = 0; k < d; ++k) {
                M[r * d + k] -= f * M[c * d + k];
                I[r * d + k] -= f * I[c * d + k];
            }
        }
    }
    std::memcpy(Ainv, I.data(), sizeof(double) * d * d);
    return true;
}

// 3x3 lower Cholesky factor
bool chol3(const double* A, double* L) {
    for (int i = 0; i < 9; ++i) L[i] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[3 * i + j];
            for (int k = 0; k < j; ++k) s -= L[3 * i + k] * L[3 * j + k];
            if (i == j) {
                if (!(s > 0)) return false;
                L[3 * i + i] = std::sqrt(s);
            } else {
                L[3 * i + j] = s / L[3 * j + j];
            }
        }
    return true;
}

void inv_lower3(const double* L, double* Li) {
    for (int i = 0; i < 9; ++i) Li[i] = 0.0;
    for (int c = 0; c < 3; ++c) {
        for (int i = 0; i < 3; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[3 * i + k] * Li[3 * k + c];
            Li[3 * i + c] = s / L[3 * i + i];
        }
    }
}

// Transposes every bs x bs block of a block array in place (the E_c kernels
// read blocks column by column).
template <typename V>
void transpose_blocks(std::vector<V>& a, int bs) {
    const size_t bb = (size_t)bs * bs;
    for (size_t o = 0; o + bb <= a.size(); o += bb)
        for (int x = 0; x < bs; ++x)
            for (int y = x + 1; y < bs; ++y) std::swap(a[o + x * bs + y], a[o + y * bs + x]);
}

// Restriction lists of level D from its finer level F (ELL over D's nodes:
// the fine nodes that interpolate from each coarse node, with weights).
int upload_restriction(rte_handle* h, const MGHostLevel& F, MGDeviceLevel& D) {
    int w = 0;
    for (int I = 0; I < D.n; ++I) w = std::max(w, F.rptr[I + 1] - F.rptr[I]);
    std::vector<int> ri((size_t)D.n * w, 0);
    std::vector<float> rwv((size_t)D.n * w, 0.f);
    for (int I = 0; I < D.n; ++I)
        for (int k = F.rptr[I]; k < F.rptr[I + 1]; ++k) {
            ri[(size_t)I * w + (k - F.rptr[I])] = F.ridx[k];
            rwv[(size_t)I * w + (k - F.rptr[I])] = F.rw[k];
        }
    RTE_TRY(upload(h, &D.ridx, ri));
    RTE_TRY(upload(h, &D.rw, rwv));
    D.rwid = w;
    return RTE_OK;
}

// Uploads the multigrid hierarchy of E_c in Kronecker form: per level the Q
// scalar stencils node-major [n][7][Qp] (Qp = Q rounded up to 4), the
// inverted diagonal blocks sum_q S_q(i,i) G_q, and the work vectors of d
// values per node; the angular blocks G_q (Q x d x d) are shared by all
// levels.
int upload_mg_kron(rte_handle* h, const MGHost& mh, int cols, int d, int Q,
                   const std::vector<double>& G, MGDevice& out) {
    out.L = (int)mh.levels.size();
    if (out.L > kMaxMGLevels) return fail(RTE_ERR_ARG, "too many multigrid levels");
    out.nu = std::max(1, std::min(h->opt.mg_sweeps, 16));
    out.cap_cols = cols;
    out.dense = mh.dense_coarse;
    out.Q = Q;
    const int Qp = (Q + 3) / 4 * 4;
    const size_t dd = (size_t)d * d;
    for (int l = 0; l < out.L; ++l) {
        const MGHostLevel& L = mh.levels[l];
        MGDeviceLevel& D = out.lev[l];
        D.m = L.m;
        D.n = (L.m + 1) * (L.m + 1);
        std::vector<double> ell;
        RTE_TRY(to_ell(L, Q, 1, ell));   // [Q][7][n]
        std::vector<float> sk((size_t)D.n * 7 * Qp, 0.f);
        for (int i = 0; i < D.n; ++i)
            for (int dir = 0; dir < 7; ++dir)
                for (int q = 0; q < Q; ++q)
                    sk[((size_t)i * 7 + dir) * Qp + q] = (float)ell[((size_t)q * 7 + dir) * D.n + i];
        RTE_TRY(upload(h, &D.sv, sk));
        std::vector<float> di((size_t)D.n * dd);
        std::vector<double> blk(dd), inv(dd);
        for (int i = 0; i < D.n; ++i) {
            std::fill(blk.begin(), blk.end(), 0.0);
            for (int q = 0; q < Q; ++q) {
                const double sq = ell[((size_t)q * 7 + 0) * D.n + i];
                if (sq == 0.0) continue;
                for (size_t t = 0; t < dd; ++t) blk[t] += sq * G[(size_t)q * dd + t];
            }
            if (!chol_inv_sym(d, blk.data(), inv.data()))
                return fail(RTE_ERR_ARG, "singular coarse multigrid diagonal block");
            for (size_t t = 0; t < dd; ++t) di[(size_t)i * dd + t] = (float)inv[t];
        }
        transpose_blocks(di, d);
        RTE_TRY(upload(h, &D.dinv, di));
        if (l > 0) RTE_TRY(upload_restriction(h, mh.levels[l - 1], D));
        const size_t nv = (size_t)D.n * cols * d;
        RTE_TRY(dalloc(h, &D.X, nv));
        RTE_TRY(dalloc(h, &D.Xt, nv));
        RTE_TRY(dalloc(h, &D.B, nv));
    }
    std::vector<float> gf(G.begin(), G.end());
    RTE_TRY(upload(h, &out.G, gf));
    return RTE_OK;
}

// Uploads a host multigrid hierarchy in ELL form; work vectors hold cols
// columns of bs values per node.
int upload_mg(rte_handle* h, const MGHost& mh, int cols, int bs, bool block_dinv,
              MGDevice& out) {
    out.L = (int)mh.levels.size();
    if (out.L > kMaxMGLevels) return fail(RTE_ERR_ARG, "too many multigrid levels");
    out.nu = std::max(1, std::min(h->opt.mg_sweeps, 16));
    out.cap_cols = cols;
    out.dense = mh.dense_coarse;
    for (int l = 0; l < out.L; ++l) {
        const MGHostLevel& L = mh.levels[l];
        MGDeviceLevel& D = out.lev[l];
        D.m = L.m;
        D.n = (L.m + 1) * (L.m + 1);
        if (bs > 1) {   // E_c blocks (the E_0 kernels use the node-major parts)
            std::vector<double> ell;
            RTE_TRY(to_ell(L, mh.slots, bs, ell));
            transpose_blocks(ell, bs);
            RTE_TRY(upload(h, &D.val, std::vector<float>(ell.begin(), ell.end())));
        }
        if (block_dinv) {
            std::vector<float> di;
            RTE_TRY(block_diag_inverse(L, bs, di));
            transpose_blocks(di, bs);
            RTE_TRY(upload(h, &D.dinv, di));
        }
        if (l > 0) RTE_TRY(upload_restriction(h, mh.levels[l - 1], D));
        const size_t nv = (size_t)D.n * cols * bs;
        RTE_TRY(dalloc(h, &D.X, nv));
        RTE_TRY(dalloc(h, &D.Xt, nv));
        RTE_TRY(dalloc(h, &D.B, nv));
    }
    return RTE_OK;
}

// The multigrid of E_c uses its Kronecker form when it has at most this many
// terms (4 + 4 per sigma class) and d^+ <= 16, else the explicit d x d blocks.
constexpr int kEcMaxTerms = 16;

// Coarsening stops at a level of at most this many nodes, which is then
// solved with a dense inverse.

int setup_multigrid(rte_handle* h, const HostSystem& hs, SetupClock* clk) {
    DevSystem& d = h->d;
    const int cap = h->opt.max_rhs;
    // ------------------------------------------------------------ E_0
    if (d.e0_direct) {
        // the level-0 coefficients alone: the factorisation reads them
        const int slots[6] = {kK11, kK12, kK22, kBx, kBy, kMt};
        const size_t nnz = hs.st.col.size();
        MGHostLevel L;
        L.m = hs.m;
        L.st = hs.st;
        L.vals.resize(6 * nnz);
        for (int q = 0; q < 6; ++q)
            std::copy(hs.sval.begin() + (size_t)slots[q] * nnz,
                      hs.sval.begin() + (size_t)(slots[q] + 1) * nnz, L.vals.begin() + q * nnz);
        std::vector<double> ell6;
        RTE_TRY(to_ell(L, 6, 1, ell6));
        const double* dell = nullptr;
        RTE_TRY(upload(h, &dell, ell6));
        double* c = nullptr;
        RTE_TRY(dalloc(h, &c, (size_t)7 * hs.nRp * hs.nSp));
        e0_coefficients(h->stream, hs.nRp, hs.nSp, dell, d.e0s, c, nullptr);
        d.e0coef = c;
        // factor: FP64 in FP64 mode, FP32 in the mixed modes; FP64 scratch
        // of one Schur complement inverse per direction, freed at the end
        const bool fp64 = !h->mixed;
        const size_t fb = e0_direct_bytes(hs.m, hs.nSp, fp64);
        double* scratch = nullptr;
        if (cudaMallocAsync(&scratch, e0_direct_scratch_bytes(hs.m, hs.nSp), h->stream) !=
            cudaSuccess)
            return fail(RTE_ERR_NOMEM, "E_0 factorisation scratch");
        int rc = RTE_OK;
        if (fp64) {
            double* f = nullptr;
            rc = dalloc(h, &f, fb / sizeof(double));
            if (rc == RTE_OK) {
                rc = e0_direct_factor(h->stream, d, scratch, nullptr, f);
                d.e0lu64 = f;
            }
        } else {
            float* f = nullptr;
            rc = dalloc(h, &f, fb / sizeof(float));
            if (rc == RTE_OK) {
                rc = e0_direct_factor(h->stream, d, scratch, f, nullptr);
                d.e0lu32 = f;
            }
        }
        cudaFreeAsync(scratch, h->stream);
        RTE_TRY(rc);
    } else {
        const int slots[6] = {kK11, kK12, kK22, kBx, kBy, kMt};
        const size_t nnz = hs.st.col.size();
        std::vector<double> v((size_t)6 * nnz);
        for (int q = 0; q < 6; ++q)
            std::copy(hs.sval.begin() + (size_t)slots[q] * nnz,
                      hs.sval.begin() + (size_t)(slots[q] + 1) * nnz, v.begin() + q * nnz);
        MGHost mh;
        RTE_TRY(build_hierarchy(hs.m, hs.st, v, 6, 1, kDenseCoarseNodes, mh));
        RTE_TRY(upload_mg(h, mh, cap * hs.nSp, 1, false, d.e0mg));
        // the six spatial parts of every level, node-major sv[i][dir][8]
        // (the kernels form each direction's coefficients from them)
        for (int l = 0; l < d.e0mg.L; ++l) {
            std::vector<double> ell;
            RTE_TRY(to_ell(mh.levels[l], 6, 1, ell));
            const size_t nl = (size_t)(mh.levels[l].m + 1) * (mh.levels[l].m + 1);
            std::vector<float> sv(nl * 7 * 8, 0.f);
            for (size_t i = 0; i < nl; ++i)
                for (int dir = 0; dir < 7; ++dir)
                    for (int q = 0; q < 6; ++q)
                        sv[(i * 7 + dir) * 8 + q] = (float)ell[((size_t)q * 7 + dir) * nl + i];
            RTE_TRY(upload(h, &d.e0mg.lev[l].sv, sv));
        }
        {
            std::vector<float> w8((size_t)hs.nSp * 8, 0.f);
            for (int k = 0; k < hs.nSp; ++k)
                for (int q = 0; q < 6; ++q) w8[(size_t)k * 8 + q] = (float)hs.e0s[6 * k + q];
            RTE_TRY(upload(h, &d.e0mg.w8, w8));
            std::vector<float> wq((size_t)6 * hs.nSp);
            for (int q = 0; q < 6; ++q)
                for (int k = 0; k < hs.nSp; ++k) wq[(size_t)q * hs.nSp + k] = (float)hs.e0s[6 * k + q];
            RTE_TRY(upload(h, &d.e0mg.wq, wq));
        }
        if (d.e0mg.dense) {
            const int nc = (mh.levels.back().m + 1) * (mh.levels.back().m + 1);
            std::vector<double> all((size_t)nc * nc * hs.nSp), one;
            for (int k = 0; k < hs.nSp; ++k) {
                std::vector<double> w(hs.e0s.begin() + 6 * k, hs.e0s.begin() + 6 * k + 6);
                coarse_dense_matrix(mh.levels.back(), w, 6, 1, one);
                std::copy(one.begin(), one.end(), all.begin() + (size_t)nc * nc * k);
            }
            std::vector<float> inv;   // [direction][i][j]
            RTE_TRY(spd_inverse_batch(h, nc, hs.nSp, all, inv));
            // rows padded with zeros to a multiple of 4 (16-byte loads)
            const size_t n4 = ((size_t)nc + 3) & ~(size_t)3;
            std::vector<float> pad((size_t)hs.nSp * nc * n4, 0.f);
            for (size_t r = 0; r < (size_t)hs.nSp * nc; ++r)
                std::copy(inv.begin() + r * nc, inv.begin() + (r + 1) * nc, pad.begin() + r * n4);
            RTE_TRY(upload(h, &d.e0mg.cinv, pad));
        }
        // level-0 operator of the CG in ELL form, per direction
        std::vector<double> ell6;
        RTE_TRY(to_ell(mh.levels[0], 6, 1, ell6));
        const double* dell = nullptr;
        RTE_TRY(upload(h, &dell, ell6));
        double* c = nullptr;
        RTE_TRY(dalloc(h, &c, (size_t)7 * hs.nRp * hs.nSp));
        e0_coefficients(h->stream, hs.nRp, hs.nSp, dell, d.e0s, c, nullptr);
        d.e0coef = c;
    }
    if (clk) clk->mark(d.e0_direct ? "E_0 factorisation" : "E_0 multigrid");
    // ------------------------------------------------------------ E_c
    if (d.dP > 0 && d.ec_direct) {
        // level-0 work vectors of the coarse CG kernel only (r in B, the
        // sweeps' result in X, their scratch row in Xt)
        MGDevice& E = d.ecmg;
        E.L = 1;
        E.nu = 1;
        E.cap_cols = cap;
        E.dense = false;
        E.Q = 0;
        MGDeviceLevel& D = E.lev[0];
        D.m = hs.m;
        D.n = hs.nRp;
        const size_t nv = (size_t)D.n * cap * d.dP;
        RTE_TRY(dalloc(h, &D.X, nv));
        RTE_TRY(dalloc(h, &D.Xt, nv));
        RTE_TRY(dalloc(h, &D.B, nv));
        MGHostLevel L0;
        L0.m = hs.m;
        L0.st = hs.st;
        L0.vals = h->h_ec;
        std::vector<double> ell;
        RTE_TRY(to_ell(L0, 1, d.dP, ell));
        transpose_blocks(ell, d.dP);
        RTE_TRY(upload(h, &d.ec_ell, ell));
        const bool fp64 = !h->mixed;
        const size_t fb = ec_direct_bytes(hs.m, d.dP, fp64);
        cusolverDnHandle_t cs = nullptr;
        RTE_TRY(solver_handle(h->stream, &cs));
        if (fp64) {
            double* f = nullptr;
            RTE_TRY(dalloc(h, &f, fb / sizeof(double)));
            RTE_TRY(ec_direct_factor(h->stream, cs, d, nullptr, f));
            d.eclu64 = f;
        } else {
            float* f = nullptr;
            RTE_TRY(dalloc(h, &f, fb / sizeof(float)));
            RTE_TRY(ec_direct_factor(h->stream, cs, d, f, nullptr));
            d.eclu32 = f;
        }
    } else if (d.dP > 0) {
        MGHost mh;
        const int dP = d.dP;
        if (h->ec_Q > 0) {   // Kronecker form: Galerkin products of Q scalar stencils
            const int Q = h->ec_Q;
            RTE_TRY(build_hierarchy(hs.m, hs.st, h->h_ecS, Q, 1, kDenseCoarseNodes, mh));
            RTE_TRY(upload_mg_kron(h, mh, cap, dP, Q, h->h_ecG, d.ecmg));
            if (d.ecmg.dense) {
                const MGHostLevel& L = mh.levels.back();
                const int n = (L.m + 1) * (L.m + 1), N = n * dP;
                const size_t nnz = L.st.col.size(), dd = (size_t)dP * dP;
                std::vector<double> A((size_t)N * N, 0.0);
                for (int i = 0; i < n; ++i)
                    for (int k = L.st.ptr[i]; k < L.st.ptr[i + 1]; ++k) {
                        const int j = L.st.col[k];
                        for (int q = 0; q < Q; ++q) {
                            const double sq = L.vals[(size_t)q * nnz + k];
                            if (sq == 0.0) continue;
                            const double* g = &h->h_ecG[(size_t)q * dd];
                            for (int a = 0; a < dP; ++a)
                                for (int b = 0; b < dP; ++b)
                                    A[(size_t)(i * dP + a) * N + j * dP + b] += sq * g[a * dP + b];
                        }
                    }
                std::vector<float> inv;
                RTE_TRY(spd_inverse_batch(h, N, 1, A, inv));
                RTE_TRY(upload(h, &d.ecmg.cinv, inv));
            }
        } else {
            RTE_TRY(build_hierarchy(hs.m, hs.st, h->h_ec, 1, dP, kDenseCoarseNodes, mh));
            RTE_TRY(upload_mg(h, mh, cap, dP, true, d.ecmg));
            if (d.ecmg.dense) {
                std::vector<double> A;
                coarse_dense_matrix(mh.levels.back(), {}, 1, dP, A);
                std::vector<float> inv;
                const int N = (mh.levels.back().m + 1) * (mh.levels.back().m + 1) * dP;
                RTE_TRY(spd_inverse_batch(h, N, 1, A, inv));
                RTE_TRY(upload(h, &d.ecmg.cinv, inv));
            }
        }
        // FP64 level-0 blocks of the CG's own apply
        MGHostLevel L0;
        L0.m = hs.m;
        L0.st = hs.st;
        L0.vals = h->h_ec;
        std::vector<double> ell;
        RTE_TRY(to_ell(L0, 1, d.dP, ell));
        transpose_blocks(ell, d.dP);
        RTE_TRY(upload(h, &d.ec_ell, ell));
    }
    // the kernels index the level descriptors at run time: keep them in
    // device memory rather than in the (then locally copied) kernel argument
    if (!d.e0_direct)
        RTE_TRY(upload(h, &d.e0mg.dev_lev,
                       std::vector<MGDeviceLevel>(d.e0mg.lev, d.e0mg.lev + d.e0mg.L)));
    if (d.dP > 0)
        RTE_TRY(upload(h, &d.ecmg.dev_lev,
                       std::vector<MGDeviceLevel>(d.ecmg.lev, d.ecmg.lev + d.ecmg.L)));
    return RTE_OK;
}

// ------------------------------------------------------------ autotuning
// Launch shapes chosen by measurement (tune.cpp) on this handle's workspace
// at max_rhs: the block size of the two SpMM kernels and, in the mixed
// modes, the tile width of each tensor-core contraction.  Results are
// cached per shape for the process.
int tune_launches(rte_handle* h) {
    if (!h->opt.autotune) return RTE_OK;
    DevSystem& d = h->d;
    const int nr = h->cap_rhs;
    cudaStream_t s = h->stream;
    auto ok = [] { return cudaGetLastError() == cudaSuccess ? RTE_OK : RTE_ERR_CUDA; };
    // defined operands (zeros) for the timing runs, sizes as in alloc_workspace
    const size_t ne = (size_t)nr * d.nRp * d.nSp, no = (size_t)nr * d.nRm * d.nSm;
    RTE_CUDA_TRY(cudaMemsetAsync(h->e1, 0, ne * sizeof(double), s));
    RTE_CUDA_TRY(cudaMemsetAsync(h->z2, 0, no * sizeof(double), s));
    if (h->mixed) {
        const size_t lo = d.lo.bf16 ? 2 : 4;
        RTE_CUDA_TRY(cudaMemsetAsync(h->zl1, 0, no * lo, s));
        RTE_CUDA_TRY(cudaMemsetAsync(h->zl2, 0, no * lo, s));
        RTE_CUDA_TRY(cudaMemsetAsync(h->f1, 0, ne * sizeof(float), s));
        RTE_CUDA_TRY(cudaMemsetAsync(h->xl, 0, ne * lo, s));
    }
    const int tpb[3] = {128, 256, 512};
    char key[200];
    int b = 1;
    std::snprintf(key, sizeof key, "apply_A m=%d nS=%d rhs=%d", d.m, d.nSp, nr);
    RTE_TRY(autotune(s, key, 3, [&](int c) {
        d.tpb_A = tpb[c];
        apply_A(s, d, h->e1, h->z1, nr);
        return ok();
    }, &b, 1));
    d.tpb_A = tpb[b];
    std::snprintf(key, sizeof key, "apply_even m=%d nS=%d rhs=%d", d.m, d.nSp, nr);
    RTE_TRY(autotune(s, key, 3, [&](int c) {
        d.tpb_even = tpb[c];
        apply_even(s, d, h->z2, h->e1, nullptr, h->e2, nr, 3);
        return ok();
    }, &b, 1));
    d.tpb_even = tpb[b];
    if (!h->mixed) return RTE_OK;
    const bool bf = d.lo.bf16;
    const int bns[2] = {128, 256};
    TcGemmArgs g{};
    g.tf32 = !bf;
    g.A = h->zl1; g.Bt = d.lo.VmT; g.C = h->zl2;
    g.M = nr * d.nRm; g.N = d.nSm; g.K = d.nSm; g.ldc = d.nSm;
    g.epi = 1; g.at = d.lo.cell_at; g.as = d.lo.cell_as; g.lam = d.lo.lamM; g.rows = d.nRm;
    g.out_bf16 = bf;
    std::snprintf(key, sizeof key, "tc_gemm %s M=%d N=%d K=%d epi=1", bf ? "bf16" : "tf32", g.M,
                  g.N, g.K);
    RTE_TRY(autotune(s, key, 2, [&](int c) { g.bn = bns[c]; return tc_gemm(s, g); }, &b,
                     g.N > 128 ? 1 : 0));
    h->bn_mk1 = bns[b];
    g.A = h->zl2; g.Bt = d.lo.Vm; g.C = h->zf; g.epi = 0; g.out_bf16 = false;
    std::snprintf(key, sizeof key, "tc_gemm %s M=%d N=%d K=%d epi=0", bf ? "bf16" : "tf32", g.M,
                  g.N, g.K);
    RTE_TRY(autotune(s, key, 2, [&](int c) { g.bn = bns[c]; return tc_gemm(s, g); }, &b,
                     g.N > 128 ? 1 : 0));
    h->bn_mk2 = bns[b];
    TcGemmArgs k{};
    k.tf32 = !bf;
    k.A = bf ? static_cast<const void*>(h->xl) : static_cast<const void*>(h->f1);
    k.Bt = d.lo.Sp; k.C = h->f3;
    k.M = nr * d.nRp; k.N = d.nSp; k.K = d.nSp; k.ldc = d.nSp; k.rows = 1;
    std::snprintf(key, sizeof key, "tc_gemm %s M=%d N=%d K=%d epi=0", bf ? "bf16" : "tf32", k.M,
                  k.N, k.K);
    RTE_TRY(autotune(s, key, 2, [&](int c) { k.bn = bns[c]; return tc_gemm(s, k); }, &b,
                     k.N > 128 ? 1 : 0));
    h->bn_kplus = bns[b];
    return tc_gemm_error(s);
}

// ------------------------------------------------------------ workspace
int ensure_workspace(rte_handle* h, int nrhs) {
    if (nrhs <= h->cap_rhs) return RTE_OK;
    return fail(RTE_ERR_ARG, "nrhs exceeds opts.max_rhs given to rte_setup");
}

int alloc_workspace(rte_handle* h, int nrhs) {
    const DevSystem& d = h->d;
    const size_t ne = (size_t)nrhs * d.nRp * d.nSp;
    const size_t no = (size_t)nrhs * d.nRm * d.nSm;
    const size_t nc = (size_t)nrhs * d.nRp * std::max(d.dP, 1);
    RTE_TRY(dalloc(h, &h->z1, no));
    RTE_TRY(dalloc(h, &h->z2, no));
    RTE_TRY(dalloc(h, &h->z3, no));
    RTE_TRY(dalloc(h, &h->z4, no));
    if (h->opt.mk_route == RTE_MK_PCG) {
        RTE_TRY(dalloc(h, &h->z5, no));
        RTE_TRY(dalloc(h, &h->z6, no));
        RTE_TRY(dalloc(h, &h->z7, no));
        RTE_TRY(dalloc(h, &h->mk_state, 4));
        RTE_CUDA_TRY(cudaMemsetAsync(h->mk_state, 0, 4 * sizeof(int), h->stream));
        if (cudaMallocHost(&h->mk_state_host, 4 * sizeof(int)) != cudaSuccess)
            return fail(RTE_ERR_NOMEM, "pinned PCG state");
        std::memset(h->mk_state_host, 0, 4 * sizeof(int));
    }
    RTE_TRY(dalloc(h, &h->zsk, (size_t)nrhs * d.nRm * d.dM));
    if (d.split_S > 0) {
        const size_t b = std::max(ozaki_slice_bytes(nrhs * d.nRm, d.nSm, d.split_S),
                                  ozaki_slice_bytes(nrhs * d.nRp, d.nSp, d.split_S));
        char* p = nullptr;
        RTE_TRY(dalloc(h, &p, b));
        h->slices = p;
    }
    double** ev[] = {&h->e1, &h->e2, &h->e3, &h->e4, &h->e5, &h->e6, &h->e7, &h->e8};
    for (auto p : ev) RTE_TRY(dalloc(h, p, ne));
    if (h->opt.p1_route == RTE_P1_PCG) {
        RTE_TRY(dalloc(h, &h->e9, ne));
        RTE_TRY(dalloc(h, &h->e10, ne));
    }
    RTE_TRY(dalloc(h, &h->c1, nc));
    RTE_TRY(dalloc(h, &h->c2, nc));
    RTE_TRY(dalloc(h, &h->partial, (size_t)nrhs * 1024));
    RTE_TRY(dalloc(h, &h->sc, (size_t)nrhs * 16));
    char* w = nullptr;
    if (!d.e0_direct) {
        h->e0bytes = e0_cg_work_bytes(d, nrhs);
        RTE_TRY(dalloc(h, &w, h->e0bytes));
        h->e0work = w;
    }
    h->cobytes = coarse_cg_work_bytes(d, nrhs);
    RTE_TRY(dalloc(h, &w, h->cobytes));
    h->cowork = w;
    RTE_TRY(dalloc(h, &h->status, 1));
    if (h->mixed) {
        const size_t lo = d.lo.bf16 ? 2 : 4;
        RTE_TRY(dalloc(h, &h->f1, ne));
        RTE_TRY(dalloc(h, &h->f2, ne));
        RTE_TRY(dalloc(h, &h->f3, ne));
        RTE_TRY(dalloc(h, &h->zf, no));
        char* p = nullptr;
        RTE_TRY(dalloc(h, &p, no * lo));
        h->zl1 = p;
        RTE_TRY(dalloc(h, &p, no * lo));
        h->zl2 = p;
        RTE_TRY(dalloc(h, &p, ne * lo));
        h->xl = p;
    }
    h->cap_rhs = nrhs;
    return RTE_OK;
}

// --------------------------------------------------------- operators
// Digit slices of the split GEMMs now: the solve's choice, else all.
int split_slices_now(const rte_handle* h) {
    return h->split_now > 0 ? std::min(h->split_now, h->d.split_S) : h->d.split_S;
}

// Slices for a solve to relative residual tol: the split product of S
// slices differs from the FP64 one by at most about S 2^-7S of the operand
// row scales (the dropped digit pairs and the truncated digits), and the
// residual's contractions are taken accurate to tol / 1000 in that measure,
// S 2^-7S <= tol / 1000: 5 slices at 1e-6, 6 at 1e-8, 7 at 1e-10 (capped by
// the slices set up, split_slices).
int slices_for_tol(double tol, int smax) {
    for (int S = 3; S < smax; ++S)
        if (S * std::ldexp(1.0, -7 * S) <= tol / 1000.0) return S;
    return smax;
}

// Z2 = (M^- - K^-)^{-1} Z1 in the full eigenbasis of (S^-, M_S^-):
// per cell j, (|T_j| (sigma_t M_S^- - sigma_s S^-))^{-1} = V diag(1/(at - lam as)) V^T
int mk_inv_eigen(rte_handle* h, const double* Z1, double* Z2, int nrhs) {
    const DevSystem& d = h->d;
    const int rows = nrhs * d.nRm;
    if (d.split_S > 0) {
        const int S = split_slices_now(h);
        int* ea = nullptr;
        {
            Scope sc(h, "split_digits");
            RTE_TRY(ozaki_split(h->stream, Z1, rows, d.nSm, S, h->slices, &ea));
        }
        {
            Scope sc(h, "dgemm_split_mk1");
            RTE_TRY(ozaki_gemm(h->stream, h->slices, ea, rows, d.sl_VmT, d.ex_VmT, d.nSm, d.nSm,
                               S, h->z4, d.nSm, 1, d.mk_rinv, d.nRm, d.split_S));
        }
        {
            Scope sc(h, "split_digits");
            RTE_TRY(ozaki_split(h->stream, h->z4, rows, d.nSm, S, h->slices, &ea));
        }
        Scope sc(h, "dgemm_split_mk2");
        RTE_TRY(ozaki_gemm(h->stream, h->slices, ea, rows, d.sl_Vm, d.ex_Vm, d.nSm, d.nSm, S,
                           Z2, d.nSm, 0, nullptr, 1, d.split_S));
        return RTE_OK;
    }
    {
        Scope sc(h, "gemm_mk_eig1");
        gemm_f64(h->stream, rows, d.nSm, d.nSm, Z1, d.nSm, d.Vm, d.nSm, h->z4, d.nSm, 1.0,
                 0.0, 1, d.cell_at, d.cell_as, d.lamM, d.nRm);
    }
    {
        Scope sc(h, "gemm_mk_eig2");
        gemm_f64(h->stream, rows, d.nSm, d.nSm, h->z4, d.nSm, d.VmT, d.nSm, Z2, d.nSm, 1.0,
                 0.0, 0, nullptr, nullptr, nullptr, 1);
    }
    return RTE_OK;
}

// x = (M^- - K^-_N)^{-1} b by eq. (MmKprecond):
// x = ((b W_N) .* (F - 1/at)) W_N^T + (b M_S^{-1}) / at
int mk_prec(rte_handle* h, const double* B, double* X, double* tmp, int nrhs) {
    const DevSystem& d = h->d;
    const int rows = nrhs * d.nRm;
    Scope sc(h, "mk_prec");
    gemm_f64(h->stream, rows, d.dM, d.nSm, B, d.nSm, d.WmN, d.dM, tmp, d.dM, 1.0, 0.0, 2,
             d.cell_at, d.cell_as, d.lamM, d.nRm);
    mk_minv_scale(h->stream, d, B, X, nrhs);
    gemm_f64(h->stream, rows, d.nSm, d.dM, tmp, d.dM, d.WmNT, d.nSm, X, d.nSm, 1.0, 1.0, 0,
             nullptr, nullptr, nullptr, 1);
    return RTE_OK;
}

// Y = (M^- - K^-) Z
int mk_apply(rte_handle* h, const double* Z, double* Y, double* G, int nrhs) {
    const DevSystem& d = h->d;
    Scope sc(h, "mk_apply");
    gemm_f64(h->stream, nrhs * d.nRm, d.nSm, d.nSm, Z, d.nSm, d.Sm, d.nSm, G, d.nSm, 1.0, 0.0,
             0, nullptr, nullptr, nullptr, 1);
    mk_combine(h->stream, d, Z, G, Y, nrhs);
    return RTE_OK;
}

__global__ void k_ratio(const double* num, const double* den, double* out, int n,
                        double sign) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = den[i] != 0.0 ? sign * num[i] / den[i] : 0.0;
}

// Y = (M^- - K^-) Z with K^- Z = diag(sigma_s |T|) Z S^- on the split
// (FP64-accurate) tensor-core GEMM: the PCG route of the mixed modes
int mk_apply_split(rte_handle* h, const double* Z, double* Y, double* G, int nrhs) {
    const DevSystem& d = h->d;
    Scope sc(h, "mk_apply");
    int* ea = nullptr;
    const int S = split_slices_now(h);
    RTE_TRY(ozaki_split(h->stream, Z, nrhs * d.nRm, d.nSm, S, h->slices, &ea));
    RTE_TRY(ozaki_gemm(h->stream, h->slices, ea, nrhs * d.nRm, d.sl_Sm, d.ex_Sm, d.nSm, d.nSm, S,
                       G, d.nSm, 0, nullptr, 1, d.split_S));
    mk_combine(h->stream, d, Z, G, Y, nrhs);
    return RTE_OK;
}

// End of one PCG iteration of Algorithm 1 inside the graph: counts it,
// records whether every right-hand side has ||r||^2 <= tol^2 ||b||^2 (or
// a residual is not finite) and sets the while node's condition.
__global__ void k_mk_check(const double* rr, const double* bb, int n, double tol2, int maxit,
                           int* state, cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int it = ++state[0];
    ++state[3];
    bool done = true, bad = false;
    for (int r = 0; r < n; ++r) {
        const double v = rr[r];
        if (!isfinite(v)) bad = true;
        if (!(v <= tol2 * bb[r])) done = false;
    }
    state[1] = done;
    state[2] = bad;
    cudaGraphSetConditional(loop, (!done && !bad && it < maxit) ? 1u : 0u);
}

// One PCG iteration for (M^- - K^-) X = B on the workspace of
// mk_inv_pcg (the body of the graph's while node).
int mk_pcg_body(rte_handle* h, int n, double* X, cudaGraphConditionalHandle loop) {
    const DevSystem& d = h->d;
    const size_t len = (size_t)d.nRm * d.nSm;
    double *R = h->z3, *P = h->z4, *AP = h->z5, *Zb = h->z6, *G = h->z7, *tmp = h->zsk;
    double* sc = h->sc;
    cudaStream_t s = h->stream;
    if (d.split_S > 0) RTE_TRY(mk_apply_split(h, P, AP, G, n));
    else RTE_TRY(mk_apply(h, P, AP, G, n));
    dot_per_rhs(s, P, AP, len, n, h->partial, sc + n);
    k_ratio<<<(n + 63) / 64, 64, 0, s>>>(sc, sc + n, sc + 2 * n, n, 1.0);
    axpby_per_rhs(s, P, X, len, n, sc + 2 * n, 0.0, nullptr, 1.0);          // x += alpha p
    k_ratio<<<(n + 63) / 64, 64, 0, s>>>(sc, sc + n, sc + 2 * n, n, -1.0);
    axpby_per_rhs(s, AP, R, len, n, sc + 2 * n, 0.0, nullptr, 1.0);         // r -= alpha Ap
    dot_per_rhs(s, R, R, len, n, h->partial, sc + 3 * n);                   // r.r
    RTE_TRY(mk_prec(h, R, Zb, tmp, n));
    dot_per_rhs(s, R, Zb, len, n, h->partial, sc + n);                      // rz_new
    k_ratio<<<(n + 63) / 64, 64, 0, s>>>(sc + n, sc, sc + 5 * n, n, 1.0);   // beta
    RTE_CUDA_TRY(cudaMemcpyAsync(sc, sc + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    axpby_per_rhs(s, Zb, P, len, n, nullptr, 1.0, sc + 5 * n, 0.0);         // p = z + beta p
    k_mk_check<<<1, 32, 0, s>>>(sc + 3 * n, sc + 4 * n, n, h->opt.mk_tol * h->opt.mk_tol,
                                h->opt.mk_maxit, h->mk_state, loop);
    count_launches(4);
    return RTE_OK;
}

// The executable graph of the loop for n right-hand sides: a while node
// whose body (captured on the handle's private stream) is mk_pcg_body.
int mk_graph_for(rte_handle* h, int n, double* X, cudaGraphExec_t* out) {
    // the body's split GEMMs bake in the slice count: one graph per both
    const int key = n * 16 + (h->d.split_S > 0 ? split_slices_now(h) : 0);
    auto it = h->mk_graph.find(key);
    if (it != h->mk_graph.end()) {
        *out = it->second;
        return RTE_OK;
    }
    if (!h->cap_stream)
        RTE_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    RTE_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle loop;
    int rc = RTE_OK;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        rc = fail(RTE_ERR_CUDA, "cudaGraphConditionalHandleCreate failed");
    if (rc == RTE_OK) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess)
            rc = fail(RTE_ERR_CUDA, "cudaGraphAddNode (while) failed");
    }
    if (rc == RTE_OK) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t saved = h->stream;
        const long long before = launches_total();
        h->stream = h->cap_stream;
        h->capturing = true;
        if (cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rc = fail(RTE_ERR_CUDA, "stream capture of the PCG body failed to begin");
        } else {
            rc = mk_pcg_body(h, n, X, loop);
            cudaGraph_t done = nullptr;
            const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &done);
            if (rc == RTE_OK && e != cudaSuccess)
                rc = fail(RTE_ERR_CUDA, std::string("capture of the PCG body: ") +
                                            cudaGetErrorString(e));
        }
        h->stream = saved;
        h->capturing = false;
        // capture launches nothing: the body's kernels are counted per replay
        h->mk_body_launches = launches_total() - before;
        count_launches(-h->mk_body_launches);
    }
    cudaGraphExec_t exec = nullptr;
    if (rc == RTE_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
        rc = fail(RTE_ERR_CUDA, "cudaGraphInstantiate of the PCG loop failed");
    cudaGraphDestroy(g);
    if (rc != RTE_OK) return rc;
    h->mk_graph[key] = exec;
    *out = exec;
    return RTE_OK;
}

// Iterations of the graph loops launched since the last call, once the
// stream has passed them (called after a synchronisation of the stream).
void settle_mk(rte_handle* h) {
    if (!h->mk_pending) return;
    h->mk_pending = false;
    h->mk_iters = h->mk_state_host[0];
    const int total = h->mk_state_host[3];
    count_launches((long long)(total - h->mk_total_seen) * h->mk_body_launches);
    h->mk_total_seen = total;
}

// Algorithm 1 line 2: (M^- - K^-) X = B by PCG preconditioned with
// eq. (MmKprecond); B = z1 and X = z2 inside Apply-E.  The set-up of the
// recurrence runs on the stream, then the iterations run as the graph's
// device-side loop: no host round trip per iteration.
int mk_inv_pcg(rte_handle* h, const double* B, double* X, int nrhs) {
    const DevSystem& d = h->d;
    if (!h->z5) return fail(RTE_ERR_ARG, "PCG route needs mk_route = RTE_MK_PCG at setup");
    const size_t len = (size_t)d.nRm * d.nSm;
    double *R = h->z3, *P = h->z4, *Zb = h->z6, *tmp = h->zsk;
    const int n = nrhs;
    double* sc = h->sc;
    cudaStream_t s = h->stream;
    RTE_CUDA_TRY(cudaMemcpyAsync(R, B, sizeof(double) * n * len, cudaMemcpyDeviceToDevice, s));
    RTE_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double) * n * len, s));
    dot_per_rhs(s, B, B, len, n, h->partial, sc + 4 * n);                  // b.b
    RTE_TRY(mk_prec(h, R, Zb, tmp, n));
    RTE_CUDA_TRY(cudaMemcpyAsync(P, Zb, sizeof(double) * n * len, cudaMemcpyDeviceToDevice, s));
    dot_per_rhs(s, R, Zb, len, n, h->partial, sc);                         // r.z
    cudaGraphExec_t exec = nullptr;
    RTE_TRY(mk_graph_for(h, n, X, &exec));
    RTE_CUDA_TRY(cudaMemsetAsync(h->mk_state, 0, 3 * sizeof(int), s));
    {
        Scope sc2(h, "mk_pcg_loop");
        RTE_CUDA_TRY(cudaGraphLaunch(exec, s));
    }
    RTE_CUDA_TRY(cudaMemcpyAsync(h->mk_state_host, h->mk_state, 4 * sizeof(int),
                                 cudaMemcpyDeviceToHost, s));
    h->mk_pending = true;
    return RTE_OK;
}

int mk_inv(rte_handle* h, const double* Z1, double* Z2, int nrhs) {
    if (h->opt.mk_route == RTE_MK_PCG) return mk_inv_pcg(h, Z1, Z2, nrhs);
    return mk_inv_eigen(h, Z1, Z2, nrhs);
}

// y = E x (with_k: y = (E - K^+) x).  Uses z1, z2 (and z3, z4 for routes).
int apply_E(rte_handle* h, const double* x, double* y, int nrhs, bool with_k) {
    const DevSystem& d = h->d;
    {
        Scope sc(h, "transport_A");
        apply_A(h->stream, d, x, h->z1, nrhs);
    }
    RTE_TRY(mk_inv(h, h->z1, h->z2, nrhs));
    double* V = nullptr;
    if (with_k) {
        V = h->e8;
        if (d.split_S > 0) {
            Scope sc(h, "dgemm_split_kplus");
            int* ea = nullptr;
            const int S = split_slices_now(h);
            RTE_TRY(ozaki_split(h->stream, x, nrhs * d.nRp, d.nSp, S, h->slices, &ea));
            RTE_TRY(ozaki_gemm(h->stream, h->slices, ea, nrhs * d.nRp, d.sl_Sp, d.ex_Sp, d.nSp,
                               d.nSp, S, V, d.nSp, 0, nullptr, 1, d.split_S));
        } else {
            Scope sc(h, "gemm_kplus");
            gemm_f64(h->stream, nrhs * d.nRp, d.nSp, d.nSp, x, d.nSp, d.Sp, d.nSp, V, d.nSp, 1.0,
                     0.0, 0, nullptr, nullptr, nullptr, 1);
        }
    }
    Scope sc(h, "apply_even");
    apply_even(h->stream, d, h->z2, x, V, y, nrhs, with_k ? 7 : 3);
    return RTE_OK;
}

// ---------------------------------------------- mixed-precision operators
// y = E x (with_k: (E - K^+) x) with FP32 vectors: transport and the fused
// gather in FP32, the eigenbasis contractions of (M^- - K^-)^{-1} and the
// scattering product U S^+ on the tensor cores (BF16 or TF32 operands, FP32
// accumulation).
int apply_E_lo(rte_handle* h, const float* x, float* y, int nrhs, bool with_k) {
    const DevSystem& d = h->d;
    const bool bf = d.lo.bf16;
    {
        Scope sc(h, "transport_A_lo");
        apply_A_lo(h->stream, d, x, h->zl1, bf, nrhs);
    }
    TcGemmArgs g{};
    g.tf32 = !bf;
    {
        Scope sc(h, "tc_gemm_mk1");
        g.A = h->zl1; g.Bt = d.lo.VmT; g.C = h->zl2;
        g.M = nrhs * d.nRm; g.N = d.nSm; g.K = d.nSm; g.ldc = d.nSm;
        g.epi = 1; g.at = d.lo.cell_at; g.as = d.lo.cell_as; g.lam = d.lo.lamM; g.rows = d.nRm;
        g.out_bf16 = bf;
        g.bn = h->bn_mk1;
        RTE_TRY(tc_gemm(h->stream, g));
    }
    {
        Scope sc(h, "tc_gemm_mk2");
        g.A = h->zl2; g.Bt = d.lo.Vm; g.C = h->zf; g.epi = 0; g.out_bf16 = false;
        g.bn = h->bn_mk2;
        RTE_TRY(tc_gemm(h->stream, g));
    }
    float* V = nullptr;
    if (with_k) {
        Scope sc(h, "tc_gemm_kplus");
        const void* xop = x;
        if (bf) {
            convert(h->stream, x, static_cast<__nv_bfloat16*>(h->xl),
                    (size_t)nrhs * d.nRp * d.nSp);
            xop = h->xl;
        }
        V = h->f3;
        TcGemmArgs k{};
        k.tf32 = !bf; k.A = xop; k.Bt = d.lo.Sp; k.C = V;
        k.M = nrhs * d.nRp; k.N = d.nSp; k.K = d.nSp; k.ldc = d.nSp; k.rows = 1;
        k.bn = h->bn_kplus;
        RTE_TRY(tc_gemm(h->stream, k));
    }
    Scope sc(h, "apply_even_lo");
    apply_even_lo(h->stream, d, h->zf, x, V, y, nrhs, with_k ? 7 : 3);
    return RTE_OK;
}

int read_status(rte_handle* h, SolveStatus& st) {
    RTE_CUDA_TRY(cudaMemcpyAsync(&st, h->status, sizeof(SolveStatus), cudaMemcpyDeviceToHost,
                                 h->stream));
    RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    settle_mk(h);
    if (st.timed_out) return fail(RTE_ERR_TIMEOUT, "a bounded grid barrier timed out");
    return RTE_OK;
}

// FP32 CG stalls near its rounding level: mixed modes stop the E_0 solves at
// a relative residual of at least this (the FP64 outer loop absorbs it).
constexpr double kLowInnerTol = 1e-5;

int e0_inv(rte_handle* h, const double* b, double* x, int nrhs) {
    if (h->d.e0_direct) {
        {
            Scope sc(h, h->mixed ? "e0_direct" : "e0_direct64");
            RTE_TRY(e0_direct_solve(h->stream, h->d, b, x, nrhs, !h->mixed));
        }
        h->e0_iters = 1;
        h->e0_launches += 1;
        h->e0_vcycles += 1.0;
        h->e0_active_vcycles += 1.0;
        return RTE_OK;
    }
    if (h->mixed) {
        Scope sc(h, "e0_cg_lo");
        RTE_TRY(e0_cg_lo(h->stream, h->d, b, x, nrhs, std::max(h->opt.e0_tol, kLowInnerTol),
                         h->opt.e0_maxit, h->e0work, h->e0bytes, h->status));
    } else {
        Scope sc(h, "e0_cg");
        RTE_TRY(e0_cg(h->stream, h->d, b, x, nrhs, h->opt.e0_tol, h->opt.e0_maxit, h->e0work,
                      h->e0bytes, h->status));
    }
    SolveStatus st;
    RTE_TRY(read_status(h, st));
    h->e0_iters = st.iterations;
    const double vc = st.iterations + 1.0, nq = nrhs * h->d.nSp / 4.0;
    h->e0_launches += 1;
    h->e0_vcycles += vc;
    h->e0_active_vcycles += st.active_quads > 0 ? st.active_quads / nq : vc;
    return RTE_OK;
}

// coarse tolerances from which the mixed modes run the coarse CG's own
// products in FP32
constexpr double kCoarseF32Tol = 1e-2;

int coarse_inv(rte_handle* h, const double* b, double* x, int nrhs) {
    {
        Scope sc(h, "coarse_cg");
        // mixed modes at a loose tolerance (the default 0.3): the CG's E_c
        // products in FP32, whose rounding lies orders below the tolerance
        const bool f32 = h->mixed && h->opt.coarse_tol >= kCoarseF32Tol;
        RTE_TRY(coarse_cg(h->stream, h->d, b, x, nrhs, h->opt.coarse_tol, h->opt.coarse_maxit,
                          h->cowork, h->cobytes, h->status, f32));
    }
    SolveStatus st;
    RTE_TRY(read_status(h, st));
    h->co_iters = st.iterations;
    return RTE_OK;
}

// z = P_1^l b (eq. applyP1).  Uses e5, e6 (and apply_E's buffers).
// E x for the inner steps: FP64, or FP32 with an FP64 interface in mixed modes
int apply_E_inner(rte_handle* h, const double* x, double* y, int nrhs, bool with_k) {
    if (!h->mixed) return apply_E(h, x, y, nrhs, with_k);
    const size_t n = (size_t)nrhs * h->d.nRp * h->d.nSp;
    convert(h->stream, x, h->f1, n);
    RTE_TRY(apply_E_lo(h, h->f1, h->f2, nrhs, with_k));
    convert(h->stream, h->f2, y, n);
    return RTE_OK;
}

// z = l steps of CG for E z = b preconditioned by E_0^{-1}, from z = 0
// (RTE_P1_PCG, Section 5.3).  Uses e5, e6, e9, e10 and sc[8n, 12n) (the
// (M^- - K^-) PCG inside the inner applies uses sc[0, 6n)); the per-RHS step
// lengths stay on the device.
int apply_P1_pcg(rte_handle* h, const double* b, double* z, int nrhs) {
    const DevSystem& d = h->d;
    const size_t len = (size_t)d.nRp * d.nSp;
    const int n = nrhs;
    cudaStream_t s = h->stream;
    double *R = h->e9, *P = h->e10, *Y = h->e6, *W = h->e5;
    double *rho = h->sc + 8 * n, *tmp = h->sc + 9 * n, *alpha = h->sc + 10 * n,
           *beta = h->sc + 11 * n;
    const unsigned rb = (unsigned)((n + 63) / 64);
    RTE_CUDA_TRY(cudaMemcpyAsync(R, b, sizeof(double) * n * len, cudaMemcpyDeviceToDevice, s));
    RTE_CUDA_TRY(cudaMemsetAsync(z, 0, sizeof(double) * n * len, s));
    RTE_TRY(e0_inv(h, R, Y, n));                       // y = E_0^{-1} r
    RTE_CUDA_TRY(cudaMemcpyAsync(P, Y, sizeof(double) * n * len, cudaMemcpyDeviceToDevice, s));
    dot_per_rhs(s, R, Y, len, n, h->partial, rho);     // rho = r.y
    for (int k = 0; k < h->opt.l; ++k) {
        RTE_TRY(apply_E_inner(h, P, W, n, false));     // w = E p
        {
            Scope sc(h, "axpy");
            dot_per_rhs(s, P, W, len, n, h->partial, tmp);
            k_ratio<<<rb, 64, 0, s>>>(rho, tmp, alpha, n, 1.0);   // alpha = rho / p.w
            count_launches(1);
            axpby_per_rhs(s, P, z, len, n, alpha, 0.0, nullptr, 1.0);   // z += alpha p
        }
        if (k + 1 == h->opt.l) break;
        {
            Scope sc(h, "axpy");
            k_ratio<<<rb, 64, 0, s>>>(rho, tmp, alpha, n, -1.0);
            count_launches(1);
            axpby_per_rhs(s, W, R, len, n, alpha, 0.0, nullptr, 1.0);   // r -= alpha w
        }
        RTE_TRY(e0_inv(h, R, Y, n));
        Scope sc(h, "axpy");
        dot_per_rhs(s, R, Y, len, n, h->partial, tmp);                  // r.y
        k_ratio<<<rb, 64, 0, s>>>(tmp, rho, beta, n, 1.0);             // beta = r.y / rho
        count_launches(1);
        RTE_CUDA_TRY(cudaMemcpyAsync(rho, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        axpby_per_rhs(s, Y, P, len, n, nullptr, 1.0, beta, 0.0);        // p = y + beta p
    }
    return RTE_OK;
}

int apply_P1(rte_handle* h, const double* b, double* z, int nrhs) {
    if (h->opt.p1_route == RTE_P1_PCG) return apply_P1_pcg(h, b, z, nrhs);
    const DevSystem& d = h->d;
    const size_t len = (size_t)d.nRp * d.nSp;
    RTE_TRY(e0_inv(h, b, z, nrhs));   // z_1 = E_0^{-1} b
    for (int k = 1; k < h->opt.l; ++k) {
        RTE_TRY(apply_E_inner(h, z, h->e5, nrhs, false));
        {
            Scope sc(h, "axpy");
            axpby_per_rhs(h->stream, b, h->e5, len, nrhs, nullptr, -1.0, nullptr, 1.0);
        }
        RTE_TRY(e0_inv(h, h->e5, h->e6, nrhs));
        Scope sc(h, "axpy");
        axpby_per_rhs(h->stream, h->e6, z, len, nrhs, nullptr, -1.0, nullptr, 1.0);
    }
    return RTE_OK;
}

// The restriction and prolongation of the coarse correction: one warp per
// row (d^+ <= 16), in FP32 products on mixed handles (a preconditioner step:
// its coarse solve stops at coarse_tol), in FP64 otherwise; the general
// FP64 GEMM for larger d^+.
int restrict_(rte_handle* h, const double* x, double* qc, int nrhs) {
    const DevSystem& d = h->d;
    Scope sc(h, "restrict");
    if (!restrict_rows(h->stream, nrhs * d.nRp, d.nSp, d.dP, x, d.WpN, h->mixed ? d.lo.WpN : nullptr,
                       qc))
        gemm_f64(h->stream, nrhs * d.nRp, d.dP, d.nSp, x, d.nSp, d.WpN, d.dP, qc, d.dP, 1.0, 0.0,
                 0, nullptr, nullptr, nullptr, 1);
    return RTE_OK;
}

int prolong_add(rte_handle* h, const double* uc, double* x, int nrhs, double beta) {
    const DevSystem& d = h->d;
    Scope sc(h, "prolong");
    if (!prolong_rows(h->stream, nrhs * d.nRp, d.nSp, d.dP, uc, d.WpNT,
                      h->mixed ? d.lo.WpNT : nullptr, x, beta))
        gemm_f64(h->stream, nrhs * d.nRp, d.nSp, d.dP, uc, d.dP, d.WpNT, d.nSp, x, d.nSp, 1.0,
                 beta, 0, nullptr, nullptr, nullptr, 1);
    return RTE_OK;
}

// s = P_2 P_1 r = P_1 r + W E_c^{-1} W^T (r - (E - K^+) P_1 r)   (eq. product_pre)
int precond(rte_handle* h, const double* r, double* s, int nrhs, bool p2) {
    const DevSystem& d = h->d;
    const size_t len = (size_t)d.nRp * d.nSp;
    RTE_TRY(apply_P1(h, r, s, nrhs));
    if (!p2 || d.dP == 0) return RTE_OK;
    RTE_TRY(apply_E_inner(h, s, h->e7, nrhs, true));
    {
        Scope sc(h, "axpy");   // e7 = r - (E - K^+) s
        axpby_per_rhs(h->stream, r, h->e7, len, nrhs, nullptr, 1.0, nullptr, -1.0);
    }
    RTE_TRY(restrict_(h, h->e7, h->c1, nrhs));   // -q_c = W^T (r - (E-K) s)
    RTE_TRY(coarse_inv(h, h->c1, h->c2, nrhs));  // -u_c
    // s <- s - W u_c, so that u_{n+1} = u_n - s = u_{n+1/2} + W u_c
    RTE_TRY(prolong_add(h, h->c2, s, nrhs, 1.0));
    return RTE_OK;
}

__global__ void k_neg(double* c, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) c[i] = -c[i];
}

bool bad(double v) { return !std::isfinite(v); }

}  // namespace

// ====================================================================== ABI
extern "C" {

const char* rte_last_error(void) { return rte::g_last_error.c_str(); }

int rte_default_options(rte_options* o) {
    if (!o) return fail(RTE_ERR_ARG, "opts is NULL");
    o->l = 0;                 // 0: per P_1 route (4 for P_1^l, 2 for the PCG steps)
    o->n_plus = 4;
    o->n_minus = 5;
    o->precision = RTE_FP64;
    o->mk_route = RTE_MK_EIGEN;
    o->mk_tol = 1e-12;
    o->mk_maxit = 500;
    o->e0_tol = 0.0;          // 0: per precision (1e-12 FP64, 0.3 mixed)
    o->e0_maxit = 20000;
    o->coarse_tol = 0.0;      // 0: per precision (1e-12 FP64, 0.3 mixed)
    o->coarse_maxit = 20000;
    o->max_iter = 200;
    o->max_rhs = 1;
    o->dgemm = RTE_DGEMM_AUTO;
    o->split_slices = 7;
    o->mg_sweeps = 2;
    o->autotune = 1;
    o->p1_route = RTE_P1_AUTO;   // P_1^l in FP64, PCG steps in the mixed modes
    o->e0_route = RTE_E0_AUTO;   // direct factorisation when the mesh allows it
    o->coarse_route = RTE_EC_AUTO;
    return RTE_OK;
}

int rte_setup(const rte_problem* prob, const rte_options* opts, void* stream,
              rte_handle** out) {
    if (!prob || !out) return fail(RTE_ERR_ARG, "NULL argument");
    *out = nullptr;
    rte_options o;
    if (opts) o = *opts; else rte_default_options(&o);
    if (o.l < 0 || o.n_minus < 1 || (o.n_minus % 2) == 0 || (o.n_plus >= 0 && o.n_plus % 2) ||
        o.max_rhs < 1 || o.mk_maxit < 1 || o.e0_maxit < 1 || o.coarse_maxit < 1)
        return fail(RTE_ERR_ARG, "invalid options (l >= 0, odd N^- >= 1, even N^+ or -1)");
    if (o.precision != RTE_FP64 && o.precision != RTE_MIXED_FP32 &&
        o.precision != RTE_MIXED_BF16)
        return fail(RTE_ERR_ARG, "unknown precision mode");
    if (o.p1_route != RTE_P1_AUTO && o.p1_route != RTE_P1_RICHARDSON &&
        o.p1_route != RTE_P1_PCG)
        return fail(RTE_ERR_ARG, "unknown P_1 route");
    if (o.p1_route == RTE_P1_AUTO)
        o.p1_route = o.precision == RTE_FP64 ? RTE_P1_RICHARDSON : RTE_P1_PCG;
    // l = 0: the paper's 4 Richardson steps for P_1^l; 2 conjugate-gradient
    // steps for the PCG route (measured on the 128 x 128 / 512-triangle
    // workload: 16 outer iterations with l = 2, 3, 4 and 6 alike, so two
    // steps take the least time; 2 and 4 within 8 % on the 96 x 96 /
    // 2048-triangle cases)
    if (o.l == 0) o.l = o.p1_route == RTE_P1_PCG ? 2 : 4;
    if (o.e0_route != RTE_E0_AUTO && o.e0_route != RTE_E0_DIRECT &&
        o.e0_route != RTE_E0_MULTIGRID)
        return fail(RTE_ERR_ARG, "unknown E_0 route");
    if (o.e0_route == RTE_E0_DIRECT && !e0_direct_fits(prob->mesh_m))
        return fail(RTE_ERR_ARG, "the direct E_0 route needs mesh_m <= 156");
    if (o.e0_route == RTE_E0_AUTO)
        o.e0_route = e0_direct_fits(prob->mesh_m) ? RTE_E0_DIRECT : RTE_E0_MULTIGRID;
    if (o.coarse_route != RTE_EC_AUTO && o.coarse_route != RTE_EC_DIRECT &&
        o.coarse_route != RTE_EC_MULTIGRID)
        return fail(RTE_ERR_ARG, "unknown coarse route");
    {
        const int dPo = o.n_plus >= 0 ? (o.n_plus + 1) * (o.n_plus + 2) / 2 : 0;
        if (o.coarse_route == RTE_EC_DIRECT && dPo > 0 && !ec_direct_fits(prob->mesh_m, dPo))
            return fail(RTE_ERR_ARG, "the direct coarse route needs (mesh_m + 1) d^+ <= 2400");
        // measured on the 128 x 128 / 512-triangle workload: a coarse solve
        // takes 4.1 ms on the multigrid route (11 CG iterations to 0.1) and
        // 9.9 ms on the direct route (one CG iteration, 514 grid-wide phases
        // of its sweeps), whose FP64 set-up adds 3.6 s: multigrid by default
        if (o.coarse_route == RTE_EC_AUTO) o.coarse_route = RTE_EC_MULTIGRID;
    }
    if (o.mk_route != RTE_MK_EIGEN && o.mk_route != RTE_MK_PCG)
        return fail(RTE_ERR_ARG, "unknown (M^- - K^-)^{-1} route");
    // inner tolerances left at 0 follow the precision mode: the plain FP64
    // method solves E_0 and E_c to 1e-12; under the mixed modes' FP64 outer
    // residual (iterative refinement) loose inner solves cost at most a few
    // outer iterations and save more inner work than those cost (E_0 to 0.3
    // and E_c to 0.3: the same outer iteration counts as 0.1 on the
    // benchmark and the 96 x 96 / 2048-triangle cases, and the least time)
    if (!(o.e0_tol > 0)) o.e0_tol = o.precision == RTE_FP64 ? 1e-12 : 0.3;
    if (!(o.coarse_tol > 0)) o.coarse_tol = o.precision == RTE_FP64 ? 1e-12 : 0.3;
    SetupClock clk{nullptr};
    HostSystem hs;
    RTE_TRY(build_host_system(*prob, o, hs));
    RTE_TRY(check_device_memory(*prob, o));
    rte_handle* h = new rte_handle();
    h->opt = o;
    h->stream = (cudaStream_t)stream;
    keep_pool_memory();
    clk.h = h;
    clk.mark("host assembly");
    auto bail = [&](int rc) {
        rte_destroy(h);
        return rc;
    };
    DevSystem& d = h->d;
    d.e0_direct = o.e0_route == RTE_E0_DIRECT;
    d.ec_direct = o.coarse_route == RTE_EC_DIRECT;
    d.m = hs.m;
    d.nRp = hs.nRp; d.nRm = hs.nRm; d.nSp = hs.nSp; d.nSm = hs.nSm;
    d.dP = hs.dP; d.dM = hs.dM; d.nnz = (int)hs.st.col.size();
    d.g = hs.g; d.c = hs.c; d.gamma = hs.gamma;
    int rc = RTE_OK;
#define UP(dst, src) do { rc = upload(h, &d.dst, src); if (rc) return bail(rc); } while (0)
    UP(cell_nodes, hs.mesh.cell_nodes);
    UP(cell_D, hs.cell_D);
    UP(cell_at, hs.cell_at);
    UP(cell_as, hs.cell_as);
    UP(adj_ptr, hs.adj_ptr);
    UP(adj_cell, hs.adj_cell);
    UP(adj_loc, hs.adj_loc);
    UP(st_ptr, hs.st.ptr);
    UP(st_col, hs.st.col);
    UP(st_diag, hs.st.diag);
    UP(sval, hs.sval);
    std::vector<double> ell4;
    {
        MGHostLevel L;
        L.m = hs.m;
        L.st = hs.st;
        const size_t nnz = hs.st.col.size();
        const int slots[4] = {kMt, kMs, kBx, kBy};
        L.vals.resize(4 * nnz);
        for (int q = 0; q < 4; ++q)
            std::copy(hs.sval.begin() + (size_t)slots[q] * nnz,
                      hs.sval.begin() + (size_t)(slots[q] + 1) * nnz, L.vals.begin() + q * nnz);
        rc = to_ell(L, 4, 1, ell4);
        if (rc) return bail(rc);
    }
    UP(ell4, ell4);
    UP(ang_m, hs.m_);
    UP(ang_omx, hs.omx);
    UP(ang_omy, hs.omy);
    UP(ang_A1, hs.A1);
    UP(ang_A2, hs.A2);
    UP(ang_MSm, hs.MSm);
    UP(ang_MSm_inv, hs.MSm_inv);
    UP(e0s, hs.e0s);
    {
        // which triangle of each pair enters through each face (x = 0, x = 1,
        // y = 0, y = 1; outward normals -e_x, e_x, -e_y, e_y): the one whose
        // direction has s.n < 0, read from the sign of its vertex sum
        std::vector<int> half((size_t)4 * hs.nSp);
        for (int k = 0; k < hs.nSp; ++k) {
            double c[2] = {0.0, 0.0};
            for (int v = 0; v < 3; ++v)
                for (int a = 0; a < 2; ++a) c[a] += hs.sphere.verts[3 * hs.sphere.tri[3 * k + v] + a];
            for (int f = 0; f < 4; ++f) {
                const double sn = (f % 2 == 0 ? -1.0 : 1.0) * c[f / 2];
                half[(size_t)f * hs.nSp + k] = sn < 0.0 ? 0 : 1;
            }
        }
        UP(inflow_half, half);
    }
    // ------------------------------------------------ S^+ and S^- (device)
    const int n = hs.nSp, nm = hs.nSm;
    QuadDev q{};
    {
        double *sp = nullptr, *sm = nullptr;
        rc = dalloc(h, &sp, (size_t)n * n); if (rc) return bail(rc);
        rc = dalloc(h, &sm, (size_t)nm * nm); if (rc) return bail(rc);
        d.Sp = sp;
        d.Sm = sm;
    }
    {
        const double *a, *b, *c, *e, *f, *g2;
        const int *pi, *ii;
        rc = upload(h, &a, hs.quad_near_pts); if (rc) return bail(rc);
        rc = upload(h, &b, hs.quad_near_w); if (rc) return bail(rc);
        rc = upload(h, &c, hs.quad_near_psi); if (rc) return bail(rc);
        rc = upload(h, &e, hs.quad_far_pts); if (rc) return bail(rc);
        rc = upload(h, &f, hs.quad_far_w); if (rc) return bail(rc);
        rc = upload(h, &g2, hs.quad_far_psi); if (rc) return bail(rc);
        rc = upload(h, &pi, hs.near_ptr); if (rc) return bail(rc);
        rc = upload(h, &ii, hs.near_idx); if (rc) return bail(rc);
        q = QuadDev{a, b, c, e, f, g2, pi, ii, 1 << (2 * kRNear), 1 << (2 * kRFar)};
    }
    assemble_scattering(h->stream, n, hs.g, q, const_cast<double*>(d.Sp),
                        const_cast<double*>(d.Sm));
    h->h_Sp.resize((size_t)n * n);
    h->h_Sm.resize((size_t)nm * nm);
    if (cudaMemcpyAsync(h->h_Sp.data(), d.Sp, sizeof(double) * n * n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->h_Sm.data(), d.Sm, sizeof(double) * (size_t)nm * nm, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return bail(fail(RTE_ERR_CUDA, "scattering assembly failed"));
    h->h_m = hs.m_; h->h_MSm = hs.MSm; h->h_A1 = hs.A1; h->h_A2 = hs.A2;
    h->h_omx = hs.omx; h->h_omy = hs.omy;

    clk.mark("uploads and scattering matrices");
    // --------------------------------------- eigenpairs of (S^+, M_S^+)
    std::vector<double> C((size_t)n * n), w;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            C[(size_t)i * n + j] = h->h_Sp[(size_t)i * n + j] / std::sqrt(hs.m_[i] * hs.m_[j]);
    rc = sym_eig(h, C, w, n);
    if (rc) return bail(rc);
    // eigenvector t (ascending) is row t of C; reorder non-increasing
    h->h_lamP.resize(n);
    std::vector<double> WpFull((size_t)n * n);
    for (int t = 0; t < n; ++t) {
        const int src = n - 1 - t;
        h->h_lamP[t] = w[src];
        for (int k = 0; k < n; ++k)
            WpFull[(size_t)k * n + t] = C[(size_t)src * n + k] / std::sqrt(hs.m_[k]);
    }
    const int dP = hs.dP;
    h->h_WpN.assign((size_t)n * std::max(dP, 1), 0.0);
    std::vector<double> WpNT((size_t)std::max(dP, 1) * n, 0.0);
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < dP; ++a) {
            h->h_WpN[(size_t)k * dP + a] = WpFull[(size_t)k * n + a];
            WpNT[(size_t)a * n + k] = WpFull[(size_t)k * n + a];
        }
    UP(WpN, h->h_WpN);
    UP(WpNT, WpNT);
    UP(lamP, h->h_lamP);

    clk.mark("eigenpairs of S+");
    // --------------------------------------- eigenpairs of (S^-, M_S^-)
    // M_S^- = L L^T blockwise; C = L^{-1} S^- L^{-T}; W = L^{-T} Q
    std::vector<double> Linv((size_t)9 * n);
    for (int k = 0; k < n; ++k) {
        double L[9];
        if (!chol3(&hs.MSm[9 * k], L)) return bail(fail(RTE_ERR_ARG, "odd mass not SPD"));
        inv_lower3(L, &Linv[9 * k]);
    }
    std::vector<double> Cm((size_t)nm * nm);
    for (int K1 = 0; K1 < n; ++K1)
        for (int K2 = 0; K2 < n; ++K2) {
            const double* Li = &Linv[9 * K1];
            const double* Lj = &Linv[9 * K2];
            double T[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k)
                        s += Li[3 * i + k] * h->h_Sm[(size_t)(3 * K1 + k) * nm + 3 * K2 + j];
                    T[3 * i + j] = s;
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += T[3 * i + k] * Lj[3 * j + k];
                    Cm[(size_t)(3 * K1 + i) * nm + 3 * K2 + j] = s;
                }
        }
    std::vector<double> wm;
    rc = sym_eig(h, Cm, wm, nm);
    if (rc) return bail(rc);
    h->h_lamM.resize(nm);
    std::vector<double> Vm((size_t)nm * nm), VmT((size_t)nm * nm);
    for (int t = 0; t < nm; ++t) {
        const int src = nm - 1 - t;
        h->h_lamM[t] = wm[src];
        const double* qv = &Cm[(size_t)src * nm];
        for (int K1 = 0; K1 < n; ++K1) {
            const double* Li = &Linv[9 * K1];
            for (int i = 0; i < 3; ++i) {
                // (L^{-T} q)_i = sum_k Linv[k][i] q_k
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += Li[3 * k + i] * qv[3 * K1 + k];
                Vm[(size_t)(3 * K1 + i) * nm + t] = s;
                VmT[(size_t)t * nm + 3 * K1 + i] = s;
            }
        }
    }
    const int dM = hs.dM;
    std::vector<double> WmN((size_t)nm * dM), WmNT((size_t)dM * nm);
    for (int r = 0; r < nm; ++r)
        for (int a = 0; a < dM; ++a) {
            WmN[(size_t)r * dM + a] = Vm[(size_t)r * nm + a];
            WmNT[(size_t)a * nm + r] = Vm[(size_t)r * nm + a];
        }
    UP(Vm, Vm);
    UP(VmT, VmT);
    UP(lamM, h->h_lamM);
    UP(WmN, WmN);
    UP(WmNT, WmNT);

    clk.mark("eigenpairs of S-");
    // ------------------------------- coarse matrix E_c = W^T (E - K^+) W
    if (dP > 0) {
        const int nnz = d.nnz;
        const int dd = dP * dP;
        h->h_ec.assign((size_t)nnz * dd, 0.0);
        const double* Mt = &hs.sval[(size_t)kMt * nnz];
        const double* Ms = &hs.sval[(size_t)kMs * nnz];
        const double* Bx = &hs.sval[(size_t)kBx * nnz];
        const double* By = &hs.sval[(size_t)kBy * nnz];
        std::vector<double> Ox(dd, 0.0), Oy(dd, 0.0);
        for (int a = 0; a < dP; ++a)
            for (int b = 0; b < dP; ++b)
                for (int k = 0; k < n; ++k) {
                    const double ww = h->h_WpN[(size_t)k * dP + a] * h->h_WpN[(size_t)k * dP + b];
                    Ox[a * dP + b] += hs.omx[k] * ww;
                    Oy[a * dP + b] += hs.omy[k] * ww;
                }
        for (int p = 0; p < nnz; ++p) {
            double* blk = &h->h_ec[(size_t)p * dd];
            for (int a = 0; a < dP; ++a) {
                blk[a * dP + a] += Mt[p] - h->h_lamP[a] * Ms[p];
                for (int b = 0; b < dP; ++b)
                    blk[a * dP + b] += Bx[p] * Ox[a * dP + b] + By[p] * Oy[a * dP + b];
            }
        }
        // transport block: G_n = V^T (A_n W_N)  (n_S^- x dP) for n = 1, 2
        std::vector<double> G((size_t)2 * nm * dP, 0.0);
        for (int nn = 0; nn < 2; ++nn) {
            const std::vector<double>& An = nn == 0 ? hs.A1 : hs.A2;
            for (int lam = 0; lam < nm; ++lam) {
                double* g = &G[((size_t)nn * nm + lam) * dP];
                for (int K1 = 0; K1 < n; ++K1)
                    for (int c = 0; c < 3; ++c) {
                        const double v = Vm[(size_t)(3 * K1 + c) * nm + lam] * An[3 * K1 + c];
                        if (v == 0.0) continue;
                        const double* wrow = &h->h_WpN[(size_t)K1 * dP];
                        for (int a = 0; a < dP; ++a) g[a] += v * wrow[a];
                    }
            }
        }
        // H(sigma_t, sigma_s) per class of cells, (2 dP)^2 entries
        std::map<std::pair<double, double>, std::vector<double>> Hc;
        const int d2 = 2 * dP;
        for (int j = 0; j < hs.nRm; ++j) {
            const double st = prob->sigma_t[j], ss = prob->sigma_s[j];
            auto key = std::make_pair(st, ss);
            if (Hc.count(key)) continue;
            std::vector<double> H((size_t)d2 * d2, 0.0);
            for (int lam = 0; lam < nm; ++lam) {
                const double f = 1.0 / (st - h->h_lamM[lam] * ss);
                for (int x = 0; x < d2; ++x) {
                    const double gx = G[((size_t)(x / dP) * nm + lam) * dP + x % dP] * f;
                    if (gx == 0.0) continue;
                    for (int y = 0; y < d2; ++y)
                        H[(size_t)x * d2 + y] += gx * G[((size_t)(y / dP) * nm + lam) * dP + y % dP];
                }
            }
            Hc[key] = std::move(H);
        }
        for (int j = 0; j < hs.nRm; ++j) {
            const std::vector<double>& H = Hc[std::make_pair(prob->sigma_t[j], prob->sigma_s[j])];
            const double A = hs.mesh.area[j];
            const int* nd = &hs.mesh.cell_nodes[3 * j];
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) {
                    const int row = nd[al], col = nd[be];
                    const int* bgn = hs.st.col.data() + hs.st.ptr[row];
                    const int* end = hs.st.col.data() + hs.st.ptr[row + 1];
                    const int pos = (int)(std::lower_bound(bgn, end, col) - hs.st.col.data());
                    double* blk = &h->h_ec[(size_t)pos * dd];
                    const double D[2][2] = {{hs.cell_D[6 * j + al], hs.cell_D[6 * j + 3 + al]},
                                            {hs.cell_D[6 * j + be], hs.cell_D[6 * j + 3 + be]}};
                    for (int nn = 0; nn < 2; ++nn)
                        for (int mm = 0; mm < 2; ++mm) {
                            const double fac = D[0][nn] * D[1][mm] / A;
                            for (int a = 0; a < dP; ++a)
                                for (int b = 0; b < dP; ++b)
                                    blk[a * dP + b] += fac * H[(size_t)(nn * dP + a) * d2 + mm * dP + b];
                        }
                }
        }
        std::vector<double> dinv((size_t)hs.nRp * dd);
        for (int i = 0; i < hs.nRp; ++i)
            if (!chol_inv_sym(dP, &h->h_ec[(size_t)hs.st.diag[i] * dd], &dinv[(size_t)i * dd]))
                return bail(fail(RTE_ERR_ARG, "singular coarse diagonal block"));
        UP(ec_val, h->h_ec);
        UP(ec_dinv, dinv);
        // Kronecker form of the same E_c for the multigrid levels: the mass,
        // scattering and boundary terms and, per sigma class, the four
        // transport terms D_n^T X D_m (x) H_c[n][m]
        const int nclass = (int)Hc.size();
        const int Q = 4 + 4 * nclass;
        if (Q <= kEcMaxTerms && dP <= 16) {
            std::map<std::pair<double, double>, int> cls;
            for (const auto& kv : Hc) cls.emplace(kv.first, (int)cls.size());
            std::vector<double> S((size_t)Q * nnz, 0.0), Gq((size_t)Q * dd, 0.0);
            std::copy(Mt, Mt + nnz, S.begin());
            std::copy(Ms, Ms + nnz, S.begin() + nnz);
            std::copy(Bx, Bx + nnz, S.begin() + 2 * (size_t)nnz);
            std::copy(By, By + nnz, S.begin() + 3 * (size_t)nnz);
            for (int a = 0; a < dP; ++a) {
                Gq[(size_t)a * dP + a] = 1.0;
                Gq[dd + (size_t)a * dP + a] = -h->h_lamP[a];
            }
            std::copy(Ox.begin(), Ox.end(), Gq.begin() + 2 * (size_t)dd);
            std::copy(Oy.begin(), Oy.end(), Gq.begin() + 3 * (size_t)dd);
            for (const auto& kv : Hc) {
                const int c = cls[kv.first];
                for (int nn = 0; nn < 2; ++nn)
                    for (int mm = 0; mm < 2; ++mm)
                        for (int a = 0; a < dP; ++a)
                            for (int b = 0; b < dP; ++b)
                                Gq[(size_t)(4 + 4 * c + 2 * nn + mm) * dd + a * dP + b] =
                                    kv.second[(size_t)(nn * dP + a) * d2 + mm * dP + b];
            }
            for (int j = 0; j < hs.nRm; ++j) {
                const int c = cls[std::make_pair(prob->sigma_t[j], prob->sigma_s[j])];
                const double A = hs.mesh.area[j];
                const int* nd = &hs.mesh.cell_nodes[3 * j];
                for (int al = 0; al < 3; ++al)
                    for (int be = 0; be < 3; ++be) {
                        const int row = nd[al], col = nd[be];
                        const int* bgn = hs.st.col.data() + hs.st.ptr[row];
                        const int* end = hs.st.col.data() + hs.st.ptr[row + 1];
                        const int pos = (int)(std::lower_bound(bgn, end, col) - hs.st.col.data());
                        const double D[2][2] = {{hs.cell_D[6 * j + al], hs.cell_D[6 * j + 3 + al]},
                                                {hs.cell_D[6 * j + be], hs.cell_D[6 * j + 3 + be]}};
                        for (int nn = 0; nn < 2; ++nn)
                            for (int mm = 0; mm < 2; ++mm)
                                S[(size_t)(4 + 4 * c + 2 * nn + mm) * nnz + pos] +=
                                    D[0][nn] * D[1][mm] / A;
                    }
            }
            // the two forms must agree: sum_q S_q G_q against the blocks
            double diff = 0.0, scale = 0.0;
            for (int p = 0; p < nnz; ++p)
                for (int t = 0; t < dd; ++t) {
                    double v = 0.0;
                    for (int q = 0; q < Q; ++q) v += S[(size_t)q * nnz + p] * Gq[(size_t)q * dd + t];
                    diff = std::max(diff, std::fabs(v - h->h_ec[(size_t)p * dd + t]));
                    scale = std::max(scale, std::fabs(h->h_ec[(size_t)p * dd + t]));
                }
            if (diff <= 1e-10 * scale) {
                h->ec_Q = Q;
                h->h_ecS.swap(S);
                h->h_ecG.swap(Gq);
            }
        }
    }
    if (o.precision != RTE_FP64) {
        h->mixed = true;
        DevLow& lo = d.lo;
        lo.bf16 = o.precision == RTE_MIXED_BF16;
        auto tof = [](const std::vector<double>& v) {
            return std::vector<float>(v.begin(), v.end());
        };
#define UPF(dst, src) do { rc = upload(h, &lo.dst, tof(src)); if (rc) return bail(rc); } while (0)
        UPF(ell4, ell4);
        UPF(cell_D, hs.cell_D);
        UPF(cell_at, hs.cell_at);
        UPF(cell_as, hs.cell_as);
        UPF(sval, hs.sval);
        UPF(m, hs.m_);
        UPF(omx, hs.omx);
        UPF(omy, hs.omy);
        UPF(A1, hs.A1);
        UPF(A2, hs.A2);
        UPF(e0s, hs.e0s);
        UPF(lamM, h->h_lamM);
        UPF(WpN, h->h_WpN);
        {
            std::vector<double> wt((size_t)std::max(dP, 1) * n, 0.0);
            for (int k = 0; k < n; ++k)
                for (int a = 0; a < dP; ++a) wt[(size_t)a * n + k] = h->h_WpN[(size_t)k * dP + a];
            UPF(WpNT, wt);
        }
#undef UPF
        // GEMM second operands, K-major: GEMM 1 multiplies by V (needs V^T),
        // GEMM 2 by V^T (needs V), the scattering product by S^+ = (S^+)^T
        const std::vector<double>* srcs[3] = {&VmT, &Vm, &h->h_Sp};
        const void** dsts[3] = {&lo.VmT, &lo.Vm, &lo.Sp};
        for (int t = 0; t < 3; ++t) {
            const std::vector<double>& v = *srcs[t];
            if (lo.bf16) {
                std::vector<__nv_bfloat16> b(v.size());
                for (size_t i = 0; i < v.size(); ++i) b[i] = __float2bfloat16_rn((float)v[i]);
                const __nv_bfloat16* p = nullptr;
                rc = upload(h, &p, b); if (rc) return bail(rc);
                *dsts[t] = p;
            } else {
                const float* p = nullptr;
                rc = upload(h, &p, tof(v)); if (rc) return bail(rc);
                *dsts[t] = p;
            }
        }
    }
    clk.mark("coarse matrix and low-precision operands");
    // ---------------------------------------- split FP64 GEMM operands
    {
        const bool split = o.dgemm == RTE_DGEMM_SPLIT ||
                           (o.dgemm == RTE_DGEMM_AUTO && o.precision != RTE_FP64);
        if (split) {
            if (o.split_slices < 1 || o.split_slices > 9)
                return bail(fail(RTE_ERR_ARG, "split_slices must be in [1, 9]"));
            d.split_S = o.split_slices;
            struct Src { const double* m; int rows, K; const void** sl; const int** ex; };
            Src srcs[4] = {{d.VmT, nm, nm, &d.sl_VmT, &d.ex_VmT},
                           {d.Vm, nm, nm, &d.sl_Vm, &d.ex_Vm},
                           {d.Sp, n, n, &d.sl_Sp, &d.ex_Sp},
                           {d.Sm, nm, nm, &d.sl_Sm, &d.ex_Sm}};
            for (auto& sr : srcs) {
                // S^- is needed as a GEMM operand only by the PCG route
                if (sr.m == d.Sm && o.mk_route != RTE_MK_PCG) continue;
                char* p = nullptr;
                rc = dalloc(h, &p, ozaki_slice_bytes(sr.rows, sr.K, d.split_S));
                if (rc) return bail(rc);
                int* ex = nullptr;
                rc = ozaki_split(h->stream, sr.m, sr.rows, sr.K, d.split_S, p, &ex);
                if (rc) return bail(rc);
                *sr.sl = p;
                *sr.ex = ex;
            }
            if (o.mk_route != RTE_MK_PCG) {
                // the eigenbasis route's diagonal 1 / (at - lam as), per cell
                // and eigenvalue, for the first contraction's epilogue
                double* t = nullptr;
                rc = dalloc(h, &t, (size_t)d.nRm * nm);
                if (rc) return bail(rc);
                rc = ozaki_recip_table(h->stream, d.cell_at, d.cell_as, d.lamM, d.nRm, nm, t);
                if (rc) return bail(rc);
                d.mk_rinv = t;
            }
        }
    }
#undef UP
    clk.mark("split FP64 operands");
    rc = setup_multigrid(h, hs, &clk);
    if (rc) return bail(rc);
    clk.mark(d.ec_direct ? "E_c factorisation" : "E_c multigrid");
    rc = alloc_workspace(h, o.max_rhs);
    if (rc) return bail(rc);
    clk.mark("workspace");
    rc = tune_launches(h);
    if (rc) return bail(rc);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(fail(RTE_ERR_CUDA, "setup synchronisation failed"));
    clk.mark("launch tuning");
    *out = h;
    return RTE_OK;
}

int rte_setup_times(const rte_handle* h, const char** names, double* ms, int cap,
                    int* count) {
    if (!h || !count || cap < 0) return fail(RTE_ERR_ARG, "bad argument");
    const int n = (int)h->setup_ms.size();
    *count = n;
    for (int i = 0; i < n && i < cap; ++i) {
        if (names) names[i] = h->setup_names[i].c_str();
        if (ms) ms[i] = h->setup_ms[i];
    }
    return RTE_OK;
}

int rte_sizes(const rte_handle* h, int* n_nodes, int* n_cells, int* n_dirs, int* n_odd,
              int* d_plus, int* d_minus) {
    if (!h) return fail(RTE_ERR_ARG, "NULL handle");
    if (n_nodes) *n_nodes = h->d.nRp;
    if (n_cells) *n_cells = h->d.nRm;
    if (n_dirs) *n_dirs = h->d.nSp;
    if (n_odd) *n_odd = h->d.nSm;
    if (d_plus) *d_plus = h->d.dP;
    if (d_minus) *d_minus = h->d.dM;
    return RTE_OK;
}

int rte_rhs(rte_handle* h, const double* q_nodal, double* q, int nrhs) {
    if (!h || !q_nodal || !q || nrhs < 1) return fail(RTE_ERR_ARG, "bad argument");
    Scope sc(h, "rhs");
    rhs_source(h->stream, h->d, q_nodal, q, nrhs);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int rte_set_stream(rte_handle* h, void* stream) {
    if (!h) return fail(RTE_ERR_ARG, "NULL handle");
    flush_timers(h);
    h->stream = (cudaStream_t)stream;
    return RTE_OK;
}

int rte_inflow(rte_handle* h, const double* g, double* q, int nrhs) {
    if (!h || !g || !q || nrhs < 1) return fail(RTE_ERR_ARG, "bad argument");
    Scope sc(h, "inflow");
    inflow_source(h->stream, h->d, g, q, nrhs);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int rte_apply(rte_handle* h, const double* x, double* y, int nrhs) {
    if (!h || !x || !y || nrhs < 1) return fail(RTE_ERR_ARG, "bad argument");
    RTE_TRY(ensure_workspace(h, nrhs));
    RTE_TRY(apply_E(h, x, y, nrhs, true));
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int rte_precond(rte_handle* h, const double* r, double* s, int nrhs, int with_p2) {
    if (!h || !r || !s || nrhs < 1) return fail(RTE_ERR_ARG, "bad argument");
    RTE_TRY(ensure_workspace(h, nrhs));
    RTE_TRY(precond(h, r, s, nrhs, with_p2 != 0));
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

int rte_operator(rte_handle* h, int op, const double* in, double* out, int nrhs) {
    if (!h || !in || !out || nrhs < 1) return fail(RTE_ERR_ARG, "bad argument");
    RTE_TRY(ensure_workspace(h, nrhs));
    const DevSystem& d = h->d;
    cudaStream_t s = h->stream;
    const size_t no = (size_t)nrhs * d.nRm * d.nSm;
    switch (op) {
        case RTE_OP_A: apply_A(s, d, in, out, nrhs); break;
        case RTE_OP_AT: apply_even(s, d, in, nullptr, nullptr, out, nrhs, 1); break;
        case RTE_OP_KPLUS:
            gemm_f64(s, nrhs * d.nRp, d.nSp, d.nSp, in, d.nSp, d.Sp, d.nSp, h->e8, d.nSp, 1.0,
                     0.0, 0, nullptr, nullptr, nullptr, 1);
            apply_even(s, d, nullptr, h->e8, h->e8, out, nrhs, 4);
            k_neg<<<(unsigned)((nrhs * (size_t)d.nRp * d.nSp + 255) / 256), 256, 0, s>>>(
                out, (size_t)nrhs * d.nRp * d.nSp);
            count_launches(1);
            break;
        case RTE_OP_MK: RTE_TRY(mk_apply(h, in, out, h->z4, nrhs)); break;
        case RTE_OP_MK_INV:
            RTE_CUDA_TRY(cudaMemcpyAsync(h->z1, in, no * 8, cudaMemcpyDeviceToDevice, s));
            RTE_TRY(mk_inv(h, h->z1, h->z2, nrhs));
            RTE_CUDA_TRY(cudaMemcpyAsync(out, h->z2, no * 8, cudaMemcpyDeviceToDevice, s));
            break;
        case RTE_OP_MK_PREC: RTE_TRY(mk_prec(h, in, out, h->z4, nrhs)); break;
        case RTE_OP_E: RTE_TRY(apply_E(h, in, out, nrhs, false)); break;
        case RTE_OP_E0_INV:
            RTE_TRY(e0_inv(h, in, out, nrhs));
            if (d.e0_direct) RTE_TRY(e0_direct_error(s));
            break;
        case RTE_OP_P1: RTE_TRY(apply_P1(h, in, out, nrhs)); break;
        case RTE_OP_RESTRICT: RTE_TRY(restrict_(h, in, out, nrhs)); break;
        case RTE_OP_PROLONG: RTE_TRY(prolong_add(h, in, out, nrhs, 0.0)); break;
        case RTE_OP_EC: coarse_apply(s, d, in, out, nrhs); break;
        case RTE_OP_EC_INV: RTE_TRY(coarse_inv(h, in, out, nrhs)); break;
        case RTE_OP_E_LO:
        case RTE_OP_EK_LO:
            if (!h->mixed) return fail(RTE_ERR_ARG, "handle was set up in FP64 mode");
            RTE_TRY(apply_E_inner(h, in, out, nrhs, op == RTE_OP_EK_LO));
            RTE_TRY(tc_gemm_error(s));
            break;
        default: return fail(RTE_ERR_ARG, "unknown operator id");
    }
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

namespace {

// ||x||_2 of one even vector (device reduction, host result)
int norm2(rte_handle* h, const double* x, double* out) {
    const size_t len = (size_t)h->d.nRp * h->d.nSp;
    dot_per_rhs(h->stream, x, x, len, 1, h->partial, h->sc);
    double v = 0.0;
    RTE_CUDA_TRY(cudaMemcpyAsync(&v, h->sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    *out = std::sqrt(std::max(v, 0.0));
    return RTE_OK;
}

// One power-iteration step: x <- y / ||y||; returns ||y|| / ||x|| (x is a
// unit vector on entry).
int power_step(rte_handle* h, double* x, const double* y, double* ratio) {
    const size_t len = (size_t)h->d.nRp * h->d.nSp;
    double ny = 0.0;
    RTE_TRY(norm2(h, y, &ny));
    *ratio = ny;
    if (!(ny > 0.0)) return RTE_OK;
    axpby_per_rhs(h->stream, y, x, len, 1, nullptr, 1.0 / ny, nullptr, 0.0);
    return RTE_OK;
}

}  // namespace

int rte_rates(rte_handle* h, int maxit, double tol, unsigned long long seed, double* rho,
              double* eta, int* iters) {
    if (!h || maxit < 1 || !(tol >= 0) || (!rho && !eta)) return fail(RTE_ERR_ARG, "bad argument");
    if (h->opt.p1_route != RTE_P1_RICHARDSON)
        return fail(RTE_ERR_ARG, "rates need the stationary P_1^l (RTE_P1_RICHARDSON)");
    const DevSystem& d = h->d;
    cudaStream_t s = h->stream;
    const size_t len = (size_t)d.nRp * d.nSp;
    double* x = h->e1;
    double* y = h->e2;
    double* t = h->e3;
    double* w = h->e4;
    int used = 0;
    auto start = [&](unsigned long long sd) -> int {
        fill_uniform(s, x, len, sd);
        double nx = 0.0;
        RTE_TRY(norm2(h, x, &nx));
        axpby_per_rhs(s, x, x, len, 1, nullptr, 1.0 / nx, nullptr, 0.0);
        return RTE_OK;
    };
    if (rho) {
        // T x = x - P_2 P_1 (E - K^+) x, the iteration matrix of Algorithm 3
        RTE_TRY(start(seed));
        double prev = 0.0, cur = 0.0;
        int k = 0;
        for (; k < maxit; ++k) {
            RTE_TRY(apply_E(h, x, y, 1, true));
            RTE_TRY(precond(h, y, t, 1, true));
            axpby_per_rhs(s, x, t, len, 1, nullptr, 1.0, nullptr, -1.0);   // t = x - P y
            RTE_TRY(power_step(h, x, t, &cur));
            if (k > 0 && std::fabs(cur - prev) <= tol * cur) { ++k; break; }
            prev = cur;
        }
        *rho = cur;
        used = std::max(used, k);
    }
    if (eta && d.dP > 0) {
        // eta^2 = largest eigenvalue of (I - P_1 A)(I - P_G)(I - P_1 A), A = E - K^+,
        // P_G = W E_c^{-1} W^T A (the A-orthogonal projection onto span W)
        RTE_TRY(start(seed ^ 0x5851F42D4C957F2Dull));
        double prev = 0.0, cur = 0.0;
        int k = 0;
        auto one_minus_p1a = [&](const double* in, double* out) -> int {   // out = in - P_1 A in
            RTE_TRY(apply_E(h, in, y, 1, true));
            RTE_TRY(apply_P1(h, y, out, 1));
            axpby_per_rhs(s, in, out, len, 1, nullptr, 1.0, nullptr, -1.0);
            return RTE_OK;
        };
        for (; k < maxit; ++k) {
            RTE_TRY(one_minus_p1a(x, t));                                   // t = (I - P_1 A) x
            RTE_TRY(apply_E(h, t, y, 1, true));                             // y = A t
            RTE_TRY(restrict_(h, y, h->c1, 1));
            RTE_TRY(coarse_inv(h, h->c1, h->c2, 1));
            axpby_per_rhs(s, nullptr, h->c2, (size_t)d.nRp * d.dP, 1, nullptr, 0.0, nullptr, -1.0);
            RTE_TRY(prolong_add(h, h->c2, t, 1, 1.0));                     // t -= W E_c^{-1} W^T A t
            RTE_TRY(one_minus_p1a(t, w));                                   // w = (I - P_1 A) t
            RTE_TRY(power_step(h, x, w, &cur));
            if (k > 0 && std::fabs(cur - prev) <= tol * cur) { ++k; break; }
            prev = cur;
        }
        *eta = std::sqrt(std::max(cur, 0.0));
        used = std::max(used, k);
    } else if (eta) {
        *eta = 0.0;
    }
    if (iters) *iters = used;
    RTE_CUDA_TRY(cudaGetLastError());
    return tc_gemm_error(s);
}

int rte_odd(rte_handle* h, const double* u_plus, const double* l_minus, double* u_minus,
            int nrhs) {
    if (!h || !u_plus || !u_minus || nrhs < 1) return fail(RTE_ERR_ARG, "bad argument");
    RTE_TRY(ensure_workspace(h, nrhs));
    const DevSystem& d = h->d;
    cudaStream_t s = h->stream;
    const size_t len = (size_t)d.nRm * d.nSm;
    apply_A(s, d, u_plus, h->z1, nrhs);                                   // z1 = A u^+
    axpby_per_rhs(s, l_minus, h->z1, len, nrhs, nullptr, 1.0, nullptr, -1.0);   // l^- - z1
    RTE_TRY(mk_inv(h, h->z1, h->z2, nrhs));
    RTE_CUDA_TRY(cudaMemcpyAsync(u_minus, h->z2, sizeof(double) * len * nrhs,
                                 cudaMemcpyDeviceToDevice, s));
    RTE_CUDA_TRY(cudaGetLastError());
    return tc_gemm_error(s);
}

int rte_solve(rte_handle* h, const double* q, double* u, int nrhs, double tol,
              rte_stats* stats) {
    if (!h || !q || !u || nrhs < 1 || !(tol >= 0)) return fail(RTE_ERR_ARG, "bad argument");
    RTE_TRY(ensure_workspace(h, nrhs));
    const auto t0 = std::chrono::steady_clock::now();
    const DevSystem& d = h->d;
    cudaStream_t s = h->stream;
    const size_t len = (size_t)d.nRp * d.nSp;
    h->e0_launches = 0;
    h->e0_vcycles = h->e0_active_vcycles = 0.0;
    // the residual's split GEMMs to the accuracy the tolerance needs
    h->split_now = d.split_S > 0 ? slices_for_tol(tol, d.split_S) : 0;
    struct Reset {
        rte_handle* h;
        ~Reset() { h->split_now = 0; }
    } reset{h};
    double* r = h->e1;       // residual r_n
    double* sv = h->e2;      // s = P_2 P_1 r
    double* rprev = h->e3;
    double* delta = h->e4;   // u_n - u_{n-1}
    std::vector<double> hq(nrhs), hr(nrhs), hd1(nrhs), hd2(nrhs);
    double* sc = h->sc;
    dot_per_rhs(s, q, q, len, nrhs, h->partial, sc);
    RTE_CUDA_TRY(cudaMemcpyAsync(hq.data(), sc, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    int it = 0, rc = RTE_OK;
    double worst = 0.0, energy = 0.0;
    for (it = 0;; ++it) {
        // r = (E - K^+) u - q   (Algorithm 3: residual)
        RTE_TRY(apply_E(h, u, r, nrhs, true));
        {
            Scope scp(h, "axpy");
            axpby_per_rhs(s, q, r, len, nrhs, nullptr, -1.0, nullptr, 1.0);
        }
        dot_per_rhs(s, r, r, len, nrhs, h->partial, sc);
        if (it > 0) {
            // ||u_n - u_{n-1}||^2_{E-K} = delta^T (r_n - r_{n-1})
            dot_per_rhs(s, delta, r, len, nrhs, h->partial, sc + nrhs);
            dot_per_rhs(s, delta, rprev, len, nrhs, h->partial, sc + 2 * nrhs);
        }
        RTE_CUDA_TRY(cudaMemcpyAsync(hr.data(), sc, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        if (it > 0) {
            RTE_CUDA_TRY(cudaMemcpyAsync(hd1.data(), sc + nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
            RTE_CUDA_TRY(cudaMemcpyAsync(hd2.data(), sc + 2 * nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        }
        RTE_CUDA_TRY(cudaStreamSynchronize(s));
        settle_mk(h);
        worst = 0.0;
        energy = 0.0;
        bool nan = false;
        for (int k = 0; k < nrhs; ++k) {
            const double rel = hq[k] > 0 ? std::sqrt(hr[k] / hq[k]) : std::sqrt(hr[k]);
            if (bad(rel)) nan = true;
            worst = std::max(worst, rel);
            if (it > 0) energy = std::max(energy, std::sqrt(std::max(0.0, hd1[k] - hd2[k])));
        }
        if (stats && stats->history && it < stats->history_cap) stats->history[it] = worst;
        if (d.e0_direct && it > 0) RTE_TRY(e0_direct_error(s));
        if (nan) { rc = fail(RTE_ERR_DIVERGED, "residual is NaN or Inf"); break; }
        if (worst <= tol) break;
        if (it >= h->opt.max_iter) { rc = fail(RTE_ERR_MAXITER, "outer iteration cap reached"); break; }
        // s = P_2 P_1 r ; u_{n+1} = u_n - s   (half step plus subspace correction)
        RTE_TRY(precond(h, r, sv, nrhs, true));
        RTE_CUDA_TRY(cudaMemcpyAsync(rprev, r, sizeof(double) * nrhs * len, cudaMemcpyDeviceToDevice, s));
        RTE_CUDA_TRY(cudaMemcpyAsync(delta, sv, sizeof(double) * nrhs * len, cudaMemcpyDeviceToDevice, s));
        {
            Scope scp(h, "axpy");
            k_neg<<<(unsigned)((nrhs * len + 255) / 256), 256, 0, s>>>(delta, nrhs * len);
            count_launches(1);
            axpby_per_rhs(s, sv, u, len, nrhs, nullptr, -1.0, nullptr, 1.0);
        }
    }
    RTE_CUDA_TRY(cudaGetLastError());
    if (stats) {
        stats->iterations = it;
        stats->rel_residual = worst;
        stats->energy_update = energy;
        stats->e0_iters_last = h->e0_iters;
        stats->coarse_iters_last = h->co_iters;
        stats->mk_iters_last = h->mk_iters;
        stats->e0_launches = h->e0_launches;
        stats->e0_vcycles = h->e0_vcycles;
        stats->e0_active_vcycles = h->e0_active_vcycles;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
}

int rte_export(const rte_handle* h, int what, double* out, size_t n) {
    if (!h || !out) return fail(RTE_ERR_ARG, "bad argument");
    const std::vector<double>* src = nullptr;
    switch (what) {
        case 0: src = &h->h_Sp; break;
        case 1: src = &h->h_Sm; break;
        case 2: src = &h->h_m; break;
        case 3: src = &h->h_MSm; break;
        case 4: src = &h->h_A1; break;
        case 5: src = &h->h_A2; break;
        case 6: src = &h->h_omx; break;
        case 7: src = &h->h_omy; break;
        case 8: src = &h->h_lamP; break;
        case 9: src = &h->h_lamM; break;
        case 10: src = &h->h_WpN; break;
        case 11: src = &h->h_ec; break;
        default: return fail(RTE_ERR_ARG, "unknown export id");
    }
    if (n < src->size()) return fail(RTE_ERR_ARG, "export buffer too small");
    std::memcpy(out, src->data(), src->size() * sizeof(double));
    return RTE_OK;
}

int rte_timing_enable(rte_handle* h, int on) {
    if (!h) return fail(RTE_ERR_ARG, "NULL handle");
    flush_timers(h);
    h->timing = on != 0;
    for (auto& v : h->tms) v = 0.0;
    for (auto& v : h->tcount) v = 0;
    return RTE_OK;
}

int rte_timing_read(rte_handle* h, const char** names, double* ms, long long* launches,
                    int cap, int* count) {
    if (!h || !count) return fail(RTE_ERR_ARG, "bad argument");
    flush_timers(h);
    const int nn = (int)h->tnames.size();
    *count = nn;
    for (int i = 0; i < nn && i < cap; ++i) {
        if (names) names[i] = h->tnames[i].c_str();
        if (ms) ms[i] = h->tms[i];
        if (launches) launches[i] = h->tcount[i];
    }
    return RTE_OK;
}

long long rte_kernel_launches(void) { return launches_total(); }

int rte_set_wait_limit(double seconds) {
    if (!(seconds > 0) || seconds > 60.0) return fail(RTE_ERR_ARG, "limit must be in (0, 60] s");
    set_wait_limit_ns((unsigned long long)(seconds * 1e9));
    // mbarrier waits count SM clock cycles: at the peak clock, so that the
    // limit is never shorter than asked at a lower clock
    int dev = 0, khz = 0;
    RTE_CUDA_TRY(cudaGetDevice(&dev));
    RTE_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long cycles = (long long)(seconds * 1e3 * std::max(khz, 1));
    RTE_TRY(e0_set_wait_cycles(cycles));
    RTE_TRY(h2_set_wait_cycles(cycles));
    return tc_set_wait_cycles(cycles);
}

constexpr int kTraceCap = 1 << 16;

int rte_trace_enable(rte_handle* h, int on) {
    if (!h) return fail(RTE_ERR_ARG, "NULL handle");
    if (on && !h->trace) RTE_TRY(dalloc(h, &h->trace, kTraceCap));
    set_phase_trace(on ? h->trace : nullptr, on ? kTraceCap : 0);
    return RTE_OK;
}

int rte_trace_read(rte_handle* h, double* us, int cap, int* count) {
    if (!h || !count) return fail(RTE_ERR_ARG, "bad argument");
    *count = 0;
    if (!h->trace) return RTE_OK;
    // the barrier struct of the last launch holds the entry count; the
    // entries themselves are in the trace buffer
    std::vector<unsigned long long> t(kTraceCap);
    RTE_CUDA_TRY(cudaStreamSynchronize(h->stream));
    RTE_CUDA_TRY(cudaMemcpy(t.data(), h->trace, t.size() * 8, cudaMemcpyDeviceToHost));
    int n = 0;
    while (n + 1 < kTraceCap && t[n + 1] > t[n] && t[n] != 0) ++n;
    for (int i = 0; i < n && i < cap; ++i) us[i] = (t[i + 1] - t[i]) * 1e-3;
    *count = n;
    return RTE_OK;
}

int rte_dgemm_split(const double* A, const double* Bt, double* C, int M, int N, int K,
                    int slices, void* stream) {
    if (!A || !Bt || !C || M < 0 || N < 0 || K < 0 || slices < 1 || slices > 9)
        return fail(RTE_ERR_ARG, "bad argument");
    if (K % 8 != 0) return fail(RTE_ERR_ARG, "K must be a multiple of 8");
    if (M == 0 || N == 0) return RTE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) {
        RTE_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * M * N, s));
        RTE_CUDA_TRY(cudaStreamSynchronize(s));
        return RTE_OK;
    }
    char *pa = nullptr, *pb = nullptr;
    if (cudaMallocAsync(&pa, ozaki_slice_bytes(M, K, slices), s) != cudaSuccess ||
        cudaMallocAsync(&pb, ozaki_slice_bytes(N, K, slices), s) != cudaSuccess) {
        cudaFreeAsync(pa, s);
        return fail(RTE_ERR_NOMEM, "split GEMM temporaries");
    }
    int *ea = nullptr, *eb = nullptr;
    int rc = ozaki_split(s, A, M, K, slices, pa, &ea);
    if (!rc) rc = ozaki_split(s, Bt, N, K, slices, pb, &eb);
    if (!rc) rc = ozaki_gemm(s, pa, ea, M, pb, eb, N, K, slices, C, N, 0, nullptr, 1);
    cudaFreeAsync(pa, s);
    cudaFreeAsync(pb, s);
    if (rc) return rc;
    return tc_gemm_error(s);
}

size_t rte_autotune_report(char* buf, size_t len) {
    const std::string r = autotune_report();
    if (buf && len > 0) {
        const size_t n = std::min(len - 1, r.size());
        std::memcpy(buf, r.data(), n);
        buf[n] = 0;
    }
    return r.size();
}

int rte_gemm_lowp(const void* A, const void* Bt, void* C, int M, int N, int K, int bf16,
                  int out_bf16, void* stream) {
    if (!A || !Bt || !C || M < 0 || N < 0 || K < 0) return fail(RTE_ERR_ARG, "bad argument");
    TcGemmArgs g{};
    g.A = A; g.Bt = Bt; g.C = C; g.M = M; g.N = N; g.K = K; g.ldc = N;
    g.tf32 = bf16 == 0; g.out_bf16 = bf16 != 0 && out_bf16 != 0; g.rows = 1;
    RTE_TRY(tc_gemm((cudaStream_t)stream, g));
    return tc_gemm_error((cudaStream_t)stream);
}

void rte_destroy(rte_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& t : h->trecs) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto& kv : h->mk_graph) cudaGraphExecDestroy(kv.second);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->mk_state_host) cudaFreeHost(h->mk_state_host);
    for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
    cudaStreamSynchronize(h->stream);
    // rte_destroy reports nothing: leave no error behind for the thread's
    // next runtime call to pick up
    cudaGetLastError();
    delete h;
}

}  // extern "C"
