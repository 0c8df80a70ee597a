/*
 * rte.h - C ABI of the GB300 library for the preconditioned Richardson
 * iteration of Dölz, Palii and Schlottbom (arXiv 2102.09038) for the
 * even-parity anisotropic radiative transfer equation.
 *
 * Discretisation (Section 4): continuous P1 elements on a uniform
 * "/"-triangulation of the unit square (n_R^+ = (m+1)^2 nodes,
 * n_R^- = 2 m^2 cells) times piecewise-constant even (n_S^+) and piecewise-
 * linear odd (n_S^- = 3 n_S^+) functions on a sphere mesh made by refining the
 * octahedron ``sphere_levels`` times (8 * 4^levels triangles, one even
 * function per antipodal pair).
 *
 * Vector layout.  Every even vector is nrhs consecutive matrices
 * U^+ (n_R^+ x n_S^+) stored row-major: element (r, i, k) at
 * ((r * n_R^+) + i) * n_S^+ + k, node i, direction k.  Odd vectors use
 * n_R^- x n_S^- the same way (odd index 3k + c).  Coarse vectors use
 * n_R^+ x d^+ (mode index fastest).
 *
 * Ownership.  The caller owns every vector pointer (device memory unless a
 * name says host).  The handle owns the assembled matrices and a workspace
 * sized for opts->max_rhs right-hand sides; it is freed by rte_destroy.
 * All work is queued on the stream given to rte_setup; functions that
 * return statistics synchronise that stream.
 *
 * Errors.  Every function returns RTE_OK (0) or one of the RTE_ERR_* codes
 * and never aborts.  rte_last_error() gives a message for the calling
 * thread's last failure.
 */
#ifndef RTE_H
#define RTE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTE_OK 0
#define RTE_ERR_ARG 1       /* invalid argument or size                      */
#define RTE_ERR_NOMEM 2     /* device or host allocation failed              */
#define RTE_ERR_DIVERGED 3  /* residual grew or became NaN/Inf               */
#define RTE_ERR_MAXITER 4   /* iteration cap reached before the tolerance   */
#define RTE_ERR_TIMEOUT 5   /* a bounded device-side wait gave up            */
#define RTE_ERR_CUDA 6      /* a CUDA runtime or library call failed         */

/* Arithmetic of the inner operators (the outer residual is always FP64). */
#define RTE_FP64 0          /* every step in FP64                            */
#define RTE_MIXED_FP32 1    /* inner applies in FP32 (TF32 tensor GEMMs)     */
#define RTE_MIXED_BF16 2    /* inner applies in FP32, scattering GEMMs BF16  */

/* How the FP64 dense contractions (eigenbasis of (M^- - K^-)^{-1}, U S^+)
 * are computed: RTE_DGEMM_AUTO picks SIMT in RTE_FP64 mode and SPLIT in the
 * mixed modes; RTE_DGEMM_SIMT uses FP64 arithmetic units; RTE_DGEMM_SPLIT
 * cuts the FP64 operands into exact BF16 digit slices whose tensor-core
 * products are summed in FP64 (about 2^-49 relative to the operand scales
 * with the default 7 slices). */
#define RTE_DGEMM_AUTO 0
#define RTE_DGEMM_SIMT 1
#define RTE_DGEMM_SPLIT 2

/* How (M^- - K^-)^{-1} is applied inside Apply-E (Algorithm 1, line 2).
 * RTE_MK_PCG runs the paper's PCG with the Lemma's preconditioner to mk_tol
 * as a device-side loop (a CUDA graph whose while node repeats one iteration
 * until a check kernel finds every right-hand side converged, or mk_maxit):
 * no host round trip per iteration.  In the mixed modes it applies to the
 * FP64 operator (the outer residual), with K^- on the split FP64-accurate
 * tensor-core GEMM; the inner FP32 applies keep the eigenbasis route. */
#define RTE_MK_EIGEN 0      /* exact, in the full eigenbasis of (S^-, M_S^-) */
#define RTE_MK_PCG 1        /* PCG with the Lemma apply_high_order_pre prec. */

/* How P_1 is realised (Section 5.3).  RTE_P1_RICHARDSON is P_1^l of eq.
 * (applyP1): l steps of the preconditioned Richardson iteration for E from
 * z = 0, a fixed SPD matrix (Lemma preconditioner_pl).  RTE_P1_PCG takes l
 * steps of conjugate gradients for E z = b preconditioned by E_0^{-1}, from
 * z = 0: the non-stationary alternative the same section names beside it.
 * Its result is the E-norm-best point of the same Krylov space (so never
 * worse than P_1^l b in that norm) but depends nonlinearly on b, so
 * rte_rates, whose power iterations need a fixed iteration matrix, refuses
 * it.  Per application: l E_0^{-1} solves (as P_1^l) and l applies of E
 * (one more than P_1^l).  RTE_P1_AUTO (the default) takes P_1^l in FP64
 * mode, the paper's method as stated, and the PCG steps in the mixed modes,
 * where they reach 1e-6 on the 128x128 / 512-triangle workload in 16 outer
 * iterations instead of 27. */
#define RTE_P1_AUTO (-1)
#define RTE_P1_RICHARDSON 0
#define RTE_P1_PCG 1

/* How E_0^{-1} is applied (its n_S^+ decoupled direction blocks, eq.
 * equivalence_bE_bE0).  RTE_E0_DIRECT factorises every block once at setup,
 * as the paper's experiments do (Section 6: a sparse direct solver for
 * E_0's blocks): the blocks are block tridiagonal over the mesh rows, and
 * the library keeps the inverses of their Schur complements ((m+1)^2 values
 * per row and direction; FP64 in RTE_FP64 mode, FP32 in the mixed modes) and
 * solves by one forward and one backward sweep, exactly up to rounding;
 * e0_tol and e0_maxit are then unused.  RTE_E0_MULTIGRID runs CG
 * preconditioned by a V-cycle per block to e0_tol, the route Section 5.5
 * names for larger problems.  RTE_E0_AUTO (0, the default) takes the direct
 * route when the mesh allows it (m <= 156) and multigrid otherwise. */
#define RTE_E0_AUTO 0
#define RTE_E0_DIRECT 1
#define RTE_E0_MULTIGRID 2

/* How the coarse system E_c u_c = q_c of the subspace correction (Section
 * 5.4) is solved: by CG to coarse_tol in every route, preconditioned by
 * RTE_EC_DIRECT: E_c's exact block factorisation over the mesh rows (the
 * inverses of its row Schur complements, ((m+1) d^+)^2 values per row,
 * computed once at setup in FP64 and kept in FP64 (FP64 mode) or FP32), so
 * the CG stops after one or two iterations; or RTE_EC_MULTIGRID: one V-cycle
 * (the paper's suggestion), whose iteration count grows with the mesh for
 * d^+ > 1.  The direct route needs (m+1) d^+ <= 2400.  RTE_EC_AUTO (0, the
 * default) takes multigrid: on the 128 x 128 / 512-triangle workload its
 * coarse solve (11 iterations to 0.1) took 4.1 ms against 9.9 ms for the
 * direct route, whose set-up also adds 3.6 s. */
#define RTE_EC_AUTO 0
#define RTE_EC_DIRECT 1
#define RTE_EC_MULTIGRID 2

typedef struct rte_handle rte_handle;

/* The problem of Section 1, eq. (rte1)-(rte2), with vacuum inflow:
 * sigma_t, sigma_s piecewise constant per cell (host arrays of length
 * 2*mesh_m^2, 0 <= sigma_s < sigma_t), Henyey-Greenstein parameter
 * 0 <= g < 1 (eq. HG-kernel1). */
typedef struct {
    int mesh_m;             /* m >= 1: m x m squares                         */
    int sphere_levels;      /* 0..5: 8*4^levels sphere triangles            */
    const double* sigma_t;  /* host, per cell                                */
    const double* sigma_s;  /* host, per cell                                */
    double g;
} rte_problem;

/* Method parameters.  Defaults (rte_default_options) follow Section 6:
 * l = 4 inner steps for P_1^l (2 for the PCG realisation of P_1), N^+ = 4
 * (d^+ = 15) for the subspace correction, N^- = 5 (d^- = 21) for the
 * preconditioner of (M^- - K^-). */
typedef struct {
    int l;                  /* steps of P_1 (eq. applyP1); 0: 4 for P_1^l
                               (Section 6), 2 for the PCG steps              */
    int n_plus;             /* even degree N^+ (0, 2, 4, ...); -1: no P_2    */
    int n_minus;            /* odd degree N^- (1, 3, 5, ...)                 */
    int precision;          /* RTE_FP64 | RTE_MIXED_FP32 | RTE_MIXED_BF16    */
    int mk_route;           /* RTE_MK_EIGEN | RTE_MK_PCG                     */
    double mk_tol;          /* relative residual of the (M^- - K^-) PCG      */
    int mk_maxit;
    double e0_tol;          /* relative residual per column of E_0 CG
                               (multigrid route);
                               0: 1e-12 (FP64) or 0.3 (mixed modes)          */
    int e0_maxit;
    double coarse_tol;      /* relative residual of the E_c CG;
                               0: 1e-12 (FP64) or 0.3 (mixed modes); from
                               1e-2 on, mixed modes run the CG's own E_c
                               products in FP32 (multigrid route), the CG
                               recurrences staying FP64                     */
    int coarse_maxit;
    int max_iter;           /* outer Richardson iterations                   */
    int max_rhs;            /* workspace is sized for this many RHS          */
    int dgemm;              /* RTE_DGEMM_AUTO | RTE_DGEMM_SIMT | _SPLIT      */
    int split_slices;       /* digit slices per operand for RTE_DGEMM_SPLIT  */
    int mg_sweeps;          /* smoothing sweeps before and after each coarse
                               correction in the multigrid preconditioners   */
    int autotune;           /* 1: time the launch shapes of the SpMM kernels
                               and tensor-core GEMMs at setup (cached per
                               shape for the process); 0: fixed shapes       */
    int p1_route;           /* RTE_P1_AUTO (default) | RTE_P1_RICHARDSON |
                               RTE_P1_PCG                                    */
    int e0_route;           /* RTE_E0_AUTO (default) | RTE_E0_DIRECT |
                               RTE_E0_MULTIGRID                              */
    int coarse_route;       /* RTE_EC_AUTO (default) | RTE_EC_DIRECT |
                               RTE_EC_MULTIGRID                              */
} rte_options;

typedef struct {
    int iterations;             /* outer iterations taken                    */
    double rel_residual;        /* max over RHS of ||r||_2 / ||q||_2 (FP64)  */
    double energy_update;       /* max over RHS of ||u_n - u_{n-1}||_{E-K}   */
    int e0_iters_last;          /* CG iterations of the last E_0^{-1}        */
    int coarse_iters_last;      /* CG iterations of the last coarse solve    */
    int mk_iters_last;          /* PCG iterations of the last (M-K)^{-1}     */
    double* history;            /* optional host array: rel. residual per it */
    int history_cap;            /* its capacity                              */
    double seconds;             /* wall time of the solve                    */
    int e0_launches;            /* E_0^{-1} applications in the solve        */
    double e0_vcycles;          /* their multigrid V-cycles, summed          */
    double e0_active_vcycles;   /* the same, each weighted by the fraction of
                                   direction columns (in groups of four) not
                                   yet converged, which are the only ones the
                                   mixed-mode kernel visits                  */
} rte_stats;

/* Fills *opts with the defaults above (FP64, eigen route, tolerances
 * 1e-12, 200 outer iterations, max_rhs 1). */
int rte_default_options(rte_options* opts);

/* Assembles the discrete system of Section 4 (eq. bKebKo, bMebMo, AR),
 * the generalised eigenpairs of (S^+, M_S^+) and (S^-, M_S^-) (Section 5.1
 * and 5.4), the direction blocks of E_0 (eq. equivalence_bE_bE0) and the
 * coarse matrix E_c = W^T (E - K^+) W (Section 5.4, Algorithm 3 lines 1-4)
 * and uploads them to the current device.  stream: a cudaStream_t (NULL
 * for the legacy default stream).  On success *out owns all of it.  A
 * problem whose estimated device memory (rte_estimate_bytes at
 * opts->max_rhs) exceeds the device's free memory plus what its default
 * memory pool holds unused is refused with RTE_ERR_NOMEM before anything is
 * allocated. */
int rte_setup(const rte_problem* prob, const rte_options* opts, void* stream,
              rte_handle** out);

/* Moves the handle's work to another stream (a cudaStream_t): functions
 * called afterwards queue on it.  Work already queued on the old stream is
 * not waited for; the caller orders the two. */
int rte_set_stream(rte_handle* h, void* stream);

/* Sizes of the discrete spaces: n_R^+, n_R^-, n_S^+, n_S^-, d^+, d^-. */
int rte_sizes(const rte_handle* h, int* n_nodes, int* n_cells, int* n_dirs,
              int* n_odd, int* d_plus, int* d_minus);

/* q = l^+ for an isotropic source with nodal values q_nodal (device,
 * nrhs x n_R^+) and vacuum inflow: q_{i,k} = (M q_h)_i * |K_k u -K_k|
 * (Section 2.4, l^+(w) = (q, w)); l^- = 0 because the odd functions
 * integrate to zero against an isotropic q. */
int rte_rhs(rte_handle* h, const double* q_nodal, double* q, int nrhs);

/* q += the inflow part of l^+ (Section 2.4: l^+(w^+) = (q, w^+) +
 * 2 (|s.n| g, w^+) over dD_- = {(s, r): r on the boundary, s.n(r) < 0})
 * for inflow data g, a device array [nrhs][4][m + 1][2 n_S^+] of values
 * piecewise constant on the sphere triangles and P1 along each face:
 * face f = 0, 1, 2, 3 is x = 0, x = 1, y = 0, y = 1; node j runs along the
 * face in increasing y (x faces) or x (y faces), i.e. node index
 * j (m+1), j (m+1) + m, j and m (m+1) + j; entry 2k is the value on K_k
 * and 2k + 1 on -K_k.  Only the triangle of each pair that points into the
 * domain through the face (s.n < 0) is read; the other entry is ignored.
 * q: device, nrhs x n_R^+ x n_S^+ (e.g. from rte_rhs); the term is added.
 * Vacuum inflow (g = 0) needs no call. */
int rte_inflow(rte_handle* h, const double* g, double* q, int nrhs);

/* y = (E - K^+) x (eq. ep_discrete; Algorithm 1 for E), device vectors. */
int rte_apply(rte_handle* h, const double* x, double* y, int nrhs);

/* s = P_2 P_1^l r: P_1^l of eq. (applyP1) and, when with_p2 != 0, the
 * subspace correction of eq. (product_pre):
 * s = P_1 r + W E_c^{-1} W^T (r - (E - K^+) P_1 r). */
int rte_precond(rte_handle* h, const double* r, double* s, int nrhs,
                int with_p2);

/* Algorithm 3: preconditioned Richardson iteration for (E - K^+) u = q,
 * eq. (Richardson_discrete), from the initial guess held in u on entry,
 * until ||r_n||_2 <= tol ||q||_2 for every RHS (r_n in FP64).  stats may be
 * NULL.  Returns RTE_ERR_MAXITER if opts.max_iter is reached and
 * RTE_ERR_DIVERGED on a NaN/Inf residual. */
int rte_solve(rte_handle* h, const double* q, double* u, int nrhs, double tol,
              rte_stats* stats);

/* Contraction estimates of Section 6.2 by power iteration on the handle's
 * own operators (nrhs = 1):
 *  rho = spectral radius of T = I - P_2 P_1^l (E - K^+) (Algorithm 3's
 *        iteration matrix, = (I - P_G)(I - P_1^l (E - K^+)));
 *  eta = its (E - K^+)-norm: eta^2 = largest eigenvalue of
 *        (I - P_1^l A)(I - P_G)(I - P_1^l A), A = E - K^+, P_G the
 *        A-orthogonal projection onto span W (needs n_plus >= 0).
 * Starts from a seeded uniform vector; stops when two successive estimates
 * differ by at most tol (relative) or after maxit steps (*iters = steps
 * taken).  rho or eta may be NULL to skip it.  Use an FP64 handle: in the
 * mixed modes the inner solves stop at loose tolerances and the operator is
 * only approximately linear.  Uses the handle's workspace (not concurrently
 * with rte_solve on the same handle). */
int rte_rates(rte_handle* h, int maxit, double tol, unsigned long long seed, double* rho,
              double* eta, int* iters);

/* The odd part of the solution from the even part: the second block row of
 * the mixed system (eq. mixed_discrete), A u^+ + (M^- - K^-) u^- = l^-, so
 * u^- = (M^- - K^-)^{-1} (l^- - A u^+) (Section 2.4).  u_plus: nrhs x n_R^+
 * x n_S^+; l_minus: nrhs x n_R^- x n_S^- or NULL for l^- = 0 (isotropic
 * source, vacuum inflow); u_minus: nrhs x n_R^- x n_S^-, odd index 3k + i.
 * Device arrays owned by the caller.  FP64 in every mode (the FP64-accurate
 * (M^- - K^-)^{-1} of the outer residual). */
int rte_odd(rte_handle* h, const double* u_plus, const double* l_minus, double* u_minus,
            int nrhs);

/* Individual steps of the iteration, for testing and profiling (device
 * vectors, sizes as in the header comment):
 *  RTE_OP_A          odd  <- even : A x = sum_n A_n (x) D_n     (eq. AR)
 *  RTE_OP_AT         even <- odd  : A^T z
 *  RTE_OP_KPLUS      even <- even : K^+ x = (S^+ (x) M_s^+) x (eq. bKebKo)
 *  RTE_OP_MK         odd  <- odd  : (M^- - K^-) z
 *  RTE_OP_MK_INV     odd  <- odd  : (M^- - K^-)^{-1} z by mk_route
 *  RTE_OP_MK_PREC    odd  <- odd  : (M^- - K^-_N)^{-1} z, eq. (MmKprecond)
 *  RTE_OP_E          even <- even : E x (Algorithm 1)
 *  RTE_OP_E0_INV     even <- even : E_0^{-1} x by per-direction CG
 *  RTE_OP_P1         even <- even : P_1^l x (Algorithm 2, eq. applyP1)
 *  RTE_OP_RESTRICT   coarse <- even: W^T x = X W_N^+
 *  RTE_OP_PROLONG    even <- coarse: W u_c = U_c (W_N^+)^T
 *  RTE_OP_EC         coarse <- coarse: E_c u_c
 *  RTE_OP_EC_INV     coarse <- coarse: E_c^{-1} u_c by CG
 *  RTE_OP_E_LO       even <- even : E x in the handle's mixed precision
 *  RTE_OP_EK_LO      even <- even : (E - K^+) x in the mixed precision
 * (the _LO ids need a handle set up with RTE_MIXED_FP32 / RTE_MIXED_BF16;
 * vectors stay FP64 at the interface)                                      */
#define RTE_OP_A 1
#define RTE_OP_AT 2
#define RTE_OP_KPLUS 3
#define RTE_OP_MK 4
#define RTE_OP_MK_INV 5
#define RTE_OP_MK_PREC 6
#define RTE_OP_E 7
#define RTE_OP_E0_INV 8
#define RTE_OP_P1 9
#define RTE_OP_RESTRICT 10
#define RTE_OP_PROLONG 11
#define RTE_OP_EC 12
#define RTE_OP_EC_INV 13
#define RTE_OP_E_LO 14
#define RTE_OP_EK_LO 15
int rte_operator(rte_handle* h, int op, const double* in, double* out,
                 int nrhs);

/* Tensor-core GEMM used by the mixed-precision paths, exposed for testing
 * and profiling: C[M x N] = A[M x K] * Bt[N x K]^T with A and Bt row-major
 * (K contiguous) device arrays of BF16 (bf16 != 0) or FP32 read as TF32,
 * FP32 accumulation, C written as FP32 (or BF16 if out_bf16 and bf16).
 * K * element size and the base addresses must be multiples of 16 bytes.
 * Queued on stream (a cudaStream_t). */
int rte_gemm_lowp(const void* A, const void* Bt, void* C, int M, int N, int K,
                  int bf16, int out_bf16, void* stream);

/* The launch shapes the autotuner chose so far in this process (one
 * "key=choice (ms per candidate);" entry per tuned kernel shape; choice is
 * the candidate index: block sizes 128/256/512 for the SpMM kernels, tile
 * widths 128/256 for the tensor-core GEMMs).  Copies at most len - 1 bytes
 * and a terminating zero into buf (buf may be NULL when len is 0); returns
 * the length of the whole report. */
size_t rte_autotune_report(char* buf, size_t len);

/* The FP64 split GEMM of RTE_DGEMM_SPLIT, exposed for testing and
 * profiling: C[M x N] = A[M x K] * Bt[N x K]^T, all FP64 row-major device
 * arrays, with `slices` digit slices per operand (1..9).  K must be a
 * multiple of 8 (refused with RTE_ERR_ARG before any device work); K = 0
 * writes C = 0.  Allocates its temporaries stream-ordered on `stream` and
 * synchronises it before returning (it reads the GEMM's timeout flag). */
int rte_dgemm_split(const double* A, const double* Bt, double* C, int M, int N, int K,
                    int slices, void* stream);

/* Allocation-free variant of rte_dgemm_split.  The paper has no counterpart:
 * this serves callers that must not allocate device memory when they call,
 * such as a process whose device memory is already handed to another
 * allocator (a framework's caching pool, a serving memory budget), or a
 * latency-critical loop in which an allocation could block or fail.
 *
 * Same arguments, kernels and result as rte_dgemm_split, but the digit
 * slices and row exponents of both operands live in one static device array
 * of RTE_SPLIT_STATIC_SCRATCH_BYTES inside the library; it allocates nothing
 * (no cudaMalloc, no pool, no library allocator).  Nothing in the scratch
 * has to start at zero: every call writes all it reads.
 *
 * Limit: the operands need ceil256(2 slices M K + 4 M + 512) +
 * 2 slices N K + 4 N + 512 bytes of scratch, at most
 * RTE_SPLIT_STATIC_SCRATCH_BYTES = 32 MiB (e.g. slices = 7 with
 * M = N = K = 1024).  Larger operands return RTE_ERR_ARG, with the bytes
 * needed in rte_last_error(), before any device work.  K must be a multiple
 * of 8 (16-byte rows of BF16 slices), also refused before any device work;
 * K = 0 writes C = 0.
 *
 * Every call looks up the scratch's device address on the current device
 * (so a device reset cannot leave a stale address) and sets the GEMM
 * kernel's shared-memory attribute; the first call on each device also
 * loads the library's device code there: make it before any stream capture
 * begins on that device.  Calls that overlap in time on one device
 * (from several host threads, or on streams whose work overlaps) share the
 * one scratch and race: order them (one stream, or an event between them).
 * Synchronises `stream` before returning (it reads the GEMM's timeout
 * flag). */
#define RTE_SPLIT_STATIC_SCRATCH_BYTES (32u << 20)
int rte_dgemm_split_static(const double* A, const double* Bt, double* C, int M, int N, int K,
                           int slices, void* stream);

/* Copies an assembled matrix to host memory (for checks against an
 * independent assembly).  what: 0 S^+ (n_S^+^2), 1 S^- (n_S^-^2),
 * 2 M_S^+ diagonal (n_S^+), 3 M_S^- blocks (n_S^+ x 9), 4 A_1 (n_S^+ x 3),
 * 5 A_2 (n_S^+ x 3), 6 omega^x (n_S^+), 7 omega^y (n_S^+), 8 Lambda^+
 * (n_S^+, non-increasing), 9 Lambda^- (n_S^-), 10 W_N^+ (n_S^+ x d^+),
 * 11 E_c nonzero blocks (count x d^+ x d^+, CSR order of the node stencil).
 * n: capacity of host_out in doubles; returns RTE_ERR_ARG if too small. */
int rte_export(const rte_handle* h, int what, double* host_out, size_t n);

/* Per-kernel device time (milliseconds) accumulated since the last reset,
 * measured with CUDA events on the handle's stream when timing is enabled:
 * names[i] and ms[i] for i < *count (capacity cap). */
int rte_timing_enable(rte_handle* h, int on);
int rte_timing_read(rte_handle* h, const char** names, double* ms,
                    long long* launches, int cap, int* count);

/* Wall-clock milliseconds of the stages of the rte_setup that made h (host
 * assembly, scattering matrices, the two angular eigen-decompositions, the
 * coarse matrix E_c, the FP64 split operands, the E_0 and E_c multigrid
 * hierarchies, the workspace, launch tuning); each stage ends with a synchronisation of the
 * handle's stream, so device work is charged to the stage that issued it.
 * names[i] and ms[i] for i < min(*count, cap); the names stay valid while
 * h lives.  Not part of the paper's method: profiling of the setup. */
int rte_setup_times(const rte_handle* h, const char** names, double* ms, int cap,
                    int* count);

/* Phase trace of the persistent solver kernels, for profiling: with on != 0
 * the next E_0 / E_c solves record the time after every grid barrier of
 * their launch; rte_trace_read copies the intervals (microseconds) of the
 * most recent launch into us[0..cap) and their number into *count. */
int rte_trace_enable(rte_handle* h, int on);
int rte_trace_read(rte_handle* h, double* us, int cap, int* count);

/* Number of CUDA kernels this library has launched in this process (all
 * handles, all threads), for counting launches inside a timed region. */
long long rte_kernel_launches(void);

/* Failure detection (not part of the paper's method).  Every device-side
 * wait of the library is bounded: a grid-barrier wait of the persistent
 * E_0 / E_c kernels, and an mbarrier wait of the tensor-core pipelines.  A
 * wait that runs out makes the kernel record the failure and return; the
 * calling function then returns RTE_ERR_TIMEOUT and the CUDA context stays
 * usable.  rte_set_wait_limit sets the limit (seconds, in (0, 60]; default
 * 2 s): for grid barriers of every launch made after the call, for mbarrier
 * waits on the current device.  Not thread-safe against concurrent
 * launches. */
int rte_set_wait_limit(double seconds);

/* Self-test of the bounded grid barrier: a cooperative launch of `blocks`
 * blocks (at most the device's resident capacity, else RTE_ERR_ARG) that
 * meet at `rounds` barriers, except block skip_block (>= 0), which leaves
 * before the first, so that the others' waits run out after the current
 * wait limit; skip_block < 0: no block leaves.  Queued on `stream` and
 * synchronised.  *timed_out = whether a wait ran out; *passed_blocks = the
 * blocks that passed every barrier.  Returns RTE_ERR_TIMEOUT if a wait ran
 * out, else RTE_OK. */
int rte_barrier_selftest(int blocks, int skip_block, int rounds, void* stream, int* timed_out,
                         int* passed_blocks);

void rte_destroy(rte_handle* h);

/* ------------------------------------------------------------------------
 * Serving and batching (not part of the paper's method).
 *
 * A server runs `slots` worker threads, each with its own CUDA stream on the
 * current device.  Submitted requests (problem + nodal source) are admitted
 * in arrival order when a slot is free and the estimated device memory of
 * the admitted requests stays within hbm_budget_bytes (a request larger than
 * the budget runs alone).  A request runs rte_setup, rte_rhs and rte_solve on
 * its slot's stream and copies u back to host memory; the device work of
 * concurrent requests overlaps.  The server copies the problem arrays and
 * the source at submission; the caller keeps ownership of its buffers.
 *
 * Operator cache: after a request the server keeps its set-up handle idle.
 * A later request with the same operator (mesh, sphere level, g and sigma
 * fields; the options are the server's) and no more right-hand sides takes
 * it and skips rte_setup: only its source, solve and copy-back run.  Idle
 * handles count against hbm_budget_bytes and are destroyed, least recently
 * used first, when an admission needs their memory.
 * ------------------------------------------------------------------------ */
typedef struct rte_server rte_server;

/* Device bytes a solve of this problem with nrhs right-hand sides needs
 * (an upper estimate used for admission). */
size_t rte_estimate_bytes(const rte_problem* prob, const rte_options* opts, int nrhs);

int rte_server_create(size_t hbm_budget_bytes, int slots, const rte_options* opts,
                      rte_server** out);

/* Queues a solve of (E - K^+) u = q with q from the host nodal source
 * q_nodal (nrhs x n_R^+) to the relative residual tol; *id identifies it. */
int rte_server_submit(rte_server* sv, const rte_problem* prob, const double* q_nodal,
                      int nrhs, double tol, long long* id);

/* Waits (timeout_s < 0: without limit) for request id, copies its solution
 * (nrhs x n_R^+ x n_S^+) into host u (u_len doubles; may be NULL), its
 * statistics, its latency from submission to completion and its queueing
 * time.  Returns the request's own status; RTE_ERR_TIMEOUT if it has not
 * finished in time (the request stays queryable). */
int rte_server_wait(rte_server* sv, long long id, double timeout_s, double* u, size_t u_len,
                    rte_stats* stats, double* latency_s, double* queue_s);

/* Finishes the running requests and stops the workers; requests still
 * queued are dropped; idle handles are destroyed. */
void rte_server_destroy(rte_server* sv);

/* Operator-cache counters: admissions that took an idle handle (*hits), that
 * set up a new one (*misses), and the bytes of the idle handles now kept.
 * Any pointer may be NULL. */
int rte_server_cache_stats(rte_server* sv, long long* hits, long long* misses,
                           size_t* idle_bytes);

/* Solves `count` independent problems at once through a temporary server:
 * q_nodal[i] (host, nrhs[i] x n_R^+), u[i] (host, nrhs[i] x n_R^+ x n_S^+). */
int rte_solve_batch(const rte_problem* probs, const double* const* q_nodal, const int* nrhs,
                    double* const* u, int count, double tol, const rte_options* opts,
                    size_t hbm_budget_bytes, int slots, rte_stats* stats);

/* ------------------------------------------------------------------------
 * H^2-compressed scattering matrices (Section 5.2; the compression
 * experiment of Section 6).  S^+ = 2 (D + M) and S^- = 2 (D - M) in the basis
 * of the representatives, with D the direct part (kernel k(s.s') over
 * K_k x K_k') and M the mirror part (k(-s.s'), K_k x (-K_k')); each part is
 * approximated by interpolating the extension K(x~, y~) = k(x.y),
 * x = x~/|x~| (eq. HGextension):
 *   cluster tree   the refinement hierarchy of the representatives; leaves
 *                  hold n_min = 64 of them (so levels >= 3);
 *   boxes          bounding boxes of each cluster's far-rule quadrature
 *                  points (negated for the mirror part's column cluster);
 *   admissibility  max(diam B_t, diam B_c) <= eta dist(B_t, B_c);
 *   interpolation  p Chebyshev points per coordinate (p^3 <= 64 per box),
 *                  nested bases (leaf bases and transfer matrices);
 *   near blocks    exact entries by the dense assembly's quadrature rules.
 * Set-up runs on the device; the apply is a sequence of block-sparse
 * products over 64-column blocks (leaf forward transform, upward transfers,
 * couplings, downward transfers, leaf backward transform, near field).
 * ------------------------------------------------------------------------ */
typedef struct rte_h2 rte_h2;

typedef struct {
    int levels;        /* sphere refinement, n_S^+ = 4 * 4^levels; 3..8    */
    double g;          /* Henyey-Greenstein asymmetry, 0 <= g < 1          */
    double eta;        /* admissibility parameter (> 0; the paper: 1.4)    */
    int p;             /* interpolation points per coordinate, 2..4        */
    int parities;      /* bit 0: S^+, bit 1: S^- (at least one)            */
    int precisions;    /* bit 0: FP64 apply, bit 1: FP32 apply, bit 2: BF16
                          tensor-core apply                                */
} rte_h2_options;

typedef struct {
    int n_plus;               /* n_S^+                                      */
    int leaves, clusters;     /* leaf clusters; clusters holding a basis    */
    int far_blocks[2];        /* admissible blocks, direct / mirror part    */
    int near_blocks[2];       /* inadmissible leaf pairs, direct / mirror   */
    int near_matrices;        /* near blocks after merging the two parts    */
    int transfers;            /* transfer matrices (clusters below the top) */
    size_t bytes;             /* device bytes of the compressed matrices    */
    double setup_ms;          /* wall time of rte_h2_create                 */
} rte_h2_info;

/* Fills the paper's parameters: eta = 1.4, p = 4, both parities, every
 * precision. */
int rte_h2_default_options(rte_h2_options* opts);

/* Builds the compressed S^+ and/or S^- on the current device (on `stream`,
 * synchronised before returning).  RTE_ERR_ARG for options out of range;
 * RTE_ERR_NOMEM when the matrices do not fit in free device memory (checked
 * on the host before allocating). */
int rte_h2_create(const rte_h2_options* opts, void* stream, rte_h2** out);

/* Y = X S^+ (parity +1) or Y = X S^- (parity -1) for `rows` row vectors:
 * X and Y are device arrays [rows][n] (n = n_S^+ for S^+, n_S^- = 3 n_S^+
 * for S^-, row-major, caller-owned, not overlapping, 16-byte aligned).
 * precision: RTE_FP64 (FP64 products on the FP64 units); RTE_MIXED_FP32
 * (FP32 products; X rounded to FP32, Y written back in FP64);
 * RTE_MIXED_BF16 (tcgen05 products with BF16 operands and FP32
 * accumulation; X, the bases, the coupling and near matrices and the
 * cluster coefficients rounded to BF16, Y accumulated in FP32).  Work
 * buffers grow on demand and are kept in the handle.  Stream-ordered on
 * `stream`; the FP64 and FP32 applies do not synchronise, the BF16 apply
 * synchronises to read its pipelines' timeout flag (RTE_ERR_TIMEOUT).
 * rows = 0 is a no-op. */
int rte_h2_apply(rte_h2* h, int parity, int precision, const double* X, double* Y, int rows,
                 void* stream);

int rte_h2_get_info(const rte_h2* h, rte_h2_info* info);

/* The host half of rte_h2_create alone: the cluster and block trees of the
 * options (no device call; bytes and setup_ms are 0).  RTE_ERR_ARG as in
 * rte_h2_create. */
int rte_h2_plan_info(const rte_h2_options* opts, rte_h2_info* info);

/* Dense S^+ or S^- (host, n x n row-major) assembled by the same device
 * quadrature as rte_setup's; for comparisons at moderate n (n_S^+ <= 4096). */
int rte_h2_dense(const rte_h2* h, int parity, double* host_out, size_t n);

void rte_h2_destroy(rte_h2* h);

/* Message of the calling thread's last error ("" if none). */
const char* rte_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RTE_H */
