// Device-resident data of one assembled problem and the kernel launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "mg.h"

namespace rte {

// FP32 copies of the operator data used by the mixed-precision paths, and
// the low-precision GEMM operands (BF16 or FP32 read as TF32), K-major.
struct DevLow {
    const float* ell4;         // M_t^+, M_s^+, B_x, B_y in ELL form [4][7][nRp]
    const float* cell_D;       // [nRm][6]
    const float* cell_at;      // [nRm]
    const float* cell_as;      // [nRm]
    const float* sval;         // [kSlots][nnz]
    const float* m;            // [nSp]
    const float* omx;
    const float* omy;
    const float* A1;           // [nSp][3]
    const float* A2;
    const float* e0s;          // [nSp][6]
    const float* lamM;         // [nSm]
    const void* VmT;           // GEMM 1 second operand (N x K = V^T)
    const void* Vm;            // GEMM 2 second operand (N x K = V)
    const void* Sp;            // scattering second operand (S^+, symmetric)
    const float* WpN;          // [nSp][dP]: restriction to the coarse space
    const float* WpNT;         // [dP][nSp]: prolongation
    bool bf16;                 // operand type: BF16, else FP32 (TF32 MMA)
};

// Raw device pointers of an assembled system (owned by rte_handle).
struct DevSystem {
    int m;                     // mesh: m x m squares
    int tpb_A = 256;           // threads per block of the transport apply (autotuned)
    int tpb_even = 256;        // threads per block of the even gather (autotuned)
    int nRp, nRm, nSp, nSm, dP, dM, nnz;
    const double* ell4;        // M_t^+, M_s^+, B_x, B_y in ELL form [4][7][nRp]
    double g, c, gamma;
    // spatial
    const int* cell_nodes;     // [nRm][3]
    const double* cell_D;      // [nRm][6]  D1[a], D2[a]
    const double* cell_at;     // [nRm]     |T| sigma_t
    const double* cell_as;     // [nRm]     |T| sigma_s
    const int* adj_ptr;        // [nRp+1]   node -> incident cells
    const int* adj_cell;
    const int* adj_loc;
    const int* st_ptr;         // [nRp+1]   7-point stencil
    const int* st_col;         // [nnz]
    const int* st_diag;        // [nRp]
    const double* sval;        // [kSlots][nnz]
    const float* sval_f;       // [kSlots][nnz] (FP32 copy)
    // angular
    const double* ang_m;       // [nSp]
    const double* ang_omx;     // [nSp]
    const double* ang_omy;     // [nSp]
    const double* ang_A1;      // [nSp][3]
    const double* ang_A2;      // [nSp][3]
    const double* ang_MSm;     // [nSp][9]
    const double* ang_MSm_inv; // [nSp][9]
    const int* inflow_half;    // [4 faces][nSp]: which triangle of pair k (0: K_k,
                               // 1: -K_k) enters the domain through the face
    const double* e0s;         // [nSp][6]  gamma a11, gamma a12, gamma a22, omx, omy, m
    const double* Sp;          // [nSp][nSp]
    const double* Sm;          // [nSm][nSm]
    const double* Vm;          // [nSm][nSm]  eigenvectors of (S^-, M_S^-) as columns
    const double* VmT;         // [nSm][nSm]
    const double* lamM;        // [nSm]       non-increasing
    const double* WmN;         // [nSm][dM]
    const double* WmNT;        // [dM][nSm]
    const double* WpN;         // [nSp][dP]
    const double* WpNT;        // [dP][nSp]
    const double* lamP;        // [nSp]
    // coarse matrix E_c: blocks [nnz][dP][dP] and inverse diagonal blocks
    const double* ec_val;
    const double* ec_dinv;     // [nRp][dP][dP]
    DevLow lo;                 // mixed-precision copies (null in FP64 mode)
    // E_0 level-0 stencil coefficients per direction, ELL [7][nRp][nSp]
    const double* e0coef;
    // direct route of E_0^{-1}: inverses of the row Schur complements of every
    // direction block, [nSp][m+1][ld][ld] (e0_direct.cu); one of the two set
    bool e0_direct = false;
    const float* e0lu32 = nullptr;
    const double* e0lu64 = nullptr;
    // direct route of E_c^{-1}: inverses of its row Schur complements,
    // [m+1][(m+1) d][ld] (ec_direct.cu); one of the two set
    bool ec_direct = false;
    const float* eclu32 = nullptr;
    const double* eclu64 = nullptr;
    const double* ec_ell;      // E_c in ELL form [7][nRp][dP][dP], blocks transposed
    // digit slices of the constant second operands for the split FP64 GEMM
    int split_S;               // 0: FP64 GEMMs on the FP64 units
    const void* sl_VmT;        // [S][nSm][nSm] BF16 (+ exponents below)
    const int* ex_VmT;
    const void* sl_Vm;
    const int* ex_Vm;
    const void* sl_Sp;
    const int* ex_Sp;
    const void* sl_Sm;         // S^- (the PCG route's K^- in the mixed modes)
    const int* ex_Sm;
    const double* mk_rinv;     // [nRm][nSm] 1 / (at - lam as), eigenbasis route
    MGDevice e0mg;             // multigrid of the E_0 direction blocks
    MGDevice ecmg;             // multigrid of E_c
};

// Status words written by persistent kernels (bounded waits, iteration counts).
struct SolveStatus {
    int iterations;
    int timed_out;
    int converged;
    int pad;
    long long active_quads;   // E_0 quad kernel: active quads summed over its V-cycles
};

// ------------------------------------------------------------- launchers
// C = alpha * op(A B) + beta * C for row-major A (M x K), B (K x N),
// C (M x N); epi selects a per-element factor applied to A B:
//   0: none
//   1: 1 / (at[r % rows] - lam[c] * as[r % rows])           eigenbasis of M-K
//   2: 1 / (at - lam as) - 1 / at                            Lemma precond.
void gemm_f64(cudaStream_t s, int M, int N, int K, const double* A, int lda,
              const double* B, int ldb, double* C, int ldc, double alpha,
              double beta, int epi, const double* at, const double* as,
              const double* lam, int rows);

// Z = A U (eq. AR): even (nrhs x nRp x nSp) -> odd (nrhs x nRm x nSm)
void apply_A(cudaStream_t s, const DevSystem& d, const double* U, double* Z,
             int nrhs);

void apply_A_lo(cudaStream_t s, const DevSystem& d, const float* U, void* Z, bool bf16,
                int nrhs);
void apply_even_lo(cudaStream_t s, const DevSystem& d, const float* Zp, const float* X,
                   const float* V, float* Y, int nrhs, int flags);
void dot_per_rhs(cudaStream_t s, const float* x, const float* y, size_t len, int nrhs,
                 double* partial, double* out);
void axpby_per_rhs(cudaStream_t s, const float* x, float* y, size_t len, int nrhs,
                   const double* a, double ca, const double* b, double cb);
// x uniform in [-1, 1), a counter-based function of (seed, index)
void fill_uniform(cudaStream_t s, double* x, size_t n, unsigned long long seed);
void convert(cudaStream_t s, const double* x, float* y, size_t n);

// Restriction qc = x W (rows x nSp times nSp x dP) and prolongation
// x = beta x + uc W^T, one warp per row, for dP <= 16 (false otherwise: the
// caller falls back to the general GEMM); W, WT in FP64 or FP32 (products and
// sums in that type, FP64 vectors at the interface).
bool restrict_rows(cudaStream_t s, int rows, int nSp, int dP, const double* x, const double* W,
                   const float* W32, double* qc);
bool prolong_rows(cudaStream_t s, int rows, int nSp, int dP, const double* uc, const double* WT,
                  const float* WT32, double* x, double beta);
void convert(cudaStream_t s, const float* x, double* y, size_t n);
void convert(cudaStream_t s, const float* x, __nv_bfloat16* y, size_t n);
void convert(cudaStream_t s, const double* x, __nv_bfloat16* y, size_t n);

// Y = [A^T Zp] + [M^+ X + R X] - [M_s^+ V] (terms selected by flags):
// flags bit0: A^T Zp, bit1: M^+ X + R X, bit2: - M_s^+ V (V = X S^+).
void apply_even(cudaStream_t s, const DevSystem& d, const double* Zp,
                const double* X, const double* V, double* Y, int nrhs,
                int flags);

// Y = M_t^- Z M_S^- - G with G already = M_s^- Z S^- scaled: here
// Y = at_j (Z_j M_S^-) - as_j G_j  (G = Z S^-).
void mk_combine(cudaStream_t s, const DevSystem& d, const double* Z,
                const double* G, double* Y, int nrhs);

// Y = (B M_S^{-1}) / at  (high-order part of eq. MmKprecond).
void mk_minv_scale(cudaStream_t s, const DevSystem& d, const double* B,
                   double* Y, int nrhs);

// q_{r,i,k} = (M q_nodal_r)_i m_k
// q += the inflow part of l^+ for data g [nrhs][4][m+1][2 nSp] (rte_inflow)
void inflow_source(cudaStream_t s, const DevSystem& d, const double* g, double* q, int nrhs);
void rhs_source(cudaStream_t s, const DevSystem& d, const double* qn,
                double* q, int nrhs);

// per-RHS reductions over blocks of length len: out[r] = sum x*y
// (deterministic two-pass; partial must hold nrhs * 1024 doubles)
void dot_per_rhs(cudaStream_t s, const double* x, const double* y, size_t len,
                 int nrhs, double* partial, double* out);

// y = a[r] * x + b[r] * y per RHS block (a, b device arrays or nullptr for
// the constants ca, cb).
void axpby_per_rhs(cudaStream_t s, const double* x, double* y, size_t len,
                   int nrhs, const double* a, double ca, const double* b,
                   double cb);

// E_0^{-1} B by one persistent CG over all (rhs, direction) columns.
int e0_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X,
          int nrhs, double tol, int maxit, void* work, size_t work_bytes,
          SolveStatus* status_dev);
size_t e0_cg_work_bytes(const DevSystem& d, int nrhs);
// The same in FP32 (vectors and coefficients), FP64 right-hand side and
// solution at the interface, reductions in FP64.
int e0_cg_lo(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
             double tol, int maxit, void* work, size_t work_bytes, SolveStatus* status_dev);

// Direct route of E_0^{-1} (e0_direct.cu): whether the mesh fits it, the
// bytes of its factor and of the setup scratch, the factorisation (setup)
// and the solve X = E_0^{-1} B (all right-hand sides, exact up to rounding).
bool e0_direct_fits(int m);
size_t e0_direct_bytes(int m, int nSp, bool fp64);
size_t e0_direct_scratch_bytes(int m, int nSp);
int e0_direct_factor(cudaStream_t s, const DevSystem& d, double* scratch, float* out32,
                     double* out64);
int e0_direct_solve(cudaStream_t s, const DevSystem& d, const double* B, double* X, int nrhs,
                    bool fp64);
// Reads and clears the flag a timed-out factor-block wait sets (synchronises s).
int e0_direct_error(cudaStream_t s);
// Limit of one such wait on the current device (SM clock cycles).
int e0_set_wait_cycles(long long cycles);

// Direct route of E_c^{-1} (ec_direct.cu): row length of its factor, bytes,
// whether the mesh fits, and the factorisation (solver: a cusolverDnHandle_t).
int ec_direct_ld(int m, int d);
size_t ec_direct_bytes(int m, int d, bool fp64);
bool ec_direct_fits(int m, int d);
int ec_direct_factor(cudaStream_t s, void* solver, const DevSystem& d, float* out32,
                     double* out64);

// E_c^{-1} B by one persistent preconditioned CG per RHS (a V-cycle of the
// multigrid, or the factor's sweeps on the direct route).  f32_products: the
// CG's own E_c products in FP32 from the multigrid's level 0 (multigrid
// route only; for loose tolerances, where their rounding is far below the
// tolerance), the recurrences staying FP64.
int coarse_cg(cudaStream_t s, const DevSystem& d, const double* B, double* X,
              int nrhs, double tol, int maxit, void* work, size_t work_bytes,
              SolveStatus* status_dev, bool f32_products = false);
size_t coarse_cg_work_bytes(const DevSystem& d, int nrhs);

// y = E_c x
void coarse_apply(cudaStream_t s, const DevSystem& d, const double* X,
                  double* Y, int nrhs);

// coef[dir][i][k] = sum_s e0s[k][s] ell6[s][dir][i]: the E_0 direction-block
// entries in ELL form (ell6: the six spatial parts K11, K12, K22, B_x, B_y,
// M_t^+ in ELL form, FP64)
void e0_coefficients(cudaStream_t s, int nRp, int nSp, const double* ell6, const double* e0s,
                     double* coef, float* coef_f);

// Assembly of S^+ and S^- by the quadrature rule (setup).
struct QuadDev {
    const double *near_pts, *near_w, *near_psi, *far_pts, *far_w, *far_psi;
    const int *near_ptr, *near_idx;
    int qn, qf;
};
void assemble_scattering(cudaStream_t s, int n, double g, const QuadDev& q,
                         double* Sp, double* Sm);

int device_sm_count();

// Phase trace of the persistent solver kernels: when buf is set, block 0
// records %globaltimer after every grid barrier (cap entries per launch).
void set_phase_trace(unsigned long long* buf, int cap);
// Limit of each grid-barrier wait of the persistent kernels launched after
// the call (nanoseconds; 0 restores the 2 s default).
void set_wait_limit_ns(unsigned long long ns);

// Count of kernel launches issued by the library (host-side counter).
void count_launches(long long n);
long long launches_total();

}  // namespace rte
