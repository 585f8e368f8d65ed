// Internal declarations shared by the libredo translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/redo.h"

namespace redo {

// ----------------------------------------------------------------------------
// Complex arithmetic on interleaved pairs (double2 / float2)
// ----------------------------------------------------------------------------
template <typename R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float> { using T = float2; };
template <typename R> using cplx = typename C2<R>::T;

template <typename R> __host__ __device__ __forceinline__ cplx<R> cmake(R re, R im) {
  cplx<R> z; z.x = re; z.y = im; return z;
}
// acc += a * b
template <typename R> __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// ----------------------------------------------------------------------------
// Table handle
// ----------------------------------------------------------------------------
constexpr int kMaxK = 64;
constexpr int kMaxN = 1024;     // N > 64 takes the global-memory (large-N) path
constexpr int kSmallN = 64;


}  // namespace redo

struct redo_table {
  int32_t N, K, base, digits;      // as stored: a level table has base = levels, digits = 1
  int32_t digit_base, digit_count; // the digit decomposition the operators were built from
  int64_t levels;
  int64_t entries;            // K * digits * base
  double dt;
  double lo[redo::kMaxK], hi[redo::kMaxK], delta[redo::kMaxK];
  double* d_lo;               // device copies [K]
  double* d_delta;            // [K]
  double2* T64;               // [entries][N][N], term 0 digit 0 folded with D
  double2* D64;               // [N][N]
  double2* Dh64;              // [N][N] half drift exp(-i dt/2 H0) of a symmetric-split table, else nullptr
  int strang;                 // calls use the symmetric step D_h E_{K-1} ... E_0 D_h
  int h0_diagonal;            // H0 (so D_h) is diagonal
  float2* T32;                // [entries][N][N] or nullptr
  int32_t* hk_ptr;            // CSR of the control operators: row pointers [K][N+1]
  int32_t* hk_col;            // column indices [nnz]
  int32_t* hk_row;            // row index of every nonzero [nnz] (COO view of the same CSR)
  double2* hk_val;            // values [nnz]
  int64_t hk_nnz;
  int32_t* hk_xmask;          // [K] m_k when every H_k has its one nonzero of row r at r ^ m_k, else nullptr
  float2* hk_xval;            // [K][N] that nonzero, H_k[r][r ^ m_k], in FP32
  void* tc_planes;            // tensor-core planes or nullptr
  size_t tc_bytes;
  int tc_nb;                  // operand block height of the large-N planes (128 or 256)
  double* sz64;               // [K][N] diagonals of the species' S_kz (amplitude/phase calls), or nullptr
  int32_t* h0_pairs;          // host: (row, column) of every off-diagonal nonzero of H0
  int64_t h0_npairs;
  cudaStream_t build_stream;
  int num_sms;
};

namespace redo {

// ----------------------------------------------------------------------------
// Event timing of a phase of launches on a stream while profiling is enabled
// (redo_profile_enable); a no-op otherwise.
// ----------------------------------------------------------------------------
struct ProfScope {
  int phase;
  cudaEvent_t a, b;
  cudaStream_t s;
  ProfScope(int phase, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;
};

// ----------------------------------------------------------------------------
// Error plumbing
// ----------------------------------------------------------------------------
redo_status set_error(redo_status s, const char* fmt, ...);
redo_status cuda_error(cudaError_t e, const char* what);
#define REDO_CUDA_TRY(call)                                   \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::redo::cuda_error(_e, #call); \
  } while (0)

// ----------------------------------------------------------------------------
// Launchers (each defined in the translation unit that holds its kernels)
// ----------------------------------------------------------------------------

// Quantizer (kernels_small.cu).
cudaError_t launch_quantize(const double* u, int64_t count, int K, const double* lo,
                            const double* delta, int64_t levels, int32_t* q, int64_t* status,
                            cudaStream_t s);

// Table: entries e = (k*digits + j)*base + c, plus the drift (entry index -1).
cudaError_t launch_table_expm(const redo_table* t, const double2* H0, const double2* Hk,
                              cudaStream_t s);
cudaError_t launch_table_fold_drift(const redo_table* t, cudaStream_t s);
cudaError_t launch_to_fp32(const double2* src, float2* dst, int64_t count, cudaStream_t s);
// Level operators E[k][q] (process 3) from the digit table; E has K*levels entries.
cudaError_t launch_table_expand(const redo_table* t, double2* E, cudaStream_t s);

// Segmented chain products for N <= 64 (SIMT, FP64 or FP32).
// Amplitude/phase calls (pd non-null): every step opens with the diagonal factor
// P_n = Z_n^dag Z_{n-1} (pd[b][n][0..N)).  The N <= 64 SIMT chains carry it as a factor
// (fps = K*digits + 1); the tensor-core chains apply it in an epilogue and the large-N chains
// between launches (fps = K*digits).
struct ChainPlan {
  int64_t B, M;
  int64_t F;          // factors per pulse = M*fps
  int64_t seg_len;    // factors per segment
  int64_t S;          // segments per pulse
  int64_t fps = 0;    // factors per step
  const double2* pd = nullptr;
  const float2* pd32 = nullptr;   // the same diagonals in FP32 (tensor-core chains)
};
ChainPlan plan_chain(const redo_table* t, int64_t B, int64_t M, int prec, bool phase = false);
size_t chain_workspace_bytes(const redo_table* t, const ChainPlan& p, int prec);
// keep non-null: every segment's partial product after each factor is also written to
// keep[chain][t] (N x N, the chain precision).
cudaError_t launch_chain_segments(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                  int prec, void* seg_out, int64_t* status, cudaStream_t s, void* keep = nullptr);
cudaError_t launch_chain_combine(const redo_table* t, const ChainPlan& p, int prec,
                                 const void* seg_in, void* prod_out, int64_t* status,
                                 cudaStream_t s);
// Segments of exactly `steps_per_segment` time steps (re-unitarisation period).
ChainPlan plan_chain_aligned(const redo_table* t, int64_t B, int64_t M, int64_t steps_per_segment,
                             bool phase = false);
// One or more Newton-Schulz polar steps on `count` N x N matrices (in may equal out
// when the precisions match); prec_in/prec_out are REDO_FP64 or REDO_FP32.
cudaError_t launch_polar(const redo_table* t, int prec_in, int prec_out, const void* in, void* out,
                         int64_t count, int iters, cudaStream_t s);

// The same Newton-Schulz steps on complex128 matrices (N <= 64), in FP64 or FP32 arithmetic.
cudaError_t launch_polar_c128(int N, int prec_arith, const double2* in, double2* out, int64_t count, int iters,
                              cudaStream_t s);

// Tensor-core chains (kernels_tc.cu), N = 64, split-FP16.
size_t tc_planes_bytes(const redo_table* t);
cudaError_t launch_build_tc_planes(const redo_table* t, cudaStream_t s);
ChainPlan plan_chain_tc(const redo_table* t, int64_t B, int64_t M);
cudaError_t launch_chain_tc(const redo_table* t, const int32_t* q, const ChainPlan& p,
                            void* seg_out, int64_t* status, cudaStream_t s);

cudaError_t launch_grape_step(double* u, const double* g, int64_t count, int64_t per_pulse, int K,
                              const double* lo, const double* delta, int64_t levels, double step,
                              const double* scale, cudaStream_t s);

cudaError_t launch_grape_adam(double* u, const double* g, double* m, double* v, int64_t count, int K,
                              const double* lo, const double* delta, int64_t levels, int step, double lr,
                              double b1, double b2, double eps, cudaStream_t s);

// Projected L-BFGS ascent step of the GRAPE loop (kernels_lbfgs.cu): per pulse the accepted
// point, its gradient, the direction, a ring of `hist` (s, y) pairs and the scalars.
struct LbfgsState {
  double *u, *g, *d, *S, *Y, *rho, *F, *alpha;
  int *count, *head;
};
size_t lbfgs_state_bytes(int64_t B, int64_t n, int hist);
LbfgsState lbfgs_state_layout(void* base, int64_t B, int64_t n, int hist);
cudaError_t launch_lbfgs_step(const redo_table* t, double* u, const double* g, const double* F, int64_t B,
                              int64_t M, int hist, int first, double step0, double c1, void* state,
                              double* u_best, double* F_best, cudaStream_t s);

// GRAPE gradient (kernels_grad.cu).
cudaError_t launch_grad_scan(const redo_table* t, int64_t B, int64_t S, int prec, const void* seg,
                             const double2* U_target, int target_batched, void* Pck, void* Rck,
                             double2* tau, double* F_out, cudaStream_t s);
// With p.pd set (amplitude/phase calls) the sweep also records Tz[b][n][k] = Tr(S_kz P R) at
// every step boundary n = 0..M ([B][M+1][K]).
cudaError_t launch_grad_sweep(const redo_table* t, const int32_t* q, const ChainPlan& p, int prec,
                              const void* Pck, const void* Rck, const double2* tau, double* grad,
                              int64_t* status, cudaStream_t s, double2* Tz = nullptr, const void* keep = nullptr);

// State simulation (kernels_sim.cu).
cudaError_t launch_state_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                              const double2* psi0, const double2* psiT, int batched, double* F_out, double* grad,
                              int64_t* status, cudaStream_t s);
// <O>(t_n) of psi_n = U_n ... U_1 psi0 for N >= 64, one CTA per pulse streaming the operators
// (the forward sweep of the state-transfer kernel); expect [B][M+1].
cudaError_t launch_sim_stream(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                              const double2* psi0, int psi0_batched, const double* obs, double* expect,
                              int64_t* status, cudaStream_t s);
cudaError_t launch_levels_closed_form(const redo_table* t, const int32_t* xm, const double2* xh, const double* xa,
                                      double2* E, cudaStream_t s);
cudaError_t launch_expect_diag(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                               const double* rho, const double* obs, double* expect, double* mean,
                               int64_t* status, cudaStream_t s);
cudaError_t launch_sim_state(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                             int prec, const double2* psi0, int psi0_batched, const double* obs,
                             double* expect, int64_t* status, cudaStream_t s);

// Warm-start MLP (kernels_mlp.cu).  `acts` and `work` end with scratch for the GEMMs' split
// operand planes (256-byte aligned after the activations / the two gradient buffers).
int64_t mlp_param_count(int L, const int32_t* sizes);
size_t gemm_plane_bytes(int64_t M, int64_t N, int64_t K);
size_t mlp_forward_plane_bytes(int L, const int32_t* sizes, int64_t batch);
size_t mlp_backward_plane_bytes(int L, const int32_t* sizes, int64_t batch);
cudaError_t mlp_forward(int L, const int32_t* sizes, const float* params, const float* x,
                        int64_t batch, float* acts, float* y, cudaStream_t s);
cudaError_t mlp_backward(int L, const int32_t* sizes, const float* params, const float* x,
                         int64_t batch, const float* acts, const float* y_target, float* grads,
                         double* loss, float* work, cudaStream_t s);
cudaError_t mlp_adam(int64_t count, float* p, const float* g, float* m, float* v, int step, float lr,
                     float b1, float b2, float eps, cudaStream_t s);

// Large-N path (kernels_large.cu), 64 < N <= 1024.
}  // namespace redo
#include <vector>
namespace redo {
cudaError_t large_table_build(redo_table* t, const double2* H0, const double2* Hk,
                              const std::vector<double>& hnorm1, double h0norm1, cudaStream_t s);
ChainPlan plan_chain_large(const redo_table* t, int64_t B, int64_t M);
cudaError_t large_table_expand(const redo_table* t, double2* E, cudaStream_t s);
size_t large_prop_workspace(const redo_table* t, const ChainPlan& p, int prec, bool reunit);
cudaError_t large_propagate(const redo_table* t, const int32_t* q, const ChainPlan& p, int prec,
                            bool reunit, void* ws, void** result, int* result_prec,
                            int64_t* status, cudaStream_t s);
size_t large_grad_workspace(const redo_table* t, const ChainPlan& p, int prec);
// With p.pd set (amplitude/phase calls, segments of whole steps) the reverse sweep also records
// Tz [B][M+1][K] at the step boundaries and undoes the step diagonals.
// reunit: every segment product is replaced by its polar factor (one Newton-Schulz step in the
// chain precision) before the checkpoint and costate scans.
cudaError_t large_grad(const redo_table* t, const int32_t* q, const ChainPlan& p, int prec,
                       const double2* UT, int tb, double* F_out, double* grad, void* ws,
                       int64_t* status, cudaStream_t s, double2* Tz = nullptr, double* grad_phase = nullptr,
                       bool reunit = false);
// The same Newton-Schulz step on the G FP32 segment products at the start of a gradient workspace
// laid out by large_grad_workspace(t, p, REDO_FP32) (its ping buffers as scratch).
cudaError_t large_reunit_segments_fp32(const redo_table* t, const ChainPlan& p, void* ws, cudaStream_t s);
size_t large_sim_workspace(const redo_table* t, int64_t B);
cudaError_t large_sim(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                      const double2* psi0, int pb, const double* obs, double* expect, void* ws,
                      cudaStream_t s);
cudaError_t large_finish_fp32(const redo_table* t, const ChainPlan& p, bool reunit, void* ws,
                              void** result, int* result_prec, cudaStream_t s);
cudaError_t large_pair_products_fp32(const float2* in, float2* out, int64_t count, int N, cudaStream_t s);
// out[h] = Pck[h-1] Rck[h] (h mod S > 0), Rck[h] (h mod S = 0), h < G, FP32.
cudaError_t large_costate_shift_fp32(const float2* Pck, const float2* Rck, float2* out, int64_t G, int64_t S, int N,
                                     cudaStream_t s);
// out[2s+1] = H[2s] Cs[s], out[2s] = Cs[s] H[2s+1], for 2s+1 < Gf (FP32).
cudaError_t large_half_costates_fp32(const float2* H, const float2* Cs, float2* out, int64_t Gf, int N,
                                     cudaStream_t s);
cudaError_t large_grad_scans_fp32(const redo_table* t, const ChainPlan& p, const double2* UT, int tb,
                                  double* F_out, void* ws, float2** Pck, float2** Rck, double2** tau,
                                  cudaStream_t s);
// Tensor-core large-N path (kernels_tc_large.cu), split FP16, 128 <= N <= 1024.
int tc_large_nb(int N);
size_t tc_large_planes_bytes(const redo_table* t);
cudaError_t launch_build_tc_large_planes(const redo_table* t, cudaStream_t s);
size_t tc_large_prop_workspace(const redo_table* t, const ChainPlan& p, bool reunit);
cudaError_t tc_large_propagate(const redo_table* t, const int32_t* q, const ChainPlan& p, bool reunit,
                               void* ws, void** result, int* result_prec, int64_t* status,
                               cudaStream_t s);
size_t tc_large_grad_workspace(const redo_table* t, const ChainPlan& p);
cudaError_t tc_large_grad(const redo_table* t, const int32_t* q, const ChainPlan& p, const double2* UT,
                          int tb, double* F_out, double* grad, void* ws, int64_t* status,
                          cudaStream_t s, bool reunit = false);

// out_b = A X_b A^dag (adjoint = 0) or A^dag X_b A (adjoint = 1), A = the table's half
// drift, FP64 out (may be X itself); X_b of precision `prec` (REDO_FP64 or REDO_FP32).
// tmp: count FP64 matrices of scratch when H0 is not diagonal (unused, may be NULL, otherwise).
cudaError_t launch_half_drift_conj(const redo_table* t, int prec, const void* X, int64_t count, int adjoint,
                                   double2* out, double2* tmp, cudaStream_t s);
// psi'_b = D_h^dag psi_b for a diagonal half drift (count vectors of N)
cudaError_t launch_half_drift_vec(const redo_table* t, const double2* psi, int64_t count, double2* out,
                                  cudaStream_t s);

// Amplitude/phase controls (kernels_phase.cu).  pd[b][n][a] = exp(i sum_k (phi[b][n][k] -
// phi[b][n-1][k]) sz[k][a]) (phi[b][-1] = 0), the diagonal of Z_n^dag Z_{n-1};
// zf[b][a] = exp(-i sum_k phi[b][M-1][k] sz[k][a]), the diagonal of Z_{M-1} (1 when M = 0).
// With pd32 non-null the diagonals go there in FP32 (pd unused).
cudaError_t launch_phase_diag(const redo_table* t, const double* phi, int64_t B, int64_t M, double2* pd,
                              float2* pd32, double2* zf, cudaStream_t s);
// Per-pulse diagonal drift: pd[b][n][a] = exp(-i dt h[b][a]) for every step n (pd32 non-null:
// FP32 there instead), the step-opening diagonals of a chain whose steps read
// U_n = E_n D diag(exp(-i dt h_b)).
cudaError_t launch_drift_diag(const redo_table* t, const double* h, int64_t B, int64_t M, double2* pd,
                              float2* pd32, cudaStream_t s);
// X_g <- P_n X_g in place for the chains g = (u, s) of a step-aligned plan, n = s*sps + i
// (chains with n >= M untouched); X of precision prec.
cudaError_t launch_phase_rows(int N, int prec, void* X, int64_t G, int64_t S, int64_t sps, int64_t i,
                              int64_t M, const double2* pd, cudaStream_t s);
// out_b = diag(conj(zf_b)) U_T (U_T[b] when batched), FP64: the target of the regrouped chain.
cudaError_t launch_phase_target(int N, int64_t B, const double2* UT, int batched, const double2* zf, double2* out,
                                cudaStream_t s);
// gphi[b][n][k] = (2/N^2) Im(conj(tau_b) (Tz[b][n+1][k] - Tz[b][n][k])), n < M.
cudaError_t launch_phase_grad_finish(int N, int64_t B, int64_t M, int K, const double2* Tz, const double2* tau,
                                     double* gphi, cudaStream_t s);
// Reverse sweep of the large-N phase gradient at offset tt from every chain's end (segments of
// whole steps): where the chain's factor opens step n, record Tz[u][n][k] = Tr(S_kz P R) and undo
// P_n (P <- P_n^dag P, R <- R P_n); tt = -1 records Tz[u][M] at the end of the last segment.
// Tz == nullptr (per-pulse drift diagonals) records nothing and only undoes P_n.
cudaError_t launch_phase_boundary(int N, int prec, void* P, void* Rm, int64_t G, int64_t S, int64_t seg_len,
                                  int64_t F, int64_t tt, int64_t kd, int64_t M, const double2* pd, const double* sz,
                                  int K, double2* Tz, cudaStream_t s);
// out_b = diag(zf_b) X_b in FP64 (X of precision prec; out may not alias X unless FP64).
cudaError_t launch_phase_final(int N, int64_t B, int prec, const void* X, const double2* zf, double2* out,
                               cudaStream_t s);

// C_b = op(A_b) op(B_b) for b < count, FP64 complex N x N, op = conjugate transpose when adj != 0;
// sA / sB are the element strides between consecutive A_b / B_b (0 broadcasts one matrix).
cudaError_t launch_batched_product(int N, int64_t count, const double2* A, int adjA, int64_t sA, const double2* B,
                                   int adjB, int64_t sB, double2* C, cudaStream_t s);

cudaError_t launch_finalize(const redo_table* t, int64_t B, int prec, const void* prod,
                            void* U_out, const double2* U_target, double* F_out, double2* tau_out,
                            cudaStream_t s);

}  // namespace redo
