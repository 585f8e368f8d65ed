/*
 * redo.h -- C ABI of libredo, a GB300 (sm_103a) implementation of REDO,
 * "Rapid Exponentiation using Discrete Operators" (Bhole & Mahesh,
 * arXiv:1707.02162).
 *
 * The library evaluates piecewise-constant quantum propagators
 *     U = U_M ... U_2 U_1,   U_n = E_{K-1,n} ... E_{0,n} D,   D = exp(-i dt H0)
 * (Section III, Eq. propUn, with the drift split off as in the Dirac-frame
 * step formula), where every per-term factor
 *     E_{k,n} = exp(-i dt u_hat_{kn} H_k)
 * is not exponentiated but assembled as a product of precomputed discrete
 * operators (Section II, processes 1 and 2, Eqs. cgrain, redoform, exp2prod).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Complex matrices are interleaved complex128 (re, im pairs of double),
 *    row-major N x N, contiguous; batches are outermost.  This is the memory
 *    layout of a contiguous torch.complex128 tensor.
 *  - Unless stated otherwise every array argument is DEVICE memory owned by the
 *    caller.  The only library-owned object is the opaque redo_table.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work on it and return without synchronising, except
 *    redo_build_table and redo_table_free, which synchronise `stream`.
 *  - Host-detectable errors (null pointers, bad sizes, non-Hermitian input,
 *    unsupported precision for a size) return a nonzero redo_status before
 *    anything is enqueued; redo_last_error() then describes the error
 *    (thread-local string, valid until the next call on the same thread).
 *  - Device-detected conditions are accumulated into a caller-provided device
 *    array `dev_status` of REDO_STATUS_WORDS int64 counters (see
 *    redo_status_word); the caller zeroes it and reads it after the stream
 *    has been synchronised.  Kernels never trap or assert.
 *  - Index conventions: the control array u and the level array q have shape
 *    [B][M][K] (pulse, time step, control term), row-major.  Time step 0 is
 *    applied first, i.e. it is the rightmost factor of the chain.
 */
#ifndef REDO_H
#define REDO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  REDO_OK = 0,
  REDO_ERR_INVALID = 1,        /* bad argument: null pointer, size, range        */
  REDO_ERR_NOT_HERMITIAN = 2,  /* H0 or some H_k is not Hermitian                */
  REDO_ERR_OOM = 3,            /* device allocation failed (build_table only)    */
  REDO_ERR_CUDA = 4,           /* a CUDA runtime call failed                     */
  REDO_ERR_UNSUPPORTED = 5     /* valid request this build does not implement    */
} redo_status;

/* Arithmetic of the product chain.  The table master copy, the quantizer and
 * the fidelity reduction are always FP64. */
typedef enum {
  REDO_FP64 = 0,     /* complex FP64 products (plain REDO)                       */
  REDO_FP32 = 1,     /* complex FP32 products on the FP32 pipes                  */
  REDO_FP16X3 = 4    /* tensor cores: each operand split hi + 2^-11-scaled lo in
                        FP16, three products hi*hi + (hi*lo + lo*hi) with FP32
                        accumulation                                            */
} redo_precision;

/* Device status counters (int64 each), indices into dev_status. */
typedef enum {
  REDO_STATUS_NONFINITE = 0,   /* control coefficients that were NaN or +-Inf    */
  REDO_STATUS_SATURATED = 1,   /* coefficients clamped to the ends of the grid   */
  REDO_STATUS_TIMEOUT = 2,     /* a bounded device wait gave up (should be 0)    */
  REDO_STATUS_BADINDEX = 3,    /* a level index outside [0, levels) was seen     */
  REDO_STATUS_WORDS = 4
} redo_status_word;

typedef struct redo_table redo_table;

/*
 * redo_build_table -- one-time discrete-operator table (Section II, process 1).
 *
 * Stores, for every control term k < K, digit j < digits and digit value
 * c < base, the operator
 *     T[k][j][c] = exp(-i dt theta_kjc H_k),
 *     theta_k0c = lo[k] + c delta_k,   theta_kjc = c base^j delta_k  (j >= 1),
 *     delta_k   = (hi[k] - lo[k]) / (base^digits - 1),
 * i.e. Eq. (redoform) with the c b^j dt scaling of the worked example of
 * Section II and the grid offset lo[k] carried by digit 0, so that
 *     prod_j T[k][j][c_j] = exp(-i dt (lo[k] + q delta_k) H_k)
 * for the level q = sum_j c_j base^j.  The drift step D = exp(-i dt H0) is
 * folded into the digit-0 operators of term 0 (T[0][0][c] <- T[0][0][c] D).
 * Exponentials are FP64 scaling-and-squaring Taylor series on the GPU.
 *
 *  N        Hilbert-space dimension, a power of two, 2 <= N <= 1024 (N > 64: FP64
 *           and FP32 chains run as batched GEMMs, one launch per chain step;
 *           REDO_FP16X3 chains as persistent tensor-core sweeps).
 *  K        number of control terms, 1 <= K <= 64.
 *  dt       time step in seconds (> 0).
 *  H0       device, complex128 [N][N], Hermitian drift (rad/s).
 *  Hk       device, complex128 [K][N][N], Hermitian control operators.
 *  lo, hi   HOST double [K], ends of each coefficient's level grid (lo < hi).
 *  base     digit base b >= 2;  digits d >= 1;  base^digits <= 2^24 levels.
 *  flags    REDO_TABLE_FP32 also builds the FP32 copy used by REDO_FP32;
 *           REDO_TABLE_FP16X3 also builds the split-FP16 operand planes used
 *           by REDO_FP16X3 (N = 64, or 128 <= N <= 1024 where two plane sets,
 *           for left and right products, are stored).  The FP64 copy is always built.
 *           REDO_TABLE_LEVELS applies process 3 of Section II to every level:
 *           after the digit table is built, each level's operator
 *           E[k][q] = T[k][d-1][c_{d-1}] ... T[k][0][c_0] is evaluated once and
 *           stored, and the table then holds K x levels operators (reported by
 *           redo_table_info as base = levels, digits = 1), so a time step costs
 *           K products instead of K*digits.  K * levels * N^2 * 16 bytes (the
 *           FP64 copy) must stay below 200 GiB; the FP32 copy and the split-FP16
 *           planes, when requested, add half and (N > 64: two sets of) half of that.
 *           REDO_TABLE_STRANG makes every call on the table use the symmetric step
 *           S_n = D_h E_{K-1} ... E_0 D_h with D_h = exp(-i dt/2 H0) (the drift split
 *           evenly around the control factors instead of applied once per step; the
 *           second-order variant of the Section III step).  The table also stores D_h;
 *           propagators are D_h (U_M ... U_1) D_h^dag of the folded chain, fidelities and
 *           gradients use the target D_h^dag U_T D_h, and redo_simulate (which then needs
 *           a diagonal H0) starts the folded chain from D_h^dag psi0.  The workspace of
 *           each call grows by B FP64 matrices (two sets when H0 is not diagonal).
 *  stream   stream for the build; synchronised before returning.
 *  out      receives the handle; free with redo_table_free.
 * Errors: REDO_ERR_INVALID, REDO_ERR_NOT_HERMITIAN (relative tolerance 1e-12
 * on max |H - H^dag|), REDO_ERR_OOM, REDO_ERR_CUDA.
 */
#define REDO_TABLE_FP32 0x1u
#define REDO_TABLE_FP16X3 0x2u
#define REDO_TABLE_LEVELS 0x4u
#define REDO_TABLE_STRANG 0x8u
redo_status redo_build_table(int32_t N, int32_t K, double dt, const void* H0, const void* Hk,
                             const double* lo, const double* hi, int32_t base, int32_t digits,
                             uint32_t flags, void* stream, redo_table** out);

/* Releases the table's device memory (synchronises the build stream). */
redo_status redo_table_free(redo_table* t);

/*
 * redo_table_info -- sizes of a table (host call, no device work).
 * Any output pointer may be NULL.  `entries` = K*digits*base operators.
 */
redo_status redo_table_info(const redo_table* t, int32_t* N, int32_t* K, int32_t* base,
                            int32_t* digits, int64_t* levels, int64_t* entries);

/*
 * redo_table_copy -- copy the FP64 table (device, complex128 [K][digits][base][N][N],
 * drift folded into term 0 digit 0) and/or the drift D (device, complex128 [N][N])
 * into caller buffers.  Either destination may be NULL.  Asynchronous on stream.
 */
redo_status redo_table_copy(const redo_table* t, void* table_out, void* drift_out, void* stream);

/*
 * redo_quantize -- coarse-grain coefficients to level indices (Eq. cgrain).
 *
 * q[b][n][k] = clamp(rint((u[b][n][k] - lo[k]) / delta_k), 0, levels - 1),
 * computed with one IEEE FP64 subtract and one IEEE FP64 divide (no fused
 * multiply-add) and round-half-to-even, so the result is bit-identical to any
 * IEEE implementation of the same formula.  (Values farther from a tie than
 * the error bound of an FP32 estimate of the quotient are decided by that
 * estimate, which gives the same level; the FP64 arithmetic decides the rest.)
 * NaN/Inf coefficients give q = 0 and count in dev_status[REDO_STATUS_NONFINITE];
 * out-of-range coefficients are clamped and counted in
 * dev_status[REDO_STATUS_SATURATED].
 *
 *  u    device double [B][M][K];  q  device int32 [B][M][K] (may not alias u).
 *  dev_status  device int64 [REDO_STATUS_WORDS] or NULL.
 */
redo_status redo_quantize(const redo_table* t, const double* u, int64_t B, int64_t M, int32_t* q,
                          int64_t* dev_status, void* stream);

/*
 * redo_propagate -- REDO propagators of B pulses (Section II process 2,
 * Section III chain U = U_M ... U_1).
 *
 * For each pulse b, multiplies the M*K*digits gathered table operators in time
 * order.  The chain is cut into segments whose products are formed in
 * parallel and then multiplied in order (association changes only rounding).
 *
 *  q           device int32 [B][M][K] level indices (from redo_quantize).
 *  prec        REDO_FP64, REDO_FP32 or REDO_FP16X3 (the last needs the table
 *              built with REDO_TABLE_FP16X3).
 *  reunit_every  R >= 0.  R = 0: no re-unitarisation.  R > 0: segments are cut
 *              at every R-th time step and each segment product -- the
 *              propagator of R consecutive steps -- is replaced by its unitary
 *              polar factor (one Newton-Schulz step P <- P(3I - P^dag P)/2 in
 *              the chain precision), and each pulse product gets one more
 *              Newton-Schulz step in FP64 before the fidelity.  This removes
 *              the norm drift of reduced-precision chains; R > M acts as R = M.
 *  U_out       device complex128 [B][N][N]; receives U_b.  May be NULL if F is wanted only.
 *  U_target    device complex128 [N][N] or NULL.
 *  F_out       device double [B] or NULL: |Tr(U_target^dag U_b)|^2 / N^2 (FP64 reduction).
 *  tau_out     device complex128 [B] (Tr(U_target^dag U_b)) or NULL.  With U_target, at
 *              least one of F_out and tau_out is required; without it both are left untouched.
 *  workspace   device scratch of at least redo_propagate_workspace() bytes,
 *              256-byte aligned; contents are overwritten.
 *  dev_status  device int64 [REDO_STATUS_WORDS] or NULL.
 * Level indices outside [0, levels) are counted in REDO_STATUS_BADINDEX and
 * replaced by 0.
 */
redo_status redo_propagate(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                           redo_precision prec, int32_t reunit_every, void* U_out,
                           const void* U_target, double* F_out, void* tau_out, void* workspace,
                           size_t workspace_bytes, int64_t* dev_status, void* stream);

/*
 * redo_propagate_steps -- the per-step propagators U_n themselves (Section III's step formula,
 * U_n = E_{K-1,n} ... E_{0,n} D, each E_k assembled from table operators as in Eq. exp2prod),
 * for callers that need every step rather than the chain: e.g. a GRAPE variant of their own,
 * or checking a pulse step by step.
 *  q           device int32 [B][M][K] levels from redo_quantize.
 *  prec        REDO_FP64 or REDO_FP32 (the latter needs REDO_TABLE_FP32); N <= 64.
 *  U_steps     device complex128 [B][M][N][N]: U_steps[b][n] = U_{n+1} of pulse b (step n applied
 *              at time index n, the rightmost factor of the chain for n = 0).  With a
 *              REDO_TABLE_STRANG table these are the symmetric steps D_h E_{K-1} ... E_0 D_h.
 *  workspace   >= redo_propagate_steps_workspace() bytes (zero for REDO_FP64 with a diagonal
 *              or no drift: then NULL is accepted), 256-byte aligned.
 * Level indices outside [0, levels) count in REDO_STATUS_BADINDEX and are replaced by 0.
 * Errors: REDO_ERR_INVALID, REDO_ERR_UNSUPPORTED (N > 64, other precisions), REDO_ERR_CUDA.
 */
redo_status redo_propagate_steps_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                           size_t* bytes);
redo_status redo_propagate_steps(const redo_table* t, const int32_t* q, int64_t B, int64_t M, redo_precision prec,
                                 void* U_steps, void* workspace, size_t workspace_bytes, int64_t* dev_status,
                                 void* stream);

/*
 * redo_reunitarize -- Newton-Schulz steps towards the unitary polar factor, the
 * re-unitarisation the reduced-precision chains apply every reunit_every steps (the paper's
 * chains are exactly unitary; the step keeps finite-precision products on the unitary group):
 *     P <- P (3 I - P^dag P) / 2,   `iters` times,
 * which converges quadratically to P (P^dag P)^(-1/2) when ||P^dag P - I|| < 1 (one step maps
 * an error e of P^dag P - I to about 3e^2/4).
 *  N        matrix dimension, a power of two, 2 <= N <= 64.
 *  prec     arithmetic of the steps, REDO_FP64 or REDO_FP32.
 *  P_in     device complex128 [count][N][N];  U_out device complex128 [count][N][N] (may equal P_in).
 * Errors: REDO_ERR_INVALID, REDO_ERR_UNSUPPORTED, REDO_ERR_CUDA.  Asynchronous on `stream`.
 */
redo_status redo_reunitarize(int32_t N, int64_t count, redo_precision prec, const void* P_in, void* U_out,
                             int32_t iters, void* stream);

/*
 * redo_plan -- the cost model of Section II (host only, no device work).  For a coefficient range
 * [0, omega_max] coarse grained to a grain eps in base b (Eq. cgrain): l is the largest integer
 * with b^l <= eps (b^l = eps when eps is a power of b), m the smallest with b^(m+1) > omega_max;
 * then p = m - l products per coefficient and s = (b - 1)(m - l + 1) stored operators (process 1,
 * identities not counted).  The worked example of Section II (eps = 1, omega_max = 2.6e5, b = 64)
 * gives l = 0, m = 2, p = 2, s = 189.  Comparisons use a relative slack of 1e-12 on eps so that a
 * decimal eps that is a power of b (1e-4 with b = 100) counts as equal.
 * Any output pointer may be NULL.  Errors: REDO_ERR_INVALID (non-positive or non-finite inputs,
 * eps > omega_max, base < 2).
 */
redo_status redo_plan(double omega_max, double eps, int32_t base, int32_t* l, int32_t* m, int32_t* p,
                      int64_t* s);

/*
 * redo_propagate_noalloc -- redo_propagate for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is a deployment variant.
 *
 * Some callers may not call cudaMalloc at all: code running inside a custom
 * allocator's callback, plug-ins whose host application owns the whole device
 * memory pool, or real-time control loops that forbid allocation after
 * start-up.  This entry point needs no workspace: its
 * scratch is a fixed array of REDO_NOALLOC_SCRATCH_BYTES bytes compiled into
 * the library as a device global, which every GPU that loads libredo holds
 * until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  The caller still passes inputs and outputs, with the
 * same meaning, layout and status words as redo_propagate (REDO_FP64 and
 * REDO_FP32 only, no re-unitarisation, N <= 64), symmetric-split tables
 * included.
 *
 *  - Requests whose segment and pulse products cannot fit the array even with
 *    one segment per pulse return REDO_ERR_INVALID with a message naming the
 *    limit.  With one segment per pulse the array holds a segment product and
 *    a pulse product per pulse: about 2*B*N*N*16 bytes for FP64 (half that for
 *    FP32), so at most 256 FP64 pulses of N = 64.  A REDO_TABLE_STRANG table
 *    adds B*N*N*16 bytes for the conjugated products (twice that when H0 is
 *    not diagonal).
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    cudaDeviceReset (or anything else that destroys the device's primary
 *    context) invalidates the kept address, and the library cannot see that
 *    happen: do not call this entry point again on a device after resetting it.
 *  - All calls on a device share the one array and it keeps the previous
 *    call's contents (nothing in it needs to start at zero).  Calls whose
 *    kernels overlap on the GPU -- on different streams or from different host
 *    threads -- race on it; serialise them.
 */
#define REDO_NOALLOC_SCRATCH_BYTES (32u << 20)
redo_status redo_propagate_noalloc(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                                   redo_precision prec, void* U_out, const void* U_target,
                                   double* F_out, void* tau_out, int64_t* dev_status, void* stream);

/*
 * redo_fidelity_grad -- fidelity and its GRAPE gradient (Section III, the
 * gradient ascent of Fig. fc with REDO propagators; the paper prints no
 * gradient formula).
 *
 * F_b = |tau_b|^2 / N^2, tau_b = Tr(U_T^dag U_b), and for every step n and term k
 *     grad[b][n][k] = dF_b/du_kn = (2 dt / N^2) Im( conj(tau_b) Tr(H_k W_nk) ),
 *     W_nk = (E_k ... E_0 D  U_{n-1} ... U_1) U_T^dag (U_M ... U_{n+1} E_{K-1} ... E_{k+1}),
 * the exact derivative of the split model U_n = E_{K-1} ... E_0 D with
 * E_k = exp(-i dt u_kn H_k), evaluated at the quantised coefficients (the
 * quantizer itself is piecewise constant; its derivative is taken as 1).
 * Units: 1/(rad/s) (multiply by Omega for a normalised amplitude).
 *
 *  q, B, M       as for redo_propagate.
 *  U_target      device complex128 [N][N], or [B][N][N] if target_batched != 0.
 *  prec          REDO_FP64 or REDO_FP32, or REDO_FP16X3 for N >= 128 (products;
 *                traces and tau in FP64).
 *  checkpoint_every  C > 0: forward checkpoints every C steps; 0: automatic.
 *  reunit_every  R >= 0.  R = 0: none.  R > 0 (requires R = checkpoint_every): every
 *                checkpoint segment product, the propagator of R consecutive steps, is
 *                replaced by its polar factor (one Newton-Schulz step in the chain
 *                precision, as in redo_propagate) before the checkpoints, costates, tau and
 *                F are formed.  Reduced-precision chains lose norm at ~3e-8 per product; over
 *                thousands of products that lowers F near 1 by more than 1e-6 unless removed.
 *  F_out         device double [B] or NULL;  grad  device double [B][M][K].
 *  workspace     >= redo_fidelity_grad_workspace() bytes, 256-byte aligned.
 * Method: segment products (one per C steps), prefix checkpoints and suffix
 * costates per segment, then one backward sweep per segment that evaluates the
 * traces with the sparse (CSR) form of H_k captured at table build time.  When
 * every forward partial product of the segment chains fits in 24 GiB (N <= 64,
 * and the tensor-core sweeps at N >= 128), the workspace holds them
 * (redo_fidelity_grad_workspace counts them) and the backward sweep reads them;
 * otherwise it undoes each factor with its adjoint (the table operators are
 * unitary), which needs memory only per segment.
 */
redo_status redo_fidelity_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                               const void* U_target, int32_t target_batched, redo_precision prec,
                               int32_t checkpoint_every, int32_t reunit_every, double* F_out, double* grad,
                               void* workspace, size_t workspace_bytes, int64_t* dev_status,
                               void* stream);
redo_status redo_fidelity_grad_workspace(const redo_table* t, int64_t B, int64_t M,
                                         redo_precision prec, int32_t checkpoint_every,
                                         size_t* bytes);

/*
 * redo_simulate -- dynamics along REDO chains (Section IV): for each pulse
 * (noise realisation) b the state psi_n = U_n ... U_1 psi_0 and the expectation
 *     expect[b][n] = <psi_n| O |psi_n> = sum_a obs_diag[a] |psi_n[a]|^2,  n = 0..M,
 * of a diagonal observable (Tr[O rho(t)] with rho = |psi><psi|), plus optionally
 * the final propagator U_M ... U_1.
 *
 * The state is advanced by one matrix-vector product per table operator, in
 * FP64 for REDO_FP64 and FP32 otherwise; U_final, if requested, is computed
 * exactly as redo_propagate(prec, reunit_every) computes U_out.
 *  psi0      device complex128 [N] (or [B][N] if psi0_batched != 0).
 *  obs_diag  device double [N];  expect  device double [B][M+1].
 *  U_final   device complex128 [B][N][N] or NULL.
 *  workspace >= redo_simulate_workspace(..., want_U = U_final != NULL) bytes.
 */
redo_status redo_simulate(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                          redo_precision prec, int32_t reunit_every, const void* psi0,
                          int32_t psi0_batched, const double* obs_diag, double* expect,
                          void* U_final, void* workspace, size_t workspace_bytes,
                          int64_t* dev_status, void* stream);

/*
 * redo_state_grad -- state-to-state GRAPE (Section III's state fidelity, the gradient
 * derived like redo_fidelity_grad's): a_b = <psi_T| U_M ... U_1 |psi0>, F_b = |a_b|^2 and
 * grad[b][n][k] = dF_b/du_kn = 2 dt Im(conj(a_b) <chi| H_k |phi>), phi the state after the last
 * digit factor of term k in step n and chi the target pulled back through the later factors.
 * Costs O(N^2) per factor (matrix-vector products, forward and then reverse, undoing each
 * unitary factor on both vectors), so it is the cheap form of GRAPE for large N.
 *  q            device int32 [B][M][K] levels.
 *  prec         REDO_FP64 or REDO_FP32 (operators of that precision; traces and a in FP64).
 *  psi0, psi_target  device complex128 [N], or [B][N] when batched != 0.
 *  F_out        device double [B] or NULL;  grad device double [B][M][K] or NULL (one of the two).
 *  workspace    >= redo_state_grad_workspace bytes (zero unless the table is a symmetric-split
 *               one, which also needs a diagonal H0).
 * Errors: REDO_ERR_INVALID, REDO_ERR_UNSUPPORTED, REDO_ERR_CUDA.  No synchronisation.
 */
redo_status redo_state_grad_workspace(const redo_table* t, int64_t B, size_t* bytes);
redo_status redo_state_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M, redo_precision prec,
                            const void* psi0, const void* psi_target, int32_t batched, double* F_out,
                            double* grad, void* workspace, size_t workspace_bytes, int64_t* dev_status,
                            void* stream);

/*
 * redo_expect_diag -- e_n = Tr[rho(t_n) O], rho(t_n) = U_n ... U_1 rho (U_n ... U_1)^dag,
 * n = 0..M, for a diagonal initial density matrix rho (mixed or a traceless deviation
 * matrix) and a diagonal observable O: e_n = sum_{r,c} rho_c O_r |(U_n ... U_1)[r][c]|^2.
 * Section IV's order parameter Q of the noisy exotic-freezing study is of this form in the
 * basis where rho(0) = O = sum_i I_ix are diagonal (the Hamiltonian terms passed to
 * redo_build_table are then given in that basis).  N <= 64.
 *  q            device int32 [B][M][K] levels from redo_quantize.
 *  prec         REDO_FP64 or REDO_FP32 (the latter needs REDO_TABLE_FP32); the reduction is FP64.
 *  rho_diag     device double [N];  obs_diag device double [N].
 *  expect       device double [B][M+1] or NULL;  expect_mean device double [B] or NULL:
 *               the mean of e_1 .. e_M (e_0 when M = 0).  At least one of the two.
 * With a symmetric-split table the drift must be diagonal (then e_n equals that of the
 * folded chain).  Errors: REDO_ERR_INVALID, REDO_ERR_UNSUPPORTED (N > 64, other
 * precisions), REDO_ERR_CUDA.  No synchronisation.
 */
redo_status redo_expect_diag(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                             redo_precision prec, const double* rho_diag, const double* obs_diag,
                             double* expect, double* expect_mean, int64_t* dev_status, void* stream);
redo_status redo_simulate_workspace(const redo_table* t, int64_t B, int64_t M,
                                    redo_precision prec, int32_t reunit_every, int32_t want_U,
                                    size_t* bytes);

/*
 * redo_grape_step -- one GRAPE ascent update in place (Section III, Fig. fc):
 *     u[b][n][k] <- clamp(u[b][n][k] + step * s_b * grad[b][n][k], lo[k], hi[k]).
 * `step` is in (rad/s)^2 when grad is dF/du from redo_fidelity_grad.
 *  u device double [B][M][K] (in/out);  grad device double [B][M][K];
 *  step_scale device double [B] (per-pulse factor s_b) or NULL (s_b = 1).
 */
redo_status redo_grape_step(const redo_table* t, double* u, const double* grad, int64_t B,
                            int64_t M, double step, const double* step_scale, void* stream);

/*
 * Learned warm start for GRAPE (no counterpart in the paper): a multilayer
 * perceptron maps problem parameters to an initial pulse.  FP32 master
 * weights, FP32 arithmetic, all device memory caller-owned.
 *
 * Network with `layers` affine maps of widths sizes[0] -> ... -> sizes[layers]
 * (host int32 array): h_0 = x, z_l = h_l W_l^T + b_l, h_{l+1} = GELU(z_l)
 * (exact erf form) for l < layers-1 and y = tanh(z_{layers-1}).  `params` is one
 * flat array holding W_0 (sizes[1] x sizes[0], row-major), b_0, W_1, b_1, ...
 *
 * redo_mlp_sizes: float counts of params, of the activation buffer `acts`
 *   (z and h of every layer for `batch` samples, then scratch for the forward
 *   GEMMs' split BF16 operand planes) and of the backward `work` buffer (two
 *   gradient buffers, then the backward GEMMs' plane scratch).  Host only.
 * redo_mlp_forward: x [batch][sizes[0]] -> y [batch][sizes[layers]], filling acts.
 * redo_mlp_backward: gradients of loss = mean over all entries of
 *   (y - y_target)^2 into grads (same layout as params), using the acts of the
 *   preceding forward call; loss (device double [1], may be NULL) receives the loss.
 * redo_mlp_adam: Adam (bias-corrected, step >= 1) on `count` parameters:
 *   m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
 *   p <- p - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 */
redo_status redo_mlp_sizes(int32_t layers, const int32_t* sizes, int64_t batch,
                           int64_t* params, int64_t* acts, int64_t* work);
redo_status redo_mlp_forward(int32_t layers, const int32_t* sizes, const float* params,
                             const float* x, int64_t batch, float* acts, float* y, void* stream);
redo_status redo_mlp_backward(int32_t layers, const int32_t* sizes, const float* params,
                              const float* x, int64_t batch, const float* acts,
                              const float* y_target, float* grads, double* loss, float* work,
                              void* stream);
redo_status redo_mlp_adam(int64_t count, float* params, const float* grads, float* m, float* v,
                          int32_t step, float lr, float beta1, float beta2, float eps,
                          void* stream);

/*
 * redo_grape_adam_step -- GRAPE ascent with Adam moments (the paper leaves the
 * update rule open): per coefficient
 *     m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *     u <- clamp(u + lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps), lo[k], hi[k]).
 * `lr` is in rad/s (the size of a typical coefficient change); m and v are
 * caller-owned device double [B][M][K], zero before step 1.
 */
redo_status redo_grape_adam_step(const redo_table* t, double* u, const double* grad, double* m,
                                 double* v, int64_t B, int64_t M, int32_t step, double lr, double beta1,
                                 double beta2, double eps, void* stream);

/*
 * redo_grape_lbfgs_step -- GRAPE ascent by projected L-BFGS with Armijo backtracking (the paper
 * leaves the update rule open; quasi-Newton ascent needs several times fewer fidelity and gradient
 * evaluations than plain or Adam ascent near F = 1).  One call per gradient evaluation:
 *   u        device double [B][M][K], in: the point just evaluated (F, grad from redo_fidelity_grad
 *            or its variants); out: the next point to evaluate.
 *   grad, F  device double [B][M][K] and [B] at that point.
 *   history  number of (s, y) pairs kept per pulse, 1..64.
 *   first    nonzero on the first call (accepts the point and starts the state).
 *   step0    size of a gradient step: its largest entry is step0 * max_k (hi_k - lo_k) / 2.
 *   c1       Armijo constant (1e-4 is usual), 0 < c1 < 1.
 *   state    device scratch of redo_grape_lbfgs_workspace() bytes, 256-byte aligned, kept between
 *            calls (nothing in it needs to start at zero).
 *   u_best, F_best  device [B][M][K] and [B] or NULL: the accepted point and its F (never falls).
 * Per pulse: a trial point is accepted when F >= F_acc + c1 grad_acc . (u - u_acc); an accepted
 * step stores the pair s = u - u_acc, y = -(grad - grad_acc) when s.y > 0, and the next direction
 * is the two-loop recursion with H0 = (s.y / y.y) I of the newest pair (the plain gradient
 * direction when no pair is kept or the result is not an ascent direction); a rejected one halves
 * the step, and below 1e-3 of it drops every pair.  The next point is clip(u_acc + alpha d, lo_k,
 * hi_k).  Errors: REDO_ERR_INVALID, REDO_ERR_CUDA.  Asynchronous on `stream`.
 */
redo_status redo_grape_lbfgs_workspace(const redo_table* t, int64_t B, int64_t M, int32_t history, size_t* bytes);
redo_status redo_grape_lbfgs_step(const redo_table* t, double* u, const double* grad, const double* F, int64_t B,
                                  int64_t M, int32_t history, int32_t first, double step0, double c1, void* state,
                                  size_t state_bytes, double* u_best, double* F_best, void* stream);

/*
 * Amplitude/phase controls (Section III, Eq. vn and the Dirac-frame step after Eq. vnd).
 *
 * A linearly polarised drive of amplitude A_kn and phase phi_kn on species k equals the
 * x-polarised drive turned about z, so a table built on the species' x-operators
 * (H_k = S_xk in redo_build_table, lo/hi spanning the amplitude range) serves every phase:
 *     U_n = Z_n E_{K-1,n} ... E_{0,n} Z_n^dag D,   Z_n = exp(-i sum_k phi_kn S_kz),
 * E_k the table operator of the quantised amplitude q[b][n][k].  The phases are not
 * quantised: Z_n is diagonal and is evaluated per basis state in FP64.
 *
 * redo_table_set_phase_axes -- attach the diagonals of S_kz to the table.
 *  sz   host double [K][N]: sz[k][a] = <a|S_kz|a>.  Copied; the caller keeps ownership.
 * Synchronous (like redo_build_table).  REDO_ERR_UNSUPPORTED when some S_kz does not commute
 * with H0 (an off-diagonal H0[a][b] != 0 with sz[k][a] != sz[k][b]): Z_n must commute with the
 * drift for the regrouping the library uses.  A second call replaces the axes.
 */
redo_status redo_table_set_phase_axes(redo_table* t, const double* sz);

/*
 * redo_propagate_phase -- U_b = U_M ... U_1 for amplitude/phase controls, and optionally
 * F_b = |Tr(U_target^dag U_b)|^2 / N^2; arguments as redo_propagate plus
 *  phi   device double [B][M][K], phases in radians (any real value).
 * REDO_FP64 and REDO_FP32 for every N; REDO_FP16X3 for N <= 64 (tensor-core chains, the
 * phase diagonals entering as split-FP16 factors).  Not on a REDO_TABLE_STRANG table.
 * REDO_ERR_INVALID when the table has no phase axes.  Workspace from
 * redo_propagate_phase_workspace.
 */
redo_status redo_propagate_phase(const redo_table* t, const int32_t* q, const double* phi, int64_t B, int64_t M,
                                 redo_precision prec, int32_t reunit_every, void* U_out, const void* U_target,
                                 double* F_out, void* tau_out, void* workspace, size_t workspace_bytes,
                                 int64_t* dev_status, void* stream);
redo_status redo_propagate_phase_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                           int32_t reunit_every, size_t* bytes);

/*
 * redo_fidelity_grad_phase -- GRAPE gradient of F = |Tr(U_target^dag U)|^2 / N^2 for amplitude/phase
 * controls (Section III: the control profiles {Omega_kn, phi_kn} are what GRAPE optimises):
 *  grad_amp    device double [B][M][K]: dF/dA_kn at the quantised amplitudes (1/(rad/s)),
 *  grad_phase  device double [B][M][K]: dF/dphi_kn (1/rad),
 * the other arguments as redo_fidelity_grad plus phi (device double [B][M][K]).  With
 * P_n = Z_n^dag Z_{n-1} the chain is Z_{M-1} (E'_M P_M) ... (E'_1 P_1); dF/dA follows from the table
 * factors as in redo_fidelity_grad, and dF/dphi_kn = (2/N^2) Im(conj(tau) (Tz_{n+1,k} - Tz_{n,k}))
 * with Tz_{n,k} = Tr(S_kz W_n) at the step boundaries (W_n the product of the chain after the
 * boundary, the transformed target and the chain before it).
 * REDO_FP64 or REDO_FP32 at every N (for N > 64 on segments of whole steps: checkpoint_every is
 * then the segment length in steps); REDO_ERR_UNSUPPORTED otherwise.  Workspace from
 * redo_fidelity_grad_phase_workspace.
 */
redo_status redo_fidelity_grad_phase(const redo_table* t, const int32_t* q, const double* phi, int64_t B, int64_t M,
                                     const void* U_target, int32_t target_batched, redo_precision prec,
                                     int32_t checkpoint_every, double* F_out, double* grad_amp, double* grad_phase,
                                     void* workspace, size_t workspace_bytes, int64_t* dev_status, void* stream);
redo_status redo_fidelity_grad_phase_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                               int32_t checkpoint_every, size_t* bytes);

/*
 * redo_propagate_drift -- U_b = U_M ... U_1 with a diagonal drift of each pulse's own:
 *   U_n = E_{K-1,n} ... E_{0,n} D diag(exp(-i dt h_b)),
 * the Lie split (Section III, the step after Eq. vnd, drift first in time) of the drift
 * H0 + diag(h_b), exact when the table's H0 is diagonal (build the table with H0 = 0 and pass
 * each pulse's whole diagonal drift in h; the NMR offsets and couplings of Section III are
 * diagonal).  One table then serves pulses on systems that differ in their offsets and couplings.
 *  h      device double [B][N]: the diagonal drift energies of pulse b (rad/s); the factors
 *         exp(-i dt h) are taken in FP64 (FP32 copies for REDO_FP16X3).
 * The other arguments, outputs and errors as redo_propagate.  REDO_ERR_UNSUPPORTED on a
 * symmetric-split table and for REDO_FP16X3 with N > 64.  Workspace from
 * redo_propagate_drift_workspace.
 */
redo_status redo_propagate_drift(const redo_table* t, const int32_t* q, const double* h, int64_t B, int64_t M,
                                 redo_precision prec, int32_t reunit_every, void* U_out, const void* U_target,
                                 double* F_out, void* tau_out, void* workspace, size_t workspace_bytes,
                                 int64_t* dev_status, void* stream);
redo_status redo_propagate_drift_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                           int32_t reunit_every, size_t* bytes);

/*
 * redo_fidelity_grad_drift -- F and dF/du of redo_fidelity_grad for the chain of
 * redo_propagate_drift (h: device double [B][N], pulse b's diagonal drift in rad/s).
 * The drift factors are constants of the pulse, so the gradient keeps Section III's form
 * g_kn = (2 dt / N^2) Im(conj(tau) Tr(H_k W_{n,k})) with each step's diagonal inside its W.
 * REDO_FP64 or REDO_FP32 at every N (for N > 64 on segments of whole steps: checkpoint_every is
 * then the segment length in steps); REDO_ERR_UNSUPPORTED otherwise and on a symmetric-split
 * table.  reunit_every as for redo_fidelity_grad (equal to checkpoint_every, or 0).
 * Workspace from redo_fidelity_grad_drift_workspace.
 */
redo_status redo_fidelity_grad_drift(const redo_table* t, const int32_t* q, const double* h, int64_t B, int64_t M,
                                     const void* U_target, int32_t target_batched, redo_precision prec,
                                     int32_t checkpoint_every, int32_t reunit_every, double* F_out, double* grad,
                                     void* workspace, size_t workspace_bytes, int64_t* dev_status, void* stream);
redo_status redo_fidelity_grad_drift_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                               int32_t checkpoint_every, size_t* bytes);

/*
 * redo_batched_product -- C_b = op(A_b) op(B_b), b < count, for the time-split layer (one pulse
 * cut into time segments, one per rank: U = S_{G-1} ... S_0, and segment r's gradient taken
 * against the target L_r^dag U_T P_r^dag with P_r = S_{r-1} ... S_0, L_r = S_{G-1} ... S_{r+1};
 * Section III's unitary fidelity is unchanged by that regrouping).
 *  N          dimension, 1..1024.
 *  A, B       device complex128 [count][N][N] when *_batched != 0, else one [N][N] used for all b.
 *  adjA/adjB  nonzero: use the conjugate transpose.
 *  C          device complex128 [count][N][N], written; must not overlap A or B (REDO_ERR_INVALID).
 * FP64 throughout; asynchronous on `stream`.
 */
redo_status redo_batched_product(int32_t N, int64_t count, const void* A, int32_t adjA, int32_t A_batched,
                                 const void* B, int32_t adjB, int32_t B_batched, void* C, void* stream);

/* Scratch bytes redo_propagate needs for (B, M, prec, reunit_every) on this table. */
redo_status redo_propagate_workspace(const redo_table* t, int64_t B, int64_t M,
                                     redo_precision prec, int32_t reunit_every, size_t* bytes);

/*
 * Kernel timing for measurement.  While enabled, the library brackets each of
 * its kernel launches with CUDA events on the launching stream.  Phases:
 *   0 quantize, 1 table, 2 chain segments, 3 chain combine, 4 finalize,
 *   5 tensor-core chain, 6 re-unitarisation, 7 gradient (all of it), and inside
 *   the tensor-core gradient for N >= 128: 8 forward sweep, 9 checkpoint and
 *   costate scans, 10 reverse sweep with traces.
 * redo_profile_read synchronises on the recorded events, adds each phase's
 * elapsed milliseconds and launch count into ms_out[p] / launches_out[p]
 * (arrays of n <= REDO_PROFILE_PHASES entries, either may be NULL) and clears
 * the record.  Not thread-safe; meant for benchmarks, not production.
 */
#define REDO_PROFILE_PHASES 11
redo_status redo_profile_enable(int32_t enable);
redo_status redo_profile_read(double* ms_out, int64_t* launches_out, int32_t n);

/* Thread-local description of the last error returned on this thread. */
const char* redo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* REDO_H */
