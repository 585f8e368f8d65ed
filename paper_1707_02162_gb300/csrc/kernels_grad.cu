// GRAPE fidelity gradient of the REDO split model (SIMT, N <= 64, FP64/FP32).
// (Section III: the gradient that GRAPE, Fig. fc, ascends; the paper prints no formula, so it is
// derived here from the split model's definitions.)
//
// With the chain of table factors A_0 ... A_{F-1} of one pulse (A_0 applied
// first), forward partial products P_f = A_f ... A_0 and backward costates
// R_f = U_T^dag A_{F-1} ... A_{f+1}, the derivative of the fidelity with respect
// to the coefficient u_kn of control term k in step n is
//     dF/du_kn = (2 dt / N^2) Im( conj(tau) Tr(H_k P_f R_f) ),
// f = the last digit factor of term k in step n, tau = Tr(U_T^dag U).  (Each
// per-term exponential commutes with its own generator H_k, so the derivative
// of the digit product exp(-i dt u H_k) is -i dt H_k times it.)
//
// Work split: the pulse is cut into S segments whose products come from the
// segment chain kernel; a scan kernel forms the checkpoints P at every segment
// end and the costates R there (suffix products), and one CTA per segment then
// sweeps its factors backwards, undoing them with their adjoints
// (P_{f-1} = A_f^dag P_f, R_{f-1} = R_f A_f, the factors being unitary) and
// evaluating the traces with the sparse (CSR) H_k.
#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "smem_mm.cuh"

#include <type_traits>

namespace redo {

// ----------------------------------------------------------------------------
// Scan: Pck[b][s] = S_s ... S_0,  Rck[b][s] = U_T^dag S_{S-1} ... S_{s+1},
// tau_b = Tr(U_T^dag U_b), F_b = |tau_b|^2 / N^2 (FP64 reduction)
// ----------------------------------------------------------------------------
template <typename R, int N>
__global__ void __launch_bounds__(SmemMM<R, N, SqTile<N>::TM, SqTile<N>::TM>::THREADS)
grad_scan_kernel(int64_t S, const cplx<R>* __restrict__ seg, const double2* __restrict__ UT,
                 int target_batched, cplx<R>* __restrict__ Pck, cplx<R>* __restrict__ Rck,
                 double2* __restrict__ tau, double* __restrict__ F_out) {
  constexpr int TM = SqTile<N>::TM;
  using MM = SmemMM<R, N, TM, TM>;
  constexpr int N2 = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cplx<R>* X = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* A = X + N2;
  __shared__ double red_re[MM::THREADS], red_im[MM::THREADS];
  const int lt = threadIdx.x;
  const int64_t b = blockIdx.x;
  const double2* Ut = UT + (target_batched ? b * N2 : 0);
  cplx<R> Y[TM][TM];
  for (int i = lt; i < N2; i += MM::THREADS) X[i] = cmake<R>((i / N == i % N) ? R(1) : R(0), R(0));
  __syncthreads();
  for (int64_t s = 0; s < S; ++s) {
    const cplx<R>* Ss = seg + (b * S + s) * N2;
    for (int i = lt; i < N2; i += MM::THREADS) A[i] = Ss[i];
    __syncthreads();
    MM::run(A, X, lt, Y);
    __syncthreads();
    MM::store(X, lt, Y);
    __syncthreads();
    cplx<R>* o = Pck + (b * S + s) * N2;
    for (int i = lt; i < N2; i += MM::THREADS) o[i] = X[i];
  }
  // tau = sum conj(U_T) .* U in FP64
  double re = 0.0, im = 0.0;
  for (int i = lt; i < N2; i += MM::THREADS) {
    const double2 g = Ut[i];
    const double ur = (double)X[i].x, ui = (double)X[i].y;
    re = fma(g.x, ur, re);
    re = fma(g.y, ui, re);
    im = fma(g.x, ui, im);
    im = fma(-g.y, ur, im);
  }
  red_re[lt] = re;
  red_im[lt] = im;
  __syncthreads();
  for (int w = MM::THREADS / 2; w > 0; w >>= 1) {
    if (lt < w) {
      red_re[lt] += red_re[lt + w];
      red_im[lt] += red_im[lt + w];
    }
    __syncthreads();
  }
  if (lt == 0) {
    tau[b] = make_double2(red_re[0], red_im[0]);
    if (F_out) F_out[b] = (red_re[0] * red_re[0] + red_im[0] * red_im[0]) / ((double)N * (double)N);
  }
  // costates: Y = U_T^dag, then Y <- Y S_s going backwards
  for (int i = lt; i < N2; i += MM::THREADS) {
    const int r = i / N, c = i % N;
    const double2 g = Ut[c * N + r];
    X[i] = cmake<R>((R)g.x, (R)(-g.y));
  }
  __syncthreads();
  for (int64_t s = S - 1; s >= 0; --s) {
    cplx<R>* o = Rck + (b * S + s) * N2;
    for (int i = lt; i < N2; i += MM::THREADS) o[i] = X[i];
    if (s == 0) break;
    const cplx<R>* Ss = seg + (b * S + s) * N2;
    for (int i = lt; i < N2; i += MM::THREADS) A[i] = Ss[i];
    __syncthreads();
    MM::run(X, A, lt, Y);
    __syncthreads();
    MM::store(X, lt, Y);
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// Backward sweep over one segment: traces at term boundaries, then undo the factor.
// ----------------------------------------------------------------------------
template <typename R>
struct GradArgs {
  const cplx<R>* T;          // table (FP64 or FP32 copy)
  const int32_t* q;
  int64_t M;
  int K, d, base;
  int64_t levels;
  int64_t S, seg_len, F;
  const cplx<R>* Pck;
  const cplx<R>* Rck;
  const double2* tau;
  const int32_t* hk_ptr;
  const int32_t* hk_col;
  const int32_t* hk_row;
  const double2* hk_val;
  double scale;              // 2 dt / N^2
  double* grad;              // [B][M][K]
  int64_t* status;
  // amplitude/phase calls: every step opens with the diagonal P_n = pd[b][n] (factor 0 of
  // fps = K*d + 1); at each such factor the sweep records Tz[b][n][k] = Tr(S_kz P R), and the
  // last segment records Tz[b][M][k] at the end of the chain.  pd == nullptr otherwise.
  int64_t fps;
  const double2* pd;
  const double* sz;          // [K][N]
  double2* Tz;               // [B][M+1][K]
  // kept forward states (the partial products of every segment, [chains][seg_len][N][N]) or
  // nullptr: with them the sweep reads P_f instead of undoing it (one product per factor)
  const cplx<R>* keep;
};

// Table operator of factor f (nullptr for a step-opening phase factor).
template <typename R, int N>
__device__ __forceinline__ const cplx<R>* grad_factor(const GradArgs<R>& a, int64_t b, int64_t f,
                                                      int* k_out, int* j_out, int64_t* n_out) {
  const int64_t n = f / a.fps;
  int r = (int)(f - n * a.fps);
  *n_out = n;
  if (a.pd) {
    if (r == 0) return nullptr;
    --r;
  }
  const int k = r / a.d, j = r - k * a.d;
  int32_t qv = a.q[(b * a.M + n) * a.K + k];
  if (qv < 0 || qv >= a.levels) {
    if (a.status) atomicAdd((unsigned long long*)&a.status[REDO_STATUS_BADINDEX], 1ull);
    qv = 0;
  }
  for (int i = 0; i < j; ++i) qv /= a.base;
  *k_out = k;
  *j_out = j;
  *n_out = n;
  return a.T + ((int64_t)(k * a.d + j) * a.base + qv % a.base) * (N * N);
}

// PH: amplitude/phase call (a.pd non-null: step-opening diagonal factors and boundary traces).
// KEEP: every forward state kept (a.keep): P_f is copied in with the factor, R starts from the
// costate carried back by the checkpoint before the segment (the kept states start from the
// identity at the segment's start), and only R <- R A_f is multiplied.  With PH and KEEP
// together a diagonal factor leaves only R <- R diag(p), and the boundary traces read the kept
// state (with R' = P_{s-1} R_s, Tr(S P_kept R') = Tr(S P R_s) for the whole prefix P).
// TZ: record the boundary traces Tz (amplitude/phase calls; not for per-pulse drift diagonals).
template <typename R, int N, bool PH, bool KEEP, bool TZ>
__global__ void __launch_bounds__(SmemMM<R, N, SqTile<N>::TM, SqTile<N>::TM>::THREADS)
grad_sweep_kernel(GradArgs<R> a) {
  constexpr int TM = SqTile<N>::TM;
  using MM = SmemMM<R, N, TM, TM>;
  constexpr int N2 = N * N;
  constexpr int STAGES = (sizeof(R) == 8 && N == 64) ? 1 : 2;   // shared memory budget
  constexpr uint32_t BYTES = (uint32_t)(N2 * sizeof(cplx<R>));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // layout: P, R, STAGES operators (KEEP: R, STAGES operators, STAGES kept states)
  cplx<R>* P = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* Rm = KEEP ? P : P + N2;
  cplx<R>* Abuf = Rm + N2;
  cplx<R>* Pbuf = Abuf + STAGES * N2;
  uint64_t* bar = reinterpret_cast<uint64_t*>(KEEP ? Pbuf + STAGES * N2 : Abuf + STAGES * N2);
  __shared__ double red_re[MM::THREADS], red_im[MM::THREADS];
  __shared__ int abort_flag;
  const int lt = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t b = g / a.S, s = g % a.S;
  const int64_t f0 = s * a.seg_len;
  int64_t f1 = f0 + a.seg_len;
  if (f1 > a.F) f1 = a.F;
  const int64_t len = f1 > f0 ? f1 - f0 : 0;
  const double2 tau = a.tau[b];

  if (lt == 0) abort_flag = 0;
  if (lt < STAGES) mbar_init(&bar[lt], 1);
  fence_mbarrier_init();
  cplx<R> Y1[TM][TM], Y2[TM][TM];
  if constexpr (KEEP) {
    // R' = P_{s-1} R_s (R_0 for the first segment of a pulse)
    for (int i = lt; i < N2; i += MM::THREADS) {
      Rm[i] = a.Rck[g * N2 + i];
      if (s > 0) Pbuf[i] = a.Pck[(g - 1) * N2 + i];
    }
    __syncthreads();
    if (s > 0) {
      MM::run(Pbuf, Rm, lt, Y2);
      __syncthreads();
      MM::store(Rm, lt, Y2);
      __syncthreads();
    }
  } else {
    for (int i = lt; i < N2; i += MM::THREADS) {
      P[i] = a.Pck[g * N2 + i];
      Rm[i] = a.Rck[g * N2 + i];
    }
    __syncthreads();
  }
  // factors are visited in reverse: t-th visit is factor f1-1-t
  // a phase factor has no operand to copy: its stage completes on the arrival alone
  auto issue = [&](int st, int64_t f) {
    int k, j;
    int64_t n;
    const cplx<R>* src = grad_factor<R, N>(a, b, f, &k, &j, &n);
    if (KEEP) {
      mbar_arrive_expect_tx(&bar[st], src ? 2 * BYTES : BYTES);
      if (src) bulk_load(Abuf + st * N2, src, BYTES, &bar[st]);
      bulk_load(Pbuf + st * N2, a.keep + (g * a.seg_len + (f - f0)) * N2, BYTES, &bar[st]);
    } else if (src) {
      mbar_arrive_expect_tx(&bar[st], BYTES);
      bulk_load(Abuf + st * N2, src, BYTES, &bar[st]);
    } else {
      mbar_arrive(&bar[st]);
    }
  };
  if (lt == 0) {
    for (int st = 0; st < STAGES && st < len; ++st) issue(st, f1 - 1 - st);
  }
  __shared__ double2 dg[64];
  // Tz[b][nz][k] = sum_a sz[k][a] (Pq R)[a][a] for every species k
  auto phase_traces = [&](int64_t nz, const cplx<R>* Pq) {
    if constexpr (!TZ) return;   // step diagonals without phase axes (per-pulse drift): no traces
    if (lt < N) {
      double re = 0.0, im = 0.0;
      for (int x = 0; x < N; ++x) {
        const cplx<R> pv = Pq[lt * N + x], rv = Rm[x * N + lt];
        re += (double)pv.x * rv.x - (double)pv.y * rv.y;
        im += (double)pv.x * rv.y + (double)pv.y * rv.x;
      }
      dg[lt] = make_double2(re, im);
    }
    __syncthreads();
    for (int kk = lt; kk < a.K; kk += MM::THREADS) {
      double re = 0.0, im = 0.0;
      for (int x = 0; x < N; ++x) {
        const double w = a.sz[(int64_t)kk * N + x];
        re += w * dg[x].x;
        im += w * dg[x].y;
      }
      a.Tz[(b * (a.M + 1) + nz) * a.K + kk] = make_double2(re, im);
    }
    __syncthreads();
  };
  if (PH && !KEEP && len > 0 && f1 == a.F) phase_traces(a.M, P);     // end of the chain
  for (int64_t t = 0; t < len; ++t) {
    const int64_t f = f1 - 1 - t;
    const int64_t n = f / a.fps;
    int r = (int)(f - n * a.fps);
    const bool phase = PH && r == 0;
    if (PH) --r;
    const int k = r / a.d, j = r - k * a.d;
    const int stage = (int)(t % STAGES);
    const uint32_t parity = (uint32_t)((t / STAGES) & 1);
    if constexpr (KEEP) {
      // the trace needs this factor's kept state: wait for the stage first
      if (!mbar_wait_bounded(&bar[stage], parity)) abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
    }
    const cplx<R>* Pt = KEEP ? Pbuf + stage * N2 : P;
    // kept states: the first visit's state is the whole segment's product, the chain's end
    if (PH && KEEP && t == 0 && f1 == a.F) phase_traces(a.M, Pt);
    if (phase) phase_traces(n, Pt);
    if (!phase && j == a.d - 1) {
      // Tr(H_k P R) = sum over nonzeros (row i, col c) of H_k[i][c] (P R)[c][i]
      const int p0 = a.hk_ptr[k * (N + 1)];
      const int p1 = a.hk_ptr[k * (N + 1) + N];
      double re = 0.0, im = 0.0;
      for (int e = p0 + lt; e < p1; e += MM::THREADS) {
        const int i = a.hk_row[e], c = a.hk_col[e];
        R dr = 0, di = 0;
        for (int x = 0; x < N; ++x) {
          const cplx<R> pv = Pt[c * N + x], rv = Rm[x * N + i];
          dr = fma(pv.x, rv.x, dr);
          dr = fma(-pv.y, rv.y, dr);
          di = fma(pv.x, rv.y, di);
          di = fma(pv.y, rv.x, di);
        }
        const double2 h = a.hk_val[e];
        re += h.x * (double)dr - h.y * (double)di;
        im += h.x * (double)di + h.y * (double)dr;
      }
      red_re[lt] = re;
      red_im[lt] = im;
      __syncthreads();
      for (int w = MM::THREADS / 2; w > 0; w >>= 1) {
        if (lt < w) {
          red_re[lt] += red_re[lt + w];
          red_im[lt] += red_im[lt + w];
        }
        __syncthreads();
      }
      if (lt == 0) {
        // Im(conj(tau) * T)
        const double tr = red_re[0], ti = red_im[0];
        a.grad[(b * a.M + n) * a.K + k] = a.scale * (tau.x * ti - tau.y * tr);
      }
    }
    if constexpr (!KEEP) {
      if (!mbar_wait_bounded(&bar[stage], parity)) abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
    }
    const cplx<R>* A = Abuf + stage * N2;
    if (PH && phase) {
      // P <- diag(p)^dag P (rows), R <- R diag(p) (columns)
      const double2* pv = a.pd + (b * a.M + n) * N;
      const int ty = lt / MM::TX, tx = lt % MM::TX;
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TM; ++v) {
          const int row = ty + MM::TY * u, col = tx + MM::TX * v;
          const R pcx = (R)pv[col].x, pcy = (R)pv[col].y;
          const cplx<R> y = Rm[row * N + col];
          if constexpr (!KEEP) {
            const R prx = (R)pv[row].x, pry = (R)pv[row].y;
            const cplx<R> x = P[row * N + col];
            Y1[u][v] = cmake<R>(prx * x.x + pry * x.y, prx * x.y - pry * x.x);
          }
          Y2[u][v] = cmake<R>(pcx * y.x - pcy * y.y, pcx * y.y + pcy * y.x);
        }
    } else if constexpr (KEEP) {
      MM::run(Rm, A, lt, Y2);        // R <- R A
    } else {
      MM::run_adj(A, P, lt, Y1);     // P <- A^dag P
      MM::run(Rm, A, lt, Y2);        // R <- R A
    }
    __syncthreads();
    if constexpr (!KEEP) MM::store(P, lt, Y1);
    MM::store(Rm, lt, Y2);
    if (lt == 0 && t + STAGES < len) {
      fence_proxy_async_smem();
      issue(stage, f1 - 1 - (t + STAGES));
    }
    __syncthreads();
  }
  if (abort_flag && lt == 0 && a.status)
    atomicAdd((unsigned long long*)&a.status[REDO_STATUS_TIMEOUT], 1ull);
}

template <typename R, int N>
static cudaError_t grad_scan_n(int64_t B, int64_t S, const void* seg, const double2* UT,
                               int target_batched, void* Pck, void* Rck, double2* tau,
                               double* F_out, cudaStream_t s) {
  using MM = SmemMM<R, N, SqTile<N>::TM, SqTile<N>::TM>;
  const size_t smem = 2 * sizeof(cplx<R>) * N * N;
  auto kern = grad_scan_kernel<R, N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)B, MM::THREADS, smem, s>>>(S, (const cplx<R>*)seg, UT, target_batched,
                                               (cplx<R>*)Pck, (cplx<R>*)Rck, tau, F_out);
  return cudaGetLastError();
}

template <typename R, int N>
static cudaError_t grad_sweep_n(const GradArgs<R>& a, int64_t B, cudaStream_t s) {
  using MM = SmemMM<R, N, SqTile<N>::TM, SqTile<N>::TM>;
  constexpr int STAGES = (sizeof(R) == 8 && N == 64) ? 1 : 2;
  const size_t smem = (a.keep ? 1 + 2 * STAGES : 2 + STAGES) * sizeof(cplx<R>) * N * N + 2 * sizeof(uint64_t);
  auto kern = a.pd ? (a.Tz ? (a.keep ? grad_sweep_kernel<R, N, true, true, true>
                                     : grad_sweep_kernel<R, N, true, false, true>)
                           : (a.keep ? grad_sweep_kernel<R, N, true, true, false>
                                     : grad_sweep_kernel<R, N, true, false, false>))
                   : (a.keep ? grad_sweep_kernel<R, N, false, true, false>
                             : grad_sweep_kernel<R, N, false, false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = B * a.S;
  if (blocks == 0) return cudaSuccess;
  kern<<<(unsigned)blocks, MM::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t grad_scan_t(const redo_table* t, int64_t B, int64_t S, const void* seg,
                               const double2* UT, int tb, void* Pck, void* Rck, double2* tau,
                               double* F, cudaStream_t s) {
  switch (t->N) {
    case 2: return grad_scan_n<R, 2>(B, S, seg, UT, tb, Pck, Rck, tau, F, s);
    case 4: return grad_scan_n<R, 4>(B, S, seg, UT, tb, Pck, Rck, tau, F, s);
    case 8: return grad_scan_n<R, 8>(B, S, seg, UT, tb, Pck, Rck, tau, F, s);
    case 16: return grad_scan_n<R, 16>(B, S, seg, UT, tb, Pck, Rck, tau, F, s);
    case 32: return grad_scan_n<R, 32>(B, S, seg, UT, tb, Pck, Rck, tau, F, s);
    case 64: return grad_scan_n<R, 64>(B, S, seg, UT, tb, Pck, Rck, tau, F, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_scan(const redo_table* t, int64_t B, int64_t S, int prec, const void* seg,
                             const double2* U_target, int target_batched, void* Pck, void* Rck,
                             double2* tau, double* F_out, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  if (prec == REDO_FP64)
    return grad_scan_t<double>(t, B, S, seg, U_target, target_batched, Pck, Rck, tau, F_out, s);
  return grad_scan_t<float>(t, B, S, seg, U_target, target_batched, Pck, Rck, tau, F_out, s);
}

template <typename R>
static cudaError_t grad_sweep_t(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                const void* Pck, const void* Rck, const double2* tau,
                                double* grad, int64_t* status, double2* Tz, const void* keep, cudaStream_t s) {
  GradArgs<R> a;
  a.keep = (const cplx<R>*)keep;
  a.fps = p.fps > 0 ? p.fps : (int64_t)t->K * t->digits;
  a.pd = p.pd;
  a.sz = t->sz64;
  a.Tz = Tz;
  a.T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  a.q = q;
  a.M = p.M;
  a.K = t->K;
  a.d = t->digits;
  a.base = t->base;
  a.levels = t->levels;
  a.S = p.S;
  a.seg_len = p.seg_len;
  a.F = p.F;
  a.Pck = (const cplx<R>*)Pck;
  a.Rck = (const cplx<R>*)Rck;
  a.tau = tau;
  a.hk_ptr = t->hk_ptr;
  a.hk_col = t->hk_col;
  a.hk_row = t->hk_row;
  a.hk_val = t->hk_val;
  a.scale = 2.0 * t->dt / ((double)t->N * (double)t->N);
  a.grad = grad;
  a.status = status;
  switch (t->N) {
    case 2: return grad_sweep_n<R, 2>(a, p.B, s);
    case 4: return grad_sweep_n<R, 4>(a, p.B, s);
    case 8: return grad_sweep_n<R, 8>(a, p.B, s);
    case 16: return grad_sweep_n<R, 16>(a, p.B, s);
    case 32: return grad_sweep_n<R, 32>(a, p.B, s);
    case 64: return grad_sweep_n<R, 64>(a, p.B, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_sweep(const redo_table* t, const int32_t* q, const ChainPlan& p, int prec,
                              const void* Pck, const void* Rck, const double2* tau, double* grad,
                              int64_t* status, cudaStream_t s, double2* Tz, const void* keep) {
  if (prec == REDO_FP64) return grad_sweep_t<double>(t, q, p, Pck, Rck, tau, grad, status, Tz, keep, s);
  return grad_sweep_t<float>(t, q, p, Pck, Rck, tau, grad, status, Tz, keep, s);
}

}  // namespace redo
