// State simulation along REDO chains (Section IV): psi_n = U_n ... U_1 psi_0 and
// the expectation <O>(t_n) = sum_a o_a |psi_n[a]|^2 of a diagonal observable.
//
// One CTA per pulse keeps psi in shared memory and applies the gathered table
// operators one matrix-vector product at a time (O(N^2) per operator instead of
// the O(N^3) operator product), reading the operators straight from the
// L2-resident table with the next operator's entries prefetched into
// registers while the current one is applied.  Thread (row r, part p) owns the
// N/P entries A[r][p*N/P ...] of every operator; the P partial sums of a row
// are combined with warp shuffles.
#include "redo_internal.cuh"

#include <type_traits>

namespace redo {

template <int N> struct SimShape {
  static constexpr int P = N >= 16 ? 256 / N : N;   // threads per row
  static constexpr int EL = N / P;                  // entries per thread
  static constexpr int THREADS = N * P;
  static_assert(P <= 32 && (P & (P - 1)) == 0, "row group must fit a warp");
};

template <typename R, int N>
__global__ void __launch_bounds__(SimShape<N>::THREADS)
sim_state_kernel(const cplx<R>* __restrict__ T, const int32_t* __restrict__ q, int64_t M, int K,
                 int d, int base, int64_t levels, const double2* __restrict__ psi0,
                 int psi0_batched, const double* __restrict__ obs, double* __restrict__ expect,
                 int64_t* status) {
  using SS = SimShape<N>;
  constexpr int P = SS::P, EL = SS::EL;
  __shared__ cplx<R> psi[N];
  __shared__ double red[SS::THREADS];
  const int tid = threadIdx.x;
  const int r = tid / P, p = tid % P;
  const int64_t b = blockIdx.x;
  const double2* ps = psi0 + (psi0_batched ? b * N : 0);
  if (tid < N) psi[tid] = cmake<R>((R)ps[tid].x, (R)ps[tid].y);
  __syncthreads();

  auto expectation = [&]() -> double {
    double v = 0.0;
    if (tid < N) {
      const double re = (double)psi[tid].x, im = (double)psi[tid].y;
      v = obs[tid] * (re * re + im * im);
    }
    red[tid] = v;
    __syncthreads();
    for (int w = SS::THREADS / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    const double out = red[0];
    __syncthreads();
    return out;
  };

  const double e0 = expectation();
  if (tid == 0) expect[b * (M + 1)] = e0;
  const int64_t kd = (int64_t)K * d;
  const int64_t F = M * kd;
  auto factor = [&](int64_t f) -> const cplx<R>* {
    const int64_t n = f / kd;
    const int rr = (int)(f - n * kd);
    const int k = rr / d, j = rr - k * d;
    int32_t qv = q[(b * M + n) * K + k];
    if (qv < 0 || qv >= levels) {
      if (status && tid == 0) atomicAdd((unsigned long long*)&status[REDO_STATUS_BADINDEX], 1ull);
      qv = 0;
    }
    for (int i = 0; i < j; ++i) qv /= base;
    return T + ((int64_t)(k * d + j) * base + qv % base) * (N * N) + r * N + p * EL;
  };
  cplx<R> cur[EL], nxt[EL];
  if (F > 0) {
    const cplx<R>* a = factor(0);
#pragma unroll
    for (int e = 0; e < EL; ++e) cur[e] = a[e];
  }
  for (int64_t f = 0; f < F; ++f) {
    if (f + 1 < F) {
      const cplx<R>* a = factor(f + 1);
#pragma unroll
      for (int e = 0; e < EL; ++e) nxt[e] = a[e];
    }
    cplx<R> acc = cmake<R>(R(0), R(0));
#pragma unroll
    for (int e = 0; e < EL; ++e) cfma<R>(acc, cur[e], psi[p * EL + e]);
    constexpr unsigned kMask = SS::THREADS >= 32 ? 0xffffffffu : ((1u << SS::THREADS) - 1u);
#pragma unroll
    for (int off = P / 2; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(kMask, acc.x, off);
      acc.y += __shfl_xor_sync(kMask, acc.y, off);
    }
    __syncthreads();
    if (p == 0) psi[r] = acc;
    __syncthreads();
    if ((f + 1) % kd == 0) {
      const double ev = expectation();
      if (tid == 0) expect[b * (M + 1) + (f + 1) / kd] = ev;
    }
#pragma unroll
    for (int e = 0; e < EL; ++e) cur[e] = nxt[e];
  }
}

template <typename R, int N>
static cudaError_t sim_n(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                         const double2* psi0, int psi0_batched, const double* obs, double* expect,
                         int64_t* status, cudaStream_t s) {
  const cplx<R>* T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  sim_state_kernel<R, N><<<(unsigned)B, SimShape<N>::THREADS, 0, s>>>(
      T, q, M, t->K, t->digits, t->base, t->levels, psi0, psi0_batched, obs, expect, status);
  return cudaGetLastError();
}

cudaError_t launch_sim_state(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                             int prec, const double2* psi0, int psi0_batched, const double* obs,
                             double* expect, int64_t* status, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const bool dbl = prec == REDO_FP64;
#define SIM_CASE(n)                                                                             \
  case n:                                                                                       \
    return dbl ? sim_n<double, n>(t, q, B, M, psi0, psi0_batched, obs, expect, status, s)       \
               : sim_n<float, n>(t, q, B, M, psi0, psi0_batched, obs, expect, status, s);
  switch (t->N) {
    SIM_CASE(2) SIM_CASE(4) SIM_CASE(8) SIM_CASE(16) SIM_CASE(32) SIM_CASE(64)
    default: return cudaErrorInvalidValue;
  }
#undef SIM_CASE
}

// ============================================================================
// Mixed diagonal states: e_n = Tr[U_n rho U_n^dag O] = sum_{r,c} rho_c o_r |U_n[r][c]|^2 for
// diagonal rho and O (Section IV's order parameter when both are diagonal in the working
// basis).  One CTA per pulse keeps U_n in shared memory (ping-pong), stages each gathered
// operator in shared memory with the next one already loaded into registers, and reduces
// e_n after every step; it writes the series and/or its mean over n = 1..M.
// ============================================================================
template <int N> struct MixShape {
  static constexpr int THREADS = N * N < 64 ? 64 : (N * N > 256 ? 256 : N * N);
  static constexpr int EPT = (N * N + THREADS - 1) / THREADS;   // entries per thread
};

template <typename R, int N>
__global__ void __launch_bounds__(MixShape<N>::THREADS)
expect_diag_kernel(const cplx<R>* __restrict__ T, const int32_t* __restrict__ q, int64_t M, int K, int d,
                   int base, int64_t levels, const double* __restrict__ rho, const double* __restrict__ obs,
                   double* __restrict__ expect, double* __restrict__ mean, int64_t* status) {
  using MS = MixShape<N>;
  constexpr int TH = MS::THREADS, EPT = MS::EPT, N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* U0 = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* U1 = U0 + N2;
  cplx<R>* A = U1 + N2;
  __shared__ double red[TH / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t b = blockIdx.x;
  for (int e = tid; e < N2; e += TH) U0[e] = cmake<R>((e / N == e % N) ? R(1) : R(0), R(0));

  auto reduce = [&](const cplx<R>* U) -> double {
    double v = 0.0;
    for (int e = tid; e < N2; e += TH) {
      const double re = (double)U[e].x, im = (double)U[e].y;
      v += rho[e % N] * obs[e / N] * (re * re + im * im);
    }
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double out = 0.0;
#pragma unroll
    for (int w = 0; w < TH / 32; ++w) out += red[w];
    return out;
  };
  auto factor = [&](int64_t f) -> const cplx<R>* {
    const int64_t kd = (int64_t)K * d;
    const int64_t n = f / kd;
    const int rr = (int)(f - n * kd);
    const int k = rr / d, j = rr - k * d;
    int32_t qv = q[(b * M + n) * K + k];
    if (qv < 0 || qv >= levels) {
      if (status && tid == 0) atomicAdd((unsigned long long*)&status[REDO_STATUS_BADINDEX], 1ull);
      qv = 0;
    }
    for (int i = 0; i < j; ++i) qv /= base;
    return T + ((int64_t)(k * d + j) * base + qv % base) * N2;
  };

  __syncthreads();
  const double e0 = reduce(U0);
  if (tid == 0 && expect) expect[b * (M + 1)] = e0;
  double acc = 0.0;
  const int64_t kd = (int64_t)K * d, F = M * kd;
  cplx<R> nxt[EPT];
  if (F > 0) {
    const cplx<R>* a = factor(0);
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * TH;
      if (e < N2) nxt[i] = a[e];
    }
  }
  cplx<R>* cur = U0;
  cplx<R>* out = U1;
  for (int64_t f = 0; f < F; ++f) {
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * TH;
      if (e < N2) A[e] = nxt[i];
    }
    __syncthreads();
    if (f + 1 < F) {
      const cplx<R>* a = factor(f + 1);
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const int e = tid + i * TH;
        if (e < N2) nxt[i] = a[e];
      }
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * TH;
      if (e < N2) {
        const int r = e / N, c = e % N;
        cplx<R> s = cmake<R>(R(0), R(0));
#pragma unroll 8
        for (int k = 0; k < N; ++k) cfma<R>(s, A[r * N + k], cur[k * N + c]);
        out[e] = s;
      }
    }
    __syncthreads();
    cplx<R>* tmp = cur;
    cur = out;
    out = tmp;
    if ((f + 1) % kd == 0) {
      const double ev = reduce(cur);
      acc += ev;
      if (tid == 0 && expect) expect[b * (M + 1) + (f + 1) / kd] = ev;
    }
  }
  if (tid == 0 && mean) mean[b] = M > 0 ? acc / (double)M : e0;
}

// Small N (<= 16) with a table that fits in shared memory: the whole table is staged once per
// CTA and every thread carries one column of one pulse's U_n in registers, so a CTA of 256
// threads serves 256/N pulses with no barrier inside the chain:
//     column c:  u <- T_f u  (N^2 complex FMAs per factor, T_f read from shared memory),
//     e_n = sum_c rho_c sum_r o_r |U_n[r][c]|^2 (the columns' parts added by shuffles within the
// pulse's N lanes; the mean needs only each lane's running sum).
constexpr int kColThreads = 256;

template <typename R, int N>
__global__ void __launch_bounds__(kColThreads, 2)
expect_cols_kernel(const cplx<R>* __restrict__ T, int64_t entries, const int32_t* __restrict__ q, int64_t B,
                   int64_t M, int K, int d, int base, int64_t levels, const double* __restrict__ rho,
                   const double* __restrict__ obs, double* __restrict__ expect, double* __restrict__ mean,
                   int64_t* status) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Ts = reinterpret_cast<cplx<R>*>(smem_raw);
  for (int64_t i = threadIdx.x; i < entries * N2; i += kColThreads) Ts[i] = T[i];
  __syncthreads();
  const int c = threadIdx.x % N;
  const int64_t b_raw = (int64_t)blockIdx.x * (kColThreads / N) + threadIdx.x / N;
  const bool active = b_raw < B;
  const int64_t b = active ? b_raw : B - 1;        // idle lanes follow the last pulse, write nothing
  R o[N];
#pragma unroll
  for (int r = 0; r < N; ++r) o[r] = (R)obs[r];
  const double rc = rho[c];
  cplx<R> u[N];
#pragma unroll
  for (int r = 0; r < N; ++r) u[r] = cmake<R>(r == c ? R(1) : R(0), R(0));
  auto part = [&]() -> double {
    R v = R(0);
#pragma unroll
    for (int r = 0; r < N; ++r) v = fma(o[r], fma(u[r].x, u[r].x, u[r].y * u[r].y), v);
    return rc * (double)v;
  };
  auto group_sum = [&](double v) -> double {
#pragma unroll
    for (int off = N / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, N);
    return v;
  };
  const double e0 = group_sum(part());
  if (expect && active && c == 0) expect[b * (M + 1)] = e0;
  double acc = 0.0;
  const int32_t* qb = q + b * M * K;
  int32_t qn = M > 0 ? qb[0] : 0;
  for (int64_t n = 0; n < M; ++n) {
    const int32_t* qrow = qb + n * K;
    for (int k = 0; k < K; ++k) {
      int32_t qv = qn;
      // next coefficient's level, loaded while this one is applied
      qn = (k + 1 < K) ? qrow[k + 1] : (n + 1 < M ? qrow[K] : 0);
      if (qv < 0 || qv >= levels) {
        if (status && active) atomicAdd((unsigned long long*)&status[REDO_STATUS_BADINDEX], 1ull);
        qv = 0;
      }
      for (int j = 0; j < d; ++j) {
        const cplx<R>* A = Ts + ((int64_t)(k * d + j) * base + qv % base) * N2;
        qv /= base;
        cplx<R> v[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
          cplx<R> sacc = cmake<R>(R(0), R(0));
          if constexpr (std::is_same<R, float>::value && N % 2 == 0) {
            // two operator entries per 16-byte load: the N lanes of a pulse read the same
            // address, so each quarter-warp phase of the load serves one pulse
            const float4* A4 = reinterpret_cast<const float4*>(A + r * N);
#pragma unroll
            for (int kk = 0; kk < N; kk += 2) {
              const float4 a2 = A4[kk / 2];
              cfma<R>(sacc, cmake<R>(a2.x, a2.y), u[kk]);
              cfma<R>(sacc, cmake<R>(a2.z, a2.w), u[kk + 1]);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < N; ++kk) cfma<R>(sacc, A[r * N + kk], u[kk]);
          }
          v[r] = sacc;
        }
#pragma unroll
        for (int r = 0; r < N; ++r) u[r] = v[r];
      }
    }
    const double pv = part();
    acc += pv;
    if (expect) {
      const double ev = group_sum(pv);
      if (active && c == 0) expect[b * (M + 1) + n + 1] = ev;
    }
  }
  const double tot = group_sum(acc);
  if (mean && active && c == 0) mean[b] = M > 0 ? tot / (double)M : e0;
}

template <typename R, int N>
static cudaError_t expect_diag_n(const redo_table* t, const int32_t* q, int64_t B, int64_t M, const double* rho,
                                 const double* obs, double* expect, double* mean, int64_t* status,
                                 cudaStream_t s) {
  const cplx<R>* T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  if constexpr (N * sizeof(R) <= 64) {            // one column in registers: N <= 16 (FP32), 8 (FP64)
    const size_t table_smem = (size_t)t->entries * N * N * sizeof(cplx<R>);
    // worth it once every SM gets a full CTA (256 / N pulses); fewer pulses keep one CTA each
    if (table_smem <= 200 * 1024 && B * N >= (int64_t)t->num_sms * kColThreads) {
      cudaError_t e = cudaFuncSetAttribute(expect_cols_kernel<R, N>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)table_smem);
      if (e != cudaSuccess) return e;
      const int64_t per = kColThreads / N;
      expect_cols_kernel<R, N><<<(unsigned)((B + per - 1) / per), kColThreads, table_smem, s>>>(
          T, t->entries, q, B, M, t->K, t->digits, t->base, t->levels, rho, obs, expect, mean, status);
      return cudaGetLastError();
    }
  }
  const size_t smem = 3 * sizeof(cplx<R>) * N * N;
  cudaError_t e = cudaFuncSetAttribute(expect_diag_kernel<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  expect_diag_kernel<R, N><<<(unsigned)B, MixShape<N>::THREADS, smem, s>>>(
      T, q, M, t->K, t->digits, t->base, t->levels, rho, obs, expect, mean, status);
  return cudaGetLastError();
}

cudaError_t launch_expect_diag(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                               const double* rho, const double* obs, double* expect, double* mean,
                               int64_t* status, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const bool dbl = prec == REDO_FP64;
#define MIX_CASE(n)                                                                                  \
  case n:                                                                                            \
    return dbl ? expect_diag_n<double, n>(t, q, B, M, rho, obs, expect, mean, status, s)             \
               : expect_diag_n<float, n>(t, q, B, M, rho, obs, expect, mean, status, s);
  switch (t->N) {
    MIX_CASE(2) MIX_CASE(4) MIX_CASE(8) MIX_CASE(16) MIX_CASE(32) MIX_CASE(64)
    default: return cudaErrorInvalidValue;
  }
#undef MIX_CASE
}

}  // namespace redo
