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

}  // namespace redo
