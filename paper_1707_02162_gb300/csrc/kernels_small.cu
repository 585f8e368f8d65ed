// SIMT kernels of libredo for N <= 64: quantizer, FP64 operator table,
// segmented product chains (FP64 / FP32) and the FP64 fidelity epilogue.
// (Section II: Eq. cgrain for the quantizer, process 1 for the table, process 2 and Eq. exp2prod
// for the products; Section III: the chain U = U_M ... U_1 and the unitary fidelity F_U.)
//
// Every product here is a complex N x N matrix product held in shared memory;
// table operators are streamed in with bulk asynchronous copies
// (cp.async.bulk + mbarrier), several stages ahead of the product that uses
// them.  All device waits are bounded and report through the status words.
#include <cstdio>
#include <type_traits>

#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "smem_mm.cuh"

namespace redo {

// ============================================================================
// Quantizer -- Eq. (cgrain): level q = clamp(rint((u - lo_k) / delta_k))
// ============================================================================
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so the FP64 divide
// decides a level only where an FP32 estimate cannot.  With u = 2^-24, the estimate
// y = fl32(fl32(fl32(v) - fl32(lo)) * fl32(1/delta)) and the FP64 quotient
// x = fl64(fl64(v - lo) / delta) differ by at most about 3u|y| + u (|v| + |lo|) / |delta|
// <= 4u|y| + 2u |lo| / |delta| (first order: three FP32 roundings of the quotient, and the
// FP32 roundings of v and lo).  The kernel takes twice that plus 2^-40 as the bound e; where y lies more
// than e from every half-integer, no half-integer lies between y and x, so rint(y) = rint(x).
// Elsewhere (near ties, non-finite or huge y, terms whose lo, delta are out of the FP32 range)
// the level comes from the FP64 subtract and divide as before.
constexpr int kQuantFastK = 256;

__global__ void quantize_kernel(const double* __restrict__ u, int64_t count, int K,
                                const double* __restrict__ lo, const double* __restrict__ delta,
                                int64_t levels, int32_t* __restrict__ q, int64_t* status) {
  // per term: fl32(lo), fl32(1/delta) and the term's part of the bound e (1 disables the screen)
  __shared__ float s_lo[kQuantFastK], s_rcp[kQuantFastK], s_e0[kQuantFastK];
  const bool screen = K <= kQuantFastK && levels <= ((int64_t)1 << 24);
  if (screen) {
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      const double l = lo[j], d = delta[j];
      const bool ok = fabs(d) > 1e-30 && fabs(d) < 1e30 && fabs(l) < 1e30;
      s_lo[j] = ok ? (float)l : 0.0f;
      s_rcp[j] = ok ? (float)(1.0 / d) : 0.0f;
      s_e0[j] = ok ? (float)fmin(4.0 * 0x1p-24 * fabs(l) / fabs(d) + 0x1p-40, 1.0) : 1.0f;
    }
  }
  __syncthreads();
  unsigned nonfinite = 0, saturated = 0;
  const double top = (double)(levels - 1);
  const float topf = (float)(levels - 1);               // exact when the screen is on
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int k = (int)(i % K);                                   // term of element i, advanced below
  const int kstep = (int)(stride % K);
  for (; i < count; i += stride) {
    const double v = u[i];
    int32_t r = 0;
    float y = 0.0f, ry = 0.0f, e = 1.0f;
    if (screen) {
      y = __fmul_rn(__fsub_rn((float)v, s_lo[k]), s_rcp[k]);
      ry = rintf(y);
      e = fmaf(fabsf(y), 0x1p-21f, s_e0[k]);
    }
    if (fabsf(y - ry) < 0.5f - e) {                       // false for NaN or infinite y
      if (ry < 0.0f) {
        ++saturated;
        r = 0;
      } else if (ry > topf) {
        ++saturated;
        r = (int32_t)(levels - 1);
      } else {
        r = (int32_t)ry;
      }
    } else if (!isfinite(v)) {
      ++nonfinite;
    } else {
      // one IEEE subtract, one IEEE divide (no contraction), round half to even
      const double x = rint(__ddiv_rn(__dsub_rn(v, lo[k]), delta[k]));
      if (x < 0.0) {
        ++saturated;
        r = 0;
      } else if (x > top) {
        ++saturated;
        r = (int32_t)(levels - 1);
      } else {
        r = (int32_t)x;
      }
    }
    q[i] = r;
    k += kstep;
    if (k >= K) k -= K;
  }
  if (status) {
    // warp-aggregate the counters, one atomic per warp and word
    for (int off = 16; off > 0; off >>= 1) {
      nonfinite += __shfl_down_sync(0xffffffffu, nonfinite, off);
      saturated += __shfl_down_sync(0xffffffffu, saturated, off);
    }
    if ((threadIdx.x & 31) == 0) {
      if (nonfinite) atomicAdd((unsigned long long*)&status[REDO_STATUS_NONFINITE], nonfinite);
      if (saturated) atomicAdd((unsigned long long*)&status[REDO_STATUS_SATURATED], saturated);
    }
  }
}

cudaError_t launch_quantize(const double* u, int64_t count, int K, const double* lo,
                            const double* delta, int64_t levels, int32_t* q, int64_t* status,
                            cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  quantize_kernel<<<(unsigned)blocks, 256, 0, s>>>(u, count, K, lo, delta, levels, q, status);
  return cudaGetLastError();
}

// ============================================================================
// GRAPE update (Section III, Fig. fc): u <- clamp(u + step * dF/du, lo_k, hi_k)
// ============================================================================
__global__ void grape_step_kernel(double* __restrict__ u, const double* __restrict__ g,
                                  int64_t count, int64_t per_pulse, int K,
                                  const double* __restrict__ lo, const double* __restrict__ delta,
                                  int64_t levels, double step, const double* __restrict__ scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % K);
    const double l = lo[k], h = l + delta[k] * (double)(levels - 1);
    const double st = scale ? step * scale[i / per_pulse] : step;
    double v = fma(st, g[i], u[i]);
    v = v < l ? l : (v > h ? h : v);
    u[i] = v;
  }
}

// Adam ascent on the coefficients: m, v moments per coefficient, bias-corrected,
// u <- clamp(u + lr * mhat / (sqrt(vhat) + eps), lo_k, hi_k)
__global__ void grape_adam_kernel(double* __restrict__ u, const double* __restrict__ g,
                                  double* __restrict__ m, double* __restrict__ v, int64_t count, int K,
                                  const double* __restrict__ lo, const double* __restrict__ delta,
                                  int64_t levels, double lr, double b1, double b2, double eps,
                                  double c1, double c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % K);
    const double l = lo[k], h = l + delta[k] * (double)(levels - 1);
    const double gi = g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    double x = u[i] + lr * (mi / c1) / (sqrt(vi / c2) + eps);
    x = x < l ? l : (x > h ? h : x);
    u[i] = x;
  }
}

cudaError_t launch_grape_adam(double* u, const double* g, double* m, double* v, int64_t count, int K,
                              const double* lo, const double* delta, int64_t levels, int step, double lr,
                              double b1, double b2, double eps, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
  grape_adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(u, g, m, v, count, K, lo, delta, levels, lr, b1,
                                                     b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_grape_step(double* u, const double* g, int64_t count, int64_t per_pulse, int K,
                              const double* lo, const double* delta, int64_t levels, double step,
                              const double* scale, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  grape_step_kernel<<<(unsigned)blocks, 256, 0, s>>>(u, g, count, per_pulse, K, lo, delta, levels,
                                                     step, scale);
  return cudaGetLastError();
}

// Per-N tiling: 256 threads per chain for N >= 16; smaller N packs several
// independent chains into one CTA.
template <int N> struct Tiling;
template <> struct Tiling<64> { static constexpr int TM = 4, TN = 4, CH = 1; };
template <> struct Tiling<32> { static constexpr int TM = 2, TN = 2, CH = 1; };
template <> struct Tiling<16> { static constexpr int TM = 1, TN = 1, CH = 1; };
template <> struct Tiling<8> { static constexpr int TM = 1, TN = 1, CH = 4; };
template <> struct Tiling<4> { static constexpr int TM = 1, TN = 1, CH = 16; };
template <> struct Tiling<2> { static constexpr int TM = 1, TN = 1, CH = 64; };

// ============================================================================
// FP64 operator table: scaling-and-squaring Taylor exponential, one CTA per
// operator.  exp(A) with A = -i dt theta H: halve A until ||A||_1 <= 1/2,
// sum the Taylor series by Horner's rule to the first degree m whose
// remainder bound ||A||^(m+1)/(m+1)! is below 1e-18, then square back.
// ============================================================================
template <int N>
__global__ void __launch_bounds__(SmemMM<double, N, (N >= 64 ? 4 : (N >= 32 ? 2 : 1)),
                                         (N >= 64 ? 4 : (N >= 32 ? 2 : 1))>::THREADS)
table_expm_kernel(const double2* __restrict__ H0, const double2* __restrict__ Hk, int K,
                  int digits, int base, double dt, const double* __restrict__ lo,
                  const double* __restrict__ delta, int64_t entries, double2* __restrict__ T,
                  double2* __restrict__ D, double2* __restrict__ Dh) {
  constexpr int TM = (N >= 64 ? 4 : (N >= 32 ? 2 : 1));
  using MM = SmemMM<double, N, TM, TM>;
  constexpr int N2 = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* P = A + N2;
  __shared__ double colsum[N];
  const int lt = threadIdx.x;
  const int64_t e = blockIdx.x;
  const double2* H;
  double theta;
  double2* out;
  if (e >= entries) {
    // the drift step, and (block entries + 1) the half drift step of the symmetric split
    H = H0;
    theta = e == entries ? 1.0 : 0.5;
    out = e == entries ? D : Dh;
  } else {
    const int c = (int)(e % base);
    const int j = (int)((e / base) % digits);
    const int k = (int)(e / ((int64_t)base * digits));
    H = Hk + (int64_t)k * N2;
    if (j == 0) {
      theta = __dadd_rn(lo[k], __dmul_rn((double)c, delta[k]));  // no contraction
    } else {
      double bj = 1.0;
      for (int i = 0; i < j; ++i) bj *= (double)base;
      theta = __dmul_rn((double)c * bj, delta[k]);
    }
    out = T + e * N2;
  }
  const double sc = dt * theta;
  for (int i = lt; i < N2; i += MM::THREADS) {
    const double2 h = H[i];
    A[i] = make_double2(sc * h.y, -sc * h.x);   // -i sc (h.x + i h.y)
  }
  __syncthreads();
  if (lt < N) {
    double s = 0.0;
    for (int r = 0; r < N; ++r) s += hypot(A[r * N + lt].x, A[r * N + lt].y);
    colsum[lt] = s;
  }
  __syncthreads();
  double nrm = 0.0;
  for (int i = 0; i < N; ++i) nrm = fmax(nrm, colsum[i]);
  int sq = 0;
  while (nrm > 0.5 && sq < 1000) {
    nrm *= 0.5;
    ++sq;
  }
  int m = 0;
  if (nrm > 0.0) {
    double term = nrm;  // nrm^(m+1)/(m+1)! for m = 0
    m = 1;
    term = term * nrm / 2.0;
    while (term > 1e-18 && m < 30) {
      ++m;
      term = term * nrm / (double)(m + 1);
    }
  }
  const double scale = ldexp(1.0, -sq);
  for (int i = lt; i < N2; i += MM::THREADS) {
    const double2 a = A[i];
    A[i] = make_double2(a.x * scale, a.y * scale);
    P[i] = make_double2((i / N == i % N) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  double2 Y[TM][TM];
  for (int it = m; it >= 1; --it) {
    MM::run(A, P, lt, Y);
    __syncthreads();
    const double inv = 1.0 / (double)it;
    const int ty = lt / MM::TX, tx = lt % MM::TX;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TM; ++c) {
        const int r = ty + MM::TY * a, col = tx + MM::TX * c;
        P[r * N + col] = make_double2(Y[a][c].x * inv + (r == col ? 1.0 : 0.0), Y[a][c].y * inv);
      }
    __syncthreads();
  }
  for (int it = 0; it < sq; ++it) {
    MM::run(P, P, lt, Y);
    __syncthreads();
    MM::store(P, lt, Y);
    __syncthreads();
  }
  for (int i = lt; i < N2; i += MM::THREADS) out[i] = P[i];
}

// T[0][0][c] <- T[0][0][c] * D  (drift applied first in time)
template <int N>
__global__ void __launch_bounds__(SmemMM<double, N, (N >= 64 ? 4 : (N >= 32 ? 2 : 1)),
                                         (N >= 64 ? 4 : (N >= 32 ? 2 : 1))>::THREADS)
table_fold_kernel(double2* __restrict__ T, const double2* __restrict__ D) {
  constexpr int TM = (N >= 64 ? 4 : (N >= 32 ? 2 : 1));
  using MM = SmemMM<double, N, TM, TM>;
  constexpr int N2 = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* X = A + N2;
  double2* Tc = T + (int64_t)blockIdx.x * N2;
  for (int i = threadIdx.x; i < N2; i += MM::THREADS) {
    A[i] = Tc[i];
    X[i] = D[i];
  }
  __syncthreads();
  double2 Y[TM][TM];
  MM::run(A, X, threadIdx.x, Y);
  __syncthreads();
  MM::store(A, threadIdx.x, Y);
  __syncthreads();
  for (int i = threadIdx.x; i < N2; i += MM::THREADS) Tc[i] = A[i];
}

// Process 3 of Section II: the operator of every level q, evaluated once as the
// product of its digit operators, E[k][q] = T[k][d-1][c_{d-1}] ... T[k][0][c_0].
template <int N>
__global__ void __launch_bounds__(SmemMM<double, N, SqTile<N>::TM, SqTile<N>::TM>::THREADS)
table_expand_kernel(const double2* __restrict__ T, int d, int base, int64_t levels,
                    double2* __restrict__ E) {
  constexpr int TM = SqTile<N>::TM;
  using MM = SmemMM<double, N, TM, TM>;
  constexpr int N2 = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);
  double2* X = A + N2;
  const int64_t e = blockIdx.x;
  const int64_t k = e / levels, q = e % levels;
  const int lt = threadIdx.x;
  int64_t qq = q;
  const double2* T0 = T + ((k * d + 0) * base + qq % base) * N2;
  for (int i = lt; i < N2; i += MM::THREADS) X[i] = T0[i];
  double2 Y[TM][TM];
  for (int j = 1; j < d; ++j) {
    qq /= base;
    const double2* Tj = T + ((k * d + j) * base + qq % base) * N2;
    __syncthreads();
    for (int i = lt; i < N2; i += MM::THREADS) A[i] = Tj[i];
    __syncthreads();
    MM::run(A, X, lt, Y);
    __syncthreads();
    MM::store(X, lt, Y);
  }
  __syncthreads();
  for (int i = lt; i < N2; i += MM::THREADS) E[e * N2 + i] = X[i];
}

template <int N>
static cudaError_t table_expand_n(const double2* T, int K, int d, int base, int64_t levels,
                                  double2* E, cudaStream_t s) {
  using MM = SmemMM<double, N, SqTile<N>::TM, SqTile<N>::TM>;
  const size_t smem = 2 * sizeof(double2) * N * N;
  cudaError_t e = cudaFuncSetAttribute(table_expand_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  table_expand_kernel<N><<<(unsigned)((int64_t)K * levels), MM::THREADS, smem, s>>>(T, d, base, levels, E);
  return cudaGetLastError();
}

cudaError_t launch_table_expand(const redo_table* t, double2* E, cudaStream_t s) {
  switch (t->N) {
    case 2: return table_expand_n<2>(t->T64, t->K, t->digits, t->base, t->levels, E, s);
    case 4: return table_expand_n<4>(t->T64, t->K, t->digits, t->base, t->levels, E, s);
    case 8: return table_expand_n<8>(t->T64, t->K, t->digits, t->base, t->levels, E, s);
    case 16: return table_expand_n<16>(t->T64, t->K, t->digits, t->base, t->levels, E, s);
    case 32: return table_expand_n<32>(t->T64, t->K, t->digits, t->base, t->levels, E, s);
    case 64: return table_expand_n<64>(t->T64, t->K, t->digits, t->base, t->levels, E, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t table_expm_n(const redo_table* t, const double2* H0, const double2* Hk,
                                cudaStream_t s) {
  constexpr int TM = (N >= 64 ? 4 : (N >= 32 ? 2 : 1));
  using MM = SmemMM<double, N, TM, TM>;
  const size_t smem = 2 * sizeof(double2) * N * N;
  cudaError_t e = cudaFuncSetAttribute(table_expm_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  table_expm_kernel<N><<<(unsigned)(t->entries + (t->Dh64 ? 2 : 1)), MM::THREADS, smem, s>>>(
      H0, Hk, t->K, t->digits, t->base, t->dt, t->d_lo, t->d_delta, t->entries, t->T64, t->D64, t->Dh64);
  return cudaGetLastError();
}

template <int N>
static cudaError_t table_fold_n(const redo_table* t, cudaStream_t s) {
  constexpr int TM = (N >= 64 ? 4 : (N >= 32 ? 2 : 1));
  using MM = SmemMM<double, N, TM, TM>;
  const size_t smem = 2 * sizeof(double2) * N * N;
  cudaError_t e = cudaFuncSetAttribute(table_fold_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  table_fold_kernel<N><<<(unsigned)t->base, MM::THREADS, smem, s>>>(t->T64, t->D64);
  return cudaGetLastError();
}

#define REDO_DISPATCH_N(N_, CALL)          \
  switch (N_) {                            \
    case 2: return CALL<2>;                \
    case 4: return CALL<4>;                \
    case 8: return CALL<8>;                \
    case 16: return CALL<16>;              \
    case 32: return CALL<32>;              \
    case 64: return CALL<64>;              \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_table_expm(const redo_table* t, const double2* H0, const double2* Hk,
                              cudaStream_t s) {
  switch (t->N) {
    case 2: return table_expm_n<2>(t, H0, Hk, s);
    case 4: return table_expm_n<4>(t, H0, Hk, s);
    case 8: return table_expm_n<8>(t, H0, Hk, s);
    case 16: return table_expm_n<16>(t, H0, Hk, s);
    case 32: return table_expm_n<32>(t, H0, Hk, s);
    case 64: return table_expm_n<64>(t, H0, Hk, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_table_fold_drift(const redo_table* t, cudaStream_t s) {
  switch (t->N) {
    case 2: return table_fold_n<2>(t, s);
    case 4: return table_fold_n<4>(t, s);
    case 8: return table_fold_n<8>(t, s);
    case 16: return table_fold_n<16>(t, s);
    case 32: return table_fold_n<32>(t, s);
    case 64: return table_fold_n<64>(t, s);
    default: return cudaErrorInvalidValue;
  }
}

// Level operators in closed form for controls with H_k^2 = a_k^2 I and one nonzero per row,
// h_k[i] at column i ^ m_k (every Pauli string):
//     exp(-i dt theta H_k) = cos(a_k dt theta) I - i sin(a_k dt theta) / a_k H_k,
// theta = lo_k + q delta_k (the level value, no contraction), with the diagonal drift of term 0
// folded on the right (column j scaled by D[j][j]).  One thread per entry of E [K][levels][N][N];
// only the two nonzeros of a row evaluate the sine and cosine.
__global__ void levels_closed_form_kernel(int N, int K, int64_t levels, double dt, const double* __restrict__ lo,
                                          const double* __restrict__ delta, const int32_t* __restrict__ xm,
                                          const double2* __restrict__ xh, const double* __restrict__ xa,
                                          const double2* __restrict__ D, double2* __restrict__ E) {
  const int64_t n2 = (int64_t)N * N;
  const int64_t total = (int64_t)K * levels * n2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / n2;
    const int r = (int)(idx - e * n2);
    const int i = r / N, j = r - i * N;
    const int k = (int)(e / levels);
    const int64_t q = e - (int64_t)k * levels;
    const int c = i ^ xm[k];
    double2 v = make_double2(0.0, 0.0);
    if (j == i || j == c) {
      const double th = __dadd_rn(lo[k], __dmul_rn((double)q, delta[k]));
      const double ak = xa[k];
      double sn, cs;
      sincos(dt * th * ak, &sn, &cs);
      if (j == c) {
        const double2 h = xh[(int64_t)k * N + i];
        v.x = sn / ak * h.y;            // -i (sin / a) h
        v.y = -sn / ak * h.x;
      }
      if (j == i) v.x += cs;
      if (k == 0) {
        const double2 dj = D[(int64_t)j * N + j];
        v = make_double2(v.x * dj.x - v.y * dj.y, v.x * dj.y + v.y * dj.x);
      }
    }
    E[idx] = v;
  }
}

cudaError_t launch_levels_closed_form(const redo_table* t, const int32_t* xm, const double2* xh, const double* xa,
                                      double2* E, cudaStream_t s) {
  const int64_t total = (int64_t)t->K * t->levels * t->N * t->N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  levels_closed_form_kernel<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(
      t->N, t->K, t->levels, t->dt, t->d_lo, t->d_delta, xm, xh, xa, t->D64, E);
  return cudaGetLastError();
}

__global__ void to_fp32_kernel(const double2* __restrict__ src, float2* __restrict__ dst,
                               int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t launch_to_fp32(const double2* src, float2* dst, int64_t count, cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  to_fp32_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

// ============================================================================
// Segmented product chains (Eq. exp2prod per term, chained over time)
// ============================================================================

// Factor f of pulse b is table operator (k, j, c) with
//   n = f / (K d), k = (f mod K d) / d, j = f mod d, c = floor(q[b][n][k] / base^j) mod base.
// Factor 0 (drift-folded digit 0 of term 0, step 0) is applied first.
// With amplitude/phase controls (pd non-null) every step opens with a diagonal factor:
// factor r = 0 of step n is P_n = diag(pd[b][n]) and r = 1.. are the table factors.
template <typename R>
struct GatherSrc {
  const cplx<R>* T;
  const int32_t* q;
  int64_t M;
  int K, d, base;
  int64_t levels;
  int64_t* status;
  int64_t fps;                // factors per step
  const double2* pd;          // [B][M][N] or nullptr
  int N;
  // diagonal of factor f when it is a phase factor, else nullptr
  __device__ __forceinline__ const double2* phase(int64_t b, int64_t f) const {
    if (!pd) return nullptr;
    const int64_t n = f / fps;
    return f - n * fps == 0 ? pd + (b * M + n) * N : nullptr;
  }
  // table operator of factor f (nullptr for a phase factor)
  __device__ __forceinline__ const cplx<R>* addr(int64_t b, int64_t f, int N2) const {
    const int64_t n = f / fps;
    int r = (int)(f - n * fps);
    if (pd) {
      if (r == 0) return nullptr;
      --r;
    }
    const int k = r / d, j = r - k * d;
    int32_t qv = q[(b * M + n) * K + k];
    if (qv < 0 || qv >= levels) {
      if (status) atomicAdd((unsigned long long*)&status[REDO_STATUS_BADINDEX], 1ull);
      qv = 0;
    }
    for (int i = 0; i < j; ++i) qv /= base;
    const int c = qv % base;
    return T + ((int64_t)(k * d + j) * base + c) * N2;
  }
};

// Factor f of unit b is P[b][f] (an ordered list of earlier segment products).
template <typename R>
struct DenseSrc {
  const cplx<R>* P;
  int64_t per_unit;
  __device__ __forceinline__ const double2* phase(int64_t, int64_t) const { return nullptr; }
  __device__ __forceinline__ const cplx<R>* addr(int64_t b, int64_t f, int N2) const {
    return P + (b * per_unit + f) * N2;
  }
};

template <typename R, int N, int STAGES, class Src>
__global__ void __launch_bounds__(SmemMM<R, N, Tiling<N>::TM, Tiling<N>::TN>::THREADS * Tiling<N>::CH)
chain_kernel(Src src, int64_t units, int64_t segs_per_unit, int64_t seg_len, int64_t total_len,
             cplx<R>* __restrict__ out, int64_t* status, cplx<R>* __restrict__ keep) {
  using TL = Tiling<N>;
  using MM = SmemMM<R, N, TL::TM, TL::TN>;
  constexpr int CH = TL::CH;
  constexpr int N2 = N * N;
  constexpr uint32_t BYTES = (uint32_t)(N2 * sizeof(cplx<R>));
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cplx<R>* Xall = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* Aall = Xall + CH * N2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Aall + CH * STAGES * N2);
  __shared__ int abort_flag;

  const int ch = threadIdx.x / MM::THREADS;
  const int lt = threadIdx.x - ch * MM::THREADS;
  const int64_t G = units * segs_per_unit;

  // every thread derives the lengths of all chains of the CTA (uniform loop bound)
  int64_t maxlen = 0, my_len = 0, my_f0 = 0, my_unit = 0;
  for (int c = 0; c < CH; ++c) {
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    int64_t len = 0, f0 = 0;
    if (g < G) {
      const int64_t s = g % segs_per_unit;
      f0 = s * seg_len;
      int64_t f1 = f0 + seg_len;
      if (f1 > total_len) f1 = total_len;
      len = f1 > f0 ? f1 - f0 : 0;
    }
    if (len > maxlen) maxlen = len;
    if (c == ch) {
      my_len = len;
      my_f0 = f0;
      my_unit = g / segs_per_unit;
    }
  }
  const int64_t my_g = (int64_t)blockIdx.x * CH + ch;
  cplx<R>* X = Xall + ch * N2;
  cplx<R>* A = Aall + ch * STAGES * N2;
  uint64_t* bar = bars + ch * STAGES;

  if (threadIdx.x == 0) abort_flag = 0;
  if (lt < STAGES) mbar_init(&bar[lt], 1);
  fence_mbarrier_init();
  for (int i = lt; i < N2; i += MM::THREADS)
    X[i] = cmake<R>((i / N == i % N) ? R(1) : R(0), R(0));
  __syncthreads();
  // a phase factor has no operand to copy: its stage completes on the arrival alone
  auto issue = [&](int st, int64_t f) {
    const cplx<R>* op = src.addr(my_unit, f, N2);
    if (op) {
      mbar_arrive_expect_tx(&bar[st], BYTES);
      bulk_load(A + st * N2, op, BYTES, &bar[st]);
    } else {
      mbar_arrive(&bar[st]);
    }
  };
  if (lt == 0) {
    for (int s = 0; s < STAGES && s < my_len; ++s) issue(s, my_f0 + s);
  }
  cplx<R> Y[TL::TM][TL::TN];
  for (int64_t t = 0; t < maxlen; ++t) {
    const int stage = (int)(t % STAGES);
    const uint32_t parity = (uint32_t)((t / STAGES) & 1);
    const bool active = t < my_len;
    if (active) {
      if (!mbar_wait_bounded(&bar[stage], parity)) {
        abort_flag = 1;
      } else {
        const double2* ph = src.phase(my_unit, my_f0 + t);
        if (ph)
          MM::scale_rows(ph, X, lt, Y);
        else
          MM::run(A + stage * N2, X, lt, Y);
      }
    }
    __syncthreads();
    if (abort_flag) break;
    if (active) {
      MM::store(X, lt, Y);
      if (keep) MM::store(keep + (my_g * seg_len + t) * N2, lt, Y);   // every partial product kept
      if (lt == 0 && t + STAGES < my_len) {
        fence_proxy_async_smem();
        issue(stage, my_f0 + t + STAGES);
      }
    }
    __syncthreads();
  }
  if (abort_flag) {
    if (threadIdx.x == 0 && status)
      atomicAdd((unsigned long long*)&status[REDO_STATUS_TIMEOUT], 1ull);
    return;
  }
  if (my_g < G) {
    cplx<R>* o = out + my_g * N2;
    for (int i = lt; i < N2; i += MM::THREADS) o[i] = X[i];
  }
}

// ----------------------------------------------------------------------------
// Small N (N * sizeof(R) <= 64: N <= 16 in FP32, <= 8 in FP64) with a table that fits in
// shared memory: the table is staged once per CTA and a thread carries one column of one
// segment product in registers, u <- T_f u factor after factor (T_f read from shared memory,
// two entries per 16-byte load in FP32), with no barrier inside the chain.
// ----------------------------------------------------------------------------
constexpr int kColsThreads = 256;
constexpr size_t kColsTableBytes = 200 * 1024;

template <typename R>
static bool cols_eligible(const redo_table* t, const ChainPlan& p) {
  const size_t table = (size_t)t->entries * t->N * t->N * sizeof(cplx<R>);
  return !p.pd && t->N * sizeof(R) <= 64 && table <= kColsTableBytes;
}

template <typename R, int N>
__global__ void __launch_bounds__(kColsThreads, 1)
chain_cols_kernel(const cplx<R>* __restrict__ T, int64_t entries, GatherSrc<R> src, int64_t units,
                  int64_t segs, int64_t seg_len, int64_t total_len, cplx<R>* __restrict__ out,
                  cplx<R>* __restrict__ keep) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* Ts = reinterpret_cast<cplx<R>*>(smem_raw);
  for (int64_t i = threadIdx.x; i < entries * N2; i += kColsThreads) Ts[i] = T[i];
  __syncthreads();
  const int c = threadIdx.x % N;
  const int64_t g = (int64_t)blockIdx.x * (kColsThreads / N) + threadIdx.x / N;
  if (g >= units * segs) return;
  const int64_t unit = g / segs, sgi = g - unit * segs;
  if (c != 0) src.status = nullptr;               // a bad level index is counted once per factor
  const int64_t f0 = sgi * seg_len;
  const int64_t f1 = f0 + seg_len < total_len ? f0 + seg_len : total_len;
  cplx<R> u[N];
#pragma unroll
  for (int r = 0; r < N; ++r) u[r] = cmake<R>(r == c ? R(1) : R(0), R(0));
  for (int64_t f = f0; f < f1; ++f) {
    const cplx<R>* A = Ts + (src.addr(unit, f, N2) - src.T);
    cplx<R> v[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      cplx<R> sacc = cmake<R>(R(0), R(0));
      if constexpr (std::is_same<R, float>::value && N % 2 == 0) {
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
    if (keep) {
      cplx<R>* kp = keep + (g * seg_len + (f - f0)) * N2;
#pragma unroll
      for (int r = 0; r < N; ++r) kp[r * N + c] = u[r];
    }
  }
  cplx<R>* o = out + g * N2;
#pragma unroll
  for (int r = 0; r < N; ++r) o[r * N + c] = u[r];
}

template <typename R, int N>
struct ChainCfg {
  static constexpr int STAGES = (N >= 64) ? 2 : ((N >= 32) ? 3 : 4);
  static constexpr int THREADS = SmemMM<R, N, Tiling<N>::TM, Tiling<N>::TN>::THREADS * Tiling<N>::CH;
  static constexpr size_t SMEM =
      (size_t)Tiling<N>::CH * (1 + STAGES) * N * N * sizeof(cplx<R>) +
      (size_t)Tiling<N>::CH * STAGES * sizeof(uint64_t);
};

template <typename R, int N, class Src>
static cudaError_t launch_chain_n(Src src, int64_t units, int64_t segs, int64_t seg_len,
                                  int64_t total_len, cplx<R>* out, int64_t* status,
                                  cudaStream_t s, cplx<R>* keep = nullptr) {
  using C = ChainCfg<R, N>;
  auto kern = chain_kernel<R, N, C::STAGES, Src>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e != cudaSuccess) return e;
  const int64_t G = units * segs;
  const int64_t blocks = (G + Tiling<N>::CH - 1) / Tiling<N>::CH;
  if (blocks == 0) return cudaSuccess;
  kern<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(src, units, segs, seg_len, total_len, out,
                                                      status, keep);
  return cudaGetLastError();
}

template <typename R>
static int chain_slots(int N, int num_sms) {
  size_t smem = 0;
  int ch = 1;
  switch (N) {
#define CASE(n)                         \
  case n:                               \
    smem = ChainCfg<R, n>::SMEM;        \
    ch = Tiling<n>::CH;                 \
    break;
    CASE(2) CASE(4) CASE(8) CASE(16) CASE(32) CASE(64)
#undef CASE
    default: break;
  }
  int per_sm = smem ? (int)((220 * 1024) / smem) : 1;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  return num_sms * per_sm * ch;
}

ChainPlan plan_chain(const redo_table* t, int64_t B, int64_t M, int prec, bool phase) {
  ChainPlan p;
  p.B = B;
  p.M = M;
  p.fps = (int64_t)t->K * t->digits + (phase ? 1 : 0);
  p.F = M * p.fps;
  int slots = prec == REDO_FP64 ? chain_slots<double>(t->N, t->num_sms)
                                : chain_slots<float>(t->N, t->num_sms);
  const bool cols = !phase && (prec == REDO_FP64 ? cols_eligible<double>(t, p) : cols_eligible<float>(t, p));
  // column chains: four CTAs of 256 / N segment products per SM, one per SM at a time
  if (cols) slots = 2 * t->num_sms * (kColsThreads / t->N);
  // about two segments per resident chain, each at least 16 factors long
  int64_t S = (2 * (int64_t)slots + B - 1) / (B > 0 ? B : 1);
  const int64_t max_s = (p.F + 15) / 16;
  if (S > max_s) S = max_s;
  if (S > 1024) S = 1024;
  if (S < 1) S = 1;
  p.seg_len = p.F > 0 ? (p.F + S - 1) / S : 0;
  p.S = p.seg_len > 0 ? (p.F + p.seg_len - 1) / p.seg_len : 1;
  return p;
}

size_t chain_workspace_bytes(const redo_table* t, const ChainPlan& p, int prec) {
  const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t n2 = (size_t)t->N * t->N;
  const size_t seg = (size_t)p.B * p.S * n2 * el;
  const size_t prod = (size_t)p.B * n2 * el;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up(seg) + up(prod);
}

template <typename R>
static cudaError_t chain_segments_t(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                    void* seg_out, int64_t* status, cudaStream_t s, void* keep) {
  cplx<R>* kp = (cplx<R>*)keep;
  GatherSrc<R> src;
  src.T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  src.q = q;
  src.M = p.M;
  src.K = t->K;
  src.d = t->digits;
  src.base = t->base;
  src.levels = t->levels;
  src.status = status;
  src.fps = p.fps > 0 ? p.fps : (int64_t)t->K * t->digits;
  src.pd = p.pd;
  src.N = t->N;
  cplx<R>* out = (cplx<R>*)seg_out;
  if (cols_eligible<R>(t, p)) {
    const size_t smem = (size_t)t->entries * t->N * t->N * sizeof(cplx<R>);
    const int64_t G = p.B * p.S;
    if (G == 0) return cudaSuccess;
#define COLS_CASE(n)                                                                                        \
  case n:                                                                                                   \
    if constexpr (n * sizeof(R) <= 64) {                                                                    \
      cudaError_t e = cudaFuncSetAttribute(chain_cols_kernel<R, n>,                                         \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
      if (e != cudaSuccess) return e;                                                                       \
      chain_cols_kernel<R, n><<<(unsigned)((G + kColsThreads / n - 1) / (kColsThreads / n)), kColsThreads,  \
                                smem, s>>>(src.T, t->entries, src, p.B, p.S, p.seg_len, p.F, out, kp);      \
      return cudaGetLastError();                                                                            \
    }                                                                                                       \
    break;
    switch (t->N) {
      COLS_CASE(2) COLS_CASE(4) COLS_CASE(8) COLS_CASE(16)
      default: break;
    }
#undef COLS_CASE
  }
  switch (t->N) {
    case 2: return launch_chain_n<R, 2>(src, p.B, p.S, p.seg_len, p.F, out, status, s, kp);
    case 4: return launch_chain_n<R, 4>(src, p.B, p.S, p.seg_len, p.F, out, status, s, kp);
    case 8: return launch_chain_n<R, 8>(src, p.B, p.S, p.seg_len, p.F, out, status, s, kp);
    case 16: return launch_chain_n<R, 16>(src, p.B, p.S, p.seg_len, p.F, out, status, s, kp);
    case 32: return launch_chain_n<R, 32>(src, p.B, p.S, p.seg_len, p.F, out, status, s, kp);
    case 64: return launch_chain_n<R, 64>(src, p.B, p.S, p.seg_len, p.F, out, status, s, kp);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chain_segments(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                  int prec, void* seg_out, int64_t* status, cudaStream_t s, void* keep) {
  if (prec == REDO_FP64) return chain_segments_t<double>(t, q, p, seg_out, status, s, keep);
  return chain_segments_t<float>(t, q, p, seg_out, status, s, keep);
}

template <typename R>
static cudaError_t chain_combine_t(const redo_table* t, const ChainPlan& p, const void* seg_in,
                                   void* prod_out, int64_t* status, cudaStream_t s) {
  DenseSrc<R> src;
  src.P = (const cplx<R>*)seg_in;
  src.per_unit = p.S;
  cplx<R>* out = (cplx<R>*)prod_out;
  const int64_t L = p.F > 0 ? p.S : 0;
  switch (t->N) {
    case 2: return launch_chain_n<R, 2>(src, p.B, 1, L, L, out, status, s);
    case 4: return launch_chain_n<R, 4>(src, p.B, 1, L, L, out, status, s);
    case 8: return launch_chain_n<R, 8>(src, p.B, 1, L, L, out, status, s);
    case 16: return launch_chain_n<R, 16>(src, p.B, 1, L, L, out, status, s);
    case 32: return launch_chain_n<R, 32>(src, p.B, 1, L, L, out, status, s);
    case 64: return launch_chain_n<R, 64>(src, p.B, 1, L, L, out, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chain_combine(const redo_table* t, const ChainPlan& p, int prec,
                                 const void* seg_in, void* prod_out, int64_t* status,
                                 cudaStream_t s) {
  if (prec == REDO_FP64) return chain_combine_t<double>(t, p, seg_in, prod_out, status, s);
  return chain_combine_t<float>(t, p, seg_in, prod_out, status, s);
}

// ============================================================================
// Re-unitarisation: Newton-Schulz polar iteration  P <- P (3I - P^dag P) / 2,
// one CTA per matrix.  Converges quadratically to the unitary polar factor
// P (P^dag P)^(-1/2) when ||P^dag P - I|| < 1; the product chains hand it
// matrices within ~1e-3 of unitary, so one step leaves ~1e-6 of that.
// ============================================================================
template <typename Rin, typename Rc, int N, typename Rout = Rc>
__global__ void __launch_bounds__(SmemMM<Rc, N, (N >= 64 ? 4 : (N >= 32 ? 2 : 1)),
                                         (N >= 64 ? 4 : (N >= 32 ? 2 : 1))>::THREADS)
polar_ns_kernel(const cplx<Rin>* __restrict__ in, cplx<Rout>* __restrict__ out, int iters) {
  constexpr int TM = (N >= 64 ? 4 : (N >= 32 ? 2 : 1));
  using MM = SmemMM<Rc, N, TM, TM>;
  constexpr int N2 = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cplx<Rc>* P = reinterpret_cast<cplx<Rc>*>(smem_raw);
  cplx<Rc>* Q = P + N2;
  const int lt = threadIdx.x;
  const int64_t b = blockIdx.x;
  for (int i = lt; i < N2; i += MM::THREADS) {
    const cplx<Rin> v = in[b * N2 + i];
    P[i] = cmake<Rc>((Rc)v.x, (Rc)v.y);
  }
  __syncthreads();
  cplx<Rc> Y[TM][TM];
  const int ty = lt / MM::TX, tx = lt % MM::TX;
  for (int it = 0; it < iters; ++it) {
    if constexpr (MM::TY == MM::TX && TM > 1) {
      MM::ns_half_gram(P, Q, lt);                        // Q = (3I - P^dag P) / 2, half the Gram tiles
    } else {
      MM::run_adj(P, P, lt, Y);                          // G = P^dag P (P read in column order)
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TM; ++c) {
          const int r = ty + MM::TY * a, col = tx + MM::TX * c;
          Q[r * N + col] = cmake<Rc>((r == col ? Rc(1.5) : Rc(0)) - Rc(0.5) * Y[a][c].x,
                                     -Rc(0.5) * Y[a][c].y);
        }
    }
    __syncthreads();
    MM::run(P, Q, lt, Y);                                // P (3I - G) / 2
    __syncthreads();
    MM::store(P, lt, Y);
    __syncthreads();
  }
  for (int i = lt; i < N2; i += MM::THREADS) {
    const cplx<Rc> v = P[i];
    out[b * N2 + i] = cmake<Rout>((Rout)v.x, (Rout)v.y);
  }
}

template <typename Rin, typename Rc, int N, typename Rout = Rc>
static cudaError_t polar_n(const void* in, void* out, int64_t count, int iters, cudaStream_t s) {
  constexpr int TM = (N >= 64 ? 4 : (N >= 32 ? 2 : 1));
  using MM = SmemMM<Rc, N, TM, TM>;
  const size_t smem = 2 * sizeof(cplx<Rc>) * N * N;
  auto kern = polar_ns_kernel<Rin, Rc, N, Rout>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  kern<<<(unsigned)count, MM::THREADS, smem, s>>>((const cplx<Rin>*)in, (cplx<Rout>*)out, iters);
  return cudaGetLastError();
}

template <typename Rin, typename Rc, typename Rout = Rc>
static cudaError_t polar_t(int N, const void* in, void* out, int64_t count, int iters,
                           cudaStream_t s) {
  switch (N) {
    case 2: return polar_n<Rin, Rc, 2, Rout>(in, out, count, iters, s);
    case 4: return polar_n<Rin, Rc, 4, Rout>(in, out, count, iters, s);
    case 8: return polar_n<Rin, Rc, 8, Rout>(in, out, count, iters, s);
    case 16: return polar_n<Rin, Rc, 16, Rout>(in, out, count, iters, s);
    case 32: return polar_n<Rin, Rc, 32, Rout>(in, out, count, iters, s);
    case 64: return polar_n<Rin, Rc, 64, Rout>(in, out, count, iters, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_polar(const redo_table* t, int prec_in, int prec_out, const void* in, void* out,
                         int64_t count, int iters, cudaStream_t s) {
  const bool din = prec_in == REDO_FP64, dout = prec_out == REDO_FP64;
  if (din && dout) return polar_t<double, double>(t->N, in, out, count, iters, s);
  if (!din && dout) return polar_t<float, double>(t->N, in, out, count, iters, s);
  if (!din && !dout) return polar_t<float, float>(t->N, in, out, count, iters, s);
  return cudaErrorInvalidValue;
}

// complex128 in and out, Newton-Schulz arithmetic in FP64 (prec_arith REDO_FP64) or FP32
cudaError_t launch_polar_c128(int N, int prec_arith, const double2* in, double2* out, int64_t count, int iters,
                              cudaStream_t s) {
  if (prec_arith == REDO_FP64) return polar_t<double, double, double>(N, in, out, count, iters, s);
  return polar_t<double, float, double>(N, in, out, count, iters, s);
}

ChainPlan plan_chain_aligned(const redo_table* t, int64_t B, int64_t M, int64_t steps_per_segment,
                             bool phase) {
  ChainPlan p;
  p.B = B;
  p.M = M;
  p.fps = (int64_t)t->K * t->digits + (phase ? 1 : 0);
  p.F = M * p.fps;
  p.seg_len = steps_per_segment * p.fps;
  p.S = p.F > 0 ? (p.F + p.seg_len - 1) / p.seg_len : 1;
  return p;
}

// ============================================================================
// Epilogue: U_out (complex128), tau = Tr(U_T^dag U) and F = |tau|^2 / N^2,
// reduced in FP64 in a fixed order (deterministic).
// ============================================================================
template <typename R>
__global__ void __launch_bounds__(256)
finalize_kernel(int N, const cplx<R>* __restrict__ prod, double2* __restrict__ U_out,
                const double2* __restrict__ U_target, double* __restrict__ F_out,
                double2* __restrict__ tau_out) {
  const int64_t b = blockIdx.x;
  const int N2 = N * N;
  const cplx<R>* P = prod + b * N2;
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < N2; i += blockDim.x) {
    const cplx<R> v = P[i];
    const double2 u = make_double2((double)v.x, (double)v.y);
    if (U_out) U_out[b * N2 + i] = u;
    if (U_target) {
      const double2 g = U_target[i];
      // conj(g) * u
      re = fma(g.x, u.x, re);
      re = fma(g.y, u.y, re);
      im = fma(g.x, u.y, im);
      im = fma(-g.y, u.x, im);
    }
  }
  if (!U_target) return;
  __shared__ double sre[256], sim[256];
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sre[threadIdx.x] += sre[threadIdx.x + w];
      sim[threadIdx.x] += sim[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tr = sre[0], ti = sim[0];
    if (F_out) F_out[b] = (tr * tr + ti * ti) / ((double)N * (double)N);
    if (tau_out) tau_out[b] = make_double2(tr, ti);
  }
}

cudaError_t launch_finalize(const redo_table* t, int64_t B, int prec, const void* prod,
                            void* U_out, const double2* U_target, double* F_out, double2* tau_out,
                            cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  if (prec == REDO_FP64)
    finalize_kernel<double><<<(unsigned)B, 256, 0, s>>>(t->N, (const double2*)prod,
                                                         (double2*)U_out, U_target, F_out, tau_out);
  else
    finalize_kernel<float><<<(unsigned)B, 256, 0, s>>>(t->N, (const float2*)prod,
                                                        (double2*)U_out, U_target, F_out, tau_out);
  return cudaGetLastError();
}

}  // namespace redo
