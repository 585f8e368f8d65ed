// State-to-state GRAPE (Section III's state fidelity): a = <psi_T| U_M ... U_1 |psi0>,
// F_S = |a|^2, and dF_S/du_kn = 2 dt Im(conj(a) <chi| H_k |phi>), where phi is the state
// after the last digit factor of term k in step n and chi = (the later factors)^dag psi_T.
//
// One CTA per pulse.  The forward pass applies the gathered table operators to psi0 one
// matrix-vector product at a time (a warp per row, lanes along the row, so operator reads are
// coalesced); the reverse pass walks the factors from the last one, evaluating the trace where
// a term's last digit sits and then undoing the factor on both vectors with adjoint products
// (a thread per column, rows in order: again coalesced).  Only two N-vectors live in shared
// memory, so the gradient costs O(N^2) per factor and needs no workspace.
#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "tcgen05.cuh"

#include <type_traits>

namespace redo {

namespace {

constexpr int kStTh = 256;

template <typename R>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double out = 0.0;
#pragma unroll
  for (int w = 0; w < kStTh / 32; ++w) out += red[w];
  return out;
}

template <typename R>
__global__ void __launch_bounds__(kStTh)
state_grad_kernel(const cplx<R>* __restrict__ T, const int32_t* __restrict__ q, int N, int64_t M, int K, int d,
                  int base, int64_t levels, const double2* __restrict__ psi0, const double2* __restrict__ psiT,
                  int batched, const int32_t* __restrict__ hk_ptr, const int32_t* __restrict__ hk_col,
                  const int32_t* __restrict__ hk_row, const double2* __restrict__ hk_val, double dt,
                  double* __restrict__ F_out, double* __restrict__ grad, int64_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* v = reinterpret_cast<cplx<R>*>(smem_raw);     // phi
  cplx<R>* w = v + N;                                      // chi
  cplx<R>* tmp = w + N;                                    // product scratch
  __shared__ double red[kStTh / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t b = blockIdx.x;
  const int64_t n2 = (int64_t)N * N;
  const double2* p0 = psi0 + (batched ? b * N : 0);
  const double2* pT = psiT + (batched ? b * N : 0);
  for (int i = tid; i < N; i += kStTh) v[i] = cmake<R>((R)p0[i].x, (R)p0[i].y);
  const int64_t kd = (int64_t)K * d, F = M * kd;
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
    return T + ((int64_t)(k * d + j) * base + qv % base) * n2;
  };
  __syncthreads();
  // forward: v <- A_f v
  for (int64_t f = 0; f < F; ++f) {
    const cplx<R>* A = factor(f);
    for (int r = warp; r < N; r += kStTh / 32) {
      cplx<R> s = cmake<R>(R(0), R(0));
      for (int c = lane; c < N; c += 32) cfma<R>(s, A[(int64_t)r * N + c], v[c]);
      for (int off = 16; off > 0; off >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
      }
      if (lane == 0) tmp[r] = s;
    }
    __syncthreads();
    for (int i = tid; i < N; i += kStTh) v[i] = tmp[i];
    __syncthreads();
  }
  // a = <psi_T | v>
  double ar = 0.0, ai = 0.0;
  for (int i = tid; i < N; i += kStTh) {
    const double2 t = pT[i];
    const double xr = (double)v[i].x, xi = (double)v[i].y;
    ar += t.x * xr + t.y * xi;
    ai += t.x * xi - t.y * xr;
  }
  ar = block_sum<R>(ar, red);
  ai = block_sum<R>(ai, red);
  if (tid == 0 && F_out) F_out[b] = ar * ar + ai * ai;
  if (!grad) return;
  for (int i = tid; i < N; i += kStTh) w[i] = cmake<R>((R)pT[i].x, (R)pT[i].y);
  __syncthreads();
  // reverse: trace at a term's last digit, then v <- A_f^dag v, w <- A_f^dag w
  for (int64_t f = F - 1; f >= 0; --f) {
    const int64_t n = f / kd;
    const int rr = (int)(f - n * kd);
    const int k = rr / d, j = rr - k * d;
    if (j == d - 1) {
      // <w| H_k |v> = sum over the nonzeros (i, c) of conj(w_i) H[i][c] v_c
      const int e0 = hk_ptr[k * (N + 1)], e1 = hk_ptr[k * (N + 1) + N];
      double tr = 0.0, ti = 0.0;
      for (int e = e0 + tid; e < e1; e += kStTh) {
        const int i = hk_row[e], c = hk_col[e];
        const double2 h = hk_val[e];
        const double wr = (double)w[i].x, wi = (double)w[i].y, vr = (double)v[c].x, vi = (double)v[c].y;
        const double hr = h.x * vr - h.y * vi, hi = h.x * vi + h.y * vr;   // H[i][c] v_c
        tr += wr * hr + wi * hi;
        ti += wr * hi - wi * hr;
      }
      tr = block_sum<R>(tr, red);
      ti = block_sum<R>(ti, red);
      if (tid == 0) grad[(b * M + n) * K + k] = 2.0 * dt * (ar * ti - ai * tr);
    }
    const cplx<R>* A = factor(f);
    for (int c = tid; c < N; c += kStTh) {
      cplx<R> sv = cmake<R>(R(0), R(0)), sw = cmake<R>(R(0), R(0));
      for (int r = 0; r < N; ++r) {
        const cplx<R> a = A[(int64_t)r * N + c];
        const cplx<R> ac = cmake<R>(a.x, -a.y);
        cfma<R>(sv, ac, v[r]);
        cfma<R>(sw, ac, w[r]);
      }
      tmp[c] = sv;
      tmp[N + c] = sw;
    }
    __syncthreads();
    for (int i = tid; i < N; i += kStTh) {
      v[i] = tmp[i];
      w[i] = tmp[N + i];
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// The same computation for N >= 64 with every operator streamed through shared memory:
// a producer warp copies each factor's rows in 64 KB chunks (bulk copies into a ring of
// stages, mbarrier-tracked), 16 compute warps consume them, so the operator stream keeps up
// to ~190 KB in flight instead of one dependent load per thread.  Forward: warps take rows
// of a chunk, lanes its columns.  Reverse: threads take columns (and, for N < 512, one of
// 512/N groups of the chunk's rows, added in shared memory at the factor's end).  The
// compute warps meet at a barrier per factor, which also carries their agreement on every
// bounded wait of that factor.
// ----------------------------------------------------------------------------
constexpr int kSgWarps = 16;
constexpr int kSgCompute = 32 * kSgWarps;
constexpr int kSgThreads = kSgCompute + 32;
constexpr uint32_t kSgChunk = 64 * 1024;
constexpr uint32_t kSgLimit = 1u << 24;

template <typename R>
__global__ void __launch_bounds__(kSgThreads, 1)
state_grad_stream_kernel(const cplx<R>* __restrict__ T, const int32_t* __restrict__ q, int N, int64_t M, int K,
                         int d, int base, int64_t levels, const double2* __restrict__ psi0,
                         const double2* __restrict__ psiT, int batched, const int32_t* __restrict__ hk_ptr,
                         const int32_t* __restrict__ hk_col, const int32_t* __restrict__ hk_row,
                         const double2* __restrict__ hk_val, double dt, double* __restrict__ F_out,
                         double* __restrict__ grad, int64_t* status, int stages, int rows,
                         const double* __restrict__ obs, double* __restrict__ expect) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint8_t* ring = smem_raw;
  cplx<R>* v = reinterpret_cast<cplx<R>*>(ring + (size_t)stages * kSgChunk);
  cplx<R>* w = v + N;
  cplx<R>* tv = w + N;
  cplx<R>* tw = tv + N;
  cplx<R>* scratch = tw + N;                         // [2][kSgCompute] reverse partial sums
  uint64_t* full = reinterpret_cast<uint64_t*>(scratch + 2 * kSgCompute);
  uint64_t* empty = full + stages;
  __shared__ double red[kSgWarps];
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t b = blockIdx.x;
  const int64_t kd = (int64_t)K * d, F = M * kd;
  const int cpf = N / rows;
  const uint32_t cbytes = (uint32_t)((size_t)rows * N * sizeof(cplx<R>));
  const int passes = grad ? 2 : 1;
  const int64_t total = (int64_t)passes * F * cpf;
  const double2* p0 = psi0 + (batched ? b * N : 0);
  const double2* pT = psiT ? psiT + (batched ? b * N : 0) : nullptr;
  if (tid == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kSgWarps);
    }
    abort_flag = 0;
    fence_mbarrier_init();
  }
  for (int i = tid; i < N; i += kSgThreads) v[i] = cmake<R>((R)p0[i].x, (R)p0[i].y);
  __syncthreads();

  if (warp == kSgWarps) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t i = 0; i < total; ++i) {
        const int64_t pass = i / (F * cpf), rem = i - pass * F * cpf;
        const int64_t fi = rem / cpf;
        const int ch = (int)(rem - fi * cpf);
        const int64_t f = pass == 0 ? fi : F - 1 - fi;
        const int s = (int)(i % stages);
        const uint32_t u = (uint32_t)(i / stages);
        if (abort_flag || (u > 0 && !mbar_wait_bounded_n(&empty[s], (u - 1) & 1, kSgLimit))) {
          abort_flag = 1;
          break;
        }
        const int64_t n = f / kd;
        const int rr = (int)(f - n * kd);
        const int k = rr / d, j = rr - k * d;
        int32_t qv = q[(b * M + n) * K + k];
        if (qv < 0 || qv >= levels) {
          if (status && pass == 0 && ch == 0) atomicAdd((unsigned long long*)&status[REDO_STATUS_BADINDEX], 1ull);
          qv = 0;
        }
        for (int x = 0; x < j; ++x) qv /= base;
        const cplx<R>* src = T + ((int64_t)(k * d + j) * base + qv % base) * N * N + (int64_t)ch * rows * N;
        mbar_arrive_expect_tx(&full[s], cbytes);
        bulk_load(ring + (size_t)s * kSgChunk, src, cbytes, &full[s]);
        issued = i + 1;
      }
      // let the copies in flight land before the CTA leaves
      for (int64_t i = issued - 1; i >= 0 && i >= issued - stages; --i)
        mbar_wait_bounded_n(&full[i % stages], (uint32_t)((i / stages) & 1), kSgLimit);
    }
    return;
  }

  // -------------------------------------------------------------------- compute warps
  int64_t idx = 0;
  bool ok = true;
  auto chunk = [&]() -> const cplx<R>* {
    const int s = (int)(idx % stages);
    if (ok && !mbar_wait_bounded_n(&full[s], (uint32_t)((idx / stages) & 1), kSgLimit)) ok = false;
    return reinterpret_cast<const cplx<R>*>(ring + (size_t)s * kSgChunk);
  };
  auto release = [&]() {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[idx % stages]);
    ++idx;
  };
  auto block_sum = [&](double x) -> double {
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    tc::named_barrier(1, kSgCompute);
    if (lane == 0) red[warp] = x;
    tc::named_barrier(1, kSgCompute);
    double o = 0.0;
#pragma unroll
    for (int i = 0; i < kSgWarps; ++i) o += red[i];
    return o;
  };
  // simulation (expect non-null): <O>(t_n) = sum_a o_a |psi_n[a]|^2 after every step
  auto observe = [&](int64_t n) {
    double x = 0.0;
    for (int i = tid; i < N; i += kSgCompute) {
      const double vr = (double)v[i].x, vi = (double)v[i].y;
      x += obs[i] * (vr * vr + vi * vi);
    }
    x = block_sum(x);
    if (tid == 0) expect[b * (M + 1) + n] = x;
  };
  if (expect) observe(0);
  // forward: v <- A_f v
  for (int64_t f = 0; f < F; ++f) {
    for (int ch = 0; ch < cpf; ++ch) {
      const cplx<R>* A = chunk();
      if (ok) {
        for (int rr = warp; rr < rows; rr += kSgWarps) {
          cplx<R> sacc = cmake<R>(R(0), R(0));
          for (int c = lane; c < N; c += 32) cfma<R>(sacc, A[(int64_t)rr * N + c], v[c]);
          for (int off = 16; off > 0; off >>= 1) {
            sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, off);
            sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, off);
          }
          if (lane == 0) tv[ch * rows + rr] = sacc;
        }
      }
      release();
    }
    ok = tc::named_barrier_and(2, kSgCompute, ok && !abort_flag);
    if (!ok) break;
    cplx<R>* x = v;
    v = tv;
    tv = x;
    if (expect && (f + 1) % kd == 0) observe((f + 1) / kd);
  }
  if (!ok) {
    if (tid == 0) {
      abort_flag = 1;
      if (status) atomicAdd((unsigned long long*)&status[REDO_STATUS_TIMEOUT], 1ull);
    }
    return;
  }
  if (!pT) return;                                  // simulation: no target state
  // a = <psi_T | v>
  double ar = 0.0, ai = 0.0;
  for (int i = tid; i < N; i += kSgCompute) {
    const double2 t = pT[i];
    const double xr = (double)v[i].x, xi = (double)v[i].y;
    ar += t.x * xr + t.y * xi;
    ai += t.x * xi - t.y * xr;
  }
  ar = block_sum(ar);
  ai = block_sum(ai);
  if (tid == 0 && F_out) F_out[b] = ar * ar + ai * ai;
  if (!grad) return;
  for (int i = tid; i < N; i += kSgCompute) w[i] = cmake<R>((R)pT[i].x, (R)pT[i].y);
  tc::named_barrier(1, kSgCompute);
  const int G = N >= kSgCompute ? 1 : kSgCompute / N;     // row groups of a chunk
  const int col = tid % N, grp = tid / N;
  // reverse: trace at a term's last digit, then v <- A_f^dag v, w <- A_f^dag w
  for (int64_t f = F - 1; f >= 0; --f) {
    const int64_t n = f / kd;
    const int rr0 = (int)(f - n * kd);
    const int k = rr0 / d, j = rr0 - k * d;
    if (j == d - 1) {
      const int e0 = hk_ptr[k * (N + 1)], e1 = hk_ptr[k * (N + 1) + N];
      double tr = 0.0, ti = 0.0;
      for (int e = e0 + tid; e < e1; e += kSgCompute) {
        const int i = hk_row[e], c = hk_col[e];
        const double2 h = hk_val[e];
        const double wr = (double)w[i].x, wi = (double)w[i].y, vr = (double)v[c].x, vi = (double)v[c].y;
        const double hr = h.x * vr - h.y * vi, hi = h.x * vi + h.y * vr;
        tr += wr * hr + wi * hi;
        ti += wr * hi - wi * hr;
      }
      tr = block_sum(tr);
      ti = block_sum(ti);
      if (tid == 0) grad[(b * M + n) * K + k] = 2.0 * dt * (ar * ti - ai * tr);
    }
    cplx<R> sv0 = cmake<R>(R(0), R(0)), sw0 = sv0, sv1 = sv0, sw1 = sv0;
    for (int ch = 0; ch < cpf; ++ch) {
      const cplx<R>* A = chunk();
      if (ok) {
        const int r0 = ch * rows;
        for (int rr = grp; rr < rows; rr += G) {
          const cplx<R> vr = v[r0 + rr], wr = w[r0 + rr];
          const cplx<R> a = A[(int64_t)rr * N + col];
          const cplx<R> ac = cmake<R>(a.x, -a.y);
          cfma<R>(sv0, ac, vr);
          cfma<R>(sw0, ac, wr);
          if (N > kSgCompute) {
            const cplx<R> a1 = A[(int64_t)rr * N + col + kSgCompute];
            const cplx<R> ac1 = cmake<R>(a1.x, -a1.y);
            cfma<R>(sv1, ac1, vr);
            cfma<R>(sw1, ac1, wr);
          }
        }
      }
      release();
    }
    if (G > 1) {
      scratch[tid] = sv0;
      scratch[kSgCompute + tid] = sw0;
      tc::named_barrier(1, kSgCompute);
      if (tid < N) {
        cplx<R> a = cmake<R>(R(0), R(0)), c2 = a;
        for (int g = 0; g < G; ++g) {
          a.x += scratch[g * N + tid].x;
          a.y += scratch[g * N + tid].y;
          c2.x += scratch[kSgCompute + g * N + tid].x;
          c2.y += scratch[kSgCompute + g * N + tid].y;
        }
        tv[tid] = a;
        tw[tid] = c2;
      }
    } else {
      tv[col] = sv0;
      tw[col] = sw0;
      if (N > kSgCompute) {
        tv[col + kSgCompute] = sv1;
        tw[col + kSgCompute] = sw1;
      }
    }
    ok = tc::named_barrier_and(2, kSgCompute, ok && !abort_flag);
    if (!ok) break;
    cplx<R>* x = v;
    v = tv;
    tv = x;
    x = w;
    w = tw;
    tw = x;
  }
  if (!ok && tid == 0) {
    abort_flag = 1;
    if (status) atomicAdd((unsigned long long*)&status[REDO_STATUS_TIMEOUT], 1ull);
  }
}

}  // namespace

template <typename R>
static cudaError_t launch_state_stream(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                                       const double2* psi0, const double2* psiT, int batched, double* F_out,
                                       double* grad, int64_t* status, cudaStream_t s, const double* obs = nullptr,
                                       double* expect = nullptr) {
  const int N = t->N;
  const size_t el = sizeof(cplx<R>);
  int rows = (int)(kSgChunk / (N * el));
  if (rows > N) rows = N;
  const size_t fixed = (4 * (size_t)N + 2 * kSgCompute) * el;
  int stages = (int)((227 * 1024 - fixed - 1024) / kSgChunk);
  if (stages > 3) stages = 3;
  if (stages < 2) return cudaErrorInvalidValue;
  const size_t smem = (size_t)stages * kSgChunk + fixed + 2 * (size_t)stages * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(state_grad_stream_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  state_grad_stream_kernel<R><<<(unsigned)B, kSgThreads, smem, s>>>(
      std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32, q, N, M, t->K, t->digits,
      t->base, t->levels, psi0, psiT, batched, t->hk_ptr, t->hk_col, t->hk_row, t->hk_val, t->dt, F_out, grad,
      status, stages, rows, obs, expect);
  return cudaGetLastError();
}

cudaError_t launch_sim_stream(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                              const double2* psi0, int psi0_batched, const double* obs, double* expect,
                              int64_t* status, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  return prec == REDO_FP64
             ? launch_state_stream<double>(t, q, B, M, psi0, nullptr, psi0_batched, nullptr, nullptr, status, s, obs,
                                           expect)
             : launch_state_stream<float>(t, q, B, M, psi0, nullptr, psi0_batched, nullptr, nullptr, status, s, obs,
                                          expect);
}

cudaError_t launch_state_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                              const double2* psi0, const double2* psiT, int batched, double* F_out, double* grad,
                              int64_t* status, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const int N = t->N;
  if (N >= 64)
    return prec == REDO_FP64 ? launch_state_stream<double>(t, q, B, M, psi0, psiT, batched, F_out, grad, status, s)
                             : launch_state_stream<float>(t, q, B, M, psi0, psiT, batched, F_out, grad, status, s);
  cudaError_t e;
  if (prec == REDO_FP64) {
    const size_t smem = 4 * sizeof(double2) * N;
    if ((e = cudaFuncSetAttribute(state_grad_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    state_grad_kernel<double><<<(unsigned)B, kStTh, smem, s>>>(
        t->T64, q, N, M, t->K, t->digits, t->base, t->levels, psi0, psiT, batched, t->hk_ptr, t->hk_col,
        t->hk_row, t->hk_val, t->dt, F_out, grad, status);
  } else {
    const size_t smem = 4 * sizeof(float2) * N;
    if ((e = cudaFuncSetAttribute(state_grad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    state_grad_kernel<float><<<(unsigned)B, kStTh, smem, s>>>(
        t->T32, q, N, M, t->K, t->digits, t->base, t->levels, psi0, psiT, batched, t->hk_ptr, t->hk_col,
        t->hk_row, t->hk_val, t->dt, F_out, grad, status);
  }
  return cudaGetLastError();
}

}  // namespace redo
