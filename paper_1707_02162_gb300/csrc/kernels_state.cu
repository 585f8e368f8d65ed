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

}  // namespace

cudaError_t launch_state_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                              const double2* psi0, const double2* psiT, int batched, double* F_out, double* grad,
                              int64_t* status, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const int N = t->N;
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
