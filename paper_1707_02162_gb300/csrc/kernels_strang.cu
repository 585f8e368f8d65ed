// Symmetric (Strang) split of a step: S_n = D_h E_{K-1} ... E_0 D_h, D_h = exp(-i dt/2 H0).
// (The Section III step with the drift split evenly around the control factors: a second-order
// variant of the paper's step.)
//
// With the drift folded into every step (U_n = E_{K-1} ... E_0 D), the symmetric chain is
// a conjugation of the folded one:
//     S_M ... S_1 = D_h (U_M ... U_1) D_h^dag,
// so propagators, fidelities (target U_T -> D_h^dag U_T D_h) and states
// (psi_0 -> D_h^dag psi_0 when the observable and D_h are both diagonal) follow from the
// folded chain.  These kernels apply the conjugation: elementwise when H0, hence D_h, is
// diagonal; otherwise by two FP64 matrix products per matrix.
#include "redo_internal.cuh"

namespace redo {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

template <typename R>
__device__ __forceinline__ double2 load_d(const cplx<R>* p, int64_t i) {
  const cplx<R> v = p[i];
  return make_double2((double)v.x, (double)v.y);
}

// Diagonal D_h = diag(d): out[i][j] = d_i X[i][j] conj(d_j), or its adjoint form
// conj(d_i) X[i][j] d_j.  One thread per entry.
template <typename R>
__global__ void conj_diag_kernel(const double2* __restrict__ Dh, const cplx<R>* X, int N, int64_t count,
                                 int adjoint, double2* out) {   // out may be X itself
  const int64_t n2 = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count * n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx % n2);
    const int i = e / N, j = e % N;
    double2 di = Dh[(int64_t)i * N + i], dj = Dh[(int64_t)j * N + j];
    if (adjoint) di = cconj(di);
    else dj = cconj(dj);
    out[idx] = cmul(cmul(di, load_d<R>(X, idx)), dj);
  }
}

// Dense D_h, first pass: tmp = X A^dag (adjoint = 0, A = D_h) or X A (adjoint = 1, A^dag = D_h^dag
// on the left later).  tmp[i][j] = sum_k X[i][k] B[k][j], B = D_h^dag or D_h.
template <typename R>
__global__ void conj_dense_right_kernel(const double2* __restrict__ Dh, const cplx<R>* __restrict__ X, int N,
                                        int64_t count, int adjoint, double2* __restrict__ tmp) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count * n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / n2;
    const int e = (int)(idx % n2);
    const int i = e / N, j = e % N;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < N; ++k) {
      const double2 x = load_d<R>(X, b * n2 + (int64_t)i * N + k);
      // B[k][j] = conj(D_h[j][k]) (D_h^dag) or D_h[k][j]
      const double2 m = adjoint ? Dh[(int64_t)k * N + j] : cconj(Dh[(int64_t)j * N + k]);
      re += x.x * m.x - x.y * m.y;
      im += x.x * m.y + x.y * m.x;
    }
    tmp[idx] = make_double2(re, im);
  }
}

// Dense D_h, second pass: out[i][j] = sum_k L[i][k] tmp[k][j], L = D_h or D_h^dag.
__global__ void conj_dense_left_kernel(const double2* __restrict__ Dh, const double2* __restrict__ tmp, int N,
                                       int64_t count, int adjoint, double2* out) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count * n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / n2;
    const int e = (int)(idx % n2);
    const int i = e / N, j = e % N;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < N; ++k) {
      const double2 l = adjoint ? cconj(Dh[(int64_t)k * N + i]) : Dh[(int64_t)i * N + k];
      const double2 x = tmp[b * n2 + (int64_t)k * N + j];
      re += l.x * x.x - l.y * x.y;
      im += l.x * x.y + l.y * x.x;
    }
    out[idx] = make_double2(re, im);
  }
}

// psi'_b[i] = conj(d_i) psi_b[i] (diagonal D_h)
__global__ void vec_diag_adj_kernel(const double2* __restrict__ Dh, const double2* __restrict__ psi, int N,
                                    int64_t count, double2* __restrict__ out) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count * N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N);
    out[idx] = cmul(cconj(Dh[(int64_t)i * N + i]), psi[idx]);
  }
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_half_drift_conj(const redo_table* t, int prec, const void* X, int64_t count, int adjoint,
                                   double2* out, double2* tmp, cudaStream_t s) {
  if (!t->Dh64) return cudaErrorInvalidValue;
  const int N = t->N;
  const int64_t n = count * (int64_t)N * N;
  if (n == 0) return cudaSuccess;
  const bool f64 = prec == REDO_FP64;
  if (t->h0_diagonal) {
    if (f64)
      conj_diag_kernel<double><<<grid_for(n), 256, 0, s>>>(t->Dh64, (const double2*)X, N, count, adjoint, out);
    else
      conj_diag_kernel<float><<<grid_for(n), 256, 0, s>>>(t->Dh64, (const float2*)X, N, count, adjoint, out);
    return cudaGetLastError();
  }
  if (!tmp) return cudaErrorInvalidValue;
  if (f64)
    conj_dense_right_kernel<double><<<grid_for(n), 256, 0, s>>>(t->Dh64, (const double2*)X, N, count, adjoint, tmp);
  else
    conj_dense_right_kernel<float><<<grid_for(n), 256, 0, s>>>(t->Dh64, (const float2*)X, N, count, adjoint, tmp);
  conj_dense_left_kernel<<<grid_for(n), 256, 0, s>>>(t->Dh64, tmp, N, count, adjoint, out);
  return cudaGetLastError();
}

cudaError_t launch_half_drift_vec(const redo_table* t, const double2* psi, int64_t count, double2* out,
                                  cudaStream_t s) {
  if (!t->Dh64 || !t->h0_diagonal) return cudaErrorInvalidValue;
  const int64_t n = count * (int64_t)t->N;
  if (n == 0) return cudaSuccess;
  vec_diag_adj_kernel<<<grid_for(n), 256, 0, s>>>(t->Dh64, psi, t->N, count, out);
  return cudaGetLastError();
}

}  // namespace redo
