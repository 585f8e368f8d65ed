// Batched FP64 complex products with optional conjugate transposes, for the time-split layer:
// a pulse cut into G time segments (one per rank) has propagator U = S_{G-1} ... S_0, and the
// gradient of segment r needs the transformed target  L_r^dag U_T P_r^dag  with the prefix
// P_r = S_{r-1} ... S_0 and the suffix L_r = S_{G-1} ... S_{r+1} (Section III: the gradient of
// |Tr(U_T^dag L S P)|^2 in the controls of S equals that of |Tr((L^dag U_T P^dag)^dag S)|^2).
// These products are few (a handful per rank and pulse), so one plain tiled kernel serves.
#include "redo_internal.cuh"

namespace redo {

namespace {

constexpr int kPT = 16;

// C_b = op_A(A_b) op_B(B_b): 16 x 16 output tiles, FP64 accumulation, any N.
__global__ void __launch_bounds__(kPT * kPT)
batched_product_kernel(int N, const double2* __restrict__ A, int adjA, int64_t sA, const double2* __restrict__ B,
                       int adjB, int64_t sB, double2* __restrict__ C, int64_t b0) {
  __shared__ double2 As[kPT][kPT + 1];
  __shared__ double2 Bs[kPT][kPT + 1];
  const int64_t b = b0 + blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * kPT + ty, j = blockIdx.x * kPT + tx;
  const double2* Ab = A + b * sA;
  const double2* Bb = B + b * sB;
  double re = 0.0, im = 0.0;
  for (int k0 = 0; k0 < N; k0 += kPT) {
    const int ka = k0 + tx, kb = k0 + ty;
    double2 av = make_double2(0.0, 0.0), bv = make_double2(0.0, 0.0);
    if (i < N && ka < N) {
      if (adjA) {
        const double2 v = Ab[(int64_t)ka * N + i];
        av = make_double2(v.x, -v.y);
      } else {
        av = Ab[(int64_t)i * N + ka];
      }
    }
    if (kb < N && j < N) {
      if (adjB) {
        const double2 v = Bb[(int64_t)j * N + kb];
        bv = make_double2(v.x, -v.y);
      } else {
        bv = Bb[(int64_t)kb * N + j];
      }
    }
    As[ty][tx] = av;
    Bs[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kPT; ++kk) {
      const double2 x = As[ty][kk], y = Bs[kk][tx];
      re = fma(x.x, y.x, fma(-x.y, y.y, re));
      im = fma(x.x, y.y, fma(x.y, y.x, im));
    }
    __syncthreads();
  }
  if (i < N && j < N) C[b * (int64_t)N * N + (int64_t)i * N + j] = make_double2(re, im);
}

}  // namespace

cudaError_t launch_batched_product(int N, int64_t count, const double2* A, int adjA, int64_t sA, const double2* B,
                                   int adjB, int64_t sB, double2* C, cudaStream_t s) {
  const unsigned tiles = (unsigned)((N + kPT - 1) / kPT);
  for (int64_t b0 = 0; b0 < count; b0 += 65535) {
    const int64_t n = count - b0 < 65535 ? count - b0 : 65535;
    batched_product_kernel<<<dim3(tiles, tiles, (unsigned)n), dim3(kPT, kPT), 0, s>>>(N, A, adjA, sA, B, adjB, sB,
                                                                                     C, b0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace redo
