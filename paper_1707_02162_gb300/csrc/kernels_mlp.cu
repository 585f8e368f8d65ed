// Multilayer perceptron for the learned warm start of GRAPE: forward,
// backward (mean-squared error) and Adam, FP32 master weights, FP32 SIMT.
//
// Network: h_0 = x; z_l = h_l W_l^T + b_l; h_{l+1} = GELU(z_l) for hidden
// layers (exact erf form) and tanh(z_l) for the output layer, whose entries are
// normalised pulse amplitudes in [-1, 1].  Parameters are one flat array with
// W_l (out x in, row-major) followed by b_l (out) for every layer.
#include "redo_internal.cuh"

namespace redo {

// C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]); optional act(C) into Cact.
// A(i,k) = A[i*sa0 + k*sa1], B(k,j) = B[k*sb0 + j*sb1], C row-major with ldc.
struct GemmArgs {
  const float* A;
  int64_t sa0, sa1;
  const float* B;
  int64_t sb0, sb1;
  float* C;
  int64_t ldc;
  int M, N, K;
  const float* bias;
  int act;          // 0 none, 1 GELU, 2 tanh
  float* Cact;
};

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float Phi = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float phi = 0.39894228040143268f * expf(-0.5f * x * x);
  return Phi + x * phi;
}

constexpr int kGT = 64, kGK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
  __shared__ float As[kGK][kGT + 1];
  __shared__ float Bs[kGK][kGT + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += kGK) {
    for (int e = tid; e < kGT * kGK; e += 256) {
      const int ii = e / kGK, kk = e % kGK;
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < g.M && k < g.K) ? g.A[i * g.sa0 + k * g.sa1] : 0.f;
      const int jj = e % kGT, kb = e / kGT;
      const int j = j0 + jj, k2 = k0 + kb;
      Bs[kb][jj] = (j < g.N && k2 < g.K) ? g.B[k2 * g.sb0 + j * g.sb1] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < g.M && j < g.N) {
        float v = acc[r][c] + (g.bias ? g.bias[j] : 0.f);
        g.C[(int64_t)i * g.ldc + j] = v;
        if (g.Cact) g.Cact[(int64_t)i * g.ldc + j] = g.act == 1 ? gelu_f(v) : (g.act == 2 ? tanhf(v) : v);
      }
    }
}

static cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M == 0 || g.N == 0) return cudaSuccess;
  dim3 grid((g.N + kGT - 1) / kGT, (g.M + kGT - 1) / kGT);
  gemm_kernel<<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// dz = dy * (1 - y^2) with dy = 2 (y - t) / count ; loss partial sums into loss (double)
__global__ void mse_tanh_grad_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                     float* __restrict__ dz, int64_t count, double* loss) {
  double part = 0.0;
  const float inv = 2.0f / (float)count;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float e = y[i] - t[i];
    part += (double)e * (double)e;
    dz[i] = inv * e * (1.0f - y[i] * y[i]);
  }
  if (loss) {
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part / (double)count);
  }
}

__global__ void gelu_back_kernel(float* __restrict__ dz, const float* __restrict__ z, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dz[i] *= gelu_grad_f(z[i]);
}

// db[j] = sum_b dz[b][j]
__global__ void colsum_kernel(const float* __restrict__ dz, int64_t rows, int cols, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int64_t b = 0; b < rows; ++b) s += dz[b * cols + j];
  db[j] = s;
}

__global__ void adam_kernel(int64_t count, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

static unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (unsigned)(b < 1 ? 1 : b);
}

int64_t mlp_param_count(int L, const int32_t* sizes) {
  int64_t n = 0;
  for (int l = 0; l < L; ++l) n += (int64_t)sizes[l + 1] * sizes[l] + sizes[l + 1];
  return n;
}

cudaError_t mlp_forward(int L, const int32_t* sizes, const float* params, const float* x,
                        int64_t batch, float* acts, float* y, cudaStream_t s) {
  const float* h = x;
  const float* p = params;
  float* a = acts;
  for (int l = 0; l < L; ++l) {
    const int in = sizes[l], out = sizes[l + 1];
    GemmArgs g{};
    g.A = h; g.sa0 = in; g.sa1 = 1;
    g.B = p; g.sb0 = 1; g.sb1 = in;              // B(k,j) = W[j][k]
    g.C = a; g.ldc = out;
    g.M = (int)batch; g.N = out; g.K = in;
    g.bias = p + (int64_t)out * in;
    g.act = l == L - 1 ? 2 : 1;
    g.Cact = a + batch * out;
    cudaError_t e = gemm(g, s);
    if (e != cudaSuccess) return e;
    h = a + batch * out;
    p += (int64_t)out * in + out;
    a += 2 * batch * out;
  }
  const int out = sizes[L];
  return cudaMemcpyAsync(y, h, sizeof(float) * batch * out, cudaMemcpyDeviceToDevice, s);
}

cudaError_t mlp_backward(int L, const int32_t* sizes, const float* params, const float* x,
                         int64_t batch, const float* acts, const float* y_target, float* grads,
                         double* loss, float* work, cudaStream_t s) {
  int maxw = 0;
  for (int l = 0; l <= L; ++l) maxw = sizes[l] > maxw ? sizes[l] : maxw;
  float* dz = work;
  float* dh = work + batch * maxw;
  // offsets of every layer's parameters and activations
  int64_t poff[64], aoff[64];
  int64_t po = 0, ao = 0;
  for (int l = 0; l < L; ++l) {
    poff[l] = po;
    aoff[l] = ao;
    po += (int64_t)sizes[l + 1] * sizes[l] + sizes[l + 1];
    ao += 2 * batch * sizes[l + 1];
  }
  const int outL = sizes[L];
  const float* yL = acts + aoff[L - 1] + batch * outL;
  if (loss) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
  }
  mse_tanh_grad_kernel<<<blocks_for(batch * outL), 256, 0, s>>>(yL, y_target, dz, batch * outL, loss);
  for (int l = L - 1; l >= 0; --l) {
    const int in = sizes[l], out = sizes[l + 1];
    const float* h = l == 0 ? x : acts + aoff[l - 1] + batch * in;
    const float* W = params + poff[l];
    float* dW = grads + poff[l];
    float* db = dW + (int64_t)out * in;
    GemmArgs g{};
    g.A = dz; g.sa0 = 1; g.sa1 = out;            // A(i,k) = dz[k][i]
    g.B = h; g.sb0 = in; g.sb1 = 1;              // B(k,j) = h[k][j]
    g.C = dW; g.ldc = in;
    g.M = out; g.N = in; g.K = (int)batch;
    cudaError_t e = gemm(g, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(out + 255) / 256, 256, 0, s>>>(dz, batch, out, db);
    if (l > 0) {
      GemmArgs h2{};
      h2.A = dz; h2.sa0 = out; h2.sa1 = 1;
      h2.B = W; h2.sb0 = in; h2.sb1 = 1;          // B(k,j) = W[k][j]
      h2.C = dh; h2.ldc = in;
      h2.M = (int)batch; h2.N = in; h2.K = out;
      e = gemm(h2, s);
      if (e != cudaSuccess) return e;
      const float* zprev = acts + aoff[l - 1];
      gelu_back_kernel<<<blocks_for(batch * in), 256, 0, s>>>(dh, zprev, batch * in);
      float* tmp = dz;
      dz = dh;
      dh = tmp;
    }
  }
  return cudaGetLastError();
}

cudaError_t mlp_adam(int64_t count, float* p, const float* g, float* m, float* v, int step, float lr,
                     float b1, float b2, float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<blocks_for(count), 256, 0, s>>>(count, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace redo
