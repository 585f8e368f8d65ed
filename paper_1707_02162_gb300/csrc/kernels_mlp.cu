// Multilayer perceptron for the learned warm start of GRAPE: forward,
// backward (mean-squared error) and Adam, FP32 master weights.
//
// Network: h_0 = x; z_l = h_l W_l^T + b_l; h_{l+1} = GELU(z_l) for hidden
// layers (exact erf form) and tanh(z_l) for the output layer, whose entries are
// normalised pulse amplitudes in [-1, 1].  Parameters are one flat array with
// W_l (out x in, row-major) followed by b_l (out) for every layer.
//
// The GEMMs run on the tensor cores (tcgen05, kind::f16 with BF16 operands): every FP32
// operand value is split as hi = bf16(v), lo = bf16(v - hi) and a product takes
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory (about 16 significant bits
// per operand, the FP32 exponent range).  A CTA computes one 128 x 128 tile of C: its threads
// stage 64-wide K slices of A and B (any strides, converted and split on the way) into
// 128-byte-swizzled K-major tiles, one thread issues the MMAs of a slice while the next slice
// is staged, and eight warps read the accumulator back for the bias and activation.
#include <cuda_bf16.h>

#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "tcgen05.cuh"

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

constexpr int kMT = 128, kNT = 128, kKT = 64;                 // C tile, K slice (bf16)
constexpr uint32_t kMPlane = kMT * kKT * 2;                      // 16 KB: 128 rows x 64 bf16
constexpr uint32_t kMStage = 4 * kMPlane;                        // A hi, A lo, B hi, B lo
constexpr uint32_t kMSmem = 2 * kMStage + 1024 + 64;
constexpr uint32_t kMLimit = 1u << 24;
// kind::f16 instruction descriptor: D f32, A and B bf16, K-major, N = 128, M = 128
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNT >> 3) << 17) |
                                ((uint32_t)(kMT >> 4) << 24);

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Stage a 128-row x 64-K tile of a strided operand (element (r, k) at X[r * s_r + k * s_k],
// zero outside rows x K) into hi / lo planes; groups of 8 consecutive k per thread, threads
// laid along whichever index is contiguous in memory.
__device__ __forceinline__ void stage_tile(const float* __restrict__ X, int64_t s_r, int64_t s_k, int rows, int K,
                                           int r0, int k0, uint8_t* hi, uint8_t* lo, int tid) {
  const bool kfast = s_k == 1;
  for (int idx = tid; idx < kMT * (kKT / 8); idx += 256) {
    const int r = kfast ? idx / (kKT / 8) : idx % kMT;
    const int g = kfast ? idx % (kKT / 8) : idx / kMT;
    const int rr = r0 + r;
    uint32_t h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float v[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = k0 + 8 * g + 2 * p + q;
        v[q] = (rr < rows && k < K) ? X[(int64_t)rr * s_r + (int64_t)k * s_k] : 0.f;
      }
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[0]), h1 = __float2bfloat16_rn(v[1]);
      h[p] = pack_bf16(h0, h1);
      l[p] = pack_bf16(__float2bfloat16_rn(v[0] - __bfloat162float(h0)),
                       __float2bfloat16_rn(v[1] - __bfloat162float(h1)));
    }
    const uint32_t o = tc::sw128((uint32_t)r, (uint32_t)(8 * g), kMT);
    *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void __launch_bounds__(256, 1) gemm_tc_kernel(GemmArgs g, int64_t* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* done = reinterpret_cast<uint64_t*>(smem + 2 * kMStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.y * kMT, j0 = blockIdx.x * kNT;
  if (tid == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, kNT);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nk = (g.K + kKT - 1) / kKT;
  bool ok = true;
  int issued = 0;                                   // slices whose MMAs were committed
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    uint8_t* base = smem + st * kMStage;
    // the MMAs that read this stage two slices ago are done
    if (kt >= 2 && !mbar_wait_bounded_n(&done[st], (uint32_t)(((kt - 2) >> 1) & 1), kMLimit)) ok = false;
    ok = __syncthreads_and(ok && !*abort_flag);
    if (!ok) break;
    stage_tile(g.A, g.sa0, g.sa1, g.M, g.K, i0, kt * kKT, base, base + kMPlane, tid);
    stage_tile(g.B, g.sb1, g.sb0, g.N, g.K, j0, kt * kKT, base + 2 * kMPlane, base + 3 * kMPlane, tid);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t a_hi = smem_u32(base), a_lo = a_hi + kMPlane;
      const uint32_t b_hi = a_hi + 2 * kMPlane, b_lo = a_hi + 3 * kMPlane;
#pragma unroll
      for (int kk = 0; kk < kKT / 16; ++kk) {
        const uint32_t o = (uint32_t)kk * 32u;
        tc::mma_f16(tmem, tc::smem_desc_sw128(a_hi + o), tc::smem_desc_sw128(b_hi + o), kIdescBf16,
                    (kt | kk) ? 1u : 0u);
        tc::mma_f16(tmem, tc::smem_desc_sw128(a_hi + o), tc::smem_desc_sw128(b_lo + o), kIdescBf16, 1u);
        tc::mma_f16(tmem, tc::smem_desc_sw128(a_lo + o), tc::smem_desc_sw128(b_hi + o), kIdescBf16, 1u);
      }
      tc::mma_commit(&done[st]);
    }
    ++issued;
  }
  // the last committed slice's MMAs (and with them every earlier one) are done
  if (issued > 0) {
    const int last = issued - 1;
    if (!mbar_wait_bounded_n(&done[last & 1], (uint32_t)((last >> 1) & 1), kMLimit)) ok = false;
  }
  ok = __syncthreads_and(ok);
  tc::tc_fence_after();
  if (!ok) {
    if (tid == 0 && status) atomicAdd((unsigned long long*)&status[REDO_STATUS_TIMEOUT], 1ull);
  } else {
    // warp w: accumulator rows 32 (w mod 4) + lane, columns 64 (w / 4) .. + 63
    const int q = warp & 3, hcol = warp >> 2;
    const int i = i0 + 32 * q + lane;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      uint32_t r[32];
      const int jb = 64 * hcol + c0;
      if (nk > 0) {
        tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)jb, r);
        tc::tmem_wait_ld();
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) r[c] = 0u;
      }
      if (i < g.M) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int j = j0 + jb + c;
          if (j < g.N) {
            const float v = __uint_as_float(r[c]) + (g.bias ? g.bias[j] : 0.f);
            g.C[(int64_t)i * g.ldc + j] = v;
            if (g.Cact) g.Cact[(int64_t)i * g.ldc + j] = g.act == 1 ? gelu_f(v) : (g.act == 2 ? tanhf(v) : v);
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kNT);
}

static cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M == 0 || g.N == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.N + kNT - 1) / kNT, (g.M + kMT - 1) / kMT);
  gemm_tc_kernel<<<grid, 256, kMSmem, s>>>(g, nullptr);
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
