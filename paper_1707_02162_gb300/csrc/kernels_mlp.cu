// Multilayer perceptron for the learned warm start of GRAPE: forward,
// backward (mean-squared error) and Adam, FP32 master weights.
// (No paper counterpart: the learned warm start extends the GRAPE application of Section III.)
//
// Network: h_0 = x; z_l = h_l W_l^T + b_l; h_{l+1} = GELU(z_l) for hidden
// layers (exact erf form) and tanh(z_l) for the output layer, whose entries are
// normalised pulse amplitudes in [-1, 1].  Parameters are one flat array with
// W_l (out x in, row-major) followed by b_l (out) for every layer.
//
// The GEMMs run on the tensor cores (tcgen05, kind::f16 with BF16 operands): every FP32
// operand value is split as hi = bf16(v), lo = bf16(v - hi) and a product takes
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory (about 16 significant bits
// per operand, the FP32 exponent range).  Each operand of a GEMM is split once, by one CTA per
// 128-row x 64-K tile, into 128-byte-swizzled K-major hi/lo planes in a scratch buffer (a weight
// or activation tile is otherwise converted again by every CTA that reads it: 40 times for the
// 5000-wide output layer).  A CTA then computes one 128 x 128 tile of C: one thread streams
// the A and B plane tiles of each 64-wide K slice through a three-stage ring of bulk copies,
// one thread issues the MMAs, and eight warps read the accumulator back for the bias and
// activation.
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
constexpr uint32_t kMLimit = 1u << 24;
// kind::f16 instruction descriptor: D f32, A and B bf16, K-major, N = 128, M = 128
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNT >> 3) << 17) |
                                ((uint32_t)(kMT >> 4) << 24);

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Split a 128-row x 64-K tile of a strided operand (element (r, k) at X[r * s_r + k * s_k],
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

// One 128-row x 64-K tile (rt, kt) of a strided FP32 operand per CTA, split into its hi and lo
// planes (16 KB each, the layout stage_tile writes) at planes + (rt * KT + kt) * 32 KB.
__global__ void __launch_bounds__(256) split_planes_kernel(const float* __restrict__ X, int64_t s_r, int64_t s_k,
                                                           int rows, int K, int KT, uint8_t* __restrict__ planes) {
  const int rt = blockIdx.y, kt = blockIdx.x;
  uint8_t* hi = planes + ((size_t)rt * KT + kt) * (2 * kMPlane);
  stage_tile(X, s_r, s_k, rows, K, rt * kMT, kt * kKT, hi, hi + kMPlane, threadIdx.x);
}

constexpr int kPStages = 3;
constexpr uint32_t kPStage = 4 * kMPlane;                        // A hi, A lo, B hi, B lo (64 KB)
constexpr uint32_t kPSmem = kPStages * kPStage + 1024 + 128;

// C tile from pre-split planes: A planes [ceil(M/128)][KT], B planes [ceil(N/128)][KT].  With
// split > 1 CTA z takes K slices [z KT / split, (z + 1) KT / split) and writes its partial tile,
// without bias or activation, to part + z M N (row-major, ldc = N).
__global__ void __launch_bounds__(256, 1) gemm_planes_kernel(GemmArgs g, const uint8_t* __restrict__ pa,
                                                             const uint8_t* __restrict__ pb, int KT, int split,
                                                             float* __restrict__ part, int64_t* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPStages * kPStage);
  uint64_t* empty = full + kPStages;
  uint64_t* done = empty + kPStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.y * kMT, j0 = blockIdx.x * kNT;
  if (tid == 0) {
    for (int st = 0; st < kPStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, kNT);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;
  const int z = blockIdx.z;
  const int k0 = (int)((int64_t)z * KT / split), k1 = (int)((int64_t)(z + 1) * KT / split);
  const int NK = k1 - k0;                                // K slices of this CTA
  const uint8_t* a_tiles = pa + ((size_t)blockIdx.y * KT + k0) * (2 * kMPlane);
  const uint8_t* b_tiles = pb + ((size_t)blockIdx.x * KT + k0) * (2 * kMPlane);
  if (tid == 0) {
    // producer: the A and B plane tiles of every K slice, kPStages slices ahead
    for (int kt = 0; kt < NK && !*abort_flag; ++kt) {
      const int st = kt % kPStages;
      if (kt >= kPStages && !mbar_wait_bounded_n(&empty[st], (uint32_t)(((kt / kPStages) - 1) & 1), kMLimit)) {
        *abort_flag = 1;
        break;
      }
      uint8_t* base = smem + st * kPStage;
      mbar_arrive_expect_tx(&full[st], kPStage);
      bulk_load(base, a_tiles + (size_t)kt * (2 * kMPlane), 2 * kMPlane, &full[st]);
      bulk_load(base + 2 * kMPlane, b_tiles + (size_t)kt * (2 * kMPlane), 2 * kMPlane, &full[st]);
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int kt = 0; kt < NK; ++kt) {
      const int st = kt % kPStages;
      if (*abort_flag || !mbar_wait_bounded_n(&full[st], (uint32_t)((kt / kPStages) & 1), kMLimit)) {
        *abort_flag = 1;
        break;
      }
      tc::tc_fence_after();
      const uint32_t a_hi = smem_u32(smem + st * kPStage), a_lo = a_hi + kMPlane;
      const uint32_t b_hi = a_hi + 2 * kMPlane, b_lo = a_hi + 3 * kMPlane;
#pragma unroll
      for (int kk = 0; kk < kKT / 16; ++kk) {
        const uint32_t o = (uint32_t)kk * 32u;
        tc::mma_f16(tmem, tc::smem_desc_sw128(a_hi + o), tc::smem_desc_sw128(b_hi + o), kIdescBf16,
                    (kt | kk) ? 1u : 0u);
        tc::mma_f16(tmem, tc::smem_desc_sw128(a_hi + o), tc::smem_desc_sw128(b_lo + o), kIdescBf16, 1u);
        tc::mma_f16(tmem, tc::smem_desc_sw128(a_lo + o), tc::smem_desc_sw128(b_hi + o), kIdescBf16, 1u);
      }
      tc::mma_commit(&empty[st]);
      if (kt == NK - 1) tc::mma_commit(done);
    }
  }
  __syncthreads();                     // the other threads wait here, not spinning, while the two work
  bool ok = true;
  if (NK > 0) ok = mbar_wait_bounded_n(done, 0u, kMLimit);
  ok = __syncthreads_and(ok && !*abort_flag);
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
      if (NK > 0) {
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
            if (split > 1) {
              part[((int64_t)z * g.M + i) * g.N + j] = __uint_as_float(r[c]);
              continue;
            }
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

// C = sum_z part[z] (+ bias) in a fixed order, optional activation into Cact.
__global__ void splitk_reduce_kernel(GemmArgs g, const float* __restrict__ part, int split) {
  const int64_t n = (int64_t)g.M * g.N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / g.N;
    const int j = (int)(idx - i * g.N);
    float v = 0.f;
    for (int z = 0; z < split; ++z) v += part[(int64_t)z * n + idx];
    if (g.bias) v += g.bias[j];
    g.C[i * g.ldc + j] = v;
    if (g.Cact) g.Cact[i * g.ldc + j] = g.act == 1 ? gelu_f(v) : (g.act == 2 ? tanhf(v) : v);
  }
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// K splits of one GEMM: when its C tiles fill less than half the GPU and its K loop is long,
// enough splits (of at least 8 K slices each) to give about one CTA per SM.
static int gemm_splits(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = ceil_div(M, kMT) * ceil_div(N, kNT), KT = ceil_div(K, kKT);
  if (tiles == 0 || tiles >= 76 || KT < 16) return 1;       // an empty GEMM takes no split
  int64_t sp = ceil_div(152, tiles);
  if (sp > KT / 8) sp = KT / 8;
  return sp < 1 ? 1 : (int)sp;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch bytes of one GEMM: split planes (A: M x K, B: N x K in tiles of 128 x 64) and, with K
// split, the partial C tiles.
size_t gemm_plane_bytes(int64_t M, int64_t N, int64_t K) {
  const int sp = gemm_splits(M, N, K);
  return up256((size_t)(ceil_div(M, kMT) + ceil_div(N, kNT)) * ceil_div(K, kKT) * (2 * kMPlane)) +
         (sp > 1 ? up256((size_t)sp * M * N * sizeof(float)) : 0);
}

// planes: scratch of gemm_plane_bytes(M, N, K) bytes, 256-byte aligned.
static cudaError_t gemm(const GemmArgs& g, cudaStream_t s, uint8_t* planes) {
  if (g.M == 0 || g.N == 0) return cudaSuccess;
  const int KT = (int)ceil_div(g.K, kKT);
  const int sp = gemm_splits(g.M, g.N, g.K);
  dim3 grid((g.N + kNT - 1) / kNT, (g.M + kMT - 1) / kMT, sp);
  uint8_t* pa = planes;
  uint8_t* pb = planes + (size_t)ceil_div(g.M, kMT) * KT * (2 * kMPlane);
  float* part = (float*)(planes + up256((size_t)(ceil_div(g.M, kMT) + ceil_div(g.N, kNT)) * KT * (2 * kMPlane)));
  if (KT > 0) {
    split_planes_kernel<<<dim3(KT, (unsigned)ceil_div(g.M, kMT)), 256, 0, s>>>(g.A, g.sa0, g.sa1, g.M, g.K, KT, pa);
    split_planes_kernel<<<dim3(KT, (unsigned)ceil_div(g.N, kNT)), 256, 0, s>>>(g.B, g.sb1, g.sb0, g.N, g.K, KT, pb);
  }
  cudaError_t e = cudaFuncSetAttribute(gemm_planes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPSmem);
  if (e != cudaSuccess) return e;
  gemm_planes_kernel<<<grid, 256, kPSmem, s>>>(g, pa, pb, KT, sp, part, nullptr);
  if (sp > 1) {
    int64_t blocks = ceil_div((int64_t)g.M * g.N, 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    splitk_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, part, sp);
  }
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
    __shared__ double red[8];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(loss, t / (double)count);
    }
  }
}

__global__ void gelu_back_kernel(float* __restrict__ dz, const float* __restrict__ z, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dz[i] *= gelu_grad_f(z[i]);
}

// db[j] = sum_b dz[b][j] in two passes of fixed order.  Pass 1: CTA (column block of 32, row
// chunk y) has its 8 warps read interleaved rows of the chunk (one coalesced 128-byte piece each)
// and writes the chunk's sums to part[y][j]; pass 2 adds the chunks' sums.
constexpr int kColChunks = 32;

__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ dz, int64_t rows, int cols,
                                                     float* __restrict__ part) {
  __shared__ float red[8][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int j = blockIdx.x * 32 + l;
  const int64_t r0 = blockIdx.y * rows / kColChunks, r1 = (blockIdx.y + 1) * rows / kColChunks;
  float s = 0.f;
  if (j < cols)
    for (int64_t b = r0 + w; b < r1; b += 8) s += dz[b * cols + j];
  red[w][l] = s;
  __syncthreads();
  if (w == 0 && j < cols) {
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += red[i][l];
    part[(int64_t)blockIdx.y * cols + j] = t;
  }
}

__global__ void colsum_finish_kernel(const float* __restrict__ part, int cols, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float t = 0.f;
  for (int y = 0; y < kColChunks; ++y) t += part[(int64_t)y * cols + j];
  db[j] = t;
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

// Scratch (bytes) for the split operand planes of the forward GEMMs and of the backward GEMMs.
size_t mlp_forward_plane_bytes(int L, const int32_t* sizes, int64_t batch) {
  size_t m = 0;
  for (int l = 0; l < L; ++l) {
    const size_t b = gemm_plane_bytes(batch, sizes[l + 1], sizes[l]);
    m = b > m ? b : m;
  }
  return m;
}

size_t mlp_backward_plane_bytes(int L, const int32_t* sizes, int64_t batch) {
  size_t m = 0;
  for (int l = 0; l < L; ++l) {
    const size_t b1 = gemm_plane_bytes(sizes[l + 1], sizes[l], batch);   // dW = dz^T h
    const size_t b2 = gemm_plane_bytes(batch, sizes[l], sizes[l + 1]);   // dh = dz W
    m = b1 > m ? b1 : m;
    m = b2 > m ? b2 : m;
  }
  return m;
}

static int64_t activation_floats(int L, const int32_t* sizes, int64_t batch) {
  int64_t a = 0;
  for (int l = 1; l <= L; ++l) a += 2 * batch * sizes[l];
  return a;
}

static uint8_t* planes_after(float* base, int64_t floats) {
  uintptr_t p = (uintptr_t)(base + floats);
  return (uint8_t*)((p + 255) & ~(uintptr_t)255);
}

cudaError_t mlp_forward(int L, const int32_t* sizes, const float* params, const float* x,
                        int64_t batch, float* acts, float* y, cudaStream_t s) {
  const float* h = x;
  const float* p = params;
  float* a = acts;
  uint8_t* planes = planes_after(acts, activation_floats(L, sizes, batch));
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
    cudaError_t e = gemm(g, s, planes);
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
  float* colpart = work + 2 * batch * maxw;              // kColChunks x maxw partial column sums
  uint8_t* planes = planes_after(work, 2 * batch * maxw + (int64_t)kColChunks * maxw);
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
    cudaError_t e = gemm(g, s, planes);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<dim3((out + 31) / 32, kColChunks), 256, 0, s>>>(dz, batch, out, colpart);
    colsum_finish_kernel<<<(out + 255) / 256, 256, 0, s>>>(colpart, out, db);
    if (l > 0) {
      GemmArgs h2{};
      h2.A = dz; h2.sa0 = out; h2.sa1 = 1;
      h2.B = W; h2.sb0 = in; h2.sb1 = 1;          // B(k,j) = W[k][j]
      h2.C = dh; h2.ldc = in;
      h2.M = (int)batch; h2.N = in; h2.K = out;
      e = gemm(h2, s, planes);
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
