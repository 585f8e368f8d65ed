// Tensor-core (tcgen05, split-FP16) lockstep chains for 128 <= N <= 1024.
//
// Every chain keeps its state as the real embedding Emb(Y) = [[Yr, -Yi], [Yi, Yr]]
// (2N x 2N) in HBM, in split FP16 (hi, lo = (v - hi) * 2^11), laid out as
// pre-swizzled tiles: tile (rt, kt) holds rows 128 rt.. and K columns 64 kt..
// as a 128-byte-swizzled K-major 128 x 64 block for hi followed by the same
// block for lo (32 KB), so a single bulk copy lands a tile in shared memory
// ready for the MMA descriptors.  Table operators are stored the same way as
// the operand B^T of Z = Y C: tile (nt, kt) holds 128 hi rows then 128 lo rows
// of B^T, row n = [Re C[:, n], Im C[:, n]].  Two operand sets exist: "row"
// planes with C = A^T (forward steps Y <- Y A^T, i.e. X <- A X for Y = X^T)
// and "column" planes with C = A (reverse gradient sweep, V <- V A, R <- R A).
//
// One launch per chain step; CTA (chain, rt, nt) computes the 128 x 128 block
// [D1 | D2] of Z with a K loop over 2N/64 tiles (3-stage bulk-copy ring):
//     D[:, 0:256]  (+)= A_hi [B_hi; B_lo]^T      (one N = 256 MMA)
//     D[:, 128:256] += A_lo B_hi^T               (one N = 128 MMA)
// and its epilogue writes Z = D1 + 2^-11 D2, split again, into the next
// state's direct and mirrored positions of the embedding.
#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "tcgen05.cuh"

#include <type_traits>

namespace redo {
namespace tcl {

using namespace tc;

constexpr uint32_t kTile = 32768;     // hi (16 KB) + lo (16 KB)
constexpr uint32_t kHalf = 16384;
constexpr uint32_t kLimit = 1u << 24;
constexpr float kScale = 2048.0f, kInv = 1.0f / 2048.0f;
constexpr int kStages = 3;

__host__ __device__ inline size_t state_bytes(int N) { return (size_t)16 * N * N; }
__host__ __device__ inline size_t entry_bytes(int N) { return (size_t)8 * N * N; }

// byte offset of the hi element (row, kcol) of an embedded state; lo at +kHalf
__device__ __forceinline__ uint32_t emb_off(int N, int row, int kcol) {
  const int KT = 2 * N / 64;
  return (uint32_t)(((row >> 7) * KT + (kcol >> 6))) * kTile + sw128(row & 127, kcol & 63, 128);
}

__device__ __forceinline__ float emb_val(const uint8_t* st, int N, int row, int kcol) {
  const uint32_t o = emb_off(N, row, kcol);
  const float h = __half2float(*reinterpret_cast<const __half*>(st + o));
  const float l = __half2float(*reinterpret_cast<const __half*>(st + o + kHalf));
  return fmaf(l, kInv, h);
}

// complex element (i, j) of the matrix Y whose embedding is st
__device__ __forceinline__ float2 emb_get(const uint8_t* st, int N, int i, int j) {
  return make_float2(emb_val(st, N, i, j), emb_val(st, N, N + i, j));
}

// ---------------------------------------------------------------------------- table planes
// grid: entries * (N/128) * KT tiles; each tile 256 rows x 8 granules
__global__ void __launch_bounds__(256) build_large_planes_kernel(const double2* __restrict__ T, int N,
                                                                 int transpose, uint8_t* __restrict__ out) {
  const int KT = 2 * N / 64, NT = N / 128;
  const int64_t tile = blockIdx.x;
  const int64_t e = tile / ((int64_t)NT * KT);
  const int rem = (int)(tile % ((int64_t)NT * KT));
  const int nt = rem / KT, kt = rem % KT;
  const double2* A = T + e * (int64_t)N * N;
  uint8_t* dst = out + tile * kTile;
  for (int gi = threadIdx.x; gi < 256 * 8; gi += blockDim.x) {
    const int r = gi >> 3, g = gi & 7;
    const int plane = r >> 7, n = nt * 128 + (r & 127);
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      __half hv[2];
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int k = kt * 64 + 8 * g + 2 * p + qq;             // 0 .. 2N-1
        const int kc = k < N ? k : k - N;
        const double2 z = transpose ? A[(int64_t)kc * N + n] : A[(int64_t)n * N + kc];
        const double v = k < N ? z.x : z.y;
        const __half h = __double2half(v);
        hv[qq] = plane == 0 ? h : __double2half((v - (double)__half2float(h)) * 2048.0);
      }
      w[p] = pack_half2(hv[0], hv[1]);
    }
    *reinterpret_cast<uint4*>(dst + sw128(r, 8 * g, 256)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------------------- state conversions
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& h, uint32_t& l) {
  const __half2 hh = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(hh);
  const __half2 ll = __floats2half2_rn((x0 - hf.x) * kScale, (x1 - hf.y) * kScale);
  h = *reinterpret_cast<const uint32_t*>(&hh);
  l = *reinterpret_cast<const uint32_t*>(&ll);
}

// Emb(Y) for Y given per chain: mode 0 Y = X^T, mode 1 Y = X^dag, mode 2 Y = X; src [G][N][N].
// One thread per (chain, row i of Y, granule of 8 columns j).
template <typename R>
__global__ void emb_from_complex_kernel(const cplx<R>* __restrict__ src, int N, int64_t G, int mode,
                                        uint8_t* __restrict__ dst) {
  const int64_t per = (int64_t)N * (N / 8);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < G * per;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / per;
    const int rem = (int)(idx % per);
    const int i = rem / (N / 8), j0 = (rem % (N / 8)) * 8;
    const cplx<R>* X = src + c * (int64_t)N * N;
    float re[8], im[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = j0 + q;
      cplx<R> v = mode == 2 ? X[(int64_t)i * N + j] : X[(int64_t)j * N + i];
      re[q] = (float)v.x;
      im[q] = mode == 1 ? -(float)v.y : (float)v.y;
    }
    uint32_t hr[4], lr[4], hi_[4], li_[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      split_pair(re[2 * p], re[2 * p + 1], hr[p], lr[p]);
      split_pair(im[2 * p], im[2 * p + 1], hi_[p], li_[p]);
    }
    uint8_t* st = dst + c * state_bytes(N);
    const uint32_t neg = 0x80008000u;
    // (i, j): Re ; (i, N+j): -Im ; (N+i, j): Im ; (N+i, N+j): Re
    uint32_t o = emb_off(N, i, j0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    o = emb_off(N, N + i, N + j0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    o = emb_off(N, N + i, j0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(li_[0], li_[1], li_[2], li_[3]);
    o = emb_off(N, i, N + j0);
    *reinterpret_cast<uint4*>(st + o) =
        make_uint4(hi_[0] ^ neg, hi_[1] ^ neg, hi_[2] ^ neg, hi_[3] ^ neg);
    *reinterpret_cast<uint4*>(st + o + kHalf) =
        make_uint4(li_[0] ^ neg, li_[1] ^ neg, li_[2] ^ neg, li_[3] ^ neg);
  }
}

// X from Emb(Y): mode 0 X = Y^T, mode 2 X = Y.  dst [G][N][N] complex<R>.
template <typename R>
__global__ void emb_to_complex_kernel(const uint8_t* __restrict__ src, int N, int64_t G, int mode,
                                      cplx<R>* __restrict__ dst) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < G * n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / n2;
    const int e = (int)(idx % n2);
    const int i = e / N, j = e % N;
    const float2 v = mode == 0 ? emb_get(src + c * state_bytes(N), N, j, i)
                               : emb_get(src + c * state_bytes(N), N, i, j);
    dst[idx] = cmake<R>((R)v.x, (R)v.y);
  }
}

__global__ void emb_identity_kernel(uint8_t* __restrict__ dst, int N, int64_t G) {
  // Emb(I) = I_{2N}: one granule of 8 per thread
  const int64_t per = (int64_t)2 * N * (2 * N / 8);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < G * per;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / per;
    const int rem = (int)(idx % per);
    const int row = rem / (2 * N / 8), k0 = (rem % (2 * N / 8)) * 8;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (row >= k0 && row < k0 + 8) {
      const int p = (row - k0) >> 1, hp = (row - k0) & 1;
      w[p] = (uint32_t)0x3C00u << (16 * hp);
    }
    uint8_t* st = dst + c * state_bytes(N);
    const uint32_t o = emb_off(N, row, k0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// ---------------------------------------------------------------------------- the step kernel
struct StepArgs {
  const uint8_t* cur;
  uint8_t* next;
  const uint8_t* planes;
  const int32_t* q;
  int64_t M;
  int K, d, base;
  int64_t levels;
  int64_t S, seg_len, F, t;
  int64_t gmod;       // chain c uses the factor of chain c % gmod
  int reverse;
  int N;
  int64_t* status;
};

__device__ __forceinline__ int64_t step_entry(const StepArgs& a, int64_t g) {
  const int64_t u = g / a.S, s = g % a.S;
  const int64_t f0 = s * a.seg_len;
  int64_t f1 = f0 + a.seg_len;
  if (f1 > a.F) f1 = a.F;
  const int64_t f = a.reverse ? f1 - 1 - a.t : f0 + a.t;
  if (f < f0 || f >= f1) return -1;
  const int64_t kd = (int64_t)a.K * a.d;
  const int64_t n = f / kd;
  const int r = (int)(f - n * kd);
  const int k = r / a.d, j = r - k * a.d;
  int32_t qv = a.q[(u * a.M + n) * a.K + k];
  if (qv < 0 || qv >= a.levels) qv = 0;
  for (int i = 0; i < j; ++i) qv /= a.base;
  return (int64_t)(k * a.d + j) * a.base + qv % a.base;
}

__global__ void __launch_bounds__(192, 1) tc_large_step_kernel(StepArgs a) {
  const int N = a.N;
  const int KT = 2 * N / 64, TM = 2 * N / 128, TN = N / 128;
  const int64_t c = blockIdx.x / (TM * TN);
  const int rem = (int)(blockIdx.x % (TM * TN));
  const int rt = rem / TN, nt = rem % TN;
  const int64_t e = step_entry(a, c % a.gmod);
  const uint8_t* Yc = a.cur + c * state_bytes(N);
  uint8_t* Yn = a.next + c * state_bytes(N);
  if (e < 0) {
    // chain finished its segment: carry this tile's destinations over unchanged
    for (int idx = threadIdx.x; idx < 128 * 16; idx += blockDim.x) {
      const int r = idx >> 4, gq = idx & 15;
      const int R = rt * 128 + r, kcol = nt * 128 + 8 * gq;
      const int Rm = R < N ? R + N : R - N;
      const uint32_t od = emb_off(N, R, kcol), om = emb_off(N, Rm, N + kcol);
      *reinterpret_cast<uint4*>(Yn + od) = *reinterpret_cast<const uint4*>(Yc + od);
      *reinterpret_cast<uint4*>(Yn + od + kHalf) = *reinterpret_cast<const uint4*>(Yc + od + kHalf);
      *reinterpret_cast<uint4*>(Yn + om) = *reinterpret_cast<const uint4*>(Yc + om);
      *reinterpret_cast<uint4*>(Yn + om + kHalf) = *reinterpret_cast<const uint4*>(Yc + om + kHalf);
    }
    return;
  }
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * 2 * kTile);
  uint64_t* empty = full + kStages;
  uint64_t* mma_done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      const uint8_t* Bbase = a.planes + (size_t)e * entry_bytes(N);
      for (int kt = 0; kt < KT; ++kt) {
        const uint32_t s = kt % kStages, u = kt / kStages;
        if (u > 0 && !mbar_wait_bounded_n(&empty[s], (u - 1) & 1, kLimit)) {
          *abort_flag = 1;
          break;
        }
        uint8_t* dA = smem + s * 2 * kTile;
        uint8_t* dB = dA + kTile;
        const uint8_t* sA = Yc + (size_t)(rt * KT + kt) * kTile;
        const uint8_t* sB = Bbase + (size_t)(nt * KT + kt) * kTile;
        mbar_arrive_expect_tx(&full[s], 2 * kTile);
        bulk_load(dA, sA, kHalf, &full[s]);
        bulk_load(dA + kHalf, sA + kHalf, kHalf, &full[s]);
        bulk_load(dB, sB, kHalf, &full[s]);
        bulk_load(dB + kHalf, sB + kHalf, kHalf, &full[s]);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      for (int kt = 0; kt < KT; ++kt) {
        const uint32_t s = kt % kStages, u = kt / kStages;
        if (*abort_flag || !mbar_wait_bounded_n(&full[s], u & 1, kLimit)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a_hi = smem_u32(smem + s * 2 * kTile);
        const uint32_t a_lo = a_hi + kHalf;
        const uint32_t b0 = a_hi + kTile;       // 256 rows: hi then lo
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t o = (uint32_t)kk * 32u;
          mma_f16(tmem, smem_desc_sw128(a_hi + o), smem_desc_sw128(b0 + o), kIdesc256,
                  (kt | kk) ? 1u : 0u);
          mma_f16(tmem + 128, smem_desc_sw128(a_lo + o), smem_desc_sw128(b0 + o), kIdesc128, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(mma_done);
    }
  } else {
    // epilogue: warps 0-3, thread = row of the output tile
    const int r = threadIdx.x;
    const int R = rt * 128 + r;
    const int Rm = R < N ? R + N : R - N;
    const uint32_t neg = R < N ? 0u : 0x80008000u;
    bool ok = mbar_wait_bounded_n(mma_done, 0, kLimit) && !*abort_flag;
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      *abort_flag = 1;
    } else {
      tc_fence_after();
      const uint32_t d1 = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
      for (int j = 0; j < 4; ++j) {
        uint32_t ra[32], rb[32];
        tmem_ld32(d1 + 32 * j, ra);
        tmem_ld32(d1 + 128 + 32 * j, rb);
        tmem_wait_ld();
        float z[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = fmaf(__uint_as_float(rb[i]), kInv, __uint_as_float(ra[i]));
#pragma unroll
        for (int gq = 0; gq < 4; ++gq) {
          uint32_t h[4], l[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) split_pair(z[8 * gq + 2 * p], z[8 * gq + 2 * p + 1], h[p], l[p]);
          const int kcol = nt * 128 + 32 * j + 8 * gq;
          const uint32_t od = emb_off(N, R, kcol), om = emb_off(N, Rm, N + kcol);
          *reinterpret_cast<uint4*>(Yn + od) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(Yn + od + kHalf) = make_uint4(l[0], l[1], l[2], l[3]);
          *reinterpret_cast<uint4*>(Yn + om) = make_uint4(h[0] ^ neg, h[1] ^ neg, h[2] ^ neg, h[3] ^ neg);
          *reinterpret_cast<uint4*>(Yn + om + kHalf) =
              make_uint4(l[0] ^ neg, l[1] ^ neg, l[2] ^ neg, l[3] ^ neg);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (*abort_flag && threadIdx.x == 0 && a.status)
    atomicAdd((unsigned long long*)&a.status[REDO_STATUS_TIMEOUT], 1ull);
  if (warp == 0) tmem_dealloc(tmem, 256);
}

constexpr uint32_t kStepSmem = kStages * 2 * kTile + 1024 + 128;

// ---------------------------------------------------------------------------- gradient traces
// Tr(H_k V^dag R) = sum_x sum_{(i,c) in nz(H_k)} H[i][c] conj(V[x][c]) R[x][i]  (V = P^dag):
// a sum over rows x of V and R, read straight from their embeddings (row x of Emb
// holds Re(row x) in K columns 0..N-1; row N+x holds Im(row x)).  Grid (chain, row block):
// each warp stages one row of V and of R in shared memory, its lanes walk the
// nonzeros, and block partials are added into acc[g]; trace_finish_kernel turns
// acc into dF/du and clears it.
__device__ __forceinline__ void emb_row_to_smem(const uint8_t* st, int N, int x, float* re, float* im,
                                                int lane) {
  for (int g = lane; g < N / 8; g += 32) {
    const uint32_t orr = emb_off(N, x, 8 * g), oi = emb_off(N, N + x, 8 * g);
    const uint4 hr = *reinterpret_cast<const uint4*>(st + orr);
    const uint4 lr = *reinterpret_cast<const uint4*>(st + orr + kHalf);
    const uint4 hi = *reinterpret_cast<const uint4*>(st + oi);
    const uint4 li = *reinterpret_cast<const uint4*>(st + oi + kHalf);
    const uint32_t hrw[4] = {hr.x, hr.y, hr.z, hr.w}, lrw[4] = {lr.x, lr.y, lr.z, lr.w};
    const uint32_t hiw[4] = {hi.x, hi.y, hi.z, hi.w}, liw[4] = {li.x, li.y, li.z, li.w};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&hrw[p]));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&lrw[p]));
      const float2 c = __half22float2(*reinterpret_cast<const __half2*>(&hiw[p]));
      const float2 d = __half22float2(*reinterpret_cast<const __half2*>(&liw[p]));
      re[8 * g + 2 * p] = fmaf(b.x, kInv, a.x);
      re[8 * g + 2 * p + 1] = fmaf(b.y, kInv, a.y);
      im[8 * g + 2 * p] = fmaf(d.x, kInv, c.x);
      im[8 * g + 2 * p + 1] = fmaf(d.y, kInv, c.y);
    }
  }
}

constexpr int kTraceRows = 8;   // rows per block (one per warp)

__global__ void __launch_bounds__(256) trace_emb_kernel(const uint8_t* __restrict__ V,
                                                        const uint8_t* __restrict__ Rs, int N, int64_t S,
                                                        int64_t seg_len, int64_t F, int64_t t, int K, int d,
                                                        const int32_t* __restrict__ hk_ptr,
                                                        const int32_t* __restrict__ hk_col,
                                                        const int32_t* __restrict__ hk_row,
                                                        const double2* __restrict__ hk_val,
                                                        double2* __restrict__ acc) {
  const int64_t g = blockIdx.x;
  const int64_t s = g % S;
  const int64_t f0 = s * seg_len;
  int64_t f1 = f0 + seg_len;
  if (f1 > F) f1 = F;
  const int64_t f = f1 - 1 - t;
  if (f < f0 || f >= f1) return;
  const int64_t kd = (int64_t)K * d;
  const int64_t n = f / kd;
  const int rr = (int)(f - n * kd);
  const int k = rr / d, j = rr - k * d;
  if (j != d - 1) return;
  extern __shared__ float rows[];            // per warp: Vre, Vim, Rre, Rim (N floats each)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* vre = rows + (size_t)warp * 4 * N;
  float* vim = vre + N;
  float* rre = vim + N;
  float* rim = rre + N;
  const int x = blockIdx.y * kTraceRows + warp;
  const uint8_t* Vg = V + g * state_bytes(N);
  const uint8_t* Rg = Rs + g * state_bytes(N);
  emb_row_to_smem(Vg, N, x, vre, vim, lane);
  emb_row_to_smem(Rg, N, x, rre, rim, lane);
  __syncwarp();
  const int p0 = hk_ptr[k * (N + 1)], p1 = hk_ptr[k * (N + 1) + N];
  double re = 0.0, im = 0.0;
  for (int e = p0 + lane; e < p1; e += 32) {
    const int i = hk_row[e], c = hk_col[e];
    // conj(V[x][c]) R[x][i]
    const float a = vre[c], b = vim[c], cr = rre[i], ci = rim[i];
    const float pr = a * cr + b * ci, pi = a * ci - b * cr;
    const double2 h = hk_val[e];
    re += h.x * pr - h.y * pi;
    im += h.x * pi + h.y * pr;
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  __shared__ double sre[8], sim[8];
  if (lane == 0) {
    sre[warp] = re;
    sim[warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < 8; ++w) {
      tr += sre[w];
      ti += sim[w];
    }
    atomicAdd(&acc[g].x, tr);
    atomicAdd(&acc[g].y, ti);
  }
}

__global__ void trace_finish_kernel(double2* __restrict__ acc, int64_t G, int64_t S, int64_t seg_len,
                                    int64_t F, int64_t t, int K, int d, const double2* __restrict__ tau,
                                    double scale, int64_t M, double* __restrict__ grad) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int64_t u = g / S, s = g % S;
  const int64_t f0 = s * seg_len;
  int64_t f1 = f0 + seg_len;
  if (f1 > F) f1 = F;
  const int64_t f = f1 - 1 - t;
  if (f < f0 || f >= f1) return;
  const int64_t kd = (int64_t)K * d;
  const int64_t n = f / kd;
  const int rr = (int)(f - n * kd);
  const int k = rr / d, j = rr - k * d;
  if (j != d - 1) return;
  const double2 T = acc[g];
  const double2 tu = tau[u];
  grad[(u * M + n) * K + k] = scale * (tu.x * T.y - tu.y * T.x);
  acc[g] = make_double2(0.0, 0.0);
}

static unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

static cudaError_t step(const redo_table* t, const int32_t* q, const ChainPlan& p, int64_t tt, int reverse,
                        int64_t chains, int64_t gmod, const uint8_t* planes, const uint8_t* cur,
                        uint8_t* next, int64_t* status, cudaStream_t s) {
  StepArgs a;
  a.cur = cur;
  a.next = next;
  a.planes = planes;
  a.q = q;
  a.M = p.M;
  a.K = t->K;
  a.d = t->digits;
  a.base = t->base;
  a.levels = t->levels;
  a.S = p.S;
  a.seg_len = p.seg_len;
  a.F = p.F;
  a.t = tt;
  a.gmod = gmod;
  a.reverse = reverse;
  a.N = t->N;
  a.status = status;
  const int64_t blocks = chains * (2 * t->N / 128) * (t->N / 128);
  tc_large_step_kernel<<<(unsigned)blocks, 192, kStepSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tcl

using namespace tcl;

size_t tc_large_planes_bytes(const redo_table* t) { return 2 * (size_t)t->entries * entry_bytes(t->N); }

cudaError_t launch_build_tc_large_planes(const redo_table* t, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(tc_large_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kStepSmem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = t->entries * (t->N / 128) * (2 * t->N / 64);
  uint8_t* rows = (uint8_t*)t->tc_planes;
  uint8_t* cols = rows + (size_t)t->entries * entry_bytes(t->N);
  build_large_planes_kernel<<<(unsigned)tiles, 256, 0, s>>>(t->T64, t->N, 0, rows);
  build_large_planes_kernel<<<(unsigned)tiles, 256, 0, s>>>(t->T64, t->N, 1, cols);
  return cudaGetLastError();
}

size_t tc_large_prop_workspace(const redo_table* t, const ChainPlan& p, bool reunit) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return large_prop_workspace(t, p, REDO_FP32, reunit) + 2 * up((size_t)p.B * p.S * state_bytes(t->N));
}

// Segment products by tensor-core chains, then the FP32 re-unitarisation, combine and
// FP64 polar step of the SIMT large-N path.
cudaError_t tc_large_propagate(const redo_table* t, const int32_t* q, const ChainPlan& p, bool reunit,
                               void* ws, void** result, int* result_prec, int64_t* status,
                               cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int N = t->N;
  const int64_t G = p.B * p.S;
  char* base = (char*)ws;
  cudaError_t e = cudaFuncSetAttribute(tc_large_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kStepSmem);
  if (e != cudaSuccess) return e;
  const size_t simt = large_prop_workspace(t, p, REDO_FP32, reunit);
  uint8_t* st0 = (uint8_t*)(base + simt);
  uint8_t* st1 = st0 + up((size_t)G * state_bytes(N));
  emb_identity_kernel<<<blocks_for(G * 2 * N * (2 * N / 8)), 256, 0, s>>>(st0, N, G);
  uint8_t* cur = st0;
  uint8_t* nxt = st1;
  const uint8_t* rows = (const uint8_t*)t->tc_planes;
  for (int64_t tt = 0; tt < p.seg_len; ++tt) {
    if ((e = step(t, q, p, tt, 0, G, G, rows, cur, nxt, status, s))) return e;
    std::swap(cur, nxt);
  }
  // segment products X = Y^T into the SIMT path's segment buffer (its first region)
  float2* seg = (float2*)base;
  emb_to_complex_kernel<float><<<blocks_for(G * (int64_t)N * N), 256, 0, s>>>(cur, N, G, 0, seg);
  return large_finish_fp32(t, p, reunit, ws, result, result_prec, s);
}

size_t tc_large_grad_workspace(const redo_table* t, const ChainPlan& p) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t G = (size_t)p.B * p.S;
  // + 2G embedded states x 2 (ping-pong) + 2G row-major FP32 transposes for the traces
  return large_grad_workspace(t, p, REDO_FP32) + 4 * up(G * state_bytes(t->N)) + up(G * sizeof(double2));
}

// Gradient: tensor-core forward segments, SIMT FP32 checkpoint/costate scans,
// tensor-core reverse sweep of (V = P^dag, R) with embedded-state traces.
cudaError_t tc_large_grad(const redo_table* t, const int32_t* q, const ChainPlan& p, const double2* UT,
                          int tb, double* F_out, double* grad, void* ws, int64_t* status,
                          cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int N = t->N;
  const int64_t G = p.B * p.S;
  const int64_t n2 = (int64_t)N * N;
  char* base = (char*)ws;
  const size_t simt = large_grad_workspace(t, p, REDO_FP32);
  const size_t sb = up((size_t)G * state_bytes(N));
  uint8_t* s0 = (uint8_t*)(base + simt);       // 2G states (V then R)
  uint8_t* s1 = s0 + 2 * sb;                   // ping
  const uint8_t* rows = (const uint8_t*)t->tc_planes;
  const uint8_t* cols = rows + (size_t)t->entries * entry_bytes(N);
  cudaError_t e = cudaFuncSetAttribute(tc_large_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kStepSmem);
  if (e != cudaSuccess) return e;
  // forward segment chains on s0 / s1 (first G states)
  emb_identity_kernel<<<blocks_for(G * 2 * N * (2 * N / 8)), 256, 0, s>>>(s0, N, G);
  uint8_t* cur = s0;
  uint8_t* nxt = s1;
  for (int64_t tt = 0; tt < p.seg_len; ++tt) {
    if ((e = step(t, q, p, tt, 0, G, G, rows, cur, nxt, status, s))) return e;
    std::swap(cur, nxt);
  }
  float2* seg = (float2*)base;                 // the SIMT layout's segment region
  emb_to_complex_kernel<float><<<blocks_for(G * n2), 256, 0, s>>>(cur, N, G, 0, seg);
  float2 *Pck = nullptr, *Rck = nullptr;
  double2* tau = nullptr;
  if ((e = large_grad_scans_fp32(t, p, UT, tb, F_out, ws, &Pck, &Rck, &tau, s))) return e;
  if (p.M == 0) return cudaGetLastError();
  // reverse sweep: chains [0, G) hold V = P^dag, [G, 2G) hold R; both right-multiplied by A_f
  emb_from_complex_kernel<float><<<blocks_for(G * N * (N / 8)), 256, 0, s>>>(Pck, N, G, 1, s0);
  emb_from_complex_kernel<float><<<blocks_for(G * N * (N / 8)), 256, 0, s>>>(Rck, N, G, 2, s0 + sb);
  cur = s0;
  nxt = s1;
  double2* acc = (double2*)(s1 + 2 * sb);      // per-chain trace accumulators
  if ((e = cudaMemsetAsync(acc, 0, sizeof(double2) * G, s))) return e;
  const size_t trace_smem = (size_t)kTraceRows * 4 * N * sizeof(float);
  if ((e = cudaFuncSetAttribute(trace_emb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)trace_smem)))
    return e;
  const double scale = 2.0 * t->dt / ((double)N * (double)N);
  const int64_t kd = (int64_t)t->K * t->digits;
  const bool aligned = (p.seg_len % kd) == 0;
  for (int64_t tt = 0; tt < p.seg_len; ++tt) {
    // traces are needed where the visited factor is a term's last digit; with
    // segments aligned to whole steps that is every d-th sweep step for all chains
    if (!aligned || ((p.seg_len - 1 - tt) % t->digits) == (t->digits - 1)) {
      dim3 grid((unsigned)G, (unsigned)(N / kTraceRows));
      trace_emb_kernel<<<grid, 256, trace_smem, s>>>(cur, cur + sb, N, p.S, p.seg_len, p.F, tt, t->K,
                                                     t->digits, t->hk_ptr, t->hk_col, t->hk_row, t->hk_val,
                                                     acc);
      trace_finish_kernel<<<(unsigned)((G + 127) / 128), 128, 0, s>>>(acc, G, p.S, p.seg_len, p.F, tt, t->K,
                                                                      t->digits, tau, scale, p.M, grad);
    }
    if ((e = step(t, q, p, tt, 1, 2 * G, G, cols, cur, nxt, status, s))) return e;
    std::swap(cur, nxt);
  }
  return cudaGetLastError();
}

}  // namespace redo
