// Tensor-core (tcgen05, split-FP16) sweeps for 128 <= N <= 1024.
// (Section II process 2, Eq. exp2prod, the Section III chain and its GRAPE gradient (Fig. fc), and
// the Section IV dynamics, on the tensor cores at large N.)
//
// State layout.  A chain state Y (N x N complex) is stored as the real N x 2N matrix
// S = [Re Y | Im Y] in split FP16 (hi = fp16(v), lo = fp16((v - hi) 2^11)), cut into tiles
// of 128 rows x 64 columns: tile (rt, kt) is the hi block (128 rows of 128 B, K-major,
// 128-byte swizzled) followed by the lo block, 32 KB, tiles row-major.  A step Y <- Y C
// gives, with the operand B^T whose row n is [Re C[:, n], Im C[:, n]],
//     Re Z = [Re Y | Im Y] [Re C; -Im C],    Im Z = [Im Y | Re Y] [Re C; Im C]:
// both halves read the same tiles of S (the Im half with its K tiles rotated by N) against
// one operand plane, and the Re half negates the products of its second K half through the
// instruction descriptor's negate-B bit.
//
// Operand planes.  Every table entry C is stored as tiles (nb, kt) holding NB rows of B^T
// hi followed by the same NB rows lo, 64 K columns wide (NB = 128 for N <= 256, else 256),
// swizzled like the states.  Two sets exist: "row" planes with C = A^T (forward steps
// X <- A X on Y = X^T) and "column" planes with C = A (reverse sweep V <- V A, R <- R A).
//
// Sweep kernel.  A right product acts on every row of Y separately, so each 128-row block
// of each chain is its own sequence of steps.  A unit of work is (step, chain, row block,
// half, column block); units are handed out in step order from a global ticket counter to
// persistent CTAs, and a unit waits only until the previous step of its own row block is
// complete (a counter per chain and row block that every finished unit increments).  In a
// CTA, a scheduler warp claims tickets and waits for the counters, up to two units ahead
// through an in-CTA unit queue; a producer warp streams the queued units' A (state) and B
// (operand) tiles through a ring of bulk copies; one thread issues the MMAs into tensor
// memory; four epilogue warps turn the FP32 accumulators into the next state's split FP16
// tiles; a publisher warp increments the counters with release semantics once a unit's
// stores are done.  In the reverse sweep of the gradient four more warps evaluate
// Tr(H_k V^dag R) for a slice of rows of the current states while the MMAs run; they
// count their finished slices per row block of a V/R pair (through the publisher), and a
// unit writes over the states of step t-1 only once all of that step's slices of its rows
// are added.  Every wait is bounded; a timed-out CTA raises a sweep-wide abort flag and
// leaves.
#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "tcgen05.cuh"

#include <cstdlib>
#include <cstring>
#include <type_traits>

namespace redo {
namespace tcl {

using namespace tc;

constexpr uint32_t kTile = 32768;     // state tile: hi (16 KB) + lo (16 KB)
constexpr uint32_t kHalf = 16384;
constexpr uint32_t kLimit = 1u << 24; // mbarrier polls before a wait gives up
constexpr uint32_t kSpin = 1u << 22;  // counter polls before a dependency wait gives up
constexpr float kScale = 2048.0f, kInv = 1.0f / 2048.0f;
constexpr uint32_t kNegB = 1u << 14;  // instruction descriptor: negate B
constexpr int kQ = 2;                 // depth of the in-CTA unit queue (1, 3, 4 and 8 measured slower)
constexpr int kSweepThreads = 384;    // 4 epilogue, producer, MMA, 4 trace warps, scheduler, publisher

__host__ __device__ inline size_t state_bytes(int N) { return (size_t)8 * N * N; }
__host__ __device__ inline size_t entry_bytes(int N) { return (size_t)8 * N * N; }
__host__ __device__ inline int trace_warps(int N) { return N >= 1024 ? 2 : 4; }

template <int NB, int ST = (NB == 256 ? 2 : 3)>
struct Geo {
  static constexpr uint32_t kB = (uint32_t)NB * 256u;      // NB rows hi + NB rows lo, 128 B each
  static constexpr uint32_t kStage = kTile + kB;
  static constexpr int kStages = ST;
  static constexpr int kAcc = 2 * NB;                       // TMEM columns of D1 | D2
  static constexpr int kBufs = 512 / kAcc;
  static constexpr uint32_t kRing = kStages * kStage;
};

// Shared memory per trace warp for rows staged by cp.async (the reverse sweep of a gradient
// with one-nonzero-per-row operators at N <= 256): SL rows of eight 16-byte granules per lane.
__host__ __device__ constexpr uint32_t trace_stage_bytes(int SL) { return (uint32_t)SL * 8 * 32 * 16; }

constexpr int kTraceRows = 6;         // staged rows in flight per trace warp

// staged: the trace rows go through shared memory (two ring stages; the row buffers of the
// general trace path are not needed then)
inline size_t sweep_smem(int NB, int N, bool staged) {
  const size_t ring = NB == 256 ? Geo<256>::kRing : (staged ? Geo<128, 2>::kRing : Geo<128>::kRing);
  const size_t rows = staged ? (size_t)trace_warps(N) * trace_stage_bytes(kTraceRows) : (size_t)trace_warps(N) * 16 * N;
  return ring + rows + 2048;
}

// byte offset of the hi element (row, kcol) of a state; lo at +kHalf
__host__ __device__ __forceinline__ uint32_t s_off(int N, int row, int kcol) {
  const int KT = 2 * N / 64;
  return (uint32_t)(((row >> 7) * KT + (kcol >> 6))) * kTile + sw128(row & 127, kcol & 63, 128);
}

__device__ __forceinline__ float s_val(const uint8_t* st, int N, int row, int kcol) {
  const uint32_t o = s_off(N, row, kcol);
  const float h = __half2float(*reinterpret_cast<const __half*>(st + o));
  const float l = __half2float(*reinterpret_cast<const __half*>(st + o + kHalf));
  return fmaf(l, kInv, h);
}

__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& h, uint32_t& l) {
  const __half2 hh = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(hh);
  const __half2 ll = __floats2half2_rn((x0 - hf.x) * kScale, (x1 - hf.y) * kScale);
  h = *reinterpret_cast<const uint32_t*>(&hh);
  l = *reinterpret_cast<const uint32_t*>(&ll);
}

// ---------------------------------------------------------------------------- operand planes
// grid: entries * (N / NB) * KT tiles; a tile is 2 NB rows (hi, lo) x 8 granules of 8 fp16.
__global__ void __launch_bounds__(256) build_planes_kernel(const double2* __restrict__ T, int N, int NB,
                                                           int transpose, uint8_t* __restrict__ out) {
  const int KT = 2 * N / 64, TNB = N / NB;
  const int64_t tile = blockIdx.x;
  const int64_t e = tile / ((int64_t)TNB * KT);
  const int rem = (int)(tile % ((int64_t)TNB * KT));
  const int nb = rem / KT, kt = rem % KT;
  const double2* A = T + e * (int64_t)N * N;
  uint8_t* dst = out + tile * (int64_t)NB * 256;
  for (int gi = threadIdx.x; gi < 2 * NB * 8; gi += blockDim.x) {
    const int r = gi >> 3, g = gi & 7;
    const int plane = r / NB, n = nb * NB + r % NB;
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
    *reinterpret_cast<uint4*>(dst + sw128(r, 8 * g, 2 * NB)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------------------- state conversions
// S from complex X per chain: mode 0 Y = X^T, mode 1 Y = X^dag, mode 2 Y = X; src [G][N][N].
// One thread per (chain, row i, granule of 8 columns j).
template <typename R>
__global__ void s_from_complex_kernel(const cplx<R>* __restrict__ src, int N, int64_t G, int mode,
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
      const cplx<R> v = mode == 2 ? X[(int64_t)i * N + j] : X[(int64_t)j * N + i];
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
    uint32_t o = s_off(N, i, j0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    o = s_off(N, i, N + j0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(li_[0], li_[1], li_[2], li_[3]);
  }
}

// X from S: mode 0 X = Y^T, mode 2 X = Y.  dst [G][N][N] complex<R>.
template <typename R>
__global__ void s_to_complex_kernel(const uint8_t* __restrict__ src, int N, int64_t G, int mode,
                                    cplx<R>* __restrict__ dst, size_t stride) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < G * n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / n2;
    const int e = (int)(idx % n2);
    const int i = e / N, j = e % N;
    const uint8_t* st = src + c * stride;
    const int row = mode == 0 ? j : i, col = mode == 0 ? i : j;
    dst[idx] = cmake<R>((R)s_val(st, N, row, col), (R)s_val(st, N, row, N + col));
  }
}

// S of the identity: one granule of 8 per thread
__global__ void s_identity_kernel(uint8_t* __restrict__ dst, int N, int64_t G) {
  const int64_t per = (int64_t)N * (2 * N / 8);
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
    const uint32_t o = s_off(N, row, k0);
    *reinterpret_cast<uint4*>(st + o) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(st + o + kHalf) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// ---------------------------------------------------------------------------- the sweep kernel
struct SweepArgs {
  uint8_t* buf0;          // states at even steps, chains x state_bytes
  uint8_t* buf1;          // states at odd steps
  const uint8_t* planes;
  const int32_t* q;
  int64_t M;
  int K, d, base;
  int64_t levels;
  int64_t S, seg_len, F;
  int64_t chains;         // forward: G; reverse: 2G (V chains, then R chains)
  int64_t gmod;           // chain c multiplies by the factor of chain c % gmod
  int64_t steps;
  int reverse;            // 0: factors in order from the segment start; 1: from its end
  int trace;              // reverse sweep of the gradient: traces and V/R coupling
  int N;
  uint32_t* cnt;          // [chains][N / 128] units per row block whose outputs are written
  uint32_t* tcnt;         // [gmod][N / 128] units per row block of a V/R pair whose trace part is added
  uint32_t* ticket;
  int* abort;
  const int32_t* hk_ptr;
  const int32_t* hk_col;
  const int32_t* hk_row;
  const double2* hk_val;
  const int32_t* xmask;   // compact operators (one nonzero per row, at r ^ m_k) or nullptr
  const float2* xval;
  double2* acc;           // [gmod][seg_len] trace accumulators
  int64_t* status;
  // Kept forward states (the gradient with every forward state kept): a forward sweep with
  // `store` writes the state after step t of chain c to store[c][t] (inputs: buf0 at t = 0,
  // store[c][t-1] after), and a reverse sweep with `vstore` has R chains only and reads the
  // trace's V = P^dag as the conjugate of the kept forward state of the same factor.
  uint8_t* store;
  const uint8_t* vstore;
};

__device__ __forceinline__ const uint8_t* state_in(const SweepArgs& a, int64_t c, int64_t t, size_t sb) {
  if (a.store) return t == 0 ? a.buf0 + c * sb : a.store + ((size_t)c * a.steps + (size_t)(t - 1)) * sb;
  return ((t & 1) ? a.buf1 : a.buf0) + c * sb;
}

__device__ __forceinline__ uint8_t* state_out(const SweepArgs& a, int64_t c, int64_t t, size_t sb) {
  if (a.store) return a.store + ((size_t)c * a.steps + (size_t)t) * sb;
  return ((t & 1) ? a.buf0 : a.buf1) + c * sb;
}

struct Unit {
  int64_t t, c;
  int rt, h, nb;
};

__device__ __forceinline__ Unit decode(const SweepArgs& a, int64_t tk, int RT, int TNB) {
  const int per_chain = RT * 2 * TNB;
  const int64_t per_step = a.chains * per_chain;
  Unit u;
  u.t = tk / per_step;
  const int64_t r = tk - u.t * per_step;
  const int64_t ci = r / per_chain;
  // the reverse sweep hands out the units of V chain g and R chain gmod + g together
  u.c = (a.trace && !a.vstore) ? ((ci & 1) ? a.gmod + (ci >> 1) : (ci >> 1)) : ci;
  const int r2 = (int)(r - ci * per_chain);
  u.rt = r2 / (2 * TNB);
  const int r3 = r2 % (2 * TNB);
  u.h = r3 / TNB;
  u.nb = r3 % TNB;
  return u;
}

// table entry multiplied at step t of chain g (or -1 past its segment); k and whether
// the factor is its term's last digit (where the gradient needs a trace)
__device__ __forceinline__ int64_t factor_entry(const SweepArgs& a, int64_t g, int64_t t, int& k, bool& last) {
  const int64_t u = g / a.S, s = g % a.S;
  const int64_t f0 = s * a.seg_len;
  int64_t f1 = f0 + a.seg_len;
  if (f1 > a.F) f1 = a.F;
  const int64_t f = a.reverse ? f1 - 1 - t : f0 + t;
  k = 0;
  last = false;
  if (f < f0 || f >= f1) return -1;
  const int64_t kd = (int64_t)a.K * a.d;
  const int64_t n = f / kd;
  const int r = (int)(f - n * kd);
  k = r / a.d;
  const int j = r - k * a.d;
  last = j == a.d - 1;
  int32_t qv = a.q[(u * a.M + n) * a.K + k];
  if (qv < 0 || qv >= a.levels) qv = 0;
  for (int i = 0; i < j; ++i) qv /= a.base;
  return (int64_t)(k * a.d + j) * a.base + qv % a.base;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Counter increment with release semantics at GPU scope: after the CTA barrier that precedes it,
// every write of the CTA's threads before that barrier is visible to a reader that acquires the
// new value (ld_acquire in wait_count).
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// false on time-out or when the sweep was aborted
__device__ bool wait_count(const uint32_t* cnt, uint32_t target, const int* abort) {
  for (uint32_t i = 0; i < kSpin; ++i) {
    if (ld_acquire(cnt) >= target) return true;
    if ((i & 63) == 63 && ld_relaxed(abort)) return false;
    __nanosleep(16);
  }
  return false;
}

// mbarrier wait that also gives up once the CTA or the sweep was aborted
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* local_abort, const int* abort) {
  for (uint32_t i = 0; i < kLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 1023) == 1023 && (*local_abort || ld_relaxed(abort))) return false;
  }
  return false;
}

__device__ __forceinline__ void unpack8(const uint4& hv, const uint4& lv, float* d) {
  const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&hw[p]));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&lw[p]));
    d[2 * p] = fmaf(b.x, kInv, a.x);
    d[2 * p + 1] = fmaf(b.y, kInv, a.y);
  }
}

// Part of Tr(H_k V^dag R) = sum_x sum_{(i,c) in nz(H_k)} H[i][c] conj(V[x][c]) R[x][i] over the
// rows x0, x0 + stride, ... (nrows of them) of the states Vs and Rs, added into (sr, si).
// Rows of V and R pass through shared memory as FP32 (vre, vim, rre, rim: N floats each);
// a lane holds GPL = N / 128 granules of a row.  For GPL <= 2 the next row's loads are
// issued before the current row's sum; larger rows are loaded in pieces of two granules.
template <int GPL>
__device__ __forceinline__ void trace_slice(const uint8_t* Vs, const uint8_t* Rs, int N, int x0, int nrows,
                                            int stride, int p0, int p1, const int32_t* __restrict__ hk_row,
                                            const int32_t* __restrict__ hk_col,
                                            const double2* __restrict__ hk_val, float* vre, float* vim,
                                            float* rre, float* rim, int lane, bool conjV, double& sr,
                                            double& si) {
  constexpr int CH = GPL < 2 ? GPL : 2;           // granules per lane held in registers
  constexpr bool kPrefetch = GPL <= 2;
  uint4 vh[CH], vl[CH], rh[CH], rl[CH];
  auto issue = [&](int x, int c0) {
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const uint32_t o = s_off(N, x, 8 * (lane + 32 * (c0 + i)));
      vh[i] = __ldcg(reinterpret_cast<const uint4*>(Vs + o));
      vl[i] = __ldcg(reinterpret_cast<const uint4*>(Vs + o + kHalf));
      rh[i] = __ldcg(reinterpret_cast<const uint4*>(Rs + o));
      rl[i] = __ldcg(reinterpret_cast<const uint4*>(Rs + o + kHalf));
    }
  };
  auto unpack = [&](int c0) {
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int kcol = 8 * (lane + 32 * (c0 + i));
      const bool re = kcol < N;
      unpack8(vh[i], vl[i], (re ? vre : vim) + (re ? kcol : kcol - N));
      unpack8(rh[i], rl[i], (re ? rre : rim) + (re ? kcol : kcol - N));
    }
  };
  if (kPrefetch && nrows > 0) issue(x0, 0);
  for (int r = 0; r < nrows; ++r) {
    if (kPrefetch) {
      unpack(0);
      if (r + 1 < nrows) issue(x0 + (r + 1) * stride, 0);
    } else {
#pragma unroll
      for (int c0 = 0; c0 < GPL; c0 += CH) {
        issue(x0 + r * stride, c0);
        unpack(c0);
      }
    }
    __syncwarp();
    float tr = 0.0f, ti = 0.0f;
    for (int e = p0 + lane; e < p1; e += 32) {
      const int i = hk_row[e], cc = hk_col[e];
      const double2 hv = hk_val[e];
      const float hx = (float)hv.x, hy = (float)hv.y;
      // conj(V[x][cc]) R[x][i]
      const float va = vre[cc], vb = conjV ? -vim[cc] : vim[cc], ra = rre[i], rb = rim[i];
      const float pr = fmaf(va, ra, vb * rb), pi = fmaf(va, rb, -vb * ra);
      tr = fmaf(hx, pr, fmaf(-hy, pi, tr));
      ti = fmaf(hx, pi, fmaf(hy, pr, ti));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, off);
      ti += __shfl_xor_sync(0xffffffffu, ti, off);
    }
    sr += (double)tr;
    si += (double)ti;
    __syncwarp();
  }
}

__device__ __forceinline__ void xor_perm8(float (&v)[8], int m7) {
  if (m7 & 1) {
#pragma unroll
    for (int w = 0; w < 8; w += 2) { const float x = v[w]; v[w] = v[w + 1]; v[w + 1] = x; }
  }
  if (m7 & 2) {
#pragma unroll
    for (int w = 0; w < 8; ++w)
      if (!(w & 2)) { const float x = v[w]; v[w] = v[w + 2]; v[w + 2] = x; }
  }
  if (m7 & 4) {
#pragma unroll
    for (int w = 0; w < 4; ++w) { const float x = v[w]; v[w] = v[w + 4]; v[w + 4] = x; }
  }
}

// One row's granule of the compact trace: ld = R Re hi, lo, R Im hi, lo, V Re hi, lo, V Im hi, lo
// (V's granule already the one at column i ^ m), h = the operator's values on the granule.
__device__ __forceinline__ void trace_row(const uint4 (&ld)[8], const float2 (&h)[8], int m7, bool conjV,
                                          float& tr, float& ti) {
  float rr[8], ri[8], vr[8], vi[8];
  unpack8(ld[0], ld[1], rr);
  unpack8(ld[2], ld[3], ri);
  unpack8(ld[4], ld[5], vr);
  unpack8(ld[6], ld[7], vi);
  if (conjV) {
#pragma unroll
    for (int w = 0; w < 8; ++w) vi[w] = -vi[w];
  }
  xor_perm8(vr, m7);
  xor_perm8(vi, m7);
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    // conj(V[x][i ^ m]) R[x][i]
    const float pr = fmaf(vr[w], rr[w], vi[w] * ri[w]);
    const float pi = fmaf(vr[w], ri[w], -vi[w] * rr[w]);
    tr = fmaf(h[w].x, pr, fmaf(-h[w].y, pi, tr));
    ti = fmaf(h[w].x, pi, fmaf(h[w].y, pr, ti));
  }
}

// The same part of the trace when H_k has one nonzero per row, h_i = H_k[i][i ^ m]:
// sum_x sum_i h_i conj(V[x][i ^ m]) R[x][i].  A lane takes the complex granules
// q = lane + 32 j (columns 8q .. 8q+7) of a row: R's own granule and V's granule q ^ (m >> 3),
// permuted inside by m & 7, straight from global memory into registers, kRB rows at a
// time.  FP32 partial sums (tr, ti) stay per lane.
__device__ __forceinline__ void trace_xor(const uint8_t* Vs, const uint8_t* Rs, int N, int x0, int nrows,
                                          int stride, int m, const float2* __restrict__ hv, int lane,
                                          bool conjV, float& tr, float& ti) {
  constexpr int kRB = 2;
  const int NG = N / 8, mq = m >> 3, m7 = m & 7;
  for (int q = lane; q < NG; q += 32) {
    const int qv = q ^ mq;
    float2 h[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) h[w] = __ldg(hv + 8 * q + w);
    const uint32_t orr = s_off(N, 0, 8 * q) , ori = s_off(N, 0, N + 8 * q);
    const uint32_t ovr = s_off(N, 0, 8 * qv), ovi = s_off(N, 0, N + 8 * qv);
    for (int r0 = 0; r0 < nrows; r0 += kRB) {
      uint4 ld[kRB][8];
#pragma unroll
      for (int b = 0; b < kRB; ++b) {
        if (r0 + b < nrows) {
          // s_off(x, kcol) = ro(x) + (s_off(0, kcol) ^ sw(x)): the row moves by 128 B inside
          // a tile and by a tile row per 128 rows, and swizzles the 16-byte granule index
          const int x = x0 + (r0 + b) * stride;
          const uint32_t ro = (uint32_t)((x >> 7) * (2 * N / 64)) * kTile + (uint32_t)(x & 127) * 128u;
          const uint32_t sw = (uint32_t)((x & 7) << 4);        // swizzle of row x
          const uint8_t* pr = Rs + ro + (orr ^ sw);
          const uint8_t* pi = Rs + ro + (ori ^ sw);
          const uint8_t* vr = Vs + ro + (ovr ^ sw);
          const uint8_t* vi = Vs + ro + (ovi ^ sw);
          ld[b][0] = __ldcg(reinterpret_cast<const uint4*>(pr));
          ld[b][1] = __ldcg(reinterpret_cast<const uint4*>(pr + kHalf));
          ld[b][2] = __ldcg(reinterpret_cast<const uint4*>(pi));
          ld[b][3] = __ldcg(reinterpret_cast<const uint4*>(pi + kHalf));
          ld[b][4] = __ldcg(reinterpret_cast<const uint4*>(vr));
          ld[b][5] = __ldcg(reinterpret_cast<const uint4*>(vr + kHalf));
          ld[b][6] = __ldcg(reinterpret_cast<const uint4*>(vi));
          ld[b][7] = __ldcg(reinterpret_cast<const uint4*>(vi + kHalf));
        } else {
#pragma unroll
          for (int z = 0; z < 8; ++z) ld[b][z] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
#pragma unroll
      for (int b = 0; b < kRB; ++b) trace_row(ld[b], h, m7, conjV, tr, ti);
    }
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

// trace_xor for N <= 256 (one granule per lane) with the granules of SL rows in flight through
// the warp's shared-memory stage (trace_stage_bytes(SL)) instead of registers: rows are fetched
// two at a time by cp.async, a pair is consumed while the next pairs are on their way.  A lane
// reads back only the granules it fetched itself.
template <int SL>
__device__ __forceinline__ void trace_xor_staged(const uint8_t* Vs, const uint8_t* Rs, int N, int x0, int nrows,
                                                 int stride, int m, const float2* __restrict__ hv, int lane,
                                                 bool conjV, float& tr, float& ti, uint8_t* stage) {
  const int NG = N / 8, mq = m >> 3, m7 = m & 7;
  const bool active = lane < NG;
  const int q = active ? lane : 0, qv = q ^ mq;
  float2 h[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) h[w] = active ? __ldg(hv + 8 * q + w) : make_float2(0.f, 0.f);
  const uint32_t orr = s_off(N, 0, 8 * q), ori = s_off(N, 0, N + 8 * q);
  const uint32_t ovr = s_off(N, 0, 8 * qv), ovi = s_off(N, 0, N + 8 * qv);
  const uint32_t sbase = smem_u32(stage);
  auto slot_off = [&](int s, int z) -> uint32_t { return (uint32_t)(((s * 8 + z) * 32 + lane) * 16); };
  auto issue = [&](int r) {
    if (active && r < nrows) {
      const int x = x0 + r * stride;
      const uint32_t ro = (uint32_t)((x >> 7) * (2 * N / 64)) * kTile + (uint32_t)(x & 127) * 128u;
      const uint32_t sw = (uint32_t)((x & 7) << 4);
      const uint8_t* pr = Rs + ro + (orr ^ sw);
      const uint8_t* pi = Rs + ro + (ori ^ sw);
      const uint8_t* vr = Vs + ro + (ovr ^ sw);
      const uint8_t* vi = Vs + ro + (ovi ^ sw);
      const int s = r % SL;
      cp_async16(sbase + slot_off(s, 0), pr);
      cp_async16(sbase + slot_off(s, 1), pr + kHalf);
      cp_async16(sbase + slot_off(s, 2), pi);
      cp_async16(sbase + slot_off(s, 3), pi + kHalf);
      cp_async16(sbase + slot_off(s, 4), vr);
      cp_async16(sbase + slot_off(s, 5), vr + kHalf);
      cp_async16(sbase + slot_off(s, 6), vi);
      cp_async16(sbase + slot_off(s, 7), vi + kHalf);
    }
  };
  auto consume = [&](int r) {
    if (active && r < nrows) {
      uint4 ld[8];
      const int s = r % SL;
#pragma unroll
      for (int z = 0; z < 8; ++z) ld[z] = *reinterpret_cast<const uint4*>(stage + slot_off(s, z));
      trace_row(ld, h, m7, conjV, tr, ti);
    }
  };
#pragma unroll
  for (int g = 0; g < SL / 2; ++g) {
    issue(2 * g);
    issue(2 * g + 1);
    cp_async_commit();
  }
  for (int r = 0; r < nrows; r += 2) {
    cp_async_wait<SL / 2 - 1>();                          // rows r, r + 1 have landed
    consume(r);
    consume(r + 1);
    __syncwarp();                                         // their slots are read before refilling
    issue(r + SL);
    issue(r + SL + 1);
    cp_async_commit();
  }
  cp_async_wait<0>();
}

// STG: the trace rows staged in shared memory by cp.async (compact operators only)
template <int NB, int ST, bool STG>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep_kernel(SweepArgs a) {
  using Gm = Geo<NB, ST>;
  constexpr int kStages = Gm::kStages, kBufs = Gm::kBufs;
  const int N = a.N;
  const int KT = 2 * N / 64, RT = N / 128, TNB = N / NB;
  const int64_t total = a.steps * a.chains * (int64_t)(RT * 2 * TNB);
  const size_t sb = state_bytes(N);
  const int TW = trace_warps(N);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* ring = smem;
  float* trace_rows = reinterpret_cast<float*>(smem + Gm::kRing);      // general trace path
  uint8_t* trace_stage = smem + Gm::kRing;                               // staged path
  uint8_t* ctrl = smem + Gm::kRing + (STG ? (size_t)TW * trace_stage_bytes(kTraceRows) : (size_t)TW * 16 * N);
  int4* uq = reinterpret_cast<int4*>(ctrl);                  // {ticket, entry, trace k, -}
  uint64_t* full = reinterpret_cast<uint64_t*>(ctrl + kQ * sizeof(int4));
  uint64_t* empty = full + kStages;
  uint64_t* mma_done = empty + kStages;
  uint64_t* tmem_empty = mma_done + kBufs;
  uint64_t* uq_full = tmem_empty + kBufs;
  uint64_t* uq_empty = uq_full + kQ;
  uint64_t* drain = uq_empty + kQ;
  uint64_t* pub_full = drain + 1;           // publisher mailboxes: two slots of a counter address
  uint64_t* pub_empty = pub_full + 2;       // (outputs) and two of a counter address and the
  uint64_t* pub_ptr = pub_empty + 2;        // count it has to reach first (traces)
  uint64_t* tpub_full = pub_ptr + 2;
  uint64_t* tpub_empty = tpub_full + 2;
  uint64_t* tpub_ptr = tpub_empty + 2;
  uint32_t* tpub_target = reinterpret_cast<uint32_t*>(tpub_ptr + 2);
  uint32_t* tmem_slot = tpub_target + 2;
  volatile int* abort_local = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&mma_done[b], 1);
      mbar_init(&tmem_empty[b], 4);
    }
    for (int i = 0; i < kQ; ++i) {
      mbar_init(&uq_full[i], 1);
      mbar_init(&uq_empty[i], 10);    // producer + MMA thread + 4 epilogue warps + 4 trace warps
    }
    mbar_init(drain, 1);
    for (int j = 0; j < 2; ++j) {
      mbar_init(&pub_full[j], 128);     // the epilogue's threads
      mbar_init(&pub_empty[j], 1);
      mbar_init(&tpub_full[j], 128);    // the trace warps' threads
      mbar_init(&tpub_empty[j], 1);
    }
    *abort_local = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&]() {
    *abort_local = 1;
    atomicExch(a.abort, 1);
  };

  if (warp == 11) {
    // ------------------------------------------------------------------ publisher
    // Makes each unit's outputs visible to the other CTAs: a release reduction on the unit's
    // row-block counter, which has to wait for the unit's stores to be performed, done here so
    // that the epilogue goes on to its next unit meanwhile.  The epilogue's threads arrive on
    // the slot's barrier after their stores (CTA-scope release), so this release covers them.
    if (lane == 0) {
      for (uint32_t k = 0;; ++k) {
        const uint32_t j = k & 1u;
        if (!wait_bar(&pub_full[j], (k >> 1) & 1u, abort_local, a.abort)) {
          fail();
          break;
        }
        const uint64_t ptr = pub_ptr[j];
        mbar_arrive(&pub_empty[j]);
        if (ptr == 0) break;
        if (!*abort_local) red_release_add(reinterpret_cast<uint32_t*>(ptr), 1u);
      }
    } else if (lane == 1 && a.trace) {
      // the trace warps' counters: a unit's slice of step t is counted only after every slice
      // of step t-1 of the same rows (so tcnt >= t * slices-per-step means steps < t are done)
      for (uint32_t k = 0;; ++k) {
        const uint32_t j = k & 1u;
        if (!wait_bar(&tpub_full[j], (k >> 1) & 1u, abort_local, a.abort)) {
          fail();
          break;
        }
        const uint64_t ptr = tpub_ptr[j];
        const uint32_t target = tpub_target[j];
        mbar_arrive(&tpub_empty[j]);
        if (ptr == 0) break;
        uint32_t* tc = reinterpret_cast<uint32_t*>(ptr);
        if (*abort_local) continue;
        if (target == 0 || wait_count(tc, target, a.abort))
          red_release_add(tc, 1u);
        else
          fail();
      }
    }
  } else if (warp == 10) {
    // ------------------------------------------------------------------ scheduler
    // Claims units in ticket (step) order, waits until the previous step of the unit's row
    // block is written, and queues it; up to kQ units run ahead of the stages below, so the
    // claim and the dependency wait of the next units overlap the current unit's copies.
    if (lane == 0) {
      uint32_t ui = 0;
      for (;;) {
        int32_t tk = -1, e = -1, trk = -1;
        if (!*abort_local && !ld_relaxed(a.abort)) {
          const uint32_t got = atomicAdd(a.ticket, 1u);
          if ((int64_t)got < total) tk = (int32_t)got;
        }
        if (tk >= 0) {
          const Unit u = decode(a, tk, RT, TNB);
          int k;
          bool last;
          e = (int32_t)factor_entry(a, u.c % a.gmod, u.t, k, last);
          if (a.trace && e >= 0 && last) trk = k;
          if (*abort_local || !wait_count(&a.cnt[u.c * RT + u.rt], (uint32_t)(u.t * 2 * TNB), a.abort)) {
            fail();
            tk = -1;
          }
        }
        const uint32_t slot = ui % kQ;
        if (ui >= kQ && !wait_bar(&uq_empty[slot], ((ui / kQ) - 1) & 1, abort_local, a.abort)) {
          fail();
          break;
        }
        uq[slot] = make_int4(tk, e, trk, 0);
        mbar_arrive(&uq_full[slot]);
        ++ui;
        if (tk < 0) break;
      }
    }
  } else if (warp == 4) {
    // ------------------------------------------------------------------ producer
    // Streams the state (A) and operand (B) tiles of the queued units through the ring,
    // one K tile of each per stage, back to back across units.
    if (lane == 0) {
      uint32_t kit = 0, ui = 0;
      for (;;) {
        const uint32_t slot = ui % kQ;
        if (!wait_bar(&uq_full[slot], (ui / kQ) & 1, abort_local, a.abort)) {
          fail();
          break;
        }
        const int4 m = uq[slot];
        mbar_arrive(&uq_empty[slot]);
        ++ui;
        if (m.x < 0) break;
        if (m.y < 0) continue;
        const Unit u = decode(a, m.x, RT, TNB);
        const uint8_t* Bb = a.planes + (size_t)m.y * entry_bytes(N) + (size_t)u.nb * KT * Gm::kB;
        // the states written by other CTAs (generic proxy) are read by bulk copies
        fence_proxy_async_global();
        const uint8_t* Sc = state_in(a, u.c, u.t, sb);
        bool ok = true;
        for (int kt = 0; kt < KT; ++kt, ++kit) {
          const uint32_t s = kit % kStages;
          uint8_t* dst = ring + s * Gm::kStage;
          if (kit >= (uint32_t)kStages &&
              !wait_bar(&empty[s], ((kit / kStages) - 1) & 1, abort_local, a.abort)) {
            fail();
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], Gm::kStage);
          bulk_load(dst + kTile, Bb + (size_t)kt * Gm::kB, Gm::kB, &full[s]);
          const int kta = u.h ? (kt + KT / 2) % KT : kt;
          bulk_load(dst, Sc + ((size_t)u.rt * KT + kta) * kTile, kTile, &full[s]);
        }
        if (!ok) break;
      }
      if (*abort_local) {
        // let the copies already issued land before the CTA leaves
        const uint32_t n = kit < (uint32_t)kStages ? kit : (uint32_t)kStages;
        for (uint32_t i = 0; i < n; ++i) {
          const uint32_t it = kit - 1 - i;
          mbar_wait_bounded_n(&full[it % kStages], (it / kStages) & 1, kLimit);
        }
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t kit = 0, ui = 0, use = 0;
      for (;;) {
        const uint32_t slot = ui % kQ;
        if (!wait_bar(&uq_full[slot], (ui / kQ) & 1, abort_local, a.abort)) {
          fail();
          break;
        }
        const int4 m = uq[slot];
        mbar_arrive(&uq_empty[slot]);
        ++ui;
        if (m.x < 0) break;
        if (m.y < 0) continue;
        const Unit u = decode(a, m.x, RT, TNB);
        const uint32_t b = use % kBufs;
        if (use >= (uint32_t)kBufs &&
            !wait_bar(&tmem_empty[b], ((use / kBufs) - 1) & 1, abort_local, a.abort)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + b * Gm::kAcc;
        bool ok = true;
        for (int kt = 0; kt < KT; ++kt, ++kit) {
          const uint32_t s = kit % kStages;
          if (!wait_bar(&full[s], (kit / kStages) & 1, abort_local, a.abort)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t neg = (u.h == 0 && kt >= KT / 2) ? kNegB : 0u;
          const uint32_t a_hi = smem_u32(ring + s * Gm::kStage);
          const uint32_t a_lo = a_hi + kHalf;
          const uint32_t b_hi = a_hi + kTile;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = (uint32_t)kk * 32u;
            const uint32_t first = (kt | kk) ? 1u : 0u;
            if (NB == 256) {
              const uint32_t b_lo = b_hi + NB * 128;
              mma_f16(d, smem_desc_sw128(a_hi + o), smem_desc_sw128(b_hi + o), kIdesc256 | neg, first);
              mma_f16(d + 256, smem_desc_sw128(a_hi + o), smem_desc_sw128(b_lo + o), kIdesc256 | neg, first);
              mma_f16(d + 256, smem_desc_sw128(a_lo + o), smem_desc_sw128(b_hi + o), kIdesc256 | neg, 1u);
            } else {
              // B rows 0..255 = hi then lo: D[0:128] = A_hi B_hi, D[128:256] = A_hi B_lo
              mma_f16(d, smem_desc_sw128(a_hi + o), smem_desc_sw128(b_hi + o), kIdesc256 | neg, first);
              mma_f16(d + 128, smem_desc_sw128(a_lo + o), smem_desc_sw128(b_hi + o), kIdesc128 | neg, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&mma_done[b]);
        ++use;
      }
      // nothing may be in flight in tensor memory when it is released
      mma_commit(drain);
      mbar_wait_bounded_n(drain, 0, kLimit);
    }
  } else if (warp < 4) {
    // ------------------------------------------------------------------ epilogue (warps 0-3)
    uint32_t ui = 0, use = 0, pubs = 0;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    // hand a counter address (0: no more) to the publisher through mailbox slot pubs & 1
    auto post = [&](uint32_t* cnt) {
      const uint32_t j = pubs & 1u;
      if (threadIdx.x == 0) {
        if (pubs >= 2 && !wait_bar(&pub_empty[j], ((pubs >> 1) - 1) & 1u, abort_local, a.abort)) fail();
        pub_ptr[j] = (uint64_t)(uintptr_t)cnt;
      }
      mbar_arrive(&pub_full[j]);
      ++pubs;
    };
    for (;;) {
      const uint32_t slot = ui % kQ;
      if (threadIdx.x == 0 && !wait_bar(&uq_full[slot], (ui / kQ) & 1, abort_local, a.abort)) fail();
      named_barrier(1, 128);
      if (*abort_local) break;
      const int4 m = uq[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&uq_empty[slot]);
      ++ui;
      if (m.x < 0) {
        post(nullptr);
        break;
      }
      const Unit u = decode(a, m.x, RT, TNB);
      const uint8_t* cur = state_in(a, u.c, u.t, sb);
      uint8_t* nxt = state_out(a, u.c, u.t, sb);
      if (a.trace && u.t > 0) {
        // the outputs overwrite the states of step t-1, which that step's traces read
        const uint32_t target = (uint32_t)(u.t * (a.vstore ? 2 : 4) * TNB);
        if (threadIdx.x == 0 && !wait_count(&a.tcnt[(u.c % a.gmod) * RT + u.rt], target, a.abort)) fail();
        named_barrier(1, 128);
      }
      const size_t region = ((size_t)u.rt * KT + (size_t)(u.h * N + u.nb * NB) / 64) * kTile;
      if (m.y < 0) {
        // past the end of its segment: carry the region over unchanged
        const uint4* src = reinterpret_cast<const uint4*>(cur + region);
        uint4* dst = reinterpret_cast<uint4*>(nxt + region);
        for (int i = threadIdx.x; i < (int)((NB / 64) * kTile / 16); i += 128) dst[i] = __ldcg(src + i);
      } else {
        const uint32_t b = use % kBufs;
        if (!wait_bar(&mma_done[b], (use / kBufs) & 1, abort_local, a.abort)) {
          fail();
        } else {
          tc_fence_after();
          const uint32_t d1 = tmem + lane_base + b * Gm::kAcc, d2 = d1 + NB;
          const int R = u.rt * 128 + 32 * warp + lane;
          uint8_t* out = nxt;
          const int kc0 = u.h * N + u.nb * NB;
#pragma unroll 1
          for (int ch = 0; ch < NB / 32; ch += 2) {
            uint32_t ra0[32], rb0[32], ra1[32], rb1[32];
            tmem_ld32(d1 + 32 * ch, ra0);
            tmem_ld32(d2 + 32 * ch, rb0);
            tmem_ld32(d1 + 32 * ch + 32, ra1);
            tmem_ld32(d2 + 32 * ch + 32, rb1);
            tmem_wait_ld();
            if (ch + 2 >= NB / 32) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&tmem_empty[b]);
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              const uint32_t* ra = half ? ra1 : ra0;
              const uint32_t* rb = half ? rb1 : rb0;
#pragma unroll
              for (int gq = 0; gq < 4; ++gq) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                  const int i0 = 8 * gq + 2 * p;
                  split_pair(fmaf(__uint_as_float(rb[i0]), kInv, __uint_as_float(ra[i0])),
                             fmaf(__uint_as_float(rb[i0 + 1]), kInv, __uint_as_float(ra[i0 + 1])), h[p], l[p]);
                }
                const uint32_t o = s_off(N, R, kc0 + 32 * (ch + half) + 8 * gq);
                *reinterpret_cast<uint4*>(out + o) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(out + o + kHalf) = make_uint4(l[0], l[1], l[2], l[3]);
              }
            }
          }
          ++use;
        }
      }
      // publish: this unit's part of step t+1 is written (by the publisher thread)
      fence_proxy_async_global();
      post(&a.cnt[u.c * RT + u.rt]);
    }
  } else {
    // ------------------------------------------------------------------ trace warps (6-9)
    const int tw = warp - 6;
    uint32_t ui = 0, tpubs = 0;
    auto tpost = [&](uint32_t* cnt, uint32_t target) {
      const uint32_t j = tpubs & 1u;
      if (threadIdx.x == 192) {
        if (tpubs >= 2 && !wait_bar(&tpub_empty[j], ((tpubs >> 1) - 1) & 1u, abort_local, a.abort)) fail();
        tpub_ptr[j] = (uint64_t)(uintptr_t)cnt;
        tpub_target[j] = target;
      }
      mbar_arrive(&tpub_full[j]);
      ++tpubs;
    };
    for (;;) {
      const uint32_t slot = ui % kQ;
      if (threadIdx.x == 192 && !wait_bar(&uq_full[slot], (ui / kQ) & 1, abort_local, a.abort)) fail();
      named_barrier(2, 128);
      if (*abort_local) break;
      const int4 m = uq[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&uq_empty[slot]);
      ++ui;
      if (m.x < 0) {
        if (a.trace) tpost(nullptr, 0);
        break;
      }
      if (!a.trace) continue;
      const Unit u = decode(a, m.x, RT, TNB);
      if (m.z >= 0 && !a.vstore) {
        // the partner chain's rows of step t are written too (this chain's are: the
        // producer waited for them before handing the unit out)
        const int64_t partner = u.c < a.gmod ? u.c + a.gmod : u.c - a.gmod;
        if (threadIdx.x == 192 && !wait_count(&a.cnt[partner * RT + u.rt], (uint32_t)(u.t * 2 * TNB), a.abort))
          fail();
        named_barrier(2, 128);
        if (*abort_local) break;
      }
      if (m.z >= 0 && tw < TW) {
        // this unit's rows of Tr(H_k V^dag R) at step t (V chain g, R chain gmod + g; or the
        // kept forward state of the same factor as conj(V) and R chain g)
        const uint8_t* cur = ((u.t & 1) ? a.buf1 : a.buf0);
        const int64_t g = u.c % a.gmod;
        const int li = (a.vstore || u.c < a.gmod ? 0 : 2 * TNB) + u.h * TNB + u.nb;
        const int rs = 128 / ((a.vstore ? 2 : 4) * TNB);
        const uint8_t* Vs = cur + g * sb;
        const uint8_t* Rs = cur + (a.gmod + g) * sb;
        if (a.vstore) {
          const int64_t f0 = (g % a.S) * a.seg_len;
          const int64_t f1 = f0 + a.seg_len < a.F ? f0 + a.seg_len : a.F;
          Vs = a.vstore + ((size_t)g * a.steps + (size_t)(f1 - f0 - 1 - u.t)) * sb;
          Rs = cur + g * sb;
        }
        const bool conjV = a.vstore != nullptr;
        float* vre = trace_rows + (size_t)tw * 4 * N;
        float* vim = vre + N;
        float* rre = vim + N;
        float* rim = rre + N;
        const int k = m.z;
        const int p0 = a.hk_ptr[k * (N + 1)], p1 = a.hk_ptr[k * (N + 1) + N];
        const int x0 = u.rt * 128 + li * rs + tw;
        const int nrows = (rs - tw + TW - 1) / TW;
        double sr = 0.0, si = 0.0;
        if (a.xval) {
          float tr = 0.0f, ti = 0.0f;
          const float2* hv = a.xval + (size_t)k * N;
          const int mk = a.xmask[k];
          if (STG)
            trace_xor_staged<kTraceRows>(Vs, Rs, N, x0, nrows, TW, mk, hv, lane, conjV, tr, ti,
                                         trace_stage + (size_t)tw * trace_stage_bytes(kTraceRows));
          else
            trace_xor(Vs, Rs, N, x0, nrows, TW, mk, hv, lane, conjV, tr, ti);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            tr += __shfl_xor_sync(0xffffffffu, tr, off);
            ti += __shfl_xor_sync(0xffffffffu, ti, off);
          }
          sr = (double)tr;
          si = (double)ti;
        } else switch (N) {
          case 128:
            trace_slice<1>(Vs, Rs, N, x0, nrows, TW, p0, p1, a.hk_row, a.hk_col, a.hk_val, vre, vim, rre, rim,
                           lane, conjV, sr, si);
            break;
          case 256:
            trace_slice<2>(Vs, Rs, N, x0, nrows, TW, p0, p1, a.hk_row, a.hk_col, a.hk_val, vre, vim, rre, rim,
                           lane, conjV, sr, si);
            break;
          case 512:
            trace_slice<4>(Vs, Rs, N, x0, nrows, TW, p0, p1, a.hk_row, a.hk_col, a.hk_val, vre, vim, rre, rim,
                           lane, conjV, sr, si);
            break;
          default:
            trace_slice<8>(Vs, Rs, N, x0, nrows, TW, p0, p1, a.hk_row, a.hk_col, a.hk_val, vre, vim, rre, rim,
                           lane, conjV, sr, si);
            break;
        }
        if (lane == 0) {
          double2* slot_acc = a.acc + g * a.seg_len + u.t;
          atomicAdd(&slot_acc->x, sr);
          atomicAdd(&slot_acc->y, si);
        }
      }
      // publish: this unit's reads of the step-t states are over (counted by the publisher
      // thread after every slice of step t-1 of these rows)
      tpost(&a.tcnt[(u.c % a.gmod) * RT + u.rt], (uint32_t)(u.t * (a.vstore ? 2 : 4) * TNB));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (*abort_local && threadIdx.x == 0 && a.status)
    atomicAdd((unsigned long long*)&a.status[REDO_STATUS_TIMEOUT], 1ull);
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// dF/du from the trace accumulators: one thread per (chain, sweep step)
__global__ void trace_finish_kernel(const double2* __restrict__ acc, int64_t G, int64_t S, int64_t seg_len,
                                    int64_t F, int K, int d, const double2* __restrict__ tau, double scale,
                                    int64_t M, double* __restrict__ grad) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= G * seg_len) return;
  const int64_t g = idx / seg_len, t = idx % seg_len;
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
  const double2 T = acc[idx];
  const double2 tu = tau[u];
  grad[(u * M + n) * K + k] = scale * (tu.x * T.y - tu.y * T.x);
}

static unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

static size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

// counters of a sweep: cnt [chains][N/128], tcnt [chains][N/128] (used up to gmod), ticket, abort
static size_t sync_words(int N, int64_t chains) { return 2 * (size_t)chains * (N / 128) + 2; }
static size_t sync_bytes(int N, int64_t chains) { return up(sync_words(N, chains) * sizeof(uint32_t)); }

// Runs `p.seg_len` steps of `chains` chains from b0; the result is in b0 (even count) or b1.
static cudaError_t sweep(const redo_table* t, const int32_t* q, const ChainPlan& p, int64_t chains,
                         int reverse, bool trace, const uint8_t* planes, uint8_t* b0, uint8_t* b1,
                         uint32_t* sync, double2* acc, int64_t* status, cudaStream_t s,
                         uint8_t* store = nullptr, const uint8_t* vstore = nullptr) {
  const int N = t->N, NB = t->tc_nb, RT = N / 128, TNB = N / NB;
  const int64_t total = p.seg_len * chains * (int64_t)(RT * 2 * TNB);
  if (total == 0) return cudaSuccess;
  if (total >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(sync, 0, sync_words(N, chains) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  SweepArgs a;
  a.buf0 = b0;
  a.buf1 = b1;
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
  a.chains = chains;
  a.gmod = (trace && !vstore) ? chains / 2 : chains;
  a.steps = p.seg_len;
  a.reverse = reverse;
  a.trace = trace ? 1 : 0;
  a.N = N;
  a.cnt = sync;
  a.tcnt = sync + (size_t)chains * RT;
  a.ticket = sync + 2 * (size_t)chains * RT;
  a.abort = reinterpret_cast<int*>(sync + 2 * (size_t)chains * RT + 1);
  a.hk_ptr = t->hk_ptr;
  a.hk_col = t->hk_col;
  a.hk_row = t->hk_row;
  a.hk_val = t->hk_val;
  a.xmask = t->hk_xmask;
  a.xval = t->hk_xval;
  a.acc = acc;
  a.status = status;
  a.store = store;
  a.vstore = vstore;
  // The gradient's reverse sweep with compact operators at N <= 256 stages its trace rows in
  // shared memory, taken from the operand ring (two stages instead of three): the traces, not
  // the MMAs, set its pace, and their loads need more bytes in flight than registers hold.
  const bool staged = trace && t->hk_xval && NB == 128 && N <= 256;
  const size_t smem = sweep_smem(NB, N, staged);
  int64_t grid = total < t->num_sms ? total : t->num_sms;
  if (NB == 256) {
    auto k = sweep_kernel<256, 2, false>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    k<<<(unsigned)grid, kSweepThreads, smem, s>>>(a);
  } else if (staged) {
    auto k = sweep_kernel<128, 2, true>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    k<<<(unsigned)grid, kSweepThreads, smem, s>>>(a);
  } else {
    auto k = sweep_kernel<128, 3, false>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    k<<<(unsigned)grid, kSweepThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace tcl

using namespace tcl;

// Operand block height, fixed when a table is built.  128 keeps two accumulator buffers
// in tensor memory (a unit's epilogue overlaps the next unit's MMAs) and gives twice the
// units per step, which pays while units are short (N = 256: K loop of 8 tiles); 256 has
// one buffer but a third less operand traffic per flop, which pays from N = 512 on.
// REDO_TCL_NB=128 or 256 overrides the choice.
int tc_large_nb(int N) {
  if (N < 256) return 128;
  const char* v = std::getenv("REDO_TCL_NB");
  if (v && std::strcmp(v, "128") == 0) return 128;
  if (v && std::strcmp(v, "256") == 0) return 256;
  return N >= 512 ? 256 : 128;
}

size_t tc_large_planes_bytes(const redo_table* t) { return 2 * (size_t)t->entries * entry_bytes(t->N); }

cudaError_t launch_build_tc_large_planes(const redo_table* t, cudaStream_t s) {
  const int NB = t->tc_nb;
  const int64_t tiles = t->entries * (t->N / NB) * (2 * t->N / 64);
  uint8_t* rows = (uint8_t*)t->tc_planes;
  uint8_t* cols = rows + (size_t)t->entries * entry_bytes(t->N);
  build_planes_kernel<<<(unsigned)tiles, 256, 0, s>>>(t->T64, t->N, NB, 0, rows);
  build_planes_kernel<<<(unsigned)tiles, 256, 0, s>>>(t->T64, t->N, NB, 1, cols);
  return cudaGetLastError();
}

size_t tc_large_prop_workspace(const redo_table* t, const ChainPlan& p, bool reunit) {
  const size_t G = (size_t)p.B * p.S;
  return large_prop_workspace(t, p, REDO_FP32, reunit) + 2 * up(G * state_bytes(t->N)) + sync_bytes(t->N, G);
}

// Segment products by tensor-core sweeps, then the FP32 re-unitarisation, combine and
// FP64 polar step of the SIMT large-N path.
cudaError_t tc_large_propagate(const redo_table* t, const int32_t* q, const ChainPlan& p, bool reunit,
                               void* ws, void** result, int* result_prec, int64_t* status,
                               cudaStream_t s) {
  const int N = t->N;
  const int64_t G = p.B * p.S;
  char* base = (char*)ws;
  const size_t simt = large_prop_workspace(t, p, REDO_FP32, reunit);
  uint8_t* st0 = (uint8_t*)(base + simt);
  uint8_t* st1 = st0 + up((size_t)G * state_bytes(N));
  uint32_t* sync = (uint32_t*)(st1 + up((size_t)G * state_bytes(N)));
  s_identity_kernel<<<blocks_for(G * N * (2 * N / 8)), 256, 0, s>>>(st0, N, G);
  cudaError_t e = sweep(t, q, p, G, 0, false, (const uint8_t*)t->tc_planes, st0, st1, sync, nullptr, status, s);
  if (e != cudaSuccess) return e;
  const uint8_t* res = (p.seg_len & 1) ? st1 : st0;
  // segment products X = Y^T into the SIMT path's segment buffer (its first region)
  float2* seg = (float2*)base;
  s_to_complex_kernel<float><<<blocks_for(G * (int64_t)N * N), 256, 0, s>>>(res, N, G, 0, seg, state_bytes(N));
  return large_finish_fp32(t, p, reunit, ws, result, result_prec, s);
}

// The forward sweep runs on two half segments per checkpoint segment when the segments alone
// would leave SMs idle.
static ChainPlan forward_plan(const redo_table* t, const ChainPlan& p) {
  const int N = t->N;
  const int64_t units = p.B * p.S * (N / 128) * 2 * (N / t->tc_nb);
  ChainPlan pf = p;
  if (units < 3 * (int64_t)t->num_sms && p.seg_len % 2 == 0 && p.seg_len >= 2) {
    pf.seg_len = p.seg_len / 2;
    pf.S = 2 * p.S;
  }
  return pf;
}

// Every forward state kept (chains x steps states; one per factor of every pulse) when they
// fit in kKeepBytes: the reverse sweep then needs no V chains (half its products).
// REDO_TCL_KEEP=0 selects the V/R form.
constexpr size_t kKeepBytes = (size_t)24 << 30;

static bool keep_states(const redo_table* t, const ChainPlan& pf) {
  const char* v = std::getenv("REDO_TCL_KEEP");
  if (v && v[0] == '0') return false;
  return (size_t)pf.B * pf.S * pf.seg_len * state_bytes(t->N) <= kKeepBytes;
}

size_t tc_large_grad_workspace(const redo_table* t, const ChainPlan& p) {
  const ChainPlan pf = forward_plan(t, p);
  if (keep_states(t, pf)) {
    const size_t G = (size_t)p.B * p.S, Gf = (size_t)pf.B * pf.S, n2 = (size_t)t->N * t->N;
    // SIMT layout over the segments + 2 Gf states (ping-pong) + kept states + half-segment
    // products and costates (FP32, Gf each) + segment costates (G) + trace accumulators +
    // sweep counters
    return large_grad_workspace(t, p, REDO_FP32) + 2 * up(Gf * state_bytes(t->N)) +
           up(Gf * (size_t)pf.seg_len * state_bytes(t->N)) + 2 * up(Gf * n2 * sizeof(float2)) +
           up(G * n2 * sizeof(float2)) + up(Gf * (size_t)pf.seg_len * sizeof(double2)) + sync_bytes(t->N, Gf);
  }
  const size_t G = (size_t)p.B * p.S;
  // + 2 x 2G states (V and R, ping-pong) + trace accumulators + sweep counters
  return large_grad_workspace(t, p, REDO_FP32) + 4 * up(G * state_bytes(t->N)) +
         up(G * (size_t)p.seg_len * sizeof(double2)) + sync_bytes(t->N, 2 * G);
}

// Gradient with every forward state kept: forward sweep of the (half) segment chains writing
// each step's state to its own slot; the segment products (halves joined in pairs) go through
// the FP32 checkpoint/costate scans; every chain's costate is carried back by the product
// before it (the kept states start from the identity at the chain's start); a reverse sweep
// of R chains only then reads conj(V) = P^T for its traces from the kept states.
static cudaError_t tc_large_grad_keep(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                      const ChainPlan& pf, const double2* UT, int tb, double* F_out, double* grad,
                                      void* ws, int64_t* status, cudaStream_t s, bool reunit) {
  const int N = t->N;
  const int64_t G = p.B * p.S, Gf = pf.B * pf.S;
  const bool split = Gf != G;
  const int64_t n2 = (int64_t)N * N;
  const size_t sb = state_bytes(N);
  char* base = (char*)ws;
  const size_t simt = large_grad_workspace(t, p, REDO_FP32);
  uint8_t* s0 = (uint8_t*)(base + simt);
  uint8_t* s1 = s0 + up((size_t)Gf * sb);
  uint8_t* keep = s1 + up((size_t)Gf * sb);
  float2* halves = (float2*)(keep + up((size_t)Gf * pf.seg_len * sb));
  float2* chain_costates = (float2*)((char*)halves + up((size_t)Gf * n2 * sizeof(float2)));
  float2* seg_costates = (float2*)((char*)chain_costates + up((size_t)Gf * n2 * sizeof(float2)));
  double2* acc = (double2*)((char*)seg_costates + up((size_t)G * n2 * sizeof(float2)));
  uint32_t* sync = (uint32_t*)((char*)acc + up((size_t)Gf * pf.seg_len * sizeof(double2)));
  const uint8_t* rows = (const uint8_t*)t->tc_planes;
  const uint8_t* cols = rows + (size_t)t->entries * entry_bytes(N);
  float2* seg = (float2*)base;                 // the SIMT layout's segment region
  cudaError_t e;
  {
    ProfScope ps(8, s);
    s_identity_kernel<<<blocks_for(Gf * N * (2 * N / 8)), 256, 0, s>>>(s0, N, Gf);
    if ((e = sweep(t, q, pf, Gf, 0, false, rows, s0, s1, sync, nullptr, status, s, keep, nullptr))) return e;
    // chain products: each chain's last kept state (the identity when there are no steps)
    float2* prods = split ? halves : seg;
    if (pf.seg_len > 0)
      s_to_complex_kernel<float><<<blocks_for(Gf * n2), 256, 0, s>>>(keep + (size_t)(pf.seg_len - 1) * sb, N, Gf,
                                                                     0, prods, (size_t)pf.seg_len * sb);
    else
      s_to_complex_kernel<float><<<blocks_for(Gf * n2), 256, 0, s>>>(s0, N, Gf, 0, prods, sb);
    if (split && (e = large_pair_products_fp32(halves, seg, G, N, s))) return e;
    if (reunit && p.M > 0 && (e = large_reunit_segments_fp32(t, p, ws, s))) return e;
  }
  float2 *Pck = nullptr, *Rck = nullptr;
  double2* tau = nullptr;
  {
    ProfScope ps(9, s);
    if ((e = large_grad_scans_fp32(t, p, UT, tb, F_out, ws, &Pck, &Rck, &tau, s))) return e;
  }
  if (p.M == 0) return cudaGetLastError();
  ProfScope ps(10, s);
  if (split) {
    if ((e = large_costate_shift_fp32(Pck, Rck, seg_costates, G, p.S, N, s))) return e;
    if ((e = large_half_costates_fp32(halves, seg_costates, chain_costates, Gf, N, s))) return e;
  } else if ((e = large_costate_shift_fp32(Pck, Rck, chain_costates, G, p.S, N, s))) {
    return e;
  }
  s_from_complex_kernel<float><<<blocks_for(Gf * N * (N / 8)), 256, 0, s>>>(chain_costates, N, Gf, 2, s0);
  if ((e = cudaMemsetAsync(acc, 0, sizeof(double2) * Gf * pf.seg_len, s))) return e;
  if ((e = sweep(t, q, pf, Gf, 1, true, cols, s0, s1, sync, acc, status, s, nullptr, keep))) return e;
  const double scale = 2.0 * t->dt / ((double)N * (double)N);
  trace_finish_kernel<<<(unsigned)((Gf * pf.seg_len + 255) / 256), 256, 0, s>>>(
      acc, Gf, pf.S, pf.seg_len, pf.F, t->K, t->digits, tau, scale, pf.M, grad);
  return cudaGetLastError();
}

cudaError_t tc_large_grad(const redo_table* t, const int32_t* q, const ChainPlan& p, const double2* UT,
                          int tb, double* F_out, double* grad, void* ws, int64_t* status,
                          cudaStream_t s, bool reunit) {
  {
    const ChainPlan pf = forward_plan(t, p);
    if (keep_states(t, pf)) return tc_large_grad_keep(t, q, p, pf, UT, tb, F_out, grad, ws, status, s, reunit);
  }
  const int N = t->N;
  const int64_t G = p.B * p.S;
  const int64_t n2 = (int64_t)N * N;
  char* base = (char*)ws;
  const size_t simt = large_grad_workspace(t, p, REDO_FP32);
  const size_t sb = up((size_t)G * state_bytes(N));
  uint8_t* s0 = (uint8_t*)(base + simt);       // 2G states (V then R)
  uint8_t* s1 = s0 + 2 * sb;                   // ping
  double2* acc = (double2*)(s1 + 2 * sb);
  uint32_t* sync = (uint32_t*)((char*)acc + up(G * (size_t)p.seg_len * sizeof(double2)));
  const uint8_t* rows = (const uint8_t*)t->tc_planes;
  const uint8_t* cols = rows + (size_t)t->entries * entry_bytes(N);
  cudaError_t e;
  float2* seg = (float2*)base;                 // the SIMT layout's segment region
  {
    ProfScope ps(8, s);                        // forward segment products
    // With few segments the forward sweep alone cannot keep every SM busy: run it on two
    // half segments per checkpoint segment (the state buffers hold 2G chains) and join
    // each pair with one FP32 product.
    const ChainPlan pf = forward_plan(t, p);
    const bool split = pf.S != p.S;
    const int64_t Gf = pf.B * pf.S;
    s_identity_kernel<<<blocks_for(Gf * N * (2 * N / 8)), 256, 0, s>>>(s0, N, Gf);
    if ((e = sweep(t, q, pf, Gf, 0, false, rows, s0, s1, sync, nullptr, status, s))) return e;
    const uint8_t* fin = (pf.seg_len & 1) ? s1 : s0;
    if (split) {
      // the checkpoint and costate regions (2G matrices, unused until the scans) hold the halves
      float2* halves = (float2*)(base + up((size_t)G * n2 * sizeof(float2)));
      s_to_complex_kernel<float><<<blocks_for(Gf * n2), 256, 0, s>>>(fin, N, Gf, 0, halves, state_bytes(N));
      if ((e = large_pair_products_fp32(halves, seg, G, N, s))) return e;
    } else {
      s_to_complex_kernel<float><<<blocks_for(G * n2), 256, 0, s>>>(fin, N, G, 0, seg, state_bytes(N));
    }
    if (reunit && p.M > 0 && (e = large_reunit_segments_fp32(t, p, ws, s))) return e;
  }
  float2 *Pck = nullptr, *Rck = nullptr;
  double2* tau = nullptr;
  {
    ProfScope ps(9, s);
    if ((e = large_grad_scans_fp32(t, p, UT, tb, F_out, ws, &Pck, &Rck, &tau, s))) return e;
  }
  if (p.M == 0) return cudaGetLastError();
  ProfScope ps(10, s);
  // reverse sweep: chains [0, G) hold V = P^dag, [G, 2G) hold R; both right-multiplied by A_f
  s_from_complex_kernel<float><<<blocks_for(G * N * (N / 8)), 256, 0, s>>>(Pck, N, G, 1, s0);
  s_from_complex_kernel<float><<<blocks_for(G * N * (N / 8)), 256, 0, s>>>(Rck, N, G, 2, s0 + G * state_bytes(N));
  if ((e = cudaMemsetAsync(acc, 0, sizeof(double2) * G * p.seg_len, s))) return e;
  if ((e = sweep(t, q, p, 2 * G, 1, true, cols, s0, s1, sync, acc, status, s))) return e;
  const double scale = 2.0 * t->dt / ((double)N * (double)N);
  trace_finish_kernel<<<(unsigned)((G * p.seg_len + 255) / 256), 256, 0, s>>>(
      acc, G, p.S, p.seg_len, p.F, t->K, t->digits, tau, scale, p.M, grad);
  return cudaGetLastError();
}

}  // namespace redo
