// Tensor-core (tcgen05) product chains for N = 64 in split-FP16 arithmetic.
// (Section II process 2, Eq. exp2prod, and the Section III chain, on the tensor cores.)
//
// One chain multiplies a segment of gathered table operators,
//     X <- A_f X,   f = f0 .. f0+len-1,
// kept on chip as Y = X^T so that the running state is the M-side operand:
//     Y <- Y A_f^T.
// With the real embedding of a complex product,
//     [Zr; Zi] = [[Yr, -Yi], [Yi, Yr]] [Cr; Ci],   C = A_f^T,
// one step is a real 128 x 64 x 128 product: the state operand (128 x 128)
// lives in shared memory, the table operand B^T (64 x 128, row n =
// [Re A_f[n,:], Im A_f[n,:]]) is streamed from the L2-resident table by bulk
// copies, and the accumulator D = [Zr; Zi] lives in tensor memory.  A table
// entry stores its hi and lo planes as one 128-row tile (rows 0-63 hi, 64-127
// lo), so  A_hi [B_hi; B_lo]^T  is a single N = 128 product.
//
// Split-FP16 arithmetic: every operand value v (|v| <= 1 for unitary
// factors) is held as hi = fp16(v) and lo = fp16((v - hi) * 2^11); a step
// accumulates  D1 = sum hi*hi'  and  D2 = sum (hi*lo' + lo*hi')  in FP32 and
// the epilogue forms Z = D1 + 2^-11 D2 (the lo*lo' term, ~2^-22 relative, is
// dropped).  Both operands of one MMA have the same type (fp16).  The
// accumulation shrinks the norm by ~3e-8 per product; redo_propagate's
// periodic re-unitarisation removes that drift.
//
// Warp roles per CTA (CH chains, EW epilogue warps per chain): warps
// 0..CH*EW-1 epilogue -- warp w serves TMEM lanes 32(w mod 4).. and, when
// EW = 8, one 32-column half of the accumulator -- then one bulk-copy
// producer warp and one MMA-issuing warp (two in the default three-block
// kernel).  Two chains per CTA let one chain's MMAs run while the other
// chain's epilogue rewrites its state.
// Every wait is bounded; a timeout sets REDO_STATUS_TIMEOUT and the CTA
// drains, frees its tensor memory and exits.
#include <cuda_fp16.h>
#include <cstdlib>

#include "redo_internal.cuh"
#include "device_sync.cuh"
#include "tcgen05.cuh"

namespace redo {
namespace tc {

constexpr int kN = 64;
constexpr uint32_t kTablePlane = 64 * 128 * 2;       // 16 KB: one 64 x 128 fp16 operand plane
constexpr uint32_t kEntryBytes = 2 * kTablePlane;    // hi + lo planes of one table operator
constexpr uint32_t kEntryAtom = 128 * 128;           // one 64-wide K column of the 128-row entry tile
constexpr uint32_t kStateAtom = 128 * 128;           // 16 KB: one 64-wide K column of the 128-row state
constexpr uint32_t kStatePlane = 2 * kStateAtom;     // 32 KB
constexpr uint32_t kStateBytes = 2 * kStatePlane;    // hi + lo
constexpr uint32_t kTcWaitLimit = 1u << 24;
constexpr float kLoScale = 2048.0f;                  // 2^11
constexpr float kLoInv = 1.0f / 2048.0f;

// --------------------------------------------------------------------------
// Table operand planes: entry e -> one 128 x 128 K-major swizzled tile whose
// rows 0-63 are hi(B^T) and rows 64-127 lo(B^T), B^T row n = [Re T_e[n,:], Im T_e[n,:]].
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) build_planes_kernel(const double2* __restrict__ T,
                                                           uint8_t* __restrict__ planes) {
  const int64_t e = blockIdx.x;
  const double2* Te = T + e * (kN * kN);
  uint8_t* tile = planes + e * kEntryBytes;
  // 64 rows x 16 granules of 8 elements
  for (int gi = threadIdx.x; gi < 64 * 16; gi += blockDim.x) {
    const int n = gi >> 4, g = gi & 15;
    uint32_t h[4], l[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      __half hh[2], ll[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = 8 * g + 2 * p + q;           // 0..127
        const double2 z = Te[n * kN + (k & 63)];
        const double v = k < 64 ? z.x : z.y;
        hh[q] = __double2half(v);
        ll[q] = __double2half((v - (double)__half2float(hh[q])) * 2048.0);
      }
      h[p] = pack_half2(hh[0], hh[1]);
      l[p] = pack_half2(ll[0], ll[1]);
    }
    *reinterpret_cast<uint4*>(tile + sw128(n, 8 * g, 128)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(tile + sw128(64 + n, 8 * g, 128)) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// --------------------------------------------------------------------------
// The chain kernel
// --------------------------------------------------------------------------
struct TcArgs {
  const uint8_t* planes;
  const int32_t* q;
  int64_t M;
  int K, d, base;
  int64_t levels;
  int64_t units, segs, seg_len, F;
  float2* out;
  int64_t* status;
  int64_t fps;                // factors per step (K * digits)
  // amplitude/phase calls: [units][M][64] diagonals P_n = Z_n^dag Z_{n-1} (FP32) that open every
  // step, applied by the epilogue of the step before (or as the initial state of a segment), else nullptr
  const float2* pd;
};

template <int CH, int EW, int STAGES>
struct TcLayout {
  static constexpr uint32_t kState = 0;
  static constexpr uint32_t kRing = CH * kStateBytes;
  static constexpr uint32_t kBars = kRing + STAGES * kEntryBytes;
  // full[STAGES], empty[STAGES], mma_done[CH], state_ready[CH]
  static constexpr uint32_t kMisc = kBars + (2 * STAGES + 2 * CH) * 8;
  static constexpr uint32_t kBytes = kMisc + 16;
  static constexpr uint32_t kAlloc = kBytes + 1024;   // slack for 1024-byte alignment
  static constexpr int kEpiThreads = 32 * EW;         // per chain
  static constexpr int kThreads = 32 * (EW * CH + 2);
  static constexpr int kCols = 128 / (EW / 4);        // accumulator columns per epilogue thread (x2 halves)
  static constexpr uint32_t kTmemCols = CH == 1 ? 128 : (CH == 2 ? 256 : 512);
  static_assert(EW == 4 || EW == 8, "4 or 8 epilogue warps per chain");
  static_assert(kAlloc <= 232448, "shared memory budget");
};

__device__ __forceinline__ int64_t tc_entry(const TcArgs& a, int64_t unit, int64_t f) {
  const int64_t n = f / a.fps;
  const int r = (int)(f - n * a.fps);
  const int k = r / a.d, j = r - k * a.d;
  int32_t qv = a.q[(unit * a.M + n) * a.K + k];
  if (qv < 0 || qv >= a.levels) {
    if (a.status) atomicAdd((unsigned long long*)&a.status[REDO_STATUS_BADINDEX], 1ull);
    qv = 0;
  }
  for (int i = 0; i < j; ++i) qv /= a.base;
  return (int64_t)(k * a.d + j) * a.base + qv % a.base;
}

// Split 8 consecutive accumulator values into hi / lo fp16 granules.
__device__ __forceinline__ void split8(const float* z, uint4& h, uint4& l) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float x0 = z[2 * p], x1 = z[2 * p + 1];
    const __half2 hh = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __floats2half2_rn((x0 - hf.x) * kLoScale, (x1 - hf.y) * kLoScale);
    hw[p] = *reinterpret_cast<const uint32_t*>(&hh);
    lw[p] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

template <int CH, int EW, int STAGES>
__global__ void __launch_bounds__(TcLayout<CH, EW, STAGES>::kThreads, 1)
chain_tc_kernel(TcArgs a) {
  using L = TcLayout<CH, EW, STAGES>;
  constexpr int HALVES = EW / 4;                  // column groups per TMEM lane quarter
  constexpr int COLS = 64 / HALVES;               // accumulator columns per epilogue thread
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBars);
  uint64_t* empty = full + STAGES;
  uint64_t* mma_done = empty + STAGES;
  uint64_t* state_ready = mma_done + CH;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = a.units * a.segs;
  int64_t len[CH], f0[CH], unit[CH];
  int64_t maxlen = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    len[c] = 0;
    f0[c] = 0;
    unit[c] = 0;
    if (g < G) {
      unit[c] = g / a.segs;
      f0[c] = (g % a.segs) * a.seg_len;
      int64_t f1 = f0[c] + a.seg_len;
      if (f1 > a.F) f1 = a.F;
      len[c] = f1 > f0[c] ? f1 - f0[c] : 0;
    }
    if (len[c] > maxlen) maxlen = len[c];
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int c = 0; c < CH; ++c) {
      mbar_init(&mma_done[c], 1);
      mbar_init(&state_ready[c], L::kEpiThreads);
    }
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, L::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < EW * CH) {
    // ------------------------------------------------------------ epilogue
    const int c = warp / EW;
    const int ew = warp % EW;
    const int quarter = ew & 3, half = ew >> 2;
    const int row = 32 * quarter + lane;                 // TMEM lane = state row, 0..127
    const int col0 = COLS * half;                        // first accumulator column of this thread
    uint8_t* st_hi = smem + L::kState + c * kStateBytes;
    uint8_t* st_lo = st_hi + kStatePlane;
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    float* out = g < G ? reinterpret_cast<float*>(a.out + g * (kN * kN)) : nullptr;
    const uint32_t d1 = tmem_base + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(c * 128);
    const uint32_t d2 = d1 + 64;
    const int mrow = row < 64 ? row + 64 : row - 64;     // mirror row of the embedding
    const uint32_t negmask = row < 64 ? 0u : 0x80008000u;
    const int m = row & 63, comp = row >> 6;
    if (len[c] == 0) {
      if (out)
        for (int n = col0; n < col0 + COLS; ++n)
          out[(n * kN + m) * 2 + comp] = (comp == 0 && n == m) ? 1.f : 0.f;
    } else {
      // initial state Y = I: embedded 128 x 128 identity, lo = 0; this thread
      // writes K granules [16*half/HALVES, ...) of its row
      for (int gi = 16 * half / HALVES; gi < 16 * (half + 1) / HALVES; ++gi) {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        const int k0 = 8 * gi;
        if (row >= k0 && row < k0 + 8) {
          const int p = (row - k0) >> 1, hp = (row - k0) & 1;
          w[p] = (uint32_t)0x3C00u << (16 * hp);         // fp16 1.0
        }
        const uint32_t off = sw128(row, k0, 128);
        *reinterpret_cast<uint4*>(st_hi + off) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(st_lo + off) = make_uint4(0u, 0u, 0u, 0u);
      }
      fence_proxy_async_smem();
      mbar_arrive(&state_ready[c]);
      for (int64_t t = 0; t < len[c]; ++t) {
        bool ok = !*abort_flag && mbar_wait_bounded_n(&mma_done[c], (uint32_t)(t & 1), kTcWaitLimit);
        ok = __all_sync(0xffffffffu, ok);                // keep the warp converged for tcgen05.ld
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const bool last = (t == len[c] - 1);
#pragma unroll
        for (int j = 0; j < COLS / 32; ++j) {
          const int cb = col0 + 32 * j;                  // 32 accumulator columns
          uint32_t ra[32], rb[32];
          tmem_ld32(d1 + cb, ra);
          tmem_ld32(d2 + cb, rb);
          tmem_wait_ld();
          float z[32];
#pragma unroll
          for (int i = 0; i < 32; ++i)
            z[i] = fmaf(__uint_as_float(rb[i]), kLoInv, __uint_as_float(ra[i]));
          if (!last) {
#pragma unroll
            for (int gq = 0; gq < 4; ++gq) {
              uint4 h, l;
              split8(z + 8 * gq, h, l);
              const uint32_t kcol = (uint32_t)(cb + 8 * gq);
              const uint32_t od = sw128((uint32_t)row, kcol, 128);
              const uint32_t om = sw128((uint32_t)mrow, 64u + kcol, 128);
              *reinterpret_cast<uint4*>(st_hi + od) = h;
              *reinterpret_cast<uint4*>(st_lo + od) = l;
              *reinterpret_cast<uint4*>(st_hi + om) =
                  make_uint4(h.x ^ negmask, h.y ^ negmask, h.z ^ negmask, h.w ^ negmask);
              *reinterpret_cast<uint4*>(st_lo + om) =
                  make_uint4(l.x ^ negmask, l.y ^ negmask, l.z ^ negmask, l.w ^ negmask);
            }
          } else if (out) {
            // row < 64 holds Re Y[row, :] = Re X[:, row]; row >= 64 holds Im X[:, row-64]
#pragma unroll
            for (int i = 0; i < 32; ++i) out[((cb + i) * kN + m) * 2 + comp] = z[i];
          }
        }
        if (!last) {
          fence_proxy_async_smem();
          tc_fence_before();
          mbar_arrive(&state_ready[c]);
        }
      }
    }
  } else if (warp == EW * CH) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t idx = 0;
      for (int64_t t = 0; t < maxlen && !*abort_flag; ++t) {
        for (int c = 0; c < CH; ++c) {
          if (t >= len[c]) continue;
          const uint32_t s = idx % STAGES, u = idx / STAGES;
          if (u > 0 && !mbar_wait_bounded_n(&empty[s], (u - 1) & 1, kTcWaitLimit)) {
            *abort_flag = 1;
            break;
          }
          const int64_t e = tc_entry(a, unit[c], f0[c] + t);
          uint8_t* dst = smem + L::kRing + s * kEntryBytes;
          const uint8_t* src = a.planes + e * kEntryBytes;
          mbar_arrive_expect_tx(&full[s], kEntryBytes);
          bulk_load(dst, src, kEntryBytes / 2, &full[s]);
          bulk_load(dst + kEntryBytes / 2, src + kEntryBytes / 2, kEntryBytes / 2, &full[s]);
          ++idx;
        }
      }
    }
  } else {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t idx = 0;
      for (int64_t t = 0; t < maxlen && !*abort_flag; ++t) {
        for (int c = 0; c < CH; ++c) {
          if (t >= len[c]) continue;
          const uint32_t s = idx % STAGES, u = idx / STAGES;
          if (!mbar_wait_bounded_n(&full[s], u & 1, kTcWaitLimit) ||
              !mbar_wait_bounded_n(&state_ready[c], (uint32_t)(t & 1), kTcWaitLimit)) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = smem_u32(smem + L::kState + c * kStateBytes);
          const uint32_t a_lo = a_hi + kStatePlane;
          const uint32_t b0 = smem_u32(smem + L::kRing + s * kEntryBytes);
          const uint32_t dd1 = tmem_base + (uint32_t)(c * 128);
          const uint32_t dd2 = dd1 + 64;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint32_t ko = (uint32_t)(kk >> 2) * kStateAtom + (uint32_t)(kk & 3) * 32u;
            const uint32_t bo = (uint32_t)(kk >> 2) * kEntryAtom + (uint32_t)(kk & 3) * 32u;
            const uint64_t ah = smem_desc_sw128(a_hi + ko), al = smem_desc_sw128(a_lo + ko);
            const uint64_t bb = smem_desc_sw128(b0 + bo);    // rows 0-63 hi, 64-127 lo
            // [D1 | D2] (+)= A_hi [B_hi; B_lo]^T ;  D2 += A_lo B_hi^T
            mma_f16(dd1, ah, bb, kIdesc128, kk > 0 ? 1u : 0u);
            mma_f16(dd2, al, bb, kIdesc64, 1u);
          }
          mma_commit(&empty[s]);
          mma_commit(&mma_done[c]);
          ++idx;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (*abort_flag && threadIdx.x == 0 && a.status)
    atomicAdd((unsigned long long*)&a.status[REDO_STATUS_TIMEOUT], 1ull);
  if (warp == 0) tmem_dealloc(tmem_base, L::kTmemCols);
}

// --------------------------------------------------------------------------
// Variant with the state operand in tensor memory.  Each chain owns 256 TMEM
// columns: A_hi (64 columns = 128 fp16 K values per lane), A_lo, D1, D2.  The
// MMA reads A from tensor memory and only the table operand from shared memory,
// which removes 64 KB of shared-memory reads per product.  Because row r of the
// embedded state needs the partner row r +- 64 of the accumulator (Re and Im
// parts of one state row sit 64 lanes apart), the epilogue swaps its split
// values with the partner thread through a small shared buffer (stored
// word-transposed, conflict-free) and writes both halves of its A row with
// tcgen05.st.
// --------------------------------------------------------------------------
template <int STAGES>
struct Tc2Layout {
  static constexpr int CH = 2, EW = 8;
  static constexpr uint32_t kRing = 0;
  static constexpr uint32_t kX = STAGES * kEntryBytes;                 // exchange: [CH][2 halves][32 words][128 rows]
  static constexpr uint32_t kXBytes = CH * 2 * 32 * 128 * 4;
  static constexpr uint32_t kBars = kX + kXBytes;
  // full[STAGES], empty[STAGES], mma_done[CH], state_ready[CH], xchg[CH]
  static constexpr uint32_t kMisc = kBars + (2 * STAGES + 3 * CH) * 8;
  static constexpr uint32_t kAlloc = kMisc + 16 + 1024;
  static constexpr int kThreads = 32 * (EW * CH + 2);
  static_assert(kAlloc <= 232448, "shared memory budget");
};

template <int STAGES>
__global__ void __launch_bounds__(Tc2Layout<STAGES>::kThreads, 1) chain_tc2_kernel(TcArgs a) {
  using L = Tc2Layout<STAGES>;
  constexpr int CH = L::CH, EW = L::EW;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint32_t* xbuf = reinterpret_cast<uint32_t*>(smem + L::kX);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBars);
  uint64_t* empty = full + STAGES;
  uint64_t* mma_done = empty + STAGES;
  uint64_t* state_ready = mma_done + CH;
  uint64_t* xchg = state_ready + CH;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = a.units * a.segs;
  int64_t len[CH], f0[CH], unit[CH];
  int64_t maxlen = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    len[c] = 0;
    f0[c] = 0;
    unit[c] = 0;
    if (g < G) {
      unit[c] = g / a.segs;
      f0[c] = (g % a.segs) * a.seg_len;
      int64_t f1 = f0[c] + a.seg_len;
      if (f1 > a.F) f1 = a.F;
      len[c] = f1 > f0[c] ? f1 - f0[c] : 0;
    }
    if (len[c] > maxlen) maxlen = len[c];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int c = 0; c < CH; ++c) {
      mbar_init(&mma_done[c], 1);
      mbar_init(&state_ready[c], 32 * EW);
      mbar_init(&xchg[c], 32 * EW);
    }
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < EW * CH) {
    const int c = warp / EW, ew = warp % EW;
    const int quarter = ew & 3, j = ew >> 2;                 // lanes 32*quarter.., columns 32j..
    const int r = 32 * quarter + lane;
    const int partner = r < 64 ? r + 64 : r - 64;
    const uint32_t negp = r < 64 ? 0x80008000u : 0u;         // partner half enters row r negated if r < 64
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const uint32_t base = tmem_base + lane_off + (uint32_t)(c * 256);
    const uint32_t a_hi = base, a_lo = base + 64, d1 = base + 128, d2 = base + 192;
    uint32_t* xw = xbuf + (size_t)(c * 2 + j) * 32 * 128;    // [32 words][128 rows]
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    float* out = g < G ? reinterpret_cast<float*>(a.out + g * (kN * kN)) : nullptr;
    const int m = r & 63, comp = r >> 6;
    if (len[c] == 0) {
      if (out)
        for (int n = 32 * j; n < 32 * j + 32; ++n) out[(n * kN + m) * 2 + comp] = (comp == 0 && n == m) ? 1.f : 0.f;
    } else {
      // Y = I: row r < 64 holds I[r,:] in K 0..63; row r >= 64 holds I[r-64,:] in K 64..127
      uint32_t own[16], oth[16], zero[16];
#pragma unroll
      for (int w = 0; w < 16; ++w) {
        own[w] = 0u;
        oth[w] = 0u;
        zero[w] = 0u;
      }
      const int col = r < 64 ? r : r - 64;                   // K position of the 1 within its half
      if (col >= 32 * j && col < 32 * j + 32) {
        const int e = col - 32 * j;
        (r < 64 ? own : oth)[e >> 1] = (uint32_t)0x3C00u << (16 * (e & 1));
      }
      tmem_st16(a_hi + 16 * j, own);
      tmem_st16(a_hi + 32 + 16 * j, oth);
      tmem_st16(a_lo + 16 * j, zero);
      tmem_st16(a_lo + 32 + 16 * j, zero);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&state_ready[c]);
      for (int64_t t = 0; t < len[c]; ++t) {
        bool ok = !*abort_flag && mbar_wait_bounded_n(&mma_done[c], (uint32_t)(t & 1), kTcWaitLimit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        uint32_t ra[32], rb[32];
        tmem_ld32(d1 + 32 * j, ra);
        tmem_ld32(d2 + 32 * j, rb);
        tmem_wait_ld();
        float z[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = fmaf(__uint_as_float(rb[i]), kLoInv, __uint_as_float(ra[i]));
        if (t == len[c] - 1) {
          if (out) {
#pragma unroll
            for (int i = 0; i < 32; ++i) out[((32 * j + i) * kN + m) * 2 + comp] = z[i];
          }
          break;
        }
        uint32_t hw[16], lw[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) {
          const __half2 hh = __floats2half2_rn(z[2 * p], z[2 * p + 1]);
          const float2 hf = __half22float2(hh);
          const __half2 ll = __floats2half2_rn((z[2 * p] - hf.x) * kLoScale, (z[2 * p + 1] - hf.y) * kLoScale);
          hw[p] = *reinterpret_cast<const uint32_t*>(&hh);
          lw[p] = *reinterpret_cast<const uint32_t*>(&ll);
        }
#pragma unroll
        for (int w = 0; w < 16; ++w) {
          xw[w * 128 + r] = hw[w];
          xw[(16 + w) * 128 + r] = lw[w];
        }
        // all 256 threads of the chain have published their halves (bounded wait, no hardware barrier)
        mbar_arrive(&xchg[c]);
        bool xok = mbar_wait_bounded_n(&xchg[c], (uint32_t)(t & 1), kTcWaitLimit);
        xok = __all_sync(0xffffffffu, xok);
        if (!xok) {
          *abort_flag = 1;
          break;
        }
#pragma unroll
        for (int w = 0; w < 16; ++w) {
          own[w] = xw[w * 128 + partner] ^ negp;
          oth[w] = xw[(16 + w) * 128 + partner] ^ negp;
        }
        tmem_st16(a_hi + 16 * j, hw);
        tmem_st16(a_lo + 16 * j, lw);
        tmem_st16(a_hi + 32 + 16 * j, own);
        tmem_st16(a_lo + 32 + 16 * j, oth);
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&state_ready[c]);
      }
    }
  } else if (warp == EW * CH) {
    if (lane == 0) {
      uint32_t idx = 0;
      for (int64_t t = 0; t < maxlen && !*abort_flag; ++t) {
        for (int c = 0; c < CH; ++c) {
          if (t >= len[c]) continue;
          const uint32_t s = idx % STAGES, u = idx / STAGES;
          if (u > 0 && !mbar_wait_bounded_n(&empty[s], (u - 1) & 1, kTcWaitLimit)) {
            *abort_flag = 1;
            break;
          }
          const int64_t e = tc_entry(a, unit[c], f0[c] + t);
          uint8_t* dst = smem + L::kRing + s * kEntryBytes;
          const uint8_t* src = a.planes + e * kEntryBytes;
          mbar_arrive_expect_tx(&full[s], kEntryBytes);
          bulk_load(dst, src, kEntryBytes / 2, &full[s]);
          bulk_load(dst + kEntryBytes / 2, src + kEntryBytes / 2, kEntryBytes / 2, &full[s]);
          ++idx;
        }
      }
    }
  } else {
    if (lane == 0) {
      uint32_t idx = 0;
      for (int64_t t = 0; t < maxlen && !*abort_flag; ++t) {
        for (int c = 0; c < CH; ++c) {
          if (t >= len[c]) continue;
          const uint32_t s = idx % STAGES, u = idx / STAGES;
          if (!mbar_wait_bounded_n(&full[s], u & 1, kTcWaitLimit) ||
              !mbar_wait_bounded_n(&state_ready[c], (uint32_t)(t & 1), kTcWaitLimit)) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t b0 = smem_u32(smem + L::kRing + s * kEntryBytes);
          const uint32_t base = tmem_base + (uint32_t)(c * 256);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint32_t bo = (uint32_t)(kk >> 2) * kEntryAtom + (uint32_t)(kk & 3) * 32u;
            const uint64_t bb = smem_desc_sw128(b0 + bo);
            mma_f16_tmem_a(base + 128, base + 8 * kk, bb, kIdesc128, kk > 0 ? 1u : 0u);
            mma_f16_tmem_a(base + 192, base + 64 + 8 * kk, bb, kIdesc64, 1u);
          }
          mma_commit(&empty[s]);
          mma_commit(&mma_done[c]);
          ++idx;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (*abort_flag && threadIdx.x == 0 && a.status)
    atomicAdd((unsigned long long*)&a.status[REDO_STATUS_TIMEOUT], 1ull);
  if (warp == 0) tmem_dealloc(tmem_base, 512);
}

// --------------------------------------------------------------------------
// Variant with a three-block state (the default): the embedding's four 64 x 64
// blocks hold only three distinct matrices, so the state operand is stored as 192
// rows [-Yi; Yr; Yi] x 64 K (48 KB for hi + lo instead of 64 KB) and each step
// runs two K halves:  D = [Yr; Yi] Cr (rows 64..191, table K atom 0)
//                   + [-Yi; Yr] Ci (rows 0..127, table K atom 1).
// The epilogue writes 48 KB of state per step instead of 64 KB, and the saved
// shared memory deepens the operand ring to four stages.  (A third chain per CTA
// fits as well, but with a two-stage ring it measured slower.)
//
// A single thread issues a tcgen05.mma only every ~80 cycles, more than the 48-64
// cycles these MMAs execute in, so each product's MMAs are split over two issuing
// threads: A_hi [B_hi; B_lo] (N = 128, into D1 | D2) and A_lo B_hi (N = 64, into a
// third accumulator D3, so the two threads never accumulate into the same columns);
// the epilogue forms Z = D1 + 2^-11 (D2 + D3).  Both threads take the two chains'
// products in the same stream order and commit each stage and each product once
// (the barriers count two arrivals).  The producer warp looks the table entries up
// 32 products at a time, a batch ahead of the copies it issues, so the level-index
// loads do not delay the operand stream.
// --------------------------------------------------------------------------
template <int CH, int STAGES>
struct Tc3Layout {
  static constexpr int EW = 8;
  static constexpr uint32_t kPlane = 192 * 128;          // 24 KB: 192 rows x 64 fp16
  static constexpr uint32_t kState = 2 * kPlane;         // hi + lo
  static constexpr uint32_t kRing = CH * kState;
  static constexpr uint32_t kBars = kRing + STAGES * kEntryBytes;
  static constexpr uint32_t kMisc = kBars + (2 * STAGES + 2 * CH) * 8;
  static constexpr uint32_t kPhase = kMisc + 16;         // per chain: the next step diagonal, 64 float2
  static constexpr uint32_t kAlloc = kPhase + CH * 64 * 8 + 1024;
  // warps: EW per chain (epilogue), one producer, two MMA issuers (hi and lo state planes)
  static constexpr int kThreads = 32 * (EW * CH + 3);
  static constexpr uint32_t kTmemPerChain = 192;         // D1 = hi.hi, D2 = hi.lo, D3 = lo.hi
  static_assert(kAlloc <= 232448, "shared memory budget");
  static_assert(CH * kTmemPerChain <= 512, "tensor memory budget");
  static_assert(CH == 2, "the operand stream interleaves exactly two chains");
};

// PH: amplitude/phase call (a.pd non-null), the step diagonals applied by the epilogue.
template <int CH, int STAGES, bool PH>
__global__ void __launch_bounds__(Tc3Layout<CH, STAGES>::kThreads, 1) chain_tc3_kernel(TcArgs a) {
  using L = Tc3Layout<CH, STAGES>;
  constexpr int EW = L::EW;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBars);
  uint64_t* empty = full + STAGES;
  uint64_t* mma_done = empty + STAGES;
  uint64_t* state_ready = mma_done + CH;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::kMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = a.units * a.segs;
  int64_t len[CH], f0[CH], unit[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    len[c] = 0;
    f0[c] = 0;
    unit[c] = 0;
    if (g < G) {
      unit[c] = g / a.segs;
      f0[c] = (g % a.segs) * a.seg_len;
      int64_t f1 = f0[c] + a.seg_len;
      if (f1 > a.F) f1 = a.F;
      len[c] = f1 > f0[c] ? f1 - f0[c] : 0;
    }
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 2);                             // both issuers commit
    }
    for (int c = 0; c < CH; ++c) {
      mbar_init(&mma_done[c], 2);
      mbar_init(&state_ready[c], 32 * EW);
    }
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < EW * CH) {
    const int c = warp / EW, ew = warp % EW;
    const int quarter = ew & 3, j = ew >> 2;
    const int r = 32 * quarter + lane;                     // accumulator row
    uint8_t* st_hi = smem + c * L::kState;
    uint8_t* st_lo = st_hi + L::kPlane;
    const int64_t g = (int64_t)blockIdx.x * CH + c;
    float* out = g < G ? reinterpret_cast<float*>(a.out + g * (kN * kN)) : nullptr;
    const uint32_t d1 = tmem_base + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(c * L::kTmemPerChain);
    const uint32_t d2 = d1 + 64, d3 = d1 + 128;
    const int m = r & 63, comp = r >> 6;
    // destinations: r < 64 (Zr row r) -> block 1 row 64+r ; r >= 64 (Zi row r-64) -> block 2
    // row 128+(r-64) and, negated, block 0 row r-64
    const int rowA = r < 64 ? 64 + r : 128 + (r - 64);
    const int rowB = r - 64;                               // used only when r >= 64
    // amplitude/phase calls: the row holding the other component of the same state entries
    const int rowP = r < 64 ? 128 + r : r;                 // Zi row m (block 2) / Zr row m (block 1)
    float2* ph = reinterpret_cast<float2*>(smem + L::kPhase) + c * 64;
    const int et = ew * 32 + lane;                         // thread index within the chain's epilogue
    const int64_t kd = a.fps;
    // split-store 16 accumulator columns cb.. of this thread's row (and its negated copy)
    auto store16 = [&](const float* z, int cb) {
#pragma unroll
      for (int gq = 0; gq < 2; ++gq) {
        uint4 hh, ll;
        split8(z + 8 * gq, hh, ll);
        const uint32_t kcol = (uint32_t)(cb + 8 * gq);
        const uint32_t oa = sw128((uint32_t)rowA, kcol, 192);
        *reinterpret_cast<uint4*>(st_hi + oa) = hh;
        *reinterpret_cast<uint4*>(st_lo + oa) = ll;
        if (r >= 64) {
          const uint32_t ob = sw128((uint32_t)rowB, kcol, 192);
          const uint32_t ng = 0x80008000u;
          *reinterpret_cast<uint4*>(st_hi + ob) = make_uint4(hh.x ^ ng, hh.y ^ ng, hh.z ^ ng, hh.w ^ ng);
          *reinterpret_cast<uint4*>(st_lo + ob) = make_uint4(ll.x ^ ng, ll.y ^ ng, ll.z ^ ng, ll.w ^ ng);
        }
      }
    };
    // the 16 stored (split) values of row `row`, columns cb..
    auto load16 = [&](int row, int cb, float* v) {
#pragma unroll
      for (int gq = 0; gq < 2; ++gq) {
        const uint32_t o = sw128((uint32_t)row, (uint32_t)(cb + 8 * gq), 192);
        const uint4 hh = *reinterpret_cast<const uint4*>(st_hi + o);
        const uint4 ll = *reinterpret_cast<const uint4*>(st_lo + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t hw = q == 0 ? hh.x : q == 1 ? hh.y : q == 2 ? hh.z : hh.w;
          const uint32_t lw = q == 0 ? ll.x : q == 1 ? ll.y : q == 2 ? ll.z : ll.w;
          const float h0 = __half2float(__ushort_as_half((unsigned short)(hw & 0xffffu)));
          const float h1 = __half2float(__ushort_as_half((unsigned short)(hw >> 16)));
          const float l0 = __half2float(__ushort_as_half((unsigned short)(lw & 0xffffu)));
          const float l1 = __half2float(__ushort_as_half((unsigned short)(lw >> 16)));
          v[8 * gq + 2 * q] = fmaf(l0, kLoInv, h0);
          v[8 * gq + 2 * q + 1] = fmaf(l1, kLoInv, h1);
        }
      }
    };
    if (len[c] == 0) {
      if (out)
        for (int n = 32 * j; n < 32 * j + 32; ++n) out[(n * kN + m) * 2 + comp] = (comp == 0 && n == m) ? 1.f : 0.f;
    } else {
      // Initial state Y = I, or the step diagonal P_n when the segment opens step n of an
      // amplitude/phase call (Y = X^T is diagonal either way): this thread sets its K columns
      // 32j..32j+31 of its rows, the diagonal entry (m, m) to its component of the value.
      double dv = comp == 0 ? 1.0 : 0.0;
      if (PH && f0[c] % kd == 0) {
        const float2 pv = a.pd[(unit[c] * a.M + f0[c] / kd) * kN + m];
        dv = comp == 0 ? pv.x : pv.y;
      }
      const __half dh = __double2half(dv);
      const __half dl = __double2half((dv - (double)__half2float(dh)) * 2048.0);
      for (int gi = 4 * j; gi < 4 * j + 4; ++gi) {
        const int k0 = 8 * gi;
        uint32_t wh[4] = {0u, 0u, 0u, 0u}, wl[4] = {0u, 0u, 0u, 0u};
        if (m >= k0 && m < k0 + 8) {
          const int p = (m - k0) >> 1, hp = (m - k0) & 1;
          wh[p] = (uint32_t)__half_as_ushort(dh) << (16 * hp);
          wl[p] = (uint32_t)__half_as_ushort(dl) << (16 * hp);
        }
        const uint32_t oa = sw128((uint32_t)rowA, (uint32_t)k0, 192);
        *reinterpret_cast<uint4*>(st_hi + oa) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4*>(st_lo + oa) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        if (r >= 64) {
          const uint32_t ob = sw128((uint32_t)rowB, (uint32_t)k0, 192);
          const uint32_t ng = 0x80008000u;
          *reinterpret_cast<uint4*>(st_hi + ob) = make_uint4(wh[0] ^ ng, wh[1] ^ ng, wh[2] ^ ng, wh[3] ^ ng);
          *reinterpret_cast<uint4*>(st_lo + ob) = make_uint4(wl[0] ^ ng, wl[1] ^ ng, wl[2] ^ ng, wl[3] ^ ng);
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&state_ready[c]);
      for (int64_t t = 0; t < len[c]; ++t) {
        const int64_t f = f0[c] + t;
        const bool last = (t == len[c] - 1);
        // amplitude/phase calls: the first product of a step (in this segment) stages the
        // diagonal that opens the next step, when that step starts inside the segment
        const bool stage_ph = PH && (t == 0 || f % kd == 0) && (f / kd + 1) * kd < f0[c] + len[c];
        const bool apply_ph = PH && !last && (f + 1) % kd == 0;
        float2 pv = make_float2(0.f, 0.f);
        if (stage_ph && et < 64) pv = a.pd[(unit[c] * a.M + f / kd + 1) * kN + et];
        bool ok = !*abort_flag && mbar_wait_bounded_n(&mma_done[c], (uint32_t)(t & 1), kTcWaitLimit);
        if (PH) {
          // the chain's epilogue warps meet at barriers below: they agree on every step
          if (stage_ph && et < 64) ph[et] = pv;
          ok = named_barrier_and(1 + c, 32 * EW, ok);
        } else {
          ok = __all_sync(0xffffffffu, ok);
        }
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cb = 32 * j + 16 * h;                  // 16 accumulator columns
          uint32_t ra[16], rb[16], rc[16];
          tmem_ld16(d1 + cb, ra);
          tmem_ld16(d2 + cb, rb);
          tmem_ld16(d3 + cb, rc);
          tmem_wait_ld();
          float z[16];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            z[i] = fmaf(__uint_as_float(rb[i]) + __uint_as_float(rc[i]), kLoInv, __uint_as_float(ra[i]));
          if (!last) {
            store16(z, cb);
          } else if (out) {
#pragma unroll
            for (int i = 0; i < 16; ++i) out[((cb + i) * kN + m) * 2 + comp] = z[i];
          }
        }
        if (apply_ph) {
          // Y <- Y P (column n scaled by p_n): each entry needs both components, which live in
          // TMEM lanes m and m + 64 (different warps), so the partners exchange them through the
          // state just written; every thread then rewrites its own rows.
          named_barrier(3 + c, 32 * EW);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cb = 32 * j + 16 * h;
            float zo[16], zp[16];
            load16(rowA, cb, zo);
            load16(rowP, cb, zp);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float2 pc = ph[cb + i];
              const float zr = comp == 0 ? zo[i] : zp[i], zi = comp == 0 ? zp[i] : zo[i];
              zo[i] = comp == 0 ? fmaf(zr, pc.x, -zi * pc.y) : fmaf(zr, pc.y, zi * pc.x);
            }
            named_barrier(3 + c, 32 * EW);               // both rows read before either is rewritten
            store16(zo, cb);
          }
        }
        if (!last) {
          fence_proxy_async_smem();
          tc_fence_before();
          mbar_arrive(&state_ready[c]);
        }
      }
    }
  } else if (warp == EW * CH) {
    // Producer: the warp's lanes look up the table entries of 32 consecutive products of the
    // stream at once (one level-index load each, issued a batch ahead), and lane 0 issues the
    // bulk copies in stream order.
    const uint32_t n0 = (uint32_t)len[0], n1 = (uint32_t)len[1];
    const uint32_t mn = n0 < n1 ? n0 : n1, total = n0 + n1;
    const uint32_t clong = n0 > n1 ? 0u : 1u;
    // stage 1 (a batch ahead): the level index and the operand slot k*d + j, digit j
    auto fetch = [&](uint32_t idx, int32_t& qv, int32_t& kd, int32_t& jd) {
      qv = 0;
      kd = 0;
      jd = 0;
      if (idx >= total) return;
      uint32_t t, c;
      if (idx < 2u * mn) {
        t = idx >> 1;
        c = idx & 1u;
      } else {
        t = idx - mn;
        c = clong;
      }
      const int64_t f = f0[c] + (int64_t)t;
      const int64_t n = f / a.fps;
      const int r = (int)(f - n * a.fps);
      const int kq = r / a.d;
      jd = r - kq * a.d;
      kd = r;
      qv = a.q[(unit[c] * a.M + n) * a.K + kq];
    };
    // stage 2 (after the current batch's copies are issued): the table entry
    auto entry = [&](int32_t qv, int32_t kd, int32_t jd) -> int64_t {
      if (qv < 0 || qv >= a.levels) {
        if (a.status) atomicAdd((unsigned long long*)&a.status[REDO_STATUS_BADINDEX], 1ull);
        qv = 0;
      }
      for (int i = 0; i < jd; ++i) qv /= a.base;
      return (int64_t)kd * a.base + qv % a.base;
    };
    int32_t qn, kn, jn;
    fetch((uint32_t)lane, qn, kn, jn);
    int64_t e_cur = (uint32_t)lane < total ? entry(qn, kn, jn) : 0;
    for (uint32_t i0 = 0; i0 < total && !*abort_flag; i0 += 32) {
      fetch(i0 + 32u + (uint32_t)lane, qn, kn, jn);
      const uint32_t nb = total - i0 < 32u ? total - i0 : 32u;
      int ok = 1;
      for (uint32_t i = 0; i < nb; ++i) {
        const int64_t ei = __shfl_sync(0xffffffffu, e_cur, (int)i);
        if (lane == 0 && ok) {
          const uint32_t id = i0 + i;
          const uint32_t s = id % STAGES, u = id / STAGES;
          if (u > 0 && !mbar_wait_bounded_n(&empty[s], (u - 1) & 1, kTcWaitLimit)) {
            *abort_flag = 1;
            ok = 0;
          } else {
            uint8_t* dst = smem + L::kRing + s * kEntryBytes;
            const uint8_t* src = a.planes + ei * kEntryBytes;
            mbar_arrive_expect_tx(&full[s], kEntryBytes);
            bulk_load(dst, src, kEntryBytes / 2, &full[s]);
            bulk_load(dst + kEntryBytes / 2, src + kEntryBytes / 2, kEntryBytes / 2, &full[s]);
          }
        }
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      e_cur = i0 + 32u + (uint32_t)lane < total ? entry(qn, kn, jn) : 0;
    }
  } else {
    // Two MMA-issuing threads share every product: `hi` issues A_hi [B_hi; B_lo] (N = 128, into
    // D1 | D2) and `lo` issues A_lo B_hi (N = 64, into D3); each commits the stage and the chain's
    // accumulators once, so both barriers complete when both halves of the product are done.
    // The two chains' products are taken in stream order (32-bit counters throughout).
    const bool hi = warp == EW * CH + 1;
    if (lane == 0) {
      const uint32_t n0 = (uint32_t)len[0], n1 = (uint32_t)len[1];
      const uint32_t mn = n0 < n1 ? n0 : n1, total = n0 + n1;
      const uint32_t clong = n0 > n1 ? 0u : 1u;
      const uint32_t st0 = smem_u32(smem) + (hi ? 0u : L::kPlane);
      const uint32_t ring = smem_u32(smem + L::kRing);
      const uint32_t dd0 = tmem_base + (hi ? 0u : 128u);
      const uint32_t idesc = hi ? kIdesc128 : kIdesc64;
      const uint64_t dst0 = smem_desc_sw128(st0), dring = smem_desc_sw128(ring);
      for (uint32_t idx = 0; idx < total; ++idx) {
        uint32_t t, c;
        if (idx < 2u * mn) {
          t = idx >> 1;
          c = idx & 1u;
        } else {
          t = idx - mn;
          c = clong;
        }
        const uint32_t s = idx % STAGES, par = (idx / STAGES) & 1u;
        if (!mbar_wait_bounded_n(&full[s], par, kTcWaitLimit) ||
            !mbar_wait_bounded_n(&state_ready[c], t & 1u, kTcWaitLimit)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t dd = dd0 + c * L::kTmemPerChain;
        const uint32_t a_pl = st0 + c * L::kState;
        const uint32_t b0 = ring + s * kEntryBytes;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t arow = h == 0 ? 64u * 128u : 0u;   // [Yr; Yi] for Cr, [-Yi; Yr] for Ci
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t ao = arow + (uint32_t)kk * 32u;
            const uint32_t bo = (uint32_t)h * kEntryAtom + (uint32_t)kk * 32u;
            mma_f16(dd, smem_desc_sw128(a_pl + ao), smem_desc_sw128(b0 + bo), idesc, (h | kk) ? 1u : 0u);
          }
        }
        mma_commit(&empty[s]);
        mma_commit(&mma_done[c]);
        if (*abort_flag) break;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (*abort_flag && threadIdx.x == 0 && a.status)
    atomicAdd((unsigned long long*)&a.status[REDO_STATUS_TIMEOUT], 1ull);
  if (warp == 0) tmem_dealloc(tmem_base, 512);
}

}  // namespace tc

// ============================================================================
// Host launchers
// ============================================================================
size_t tc_planes_bytes(const redo_table* t) { return (size_t)t->entries * tc::kEntryBytes; }

cudaError_t launch_build_tc_planes(const redo_table* t, cudaStream_t s) {
  if (t->N != tc::kN) return cudaErrorInvalidValue;
  tc::build_planes_kernel<<<(unsigned)t->entries, 256, 0, s>>>(t->T64, (uint8_t*)t->tc_planes);
  return cudaGetLastError();
}

constexpr int kTcChains = 2;
constexpr int kTcEpiWarps = 8;
constexpr int kTcStages = 3;

ChainPlan plan_chain_tc(const redo_table* t, int64_t B, int64_t M) {
  ChainPlan p;
  p.B = B;
  p.M = M;
  p.fps = (int64_t)t->K * t->digits;
  p.F = M * p.fps;
  const int64_t slots = (int64_t)t->num_sms * kTcChains;
  // pick the segment count minimising (waves x segment length) + combine cost
  int64_t bestS = 1;
  double best = 1e300;
  for (int64_t S = 1; S <= 256; ++S) {
    const int64_t seg_len = p.F > 0 ? (p.F + S - 1) / S : 0;
    if (S > 1 && seg_len < 64) break;
    const int64_t segs = seg_len > 0 ? (p.F + seg_len - 1) / seg_len : 1;
    const int64_t waves = (B * segs + slots - 1) / slots;
    const double cost = (double)waves * (double)seg_len + 8.0 * (double)segs;
    if (cost < best) {
      best = cost;
      bestS = S;
    }
  }
  p.seg_len = p.F > 0 ? (p.F + bestS - 1) / bestS : 0;
  p.S = p.seg_len > 0 ? (p.F + p.seg_len - 1) / p.seg_len : 1;
  return p;
}

// Which chain kernel runs (all exact alternatives):
//   3 (default) three-block state in shared memory, 2 chains, 4-stage ring,
//     two MMA issuers, batched operand lookups:                              33.0 ms
//     (one issuer and per-product lookups: 35.1 ms)
//   1 embedded state in shared memory, 2 chains, 3-stage ring:               37.3 ms
//   2 embedded state in tensor memory, 2 chains, 4-stage ring:               39.1 ms
// (GB300, 256 pulses x 2000 steps x 12 products).  Each chain's step is serial: MMAs,
// then the epilogue that rewrites the state; at 33.0 ms the default's operand stream
// reads the level table at ~0.9 of the measured HBM copy bandwidth.
static int tc_variant() {
  const char* v = getenv("REDO_TC_VARIANT");
  if (v && v[0] == '1') return 1;
  if (v && v[0] == '2') return 2;
  return 3;
}

constexpr int kTc3Chains = 2, kTc3Stages = 4;

cudaError_t launch_chain_tc(const redo_table* t, const int32_t* q, const ChainPlan& p,
                            void* seg_out, int64_t* status, cudaStream_t s) {
  // amplitude/phase calls run on the three-block kernel only (its epilogue applies the step diagonals)
  if (p.pd32 || tc_variant() == 3) {
    using L3 = tc::Tc3Layout<kTc3Chains, kTc3Stages>;
    auto kern3 = p.pd32 ? tc::chain_tc3_kernel<kTc3Chains, kTc3Stages, true>
                        : tc::chain_tc3_kernel<kTc3Chains, kTc3Stages, false>;
    cudaError_t e = cudaFuncSetAttribute(kern3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L3::kAlloc);
    if (e != cudaSuccess) return e;
    tc::TcArgs a{};
    a.planes = (const uint8_t*)t->tc_planes;
    a.q = q;
    a.M = p.M;
    a.K = t->K;
    a.d = t->digits;
    a.base = t->base;
    a.levels = t->levels;
    a.units = p.B;
    a.segs = p.S;
    a.seg_len = p.seg_len;
    a.F = p.F;
    a.out = (float2*)seg_out;
    a.status = status;
    a.fps = p.fps > 0 ? p.fps : (int64_t)t->K * t->digits;
    a.pd = p.pd32;
    const int64_t G = p.B * p.S;
    const int64_t blocks = (G + kTc3Chains - 1) / kTc3Chains;
    if (blocks == 0) return cudaSuccess;
    kern3<<<(unsigned)blocks, L3::kThreads, L3::kAlloc, s>>>(a);
    return cudaGetLastError();
  }
  if (tc_variant() == 2) {
    constexpr int ST = 4;
    using L2 = tc::Tc2Layout<ST>;
    auto kern2 = tc::chain_tc2_kernel<ST>;
    cudaError_t e = cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L2::kAlloc);
    if (e != cudaSuccess) return e;
    tc::TcArgs a{};
    a.planes = (const uint8_t*)t->tc_planes;
    a.q = q;
    a.M = p.M;
    a.K = t->K;
    a.d = t->digits;
    a.base = t->base;
    a.levels = t->levels;
    a.units = p.B;
    a.segs = p.S;
    a.seg_len = p.seg_len;
    a.F = p.F;
    a.out = (float2*)seg_out;
    a.status = status;
    a.fps = p.fps > 0 ? p.fps : (int64_t)t->K * t->digits;
    a.pd = p.pd32;
    const int64_t G = p.B * p.S;
    const int64_t blocks = (G + L2::CH - 1) / L2::CH;
    if (blocks == 0) return cudaSuccess;
    kern2<<<(unsigned)blocks, L2::kThreads, L2::kAlloc, s>>>(a);
    return cudaGetLastError();
  }
  using L = tc::TcLayout<kTcChains, kTcEpiWarps, kTcStages>;
  auto kern = tc::chain_tc_kernel<kTcChains, kTcEpiWarps, kTcStages>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::kAlloc);
  if (e != cudaSuccess) return e;
  tc::TcArgs a{};
  a.planes = (const uint8_t*)t->tc_planes;
  a.q = q;
  a.M = p.M;
  a.K = t->K;
  a.d = t->digits;
  a.base = t->base;
  a.levels = t->levels;
  a.units = p.B;
  a.segs = p.S;
  a.seg_len = p.seg_len;
  a.F = p.F;
  a.out = (float2*)seg_out;
  a.status = status;
  a.fps = p.fps > 0 ? p.fps : (int64_t)t->K * t->digits;
  const int64_t G = p.B * p.S;
  const int64_t blocks = (G + kTcChains - 1) / kTcChains;
  if (blocks == 0) return cudaSuccess;
  kern<<<(unsigned)blocks, L::kThreads, L::kAlloc, s>>>(a);
  return cudaGetLastError();
}

}  // namespace redo
