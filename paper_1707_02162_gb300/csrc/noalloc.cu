// redo_propagate_noalloc: the propagation entry point for callers that cannot
// allocate device memory.  Its scratch lives in a fixed, file-scope device
// array instead of a caller- or library-allocated workspace.
#include <mutex>

#include "redo_internal.cuh"

namespace redo {

// Every GPU that loads libredo holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[REDO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.  The host-side
// symbol g_noalloc_scratch is only a stand-in and must never reach a kernel;
// the real address comes from cudaGetSymbolAddress, once per device.
static redo_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(REDO_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return REDO_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Symmetric-split tables: the pulse products are conjugated by the half drift,
// D_h (U_M ... U_1) D_h^dag, into B FP64 matrices (plus as many for the dense
// product's intermediate when H0 is not diagonal), as redo_propagate does.
static size_t strang_scratch(const redo_table* t, int64_t B) {
  if (!t->strang) return 0;
  const size_t m = up256((size_t)B * t->N * t->N * sizeof(double2));
  return t->h0_diagonal ? m : 2 * m;
}

static size_t scratch_need(const redo_table* t, const ChainPlan& p, int prec, int64_t B) {
  return up256(chain_workspace_bytes(t, p, prec)) + strang_scratch(t, B);
}

// Same segmented plan as the allocating path, with the number of segments per
// pulse lowered until segment products, pulse products and (symmetric split)
// the conjugated products fit the array.
static bool plan_fits(const redo_table* t, int64_t B, int64_t M, int prec, ChainPlan* out) {
  ChainPlan p = plan_chain(t, B, M, prec);
  while (scratch_need(t, p, prec, B) > (size_t)REDO_NOALLOC_SCRATCH_BYTES && p.S > 1) {
    int64_t S = p.S - 1;
    p.seg_len = p.F > 0 ? (p.F + S - 1) / S : 0;
    p.S = p.seg_len > 0 ? (p.F + p.seg_len - 1) / p.seg_len : 1;
  }
  *out = p;
  return scratch_need(t, p, prec, B) <= (size_t)REDO_NOALLOC_SCRATCH_BYTES;
}

}  // namespace redo

using namespace redo;

extern "C" redo_status redo_propagate_noalloc(const redo_table* t, const int32_t* q, int64_t B,
                                              int64_t M, redo_precision prec, void* U_out,
                                              const void* U_target, double* F_out, void* tau_out,
                                              int64_t* dev_status, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "redo_propagate_noalloc supports REDO_FP64 and REDO_FP32");
  if (t->N > kSmallN) return set_error(REDO_ERR_UNSUPPORTED, "redo_propagate_noalloc supports N <= 64");
  if (prec == REDO_FP32 && !t->T32)
    return set_error(REDO_ERR_INVALID, "REDO_FP32 needs a table built with REDO_TABLE_FP32");
  if (B == 0) return REDO_OK;
  if (M > 0 && !q) return set_error(REDO_ERR_INVALID, "q is NULL");
  if (U_target && !F_out && !tau_out)
    return set_error(REDO_ERR_INVALID, "U_target given without F_out or tau_out");
  if (!U_out && !U_target) return set_error(REDO_ERR_INVALID, "nothing to compute");
  ChainPlan p;
  if (!plan_fits(t, B, M, prec, &p))
    return set_error(REDO_ERR_INVALID,
                     "B=%lld pulses of N=%d need %zu scratch bytes; redo_propagate_noalloc holds "
                     "at most %zu (REDO_NOALLOC_SCRATCH_BYTES): use fewer pulses per call or "
                     "redo_propagate with a workspace",
                     (long long)B, t->N, scratch_need(t, p, prec, B),
                     (size_t)REDO_NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  redo_status st = scratch_for_current_device(&scratch);
  if (st != REDO_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t n2 = (size_t)t->N * t->N;
  char* seg = (char*)scratch;
  char* prod = seg + up256((size_t)p.B * p.S * n2 * el);
  cudaError_t e;
  if ((e = launch_chain_segments(t, q, p, prec, seg, dev_status, s)) != cudaSuccess)
    return cuda_error(e, "chain segments");
  if ((e = launch_chain_combine(t, p, prec, seg, prod, dev_status, s)) != cudaSuccess)
    return cuda_error(e, "chain combine");
  const void* fin = prod;
  int fin_prec = prec;
  if (t->strang) {
    // S_M ... S_1 = D_h (U_M ... U_1) D_h^dag, D_h = exp(-i dt/2 H0)
    char* sb = (char*)scratch + up256(chain_workspace_bytes(t, p, prec));
    const size_t m = up256((size_t)B * n2 * sizeof(double2));
    if ((e = launch_half_drift_conj(t, prec, prod, B, 0, (double2*)sb,
                                    t->h0_diagonal ? nullptr : (double2*)(sb + m), s)) != cudaSuccess)
      return cuda_error(e, "half-drift conjugation");
    fin = sb;
    fin_prec = REDO_FP64;
  }
  if ((e = launch_finalize(t, B, fin_prec, fin, U_out, (const double2*)U_target, F_out,
                           (double2*)tau_out, s)) != cudaSuccess)
    return cuda_error(e, "finalize");
  return REDO_OK;
}
