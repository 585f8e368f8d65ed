// Host side of the libredo C ABI: argument checks, table ownership, launch order.
// (Each entry point is declared with the passage it implements -- Sections II to IV -- in redo.h.)
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "redo_internal.cuh"

namespace redo {

static thread_local char g_err[512] = "";

redo_status set_error(redo_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

redo_status cuda_error(cudaError_t e, const char* what) {
  return set_error(REDO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Optional event timing of the library's own launches (benchmarks only)
// ---------------------------------------------------------------------------
struct ProfRecord {
  int phase;
  cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRecord> g_prof;

ProfScope::ProfScope(int ph, cudaStream_t st) : phase(-1), a(nullptr), b(nullptr), s(st) {
  if (!g_prof_on) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
  phase = ph;
  cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
  if (phase < 0) return;
  cudaEventRecord(b, s);
  g_prof.push_back(ProfRecord{phase, a, b});
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static redo_status check_hermitian(const std::vector<double>& h, int N, const char* name, int k) {
  double mx = 0.0, dev = 0.0;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      const double ar = h[2 * (i * N + j)], ai = h[2 * (i * N + j) + 1];
      const double br = h[2 * (j * N + i)], bi = h[2 * (j * N + i) + 1];
      mx = std::fmax(mx, std::hypot(ar, ai));
      dev = std::fmax(dev, std::hypot(ar - br, ai + bi));
      if (!std::isfinite(ar) || !std::isfinite(ai))
        return set_error(REDO_ERR_INVALID, "%s[%d] has a non-finite entry", name, k);
    }
  if (dev > 1e-12 * (mx > 0 ? mx : 1.0))
    return set_error(REDO_ERR_NOT_HERMITIAN, "%s[%d] is not Hermitian (max |H-H^dag| = %g)", name,
                     k, dev);
  return REDO_OK;
}

}  // namespace redo

using namespace redo;

extern "C" {

const char* redo_last_error(void) { return g_err; }

redo_status redo_profile_enable(int32_t enable) {
  g_prof_on = enable != 0;
  return REDO_OK;
}

redo_status redo_profile_read(double* ms_out, int64_t* launches_out, int32_t n) {
  if (n < 0 || n > REDO_PROFILE_PHASES) return set_error(REDO_ERR_INVALID, "n out of range");
  for (auto& r : g_prof) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess &&
        r.phase < n) {
      if (ms_out) ms_out[r.phase] += ms;
      if (launches_out) launches_out[r.phase] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  return REDO_OK;
}

redo_status redo_build_table(int32_t N, int32_t K, double dt, const void* H0, const void* Hk,
                             const double* lo, const double* hi, int32_t base, int32_t digits,
                             uint32_t flags, void* stream, redo_table** out) {
  if (!out) return set_error(REDO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!H0 || !Hk || !lo || !hi) return set_error(REDO_ERR_INVALID, "null input pointer");
  if (N < 2 || N > kMaxN || !is_pow2(N))
    return set_error(REDO_ERR_UNSUPPORTED, "N=%d: this build supports N in {2,4,...,1024}", N);
  if (K < 1 || K > kMaxK) return set_error(REDO_ERR_INVALID, "K=%d out of [1, %d]", K, kMaxK);
  if (!(dt > 0) || !std::isfinite(dt)) return set_error(REDO_ERR_INVALID, "dt must be > 0");
  if (base < 2 || digits < 1) return set_error(REDO_ERR_INVALID, "base >= 2 and digits >= 1");
  double lv = 1.0;
  for (int j = 0; j < digits; ++j) lv *= base;
  if (lv > (double)(1 << 24)) return set_error(REDO_ERR_INVALID, "base^digits > 2^24 levels");
  for (int k = 0; k < K; ++k)
    if (!(hi[k] > lo[k]) || !std::isfinite(lo[k]) || !std::isfinite(hi[k]))
      return set_error(REDO_ERR_INVALID, "term %d: need finite lo < hi", k);
  if ((flags & REDO_TABLE_FP16X3) && N != 64 && N < 128)
    return set_error(REDO_ERR_UNSUPPORTED, "REDO_TABLE_FP16X3 needs N = 64 or N >= 128");
  if ((flags & REDO_TABLE_LEVELS) &&
      (double)K * lv * (double)N * N * 16.0 > 200.0 * 1024 * 1024 * 1024)
    return set_error(REDO_ERR_INVALID, "level table above 200 GiB (K * levels * N^2 * 16 bytes)");
  cudaStream_t s = (cudaStream_t)stream;

  // Hermitian check on the host (one synchronous copy, build time only)
  const size_t n2 = (size_t)N * N;
  std::vector<double> h(2 * n2 * (K + 1));
  REDO_CUDA_TRY(cudaMemcpyAsync(h.data(), H0, 2 * n2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  REDO_CUDA_TRY(cudaMemcpyAsync(h.data() + 2 * n2, Hk, 2 * n2 * K * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
  REDO_CUDA_TRY(cudaStreamSynchronize(s));
  {
    std::vector<double> one(2 * n2);
    for (int k = -1; k < K; ++k) {
      std::memcpy(one.data(), h.data() + 2 * n2 * (k + 1), 2 * n2 * sizeof(double));
      redo_status st = check_hermitian(one, N, k < 0 ? "H0" : "Hk", k < 0 ? 0 : k);
      if (st != REDO_OK) return st;
    }
  }

  redo_table* t = (redo_table*)std::calloc(1, sizeof(redo_table));
  if (!t) return set_error(REDO_ERR_OOM, "host allocation failed");
  t->N = N;
  t->K = K;
  t->base = base;
  t->digits = digits;
  t->digit_base = base;
  t->digit_count = digits;
  t->levels = (int64_t)lv;
  t->entries = (int64_t)K * digits * base;
  t->dt = dt;
  t->build_stream = s;
  for (int k = 0; k < K; ++k) {
    t->lo[k] = lo[k];
    t->hi[k] = hi[k];
    t->delta[k] = (hi[k] - lo[k]) / (double)(t->levels - 1);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (t->num_sms <= 0) t->num_sms = 148;

  auto fail = [&](redo_status st) {
    redo_table_free(t);
    return st;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&t->d_lo, sizeof(double) * K)) != cudaSuccess ||
      (e = cudaMalloc(&t->d_delta, sizeof(double) * K)) != cudaSuccess ||
      (e = cudaMalloc(&t->T64, sizeof(double2) * n2 * t->entries)) != cudaSuccess ||
      (e = cudaMalloc(&t->D64, sizeof(double2) * n2)) != cudaSuccess)
    return fail(set_error(REDO_ERR_OOM, "table allocation: %s", cudaGetErrorString(e)));
  if (flags & REDO_TABLE_STRANG) {
    t->strang = 1;
    if ((e = cudaMalloc(&t->Dh64, sizeof(double2) * n2)) != cudaSuccess)
      return fail(set_error(REDO_ERR_OOM, "half drift allocation: %s", cudaGetErrorString(e)));
  }
  {
    // off-diagonal nonzeros of H0 (the commutation check of the amplitude/phase calls)
    std::vector<int32_t> pairs;
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c)
        if (r != c && (h[2 * (r * N + c)] != 0.0 || h[2 * (r * N + c) + 1] != 0.0)) {
          pairs.push_back(r);
          pairs.push_back(c);
        }
    t->h0_diagonal = pairs.empty() ? 1 : 0;
    t->h0_npairs = (int64_t)pairs.size() / 2;
    if (!pairs.empty()) {
      t->h0_pairs = (int32_t*)std::malloc(sizeof(int32_t) * pairs.size());
      if (!t->h0_pairs) return fail(set_error(REDO_ERR_OOM, "host allocation"));
      std::memcpy(t->h0_pairs, pairs.data(), sizeof(int32_t) * pairs.size());
    }
  }
  // one-nonzero-per-row operators (row r at column r ^ m_k, value h_k[r]) with H_k^2 = a_k^2 I:
  // their level operators have a closed form (Pauli strings)
  std::vector<int32_t> mono_m(K, 0);
  std::vector<double2> mono_h((size_t)K * N);
  std::vector<double> mono_a(K, 0.0);
  bool mono_involutory = false;
  {
    // sparse (CSR) copy of the control operators for the gradient traces Tr(H_k W)
    std::vector<int32_t> ptr((size_t)K * (N + 1)), col, rowi;
    std::vector<double2> val;
    for (int k = 0; k < K; ++k) {
      const double* hk = h.data() + 2 * n2 * (k + 1);
      for (int r = 0; r < N; ++r) {
        ptr[(size_t)k * (N + 1) + r] = (int32_t)col.size();
        for (int c = 0; c < N; ++c) {
          const double re = hk[2 * (r * N + c)], im = hk[2 * (r * N + c) + 1];
          if (re != 0.0 || im != 0.0) {
            col.push_back(c);
            rowi.push_back(r);
            val.push_back(make_double2(re, im));
          }
        }
      }
      ptr[(size_t)k * (N + 1) + N] = (int32_t)col.size();
    }
    t->hk_nnz = (int64_t)col.size();
    const size_t nz = col.empty() ? 1 : col.size();
    if ((e = cudaMalloc(&t->hk_ptr, sizeof(int32_t) * ptr.size())) != cudaSuccess ||
        (e = cudaMalloc(&t->hk_col, sizeof(int32_t) * nz)) != cudaSuccess ||
        (e = cudaMalloc(&t->hk_row, sizeof(int32_t) * nz)) != cudaSuccess ||
        (e = cudaMalloc(&t->hk_val, sizeof(double2) * nz)) != cudaSuccess)
      return fail(set_error(REDO_ERR_OOM, "operator CSR allocation: %s", cudaGetErrorString(e)));
    if ((e = cudaMemcpy(t->hk_ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice)) ||
        (!col.empty() &&
         ((e = cudaMemcpy(t->hk_col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice)) ||
          (e = cudaMemcpy(t->hk_row, rowi.data(), sizeof(int32_t) * rowi.size(), cudaMemcpyHostToDevice)) ||
          (e = cudaMemcpy(t->hk_val, val.data(), sizeof(double2) * val.size(), cudaMemcpyHostToDevice)))))
      return fail(cuda_error(e, "operator CSR upload"));
    // Operators with exactly one nonzero per row, at column r ^ m_k (every Pauli string:
    // X/Y flip bits, Z only sets phases) also get the compact form m_k, h_k[r] in FP32
    // that the tensor-core gradient's trace reads without gathering.
    bool mono = true;
    std::vector<int32_t>& xm = mono_m;
    std::vector<float2> xv((size_t)K * N);
    for (int k = 0; k < K && mono; ++k)
      for (int r = 0; r < N && mono; ++r) {
        const size_t a = (size_t)k * (N + 1) + r;
        if (ptr[a + 1] - ptr[a] != 1) {
          mono = false;
          break;
        }
        const int m = col[ptr[a]] ^ r;
        if (r == 0) xm[k] = m;
        if (m != xm[k]) mono = false;
        mono_h[(size_t)k * N + r] = val[ptr[a]];
        xv[(size_t)k * N + r] = make_float2((float)val[ptr[a]].x, (float)val[ptr[a]].y);
      }
    if (mono) {
      // H_k^2 is diagonal with entries h_r h_{r ^ m}; involutory up to scale when they all equal a^2 > 0
      mono_involutory = true;
      for (int k = 0; k < K && mono_involutory; ++k) {
        const double2* h = mono_h.data() + (size_t)k * N;
        const double2 p0 = h[0], p1 = h[xm[k]];
        const double a2 = p0.x * p1.x - p0.y * p1.y;
        if (!(a2 > 0.0)) mono_involutory = false;
        for (int r = 0; r < N && mono_involutory; ++r) {
          const double2 x = h[r], y = h[r ^ xm[k]];
          const double re = x.x * y.x - x.y * y.y, im = x.x * y.y + x.y * y.x;
          if (std::fabs(re - a2) > 1e-14 * a2 || std::fabs(im) > 1e-14 * a2) mono_involutory = false;
        }
        mono_a[k] = std::sqrt(a2);
      }
    }
    const bool xr = mono && N > kSmallN;
    if (xr) {
      if ((e = cudaMalloc(&t->hk_xmask, sizeof(int32_t) * K)) != cudaSuccess ||
          (e = cudaMalloc(&t->hk_xval, sizeof(float2) * K * N)) != cudaSuccess)
        return fail(set_error(REDO_ERR_OOM, "operator allocation: %s", cudaGetErrorString(e)));
      if ((e = cudaMemcpy(t->hk_xmask, xm.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice)) ||
          (e = cudaMemcpy(t->hk_xval, xv.data(), sizeof(float2) * K * N, cudaMemcpyHostToDevice)))
        return fail(cuda_error(e, "operator upload"));
    }
  }
  if ((flags & (REDO_TABLE_FP32 | REDO_TABLE_FP16X3)) &&
      (e = cudaMalloc(&t->T32, sizeof(float2) * n2 * t->entries)) != cudaSuccess)
    return fail(set_error(REDO_ERR_OOM, "FP32 table allocation: %s", cudaGetErrorString(e)));
  if ((e = cudaMemcpyAsync(t->d_lo, t->lo, sizeof(double) * K, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(t->d_delta, t->delta, sizeof(double) * K, cudaMemcpyHostToDevice, s)))
    return fail(cuda_error(e, "copy lo/delta"));
  if (N <= kSmallN) {
    if ((e = launch_table_expm(t, (const double2*)H0, (const double2*)Hk, s)) != cudaSuccess)
      return fail(cuda_error(e, "table exponentials"));
    if ((e = launch_table_fold_drift(t, s)) != cudaSuccess)
      return fail(cuda_error(e, "drift fold"));
  } else {
    // 1-norms (max column sum) of the generators bound the Taylor scaling
    std::vector<double> hn(K);
    double h0n = 0.0;
    for (int k = -1; k < K; ++k) {
      const double* hk = h.data() + 2 * n2 * (k + 1);
      double mx = 0.0;
      for (int c = 0; c < N; ++c) {
        double sum = 0.0;
        for (int r = 0; r < N; ++r) sum += std::hypot(hk[2 * (r * N + c)], hk[2 * (r * N + c) + 1]);
        mx = std::fmax(mx, sum);
      }
      if (k < 0) h0n = mx; else hn[k] = mx;
    }
    if ((e = large_table_build(t, (const double2*)H0, (const double2*)Hk, hn, h0n, s)) != cudaSuccess)
      return fail(cuda_error(e, "large-N table"));
  }
  if (flags & REDO_TABLE_LEVELS) {
    // process 3: evaluate each level's operator once as the product of its digit operators
    double2* E = nullptr;
    const int64_t ne = (int64_t)K * t->levels;
    if ((e = cudaMalloc(&E, sizeof(double2) * n2 * ne)) != cudaSuccess)
      return fail(set_error(REDO_ERR_OOM, "level table allocation: %s", cudaGetErrorString(e)));
    if (mono_involutory && t->h0_diagonal) {
      // every level's operator in closed form (equal to the digit product up to rounding)
      int32_t* d_m = nullptr;
      double2* d_h = nullptr;
      double* d_a = nullptr;
      e = cudaMalloc(&d_m, sizeof(int32_t) * K);
      if (e == cudaSuccess) e = cudaMalloc(&d_h, sizeof(double2) * K * N);
      if (e == cudaSuccess) e = cudaMalloc(&d_a, sizeof(double) * K);
      if (e == cudaSuccess) e = cudaMemcpy(d_m, mono_m.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(d_h, mono_h.data(), sizeof(double2) * K * N, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(d_a, mono_a.data(), sizeof(double) * K, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = launch_levels_closed_form(t, d_m, d_h, d_a, E, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(d_m);
      cudaFree(d_h);
      cudaFree(d_a);
    } else {
      e = N > kSmallN ? large_table_expand(t, E, s) : launch_table_expand(t, E, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
      cudaFree(E);
      return fail(cuda_error(e, "level table"));
    }
    cudaFree(t->T64);
    t->T64 = E;
    t->entries = ne;
    t->base = (int32_t)t->levels;
    t->digits = 1;
    if (t->T32) {
      cudaFree(t->T32);
      t->T32 = nullptr;
      if ((e = cudaMalloc(&t->T32, sizeof(float2) * n2 * ne)) != cudaSuccess)
        return fail(set_error(REDO_ERR_OOM, "FP32 level table allocation: %s", cudaGetErrorString(e)));
    }
  }
  if (t->T32 && (e = launch_to_fp32(t->T64, t->T32, (int64_t)n2 * t->entries, s)) != cudaSuccess)
    return fail(cuda_error(e, "FP32 copy"));
  if (flags & REDO_TABLE_FP16X3) {
    t->tc_nb = N > kSmallN ? tc_large_nb(N) : 0;
    t->tc_bytes = N > kSmallN ? tc_large_planes_bytes(t) : tc_planes_bytes(t);
    if ((e = cudaMalloc(&t->tc_planes, t->tc_bytes)) != cudaSuccess)
      return fail(set_error(REDO_ERR_OOM, "FP16x3 planes allocation: %s", cudaGetErrorString(e)));
    e = N > kSmallN ? launch_build_tc_large_planes(t, s) : launch_build_tc_planes(t, s);
    if (e != cudaSuccess) return fail(cuda_error(e, "FP16x3 planes"));
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_error(e, "table build"));
  *out = t;
  return REDO_OK;
}

redo_status redo_table_free(redo_table* t) {
  if (!t) return REDO_OK;
  if (t->build_stream) cudaStreamSynchronize(t->build_stream);
  cudaFree(t->d_lo);
  cudaFree(t->d_delta);
  cudaFree(t->T64);
  cudaFree(t->D64);
  cudaFree(t->Dh64);
  cudaFree(t->T32);
  cudaFree(t->tc_planes);
  cudaFree(t->hk_ptr);
  cudaFree(t->hk_col);
  cudaFree(t->hk_row);
  cudaFree(t->hk_val);
  cudaFree(t->hk_xmask);
  cudaFree(t->hk_xval);
  cudaFree(t->sz64);
  std::free(t->h0_pairs);
  std::free(t);
  return REDO_OK;
}

redo_status redo_table_set_phase_axes(redo_table* t, const double* sz) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (!sz) return set_error(REDO_ERR_INVALID, "sz is NULL");
  const int N = t->N, K = t->K;
  for (int64_t i = 0; i < (int64_t)K * N; ++i)
    if (!std::isfinite(sz[i])) return set_error(REDO_ERR_INVALID, "sz[%lld] is not finite", (long long)i);
  // Z_n commutes with the drift (Section III): H0[a][b] != 0 needs sz[k][a] == sz[k][b]
  for (int64_t e = 0; e < t->h0_npairs; ++e) {
    const int a = t->h0_pairs[2 * e], b = t->h0_pairs[2 * e + 1];
    for (int k = 0; k < K; ++k)
      if (sz[(int64_t)k * N + a] != sz[(int64_t)k * N + b])
        return set_error(REDO_ERR_UNSUPPORTED, "S_z of term %d does not commute with H0 (entry %d, %d)", k, a, b);
  }
  if (!t->sz64) {
    cudaError_t e = cudaMalloc(&t->sz64, sizeof(double) * K * N);
    if (e != cudaSuccess) {
      t->sz64 = nullptr;
      return set_error(REDO_ERR_OOM, "phase axes: %s", cudaGetErrorString(e));
    }
  }
  REDO_CUDA_TRY(cudaMemcpy(t->sz64, sz, sizeof(double) * K * N, cudaMemcpyHostToDevice));
  return REDO_OK;
}

redo_status redo_table_info(const redo_table* t, int32_t* N, int32_t* K, int32_t* base,
                            int32_t* digits, int64_t* levels, int64_t* entries) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (N) *N = t->N;
  if (K) *K = t->K;
  if (base) *base = t->base;
  if (digits) *digits = t->digits;
  if (levels) *levels = t->levels;
  if (entries) *entries = t->entries;
  return REDO_OK;
}

redo_status redo_table_copy(const redo_table* t, void* table_out, void* drift_out, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  const size_t n2 = (size_t)t->N * t->N;
  cudaStream_t s = (cudaStream_t)stream;
  if (table_out)
    REDO_CUDA_TRY(cudaMemcpyAsync(table_out, t->T64, sizeof(double2) * n2 * t->entries,
                                  cudaMemcpyDeviceToDevice, s));
  if (drift_out)
    REDO_CUDA_TRY(
        cudaMemcpyAsync(drift_out, t->D64, sizeof(double2) * n2, cudaMemcpyDeviceToDevice, s));
  return REDO_OK;
}

redo_status redo_quantize(const redo_table* t, const double* u, int64_t B, int64_t M, int32_t* q,
                          int64_t* dev_status, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  const int64_t count = B * M * t->K;
  if (count == 0) return REDO_OK;
  if (!u || !q) return set_error(REDO_ERR_INVALID, "null u or q");
  ProfScope ps(0, (cudaStream_t)stream);
  cudaError_t e = launch_quantize(u, count, t->K, t->d_lo, t->d_delta, t->levels, q, dev_status,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "quantize");
  return REDO_OK;
}

static redo_status check_prec(const redo_table* t, redo_precision prec) {
  if (prec == REDO_FP64) return REDO_OK;
  if (prec == REDO_FP32) {
    if (!t->T32) return set_error(REDO_ERR_INVALID, "REDO_FP32 needs a table built with REDO_TABLE_FP32");
    return REDO_OK;
  }
  if (prec == REDO_FP16X3) {
    if (!t->tc_planes)
      return set_error(REDO_ERR_INVALID, "REDO_FP16X3 needs a table built with REDO_TABLE_FP16X3");
    return REDO_OK;
  }
  return set_error(REDO_ERR_INVALID, "unknown precision %d", (int)prec);
}

// Plan and workspace layout shared by redo_propagate and redo_propagate_workspace.
struct PropLayout {
  ChainPlan p;
  int eff_prec;       // precision of segment and pulse products
  size_t seg_off, prod_off, prod64_off, total;
  size_t strang_off, strang_tmp_off;   // symmetric split: conjugated products (+ dense-drift scratch)
  size_t pd_off, zf_off, phout_off;     // amplitude/phase calls
};

// FP64 matrices appended to a workspace for the symmetric split's conjugation
static size_t strang_bytes(const redo_table* t, int64_t count) {
  if (!t->strang) return 0;
  const size_t m = ((size_t)count * t->N * t->N * sizeof(double2) + 255) & ~(size_t)255;
  return t->h0_diagonal ? m : 2 * m;
}

static void add_strang(const redo_table* t, int64_t count, size_t& total, size_t& off, size_t& tmp_off) {
  const size_t m = ((size_t)count * t->N * t->N * sizeof(double2) + 255) & ~(size_t)255;
  off = total;
  tmp_off = total + m;
  total += strang_bytes(t, count);
}

// amplitude/phase calls: step diagonals, final rotation and the rotated FP64 product
static void add_phase(const redo_table* t, int64_t B, int64_t M, size_t& total, size_t& pd_off, size_t& zf_off,
                      size_t& out_off) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  pd_off = total;
  zf_off = pd_off + up((size_t)B * M * t->N * sizeof(double2));
  out_off = zf_off + up((size_t)B * t->N * sizeof(double2));
  total = out_off + up((size_t)B * t->N * t->N * sizeof(double2));
}

static PropLayout prop_layout(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                              int32_t reunit_every, bool phase = false) {
  PropLayout L;
  L.pd_off = L.zf_off = L.phout_off = 0;
  if (t->N > kSmallN) {
    L.eff_prec = prec == REDO_FP16X3 ? REDO_FP32 : prec;
    if (reunit_every > 0) {
      L.p = plan_chain_aligned(t, B, M, reunit_every);
    } else {
      L.p = plan_chain_large(t, B, M);
      if (phase) {
        // whole steps per segment, so that the step diagonals fall between launches
        const int64_t kd = (int64_t)t->K * t->digits;
        L.p = plan_chain_aligned(t, B, M, L.p.seg_len > 0 ? (L.p.seg_len + kd - 1) / kd : 1);
      }
    }
    L.seg_off = L.prod_off = L.prod64_off = 0;
    L.total = prec == REDO_FP16X3 ? tc_large_prop_workspace(t, L.p, reunit_every > 0)
                                  : large_prop_workspace(t, L.p, prec, reunit_every > 0);
    add_strang(t, B, L.total, L.strang_off, L.strang_tmp_off);
    if (phase) add_phase(t, B, M, L.total, L.pd_off, L.zf_off, L.phout_off);
    return L;
  }
  // the tensor-core path forms segment products in split FP16 and combines them in FP32
  L.eff_prec = prec == REDO_FP16X3 ? REDO_FP32 : prec;
  // amplitude/phase calls: the SIMT chains carry each step's diagonal as an extra factor, the
  // tensor-core chains apply it in the epilogue of the step's last product
  const bool phase_factors = phase && prec != REDO_FP16X3;
  if (reunit_every > 0)
    L.p = plan_chain_aligned(t, B, M, reunit_every, phase_factors);
  else
    L.p = prec == REDO_FP16X3 ? plan_chain_tc(t, B, M) : plan_chain(t, B, M, L.eff_prec, phase_factors);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t el = L.eff_prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t n2 = (size_t)t->N * t->N;
  L.seg_off = 0;
  L.prod_off = up((size_t)L.p.B * L.p.S * n2 * el);
  L.prod64_off = L.prod_off + up((size_t)L.p.B * n2 * el);
  L.total = L.prod64_off + (reunit_every > 0 ? up((size_t)L.p.B * n2 * sizeof(double2)) : 0);
  add_strang(t, B, L.total, L.strang_off, L.strang_tmp_off);
  if (phase) add_phase(t, B, M, L.total, L.pd_off, L.zf_off, L.phout_off);
  return L;
}

redo_status redo_propagate_workspace(const redo_table* t, int64_t B, int64_t M,
                                     redo_precision prec, int32_t reunit_every, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || reunit_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if (reunit_every > M) reunit_every = M > 0 ? (int32_t)M : 0;
  *bytes = prop_layout(t, B, M, prec, reunit_every).total;
  return REDO_OK;
}

// Shared body of redo_propagate, redo_propagate_phase (phi non-null: amplitude/phase controls) and
// redo_propagate_drift (h non-null: a diagonal drift per pulse).
static redo_status propagate_core(const redo_table* t, const int32_t* q, const double* phi, const double* h,
                                  int64_t B, int64_t M, redo_precision prec, int32_t reunit_every, void* U_out,
                                  const void* U_target,
                                  double* F_out, void* tau_out, void* workspace, size_t workspace_bytes,
                                  int64_t* dev_status, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  if (reunit_every < 0) return set_error(REDO_ERR_INVALID, "reunit_every must be >= 0");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  const bool phase = phi != nullptr;
  const bool diag = phase || h != nullptr;   // step-opening diagonal factors
  if (B == 0) return REDO_OK;
  if (M > 0 && !q) return set_error(REDO_ERR_INVALID, "q is NULL");
  if (U_target && !F_out && !tau_out)
    return set_error(REDO_ERR_INVALID, "U_target given without F_out or tau_out");
  if (!U_out && !U_target) return set_error(REDO_ERR_INVALID, "nothing to compute");
  if (reunit_every > M) reunit_every = M > 0 ? (int32_t)M : 0;
  PropLayout L = prop_layout(t, B, M, prec, reunit_every, diag);
  if (!workspace || workspace_bytes < L.total)
    return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", L.total);
  if (((uintptr_t)workspace & 255) != 0) return set_error(REDO_ERR_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  double2* zf = nullptr;
  if (diag) {
    double2* pd = (double2*)((char*)workspace + L.pd_off);
    zf = (double2*)((char*)workspace + L.zf_off);
    const bool tc = prec == REDO_FP16X3 && t->N <= kSmallN;     // the split-FP16 chains take FP32 diagonals
    e = phase ? launch_phase_diag(t, phi, B, M, tc ? nullptr : pd, tc ? (float2*)pd : nullptr, zf, s)
              : launch_drift_diag(t, h, B, M, tc ? nullptr : pd, tc ? (float2*)pd : nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, phase ? "phase diagonals" : "drift diagonals");
    if (tc)
      L.p.pd32 = (const float2*)pd;
    else
      L.p.pd = pd;
  }
  // the last rotation Z_{M-1} of an amplitude/phase call, applied before the fidelity
  auto rotate = [&](const void*& fin, int& fin_prec) -> cudaError_t {
    if (!phase) return cudaSuccess;
    double2* o = (double2*)((char*)workspace + L.phout_off);
    cudaError_t er = launch_phase_final(t->N, B, fin_prec, fin, zf, o, s);
    fin = o;
    fin_prec = REDO_FP64;
    return er;
  };
  const ChainPlan& p = L.p;
  const int eff = L.eff_prec;
  char* seg = (char*)workspace + L.seg_off;
  char* prod = (char*)workspace + L.prod_off;
  char* prod64 = (char*)workspace + L.prod64_off;
  if (t->N > kSmallN) {
    void* res = nullptr;
    int res_prec = eff;
    {
      ProfScope ps(2, s);
      e = prec == REDO_FP16X3
              ? tc_large_propagate(t, q, p, reunit_every > 0, workspace, &res, &res_prec, dev_status, s)
              : large_propagate(t, q, p, eff, reunit_every > 0, workspace, &res, &res_prec,
                                dev_status, s);
      if (e != cudaSuccess) return cuda_error(e, "large-N chains");
    }
    if (t->strang) {
      // symmetric split: S_M ... S_1 = D_h (U_M ... U_1) D_h^dag
      double2* sb = (double2*)((char*)workspace + L.strang_off);
      if ((e = launch_half_drift_conj(t, res_prec, res, B, 0, sb,
                                      (double2*)((char*)workspace + L.strang_tmp_off), s)) != cudaSuccess)
        return cuda_error(e, "half-drift conjugation");
      res = sb;
      res_prec = REDO_FP64;
    }
    const void* rc = res;
    if ((e = rotate(rc, res_prec)) != cudaSuccess) return cuda_error(e, "phase rotation");
    res = const_cast<void*>(rc);
    ProfScope ps(4, s);
    if ((e = launch_finalize(t, B, res_prec, res, U_out, (const double2*)U_target, F_out,
                             (double2*)tau_out, s)) != cudaSuccess)
      return cuda_error(e, "finalize");
    return REDO_OK;
  }
  if (prec == REDO_FP16X3) {
    ProfScope ps(5, s);
    if ((e = launch_chain_tc(t, q, p, seg, dev_status, s)) != cudaSuccess)
      return cuda_error(e, "tensor-core chain segments");
  } else {
    ProfScope ps(2, s);
    if ((e = launch_chain_segments(t, q, p, eff, seg, dev_status, s)) != cudaSuccess)
      return cuda_error(e, "chain segments");
  }
  if (reunit_every > 0 && M > 0) {
    ProfScope ps(6, s);
    if ((e = launch_polar(t, eff, eff, seg, seg, p.B * p.S, 1, s)) != cudaSuccess)
      return cuda_error(e, "segment re-unitarisation");
  }
  {
    ProfScope ps(3, s);
    if ((e = launch_chain_combine(t, p, eff, seg, prod, dev_status, s)) != cudaSuccess)
      return cuda_error(e, "chain combine");
  }
  const void* fin = prod;
  int fin_prec = eff;
  if (reunit_every > 0 && M > 0) {
    ProfScope ps(6, s);
    if ((e = launch_polar(t, eff, REDO_FP64, prod, prod64, B, 1, s)) != cudaSuccess)
      return cuda_error(e, "final re-unitarisation");
    fin = prod64;
    fin_prec = REDO_FP64;
  }
  if (t->strang) {
    double2* sb = (double2*)((char*)workspace + L.strang_off);
    if ((e = launch_half_drift_conj(t, fin_prec, fin, B, 0, sb,
                                    (double2*)((char*)workspace + L.strang_tmp_off), s)) != cudaSuccess)
      return cuda_error(e, "half-drift conjugation");
    fin = sb;
    fin_prec = REDO_FP64;
  }
  if ((e = rotate(fin, fin_prec)) != cudaSuccess) return cuda_error(e, "phase rotation");
  {
    ProfScope ps(4, s);
    if ((e = launch_finalize(t, B, fin_prec, fin, U_out, (const double2*)U_target, F_out,
                             (double2*)tau_out, s)) != cudaSuccess)
      return cuda_error(e, "finalize");
  }
  return REDO_OK;
}

redo_status redo_propagate(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                           redo_precision prec, int32_t reunit_every, void* U_out,
                           const void* U_target, double* F_out, void* tau_out, void* workspace,
                           size_t workspace_bytes, int64_t* dev_status, void* stream) {
  return propagate_core(t, q, nullptr, nullptr, B, M, prec, reunit_every, U_out, U_target, F_out, tau_out,
                        workspace, workspace_bytes, dev_status, stream);
}

static redo_status check_phase(const redo_table* t, redo_precision prec) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (!t->sz64) return set_error(REDO_ERR_INVALID, "no phase axes: call redo_table_set_phase_axes first");
  if (t->strang) return set_error(REDO_ERR_UNSUPPORTED, "amplitude/phase calls on a symmetric-split table");
  if (prec == REDO_FP16X3 && t->N > kSmallN)
    return set_error(REDO_ERR_UNSUPPORTED, "amplitude/phase calls in REDO_FP16X3 need N <= 64");
  return REDO_OK;
}

redo_status redo_propagate_phase_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                           int32_t reunit_every, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || reunit_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if ((st = check_phase(t, prec)) != REDO_OK) return st;
  if (reunit_every > M) reunit_every = M > 0 ? (int32_t)M : 0;
  *bytes = prop_layout(t, B, M, prec, reunit_every, true).total;
  return REDO_OK;
}

redo_status redo_propagate_phase(const redo_table* t, const int32_t* q, const double* phi, int64_t B, int64_t M,
                                 redo_precision prec, int32_t reunit_every, void* U_out, const void* U_target,
                                 double* F_out, void* tau_out, void* workspace, size_t workspace_bytes,
                                 int64_t* dev_status, void* stream) {
  redo_status st = check_phase(t, prec);
  if (st != REDO_OK) return st;
  if (B > 0 && M > 0 && !phi) return set_error(REDO_ERR_INVALID, "phi is NULL");
  static const double kNoPhase = 0.0;
  return propagate_core(t, q, phi ? phi : &kNoPhase, nullptr, B, M, prec, reunit_every, U_out, U_target, F_out,
                        tau_out, workspace, workspace_bytes, dev_status, stream);
}

static redo_status check_drift(const redo_table* t, redo_precision prec) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (t->strang) return set_error(REDO_ERR_UNSUPPORTED, "per-pulse drift on a symmetric-split table");
  if (prec == REDO_FP16X3 && t->N > kSmallN)
    return set_error(REDO_ERR_UNSUPPORTED, "per-pulse drift in REDO_FP16X3 needs N <= 64");
  return check_prec(t, prec);
}

redo_status redo_propagate_drift_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                           int32_t reunit_every, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || reunit_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_drift(t, prec);
  if (st != REDO_OK) return st;
  if (reunit_every > M) reunit_every = M > 0 ? (int32_t)M : 0;
  *bytes = prop_layout(t, B, M, prec, reunit_every, true).total;
  return REDO_OK;
}

redo_status redo_propagate_drift(const redo_table* t, const int32_t* q, const double* h, int64_t B, int64_t M,
                                 redo_precision prec, int32_t reunit_every, void* U_out, const void* U_target,
                                 double* F_out, void* tau_out, void* workspace, size_t workspace_bytes,
                                 int64_t* dev_status, void* stream) {
  redo_status st = check_drift(t, prec);
  if (st != REDO_OK) return st;
  if (B > 0 && M > 0 && !h) return set_error(REDO_ERR_INVALID, "h is NULL");
  static const double kNoDrift = 0.0;
  return propagate_core(t, q, nullptr, h ? h : &kNoDrift, B, M, prec, reunit_every, U_out, U_target, F_out,
                        tau_out, workspace, workspace_bytes, dev_status, stream);
}

// ---------------------------------------------------------------------------
// Per-step propagators, re-unitarisation, cost model
// ---------------------------------------------------------------------------
static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// FP32 step products (converted to complex128 afterwards) and, for a symmetric-split table with
// a dense drift, the intermediate of the conjugation.
static size_t steps_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec, size_t* conj_off) {
  const size_t count = (size_t)B * M, n2 = (size_t)t->N * t->N;
  size_t total = prec == REDO_FP32 ? up256(count * n2 * sizeof(float2)) : 0;
  *conj_off = total;
  if (t->strang && !t->h0_diagonal) total += up256(count * n2 * sizeof(double2));
  return total;
}

static redo_status check_steps(const redo_table* t, redo_precision prec) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "per-step propagators in REDO_FP64 or REDO_FP32 only");
  if (t->N > kSmallN) return set_error(REDO_ERR_UNSUPPORTED, "per-step propagators for N <= 64 only");
  return check_prec(t, prec);
}

redo_status redo_propagate_steps_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                           size_t* bytes) {
  redo_status st = check_steps(t, prec);
  if (st != REDO_OK) return st;
  if (!bytes) return set_error(REDO_ERR_INVALID, "bytes is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  size_t off;
  *bytes = steps_workspace(t, B, M, prec, &off);
  return REDO_OK;
}

redo_status redo_propagate_steps(const redo_table* t, const int32_t* q, int64_t B, int64_t M, redo_precision prec,
                                 void* U_steps, void* workspace, size_t workspace_bytes, int64_t* dev_status,
                                 void* stream) {
  redo_status st = check_steps(t, prec);
  if (st != REDO_OK) return st;
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  if (B == 0 || M == 0) return REDO_OK;
  if (!q || !U_steps) return set_error(REDO_ERR_INVALID, "q or U_steps is NULL");
  size_t conj_off;
  const size_t need = steps_workspace(t, B, M, prec, &conj_off);
  if (need > 0 && (!workspace || workspace_bytes < need))
    return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", need);
  if (need > 0 && ((uintptr_t)workspace & 255) != 0)
    return set_error(REDO_ERR_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  // one segment per time step: segment (b, n) is U_n = E_{K-1} ... E_0 D of pulse b
  const ChainPlan p = plan_chain_aligned(t, B, M, 1);
  const int64_t count = B * M;
  void* seg = prec == REDO_FP64 ? U_steps : workspace;
  cudaError_t e = launch_chain_segments(t, q, p, prec, seg, dev_status, s);
  if (e != cudaSuccess) return cuda_error(e, "step products");
  if (t->strang) {
    // symmetric step S_n = D_h E_{K-1} ... E_0 D_h = D_h U_n D_h^dag of the folded step
    double2* tmp = t->h0_diagonal ? nullptr : (double2*)((char*)workspace + conj_off);
    if ((e = launch_half_drift_conj(t, prec, seg, count, 0, (double2*)U_steps, tmp, s)) != cudaSuccess)
      return cuda_error(e, "half-drift conjugation");
  } else if (prec == REDO_FP32) {
    if ((e = launch_finalize(t, count, REDO_FP32, seg, U_steps, nullptr, nullptr, nullptr, s)) != cudaSuccess)
      return cuda_error(e, "widen to complex128");
  }
  return REDO_OK;
}

redo_status redo_reunitarize(int32_t N, int64_t count, redo_precision prec, const void* P_in, void* U_out,
                             int32_t iters, void* stream) {
  if (N < 2 || N > kSmallN || (N & (N - 1)) != 0)
    return set_error(REDO_ERR_UNSUPPORTED, "redo_reunitarize takes N a power of two, 2 <= N <= 64 (N=%d)", N);
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "redo_reunitarize arithmetic is REDO_FP64 or REDO_FP32");
  if (count < 0 || iters < 0) return set_error(REDO_ERR_INVALID, "negative count or iters");
  if (count == 0) return REDO_OK;
  if (!P_in || !U_out) return set_error(REDO_ERR_INVALID, "null matrix pointer");
  cudaError_t e = launch_polar_c128(N, prec, (const double2*)P_in, (double2*)U_out, count, iters,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "Newton-Schulz polar steps");
  return REDO_OK;
}

redo_status redo_plan(double omega_max, double eps, int32_t base, int32_t* l_out, int32_t* m_out, int32_t* p_out,
                      int64_t* s_out) {
  if (!(omega_max > 0.0) || !(eps > 0.0) || !std::isfinite(omega_max) || !std::isfinite(eps))
    return set_error(REDO_ERR_INVALID, "omega_max and eps must be positive and finite");
  if (base < 2) return set_error(REDO_ERR_INVALID, "base must be >= 2");
  if (eps > omega_max) return set_error(REDO_ERR_INVALID, "eps larger than omega_max");
  const double b = (double)base, rel = 1e-12;
  // l: the largest integer with b^l <= eps (b^l = eps when eps is a power of b)
  int l = 0;
  if (1.0 <= eps * (1.0 + rel)) {
    while (std::pow(b, l + 1) <= eps * (1.0 + rel)) ++l;
  } else {
    while (std::pow(b, l) > eps * (1.0 + rel)) --l;
  }
  // m: the smallest integer with b^(m+1) > omega_max
  int m = l - 1;
  while (std::pow(b, m + 1) <= omega_max) ++m;
  if (l_out) *l_out = l;
  if (m_out) *m_out = m;
  if (p_out) *p_out = m - l;
  if (s_out) *s_out = (int64_t)(base - 1) * (int64_t)(m - l + 1);
  return REDO_OK;
}

redo_status redo_batched_product(int32_t N, int64_t count, const void* A, int32_t adjA, int32_t A_batched,
                                 const void* B, int32_t adjB, int32_t B_batched, void* C, void* stream) {
  if (N <= 0 || N > kMaxN) return set_error(REDO_ERR_INVALID, "N=%d out of range", N);
  if (count < 0) return set_error(REDO_ERR_INVALID, "negative count");
  if (count == 0) return REDO_OK;
  if (!A || !B || !C) return set_error(REDO_ERR_INVALID, "null matrix pointer");
  const int64_t n2 = (int64_t)N * N;
  const char *a0 = (const char*)A, *b0 = (const char*)B, *c0 = (const char*)C;
  const int64_t ab = (A_batched ? count : 1) * n2 * 16, bb = (B_batched ? count : 1) * n2 * 16, cb = count * n2 * 16;
  if ((c0 < a0 + ab && a0 < c0 + cb) || (c0 < b0 + bb && b0 < c0 + cb))
    return set_error(REDO_ERR_INVALID, "C overlaps A or B");
  cudaError_t e = launch_batched_product(N, count, (const double2*)A, adjA ? 1 : 0, A_batched ? n2 : 0,
                                         (const double2*)B, adjB ? 1 : 0, B_batched ? n2 : 0, (double2*)C,
                                         (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "batched product");
  return REDO_OK;
}

// ---------------------------------------------------------------------------
// GRAPE gradient
// ---------------------------------------------------------------------------
struct GradLayout {
  ChainPlan p;
  size_t seg_off, pck_off, rck_off, tau_off, total;
  size_t keep_off = 0;                 // N <= 64: every forward state kept (0: not kept)
  bool keep = false;
  size_t strang_off, strang_tmp_off;   // symmetric split: transformed targets (+ scratch)
};

static GradLayout grad_layout(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                              int32_t checkpoint_every) {
  GradLayout L;
  if (t->N > kSmallN) {
    L.p = checkpoint_every > 0 ? plan_chain_aligned(t, B, M, checkpoint_every)
                               : plan_chain_large(t, B, M);
    L.seg_off = L.pck_off = L.rck_off = L.tau_off = 0;
    L.total = prec == REDO_FP16X3 ? tc_large_grad_workspace(t, L.p) : large_grad_workspace(t, L.p, prec);
    add_strang(t, B, L.total, L.strang_off, L.strang_tmp_off);
    return L;
  }
  L.p = checkpoint_every > 0 ? plan_chain_aligned(t, B, M, checkpoint_every)
                             : plan_chain(t, B, M, prec);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t mats = up((size_t)L.p.B * L.p.S * t->N * t->N * el);
  L.seg_off = 0;
  L.pck_off = mats;
  L.rck_off = 2 * mats;
  L.tau_off = 3 * mats;
  L.total = L.tau_off + up((size_t)B * sizeof(double2));
  // every forward state kept when they fit in 24 GiB: the sweep then multiplies only the
  // costates (one product per factor instead of two)
  const size_t keep_bytes = (size_t)L.p.B * L.p.S * L.p.seg_len * t->N * t->N * el;
  if (M > 0 && keep_bytes <= ((size_t)24 << 30)) {
    L.keep = true;
    L.keep_off = L.total;
    L.total += up(keep_bytes);
  }
  add_strang(t, B, L.total, L.strang_off, L.strang_tmp_off);
  return L;
}

redo_status redo_fidelity_grad_workspace(const redo_table* t, int64_t B, int64_t M,
                                         redo_precision prec, int32_t checkpoint_every,
                                         size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || checkpoint_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  if (prec != REDO_FP64 && prec != REDO_FP32 && !(prec == REDO_FP16X3 && t->N > kSmallN))
    return set_error(REDO_ERR_UNSUPPORTED,
                     "the gradient supports REDO_FP64, REDO_FP32 and, for N >= 128, REDO_FP16X3");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if (checkpoint_every > M) checkpoint_every = M > 0 ? (int32_t)M : 0;
  *bytes = grad_layout(t, B, M, prec, checkpoint_every).total;
  return REDO_OK;
}

redo_status redo_fidelity_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                               const void* U_target, int32_t target_batched, redo_precision prec,
                               int32_t checkpoint_every, int32_t reunit_every, double* F_out, double* grad,
                               void* workspace, size_t workspace_bytes, int64_t* dev_status,
                               void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0 || checkpoint_every < 0 || reunit_every < 0)
    return set_error(REDO_ERR_INVALID, "negative size");
  if (reunit_every > 0 && reunit_every != checkpoint_every)
    return set_error(REDO_ERR_INVALID, "reunit_every (%d) must equal checkpoint_every (%d): the segment products "
                     "of the checkpoints are what is re-unitarised", reunit_every, checkpoint_every);
  if (prec != REDO_FP64 && prec != REDO_FP32 && !(prec == REDO_FP16X3 && t->N > kSmallN))
    return set_error(REDO_ERR_UNSUPPORTED,
                     "the gradient supports REDO_FP64, REDO_FP32 and, for N >= 128, REDO_FP16X3");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if (B == 0) return REDO_OK;
  if (!U_target) return set_error(REDO_ERR_INVALID, "U_target is NULL");
  if (M > 0 && (!q || !grad)) return set_error(REDO_ERR_INVALID, "q or grad is NULL");
  if (checkpoint_every > M) checkpoint_every = M > 0 ? (int32_t)M : 0;
  const GradLayout L = grad_layout(t, B, M, prec, checkpoint_every);
  if (!workspace || workspace_bytes < L.total)
    return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", L.total);
  if (((uintptr_t)workspace & 255) != 0) return set_error(REDO_ERR_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)workspace;
  double2* tau = (double2*)(w + L.tau_off);
  cudaError_t e;
  ProfScope ps(7, s);
  if (t->strang) {
    // symmetric split: F(U_T, D_h U D_h^dag) = F(D_h^dag U_T D_h, U) for the folded chain U
    double2* sb = (double2*)(w + L.strang_off);
    if ((e = launch_half_drift_conj(t, REDO_FP64, U_target, target_batched ? B : 1, 1, sb,
                                    (double2*)(w + L.strang_tmp_off), s)) != cudaSuccess)
      return cuda_error(e, "half-drift conjugation of the target");
    U_target = sb;
  }
  if (t->N > kSmallN) {
    const bool reunit = reunit_every > 0;
    e = prec == REDO_FP16X3
            ? tc_large_grad(t, q, L.p, (const double2*)U_target, target_batched, F_out, grad,
                            workspace, dev_status, s, reunit)
            : large_grad(t, q, L.p, prec, (const double2*)U_target, target_batched, F_out, grad,
                         workspace, dev_status, s, nullptr, nullptr, reunit);
    if (e != cudaSuccess) return cuda_error(e, "large-N gradient");
    return REDO_OK;
  }
  void* keep = L.keep ? w + L.keep_off : nullptr;
  if ((e = launch_chain_segments(t, q, L.p, prec, w + L.seg_off, dev_status, s, keep)) != cudaSuccess)
    return cuda_error(e, "gradient segments");
  if (reunit_every > 0 && M > 0 &&
      (e = launch_polar(t, prec, prec, w + L.seg_off, w + L.seg_off, B * L.p.S, 1, s)) != cudaSuccess)
    return cuda_error(e, "segment re-unitarisation");
  if ((e = launch_grad_scan(t, B, L.p.S, prec, w + L.seg_off, (const double2*)U_target,
                            target_batched, w + L.pck_off, w + L.rck_off, tau, F_out, s)) !=
      cudaSuccess)
    return cuda_error(e, "gradient checkpoints");
  if (M > 0 && (e = launch_grad_sweep(t, q, L.p, prec, w + L.pck_off, w + L.rck_off, tau, grad,
                                      dev_status, s, nullptr, keep)) != cudaSuccess)
    return cuda_error(e, "gradient sweep");
  return REDO_OK;
}

// Amplitude/phase GRAPE gradient (N <= 64, SIMT): the chain with the step diagonals as
// factors, against the target Z_{M-1}^dag U_T of the regrouped chain.
struct PhaseGradLayout {
  GradLayout g;
  size_t pd_off, zf_off, ut_off, tz_off, total;
};

static PhaseGradLayout phase_grad_layout(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                         int32_t checkpoint_every, bool phase = true) {
  PhaseGradLayout L;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  if (t->N > kSmallN) {
    // lockstep SIMT sweeps on segments of whole steps (the diagonals fall between launches)
    const int64_t kd = (int64_t)t->K * t->digits;
    int64_t sps = checkpoint_every;
    if (sps <= 0) {
      const ChainPlan p0 = plan_chain_large(t, B, M);
      sps = p0.seg_len > 0 ? (p0.seg_len + kd - 1) / kd : 1;
    }
    L.g.p = plan_chain_aligned(t, B, M, sps);
    L.g.seg_off = L.g.pck_off = L.g.rck_off = L.g.tau_off = 0;
    L.pd_off = up(large_grad_workspace(t, L.g.p, prec));
  } else {
    L.g.p = checkpoint_every > 0 ? plan_chain_aligned(t, B, M, checkpoint_every, true)
                                 : plan_chain(t, B, M, prec, true);
    const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t mats = up((size_t)L.g.p.B * L.g.p.S * t->N * t->N * el);
    L.g.seg_off = 0;
    L.g.pck_off = mats;
    L.g.rck_off = 2 * mats;
    L.g.tau_off = 3 * mats;
    L.pd_off = L.g.tau_off + up((size_t)B * sizeof(double2));
  }
  // the per-pulse drift form has no final rotation, transformed target or boundary traces
  const size_t ph = phase ? 1 : 0;
  L.zf_off = L.pd_off + up((size_t)B * M * t->N * sizeof(double2));
  L.ut_off = L.zf_off + ph * up((size_t)B * t->N * sizeof(double2));
  L.tz_off = L.ut_off + ph * up((size_t)B * t->N * t->N * sizeof(double2));
  L.total = L.tz_off + ph * up((size_t)B * (M + 1) * t->K * sizeof(double2));
  if (t->N <= kSmallN) {
    // N <= 64: every forward state kept when they fit in 24 GiB (the sweep then multiplies only
    // the costates), as in the plain gradient
    const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t keep_bytes = (size_t)L.g.p.B * L.g.p.S * L.g.p.seg_len * t->N * t->N * el;
    if (M > 0 && keep_bytes <= ((size_t)24 << 30)) {
      L.g.keep = true;
      L.g.keep_off = L.total;
      L.total += up(keep_bytes);
    }
  }
  return L;
}

static redo_status check_phase_grad(const redo_table* t, redo_precision prec) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (!t->sz64) return set_error(REDO_ERR_INVALID, "no phase axes: call redo_table_set_phase_axes first");
  if (t->strang) return set_error(REDO_ERR_UNSUPPORTED, "amplitude/phase calls on a symmetric-split table");
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "the amplitude/phase gradient supports REDO_FP64 and REDO_FP32");
  return check_prec(t, prec);
}

redo_status redo_fidelity_grad_phase_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                               int32_t checkpoint_every, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || checkpoint_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_phase_grad(t, prec);
  if (st != REDO_OK) return st;
  if (checkpoint_every > M) checkpoint_every = M > 0 ? (int32_t)M : 0;
  *bytes = phase_grad_layout(t, B, M, prec, checkpoint_every).total;
  return REDO_OK;
}

redo_status redo_fidelity_grad_phase(const redo_table* t, const int32_t* q, const double* phi, int64_t B, int64_t M,
                                     const void* U_target, int32_t target_batched, redo_precision prec,
                                     int32_t checkpoint_every, double* F_out, double* grad_amp, double* grad_phase,
                                     void* workspace, size_t workspace_bytes, int64_t* dev_status, void* stream) {
  redo_status st = check_phase_grad(t, prec);
  if (st != REDO_OK) return st;
  if (B < 0 || M < 0 || checkpoint_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  if (B == 0) return REDO_OK;
  if (!U_target) return set_error(REDO_ERR_INVALID, "U_target is NULL");
  if (M > 0 && (!q || !phi || !grad_amp || !grad_phase))
    return set_error(REDO_ERR_INVALID, "q, phi, grad_amp or grad_phase is NULL");
  if (checkpoint_every > M) checkpoint_every = M > 0 ? (int32_t)M : 0;
  PhaseGradLayout L = phase_grad_layout(t, B, M, prec, checkpoint_every);
  if (!workspace || workspace_bytes < L.total)
    return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", L.total);
  if (((uintptr_t)workspace & 255) != 0) return set_error(REDO_ERR_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)workspace;
  double2* tau = (double2*)(w + L.g.tau_off);
  double2* pd = (double2*)(w + L.pd_off);
  double2* zf = (double2*)(w + L.zf_off);
  double2* ut = (double2*)(w + L.ut_off);
  double2* tz = (double2*)(w + L.tz_off);
  static const double kNoPhase = 0.0;
  cudaError_t e;
  ProfScope ps(7, s);
  if ((e = launch_phase_diag(t, M > 0 ? phi : &kNoPhase, B, M, pd, nullptr, zf, s)) != cudaSuccess)
    return cuda_error(e, "phase diagonals");
  if ((e = launch_phase_target(t->N, B, (const double2*)U_target, target_batched, zf, ut, s)) != cudaSuccess)
    return cuda_error(e, "phase target");
  L.g.p.pd = pd;
  if (t->N > kSmallN) {
    if ((e = large_grad(t, q, L.g.p, prec, ut, 1, F_out, grad_amp, workspace, dev_status, s, tz, grad_phase)) !=
        cudaSuccess)
      return cuda_error(e, "large-N phase gradient");
    return REDO_OK;
  }
  void* keep = L.g.keep ? w + L.g.keep_off : nullptr;
  if ((e = launch_chain_segments(t, q, L.g.p, prec, w + L.g.seg_off, dev_status, s, keep)) != cudaSuccess)
    return cuda_error(e, "gradient segments");
  if ((e = launch_grad_scan(t, B, L.g.p.S, prec, w + L.g.seg_off, ut, 1, w + L.g.pck_off, w + L.g.rck_off, tau,
                            F_out, s)) != cudaSuccess)
    return cuda_error(e, "gradient checkpoints");
  if (M > 0) {
    if ((e = launch_grad_sweep(t, q, L.g.p, prec, w + L.g.pck_off, w + L.g.rck_off, tau, grad_amp, dev_status, s,
                               tz, keep)) != cudaSuccess)
      return cuda_error(e, "gradient sweep");
    if ((e = launch_phase_grad_finish(t->N, B, M, t->K, tz, tau, grad_phase, s)) != cudaSuccess)
      return cuda_error(e, "phase gradient");
  }
  return REDO_OK;
}

// GRAPE gradient with a diagonal drift per pulse: the chain with the step diagonals
// diag(exp(-i dt h_b)) as factors, against the caller's target (SIMT sweeps, FP64 or FP32).
static redo_status check_drift_grad(const redo_table* t, redo_precision prec) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (t->strang) return set_error(REDO_ERR_UNSUPPORTED, "per-pulse drift on a symmetric-split table");
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "the per-pulse drift gradient supports REDO_FP64 and REDO_FP32");
  return check_prec(t, prec);
}

redo_status redo_fidelity_grad_drift_workspace(const redo_table* t, int64_t B, int64_t M, redo_precision prec,
                                               int32_t checkpoint_every, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || checkpoint_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_drift_grad(t, prec);
  if (st != REDO_OK) return st;
  if (checkpoint_every > M) checkpoint_every = M > 0 ? (int32_t)M : 0;
  *bytes = phase_grad_layout(t, B, M, prec, checkpoint_every, false).total;
  return REDO_OK;
}

redo_status redo_fidelity_grad_drift(const redo_table* t, const int32_t* q, const double* h, int64_t B, int64_t M,
                                     const void* U_target, int32_t target_batched, redo_precision prec,
                                     int32_t checkpoint_every, int32_t reunit_every, double* F_out, double* grad,
                                     void* workspace, size_t workspace_bytes, int64_t* dev_status, void* stream) {
  redo_status st = check_drift_grad(t, prec);
  if (st != REDO_OK) return st;
  if (B < 0 || M < 0 || checkpoint_every < 0 || reunit_every < 0)
    return set_error(REDO_ERR_INVALID, "negative size");
  if (reunit_every > 0 && reunit_every != checkpoint_every)
    return set_error(REDO_ERR_INVALID, "reunit_every (%d) must equal checkpoint_every (%d)", reunit_every,
                     checkpoint_every);
  if (B == 0) return REDO_OK;
  if (!U_target) return set_error(REDO_ERR_INVALID, "U_target is NULL");
  if (M > 0 && (!q || !h || !grad)) return set_error(REDO_ERR_INVALID, "q, h or grad is NULL");
  if (checkpoint_every > M) checkpoint_every = M > 0 ? (int32_t)M : 0;
  PhaseGradLayout L = phase_grad_layout(t, B, M, prec, checkpoint_every, false);
  if (!workspace || workspace_bytes < L.total)
    return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", L.total);
  if (((uintptr_t)workspace & 255) != 0) return set_error(REDO_ERR_INVALID, "workspace not 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)workspace;
  double2* tau = (double2*)(w + L.g.tau_off);
  double2* pd = (double2*)(w + L.pd_off);
  const double2* ut = (const double2*)U_target;
  cudaError_t e;
  ProfScope ps(7, s);
  if (M > 0 && (e = launch_drift_diag(t, h, B, M, pd, nullptr, s)) != cudaSuccess)
    return cuda_error(e, "drift diagonals");
  L.g.p.pd = pd;
  if (t->N > kSmallN) {
    if ((e = large_grad(t, q, L.g.p, prec, ut, target_batched, F_out, grad, workspace, dev_status, s, nullptr,
                        nullptr, reunit_every > 0)) != cudaSuccess)
      return cuda_error(e, "large-N drift gradient");
    return REDO_OK;
  }
  void* keep = L.g.keep ? w + L.g.keep_off : nullptr;
  if ((e = launch_chain_segments(t, q, L.g.p, prec, w + L.g.seg_off, dev_status, s, keep)) != cudaSuccess)
    return cuda_error(e, "gradient segments");
  if (reunit_every > 0 && M > 0 &&
      (e = launch_polar(t, prec, prec, w + L.g.seg_off, w + L.g.seg_off, B * L.g.p.S, 1, s)) != cudaSuccess)
    return cuda_error(e, "segment re-unitarisation");
  if ((e = launch_grad_scan(t, B, L.g.p.S, prec, w + L.g.seg_off, ut, target_batched, w + L.g.pck_off,
                            w + L.g.rck_off, tau, F_out, s)) != cudaSuccess)
    return cuda_error(e, "gradient checkpoints");
  if (M > 0 && (e = launch_grad_sweep(t, q, L.g.p, prec, w + L.g.pck_off, w + L.g.rck_off, tau, grad, dev_status,
                                      s, nullptr, keep)) != cudaSuccess)
    return cuda_error(e, "gradient sweep");
  return REDO_OK;
}

redo_status redo_simulate_workspace(const redo_table* t, int64_t B, int64_t M,
                                    redo_precision prec, int32_t reunit_every, int32_t want_U,
                                    size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0 || reunit_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  // the lockstep state simulation (N > 64 with fewer pulses than SMs) needs two state vectors
  size_t state = t->N > kSmallN && B < t->num_sms ? large_sim_workspace(t, B) : 0;
  if (t->strang) state += ((size_t)B * t->N * sizeof(double2) + 255) & ~(size_t)255;   // D_h^dag psi0
  size_t prop = 0;
  if (want_U) {
    st = redo_propagate_workspace(t, B, M, prec, reunit_every, &prop);
    if (st != REDO_OK) return st;
  }
  *bytes = state > prop ? state : prop;   // the two phases run one after the other
  return REDO_OK;
}

redo_status redo_simulate(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                          redo_precision prec, int32_t reunit_every, const void* psi0,
                          int32_t psi0_batched, const double* obs_diag, double* expect,
                          void* U_final, void* workspace, size_t workspace_bytes,
                          int64_t* dev_status, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0 || reunit_every < 0) return set_error(REDO_ERR_INVALID, "negative size");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if (prec == REDO_FP16X3 && !t->T32)
    return set_error(REDO_ERR_INVALID, "state simulation needs the FP32 table copy");
  if (B == 0) return REDO_OK;
  if (!psi0 || !obs_diag || !expect) return set_error(REDO_ERR_INVALID, "null psi0, obs_diag or expect");
  if (M > 0 && !q) return set_error(REDO_ERR_INVALID, "q is NULL");
  if (t->strang && !t->h0_diagonal)
    return set_error(REDO_ERR_UNSUPPORTED,
                     "state simulation with the symmetric split needs a diagonal drift H0");
  cudaStream_t s = (cudaStream_t)stream;
  {
    ProfScope ps(2, s);
    cudaError_t e;
    const bool lockstep = t->N > kSmallN && B < t->num_sms;
    const size_t need_state = lockstep ? large_sim_workspace(t, B) : 0;
    if (t->strang) {
      // symmetric split with a diagonal drift and observable: the symmetric states give the
      // same expectations as the folded chain started from D_h^dag psi0
      const size_t need = need_state + (((size_t)B * t->N * sizeof(double2) + 255) & ~(size_t)255);
      if (!workspace || workspace_bytes < need)
        return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", need);
      double2* pw = (double2*)((char*)workspace + need_state);
      if ((e = launch_half_drift_vec(t, (const double2*)psi0, psi0_batched ? B : 1, pw, s)) != cudaSuccess)
        return cuda_error(e, "half-drift of the initial state");
      psi0 = pw;
    }
    if (lockstep) {
      // fewer pulses than SMs: every SM works on every step (one launch per factor)
      if (!workspace || workspace_bytes < need_state)
        return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", need_state);
      e = large_sim(t, q, B, M, prec == REDO_FP64 ? REDO_FP64 : REDO_FP32, (const double2*)psi0,
                    psi0_batched, obs_diag, expect, workspace, s);
    } else if (t->N > kSmallN) {
      // a pulse per CTA, its operators streamed through shared memory
      e = launch_sim_stream(t, q, B, M, prec == REDO_FP64 ? REDO_FP64 : REDO_FP32, (const double2*)psi0,
                            psi0_batched, obs_diag, expect, dev_status, s);
    } else {
      e = launch_sim_state(t, q, B, M, prec == REDO_FP64 ? REDO_FP64 : REDO_FP32,
                           (const double2*)psi0, psi0_batched, obs_diag, expect, dev_status, s);
    }
    if (e != cudaSuccess) return cuda_error(e, "state simulation");
  }
  if (U_final)
    return redo_propagate(t, q, B, M, prec, reunit_every, U_final, nullptr, nullptr, nullptr,
                          workspace, workspace_bytes, dev_status, stream);
  return REDO_OK;
}

redo_status redo_state_grad_workspace(const redo_table* t, int64_t B, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0) return set_error(REDO_ERR_INVALID, "negative B");
  *bytes = t->strang ? 2 * (((size_t)B * t->N * sizeof(double2) + 255) & ~(size_t)255) : 0;
  return REDO_OK;
}

redo_status redo_state_grad(const redo_table* t, const int32_t* q, int64_t B, int64_t M, redo_precision prec,
                            const void* psi0, const void* psi_target, int32_t batched, double* F_out,
                            double* grad, void* workspace, size_t workspace_bytes, int64_t* dev_status,
                            void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative size");
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "redo_state_grad supports REDO_FP64 and REDO_FP32");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if (t->strang && !t->h0_diagonal)
    return set_error(REDO_ERR_UNSUPPORTED, "symmetric split with a non-diagonal drift");
  if (B == 0) return REDO_OK;
  if (!psi0 || !psi_target) return set_error(REDO_ERR_INVALID, "null psi0 or psi_target");
  if (!F_out && !grad) return set_error(REDO_ERR_INVALID, "nothing to compute");
  if (M > 0 && !q) return set_error(REDO_ERR_INVALID, "q is NULL");
  size_t need = 0;
  redo_state_grad_workspace(t, B, &need);
  if (need && (!workspace || workspace_bytes < need))
    return set_error(REDO_ERR_INVALID, "workspace of %zu bytes needed", need);
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(7, s);
  cudaError_t e;
  const double2* p0 = (const double2*)psi0;
  const double2* pT = (const double2*)psi_target;
  if (t->strang) {
    // <psi_T| D_h U D_h^dag |psi0> = <D_h^dag psi_T| U |D_h^dag psi0>
    const int64_t nv = batched ? B : 1;
    double2* w0 = (double2*)workspace;
    double2* wT = (double2*)((char*)workspace + need / 2);
    if ((e = launch_half_drift_vec(t, p0, nv, w0, s)) != cudaSuccess ||
        (e = launch_half_drift_vec(t, pT, nv, wT, s)) != cudaSuccess)
      return cuda_error(e, "half-drift of the states");
    p0 = w0;
    pT = wT;
  }
  if ((e = launch_state_grad(t, q, B, M, prec, p0, pT, batched, F_out, grad, dev_status, s)) != cudaSuccess)
    return cuda_error(e, "state-transfer gradient");
  return REDO_OK;
}

redo_status redo_expect_diag(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                             redo_precision prec, const double* rho_diag, const double* obs_diag,
                             double* expect, double* expect_mean, int64_t* dev_status, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative size");
  if (prec != REDO_FP64 && prec != REDO_FP32)
    return set_error(REDO_ERR_UNSUPPORTED, "redo_expect_diag supports REDO_FP64 and REDO_FP32");
  redo_status st = check_prec(t, prec);
  if (st != REDO_OK) return st;
  if (t->N > kSmallN) return set_error(REDO_ERR_UNSUPPORTED, "redo_expect_diag needs N <= 64");
  if (t->strang && !t->h0_diagonal)
    return set_error(REDO_ERR_UNSUPPORTED, "symmetric split with a non-diagonal drift");
  if (B == 0) return REDO_OK;
  if (!rho_diag || !obs_diag) return set_error(REDO_ERR_INVALID, "null rho_diag or obs_diag");
  if (!expect && !expect_mean) return set_error(REDO_ERR_INVALID, "nothing to compute");
  if (M > 0 && !q) return set_error(REDO_ERR_INVALID, "q is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(2, s);
  cudaError_t e = launch_expect_diag(t, q, B, M, prec, rho_diag, obs_diag, expect, expect_mean, dev_status, s);
  if (e != cudaSuccess) return cuda_error(e, "mixed-state expectations");
  return REDO_OK;
}

static redo_status check_mlp(int32_t layers, const int32_t* sizes) {
  if (layers < 1 || layers > 32 || !sizes) return set_error(REDO_ERR_INVALID, "1 <= layers <= 32");
  for (int l = 0; l <= layers; ++l)
    if (sizes[l] < 1 || sizes[l] > (1 << 20)) return set_error(REDO_ERR_INVALID, "bad layer width");
  return REDO_OK;
}

redo_status redo_mlp_sizes(int32_t layers, const int32_t* sizes, int64_t batch,
                           int64_t* params, int64_t* acts, int64_t* work) {
  redo_status st = check_mlp(layers, sizes);
  if (st != REDO_OK) return st;
  if (batch < 0) return set_error(REDO_ERR_INVALID, "negative batch");
  int64_t a = 0, mw = 0;
  for (int l = 0; l <= layers; ++l) {
    if (l > 0) a += 2 * batch * sizes[l];
    if (sizes[l] > mw) mw = sizes[l];
  }
  // plus the split operand planes of the GEMMs, 256-byte aligned after the float buffers
  const int64_t slack = 256 / sizeof(float);
  if (params) *params = mlp_param_count(layers, sizes);
  if (acts) *acts = a + slack + (int64_t)((mlp_forward_plane_bytes(layers, sizes, batch) + 3) / 4);
  // the backward buffer also holds 32 rows of partial column sums for the bias gradients
  if (work) *work = 2 * batch * mw + 32 * mw + slack + (int64_t)((mlp_backward_plane_bytes(layers, sizes, batch) + 3) / 4);
  return REDO_OK;
}

redo_status redo_mlp_forward(int32_t layers, const int32_t* sizes, const float* params,
                             const float* x, int64_t batch, float* acts, float* y, void* stream) {
  redo_status st = check_mlp(layers, sizes);
  if (st != REDO_OK) return st;
  if (batch < 0) return set_error(REDO_ERR_INVALID, "negative batch");
  if (batch == 0) return REDO_OK;
  if (!params || !x || !acts || !y) return set_error(REDO_ERR_INVALID, "null pointer");
  cudaError_t e = mlp_forward(layers, sizes, params, x, batch, acts, y, (cudaStream_t)stream);
  return e == cudaSuccess ? REDO_OK : cuda_error(e, "mlp forward");
}

redo_status redo_mlp_backward(int32_t layers, const int32_t* sizes, const float* params,
                              const float* x, int64_t batch, const float* acts,
                              const float* y_target, float* grads, double* loss, float* work,
                              void* stream) {
  redo_status st = check_mlp(layers, sizes);
  if (st != REDO_OK) return st;
  if (batch < 1) return set_error(REDO_ERR_INVALID, "batch must be >= 1");
  if (!params || !x || !acts || !y_target || !grads || !work)
    return set_error(REDO_ERR_INVALID, "null pointer");
  cudaError_t e = mlp_backward(layers, sizes, params, x, batch, acts, y_target, grads, loss, work,
                               (cudaStream_t)stream);
  return e == cudaSuccess ? REDO_OK : cuda_error(e, "mlp backward");
}

redo_status redo_mlp_adam(int64_t count, float* params, const float* grads, float* m, float* v,
                          int32_t step, float lr, float beta1, float beta2, float eps,
                          void* stream) {
  if (count < 0 || step < 1) return set_error(REDO_ERR_INVALID, "count >= 0 and step >= 1");
  if (count == 0) return REDO_OK;
  if (!params || !grads || !m || !v) return set_error(REDO_ERR_INVALID, "null pointer");
  cudaError_t e = mlp_adam(count, params, grads, m, v, step, lr, beta1, beta2, eps,
                           (cudaStream_t)stream);
  return e == cudaSuccess ? REDO_OK : cuda_error(e, "adam");
}

redo_status redo_grape_lbfgs_workspace(const redo_table* t, int64_t B, int64_t M, int32_t history, size_t* bytes) {
  if (!t || !bytes) return set_error(REDO_ERR_INVALID, "null argument");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  if (history < 1 || history > 64) return set_error(REDO_ERR_INVALID, "history must be 1..64");
  *bytes = lbfgs_state_bytes(B, M * t->K, history);
  return REDO_OK;
}

redo_status redo_grape_lbfgs_step(const redo_table* t, double* u, const double* grad, const double* F, int64_t B,
                                  int64_t M, int32_t history, int32_t first, double step0, double c1, void* state,
                                  size_t state_bytes, double* u_best, double* F_best, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  if (history < 1 || history > 64) return set_error(REDO_ERR_INVALID, "history must be 1..64");
  if (!(step0 > 0.0) || !std::isfinite(step0) || !(c1 > 0.0 && c1 < 1.0))
    return set_error(REDO_ERR_INVALID, "step0 > 0 and 0 < c1 < 1 required");
  if (B == 0 || M == 0) return REDO_OK;
  if (!u || !grad || !F || !state) return set_error(REDO_ERR_INVALID, "null pointer");
  const size_t need = lbfgs_state_bytes(B, M * t->K, history);
  if (state_bytes < need) return set_error(REDO_ERR_INVALID, "state of %zu bytes needed", need);
  if (((uintptr_t)state & 255) != 0) return set_error(REDO_ERR_INVALID, "state not 256-byte aligned");
  cudaError_t e = launch_lbfgs_step(t, u, grad, F, B, M, history, first ? 1 : 0, step0, c1, state, u_best, F_best,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "grape L-BFGS step");
  return REDO_OK;
}

redo_status redo_grape_adam_step(const redo_table* t, double* u, const double* grad, double* m,
                                 double* v, int64_t B, int64_t M, int32_t step, double lr, double beta1,
                                 double beta2, double eps, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0 || step < 1) return set_error(REDO_ERR_INVALID, "B, M >= 0 and step >= 1");
  if (!std::isfinite(lr) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return set_error(REDO_ERR_INVALID, "bad Adam hyper-parameters");
  const int64_t count = B * M * t->K;
  if (count == 0) return REDO_OK;
  if (!u || !grad || !m || !v) return set_error(REDO_ERR_INVALID, "null pointer");
  cudaError_t e = launch_grape_adam(u, grad, m, v, count, t->K, t->d_lo, t->d_delta, t->levels, step,
                                    lr, beta1, beta2, eps, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "grape adam step");
  return REDO_OK;
}

redo_status redo_grape_step(const redo_table* t, double* u, const double* grad, int64_t B,
                            int64_t M, double step, const double* step_scale, void* stream) {
  if (!t) return set_error(REDO_ERR_INVALID, "table is NULL");
  if (B < 0 || M < 0) return set_error(REDO_ERR_INVALID, "negative B or M");
  if (!std::isfinite(step)) return set_error(REDO_ERR_INVALID, "step must be finite");
  const int64_t count = B * M * t->K;
  if (count == 0) return REDO_OK;
  if (!u || !grad) return set_error(REDO_ERR_INVALID, "null u or grad");
  cudaError_t e = launch_grape_step(u, grad, count, M * t->K, t->K, t->d_lo, t->d_delta,
                                    t->levels, step, step_scale, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "grape step");
  return REDO_OK;
}

}  // extern "C"
