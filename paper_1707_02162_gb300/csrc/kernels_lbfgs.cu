// GRAPE update by projected L-BFGS with Armijo backtracking (Section III's ascent loop, Fig. fc;
// the paper leaves the update rule open).  One CTA per pulse: every step is a handful of block
// reductions and element-wise passes over the pulse's M*K coefficients, with the pulse's pair
// history (a ring of s and y vectors) in global memory.
//
// For f = -F (gradient -g) the pair of an accepted step is s = u_new - u, y = -(g_new - g); the
// direction is the two-loop recursion of Nocedal & Wright (Algorithm 7.4) with H0 = gamma I,
// gamma = s.y / y.y of the newest pair, negated into an ascent direction for F.
#include "redo_internal.cuh"

namespace redo {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct Bounds {
  double lo[kMaxK], hi[kMaxK];
};

// Sum over the block of one double per thread (fixed order: warps, then warp partials).
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) t += red[i];
  return t;
}

__device__ double block_max(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) t = fmax(t, red[i]);
  return t;
}

__global__ void __launch_bounds__(kThreads) lbfgs_step_kernel(
    double* __restrict__ u, const double* __restrict__ gt, const double* __restrict__ Ft, int64_t n, int K,
    int hist, int first, double step0, double span, double c1, Bounds bd, LbfgsState st,
    double* __restrict__ u_best, double* __restrict__ F_best) {
  __shared__ double red[kWarps];
  __shared__ double a_s[64];
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  double* ut = u + b * n;                       // in: the evaluated point; out: the next one
  const double* g_t = gt + b * n;
  double* ua = st.u + b * n;
  double* ga = st.g + b * n;
  double* d = st.d + b * n;
  double* S = st.S + b * (int64_t)hist * n;
  double* Y = st.Y + b * (int64_t)hist * n;
  double* rho = st.rho + b * hist;
  double& F = st.F[b];
  double& alpha = st.alpha[b];
  int& count = st.count[b];
  int& head = st.head[b];
  const double ft = Ft[b];
  bool new_dir = false;
  if (first) {
    for (int64_t i = tid; i < n; i += kThreads) {
      ua[i] = ut[i];
      ga[i] = g_t[i];
    }
    if (tid == 0) {
      F = ft;
      count = 0;
      head = hist - 1;
    }
    new_dir = true;
  } else {
    double gp = 0.0;
    for (int64_t i = tid; i < n; i += kThreads) gp += ga[i] * (ut[i] - ua[i]);
    gp = block_sum(gp, red);
    const double Fa = F;
    if (ft >= Fa + c1 * gp) {
      // accepted: the pair (s, y), stored when s.y > 0
      double sy = 0.0;
      for (int64_t i = tid; i < n; i += kThreads) sy += (ut[i] - ua[i]) * -(g_t[i] - ga[i]);
      sy = block_sum(sy, red);
      if (sy > 0.0) {
        const int slot = (head + 1) % hist;
        for (int64_t i = tid; i < n; i += kThreads) {
          S[(int64_t)slot * n + i] = ut[i] - ua[i];
          Y[(int64_t)slot * n + i] = -(g_t[i] - ga[i]);
        }
        __syncthreads();
        if (tid == 0) {
          rho[slot] = 1.0 / sy;
          head = slot;
          count = count < hist ? count + 1 : hist;
        }
      }
      for (int64_t i = tid; i < n; i += kThreads) {
        ua[i] = ut[i];
        ga[i] = g_t[i];
      }
      if (tid == 0) F = ft;
      new_dir = true;
    } else {
      const double a2 = alpha * 0.5;
      __syncthreads();
      if (tid == 0) alpha = a2;
      if (a2 < 1e-3) {
        if (tid == 0) count = 0;
        new_dir = true;
      }
    }
  }
  __syncthreads();
  if (new_dir) {
    const int cnt = count, hd = head;
    bool grad_dir = cnt == 0;
    if (!grad_dir) {
      // q = -g (the gradient of f) in d; first loop newest to oldest
      for (int64_t i = tid; i < n; i += kThreads) d[i] = -ga[i];
      for (int j = 0; j < cnt; ++j) {
        const int slot = (hd - j + hist) % hist;
        const double* s = S + (int64_t)slot * n;
        const double* y = Y + (int64_t)slot * n;
        double sq = 0.0;
        for (int64_t i = tid; i < n; i += kThreads) sq += s[i] * d[i];
        const double a = rho[slot] * block_sum(sq, red);
        if (tid == 0) a_s[slot] = a;
        for (int64_t i = tid; i < n; i += kThreads) d[i] -= a * y[i];
      }
      // r = gamma q, gamma = s.y / y.y of the newest pair
      {
        const double* y = Y + (int64_t)hd * n;
        double yy = 0.0;
        for (int64_t i = tid; i < n; i += kThreads) yy += y[i] * y[i];
        yy = block_sum(yy, red);
        const double gamma = (1.0 / rho[hd]) / yy;
        for (int64_t i = tid; i < n; i += kThreads) d[i] *= gamma;
      }
      // second loop oldest to newest
      for (int j = cnt - 1; j >= 0; --j) {
        const int slot = (hd - j + hist) % hist;
        const double* s = S + (int64_t)slot * n;
        const double* y = Y + (int64_t)slot * n;
        double yr = 0.0;
        for (int64_t i = tid; i < n; i += kThreads) yr += y[i] * d[i];
        const double beta = rho[slot] * block_sum(yr, red);
        const double coef = a_s[slot] - beta;
        for (int64_t i = tid; i < n; i += kThreads) d[i] += coef * s[i];
      }
      // ascent direction for F; not an ascent direction: drop the pairs, use the gradient
      double gd = 0.0;
      for (int64_t i = tid; i < n; i += kThreads) {
        d[i] = -d[i];
        gd += ga[i] * d[i];
      }
      gd = block_sum(gd, red);
      if (!(gd > 0.0)) {
        grad_dir = true;
        if (tid == 0) count = 0;
      }
    }
    if (grad_dir) {
      double m = 0.0;
      for (int64_t i = tid; i < n; i += kThreads) m = fmax(m, fabs(ga[i]));
      m = block_max(m, red);
      const double sc = m > 0.0 ? step0 * span / m : 0.0;
      for (int64_t i = tid; i < n; i += kThreads) d[i] = ga[i] * sc;
    }
    __syncthreads();
    if (tid == 0) alpha = 1.0;
  }
  __syncthreads();
  const double al = alpha;
  for (int64_t i = tid; i < n; i += kThreads) {
    const int k = (int)(i % K);
    double x = ua[i] + al * d[i];
    x = x < bd.lo[k] ? bd.lo[k] : (x > bd.hi[k] ? bd.hi[k] : x);
    ut[i] = x;
    if (u_best) u_best[b * n + i] = ua[i];
  }
  if (F_best && tid == 0) F_best[b] = F;
}

}  // namespace

size_t lbfgs_state_bytes(int64_t B, int64_t n, int hist) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up((size_t)B * n * 8) * 3 + up((size_t)B * hist * n * 8) * 2 + up((size_t)B * hist * 8) +
         up((size_t)B * 8) * 2 + up((size_t)B * 4) * 2;
}

LbfgsState lbfgs_state_layout(void* base, int64_t B, int64_t n, int hist) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = (char*)base;
  LbfgsState s;
  s.u = (double*)p;
  p += up((size_t)B * n * 8);
  s.g = (double*)p;
  p += up((size_t)B * n * 8);
  s.d = (double*)p;
  p += up((size_t)B * n * 8);
  s.S = (double*)p;
  p += up((size_t)B * hist * n * 8);
  s.Y = (double*)p;
  p += up((size_t)B * hist * n * 8);
  s.rho = (double*)p;
  p += up((size_t)B * hist * 8);
  s.F = (double*)p;
  p += up((size_t)B * 8);
  s.alpha = (double*)p;
  p += up((size_t)B * 8);
  s.count = (int*)p;
  p += up((size_t)B * 4);
  s.head = (int*)p;
  return s;
}

cudaError_t launch_lbfgs_step(const redo_table* t, double* u, const double* g, const double* F, int64_t B,
                              int64_t M, int hist, int first, double step0, double c1, void* state,
                              double* u_best, double* F_best, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  Bounds bd{};
  double span = 0.0;
  for (int k = 0; k < t->K; ++k) {
    bd.lo[k] = t->lo[k];
    bd.hi[k] = t->hi[k];
    span = fmax(span, 0.5 * (t->hi[k] - t->lo[k]));
  }
  const int64_t n = M * t->K;
  const LbfgsState st = lbfgs_state_layout(state, B, n, hist);
  lbfgs_step_kernel<<<(unsigned)B, kThreads, 0, s>>>(u, g, F, n, t->K, hist, first, step0, span, c1, bd, st,
                                                     u_best, F_best);
  return cudaGetLastError();
}

}  // namespace redo
