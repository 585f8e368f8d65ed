// Amplitude/phase controls (Section III, Eq. vn and the Dirac-frame step after Eq. vnd).
//
// A drive of amplitude A_kn and phase phi_kn on species k is the x-polarised drive turned
// about z, so with one x-table per species the step is
//     U_n = Z_n E_n Z_n^dag D,   Z_n = exp(-i sum_k phi_kn S_kz),   E_n = E_{K-1,n} ... E_{0,n}.
// When D commutes with every S_kz the chain regroups as
//     U_M ... U_1 = Z_{M-1} (E'_M P_M) ... (E'_1 P_1),   P_n = Z_n^dag Z_{n-1},  E'_n = E_n D,
// (0-based steps in the code, Z_{-1} = I): the folded table serves unchanged and each step
// gains one diagonal factor.  These kernels evaluate the diagonals in FP64 and apply them
// where the chain kernels do not (the large-N chains and the final Z_{M-1}).
#include "redo_internal.cuh"

namespace redo {

namespace {

// one thread per (b, n, a): pd[b][n][a] = exp(i sum_k (phi[b][n][k] - phi[b][n-1][k]) sz[k][a]);
// the threads of step M (n == M) write zf[b][a] = exp(-i sum_k phi[b][M-1][k] sz[k][a]).
// With pd32 non-null the step diagonals are written in FP32 instead (for the split-FP16 chains):
// the angle is summed and reduced to [-pi, pi] in FP64, its sine and cosine taken in FP32.
__global__ void phase_diag_kernel(const double* __restrict__ phi, const double* __restrict__ sz, int64_t B,
                                  int64_t M, int K, int N, double2* __restrict__ pd, float2* __restrict__ pd32,
                                  double2* __restrict__ zf) {
  const int64_t total = B * (M + 1) * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % N);
    const int64_t bn = idx / N;
    const int64_t n = bn % (M + 1), b = bn / (M + 1);
    const double* cur = phi + (b * M + n) * K;
    double th = 0.0;
    if (n < M) {
      for (int k = 0; k < K; ++k) {
        const double prev = n > 0 ? cur[k - K] : 0.0;
        th += (cur[k] - prev) * sz[(int64_t)k * N + a];
      }
      if (pd32) {
        const double red = th - 6.283185307179586 * rint(th * 0.15915494309189535);
        float sf, cf;
        sincosf((float)red, &sf, &cf);
        pd32[(b * M + n) * N + a] = make_float2(cf, sf);
      } else {
        double sn, cs;
        sincos(th, &sn, &cs);
        pd[(b * M + n) * N + a] = make_double2(cs, sn);
      }
    } else {
      for (int k = 0; k < K && M > 0; ++k) th += cur[k - K] * sz[(int64_t)k * N + a];
      double sn, cs;
      sincos(th, &sn, &cs);
      zf[b * N + a] = make_double2(cs, -sn);
    }
  }
}

// Per-pulse diagonal drift: pd[b][n][a] = exp(-i dt h[b][a]) for every step n, so that each
// step reads U_n = E_n D diag(exp(-i dt h_b)) (the Lie split of the drift H0 + diag(h_b), exact
// when H0 is diagonal).  Each (b, a) takes its sine and cosine once, in FP64, and writes them
// for a run of kDriftSteps steps; pd32 non-null writes them in FP32 instead.
constexpr int64_t kDriftSteps = 64;

__global__ void drift_diag_kernel(const double* __restrict__ h, double dt, int64_t B, int64_t M, int N,
                                  double2* __restrict__ pd, float2* __restrict__ pd32) {
  const int64_t runs = (M + kDriftSteps - 1) / kDriftSteps;
  for (int64_t w = blockIdx.x; w < B * runs; w += gridDim.x) {
    const int64_t b = w / runs, n0 = (w % runs) * kDriftSteps;
    const int64_t n1 = n0 + kDriftSteps < M ? n0 + kDriftSteps : M;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      double sn, cs;
      sincos(dt * h[b * N + a], &sn, &cs);
      for (int64_t n = n0; n < n1; ++n) {
        if (pd32)
          pd32[(b * M + n) * N + a] = make_float2((float)cs, (float)-sn);
        else
          pd[(b * M + n) * N + a] = make_double2(cs, -sn);
      }
    }
  }
}

// X_g <- diag(pd[u][n]) X_g, n = s * sps + i, for the chains g = u * S + s with n < M
template <typename R>
__global__ void phase_rows_kernel(cplx<R>* __restrict__ X, int N, int64_t S, int64_t sps, int64_t i,
                                  int64_t M, const double2* __restrict__ pd) {
  const int64_t g = blockIdx.x;
  const int64_t u = g / S, sg = g - u * S;
  const int64_t n = sg * sps + i;
  if (n >= M) return;
  const int64_t n2 = (int64_t)N * N;
  cplx<R>* Xg = X + g * n2;
  const double2* p = pd + (u * M + n) * N;
  for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.y * blockDim.x) {
    const double2 pv = p[e / N];
    const cplx<R> x = Xg[e];
    const double xr = (double)x.x, xi = (double)x.y;
    Xg[e] = cmake<R>((R)(pv.x * xr - pv.y * xi), (R)(pv.x * xi + pv.y * xr));
  }
}

template <typename R>
__global__ void phase_final_kernel(const cplx<R>* __restrict__ X, int N, const double2* __restrict__ zf,
                                   double2* __restrict__ out) {
  const int64_t b = blockIdx.x;
  const int64_t n2 = (int64_t)N * N;
  for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.y * blockDim.x) {
    const double2 z = zf[b * N + e / N];
    const cplx<R> x = X[b * n2 + e];
    const double xr = (double)x.x, xi = (double)x.y;
    out[b * n2 + e] = make_double2(z.x * xr - z.y * xi, z.x * xi + z.y * xr);
  }
}

__global__ void phase_target_kernel(const double2* __restrict__ UT, int batched, int N,
                                    const double2* __restrict__ zf, double2* __restrict__ out) {
  const int64_t b = blockIdx.x;
  const int64_t n2 = (int64_t)N * N;
  const double2* U = UT + (batched ? b * n2 : 0);
  for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.y * blockDim.x) {
    const double2 z = zf[b * N + e / N];
    const double2 u = U[e];
    out[b * n2 + e] = make_double2(z.x * u.x + z.y * u.y, z.x * u.y - z.y * u.x);   // conj(z) u
  }
}

__global__ void phase_grad_finish_kernel(int N, int64_t B, int64_t M, int K, const double2* __restrict__ Tz,
                                         const double2* __restrict__ tau, double* __restrict__ gphi) {
  const int64_t total = B * M * K;
  const double scale = 2.0 / ((double)N * (double)N);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % K);
    const int64_t bn = idx / K;
    const int64_t n = bn % M, b = bn / M;
    const double2 t1 = Tz[(b * (M + 1) + n + 1) * K + k], t0 = Tz[(b * (M + 1) + n) * K + k];
    const double dr = t1.x - t0.x, di = t1.y - t0.y;
    const double2 ta = tau[b];
    gphi[idx] = scale * (ta.x * di - ta.y * dr);
  }
}

// Reverse sweeps of the large-N gradient (segments of whole steps, every chain at the same
// offset tt from its end): the chain's factor f = f1 - 1 - tt.  With tt = -1 the chain end itself
// (f = f1), a step boundary only for the last segment.
__device__ __forceinline__ int64_t boundary_factor(int64_t g, int64_t S, int64_t seg_len, int64_t F, int64_t tt,
                                                   int64_t* f0_out) {
  const int64_t sg = g % S;
  const int64_t f0 = sg * seg_len;
  const int64_t f1 = f0 + seg_len < F ? f0 + seg_len : F;
  *f0_out = f0;
  return f1 - 1 - tt;
}

// Tz[u][n][k] = sum_a sz[k][a] (P R)[a][a] at the boundary n = f / kd of every chain g = u S + s
// whose factor f opens step n (or, with tt = -1, at the end of the last segment: n = M).
template <typename R>
__global__ void __launch_bounds__(256) phase_boundary_tz_kernel(const cplx<R>* __restrict__ P,
                                                                const cplx<R>* __restrict__ Rm, int N, int64_t S,
                                                                int64_t seg_len, int64_t F, int64_t tt, int64_t kd,
                                                                int64_t M, const double* __restrict__ sz, int K,
                                                                double2* __restrict__ Tz) {
  __shared__ double2 dg[1024];
  const int64_t g = blockIdx.x;
  int64_t f0;
  const int64_t f = boundary_factor(g, S, seg_len, F, tt, &f0);
  if (tt < 0 ? f != F : (f < f0 || f % kd != 0)) return;
  const int64_t n = f / kd;
  const int64_t u = g / S;
  const int64_t n2 = (int64_t)N * N;
  const cplx<R>* Pg = P + g * n2;
  const cplx<R>* Rg = Rm + g * n2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int a = warp; a < N; a += 8) {
    double re = 0.0, im = 0.0;
    for (int x = lane; x < N; x += 32) {
      const cplx<R> pv = Pg[(int64_t)a * N + x], rv = Rg[(int64_t)x * N + a];
      re += (double)pv.x * rv.x - (double)pv.y * rv.y;
      im += (double)pv.x * rv.y + (double)pv.y * rv.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) dg[a] = make_double2(re, im);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int a = 0; a < N; ++a) {
      const double w = sz[(int64_t)k * N + a];
      re += w * dg[a].x;
      im += w * dg[a].y;
    }
    Tz[(u * (M + 1) + n) * K + k] = make_double2(re, im);
  }
}

// Undo the step-opening diagonal P_n of every chain at a boundary: P <- diag(p_n)^dag P,
// R <- R diag(p_n).
template <typename R>
__global__ void phase_undo_kernel(cplx<R>* __restrict__ P, cplx<R>* __restrict__ Rm, int N, int64_t S,
                                  int64_t seg_len, int64_t F, int64_t tt, int64_t kd, int64_t M,
                                  const double2* __restrict__ pd) {
  const int64_t g = blockIdx.x;
  int64_t f0;
  const int64_t f = boundary_factor(g, S, seg_len, F, tt, &f0);
  if (f < f0 || f % kd != 0) return;
  const int64_t n = f / kd, u = g / S;
  const int64_t n2 = (int64_t)N * N;
  const double2* p = pd + (u * M + n) * N;
  cplx<R>* Pg = P + g * n2;
  cplx<R>* Rg = Rm + g * n2;
  for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.y * blockDim.x) {
    const double2 pr = p[e / N], pc = p[e % N];
    const cplx<R> x = Pg[e], y = Rg[e];
    Pg[e] = cmake<R>((R)(pr.x * (double)x.x + pr.y * (double)x.y), (R)(pr.x * (double)x.y - pr.y * (double)x.x));
    Rg[e] = cmake<R>((R)(pc.x * (double)y.x - pc.y * (double)y.y), (R)(pc.x * (double)y.y + pc.y * (double)y.x));
  }
}

unsigned grid_y(int64_t n2) {
  int64_t b = (n2 + 255) / 256;
  if (b > 64) b = 64;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_phase_diag(const redo_table* t, const double* phi, int64_t B, int64_t M, double2* pd,
                              float2* pd32, double2* zf, cudaStream_t s) {
  const int64_t total = B * (M + 1) * t->N;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)t->num_sms * 32) blocks = (int64_t)t->num_sms * 32;
  phase_diag_kernel<<<(unsigned)blocks, 256, 0, s>>>(phi, t->sz64, B, M, t->K, t->N, pd, pd32, zf);
  return cudaGetLastError();
}

cudaError_t launch_drift_diag(const redo_table* t, const double* h, int64_t B, int64_t M, double2* pd,
                              float2* pd32, cudaStream_t s) {
  const int64_t work = B * ((M + kDriftSteps - 1) / kDriftSteps);
  if (work == 0) return cudaSuccess;
  const int64_t blocks = work < (int64_t)t->num_sms * 16 ? work : (int64_t)t->num_sms * 16;
  drift_diag_kernel<<<(unsigned)blocks, 128, 0, s>>>(h, t->dt, B, M, t->N, pd, pd32);
  return cudaGetLastError();
}

cudaError_t launch_phase_rows(int N, int prec, void* X, int64_t G, int64_t S, int64_t sps, int64_t i,
                              int64_t M, const double2* pd, cudaStream_t s) {
  if (G == 0) return cudaSuccess;
  const dim3 grid((unsigned)G, grid_y((int64_t)N * N));
  if (prec == REDO_FP64)
    phase_rows_kernel<double><<<grid, 256, 0, s>>>((double2*)X, N, S, sps, i, M, pd);
  else
    phase_rows_kernel<float><<<grid, 256, 0, s>>>((float2*)X, N, S, sps, i, M, pd);
  return cudaGetLastError();
}

cudaError_t launch_phase_target(int N, int64_t B, const double2* UT, int batched, const double2* zf, double2* out,
                                cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  phase_target_kernel<<<dim3((unsigned)B, grid_y((int64_t)N * N)), 256, 0, s>>>(UT, batched, N, zf, out);
  return cudaGetLastError();
}

cudaError_t launch_phase_grad_finish(int N, int64_t B, int64_t M, int K, const double2* Tz, const double2* tau,
                                     double* gphi, cudaStream_t s) {
  const int64_t total = B * M * K;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  phase_grad_finish_kernel<<<(unsigned)blocks, 256, 0, s>>>(N, B, M, K, Tz, tau, gphi);
  return cudaGetLastError();
}

cudaError_t launch_phase_boundary(int N, int prec, void* P, void* Rm, int64_t G, int64_t S, int64_t seg_len,
                                  int64_t F, int64_t tt, int64_t kd, int64_t M, const double2* pd, const double* sz,
                                  int K, double2* Tz, cudaStream_t s) {
  if (G == 0) return cudaSuccess;
  if (prec == REDO_FP64) {
    if (Tz)
      phase_boundary_tz_kernel<double><<<(unsigned)G, 256, 0, s>>>((const double2*)P, (const double2*)Rm, N, S,
                                                                    seg_len, F, tt, kd, M, sz, K, Tz);
    if (tt >= 0)
      phase_undo_kernel<double><<<dim3((unsigned)G, grid_y((int64_t)N * N)), 256, 0, s>>>(
          (double2*)P, (double2*)Rm, N, S, seg_len, F, tt, kd, M, pd);
  } else {
    if (Tz)
      phase_boundary_tz_kernel<float><<<(unsigned)G, 256, 0, s>>>((const float2*)P, (const float2*)Rm, N, S,
                                                                   seg_len, F, tt, kd, M, sz, K, Tz);
    if (tt >= 0)
      phase_undo_kernel<float><<<dim3((unsigned)G, grid_y((int64_t)N * N)), 256, 0, s>>>(
          (float2*)P, (float2*)Rm, N, S, seg_len, F, tt, kd, M, pd);
  }
  return cudaGetLastError();
}

cudaError_t launch_phase_final(int N, int64_t B, int prec, const void* X, const double2* zf, double2* out,
                               cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const dim3 grid((unsigned)B, grid_y((int64_t)N * N));
  if (prec == REDO_FP64)
    phase_final_kernel<double><<<grid, 256, 0, s>>>((const double2*)X, N, zf, out);
  else
    phase_final_kernel<float><<<grid, 256, 0, s>>>((const float2*)X, N, zf, out);
  return cudaGetLastError();
}

}  // namespace redo
