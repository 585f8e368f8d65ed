// Large-N path (N = 128 ... 1024, powers of two): operators and states live in
// global memory and every product is a batched complex GEMM, one launch per
// chain step over all chains at once ("lockstep" chains).  SIMT FP64/FP32.
// (Section II processes 1 and 2 -- the table and the products of Eq. exp2prod -- and the
// Section III chain U = U_M ... U_1, gradient and Section IV dynamics for large N.)
//
// Everything the N <= 64 path does in shared memory is expressed here with
// one GEMM kernel, templated on a small functor that names the three
// matrices of batch item b (gathered table operators, checkpoints, states):
//     C_b = alpha * opA(A_b) B_b + diag * I,    opA = A or A^dag.
// A null A_b means "identity": the tile of B_b is copied to C_b (chains whose
// segment ended early pass their state through).
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "redo_internal.cuh"

namespace redo {
namespace large {

constexpr int kT = 64;    // output tile (complex)
constexpr int kBK = 16;   // K chunk

template <typename R, bool ADJA, class Ops>
__global__ void __launch_bounds__(256) cgemm_kernel(Ops ops, int N, R alpha, R diag) {
  __shared__ cplx<R> As[kBK][kT + 1];
  __shared__ cplx<R> Bs[kBK][kT + 1];
  // blockIdx.x = (batch item, row tile, column tile)
  const int tiles = N / kT;
  const int64_t b = blockIdx.x / ((int64_t)tiles * tiles);
  const int tile = (int)(blockIdx.x % ((int64_t)tiles * tiles));
  const cplx<R>* A;
  const cplx<R>* Bm;
  cplx<R>* C;
  ops.get(b, A, Bm, C);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = (tile / tiles) * kT, j0 = (tile % tiles) * kT;
  if (C == nullptr) return;
  if (A == nullptr) {
    // identity: copy the tile
    for (int e = tid; e < kT * kT; e += 256) {
      const int r = e / kT, c = e % kT;
      C[(int64_t)(i0 + r) * N + j0 + c] = Bm[(int64_t)(i0 + r) * N + j0 + c];
    }
    return;
  }
  cplx<R> acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = cmake<R>(R(0), R(0));
  for (int k0 = 0; k0 < N; k0 += kBK) {
#pragma unroll
    for (int x = 0; x < (kT * kBK) / 256; ++x) {
      const int e = tid + 256 * x;
      if (!ADJA) {
        const int r = e / kBK, kk = e % kBK;
        As[kk][r] = A[(int64_t)(i0 + r) * N + k0 + kk];
      } else {
        const int kk = e / kT, r = e % kT;
        const cplx<R> v = A[(int64_t)(k0 + kk) * N + i0 + r];
        As[kk][r] = cmake<R>(v.x, -v.y);
      }
      const int kb = e / kT, c = e % kT;
      Bs[kb][c] = Bm[(int64_t)(k0 + kb) * N + j0 + c];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      cplx<R> a[4], bb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cfma<R>(acc[r][c], a[r], bb[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      C[(int64_t)i * N + j] = cmake<R>(alpha * acc[r][c].x + (i == j ? diag : R(0)), alpha * acc[r][c].y);
    }
}

template <typename R, bool ADJA, class Ops>
static cudaError_t cgemm(const Ops& ops, int64_t batch, int N, R alpha, R diag, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  const int64_t blocks = batch * (N / kT) * (N / kT);
  cgemm_kernel<R, ADJA, Ops><<<(unsigned)blocks, 256, 0, s>>>(ops, N, alpha, diag);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------- functors

// Strided dense batches: A_b = A + b*sA etc. (sA = 0 broadcasts one matrix)
template <typename R>
struct DenseOps {
  const cplx<R>* A;
  const cplx<R>* B;
  cplx<R>* C;
  int64_t sA, sB, sC;
  __device__ void get(int64_t b, const cplx<R>*& a, const cplx<R>*& bb, cplx<R>*& c) const {
    a = A + b * sA;
    bb = B + b * sB;
    c = C + b * sC;
  }
};

// Index lists: C[ic[b]] = A[ia[b]] * B[ib[b]] within one array of matrices.
template <typename R>
struct IndexOps {
  const cplx<R>* A;
  const cplx<R>* B;
  cplx<R>* C;
  const int32_t* ia;
  const int32_t* ib;
  const int32_t* ic;
  int64_t n2;
  __device__ void get(int64_t b, const cplx<R>*& a, const cplx<R>*& bb, cplx<R>*& c) const {
    a = A + (int64_t)ia[b] * n2;
    bb = B + (int64_t)ib[b] * n2;
    c = C + (int64_t)ic[b] * n2;
  }
};

// Gathered table factor f of chain g (segment s of unit u):
//   gather_left:  C_g = A_f X_g    (forward step, or A_f^dag P_g with ADJA)
//   gather_right: C_g = X_g A_f    (costate step)
// `t` counts steps from the segment start (forward) or from its end (reverse).
template <typename R>
struct GatherStepOps {
  const cplx<R>* T;
  const int32_t* q;
  int64_t M;
  int K, d, base;
  int64_t levels;
  int64_t S, seg_len, F;
  int64_t t;
  bool reverse;
  bool right;
  const cplx<R>* X;
  cplx<R>* Y;
  int64_t n2;
  int64_t* status;
  __device__ const cplx<R>* factor(int64_t g) const {
    const int64_t u = g / S, s = g % S;
    const int64_t f0 = s * seg_len;
    int64_t f1 = f0 + seg_len;
    if (f1 > F) f1 = F;
    const int64_t f = reverse ? f1 - 1 - t : f0 + t;
    if (f < f0 || f >= f1) return nullptr;
    const int64_t kd = (int64_t)K * d;
    const int64_t n = f / kd;
    const int r = (int)(f - n * kd);
    const int k = r / d, j = r - k * d;
    int32_t qv = q[(u * M + n) * K + k];
    if (qv < 0 || qv >= levels) {
      if (status && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0)
        atomicAdd((unsigned long long*)&status[REDO_STATUS_BADINDEX], 1ull);
      qv = 0;
    }
    for (int i = 0; i < j; ++i) qv /= base;
    return T + ((int64_t)(k * d + j) * base + qv % base) * n2;
  }
  __device__ void get(int64_t g, const cplx<R>*& a, const cplx<R>*& bb, cplx<R>*& c) const {
    const cplx<R>* A = factor(g);
    c = Y + g * n2;
    if (!right) {
      a = A;
      bb = X + g * n2;
    } else if (A == nullptr) {
      a = nullptr;                 // identity on the right: pass X through
      bb = X + g * n2;
    } else {
      a = X + g * n2;
      bb = A;
    }
  }
};

// Dense step over a list of per-unit matrices: C_u = L_u[t] X_u (left) or X_u L_u[t] (right)
template <typename R>
struct ListStepOps {
  const cplx<R>* L;
  int64_t per_unit;
  int64_t t;
  bool right;
  const cplx<R>* X;
  cplx<R>* Y;
  int64_t n2;
  __device__ void get(int64_t u, const cplx<R>*& a, const cplx<R>*& bb, cplx<R>*& c) const {
    const cplx<R>* Lm = L + (u * per_unit + t) * n2;
    c = Y + u * n2;
    if (!right) {
      a = Lm;
      bb = X + u * n2;
    } else {
      a = X + u * n2;
      bb = Lm;
    }
  }
};

// --------------------------------------------------------------------------- elementwise

template <typename R>
__global__ void set_identity_kernel(cplx<R>* X, int64_t count, int N) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count * n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i % n2;
    X[i] = cmake<R>((e / N == e % N) ? R(1) : R(0), R(0));
  }
}

template <typename R>
__global__ void copy_kernel(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Q = 1.5 I - 0.5 G (Newton-Schulz)
template <typename R>
__global__ void ns_mid_kernel(cplx<R>* G, int64_t count, int N) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count * n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i % n2;
    const cplx<R> g = G[i];
    G[i] = cmake<R>(((e / N == e % N) ? R(1.5) : R(0)) - R(0.5) * g.x, -R(0.5) * g.y);
  }
}

template <typename Rin, typename Rout>
__global__ void convert_kernel(const cplx<Rin>* __restrict__ src, cplx<Rout>* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = cmake<Rout>((Rout)src[i].x, (Rout)src[i].y);
}

// X_b = -i c_b H_{k_b}  (scaled generators for the Taylor series)
__global__ void scaled_generator_kernel(const double2* __restrict__ Hk, const int32_t* __restrict__ kidx,
                                        const double* __restrict__ coef, double2* __restrict__ X,
                                        int64_t count, int64_t n2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count * n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / n2, e = i % n2;
    const double2 h = Hk[(int64_t)kidx[b] * n2 + e];
    const double c = coef[b];
    X[i] = make_double2(c * h.y, -c * h.x);
  }
}

static unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

template <typename R>
static cudaError_t set_identity(cplx<R>* X, int64_t count, int N, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  set_identity_kernel<R><<<blocks_for(count * N * N), 256, 0, s>>>(X, count, N);
  return cudaGetLastError();
}

}  // namespace large

using namespace large;

// ============================================================================
// Table: exponentials by scaling and squaring Taylor series (batched GEMMs),
// then digit powers  T[k][j][c] = E_kj^c  (j >= 1, E_kj = exp(-i dt c b^j delta H_k)
// at c = 1) and  T[k][0][c] = S_k^c O_k  (S_k = exp(-i dt delta H_k),
// O_k = exp(-i dt lo_k H_k)), powers by a binary tree (c = 2^l + r  ->
// P[2^l] P[r]); finally T[0][0][c] <- T[0][0][c] D.
// ============================================================================
static cudaError_t batched_expm(int N, const double2* Hk, const std::vector<int32_t>& kidx,
                                const std::vector<double>& coef, const std::vector<double>& hnorm1,
                                double2* out, double2* work, int32_t* d_kidx, double* d_coef,
                                cudaStream_t s) {
  // exp(-i coef_b H_{k_b}) for every b; work holds X (count matrices) and a ping buffer
  const int64_t count = (int64_t)kidx.size();
  const int64_t n2 = (int64_t)N * N;
  double nrm = 0.0;
  for (int64_t b = 0; b < count; ++b) nrm = std::fmax(nrm, std::fabs(coef[b]) * hnorm1[kidx[b]]);
  int sq = 0;
  while (nrm > 0.5 && sq < 60) {
    nrm *= 0.5;
    ++sq;
  }
  int m = 0;
  if (nrm > 0.0) {
    double term = nrm * nrm / 2.0;
    m = 1;
    while (term > 1e-18 && m < 30) {
      ++m;
      term = term * nrm / (double)(m + 1);
    }
  }
  std::vector<double> c2(coef);
  for (auto& c : c2) c = std::ldexp(c, -sq);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_kidx, kidx.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(d_coef, c2.data(), sizeof(double) * count, cudaMemcpyHostToDevice, s)))
    return e;
  double2* X = work;
  double2* tmp = work + count * n2;
  scaled_generator_kernel<<<blocks_for(count * n2), 256, 0, s>>>(Hk, d_kidx, d_coef, X, count, n2);
  if ((e = set_identity<double>(out, count, N, s))) return e;
  DenseOps<double> op{X, out, tmp, n2, n2, n2};
  for (int it = m; it >= 1; --it) {
    // out = I + X out / it
    if ((e = cgemm<double, false>(op, count, N, 1.0 / it, 1.0, s))) return e;
    copy_kernel<double><<<blocks_for(count * n2), 256, 0, s>>>(tmp, out, count * n2);
  }
  DenseOps<double> sqop{out, out, tmp, n2, n2, n2};
  for (int it = 0; it < sq; ++it) {
    if ((e = cgemm<double, false>(sqop, count, N, 1.0, 0.0, s))) return e;
    copy_kernel<double><<<blocks_for(count * n2), 256, 0, s>>>(tmp, out, count * n2);
  }
  return cudaGetLastError();
}

cudaError_t large_table_build(redo_table* t, const double2* H0, const double2* Hk,
                              const std::vector<double>& hnorm1, double h0norm1, cudaStream_t s) {
  const int N = t->N, K = t->K, d = t->digits, base = t->base;
  const int64_t n2 = (int64_t)N * N;
  // exponentials: per k: O_k (lo), S_k (delta), E_kj (j >= 1); plus the drift
  std::vector<int32_t> kidx;
  std::vector<double> coef;
  for (int k = 0; k < K; ++k) {
    kidx.push_back(k);
    coef.push_back(t->dt * t->lo[k]);
    kidx.push_back(k);
    coef.push_back(t->dt * t->delta[k]);
    double bj = 1.0;
    for (int j = 1; j < d; ++j) {
      bj *= base;
      kidx.push_back(k);
      coef.push_back(t->dt * (bj * t->delta[k]));
    }
  }
  const int64_t ne = (int64_t)kidx.size();   // K * (d + 1)
  double2 *ex = nullptr, *work = nullptr, *tmp = nullptr;
  int32_t* d_idx = nullptr;
  double* d_coef = nullptr;
  int32_t *ia = nullptr, *ib = nullptr, *ic = nullptr;
  cudaError_t e;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    cudaFree(ex);
    cudaFree(work);
    cudaFree(tmp);
    cudaFree(d_idx);
    cudaFree(d_coef);
    cudaFree(ia);
    cudaFree(ib);
    cudaFree(ic);
  };
  const int64_t nb = (int64_t)K * d * base;
  if ((e = cudaMalloc(&ex, sizeof(double2) * n2 * ne)) ||
      (e = cudaMalloc(&work, sizeof(double2) * n2 * 2 * (ne > 1 ? ne : 1))) ||
      (e = cudaMalloc(&tmp, sizeof(double2) * n2 * base)) ||
      (e = cudaMalloc(&d_idx, sizeof(int32_t) * (ne + 1))) ||
      (e = cudaMalloc(&d_coef, sizeof(double) * (ne + 1))) ||
      (e = cudaMalloc(&ia, sizeof(int32_t) * nb)) || (e = cudaMalloc(&ib, sizeof(int32_t) * nb)) ||
      (e = cudaMalloc(&ic, sizeof(int32_t) * nb))) {
    cleanup();
    return e;
  }
  if ((e = batched_expm(N, Hk, kidx, coef, hnorm1, ex, work, d_idx, d_coef, s))) {
    cleanup();
    return e;
  }
  {
    // drift D = exp(-i dt H0)
    std::vector<int32_t> k0{0};
    std::vector<double> c0{t->dt};
    std::vector<double> hn{h0norm1};
    if ((e = batched_expm(N, H0, k0, c0, hn, t->D64, work, d_idx, d_coef, s))) {
      cleanup();
      return e;
    }
    // half drift exp(-i dt/2 H0) of the symmetric split
    std::vector<double> ch{0.5 * t->dt};
    if (t->Dh64 && (e = batched_expm(N, H0, k0, ch, hn, t->Dh64, work, d_idx, d_coef, s))) {
      cleanup();
      return e;
    }
  }
  // digit powers: slot (k, j, 1) = generator G_kj (S_k for j = 0), slot c = 0 identity
  double2* T = t->T64;
  auto slot = [&](int k, int j, int c) { return ((int64_t)(k * d + j) * base + c); };
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < d; ++j) {
      if ((e = set_identity<double>(T + slot(k, j, 0) * n2, 1, N, s))) { cleanup(); return e; }
      const int64_t src = (int64_t)k * (d + 1) + (j == 0 ? 1 : j + 1);
      if (base > 1)
        copy_kernel<double><<<blocks_for(n2), 256, 0, s>>>(ex + src * n2, T + slot(k, j, 1) * n2, n2);
    }
  // powers: level p2 = 2, 4, 8, ...: P[p2] = P[p2/2]^2, then P[c] = P[c - p2] P[p2] for
  // p2 < c < 2 p2 (both factors computed at earlier levels; powers commute)
  for (int p2 = 2; p2 < base; p2 *= 2) {
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<int32_t> A_, B_, C_;
      for (int k = 0; k < K; ++k)
        for (int j = 0; j < d; ++j) {
          if (pass == 0) {
            A_.push_back((int32_t)slot(k, j, p2 / 2));
            B_.push_back((int32_t)slot(k, j, p2 / 2));
            C_.push_back((int32_t)slot(k, j, p2));
          } else {
            for (int c = p2 + 1; c < 2 * p2 && c < base; ++c) {
              A_.push_back((int32_t)slot(k, j, c - p2));
              B_.push_back((int32_t)slot(k, j, p2));
              C_.push_back((int32_t)slot(k, j, c));
            }
          }
        }
      const int64_t cnt = (int64_t)C_.size();
      if (cnt == 0) continue;
      if ((e = cudaMemcpyAsync(ia, A_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)) ||
          (e = cudaMemcpyAsync(ib, B_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)) ||
          (e = cudaMemcpyAsync(ic, C_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s))) {
        cleanup();
        return e;
      }
      IndexOps<double> op{T, T, T, ia, ib, ic, n2};
      if ((e = cgemm<double, false>(op, cnt, N, 1.0, 0.0, s))) { cleanup(); return e; }
      if ((e = cudaStreamSynchronize(s))) { cleanup(); return e; }   // index buffers are reused
    }
  }
  // digit 0 offset and drift: T[k][0][c] <- S_k^c O_k ; T[0][0][c] <- T[0][0][c] D
  for (int k = 0; k < K; ++k) {
    DenseOps<double> op{T + slot(k, 0, 0) * n2, ex + (int64_t)k * (d + 1) * n2, tmp, n2, 0, n2};
    if ((e = cgemm<double, false>(op, base, N, 1.0, 0.0, s))) { cleanup(); return e; }
    if (k == 0) {
      DenseOps<double> op2{tmp, t->D64, T + slot(0, 0, 0) * n2, n2, 0, n2};
      if ((e = cgemm<double, false>(op2, base, N, 1.0, 0.0, s))) { cleanup(); return e; }
    } else {
      copy_kernel<double><<<blocks_for(n2 * base), 256, 0, s>>>(tmp, T + slot(k, 0, 0) * n2, n2 * base);
    }
  }
  e = cudaStreamSynchronize(s);
  cleanup();
  return e;
}

// Level operators (process 3) for large N: E[k][q] = T[k][d-1][c_{d-1}] ... T[k][0][c_0],
// built with batched GEMMs over chunks of levels (two chunk-sized ping-pong buffers).
cudaError_t large_table_expand(const redo_table* t, double2* E, cudaStream_t s) {
  const int N = t->N, K = t->K, d = t->digits, base = t->base;
  const int64_t n2 = (int64_t)N * N, L = t->levels;
  const int64_t chunk = L < 1024 ? L : 1024;
  double2* buf = nullptr;
  int32_t *ia = nullptr, *ib = nullptr, *ic = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&buf, sizeof(double2) * n2 * chunk)) || (e = cudaMalloc(&ia, sizeof(int32_t) * chunk)) ||
      (e = cudaMalloc(&ib, sizeof(int32_t) * chunk)) || (e = cudaMalloc(&ic, sizeof(int32_t) * chunk))) {
    cudaFree(buf);
    cudaFree(ia);
    cudaFree(ib);
    cudaFree(ic);
    return e;
  }
  std::vector<int32_t> A_(chunk), B_(chunk), C_(chunk);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    for (int64_t q0 = 0; q0 < L && e == cudaSuccess; q0 += chunk) {
      const int64_t cnt = (q0 + chunk <= L) ? chunk : L - q0;
      double2* dst = E + ((int64_t)k * L + q0) * n2;
      // start: digit-0 operators (the product accumulates into dst / buf alternately)
      double2* cur = (d % 2 == 1) ? dst : buf;
      double2* nxt = (d % 2 == 1) ? buf : dst;
      for (int64_t i = 0; i < cnt; ++i) {
        A_[i] = (int32_t)((int64_t)(k * d + 0) * base + (q0 + i) % base);
        C_[i] = (int32_t)i;
      }
      if ((e = cudaMemcpyAsync(ia, A_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)) ||
          (e = cudaMemcpyAsync(ic, C_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)))
        break;
      for (int64_t i = 0; i < cnt; ++i) {
        const double2* src = t->T64 + (int64_t)A_[i] * n2;
        if ((e = cudaMemcpyAsync(cur + i * n2, src, sizeof(double2) * n2, cudaMemcpyDeviceToDevice, s))) break;
      }
      for (int j = 1; j < d && e == cudaSuccess; ++j) {
        int64_t bj = 1;
        for (int x = 0; x < j; ++x) bj *= base;
        for (int64_t i = 0; i < cnt; ++i) {
          A_[i] = (int32_t)((int64_t)(k * d + j) * base + ((q0 + i) / bj) % base);
          B_[i] = (int32_t)i;
          C_[i] = (int32_t)i;
        }
        if ((e = cudaMemcpyAsync(ia, A_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(ib, B_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemcpyAsync(ic, C_.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s)))
          break;
        // A from the table, B and C chunk-relative (IndexOps with separate base pointers)
        IndexOps<double> op{t->T64, cur, nxt, ia, ib, ic, n2};
        if ((e = cgemm<double, false>(op, cnt, N, 1.0, 0.0, s))) break;
        if ((e = cudaStreamSynchronize(s))) break;    // host index vectors are reused
        std::swap(cur, nxt);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(buf);
  cudaFree(ia);
  cudaFree(ib);
  cudaFree(ic);
  return e;
}

// ============================================================================
// Chains, combine, re-unitarisation
// ============================================================================
template <typename R>
static cudaError_t large_chain_t(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                 cplx<R>* seg, cplx<R>* ping, int64_t* status, cudaStream_t s) {
  const int N = t->N;
  const int64_t n2 = (int64_t)N * N, G = p.B * p.S;
  GatherStepOps<R> op{};
  op.T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  op.q = q;
  op.M = p.M;
  op.K = t->K;
  op.d = t->digits;
  op.base = t->base;
  op.levels = t->levels;
  op.S = p.S;
  op.seg_len = p.seg_len;
  op.F = p.F;
  op.reverse = false;
  op.right = false;
  op.n2 = n2;
  op.status = status;
  cudaError_t e = set_identity<R>(seg, G, N, s);
  if (e) return e;
  cplx<R>* cur = seg;
  cplx<R>* nxt = ping;
  const int64_t kd = (int64_t)t->K * t->digits;
  for (int64_t tt = 0; tt < p.seg_len; ++tt) {
    // amplitude/phase calls: the segments hold whole steps, each opened by its diagonal P_n
    if (p.pd && tt % kd == 0 &&
        (e = launch_phase_rows(N, std::is_same<R, double>::value ? REDO_FP64 : REDO_FP32, cur, G, p.S,
                               p.seg_len / kd, tt / kd, p.M, p.pd, s)))
      return e;
    op.t = tt;
    op.X = cur;
    op.Y = nxt;
    if ((e = cgemm<R, false>(op, G, N, R(1), R(0), s))) return e;
    std::swap(cur, nxt);
  }
  if (cur != seg) copy_kernel<R><<<blocks_for(G * n2), 256, 0, s>>>(cur, seg, G * n2);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t large_combine_t(int N, const ChainPlan& p, const cplx<R>* seg, cplx<R>* prod,
                                   cplx<R>* ping, cudaStream_t s) {
  const int64_t n2 = (int64_t)N * N;
  cudaError_t e = set_identity<R>(prod, p.B, N, s);
  if (e) return e;
  ListStepOps<R> op{seg, p.S, 0, false, nullptr, nullptr, n2};
  cplx<R>* cur = prod;
  cplx<R>* nxt = ping;
  const int64_t L = p.F > 0 ? p.S : 0;
  for (int64_t tt = 0; tt < L; ++tt) {
    op.t = tt;
    op.X = cur;
    op.Y = nxt;
    if ((e = cgemm<R, false>(op, p.B, N, R(1), R(0), s))) return e;
    std::swap(cur, nxt);
  }
  if (cur != prod) copy_kernel<R><<<blocks_for(p.B * n2), 256, 0, s>>>(cur, prod, p.B * n2);
  return cudaGetLastError();
}

// one Newton-Schulz step on `count` matrices in place; tmp holds 2*count matrices
template <typename R>
static cudaError_t large_polar_t(int N, cplx<R>* P, int64_t count, cplx<R>* tmp, cudaStream_t s) {
  const int64_t n2 = (int64_t)N * N;
  cplx<R>* G = tmp;
  cplx<R>* Pn = tmp + count * n2;
  DenseOps<R> g{P, P, G, n2, n2, n2};
  cudaError_t e = cgemm<R, true>(g, count, N, R(1), R(0), s);
  if (e) return e;
  ns_mid_kernel<R><<<blocks_for(count * n2), 256, 0, s>>>(G, count, N);
  DenseOps<R> m{P, G, Pn, n2, n2, n2};
  if ((e = cgemm<R, false>(m, count, N, R(1), R(0), s))) return e;
  copy_kernel<R><<<blocks_for(count * n2), 256, 0, s>>>(Pn, P, count * n2);
  return cudaGetLastError();
}

size_t large_prop_workspace(const redo_table* t, const ChainPlan& p, int prec, bool reunit) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t n2 = (size_t)t->N * t->N;
  const size_t G = (size_t)p.B * p.S;
  // seg, ping (G each), prod (B), NS scratch (2G), prod64 (B, FP64)
  return up(G * n2 * el) * 2 + up(p.B * n2 * el) + up(2 * G * n2 * el) +
         (reunit ? up(p.B * n2 * sizeof(double2)) + up(2 * p.B * n2 * sizeof(double2)) : 0);
}

// After the segment products sit in the first region of the workspace: optional FP32/FP64
// re-unitarisation of segments, ordered combine, optional FP64 polar step of pulse products.
template <typename R>
static cudaError_t large_finish_t(const redo_table* t, const ChainPlan& p, bool reunit, char* ws,
                                  void** result, int* result_prec, cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int N = t->N;
  const size_t n2 = (size_t)N * N, G = (size_t)p.B * p.S;
  cplx<R>* seg = (cplx<R>*)ws;
  cplx<R>* ping = (cplx<R>*)(ws + up(G * n2 * sizeof(cplx<R>)));
  cplx<R>* prod = (cplx<R>*)((char*)ping + up(G * n2 * sizeof(cplx<R>)));
  cplx<R>* nsbuf = (cplx<R>*)((char*)prod + up(p.B * n2 * sizeof(cplx<R>)));
  char* tail = (char*)nsbuf + up(2 * G * n2 * sizeof(cplx<R>));
  cudaError_t e = cudaSuccess;
  if (reunit && p.M > 0 && (e = large_polar_t<R>(N, seg, G, nsbuf, s))) return e;
  if ((e = large_combine_t<R>(N, p, seg, prod, ping, s))) return e;
  *result = prod;
  *result_prec = std::is_same<R, double>::value ? REDO_FP64 : REDO_FP32;
  if (reunit && p.M > 0) {
    double2* p64 = (double2*)tail;
    double2* ns64 = (double2*)(tail + up(p.B * n2 * sizeof(double2)));
    convert_kernel<R, double><<<blocks_for(p.B * n2), 256, 0, s>>>(prod, p64, p.B * n2);
    if ((e = large_polar_t<double>(N, p64, p.B, ns64, s))) return e;
    *result = p64;
    *result_prec = REDO_FP64;
  }
  return cudaGetLastError();
}

template <typename R>
static cudaError_t large_propagate_t(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                     bool reunit, char* ws, void** result, int* result_prec,
                                     int64_t* status, cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t n2 = (size_t)t->N * t->N, G = (size_t)p.B * p.S;
  cplx<R>* seg = (cplx<R>*)ws;
  cplx<R>* ping = (cplx<R>*)(ws + up(G * n2 * sizeof(cplx<R>)));
  cudaError_t e = large_chain_t<R>(t, q, p, seg, ping, status, s);
  if (e) return e;
  return large_finish_t<R>(t, p, reunit, ws, result, result_prec, s);
}

cudaError_t large_finish_fp32(const redo_table* t, const ChainPlan& p, bool reunit, void* ws,
                              void** result, int* result_prec, cudaStream_t s) {
  return large_finish_t<float>(t, p, reunit, (char*)ws, result, result_prec, s);
}

// out[b] = in[2b + 1] in[2b] for b < count (FP32): joins pairs of consecutive sub-segment
// products (the later one on the left) into segment products.
// out[h] = Pck[h-1] Rck[h] for the chains h = u S + s with s > 0, Rck[h] for s = 0 (FP32): the
// costate of a segment carried back by the checkpoint before it, so that a trace against the
// segment's own partial products (which start from the identity) is a trace against P_f.
struct CostateShiftOps {
  const float2* P;
  const float2* Rc;
  float2* C;
  int64_t S, n2;
  __device__ void get(int64_t h, const float2*& a, const float2*& bb, float2*& c) const {
    a = (h % S == 0) ? nullptr : P + (h - 1) * n2;
    bb = Rc + h * n2;
    c = C + h * n2;
  }
};

cudaError_t large_costate_shift_fp32(const float2* Pck, const float2* Rck, float2* out, int64_t G, int64_t S, int N,
                                     cudaStream_t s) {
  const int64_t n2 = (int64_t)N * N;
  CostateShiftOps op{Pck, Rck, out, S, n2};
  return cgemm<float, false>(op, G, N, 1.0f, 0.0f, s);
}

// Costates of half segments from their segment's shifted costate C_s (h = 2s + i):
//     out[2s+1] = H[2s] C_s,   out[2s] = C_s H[2s+1]   (FP32),
// H the half-segment products: the later half sees the earlier half as part of its prefix,
// the earlier half sees the later one as part of its suffix.
struct HalfCostateOps {
  const float2* H;
  const float2* Cs;
  float2* C;
  int64_t n2;
  __device__ void get(int64_t h, const float2*& a, const float2*& bb, float2*& c) const {
    if (h & 1) {
      a = H + (h - 1) * n2;
      bb = Cs + (h >> 1) * n2;
    } else {
      a = Cs + (h >> 1) * n2;
      bb = H + (h + 1) * n2;
    }
    c = C + h * n2;
  }
};

cudaError_t large_half_costates_fp32(const float2* H, const float2* Cs, float2* out, int64_t Gf, int N,
                                     cudaStream_t s) {
  HalfCostateOps op{H, Cs, out, (int64_t)N * N};
  return cgemm<float, false>(op, Gf, N, 1.0f, 0.0f, s);
}

cudaError_t large_pair_products_fp32(const float2* in, float2* out, int64_t count, int N, cudaStream_t s) {
  const int64_t n2 = (int64_t)N * N;
  DenseOps<float> op{in + n2, in, out, 2 * n2, 2 * n2, n2};
  return cgemm<float, false>(op, count, N, 1.0f, 0.0f, s);
}

cudaError_t large_propagate(const redo_table* t, const int32_t* q, const ChainPlan& p, int prec,
                            bool reunit, void* ws, void** result, int* result_prec,
                            int64_t* status, cudaStream_t s) {
  if (prec == REDO_FP64)
    return large_propagate_t<double>(t, q, p, reunit, (char*)ws, result, result_prec, status, s);
  return large_propagate_t<float>(t, q, p, reunit, (char*)ws, result, result_prec, status, s);
}

ChainPlan plan_chain_large(const redo_table* t, int64_t B, int64_t M) {
  ChainPlan p;
  p.B = B;
  p.M = M;
  p.F = M * (int64_t)t->K * t->digits;
  // enough chains to give every SM a few tiles per step
  const int64_t tiles = (int64_t)(t->N / kT) * (t->N / kT);
  const int64_t bt = B * tiles;                         // 0 for an empty batch: one segment
  int64_t S = bt > 0 ? (4 * (int64_t)t->num_sms + bt - 1) / bt : 1;
  const int64_t max_s = (p.F + 15) / 16;
  if (S > max_s) S = max_s;
  if (S > 256) S = 256;
  if (S < 1) S = 1;
  p.seg_len = p.F > 0 ? (p.F + S - 1) / S : 0;
  p.S = p.seg_len > 0 ? (p.F + p.seg_len - 1) / p.seg_len : 1;
  return p;
}

// ============================================================================
// Gradient: segment products, checkpoints and costates, reverse sweep with traces
// ============================================================================

// Tr(H_k P_g R_g) for every chain g, H_k sparse (CSR); one CTA per chain.
template <typename R>
__global__ void __launch_bounds__(256) trace_kernel(const cplx<R>* __restrict__ P,
                                                    const cplx<R>* __restrict__ Rm, int N,
                                                    int64_t S, int64_t seg_len, int64_t F,
                                                    int64_t t, int K, int d,
                                                    const int32_t* __restrict__ hk_ptr,
                                                    const int32_t* __restrict__ hk_col, const int32_t* __restrict__ hk_row,
                                                    const double2* __restrict__ hk_val,
                                                    const double2* __restrict__ tau, double scale,
                                                    int64_t M, double* __restrict__ grad) {
  const int64_t g = blockIdx.x;
  const int64_t u = g / S, s = g % S;
  const int64_t f0 = s * seg_len;
  int64_t f1 = f0 + seg_len;
  if (f1 > F) f1 = F;
  const int64_t f = f1 - 1 - t;
  if (f < f0 || f >= f1) return;
  const int64_t kd = (int64_t)K * d;
  const int64_t n = f / kd;
  const int r = (int)(f - n * kd);
  const int k = r / d, j = r - k * d;
  if (j != d - 1) return;
  const int64_t n2 = (int64_t)N * N;
  const cplx<R>* Pg = P + g * n2;
  const cplx<R>* Rg = Rm + g * n2;
  const int p0 = hk_ptr[k * (N + 1)], p1 = hk_ptr[k * (N + 1) + N];
  double re = 0.0, im = 0.0;
  // one warp per nonzero: (row i, col c): H[i][c] * sum_x P[c][x] R[x][i]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = p0 + warp; e < p1; e += 8) {
    const int i = hk_row[e], c = hk_col[e];
    double dr = 0.0, di = 0.0;
    for (int x = lane; x < N; x += 32) {
      const cplx<R> pv = Pg[(int64_t)c * N + x], rv = Rg[(int64_t)x * N + i];
      dr += (double)pv.x * rv.x - (double)pv.y * rv.y;
      di += (double)pv.x * rv.y + (double)pv.y * rv.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
      dr += __shfl_down_sync(0xffffffffu, dr, off);
      di += __shfl_down_sync(0xffffffffu, di, off);
    }
    if (lane == 0) {
      const double2 h = hk_val[e];
      re += h.x * dr - h.y * di;
      im += h.x * di + h.y * dr;
    }
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
    const double2 tu = tau[u];
    grad[(u * M + n) * K + k] = scale * (tu.x * ti - tu.y * tr);
  }
}

// tau_u = Tr(U_T^dag X_u) (FP64), F_u
// tau_u = Tr(U_T^dag X_u) = sum_ij conj(U_T[i][j]) X_u[i][j], in FP64: grid (pulse, part),
// each block sums 1/kTauParts of the entries and adds into tau[u] (zeroed beforehand).
constexpr int kTauParts = 32;

template <typename R>
__global__ void __launch_bounds__(256) tau_kernel(const cplx<R>* __restrict__ X, const double2* __restrict__ UT,
                                                  int tb, int N, double2* __restrict__ tau) {
  const int64_t u = blockIdx.x / kTauParts;
  const int part = blockIdx.x % kTauParts;
  const int64_t n2 = (int64_t)N * N;
  const int64_t i0 = n2 * part / kTauParts, i1 = n2 * (part + 1) / kTauParts;
  const double2* Ut = UT + (tb ? u * n2 : 0);
  double re = 0.0, im = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
    const double2 g = Ut[i];
    const double xr = (double)X[u * n2 + i].x, xi = (double)X[u * n2 + i].y;
    re += g.x * xr + g.y * xi;
    im += g.x * xi - g.y * xr;
  }
  __shared__ double sre[256], sim[256];
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sre[threadIdx.x] += sre[threadIdx.x + w];
      sim[threadIdx.x] += sim[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&tau[u].x, sre[0]);
    atomicAdd(&tau[u].y, sim[0]);
  }
}

__global__ void fidelity_from_tau_kernel(const double2* __restrict__ tau, int64_t B, int N, double* __restrict__ F) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u < B) F[u] = (tau[u].x * tau[u].x + tau[u].y * tau[u].y) / ((double)N * (double)N);
}

// X_u = U_T^dag (converted)
template <typename R>
__global__ void adjoint_target_kernel(const double2* __restrict__ UT, int tb, int N, int64_t count,
                                      cplx<R>* __restrict__ X) {
  const int64_t n2 = (int64_t)N * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count * n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = i / n2, e = i % n2;
    const int r = (int)(e / N), c = (int)(e % N);
    const double2 g = UT[(tb ? u * n2 : 0) + (int64_t)c * N + r];
    X[i] = cmake<R>((R)g.x, (R)(-g.y));
  }
}

size_t large_grad_workspace(const redo_table* t, const ChainPlan& p, int prec) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t el = prec == REDO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t n2 = (size_t)t->N * t->N;
  const size_t G = (size_t)p.B * p.S;
  // seg, Pck, Rck, ping x2 (G each), running (B) x2, tau
  return 5 * up(G * n2 * el) + 2 * up(p.B * n2 * el) + up(p.B * sizeof(double2));
}

// One round of the log-depth (Hillis-Steele) scans over the S segment products of every
// pulse, prefix and suffix in one launch.  Items [0, B S) are prefix entries,
//     P_s <- P_s P_{s-off}            (s >= off; else copied),
// items [B S, 2 B S) suffix entries,
//     Q_s <- Q_{s+off} Q_s            (s + off < S; else copied),
// so after rounds off = 1, 2, 4, ... < S, P_s = X_s ... X_0 and Q_s = X_{S-1} ... X_s.
template <typename R>
struct ScanRoundOps {
  const cplx<R>* ps;
  cplx<R>* pd;
  const cplx<R>* qs;
  cplx<R>* qd;
  int64_t BS, S, off, n2;
  __device__ void get(int64_t b, const cplx<R>*& a, const cplx<R>*& bb, cplx<R>*& c) const {
    const bool suffix = b >= BS;
    const int64_t i = suffix ? b - BS : b;
    const int64_t s = i % S;
    if (!suffix) {
      a = s >= off ? ps + i * n2 : nullptr;
      bb = s >= off ? ps + (i - off) * n2 : ps + i * n2;
      c = pd + i * n2;
    } else {
      a = s + off < S ? qs + (i + off) * n2 : nullptr;
      bb = qs + i * n2;
      c = qd + i * n2;
    }
  }
};

// Costates R_s = U_T^dag Q_{s+1} (U_T^dag alone for the last segment) and a contiguous copy
// of every pulse's full product P_{S-1} (items [B S, B S + B)).
template <typename R>
struct CostateOps {
  const cplx<R>* Q;
  const cplx<R>* Uadj;     // [B] U_T^dag
  const cplx<R>* P;
  cplx<R>* Rck;
  cplx<R>* last;           // [B]
  int64_t BS, S, n2;
  __device__ void get(int64_t b, const cplx<R>*& a, const cplx<R>*& bb, cplx<R>*& c) const {
    if (b < BS) {
      const int64_t s = b % S, u = b / S;
      a = s + 1 < S ? Uadj + u * n2 : nullptr;
      bb = s + 1 < S ? Q + (b + 1) * n2 : Uadj + u * n2;
      c = Rck + b * n2;
    } else {
      const int64_t u = b - BS;
      a = nullptr;
      bb = P + (u * S + S - 1) * n2;
      c = last + u * n2;
    }
  }
};

// Prefix checkpoints, tau/F and suffix costates from the segment products in the first
// workspace region, by log-depth scans (ceil(log2 S) batched rounds instead of 2S
// dependent products).
template <typename R>
static cudaError_t large_scans_t(const redo_table* t, const ChainPlan& p, const double2* UT, int tb,
                                 double* F_out, char* ws, cplx<R>** Pck_out, cplx<R>** Rck_out,
                                 double2** tau_out, cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int N = t->N;
  const int64_t n2 = (int64_t)N * N, G = p.B * p.S;
  const size_t mat = up((size_t)G * n2 * sizeof(cplx<R>));
  cplx<R>* seg = (cplx<R>*)ws;
  cplx<R>* Pck = (cplx<R>*)(ws + mat);
  cplx<R>* Rck = (cplx<R>*)(ws + 2 * mat);
  cplx<R>* ping = (cplx<R>*)(ws + 3 * mat);
  cplx<R>* pong = (cplx<R>*)(ws + 4 * mat);
  cplx<R>* run = (cplx<R>*)(ws + 5 * mat);
  cplx<R>* run2 = (cplx<R>*)(ws + 5 * mat + up(p.B * n2 * sizeof(cplx<R>)));
  double2* tau = (double2*)(ws + 5 * mat + 2 * up(p.B * n2 * sizeof(cplx<R>)));
  cudaError_t e;
  // prefix in Pck / ping, suffix in pong / Rck; the first round reads the segment products
  const cplx<R>* ps = seg;
  const cplx<R>* qs = seg;
  cplx<R>* pbuf[2] = {Pck, ping};
  cplx<R>* qbuf[2] = {pong, Rck};
  int r = 0;
  for (int64_t off = 1; off < p.S || r == 0; off *= 2, ++r) {
    ScanRoundOps<R> op{ps, pbuf[r & 1], qs, qbuf[r & 1], G, p.S, off, n2};
    if ((e = cgemm<R, false>(op, 2 * G, N, R(1), R(0), s))) return e;
    ps = pbuf[r & 1];
    qs = qbuf[r & 1];
  }
  // checkpoints end in Pck and the suffix products in pong (copy over when they did not)
  if (ps != Pck) {
    DenseOps<R> cp{nullptr, ps, Pck, 0, n2, n2};
    if ((e = cgemm<R, false>(cp, G, N, R(1), R(0), s))) return e;
  }
  if (qs != pong) {
    DenseOps<R> cp{nullptr, qs, pong, 0, n2, n2};
    if ((e = cgemm<R, false>(cp, G, N, R(1), R(0), s))) return e;
  }
  adjoint_target_kernel<R><<<blocks_for(p.B * n2), 256, 0, s>>>(UT, tb, N, p.B, run);
  CostateOps<R> co{pong, run, Pck, Rck, run2, G, p.S, n2};
  if ((e = cgemm<R, false>(co, G + p.B, N, R(1), R(0), s))) return e;
  if ((e = cudaMemsetAsync(tau, 0, sizeof(double2) * p.B, s))) return e;
  tau_kernel<R><<<(unsigned)(p.B * kTauParts), 256, 0, s>>>(run2, UT, tb, N, tau);
  if (F_out) fidelity_from_tau_kernel<<<(unsigned)((p.B + 127) / 128), 128, 0, s>>>(tau, p.B, N, F_out);
  *Pck_out = Pck;
  *Rck_out = Rck;
  *tau_out = tau;
  return cudaGetLastError();
}

cudaError_t large_grad_scans_fp32(const redo_table* t, const ChainPlan& p, const double2* UT, int tb,
                                  double* F_out, void* ws, float2** Pck, float2** Rck, double2** tau,
                                  cudaStream_t s) {
  return large_scans_t<float>(t, p, UT, tb, F_out, (char*)ws, Pck, Rck, tau, s);
}

cudaError_t large_reunit_segments_fp32(const redo_table* t, const ChainPlan& p, void* ws, cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t n2 = (int64_t)t->N * t->N, G = p.B * p.S;
  const size_t mat = up((size_t)G * n2 * sizeof(float2));
  // seg, Pck, Rck, then two ping buffers: contiguous scratch for 2G matrices
  return large_polar_t<float>(t->N, (float2*)ws, G, (float2*)((char*)ws + 3 * mat), s);
}

template <typename R>
static cudaError_t large_grad_t(const redo_table* t, const int32_t* q, const ChainPlan& p,
                                const double2* UT, int tb, double* F_out, double* grad, char* ws,
                                int64_t* status, cudaStream_t s, double2* Tz, double* grad_phase,
                                bool reunit) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int N = t->N;
  const int64_t n2 = (int64_t)N * N, G = p.B * p.S;
  const size_t mat = up((size_t)G * n2 * sizeof(cplx<R>));
  cplx<R>* seg = (cplx<R>*)ws;
  cplx<R>* pA = (cplx<R>*)(ws + 3 * mat);
  cplx<R>* pB = (cplx<R>*)(ws + 4 * mat);
  cudaError_t e = large_chain_t<R>(t, q, p, seg, pA, status, s);
  if (e) return e;
  if (reunit && p.M > 0 && (e = large_polar_t<R>(N, seg, G, pA, s))) return e;
  cplx<R>* Pck;
  cplx<R>* Rck;
  double2* tau;
  if ((e = large_scans_t<R>(t, p, UT, tb, F_out, ws, &Pck, &Rck, &tau, s))) return e;
  if (p.M == 0) return cudaGetLastError();
  // reverse sweep: traces, then P <- A^dag P, R <- R A
  GatherStepOps<R> left{}, right{};
  left.T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  left.q = q;
  left.M = p.M;
  left.K = t->K;
  left.d = t->digits;
  left.base = t->base;
  left.levels = t->levels;
  left.S = p.S;
  left.seg_len = p.seg_len;
  left.F = p.F;
  left.reverse = true;
  left.right = false;
  left.n2 = n2;
  left.status = status;
  right = left;
  right.right = true;
  right.status = nullptr;
  cplx<R>* P = Pck;
  cplx<R>* Pn = pA;
  cplx<R>* Rr = Rck;
  cplx<R>* Rn = pB;
  const double scale = 2.0 * t->dt / ((double)N * (double)N);
  const int prec = std::is_same<R, double>::value ? REDO_FP64 : REDO_FP32;
  const int64_t kd = (int64_t)t->K * t->digits;
  if (p.pd && (e = launch_phase_boundary(N, prec, P, Rr, G, p.S, p.seg_len, p.F, -1, kd, p.M, p.pd, t->sz64,
                                         t->K, Tz, s)))
    return e;
  for (int64_t tt = 0; tt < p.seg_len; ++tt) {
    trace_kernel<R><<<(unsigned)G, 256, 0, s>>>(P, Rr, N, p.S, p.seg_len, p.F, tt, t->K, t->digits,
                                                t->hk_ptr, t->hk_col, t->hk_row, t->hk_val, tau, scale, p.M,
                                                grad);
    left.t = tt;
    left.X = P;
    left.Y = Pn;
    if ((e = cgemm<R, true>(left, G, N, R(1), R(0), s))) return e;
    right.t = tt;
    right.X = Rr;
    right.Y = Rn;
    if ((e = cgemm<R, false>(right, G, N, R(1), R(0), s))) return e;
    std::swap(P, Pn);
    std::swap(Rr, Rn);
    // the factor just undone opened its step: record the boundary trace, undo the diagonal
    if (p.pd && (tt + 1) % kd == 0 &&
        (e = launch_phase_boundary(N, prec, P, Rr, G, p.S, p.seg_len, p.F, tt, kd, p.M, p.pd, t->sz64, t->K, Tz,
                                   s)))
      return e;
  }
  if (p.pd && Tz && (e = launch_phase_grad_finish(N, p.B, p.M, t->K, Tz, tau, grad_phase, s))) return e;
  return cudaGetLastError();
}

cudaError_t large_grad(const redo_table* t, const int32_t* q, const ChainPlan& p, int prec,
                       const double2* UT, int tb, double* F_out, double* grad, void* ws,
                       int64_t* status, cudaStream_t s, double2* Tz, double* grad_phase, bool reunit) {
  if (prec == REDO_FP64)
    return large_grad_t<double>(t, q, p, UT, tb, F_out, grad, (char*)ws, status, s, Tz, grad_phase, reunit);
  return large_grad_t<float>(t, q, p, UT, tb, F_out, grad, (char*)ws, status, s, Tz, grad_phase, reunit);
}

// ============================================================================
// State simulation for large N: psi_b <- A(b, f) psi_b, one launch per factor,
// CTA (b, row block of 64) with a warp per 8 rows; <O> at step ends.
// ============================================================================
template <typename R>
__global__ void __launch_bounds__(256) matvec_step_kernel(const cplx<R>* __restrict__ T,
                                                          const int32_t* __restrict__ q,
                                                          int64_t M, int K, int d, int base,
                                                          int64_t levels, int N, int64_t f,
                                                          const cplx<R>* __restrict__ x,
                                                          cplx<R>* __restrict__ y) {
  const int64_t b = blockIdx.y;
  const int64_t kd = (int64_t)K * d;
  const int64_t n = f / kd;
  const int r = (int)(f - n * kd);
  const int k = r / d, j = r - k * d;
  int32_t qv = q[(b * M + n) * K + k];
  if (qv < 0 || qv >= levels) qv = 0;
  for (int i = 0; i < j; ++i) qv /= base;
  const cplx<R>* A = T + ((int64_t)(k * d + j) * base + qv % base) * (int64_t)N * N;
  const cplx<R>* xb = x + b * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int row = blockIdx.x * 64 + warp; row < (int)(blockIdx.x + 1) * 64 && row < N; row += 8) {
    R sr = 0, si = 0;
    for (int c = lane; c < N; c += 32) {
      const cplx<R> a = A[(int64_t)row * N + c], v = xb[c];
      sr = fma(a.x, v.x, sr);
      sr = fma(-a.y, v.y, sr);
      si = fma(a.x, v.y, si);
      si = fma(a.y, v.x, si);
    }
    for (int off = 16; off > 0; off >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, off);
      si += __shfl_down_sync(0xffffffffu, si, off);
    }
    if (lane == 0) y[b * N + row] = cmake<R>(sr, si);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) expect_kernel(const cplx<R>* __restrict__ x, const double* __restrict__ obs,
                                                     int N, int64_t M, int64_t n, double* __restrict__ expect) {
  const int64_t b = blockIdx.x;
  double v = 0.0;
  for (int i = threadIdx.x; i < N; i += 256) {
    const double re = (double)x[b * N + i].x, im = (double)x[b * N + i].y;
    v += obs[i] * (re * re + im * im);
  }
  __shared__ double sv[256];
  sv[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sv[threadIdx.x] += sv[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) expect[b * (M + 1) + n] = sv[0];
}

size_t large_sim_workspace(const redo_table* t, int64_t B) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return 2 * up((size_t)B * t->N * sizeof(double2));
}

template <typename R>
static cudaError_t large_sim_t(const redo_table* t, const int32_t* q, int64_t B, int64_t M,
                               const double2* psi0, int pb, const double* obs, double* expect,
                               char* ws, cudaStream_t s) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int N = t->N;
  cplx<R>* x = (cplx<R>*)ws;
  cplx<R>* y = (cplx<R>*)(ws + up((size_t)B * N * sizeof(double2)));
  // x_b = psi0 (converted)
  for (int64_t b = 0; b < B; ++b)
    convert_kernel<double, R><<<blocks_for(N), 256, 0, s>>>(psi0 + (pb ? b * N : 0), x + b * N, N);
  expect_kernel<R><<<(unsigned)B, 256, 0, s>>>(x, obs, N, M, 0, expect);
  const cplx<R>* T = std::is_same<R, double>::value ? (const cplx<R>*)t->T64 : (const cplx<R>*)t->T32;
  const int64_t kd = (int64_t)t->K * t->digits;
  dim3 grid((N + 63) / 64, (unsigned)B);
  for (int64_t f = 0; f < M * kd; ++f) {
    matvec_step_kernel<R><<<grid, 256, 0, s>>>(T, q, M, t->K, t->digits, t->base, t->levels, N, f, x, y);
    std::swap(x, y);
    if ((f + 1) % kd == 0) expect_kernel<R><<<(unsigned)B, 256, 0, s>>>(x, obs, N, M, (f + 1) / kd, expect);
  }
  return cudaGetLastError();
}

cudaError_t large_sim(const redo_table* t, const int32_t* q, int64_t B, int64_t M, int prec,
                      const double2* psi0, int pb, const double* obs, double* expect, void* ws,
                      cudaStream_t s) {
  if (prec == REDO_FP64) return large_sim_t<double>(t, q, B, M, psi0, pb, obs, expect, (char*)ws, s);
  return large_sim_t<float>(t, q, B, M, psi0, pb, obs, expect, (char*)ws, s);
}

}  // namespace redo
