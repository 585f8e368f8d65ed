// Shared-memory complex matrix products for N <= 64 (SIMT, FP64 or FP32).
#pragma once
#include "redo_internal.cuh"

namespace redo {

// ============================================================================
// Shared-memory complex matrix product  Y = A * X  (N x N, row-major)
// Thread lt of a chain owns rows ty + TY*a and columns tx + TX*c.
// ============================================================================
template <typename R, int N, int TM, int TN>
struct SmemMM {
  static constexpr int TY = N / TM, TX = N / TN, THREADS = TY * TX;
  static_assert(TY * TM == N && TX * TN == N, "tile must divide N");
  __device__ __forceinline__ static void run(const cplx<R>* __restrict__ A,
                                             const cplx<R>* __restrict__ X, int lt,
                                             cplx<R> (&Y)[TM][TN]) {
    const int ty = lt / TX, tx = lt % TX;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) Y[a][c] = cmake<R>(R(0), R(0));
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      cplx<R> av[TM], xv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = A[(ty + TY * a) * N + k];
#pragma unroll
      for (int c = 0; c < TN; ++c) xv[c] = X[k * N + tx + TX * c];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) cfma<R>(Y[a][c], av[a], xv[c]);
    }
  }
  // Y = A^dag X
  __device__ __forceinline__ static void run_adj(const cplx<R>* __restrict__ A,
                                                 const cplx<R>* __restrict__ X, int lt,
                                                 cplx<R> (&Y)[TM][TN]) {
    const int ty = lt / TX, tx = lt % TX;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) Y[a][c] = cmake<R>(R(0), R(0));
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      cplx<R> av[TM], xv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) {
        const cplx<R> v = A[k * N + ty + TY * a];
        av[a] = cmake<R>(v.x, -v.y);
      }
#pragma unroll
      for (int c = 0; c < TN; ++c) xv[c] = X[k * N + tx + TX * c];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) cfma<R>(Y[a][c], av[a], xv[c]);
    }
  }
  // Q = (3I - A^dag A) / 2 written to Q, computing only half of the Hermitian Gram matrix: the
  // T(T+1)/2 tiles (ty <= tx) of a square tiling go to the first threads (whole warps), each writes
  // its entries and, off the tile diagonal ty == tx, their conjugate mirrors (tile (ty, tx) and
  // tile (tx, ty) hold transposed entries).  Returns after the caller's barrier is due.
  __device__ __forceinline__ static void ns_half_gram(const cplx<R>* __restrict__ A, cplx<R>* __restrict__ Q,
                                                      int lt) {
    static_assert(TY == TX && TM == TN, "square tiling");
    constexpr int T = TY, HALF = T * (T + 1) / 2;
    if (lt >= HALF) return;
    int ty = 0, rem = lt;
    while (rem >= T - ty) {
      rem -= T - ty;
      ++ty;
    }
    const int tx = ty + rem;
    cplx<R> Y[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) Y[a][c] = cmake<R>(R(0), R(0));
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      cplx<R> av[TM], xv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) {
        const cplx<R> v = A[k * N + ty + TY * a];
        av[a] = cmake<R>(v.x, -v.y);
      }
#pragma unroll
      for (int c = 0; c < TN; ++c) xv[c] = A[k * N + tx + TX * c];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) cfma<R>(Y[a][c], av[a], xv[c]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int r = ty + TY * a, col = tx + TX * c;
        Q[r * N + col] = cmake<R>((r == col ? R(1.5) : R(0)) - R(0.5) * Y[a][c].x, -R(0.5) * Y[a][c].y);
        if (ty != tx) Q[col * N + r] = cmake<R>(-R(0.5) * Y[a][c].x, R(0.5) * Y[a][c].y);
      }
  }
  // Y = diag(p) X (a row scaling, p in FP64)
  __device__ __forceinline__ static void scale_rows(const double2* __restrict__ p,
                                                    const cplx<R>* __restrict__ X, int lt,
                                                    cplx<R> (&Y)[TM][TN]) {
    const int ty = lt / TX, tx = lt % TX;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const double2 pv = p[ty + TY * a];
      const cplx<R> pa = cmake<R>((R)pv.x, (R)pv.y);
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        Y[a][c] = cmake<R>(R(0), R(0));
        cfma<R>(Y[a][c], pa, X[(ty + TY * a) * N + tx + TX * c]);
      }
    }
  }
  __device__ __forceinline__ static void store(cplx<R>* __restrict__ X, int lt,
                                               const cplx<R> (&Y)[TM][TN]) {
    const int ty = lt / TX, tx = lt % TX;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) X[(ty + TY * a) * N + tx + TX * c] = Y[a][c];
  }
};


// Square register tiles used by the one-matrix-per-CTA kernels.
template <int N> struct SqTile { static constexpr int TM = N >= 64 ? 4 : (N >= 32 ? 2 : 1); };

}  // namespace redo
