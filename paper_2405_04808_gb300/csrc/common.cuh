// Shared device-side definitions of the pintmg kernels (sm_103a).
//
// Vectors are the ABI's type-major layout (Fig. 4): the time-major
// permutation of Sec. 5.2 is never materialised; each kernel indexes the five
// type arrays directly.  Time block j = 0..n (the paper's block j + 1 of
// Fig. 5) owns u_j, z_j, lambda_j (j < n) and v_{j-1}, mu_{j-1} (j >= 1), with
// 0-based step indices.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pintmg.h"

namespace pintmg {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kDenseMax = 4;     // dense layout: p, q <= 4 (one thread per time block)
// tridiagonal: per time block, the 2x2 maps each lane composes in each of the
// 5 rounds of the forward and backward warp scans (precomputed at setup),
// laid out [direction][round][entry][lane] so that lanes read consecutively
constexpr int kScanRounds = 5;
constexpr int kScanPerBlock = 2 * kScanRounds * 4 * 32;
__host__ __device__ constexpr int scan_index(int dir, int round, int entry, int lane) {
  return ((dir * kScanRounds + round) * 4 + entry) * 32 + lane;
}

// Coefficients of one grid level (device pointers), in the kernels' precision T.
//   N, V, Z: per-step blocks (tridiagonal: 3 band rows of p; dense: p*p, p*p, p*q)
//   stride 0 means the same block at every step.
//   fac:  tridiagonal: LDL^T of S = N N^T + Z Z^T as [a(p) | b(p) | dinv(p)]
//         (a_i = L[i][i-1], b_i = L[i][i-2], dinv_i = 1 / D_i);
//         dense: Cholesky factor of S, row-major p*p, diagonal stored inverted.
//   scan: tridiagonal only: per step, kScanPerBlock entries: for each lane and
//         round of the forward / backward warp scans, the composed 2x2 map of
//         that lane's LDL^T recurrence chunks (scan_index layout).
//   CT: storage type of the N, V, Z bands (T, or BF16 with T = float: the
//   bands are read as BF16 and every product is formed in FP32).
template <typename T, typename CT = T>
struct LevelView {
  int n, p, q, layout;
  const CT *N, *V, *Z;
  long long sN, sV, sZ;
  const T *fac;
  long long sFac;
  const T *scan;
  T kappa;  // != 0: V_k = kappa Z_k for every step (theta = 1, d_z f a multiple of M), else 0
  // tridiagonal blocks too large for one warp's registers (p > 128): workspaces of the block
  // solve's three launches, (n + 1) x p each (right-hand sides of S lambda = rhs, and lambda)
  T *ws_rhs, *ws_lam;
};

template <typename T>
struct Vec {
  T *u, *v, *z, *l, *m;
};

template <typename T>
__host__ __device__ inline Vec<T> make_vec(T *base, int n, int p, int q) {
  Vec<T> x;
  long long np = (long long)n * p;
  x.u = base;
  x.v = base + np;
  x.z = base + 2 * np;
  x.l = base + 2 * np + (long long)n * q;
  x.m = base + 3 * np + (long long)n * q;
  return x;
}

template <typename T>
__host__ __device__ inline Vec<const T> make_cvec(const T *base, int n, int p, int q) {
  Vec<const T> x;
  long long np = (long long)n * p;
  x.u = base;
  x.v = base + np;
  x.z = base + 2 * np;
  x.l = base + 2 * np + (long long)n * q;
  x.m = base + 3 * np + (long long)n * q;
  return x;
}

// a band coefficient in the arithmetic type
__device__ __forceinline__ double coef(double a) { return a; }
__device__ __forceinline__ float coef(float a) { return a; }
__device__ __forceinline__ float coef(__nv_bfloat16 a) { return __bfloat162float(a); }

// ---------------------------------------------------------------------------
// Warp-cooperative tridiagonal helpers.  Lane `ln` owns the contiguous chunk
// [ln*C, ln*C + C) of a length-p vector (p <= 32 C); entries at i >= p are 0.

template <typename T, int C>
__device__ __forceinline__ void chunk_load(T (&x)[C], const T *src, int p, int ln) {
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    x[e] = (i < p) ? src[i] : T(0);
  }
}

template <typename T, int C>
__device__ __forceinline__ void chunk_store(T *dst, const T (&x)[C], int p, int ln) {
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    if (i < p) dst[i] = x[e];
  }
}

// neighbours of the chunk: x_{lo-1} and x_{lo+C} (0 outside [0, p))
template <typename T, int C>
__device__ __forceinline__ void chunk_halo(const T (&x)[C], int p, int ln, T &prev, T &next) {
  prev = __shfl_up_sync(kFull, x[C - 1], 1);
  next = __shfl_down_sync(kFull, x[0], 1);
  if (ln == 0) prev = T(0);
  if (ln * C + C >= p) next = T(0);
}

// y (+)= A x for a tridiagonal band A (3 rows of p, stored as CT)
template <typename T, int C, bool kAccumulate, typename CT>
__device__ __forceinline__ void tri_mv(T (&y)[C], const CT *A, const T (&x)[C], int p, int ln, T sign) {
  T prev, next;
  chunk_halo<T, C>(x, p, ln, prev, next);
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    T acc = T(0);
    if (i < p) {
      T xm = (e == 0) ? prev : x[e - 1];
      T xp = (e == C - 1) ? next : x[e + 1];
      acc = fma(T(coef(A[i])), xm, fma(T(coef(A[p + i])), x[e], T(coef(A[2 * p + i])) * xp));
    }
    y[e] = kAccumulate ? fma(sign, acc, y[e]) : sign * acc;
  }
}

// y (+)= A^T x for a tridiagonal band A: (A^T x)_i = A[i-1][i] x_{i-1} + A[i][i] x_i + A[i+1][i] x_{i+1}
template <typename T, int C, bool kAccumulate, typename CT>
__device__ __forceinline__ void tri_mtv(T (&y)[C], const CT *A, const T (&x)[C], int p, int ln, T sign) {
  T prev, next;
  chunk_halo<T, C>(x, p, ln, prev, next);
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    T acc = T(0);
    if (i < p) {
      T xm = (e == 0) ? prev : x[e - 1];
      T xp = (e == C - 1) ? next : x[e + 1];
      T up = (i > 0) ? T(coef(A[2 * p + i - 1])) : T(0);     // A[i-1][i]
      T lo = (i + 1 < p) ? T(coef(A[i + 1])) : T(0);         // A[i+1][i]
      acc = fma(up, xm, fma(T(coef(A[p + i])), x[e], lo * xp));
    }
    y[e] = kAccumulate ? fma(sign, acc, y[e]) : sign * acc;
  }
}

// Inclusive Kogge-Stone scan of affine maps s -> H s + t over the warp's
// lanes when the linear parts are known in advance: in round d lane ln
// composes with lane ln - 2^d (forward) or ln + 2^d (backward), and
// Hd[round] is the composed linear part lane ln holds at the start of that
// round, precomputed from the operator.  Only the offsets move at run time:
// t <- t + H t'  (4 FMAs per round instead of 12).
template <typename T, bool kForward>
__device__ __forceinline__ void warp_affine_scan_pre(T (&t)[2], const T *scan, int dir, int ln) {
#pragma unroll
  for (int d = 0; d < kScanRounds; ++d) {
    const int off = 1 << d;
    T t0, t1;
    if (kForward) {
      t0 = __shfl_up_sync(kFull, t[0], off);
      t1 = __shfl_up_sync(kFull, t[1], off);
    } else {
      t0 = __shfl_down_sync(kFull, t[0], off);
      t1 = __shfl_down_sync(kFull, t[1], off);
    }
    const bool take = kForward ? (ln >= off) : (ln + off < kWarp);
    if (take) {
      const T h0 = scan[scan_index(dir, d, 0, ln)], h1 = scan[scan_index(dir, d, 1, ln)];
      const T h2 = scan[scan_index(dir, d, 2, ln)], h3 = scan[scan_index(dir, d, 3, ln)];
      const T n0 = fma(h0, t0, fma(h1, t1, t[0]));
      const T n1 = fma(h2, t0, fma(h3, t1, t[1]));
      t[0] = n0;
      t[1] = n1;
    }
  }
}

// Solve S x = r with S = L D L^T pentadiagonal (a, b = first and second
// sub-diagonals of the unit lower L, dinv = 1/D), r and x held as lane chunks.
//   forward   g_i = r_i - a_i g_{i-1} - b_i g_{i-2}
//   scale     h_i = g_i dinv_i
//   backward  x_i = h_i - a_{i+1} x_{i+1} - b_{i+2} x_{i+2}
// Each lane runs its chunk from a zero incoming state, a warp scan of the
// chunks' 2x2 affine maps (linear parts and their compositions precomputed
// in `scan`) gives every chunk's true incoming state, and the chunk is run
// again from it.
template <typename T, int C>
__device__ __forceinline__ void penta_solve(T (&x)[C], const T (&r)[C], const T *fac, const T *scan,
                                            int p, int ln) {
  const T *a = fac, *b = fac + p, *dinv = fac + 2 * p;
  T ca[C], cb[C];
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    ca[e] = (i < p) ? a[i] : T(0);
    cb[e] = (i < p) ? b[i] : T(0);
  }
  // forward: state (g_{i-2}, g_{i-1})
  T s1 = 0, s2 = 0;
#pragma unroll
  for (int e = 0; e < C; ++e) {
    T g = fma(-ca[e], s2, fma(-cb[e], s1, r[e]));
    s1 = s2;
    s2 = g;
  }
  T t[2] = {s1, s2};
  warp_affine_scan_pre<T, true>(t, scan, 0, ln);
  s1 = __shfl_up_sync(kFull, t[0], 1);
  s2 = __shfl_up_sync(kFull, t[1], 1);
  if (ln == 0) { s1 = 0; s2 = 0; }
  T g[C];
#pragma unroll
  for (int e = 0; e < C; ++e) {
    g[e] = fma(-ca[e], s2, fma(-cb[e], s1, r[e]));
    s1 = s2;
    s2 = g[e];
  }
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    g[e] = (i < p) ? g[e] * dinv[i] : T(0);
  }
  // backward: state (x_{i+1}, x_{i+2}); coefficients a_{i+1}, b_{i+2}
  T na[C], nb[C];
#pragma unroll
  for (int e = 0; e < C; ++e) {
    int i = ln * C + e;
    na[e] = (i + 1 < p) ? a[i + 1] : T(0);
    nb[e] = (i + 2 < p) ? b[i + 2] : T(0);
  }
  s1 = 0; s2 = 0;
#pragma unroll
  for (int e = C - 1; e >= 0; --e) {
    T xi = fma(-na[e], s1, fma(-nb[e], s2, g[e]));
    s2 = s1;
    s1 = xi;
  }
  T tb[2] = {s1, s2};
  warp_affine_scan_pre<T, false>(tb, scan, 1, ln);
  s1 = __shfl_down_sync(kFull, tb[0], 1);
  s2 = __shfl_down_sync(kFull, tb[1], 1);
  if (ln == kWarp - 1) { s1 = 0; s2 = 0; }
#pragma unroll
  for (int e = C - 1; e >= 0; --e) {
    T xi = fma(-na[e], s1, fma(-nb[e], s2, g[e]));
    s2 = s1;
    s1 = xi;
    x[e] = xi;
  }
}

// ---------------------------------------------------------------------------
// Dense blocks up to kDenseWarpMax: one warp per time block, lane i owning
// entry i of every vector (entries at i >= the length are 0).  A is row-major.

constexpr int kDenseWarpMax = 32;

template <typename T>
__device__ __forceinline__ T dw_load(const T *src, int len, int ln) {
  return ln < len ? src[ln] : T(0);
}

// y (+)= sign A x, A rows x cols (lane i forms row i; x held by lane k)
template <typename T>
__device__ __forceinline__ T dw_mv(const T *A, T x, int rows, int cols, int ln) {
  T acc = T(0);
  for (int k = 0; k < cols; ++k) {
    const T xk = __shfl_sync(kFull, x, k);
    if (ln < rows) acc = fma(A[ln * cols + k], xk, acc);
  }
  return acc;
}

// A^T x, A rows x cols (lane i forms entry i of the cols-vector)
template <typename T>
__device__ __forceinline__ T dw_mtv(const T *A, T x, int rows, int cols, int ln) {
  T acc = T(0);
  for (int k = 0; k < rows; ++k) {
    const T xk = __shfl_sync(kFull, x, k);
    if (ln < cols) acc = fma(A[k * cols + ln], xk, acc);
  }
  return acc;
}

// x = S^-1 r with S = L L^T (L row-major p x p, diagonal stored inverted):
// column-oriented substitutions, one broadcast per column
template <typename T>
__device__ __forceinline__ T dw_chol_solve(const T *L, T r, int p, int ln) {
  T y = r;
  for (int k = 0; k < p; ++k) {  // forward: y_k = (r_k - sum_{i<k} L_ki y_i) / L_kk
    const T yk = __shfl_sync(kFull, y, k) * L[k * p + k];
    if (ln == k) y = yk;
    if (ln > k && ln < p) y = fma(-L[ln * p + k], yk, y);
  }
  T x = y;
  for (int k = p - 1; k >= 0; --k) {  // backward with L^T
    const T xk = __shfl_sync(kFull, x, k) * L[k * p + k];
    if (ln == k) x = xk;
    if (ln < k) x = fma(-L[k * p + ln], xk, x);
  }
  return ln < p ? x : T(0);
}

// ---------------------------------------------------------------------------
// Dense small-block helpers (one thread per time block, p, q <= kDenseMax)

// y = A x (A p x m row-major) or y = A^T x (A m x p), sign applied
template <typename T>
__device__ __forceinline__ void dn_mv(T *y, const T *A, const T *x, int rows, int cols, T sign,
                                      bool accumulate) {
#pragma unroll
  for (int i = 0; i < kDenseMax; ++i) {
    if (i < rows) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < kDenseMax; ++k)
        if (k < cols) acc = fma(A[i * cols + k], x[k], acc);
      y[i] = accumulate ? fma(sign, acc, y[i]) : sign * acc;
    }
  }
}

template <typename T>
__device__ __forceinline__ void dn_mtv(T *y, const T *A, const T *x, int rows, int cols, T sign,
                                       bool accumulate) {
  // A is rows x cols; y (cols) = A^T x (rows)
#pragma unroll
  for (int i = 0; i < kDenseMax; ++i) {
    if (i < cols) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < kDenseMax; ++k)
        if (k < rows) acc = fma(A[k * cols + i], x[k], acc);
      y[i] = accumulate ? fma(sign, acc, y[i]) : sign * acc;
    }
  }
}

// x = S^-1 r with S = L L^T (L row-major, diagonal stored inverted)
template <typename T>
__device__ __forceinline__ void dn_chol_solve(T *x, const T *r, const T *L, int p) {
  T y[kDenseMax];
#pragma unroll
  for (int i = 0; i < kDenseMax; ++i) {
    if (i < p) {
      T acc = r[i];
#pragma unroll
      for (int k = 0; k < kDenseMax; ++k)
        if (k < i) acc = fma(-L[i * p + k], y[k], acc);
      y[i] = acc * L[i * p + i];
    }
  }
#pragma unroll
  for (int i = kDenseMax - 1; i >= 0; --i) {
    if (i < p) {
      T acc = y[i];
#pragma unroll
      for (int k = 0; k < kDenseMax; ++k)
        if (k > i && k < p) acc = fma(-L[k * p + i], x[k], acc);
      x[i] = acc * L[i * p + i];
    }
  }
}

}  // namespace pintmg
