// FP64 Krylov kernels for flexible GMRES (Saad 1993) and the coarse GMRES:
// multi-dot products with fixed-order reductions (bitwise reproducible),
// multi-axpy, and the Arnoldi/Givens bookkeeping on the device.
#pragma once

#include "common.cuh"

namespace pintmg {

constexpr int kDotThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kDotThreads / kWarp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  const int w = threadIdx.x / kWarp, ln = threadIdx.x & (kWarp - 1);
  if (ln == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kDotThreads / kWarp; ++i) s += red[i];
  }
  return s;
}

// partial[i * G + blockIdx.x] = sum over this CTA's slice of V_i . w,
// V_i = V + i * ldv, i = blockIdx.y.  gate (optional device flag): 0 skips
// the work (the reorthogonalisation pass that the DGKS test did not ask for).
__global__ void __launch_bounds__(kDotThreads) k_multidot_partial(const double *__restrict__ V, long long ldv,
                                                                  const double *__restrict__ w, long long len,
                                                                  double *partial, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  const int i = blockIdx.y;
  const double *vi = V + i * ldv;
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)kDotThreads + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * kDotThreads)
    acc = fma(vi[idx], w[idx], acc);
  double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(long long)i * gridDim.x + blockIdx.x] = s;
}

// The same for VB vectors per CTA: each thread streams its slice of w once
// against VB basis vectors (VB independent accumulators), so the per-CTA
// reduction is amortised over VB times more fused multiply-adds.
// partial[i * gridDim.x + blockIdx.x] for i = blockIdx.y * VB + v < m.
template <int VB>
__global__ void __launch_bounds__(kDotThreads) k_multidot_blocked(const double *__restrict__ V, long long ldv, int m,
                                                                  const double *__restrict__ w, long long len,
                                                                  double *partial, const int *gate) {
  if (gate && *gate == 0) return;
  __shared__ double red[kDotThreads / kWarp][VB];
  const int vb = blockIdx.y * VB;
  const int nv = min(VB, m - vb);
  double acc[VB];
#pragma unroll
  for (int v = 0; v < VB; ++v) acc[v] = 0.0;
  for (long long idx = blockIdx.x * (long long)kDotThreads + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * kDotThreads) {
    const double wv = w[idx];
#pragma unroll
    for (int v = 0; v < VB; ++v)
      if (v < nv) acc[v] = fma(V[(long long)(vb + v) * ldv + idx], wv, acc[v]);
  }
  const int wp = threadIdx.x / kWarp, ln = threadIdx.x & (kWarp - 1);
#pragma unroll
  for (int v = 0; v < VB; ++v) {
    double x = acc[v];
    if (v < nv) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
    }
    if (ln == 0) red[wp][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double sum = 0.0;
    for (int i = 0; i < kDotThreads / kWarp; ++i) sum += red[i][threadIdx.x];
    partial[(long long)(vb + threadIdx.x) * gridDim.x + blockIdx.x] = sum;
  }
}

// out[i] (+)= sum_g partial[i * G + g], fixed order.  One warp per i.
__global__ void k_reduce_partials(const double *__restrict__ partial, int G, int m, double *out, int accumulate,
                                  const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  const int i = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  const int ln = threadIdx.x & (kWarp - 1);
  if (i >= m) return;
  double s = 0.0;
  for (int g = ln; g < G; g += kWarp) s += partial[(long long)i * G + g];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
  if (ln == 0) out[i] = accumulate ? out[i] + s : s;
}

// y[idx] += sign * sum_{i < m} c[i] X_i[idx],  X_i = X + i * ldx
// (coefficients staged in shared memory; m <= 512; the vector loop is unrolled
// so that several basis loads are in flight per thread)
__global__ void k_multi_axpy(double *y, const double *__restrict__ X, long long ldx, const double *__restrict__ c,
                             int m, double sign, long long len, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  __shared__ double cs[512];
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int i = 0; i < m; ++i) acc = fma(cs[i], X[i * ldx + idx], acc);
    y[idx] = fma(sign, acc, y[idx]);
  }
}

// y -= sum_{i < m} c[i] X_i, and the CTA's partial sum of the new y^2 into
// partial[blockIdx.x] (fixed order), for the norm of the orthogonalised vector
__global__ void __launch_bounds__(kDotThreads) k_multi_axpy_norm(double *y, const double *__restrict__ X, long long ldx,
                                                                 const double *__restrict__ c, int m, long long len,
                                                                 double *partial) {
  __shared__ double cs[512];
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  double sq = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
#pragma unroll 8
    for (int i = 0; i < m; ++i) acc = fma(cs[i], X[i * ldx + idx], acc);
    const double v = y[idx] - acc;
    y[idx] = v;
    sq = fma(v, v, sq);
  }
  const double s = block_sum(sq);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// y[i] += x[i], i < m
__global__ void k_add_inplace(double *y, const double *__restrict__ x, int m, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) y[i] += x[i];
}

// y = x * s[0]
__global__ void k_scale(double *y, const double *__restrict__ x, const double *__restrict__ s, long long len) {
  const double a = s[0];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x)
    y[idx] = x[idx] * a;
}

// scal[0] = sqrt(nrm2[0]); scal[1] = 1 / scal[0] (0 if zero)
__global__ void k_norm_from_sq(const double *nrm2, double *scal) {
  double b = sqrt(nrm2[0]);
  scal[0] = b;
  scal[1] = b > 0.0 ? 1.0 / b : 0.0;
}

// Arnoldi column j: H[0..j][j] = h, H[j+1][j] = ||w||; apply the previous
// Givens rotations, form rotation j, update g.  H is column-major with leading
// dimension ldh.  scal: [0] |g_{j+1}|, [1] 1/h_{j+1,j}, [2] h_{j+1,j}.
__global__ void k_arnoldi_step(int j, const double *__restrict__ h, const double *__restrict__ w2, double *H,
                               int ldh, double *cs, double *sn, double *g, double *scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *col = H + (long long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h[i];
  const double hj1 = sqrt(w2[0]);
  col[j + 1] = hj1;
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j], b = col[j + 1];
  const double den = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (den != 0.0) {
    c = a / den;
    s = b / den;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = c * a + s * b;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  scal[0] = fabs(g[j + 1]);
  scal[1] = hj1 > 0.0 ? 1.0 / hj1 : 0.0;
  scal[2] = hj1;
}

// g = (beta, 0, ...), scal[0] = beta
__global__ void k_arnoldi_init(const double *beta_scal, double *g, int m) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta_scal[0] : 0.0;
}

// y = R^-1 g for the leading k x k upper triangle of the rotated H, one CTA,
// column-oriented: y_i = g_i / R_ii, then every g_r (r < i) -= R_ri y_i in parallel.
__global__ void k_backsolve(int k, const double *__restrict__ H, int ldh, const double *__restrict__ g, double *y) {
  extern __shared__ double gs[];
  for (int r = threadIdx.x; r < k; r += blockDim.x) gs[r] = g[r];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double yi = gs[i] / H[(long long)i * ldh + i];
    __syncthreads();
    if (threadIdx.x == 0) y[i] = yi;
    const double *col = H + (long long)i * ldh;
    for (int r = threadIdx.x; r < i; r += blockDim.x) gs[r] = fma(-col[r], yi, gs[r]);
    __syncthreads();
  }
}

}  // namespace pintmg
