// FP64 Krylov kernels for flexible GMRES (Saad 1993) and the coarse GMRES:
// multi-dot products with fixed-order reductions (bitwise reproducible),
// multi-axpy, and the Arnoldi/Givens bookkeeping on the device.  The
// FP32-pair basis option's kernels are in pair_kernels.cuh.
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
// V_i = V + i * ldv, i = blockIdx.y (the residual check that allocates
// nothing).  gate (optional device flag): 0 skips the work.
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

// Partition of the blocked dot products: the m vectors in ceil(m / VB)
// blocks, each block's length split into G chunks; a (block, chunk) pair is
// one work item with its own partial sum.  G depends on m only, so a launch
// whose m is read on the device (graph-captured solves) partitions exactly
// like one with m known on the host: the same partial sums, the same order.
// Few vectors: more, shorter chunks to fill the GPU; many vectors: fewer,
// longer ones (the per-item reduction is amortised, ~1200 items in flight);
// short vectors: at least 4 entries per thread and chunk.
__host__ __device__ inline int dot_parts(int m, int VB, long long len) {
  const int nb = (m + VB - 1) / VB;
  int G = nb <= 1 ? 304 : 1216 / nb;
  G = G < 40 ? 40 : (G > 152 && nb > 1 ? 152 : G);
  const long long cap = len / (4LL * kDotThreads);
  return cap < 1 ? 1 : (G > cap ? (int)cap : G);
}
constexpr int kDotGridCap = 1216;  // CTAs of a dot-product launch (8 per SM)

// Fixed-order sum over g < G of partial[i * G + g] by one warp (lane-strided
// sums, then a shuffle tree): the order of k_reduce_partials, so a fused
// reduction gives the same bits.  The result is valid in lane 0.
__device__ __forceinline__ double warp_partial_sum(const double *partial, int G, long long i, int ln) {
  double s = 0.0;
  for (int g = ln; g < G; g += kWarp) s += __ldcg(partial + i * G + g);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
  return s;
}

// true in every thread of the CTA that finishes last (its partial sums and
// those of every other CTA of the launch are then visible); the ticket counts
// the CTAs that have finished and is reset by the last one
__device__ __forceinline__ bool last_cta(unsigned *ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Sums over the 32 lanes of VB accumulators (VB = 2^b, b <= 5) as a
// reduce-scatter: in round r (partner lane ln ^ (16 >> r)) a lane keeps half
// of the values it still carries, the half picked by lane bit 4 - r, and adds
// the partner's copy of that half; after b rounds it carries one value, which
// the remaining rounds add up in full.  Every total follows the butterfly of a
// shuffle-down tree (leaves paired by lane bits 4, 3, 2, 1, 0 in that order,
// operands of an addition possibly swapped), so the totals are bitwise those
// of one such tree per accumulator, for every VB; a lane adds VB - 1 + 5 - b
// values instead of 5 VB (the FP64 adds compete with the dot products' FMAs
// for GB300's FP64 pipe).  Returns the total of accumulator ln / (32 / VB),
// held by every lane with those top b bits.
template <int VB>
__device__ __forceinline__ double warp_sum_scatter(const double (&acc)[VB], int ln) {
  static_assert(VB >= 1 && VB <= 32 && (VB & (VB - 1)) == 0, "VB must be a power of two up to 32");
  double cur[VB];
#pragma unroll
  for (int v = 0; v < VB; ++v) cur[v] = acc[v];
  int o = kWarp / 2;
#pragma unroll
  for (int n = VB; n > 1; n >>= 1, o >>= 1) {
    const bool upper = (ln & o) != 0;  // this round's lane bit: keep the upper half
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double keep = upper ? cur[n / 2 + i] : cur[i];
      const double send = upper ? cur[i] : cur[n / 2 + i];
      cur[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  double x = cur[0];
  for (; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// partial[i * G + g] = sum over chunk g of V_i . w for i < m, VB vectors per
// work item, G = dot_parts(m, VB, len); a persistent grid walks the items.  kPair:
// two consecutive entries per thread and step (16-byte loads; needs len and
// ldv even and 16-byte aligned V, w).  Each thread streams its slice of w once
// against VB basis vectors (VB independent accumulators), so the per-item
// reduction is amortised over VB times more fused multiply-adds.
// ticket non-null: the CTA that finishes last also reduces the partial sums
// into out[i] (+= with accumulate), in k_reduce_partials' order (one launch
// instead of two, the same bits).
template <int VB, bool kPair>
__global__ void __launch_bounds__(kDotThreads) k_multidot_blocked(const double *__restrict__ V, long long ldv, int m,
                                                                  const double *__restrict__ w, long long len,
                                                                  double *partial, const int *gate,
                                                                  const int *m_dev = nullptr,
                                                                  unsigned *ticket = nullptr, double *out = nullptr,
                                                                  int accumulate = 0) {
  if (gate && *gate == 0) return;
  if (m_dev) m = *m_dev;  // vector count held on the device (graph-captured solves)
  __shared__ double red[kDotThreads / kWarp][VB];
  const int G = dot_parts(m, VB, len);
  const int items = ((m + VB - 1) / VB) * G;
  const int wp = threadIdx.x / kWarp, ln = threadIdx.x & (kWarp - 1);
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int vb = (item / G) * VB, g = item % G;
    const int nv = min(VB, m - vb);
    double acc[VB];
#pragma unroll
    for (int v = 0; v < VB; ++v) acc[v] = 0.0;
    if (kPair) {
      const double2 *w2 = reinterpret_cast<const double2 *>(w);
      for (long long idx = g * (long long)kDotThreads + threadIdx.x; idx < len / 2;
           idx += (long long)G * kDotThreads) {
        const double2 wv = w2[idx];
#pragma unroll
        for (int v = 0; v < VB; ++v)
          if (v < nv) {
            // basis vectors are streamed once: load them evict-first so that w stays in L2
            const double2 x = __ldcs(reinterpret_cast<const double2 *>(V + (long long)(vb + v) * ldv) + idx);
            acc[v] = fma(x.x, wv.x, acc[v]);
            acc[v] = fma(x.y, wv.y, acc[v]);
          }
      }
    } else {
      for (long long idx = g * (long long)kDotThreads + threadIdx.x; idx < len; idx += (long long)G * kDotThreads) {
        const double wv = w[idx];
#pragma unroll
        for (int v = 0; v < VB; ++v)
          if (v < nv) acc[v] = fma(V[(long long)(vb + v) * ldv + idx], wv, acc[v]);
      }
    }
    // warp sums of the VB accumulators by a reduce-scatter: lane ln ends with
    // the sum of accumulator ln / (32 / VB) (the unused accumulators are 0)
    const double x = warp_sum_scatter<VB>(acc, ln);
    if ((ln & (kWarp / VB - 1)) == 0) red[wp][ln / (kWarp / VB)] = x;
    __syncthreads();
    if (threadIdx.x < nv) {
      double sum = 0.0;
      for (int i = 0; i < kDotThreads / kWarp; ++i) sum += red[i][threadIdx.x];
      partial[(long long)(vb + threadIdx.x) * G + g] = sum;
    }
    __syncthreads();  // red is reused by the next item
  }
  if (ticket && last_cta(ticket)) {
    for (int i = wp; i < m; i += kDotThreads / kWarp) {
      const double sum = warp_partial_sum(partial, G, i, ln);
      if (ln == 0) out[i] = accumulate ? out[i] + sum : sum;
    }
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

// out[i] (+)= sum_g partial[i * G + g], fixed order.  One warp per i.  With
// vb > 0, G = dot_parts(m, vb, len) (the partition of k_multidot_blocked).
// nr > 1: nr right-hand sides' sums of the same partition, out[r m + i]
__global__ void k_reduce_partials(const double *__restrict__ partial, int G, int m, double *out, int accumulate,
                                  const int *gate = nullptr, const int *m_dev = nullptr, int vb = 0,
                                  long long len = 0, int nr = 1) {
  if (gate && *gate == 0) return;
  if (m_dev) m = *m_dev;
  if (vb > 0) G = dot_parts(m, vb, len);
  const int i = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  const int ln = threadIdx.x & (kWarp - 1);
  if (i >= m * nr) return;
  double s = 0.0;
  for (int g = ln; g < G; g += kWarp) s += partial[(long long)i * G + g];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
  if (ln == 0) out[i] = accumulate ? out[i] + s : s;
}

// Arnoldi column j: H[0..j][j] = h, H[j+1][j] = ||w||; apply the previous
// Givens rotations, form rotation j, update g.  H is column-major with leading
// dimension ldh.  scal: [0] |g_{j+1}|, [1] 1/h_{j+1,j}, [2] h_{j+1,j}.
// One warp.  The previous rotations act on the new column as a first-order
// linear recurrence: with t_0 = h_0, rotation i gives
//   col_i = c_i t_i + s_i h_{i+1},   t_{i+1} = -s_i t_i + c_i h_{i+1},
// so each lane composes the affine maps of its chunk of rotations, a warp
// scan gives every chunk its incoming t, and the chunk is re-run; t_j meets
// h_{j+1,j} = ||w|| in the new rotation j.
__device__ __forceinline__ void arnoldi_column(int j, const double *h, double w2, double *H, int ldh, double *cs,
                                               double *sn, double *g, double *scal, int ln) {
  double *col = H + (long long)j * ldh;
  const double hj1 = sqrt(w2);
  const int ch = (j + kWarp - 1) / kWarp;
  const int i0 = min(ln * ch, j), i1 = min(i0 + ch, j);
  double A = 1.0, B = 0.0;  // this chunk's map t -> A t + B
  for (int i = i0; i < i1; ++i) {
    const double a = -sn[i];
    B = fma(a, B, cs[i] * h[i + 1]);
    A *= a;
  }
#pragma unroll
  for (int off = 1; off < kWarp; off <<= 1) {  // inclusive scan: compose with the lanes below
    const double Ap = __shfl_up_sync(kFull, A, off), Bp = __shfl_up_sync(kFull, B, off);
    if (ln >= off) {
      B = fma(A, Bp, B);
      A *= Ap;
    }
  }
  double Ae = __shfl_up_sync(kFull, A, 1), Be = __shfl_up_sync(kFull, B, 1);
  if (ln == 0) {
    Ae = 1.0;
    Be = 0.0;
  }
  double t = fma(Ae, h[0], Be);
  for (int i = i0; i < i1; ++i) {
    const double hi1 = h[i + 1];
    col[i] = fma(cs[i], t, sn[i] * hi1);
    t = fma(-sn[i], t, cs[i] * hi1);
  }
  const double Aall = __shfl_sync(kFull, A, kWarp - 1), Ball = __shfl_sync(kFull, B, kWarp - 1);
  if (ln != 0) return;
  const double a = fma(Aall, h[0], Ball), b = hj1;
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

__global__ void k_arnoldi_step(int j, const double *__restrict__ h, const double *__restrict__ w2, double *H,
                               int ldh, double *cs, double *sn, double *g, double *scal, const int *j_dev = nullptr) {
  if (blockIdx.x != 0 || threadIdx.x >= kWarp) return;
  if (j_dev) j = *j_dev;
  arnoldi_column(j, h, w2[0], H, ldh, cs, sn, g, scal, threadIdx.x);
}

// The end of a CGS2 step, run by the CTA that finishes the second
// orthogonalisation last: ||w||^2 from the CTAs' partial sums (the order of
// k_reduce_partials), h += h2 (the two passes' coefficients), then the
// Arnoldi column j with its Givens rotations (k_arnoldi_step).  One launch
// less than reduce + add + step, the same bits.
struct ArnoldiTail {
  unsigned *ticket;
  double *h;          // first pass's coefficients, summed in place with h2
  const double *h2;   // second pass's coefficients
  double *nrm2;       // receives ||w||^2
  double *H, *cs, *sn, *g, *scal;
  int ldh, j;
  const int *j_dev;   // the Arnoldi index on the device (graph-captured solves), else null
};

__device__ __forceinline__ void arnoldi_tail(const ArnoldiTail &t, const double *partial, int m) {
  const int wp = threadIdx.x / kWarp, ln = threadIdx.x & (kWarp - 1);
  __shared__ double s_w2;
  if (wp == 0) {
    const double sum = warp_partial_sum(partial, gridDim.x, 0, ln);
    if (ln == 0) {
      t.nrm2[0] = sum;
      s_w2 = sum;
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) t.h[i] += t.h2[i];
  __syncthreads();
  if (wp == 0) arnoldi_column(t.j_dev ? *t.j_dev : t.j, t.h, s_w2, t.H, t.ldh, t.cs, t.sn, t.g, t.scal, ln);
  if (threadIdx.x == 0) *t.ticket = 0u;
}

// y[idx] += sign * sum_{i < m} c[i] X_i[idx],  X_i = X + i * ldx
// (coefficients staged in shared memory; m <= 512; the vector loop is unrolled
// so that several basis loads are in flight per thread).  kPair: two
// consecutive entries per thread (16-byte loads; len, ldx even, y, X aligned);
// each entry's sum runs over i in the same order either way.
template <bool kPair>
__global__ void k_multi_axpy(double *y, const double *__restrict__ X, long long ldx, const double *__restrict__ c,
                             int m, double sign, long long len, const int *gate = nullptr,
                             const int *m_dev = nullptr) {
  if (gate && *gate == 0) return;
  if (m_dev) m = *m_dev;
  __shared__ double cs[512];
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  if (kPair) {
    double2 *y2 = reinterpret_cast<double2 *>(y);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len / 2;
         idx += (long long)gridDim.x * blockDim.x) {
      double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
      for (int i = 0; i < m; ++i) {
        const double2 x = reinterpret_cast<const double2 *>(X + i * ldx)[idx];
        a0 = fma(cs[i], x.x, a0);
        a1 = fma(cs[i], x.y, a1);
      }
      double2 v = y2[idx];
      v.x = fma(sign, a0, v.x);
      v.y = fma(sign, a1, v.y);
      y2[idx] = v;
    }
  } else {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
         idx += (long long)gridDim.x * blockDim.x) {
      double acc = 0.0;
#pragma unroll 8
      for (int i = 0; i < m; ++i) acc = fma(cs[i], X[i * ldx + idx], acc);
      y[idx] = fma(sign, acc, y[idx]);
    }
  }
}

// y -= sum_{i < m} c[i] X_i, and the CTA's partial sum of the new y^2 into
// partial[blockIdx.x] (fixed order), for the norm of the orthogonalised vector
template <bool kPair>
__global__ void __launch_bounds__(kDotThreads) k_multi_axpy_norm(double *y, const double *__restrict__ X, long long ldx,
                                                                 const double *__restrict__ c, int m, long long len,
                                                                 double *partial, const int *m_dev = nullptr,
                                                                 ArnoldiTail tail = {}) {
  if (m_dev) m = *m_dev;
  __shared__ double cs[512];
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  double sq = 0.0;
  if (kPair) {
    double2 *y2 = reinterpret_cast<double2 *>(y);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len / 2;
         idx += (long long)gridDim.x * blockDim.x) {
      double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
      for (int i = 0; i < m; ++i) {
        const double2 x = reinterpret_cast<const double2 *>(X + i * ldx)[idx];
        a0 = fma(cs[i], x.x, a0);
        a1 = fma(cs[i], x.y, a1);
      }
      double2 v = y2[idx];
      v.x -= a0;
      v.y -= a1;
      y2[idx] = v;
      sq = fma(v.x, v.x, sq);
      sq = fma(v.y, v.y, sq);
    }
  } else {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
         idx += (long long)gridDim.x * blockDim.x) {
      double acc = 0.0;
#pragma unroll 8
      for (int i = 0; i < m; ++i) acc = fma(cs[i], X[i * ldx + idx], acc);
      const double v = y[idx] - acc;
      y[idx] = v;
      sq = fma(v, v, sq);
    }
  }
  const double s = block_sum(sq);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (tail.ticket && last_cta(tail.ticket)) arnoldi_tail(tail, partial, m);
}

// y[i] += x[i], i < m
__global__ void k_add_inplace(double *y, const double *__restrict__ x, int m, const int *gate = nullptr,
                              const int *m_dev = nullptr) {
  if (gate && *gate == 0) return;
  if (m_dev) m = *m_dev;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) y[i] += x[i];
}

// y = x * s[0]; with idx non-null the destination is y + (idx[0] + shift) * len
// (a basis slot chosen on the device); guard non-null and 0 skips the work.
// also (optional): a second destination of the same values (the next iteration's
// preconditioner input, saving its copy from the basis)
__global__ void k_scale(double *y, const double *__restrict__ x, const double *__restrict__ s, long long len,
                        const int *idx = nullptr, int shift = 0, const int *guard = nullptr, double *also = nullptr) {
  if (guard && *guard == 0) return;
  if (idx) y += (long long)(idx[0] + shift) * len;
  const double a = s[0];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len;
       idx += (long long)gridDim.x * blockDim.x) {
    const double v = x[idx] * a;
    y[idx] = v;
    if (also) also[idx] = v;
  }
}

// scal[0] = sqrt(nrm2[0]); scal[1] = 1 / scal[0] (0 if zero)
__global__ void k_norm_from_sq(const double *nrm2, double *scal, const int *guard = nullptr) {
  if (guard && *guard == 0) return;
  double b = sqrt(nrm2[0]);
  scal[0] = b;
  scal[1] = b > 0.0 ? 1.0 / b : 0.0;
}

// g = (beta, 0, ...), scal[0] = beta
__global__ void k_arnoldi_init(const double *beta_scal, double *g, int m, const int *guard = nullptr) {
  if (guard && *guard == 0) return;
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = (i == 0) ? beta_scal[0] : 0.0;
}

// y = R^-1 g for the leading k x k upper triangle of the rotated H, one CTA,
// column-oriented: y_i = g_i / R_ii, then every g_r (r < i) -= R_ri y_i in parallel.
__global__ void k_backsolve(int k, const double *__restrict__ H, int ldh, const double *__restrict__ g, double *y,
                            const int *k_dev = nullptr, const int *guard = nullptr) {
  if (guard && *guard == 0) return;
  if (k_dev) k = *k_dev;
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

// start of a DCGS2 cycle: eta = ||r|| (scal[0]), 1 / eta (scal[1])
__global__ void k_dcgs2_start(const double *__restrict__ scal, double *dc, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  if (threadIdx.x == 0) {
    dc[3] = scal[0];
    dc[0] = scal[1];
  }
}

// DCGS2 step j (one warp; j from j_dev when given).  out: the pass's dot
// products, out[i] = V_i . u and out[j + i] = V_i . w (i < j); dc as in
// k_multi_axpy2_pair, with dc[4] = u . w.  With s = out[0..j) / eta and
// nu = (1 - |s|^2)^(1/2):
//   j >= 1: column j - 1 of H becomes hp + eta s with H[j][j-1] = eta nu, and
//           is rotated (arnoldi_column: scal[0] = |g_j|, the residual estimate
//           of the first j columns);
//   close == 0: the coefficients of the update pass, c1 = s, c2 = t =
//           out[j..2j), dc[1] = 1 / nu, dc[2] = h_j = (u . w / eta - s . t) / nu,
//           and the pending column j, hp = (t, h_j).
// close = 1 ends a cycle: only column j - 1 (out[j..) is not read).  A
// non-positive 1 - |s|^2 makes nu NaN (breakdown, seen in the estimate).
__global__ void k_dcgs2_coef(int j, const int *j_dev, const double *__restrict__ out, double *dc, double *c1,
                             double *c2, double *hp, double *H, int ldh, double *cs, double *sn, double *g,
                             double *scal, int close, const int *gate = nullptr) {
  if (gate && *gate == 0) return;
  if (j_dev) j = *j_dev;
  if (threadIdx.x >= kWarp) return;
  const int ln = threadIdx.x;
  __shared__ double hcol[512];
  const double inv_eta = dc[0], eta = dc[3];
  double ss = 0.0, st = 0.0;
  for (int i = ln; i < j; i += kWarp) {
    const double si = out[i] * inv_eta;
    ss = fma(si, si, ss);
    if (!close) st = fma(si, out[j + i], st);
    hcol[i] = fma(eta, si, hp[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(kFull, ss, o);
    st += __shfl_xor_sync(kFull, st, o);
  }
  const double nu2 = 1.0 - ss;
  const double nu = nu2 > 0.0 ? sqrt(nu2) : __longlong_as_double(0x7FF8000000000000LL);
  __syncwarp();
  if (j >= 1) arnoldi_column(j - 1, hcol, eta * eta * nu2, H, ldh, cs, sn, g, scal, ln);
  if (close) return;
  for (int i = ln; i < j; i += kWarp) {
    c1[i] = out[i] * inv_eta;
    c2[i] = out[j + i];
    hp[i] = out[j + i];
  }
  if (ln == 0) {
    const double hj = (dc[4] * inv_eta - st) / nu;
    hp[j] = hj;
    dc[1] = 1.0 / nu;
    dc[2] = hj;
  }
}

// ---------------------------------------------------------------------------
// Device-side control of the Krylov loops for graph-captured solves: the
// loop state lives on the device and a control kernel sets the condition of
// the enclosing WHILE node (no host round trip per iteration).

struct KState {
  int j;          // Arnoldi index within the current cycle
  int m1;         // j + 1: vectors to orthogonalise against
  int total;      // iterations of this solve
  int done;       // solve finished (converged, breakdown or iteration cap)
  int cycle_end;  // the current cycle must be closed (least squares + update)
  int restart;    // cycle_end && !done: a new cycle starts from the true residual
  int kcount;     // columns of the current least-squares problem
  int breakdown;  // non-finite Hessenberg entry
  int converged;
  int pad;
  int go;         // DCGS2: the step's update pass runs (the cycle did not end at its lagged column)
  int close;      // DCGS2: the cycle ends with the closing pass over V^T u
  int bodies;     // DCGS2: loop bodies executed in this solve (a step that ends a cycle adds no column)
  int pad2;
  long long calls;      // solves since setup
  long long iters_all;  // iterations summed over calls
  double bnorm, rtol;
  double est;           // last Arnoldi residual estimate |g_{j+1}|
};

// start of a solve: beta = scal[0] (= ||r||); nothing to do if beta == 0
// admitted (optional): the learned coarse correction was accepted, nothing to iterate
__global__ void k_ctl_start(KState *st, const double *scal, double rtol, cudaGraphConditionalHandle h,
                            const int *admitted = nullptr) {
  const double beta = scal[0];
  st->go = 0;
  st->close = 0;
  st->bodies = 0;
  st->j = 0;
  st->m1 = 1;
  st->total = 0;
  st->kcount = 0;
  st->cycle_end = 0;
  st->restart = 0;
  st->breakdown = 0;
  st->converged = 0;
  st->bnorm = beta;
  st->rtol = rtol;
  st->done = (beta > 0.0 && !(admitted && admitted[0])) ? 0 : 1;
  st->calls += 1;
  cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

// after Arnoldi step j (scal: [0] |g_{j+1}|, [2] h_{j+1,j}): advance and test.
// cycle = restart length; for the coarse loop (restart none) the WHILE
// condition is set here; for the outer loop k_ctl_continue sets it.
__global__ void k_ctl_step(KState *st, const double *scal, int cycle, int maxit, int set_here,
                           cudaGraphConditionalHandle h) {
  const double est = scal[0], hj1 = scal[2];
  st->est = est;
  st->j += 1;
  st->m1 = st->j + 1;
  st->total += 1;
  st->iters_all += 1;
  st->kcount = st->j;
  const bool bad = !isfinite(est) || !isfinite(hj1);
  const bool conv = !bad && (est <= st->rtol * st->bnorm || hj1 == 0.0);
  st->breakdown = bad ? 1 : 0;
  st->converged = conv ? 1 : 0;
  const bool last = st->total >= maxit;
  st->cycle_end = (bad || conv || last || st->j >= cycle) ? 1 : 0;
  st->done = (bad || conv || last) ? 1 : 0;
  st->restart = (st->cycle_end && !st->done) ? 1 : 0;
  if (set_here) cudaGraphSetConditional(h, st->cycle_end ? 0u : 1u);
}

// DCGS2, after k_dcgs2_coef of step j (graph-captured solves): j >= 1 has
// just finished column j - 1 (scal: [0] |g_j|, [2] its subdiagonal); a
// converged or broken-down column ends the cycle with j columns (no update
// pass, no closing pass).  Otherwise the update pass runs (go) and, when this
// step fills the cycle (j + 1 = cycle) or reaches the iteration cap, the
// closing pass follows (close).  total counts finished columns.
__global__ void k_dcgs2_ctl(KState *st, const double *scal, int cycle, int maxit) {
  const int j = st->j;
  st->bodies += 1;
  st->go = 1;
  st->close = 0;
  st->cycle_end = 0;
  st->restart = 0;
  // every body either finishes a column or ends a cycle, so a solve needs at most about
  // 2 maxit bodies; past that the loop ends as a breakdown rather than running on
  if (st->bodies > 2 * maxit + 64) {
    st->breakdown = 1;
    st->converged = 0;
    st->kcount = j;
    st->go = 0;
    st->cycle_end = 1;
    st->done = 1;
    return;
  }
  if (j >= 1) {
    const double est = scal[0], hj1 = scal[2];
    st->est = est;
    const bool bad = !isfinite(est) || !isfinite(hj1);
    const bool conv = !bad && (est <= st->rtol * st->bnorm || hj1 == 0.0);
    if (bad || conv) {
      st->breakdown = bad ? 1 : 0;
      st->converged = conv ? 1 : 0;
      st->kcount = j;
      st->total += j;
      st->iters_all += j;
      st->go = 0;
      st->cycle_end = 1;
      st->done = 1;
      st->restart = 0;
      return;
    }
  }
  if (j + 1 >= cycle || st->total + j + 1 >= maxit) {
    st->close = 1;
    st->cycle_end = 1;
  }
}

// DCGS2: after a step's update pass, one more final basis vector
__global__ void k_dcgs2_adv(KState *st) {
  if (st->go) st->j += 1;
}

// DCGS2: after the closing pass (k_dcgs2_coef with close = 1) the cycle holds j columns
__global__ void k_dcgs2_closed(KState *st, const double *scal, int maxit) {
  if (!st->close) return;
  const int j = st->j;
  const double est = scal[0], hj1 = scal[2];
  st->est = est;
  const bool bad = !isfinite(est) || !isfinite(hj1);
  const bool conv = !bad && (est <= st->rtol * st->bnorm || hj1 == 0.0);
  st->breakdown = bad ? 1 : 0;
  st->converged = conv ? 1 : 0;
  st->kcount = j;
  st->total += j;
  st->iters_all += j;
  st->done = (bad || conv || st->total >= maxit) ? 1 : 0;
  st->restart = st->done ? 0 : 1;
}

// dst = src (len entries) when the gate is open
__global__ void k_copy_gated(double *dst, const double *__restrict__ src, long long len, const int *gate) {
  if (gate && *gate == 0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// end of an outer iteration: a closed cycle that is not the last restarts at j = 0
__global__ void k_ctl_continue(KState *st, cudaGraphConditionalHandle h) {
  if (st->restart) {
    st->j = 0;
    st->m1 = 1;
    st->cycle_end = 0;
  }
  cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

// dst = src_base + idx[0] * len (copy a basis slot chosen on the device) or the reverse
__global__ void k_copy_indexed(double *dst, const double *__restrict__ src, long long len, const int *idx,
                               int dst_indexed) {
  const long long off = (long long)idx[0] * len;
  const double *sp = dst_indexed ? src : src + off;
  double *dp = dst_indexed ? dst + off : dst;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dp[i] = sp[i];
}

// learned coarse correction: admitted if ||r - A e|| <= admit ||r||
// (rr2 = ||r - A e||^2, scal[0] = ||r||); flag[0] = decision, flag[1] counts admissions
__global__ void k_net_admit(const double *rr2, const double *scal, double admit, int *flag) {
  const bool ok = sqrt(rr2[0]) <= admit * scal[0] && scal[0] > 0.0;
  flag[0] = ok ? 1 : 0;
  if (ok) flag[1] += 1;
}

// dst = src where flag[0] != 0
__global__ void k_copy_if(double *dst, const double *__restrict__ src, long long n, const int *flag) {
  if (!flag[0]) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// a training pair: r / rms(r) and y / rms(r) in FP32 (inv = 1 / rms(r) = sqrt(n) / ||r||)
__global__ void k_record_pair(const double *__restrict__ r, const double *__restrict__ y, double inv, float *rr,
                              float *yy, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    rr[i] = (float)(r[i] * inv);
    yy[i] = (float)(y[i] * inv);
  }
}

// power iteration: x = y / ||y|| (nrm2[0] = ||y||^2); acc[0] += log ||y||, acc[1] += 1 when counting
__global__ void k_power_step(const double *__restrict__ y, double *x, long long n, const double *nrm2, double *acc,
                             int counting) {
  const double nr = sqrt(nrm2[0]);
  const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = y[i] * inv;
  if (counting && blockIdx.x == 0 && threadIdx.x == 0 && nr > 0.0) {
    acc[0] += log(nr);
    acc[1] += 1.0;
  }
}

// a fixed, non-degenerate start vector for the power iteration
__global__ void k_power_start(double *x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = 1.0 + 0.5 * (double)((i * 2654435761ULL) % 1000ULL) / 1000.0;
}

}  // namespace pintmg
