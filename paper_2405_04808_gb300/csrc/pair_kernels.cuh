// Krylov basis vectors stored as pairs of FP32 values, and the dot products
// and axpys against them in compensated FP32 arithmetic.
//
// GB300 issues FP64 fused multiply-adds at 1/64 of its FP32 rate, so the
// FP64 multi-dot products and multi-axpys of the Gram-Schmidt passes are
// bound by the FP64 pipe, not by HBM.  Here a basis entry x is stored as
// (hi, lo), hi = x rounded to 24 significant bits and lo = the remainder
// rounded to FP32 (8 bytes, as in FP64; x is kept to about 48 bits), and each
// product with an FP64 operand split the same way is evaluated as in the Dot2
// algorithm of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J.
// Sci. Comput. 26, 2005): the leading product hi*hi' exactly as a sum of two
// floats (TwoProduct by FMA), its running sum exactly by Knuth's TwoSum, and
// the cross terms hi*lo' + lo*hi' and all rounding errors in a second FP32
// accumulator.  Each thread's result is a double-single value with about 48
// significant bits; the warp and block reductions and the final scaling are
// done in FP64.  The FP32 exponent range is handled by scaling the FP64
// operand by a power of two (exactly, in the exponent field) chosen per warp
// or per CTA from the largest exponent it holds.
#pragma once

#include "common.cuh"

namespace pintmg {

// biased FP64 exponent field of x
__device__ __forceinline__ unsigned f64_exponent(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu;
}

// x * 2^(896 - eoff) as (hi, lo) FP32: hi = the 53-bit significand rounded to
// 24 bits (ties away from zero, by integer arithmetic), lo = the remainder
// (at most 29 bits, signed) rounded to FP32 by the integer-to-float
// conversion.  eoff = 896 keeps the value.  Zero and FP64 subnormals give 0,
// values whose scaled hi is below the FP32 normal range are flushed to 0, a
// remainder below it is dropped; NaN and infinity give NaN.
__device__ __forceinline__ float2 split48(double x, int eoff) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int eh = e - eoff;  // FP32 exponent field of the scaled hi (before a rounding carry)
  if (e == 0x7FF) return make_float2(__int_as_float(0x7FC00000), 0.0f);
  if (e == 0 || eh < 1) return make_float2(0.0f, 0.0f);
  if (eh > 253) return make_float2(__int_as_float((int)(sign | 0x7F800000u)), 0.0f);
  // rounding: add half an ulp of the 24-bit result; a carry runs into the exponent
  const unsigned long long a = (b & 0x7FFFFFFFFFFFFFFFull) + (1ull << 28);
  const unsigned hbits = (unsigned)(a >> 29) - ((unsigned)eoff << 23);
  // remainder: the low 29 bits as a signed value (negative when hi was rounded up)
  const int r = ((int)((unsigned)b << 3)) >> 3;
  const int el = eh - 52;  // FP32 exponent field of the remainder's unit 2^(e - 1075), scaled
  float lo = 0.0f;
  if (el >= 1) lo = __fmul_rn(__int2float_rn(r), __int_as_float(el << 23));
  return make_float2(__int_as_float((int)(hbits | sign)), __int_as_float(__float_as_int(lo) ^ (int)sign));
}

// 2^(e - 1023) for a biased FP64 exponent field e in [1, 2046]; 0 for e = 0
__device__ __forceinline__ double pow2_of_exponent(unsigned e) {
  return e == 0 ? 0.0 : __longlong_as_double((long long)e << 52);
}

// (hi + lo) * 2^(eoff - 896) in FP64
__device__ __forceinline__ double pair_value(float2 p, double scale) {
  return ((double)p.x + (double)p.y) * scale;
}

// s + c += (vh + vl) * (wh + wl): TwoProduct of the leading terms, TwoSum into
// s, everything else into c.  The intrinsics keep each operation rounded on
// its own (no contraction into FMAs).
__device__ __forceinline__ void dot2_step(float &s, float &c, float vh, float vl, float wh, float wl) {
  const float p = __fmul_rn(vh, wh);
  const float e = __fmaf_rn(vh, wh, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, e));
  c = __fmaf_rn(vh, wl, c);
  c = __fmaf_rn(vl, wh, c);
}

// (s, c) += (s2, c2) with the TwoSum of the leading parts
__device__ __forceinline__ void ds_add(float &s, float &c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, c2));
}

// dst[i] = split48(src[i] * mul) (mul = 1/||w|| for a new basis vector, or
// read from the device); the basis slot may be chosen on the device
// (dst + idx[0] * len)
// also (optional): the stored pair's FP64 value (what k_join_basis would read back), for the next
// iteration's preconditioner input
__global__ void k_split_basis(float2 *dst, const double *__restrict__ src, const double *mul, long long len,
                              const int *idx = nullptr, int idx_add = 0, const int *gate = nullptr,
                              double *also = nullptr) {
  if (gate && *gate == 0) return;
  const double a = mul ? *mul : 1.0;
  if (idx) dst += (long long)(idx[0] + idx_add) * len;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = split48(src[i] * a, 896);
    dst[i] = v;
    if (also) also[i] = pair_value(v, 1.0);
  }
}

// dst[i] = hi + lo of basis slot idx[0] (or of src itself when idx is null), in FP64
__global__ void k_join_basis(double *dst, const float2 *__restrict__ src, long long len, const int *idx = nullptr) {
  if (idx) src += (long long)idx[0] * len;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = pair_value(src[i], 1.0);
}

// y += sign * sum_{i < m} c[i] X_i (X_i = X + i * ldx, pairs), each entry's
// sum in double-single FP32 over i with the coefficients scaled by
// 2^(1023 - emax(c)) and split in shared memory; the update of y in FP64.
// kNorm: also the CTA's partial sum of the new y^2 into partial[blockIdx.x].
// len and ldx even, y and X 16-byte aligned; m <= 512.
template <bool kNorm>
__global__ void __launch_bounds__(kDotThreads) k_multi_axpy_pair(double *y, const float2 *__restrict__ X, long long ldx,
                                                                 const double *__restrict__ c, int m, double sign,
                                                                 long long len, double *partial, const int *gate,
                                                                 const int *m_dev = nullptr, ArnoldiTail tail = {}) {
  if (gate && *gate == 0) return;
  if (m_dev) m = *m_dev;
  __shared__ float2 cs[512];
  __shared__ unsigned cmax[kDotThreads / kWarp];
  unsigned e = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) e = max(e, f64_exponent(c[i]));
  e = __reduce_max_sync(kFull, e);
  if ((threadIdx.x & (kWarp - 1)) == 0) cmax[threadIdx.x / kWarp] = e;
  __syncthreads();
  unsigned emax = 0;
#pragma unroll
  for (int i = 0; i < kDotThreads / kWarp; ++i) emax = max(emax, cmax[i]);
  const int eoff = (int)emax - 127;
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = split48(c[i], eoff);
  __syncthreads();
  const double scale = sign * pow2_of_exponent(emax);
  double sq = 0.0;
  double2 *y2 = reinterpret_cast<double2 *>(y);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len / 2;
       idx += (long long)gridDim.x * blockDim.x) {
    float s0 = 0.0f, c0 = 0.0f, s1 = 0.0f, c1 = 0.0f;
#pragma unroll 8
    for (int i = 0; i < m; ++i) {
      const float4 x = reinterpret_cast<const float4 *>(X + i * ldx)[idx];
      const float2 ci = cs[i];
      dot2_step(s0, c0, x.x, x.y, ci.x, ci.y);
      dot2_step(s1, c1, x.z, x.w, ci.x, ci.y);
    }
    double2 v = y2[idx];
    v.x = fma(scale, (double)s0 + (double)c0, v.x);
    v.y = fma(scale, (double)s1 + (double)c1, v.y);
    y2[idx] = v;
    if (kNorm) {
      sq = fma(v.x, v.x, sq);
      sq = fma(v.y, v.y, sq);
    }
  }
  if (kNorm) {
    const double t = block_sum(sq);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
    if (tail.ticket && last_cta(tail.ticket)) arnoldi_tail(tail, partial, m);
  }
}

// ---------------------------------------------------------------------------
// Delayed reorthogonalisation (DCGS2; Bielich, Langou, Thomas, Swirydowicz,
// Yamazaki and Boman, Parallel Computing 2022) on the pair basis.  At Arnoldi
// step j the basis holds the final orthonormal V_0 .. V_{j-1} and, in slot j,
// the tentative vector vt_j = u / eta of the previous step (u its FP64 copy,
// eta = ||u||); w = A z_j.  One pass over V_0 .. V_{j-1} forms
// s' = V^T u and t = V^T w (k_multidot_pair_tma with two right-hand sides),
// k_dcgs2_coef finishes column j - 1 of the Hessenberg matrix with s = s' /
// eta and nu = (1 - |s|^2)^(1/2) (u's component outside the basis) and forms
// h_j = (vt_j . w - s . t) / nu, and one more pass (k_multi_axpy2_pair) writes
// the final V_j = (vt_j - V s) / nu and w' = w - V t - h_j V_j: two passes over
// the basis per step instead of CGS2's four.
//
// dc: the step's scalars, [0] 1 / eta, [1] 1 / nu, [2] h_j, [3] eta, [4]
// u . w (FP64 dot product of the step), [5] ||w'||^2.

// y = u dc[0] - sum_i s_i V_i, scaled by dc[1], into basis slot m (m = the
// final vectors, read from m_dev when given) as a pair; then u = w - sum_i t_i V_i
// - dc[2] y (FP64) and the CTA's partial sum of u^2; the last CTA (ticket)
// reduces the partials into dc[5], dc[3] = ||u||, dc[0] = 1 / ||u||.  s, t:
// the coefficients (m each), scaled per CTA by powers of two and split as in
// k_multi_axpy_pair.  len and ldx even, u, w, V 16-byte aligned; m <= 512.
__global__ void __launch_bounds__(kDotThreads) k_multi_axpy2_pair(float2 *V, long long ldx, const double *__restrict__ s,
                                                                  const double *__restrict__ t, int m, double *u,
                                                                  const double *__restrict__ w, long long len,
                                                                  double *dc, double *partial, unsigned *ticket,
                                                                  const int *gate, const int *m_dev) {
  if (gate && *gate == 0) return;
  if (m_dev) m = *m_dev;
  __shared__ float2 cs1[512], cs2[512];
  __shared__ unsigned cmax[2][kDotThreads / kWarp];
  unsigned e1 = 0, e2 = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    e1 = max(e1, f64_exponent(s[i]));
    e2 = max(e2, f64_exponent(t[i]));
  }
  e1 = __reduce_max_sync(kFull, e1);
  e2 = __reduce_max_sync(kFull, e2);
  if ((threadIdx.x & (kWarp - 1)) == 0) {
    cmax[0][threadIdx.x / kWarp] = e1;
    cmax[1][threadIdx.x / kWarp] = e2;
  }
  __syncthreads();
  unsigned emax1 = 0, emax2 = 0;
#pragma unroll
  for (int i = 0; i < kDotThreads / kWarp; ++i) {
    emax1 = max(emax1, cmax[0][i]);
    emax2 = max(emax2, cmax[1][i]);
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    cs1[i] = split48(s[i], (int)emax1 - 127);
    cs2[i] = split48(t[i], (int)emax2 - 127);
  }
  __syncthreads();
  const double sc1 = pow2_of_exponent(emax1), sc2 = pow2_of_exponent(emax2);
  const double inv_eta = dc[0], inv_nu = dc[1], hj = dc[2];
  float4 *slot = reinterpret_cast<float4 *>(V + (long long)m * ldx);
  double2 *u2 = reinterpret_cast<double2 *>(u);
  const double2 *w2 = reinterpret_cast<const double2 *>(w);
  double sq = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < len / 2;
       idx += (long long)gridDim.x * blockDim.x) {
    float a0 = 0.f, ca0 = 0.f, a1 = 0.f, ca1 = 0.f, b0 = 0.f, cb0 = 0.f, b1 = 0.f, cb1 = 0.f;
    auto step = [&](const float4 &x, int i) {
      const float2 p = cs1[i], q = cs2[i];
      dot2_step(a0, ca0, x.x, x.y, p.x, p.y);
      dot2_step(a1, ca1, x.z, x.w, p.x, p.y);
      dot2_step(b0, cb0, x.x, x.y, q.x, q.y);
      dot2_step(b1, cb1, x.z, x.w, q.x, q.y);
    };
    int i = 0;
    for (; i + 8 <= m; i += 8) {  // eight basis loads in flight, then their products in order
      float4 x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = reinterpret_cast<const float4 *>(V + (i + k) * ldx)[idx];
#pragma unroll
      for (int k = 0; k < 8; ++k) step(x[k], i + k);
    }
    for (; i < m; ++i) step(reinterpret_cast<const float4 *>(V + i * ldx)[idx], i);
    const double2 uv = u2[idx], wv = w2[idx];
    const double y0 = (uv.x * inv_eta - sc1 * ((double)a0 + (double)ca0)) * inv_nu;
    const double y1 = (uv.y * inv_eta - sc1 * ((double)a1 + (double)ca1)) * inv_nu;
    const float2 p0 = split48(y0, 896), p1 = split48(y1, 896);
    slot[idx] = make_float4(p0.x, p0.y, p1.x, p1.y);
    double2 nu;
    nu.x = fma(-hj, y0, fma(-sc2, (double)b0 + (double)cb0, wv.x));
    nu.y = fma(-hj, y1, fma(-sc2, (double)b1 + (double)cb1, wv.y));
    u2[idx] = nu;
    sq = fma(nu.x, nu.x, sq);
    sq = fma(nu.y, nu.y, sq);
  }
  const double tt = block_sum(sq);
  if (threadIdx.x == 0) partial[blockIdx.x] = tt;
  if (last_cta(ticket)) {
    if (threadIdx.x < kWarp) {
      const double n2 = warp_partial_sum(partial, gridDim.x, 0, threadIdx.x);
      if (threadIdx.x == 0) {
        const double eta = sqrt(n2);
        dc[5] = n2;
        dc[3] = eta;
        dc[0] = eta > 0.0 ? 1.0 / eta : 0.0;
      }
    }
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

// ---------------------------------------------------------------------------
// Multi-dot products against the pair basis with the basis streamed into
// shared memory by bulk asynchronous copies (TMA, cp.async.bulk) through a
// ring of NS stages, each holding kPairStageLen entries of VB basis
// vectors and of w.  One producer warp issues the copies; eight consumer
// warps evaluate the compensated products from shared memory, so the number
// of bytes in flight per SM no longer depends on registers.  Every wait on an
// mbarrier is bounded; a wait that runs out sets err[0] and the CTA stops
// issuing and consuming (after waiting, again bounded, for its copies).

constexpr int kPairStageLen = 512;     // entries per stage (two per consumer thread)
constexpr int kPairConsumers = 8;      // consumer warps
constexpr int kPairTmaThreads = (kPairConsumers + 1) * kWarp;
constexpr unsigned long long kPairWaitNs = 2000000000ull;  // longest wait on an mbarrier (2 s) before giving up

// chunk length of the TMA multi-dot partition: the vectors' length in G
// contiguous even-length chunks (the last may be shorter or empty)
__host__ __device__ inline long long pair_chunk(long long len, int G) {
  const long long c = (len + G - 1) / G;
  return (c + 1) & ~1ll;
}

template <int VB, int NS, int NR = 1>
__host__ __device__ constexpr size_t pair_tma_smem() {
  return (size_t)NS * kPairStageLen * (VB * sizeof(float2) + NR * sizeof(double)) +
         2 * NS * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
// wait until the phase with the given parity has completed; false once
// kPairWaitNs have passed (checked every 64 polls)
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > kPairWaitNs) return false;
  }
}
// bulk copy of bytes (a multiple of 16, both addresses 16-byte aligned) into shared memory
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar,
                                          unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// partial[i * G + g] = sum over chunk g (entries [g C, min(len, (g+1) C)),
// C = pair_chunk(len, G), G = dot_parts(m, VB, len)) of V_i . w.  Requires
// len and ldv even and V, w 16-byte aligned; dynamic shared memory
// pair_tma_smem<VB>(); blockDim = kPairTmaThreads.  Each consumer warp keeps a
// running scale 2^(emax - 1023) for its entries of w (emax: the largest FP64
// exponent seen so far); when a stage raises it, the FP32 accumulators are
// rescaled by the (exact) power of two.  A wait that runs out sets err[0];
// later launches with err[0] set return at once.
// NR = 2: a second right-hand side w2 streamed beside w (DCGS2's pass over the
// basis, Q^T [u, w]); the partial sums of w2 follow those of w:
// partial[(r m + i) G + g] for right-hand side r.
template <int VB, int NS, int kMinBlocks, int NR = 1>
__global__ void __launch_bounds__(kPairTmaThreads, kMinBlocks)
    k_multidot_pair_tma(const float2 *__restrict__ V, long long ldv, int m, const double *__restrict__ w, long long len,
                        double *partial, const int *gate, const int *m_dev, int *err, int stall = 0,
                        const double *__restrict__ w2 = nullptr) {
  if (gate && *gate == 0) return;
  if (*(volatile int *)err) return;  // an earlier launch of this solve timed out: its results are void anyway
  if (m_dev) m = *m_dev;
  extern __shared__ __align__(128) unsigned char pair_smem[];
  float2 *sv = reinterpret_cast<float2 *>(pair_smem);  // [stage][VB][kPairStageLen]
  double *sw = reinterpret_cast<double *>(sv + (size_t)NS * VB * kPairStageLen);  // [stage][NR][len]
  unsigned long long *full = reinterpret_cast<unsigned long long *>(sw + (size_t)NS * NR * kPairStageLen);
  unsigned long long *empty = full + NS;
  __shared__ double red[kPairConsumers][NR][VB];
  __shared__ int abort_flag;
  const int G = dot_parts(m, VB, len);
  const long long C = pair_chunk(len, G);
  const int items = ((m + VB - 1) / VB) * G;
  const int wp = threadIdx.x / kWarp, ln = threadIdx.x & (kWarp - 1);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kPairConsumers);
    }
    abort_flag = 0;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  if (wp == kPairConsumers) {  // producer warp: one lane issues the copies
    // stall == 1 (failure-detection tests only): issue nothing, so that the
    // consumers' waits run out and the launch reports a timeout
    if (ln == 0 && stall != 1) {
      unsigned long long policy;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(policy));
      unsigned long long keep;
      asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(keep));
      long long q = 0;  // stages issued
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const int vb = (item / G) * VB, g = item % G;
        const int nv = min(VB, m - vb);
        const long long c0 = g * C, c1 = min(len, c0 + C);
        for (long long pos = c0; pos < c1; pos += kPairStageLen, ++q) {
          const int slot = (int)(q % NS);
          const unsigned use = (unsigned)(q / NS);
          if (!mbar_wait(&empty[slot], (use & 1u) ^ 1u) || *(volatile int *)&abort_flag) {
            ok = false;
            break;
          }
          const unsigned ne = (unsigned)min((long long)kPairStageLen, c1 - pos);
          mbar_expect_tx(&full[slot], ne * (unsigned)(nv * sizeof(float2) + NR * sizeof(double)));
          bulk_load(sw + (size_t)slot * NR * kPairStageLen, w + pos, ne * (unsigned)sizeof(double), &full[slot], keep);
          if (NR == 2)
            bulk_load(sw + ((size_t)slot * NR + 1) * kPairStageLen, w2 + pos, ne * (unsigned)sizeof(double),
                      &full[slot], keep);
          for (int v = 0; v < nv; ++v)
            bulk_load(sv + ((size_t)slot * VB + v) * kPairStageLen, V + (long long)(vb + v) * ldv + pos,
                      ne * (unsigned)sizeof(float2), &full[slot], policy);
        }
      }
      if (!ok) {
        atomicOr(err, 1);
        *(volatile int *)&abort_flag = 1;
      }
      // Let every copy this lane issued land before it returns, whether or not
      // the consumers still wait for them (a consumer that gives up skips its
      // waits, and the CTA must not exit with bulk copies in flight).  Stage k
      // is the last use of its slot for k >= q - NS, so its full barrier's
      // phase (k / NS) & 1 completes exactly when its bytes have arrived; in a
      // healthy run these phases have completed already.
      for (long long k = (q > NS ? q - NS : 0); k < q; ++k)
        mbar_wait(&full[(int)(k % NS)], (unsigned)(k / NS) & 1u);
    }
    return;
  }
  // consumer warps; a warp that gave up (dead) keeps walking the items so that
  // the named barriers of the consumer warps still match
  long long q = 0;
  bool dead = false;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int vb = (item / G) * VB, g = item % G;
    const int nv = min(VB, m - vb);
    const long long c0 = g * C, c1 = min(len, c0 + C);
    float s[NR][VB], c[NR][VB];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int v = 0; v < VB; ++v) s[r][v] = c[r][v] = 0.0f;
    unsigned emax[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) emax[r] = 0;
    for (long long pos = c0; pos < c1; pos += kPairStageLen, ++q) {
      const int slot = (int)(q % NS);
      const unsigned use = (unsigned)(q / NS);
      if (!dead) {
        const bool ok = !*(volatile int *)&abort_flag && mbar_wait(&full[slot], use & 1u);
        dead = __any_sync(kFull, !ok);
        if (dead && ln == 0) {
          atomicOr(err, 1);
          *(volatile int *)&abort_flag = 1;
        }
      }
      if (dead) continue;
      const int ne = (int)min((long long)kPairStageLen, c1 - pos);
      const int e0 = 2 * ln + 2 * kWarp * wp;  // this thread's two entries of the stage
      const bool mine = e0 < ne;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        double2 wv = make_double2(0.0, 0.0);
        if (mine) wv = reinterpret_cast<const double2 *>(sw + ((size_t)slot * NR + r) * kPairStageLen)[e0 / 2];
        const unsigned en = __reduce_max_sync(kFull, max(f64_exponent(wv.x), f64_exponent(wv.y)));
        if (en > emax[r]) {
          if (emax[r] != 0) {
            const unsigned d = en - emax[r];
            const float f = d > 120 ? 0.0f : __int_as_float((int)(127 - d) << 23);
#pragma unroll
            for (int v = 0; v < VB; ++v) {
              s[r][v] = __fmul_rn(s[r][v], f);
              c[r][v] = __fmul_rn(c[r][v], f);
            }
          }
          emax[r] = en;
        }
        if (mine) {
          const int eoff = (int)emax[r] - 127;
          const float2 a0 = split48(wv.x, eoff), a1 = split48(wv.y, eoff);
          const float2 *base = sv + (size_t)slot * VB * kPairStageLen;
#pragma unroll
          for (int v = 0; v < VB; ++v)
            if (v < nv) {
              const float4 x = reinterpret_cast<const float4 *>(base + (size_t)v * kPairStageLen)[e0 / 2];
              dot2_step(s[r][v], c[r][v], x.x, x.y, a0.x, a0.y);
              dot2_step(s[r][v], c[r][v], x.z, x.w, a1.x, a1.y);
            }
        }
      }
      __syncwarp();
      if (ln == 0) mbar_arrive(&empty[slot]);
      // stall == 2 (failure-detection tests only): the first consumer warp of
      // CTA 0 gives up after its first stage, possibly after the producer has
      // issued every copy; the other warps then skip their waits
      if (stall == 2 && blockIdx.x == 0 && wp == 0 && q == 0 && ln == 0) {
        atomicOr(err, 1);
        *(volatile int *)&abort_flag = 1;
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double scale = pow2_of_exponent(emax[r]);
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        float svv = s[r][v], cvv = c[r][v];
        if (v < nv) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(kFull, svv, o), c2 = __shfl_down_sync(kFull, cvv, o);
            ds_add(svv, cvv, s2, c2);
          }
        }
        if (ln == 0) red[wp][r][v] = ((double)svv + (double)cvv) * scale;
      }
    }
    asm volatile("bar.sync 1, %0;\n" ::"n"(kPairConsumers * kWarp) : "memory");
    if (threadIdx.x < NR * VB && threadIdx.x % VB < nv) {
      const int r = threadIdx.x / VB, v = threadIdx.x % VB;
      double sum = 0.0;
      for (int i = 0; i < kPairConsumers; ++i) sum += red[i][r][v];
      partial[((long long)r * m + vb + v) * G + g] = sum;
    }
    asm volatile("bar.sync 1, %0;\n" ::"n"(kPairConsumers * kWarp) : "memory");
  }
}

}  // namespace pintmg
