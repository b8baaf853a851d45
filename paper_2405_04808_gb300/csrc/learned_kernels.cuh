// Learned coarse-grid correction: a small convolutional network over
// (time, space) that proposes the coarse solve from the coarse residual.
// Forward, backward and optimiser kernels (FP32 training, BF16-storage
// inference with FP32 accumulation).  Tensors are NCHW with H = time steps,
// W = space nodes; a coarse type-major vector (u, v, z, lambda, mu, each
// n x p) is exactly a (5, n, p) tensor.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace pintmg {

constexpr int kNetLayers = 4;
constexpr int kNetKT = 3, kNetKX = 7;
constexpr float kNetSlope = 0.1f;

// channels between layers: 5 -> 32 -> 32 -> 32 -> 5
__host__ __device__ constexpr int net_ch(int l) { return (l == 0 || l == kNetLayers) ? 5 : 32; }

__host__ __device__ constexpr long long net_layer_params(int l) {
  return (long long)net_ch(l + 1) * net_ch(l) * kNetKT * kNetKX + net_ch(l + 1);
}
__host__ __device__ constexpr long long net_layer_offset(int l) {
  return l == 0 ? 0 : net_layer_offset(l - 1) + net_layer_params(l - 1);
}
constexpr long long kNetParams = net_layer_offset(kNetLayers);

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T from_f(float v) { return (T)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16(v); }

// z[b,o,t,s] = bias[o] + sum_{c,i,j} W[o,c,i,j] x[b,c,t+i-1,s+j-3] (zero outside);
// y = z (last layer) or leaky(z); z kept in FP32 when requested (training).
// Tiled direct convolution with FP32 accumulation: a CTA computes a
// 16 (time) x 64 (space) tile of positions for OB output channels; each thread
// 2 x 2 positions (rows 2ty, 2ty+1; columns tx, tx+32) x OB channels in FP32
// registers.  Input channels are staged in chunks of kConvCC into shared
// memory with their halo (zero outside the grid), converted to FP32, and the
// chunk's weights as [c][tap][o] so that one 16-byte broadcast load feeds
// four channels.  W is [O][C][3][7] in storage type T; bias may be NULL.
// Grid: (ceil(Wd / 64), ceil(H / 16), B * ceil(O / OB)), 256 threads.
constexpr int kConvTT = 16, kConvTX = 64, kConvCC = 4;

template <typename T, int OB>
__global__ void __launch_bounds__(256) k_conv_tiled(const T *__restrict__ x, const T *__restrict__ W,
                                                    const T *__restrict__ bias, T *y, float *z, int B, int C, int O,
                                                    int H, int Wd, int act) {
  constexpr int K = kNetKT * kNetKX;
  constexpr int RH = kConvTT + kNetKT - 1, RW = kConvTX + kNetKX - 1;
  __shared__ float sx[kConvCC][RH][RW];
  __shared__ __align__(16) float sw[kConvCC][K][OB];
  const int nob = (O + OB - 1) / OB;
  const int b = blockIdx.z / nob, ob = (blockIdx.z % nob) * OB;
  const int t0 = blockIdx.y * kConvTT, s0 = blockIdx.x * kConvTX;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[2][2][OB];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int o = 0; o < OB; ++o) acc[r][q][o] = 0.f;
  for (int c0 = 0; c0 < C; c0 += kConvCC) {
    // stage the input chunk with its halo, and the chunk's weights
    for (int e = threadIdx.x; e < kConvCC * RH * RW; e += blockDim.x) {
      const int cc = e / (RH * RW), rr = (e / RW) % RH, col = e % RW;
      const int c = c0 + cc, t = t0 + rr - kNetKT / 2, sp = s0 + col - kNetKX / 2;
      float v = 0.f;
      if (c < C && t >= 0 && t < H && sp >= 0 && sp < Wd) v = to_f(x[(((long long)b * C + c) * H + t) * Wd + sp]);
      sx[cc][rr][col] = v;
    }
    for (int e = threadIdx.x; e < kConvCC * K * OB; e += blockDim.x) {
      const int cc = e / (K * OB), k = (e / OB) % K, o = e % OB;
      const int c = c0 + cc;
      sw[cc][k][o] = (c < C && ob + o < O) ? to_f(W[((long long)(ob + o) * C + c) * K + k]) : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int cc = 0; cc < kConvCC; ++cc) {
#pragma unroll
      for (int i = 0; i < kNetKT; ++i) {
#pragma unroll
        for (int j = 0; j < kNetKX; ++j) {
          const float x00 = sx[cc][2 * ty + i][tx + j], x01 = sx[cc][2 * ty + i][tx + 32 + j];
          const float x10 = sx[cc][2 * ty + 1 + i][tx + j], x11 = sx[cc][2 * ty + 1 + i][tx + 32 + j];
          const float4 *wv = reinterpret_cast<const float4 *>(&sw[cc][i * kNetKX + j][0]);
#pragma unroll
          for (int o4 = 0; o4 < OB / 4; ++o4) {
            const float4 w4 = wv[o4];
            const float wo[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              acc[0][0][4 * o4 + u] = fmaf(wo[u], x00, acc[0][0][4 * o4 + u]);
              acc[0][1][4 * o4 + u] = fmaf(wo[u], x01, acc[0][1][4 * o4 + u]);
              acc[1][0][4 * o4 + u] = fmaf(wo[u], x10, acc[1][0][4 * o4 + u]);
              acc[1][1][4 * o4 + u] = fmaf(wo[u], x11, acc[1][1][4 * o4 + u]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int t = t0 + 2 * ty + r;
    if (t >= H) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int sp = s0 + tx + 32 * q;
      if (sp >= Wd) continue;
#pragma unroll
      for (int o = 0; o < OB; ++o) {
        if (ob + o >= O) continue;
        const float v = acc[r][q][o] + (bias ? to_f(bias[ob + o]) : 0.f);
        const long long idx = (((long long)b * O + ob + o) * H + t) * Wd + sp;
        if (z) z[idx] = v;
        y[idx] = from_f<T>(act ? (v > 0.f ? v : kNetSlope * v) : v);
      }
    }
  }
}

// BF16 inference on the tensor cores: the same convolution as an implicit
// GEMM, out[position][o] = sum_k A[position][k] B[k][o] with k = (tap, input
// channel), by mma.sync m16n8k16 (BF16 operands, FP32 accumulation).  A CTA
// of 4 warps owns 4 rows x 64 columns of positions; warp w computes row w as
// 4 m-tiles of 16 columns x NT n-tiles of 8 output channels.  The input tile
// with its halo is staged channel-innermost (channels padded to CB*16, rows of
// CB*16+8 values so that the 8 row addresses of an ldmatrix fall in distinct
// banks), the weights as [tap][channel block][o][k] rows of 24 values.  For a
// tap (i, j) the A fragment of positions s..s+15 is the staged rows at column
// s + j of input row w + i, so no im2col copy is made.  The weights come as the
// layer's image (k_conv_mma_image, 16-byte aligned).  Dynamic shared memory:
// conv_mma_smem(CB, NT) bytes.  Grid: (ceil(Wd / 64), ceil(H / 4), B), 128 threads.
constexpr int kMmaRows = 4, kMmaCols = 64;

__host__ __device__ constexpr int conv_mma_cs(int CB) { return CB * 16 + 8; }
__host__ __device__ constexpr int conv_mma_smem(int CB, int NT) {
  return (kMmaRows + kNetKT - 1) * (kMmaCols + kNetKX - 1) * conv_mma_cs(CB) * 2 +
         kNetKT * kNetKX * CB * NT * 8 * 24 * 2;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// The weights of one layer in k_conv_mma's shared-memory order, [tap][channel
// block][o][k] with rows of 24 values (zero padding), written once per
// parameter change so that the kernel stages them with 16-byte copies.
__host__ __device__ constexpr int conv_mma_wimg(int CB, int NT) { return kNetKT * kNetKX * CB * NT * 8 * 24; }
// (CB, NT) of layer l: input channels in blocks of 16, output channels in tiles of 8
__host__ __device__ constexpr int conv_mma_cb(int l) { return net_ch(l) <= 16 ? 1 : 2; }
__host__ __device__ constexpr int conv_mma_nt(int l) { return net_ch(l + 1) <= 8 ? 1 : 4; }
__host__ __device__ constexpr long long conv_mma_wimg_offset(int l) {
  return l == 0 ? 0 : conv_mma_wimg_offset(l - 1) + conv_mma_wimg(conv_mma_cb(l - 1), conv_mma_nt(l - 1));
}
constexpr long long kConvMmaWimg = conv_mma_wimg_offset(kNetLayers);

template <int CB, int NT>
__global__ void k_conv_mma_image(const __nv_bfloat16 *__restrict__ W, int C, int O, __nv_bfloat16 *img) {
  constexpr int K = kNetKT * kNetKX, NO = NT * 8, KS = 24;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * CB * NO * KS; e += gridDim.x * blockDim.x) {
    const int k = e % KS, n = (e / KS) % NO, cb = (e / (KS * NO)) % CB, tap = e / (KS * NO * CB);
    const int c = cb * 16 + k;
    img[e] = (k < 16 && n < O && c < C) ? W[((long long)n * C + c) * K + tap] : __float2bfloat16(0.f);
  }
}

template <int CB, int NT>
__global__ void __launch_bounds__(128) k_conv_mma(const __nv_bfloat16 *__restrict__ x,
                                                  const __nv_bfloat16 *__restrict__ wimg,
                                                  const __nv_bfloat16 *__restrict__ bias, __nv_bfloat16 *y, int B,
                                                  int C, int O, int H, int Wd, int act) {
  constexpr int K = kNetKT * kNetKX;
  constexpr int HR = kMmaRows + kNetKT - 1, HC = kMmaCols + kNetKX - 1;
  constexpr int CS = conv_mma_cs(CB), KS = 24, NO = NT * 8;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  __nv_bfloat16 *sx = reinterpret_cast<__nv_bfloat16 *>(conv_smem);
  __nv_bfloat16 *sw = sx + HR * HC * CS;
  const int b = blockIdx.z, t0 = blockIdx.y * kMmaRows, s0 = blockIdx.x * kMmaCols;
  // input tile: a thread per (position, 8 channels): 8 loads coalesced along
  // the columns, one 16-byte store into the channel-innermost row
  for (int e = threadIdx.x; e < CB * 2 * HR * HC; e += blockDim.x) {
    const int col = e % HC, r = (e / HC) % HR, grp = e / (HC * HR);
    const int t = t0 + r - kNetKT / 2, sp = s0 + col - kNetKX / 2;
    __align__(16) __nv_bfloat16 v[8];
    const bool in = t >= 0 && t < H && sp >= 0 && sp < Wd;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = grp * 8 + u;
      v[u] = (in && c < C) ? x[(((long long)b * C + c) * H + t) * Wd + sp] : __float2bfloat16(0.f);
    }
    *reinterpret_cast<uint4 *>(sx + (r * HC + col) * CS + grp * 8) = *reinterpret_cast<const uint4 *>(v);
  }
  // weights: a straight copy of the layer's image
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(wimg);
    uint4 *dst = reinterpret_cast<uint4 *>(sw);
    for (int e = threadIdx.x; e < K * CB * NO * KS / 8; e += blockDim.x) dst[e] = src[e];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int mi = lane >> 3, rr = lane & 7;
  const int arow = rr + ((mi & 1) ? 8 : 0), akoff = (mi >> 1) ? 8 : 0;
  float acc[4][NT][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[mt][nt][u] = 0.f;
#pragma unroll 1
  for (int tap = 0; tap < K; ++tap) {
    const int i = tap / kNetKX, j = tap % kNetKX;
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      unsigned bf[NT][2];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const __nv_bfloat16 *wp = sw + ((tap * CB + cb) * NO + nt * 8 + g) * KS + 2 * q;
        bf[nt][0] = *reinterpret_cast<const unsigned *>(wp);
        bf[nt][1] = *reinterpret_cast<const unsigned *>(wp + 8);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const __nv_bfloat16 *ap = sx + ((warp + i) * HC + mt * 16 + arow + j) * CS + cb * 16 + akoff;
        unsigned a0, a1, a2, a3;
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                     : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                     : "r"(smem_u32(ap)));
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
              "{%0, %1, %2, %3};\n"
              : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
              : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(bf[nt][0]), "r"(bf[nt][1]));
        }
      }
    }
  }
  const int t = t0 + warp;
  if (t >= H) return;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int sp = s0 + mt * 16 + g + ((u & 2) ? 8 : 0);
        const int o = nt * 8 + 2 * q + (u & 1);
        if (o >= O || sp >= Wd) continue;
        float v = acc[mt][nt][u] + (bias ? __bfloat162float(bias[o]) : 0.f);
        if (act) v = v > 0.f ? v : kNetSlope * v;
        y[(((long long)b * O + o) * H + t) * Wd + sp] = __float2bfloat16(v);
      }
}

// Wt[c][o][i][j] = W[o][c][KT-1-i][KX-1-j]: the gradient with respect to a
// layer's input is the convolution of the output gradient with these weights
__global__ void k_flip_transpose(const float *__restrict__ W, float *Wt, int C, int O) {
  constexpr int K = kNetKT * kNetKX;
  const long long n = (long long)O * C * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % K), c = (int)((e / K) % C), o = (int)(e / ((long long)K * C));
    const int i = k / kNetKX, j = k % kNetKX;
    Wt[((long long)c * O + o) * K + (kNetKT - 1 - i) * kNetKX + (kNetKX - 1 - j)] = W[e];
  }
}

// g *= leaky'(z) elementwise (gradient through the activation)
__global__ void k_leaky_bwd(float *g, const float *__restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(z[i] > 0.f)) g[i] *= kNetSlope;
}

// Weight gradient gW[o,c,i,j] = sum_{b,t,s} gz[b,o,t,s] x[b,c,t+i-1,s+j-3].
// CTA (o-block of 16, c-block of 4, slice p of P): walks the position tiles
// p, p + P, ... (4 rows x 64 columns of one sample, in a fixed order), staging
// the tile's output gradient and the input with its halo in shared memory.
// Thread (o, c, i) keeps the 7 sums of j; per run of 8 positions it reads 8
// gradients and 14 inputs for 56 fused multiply-adds.  Writes
// partial[p][o][c][i][j]; k_wgrad_reduce sums the P slices in order.
// Grid: (ceil(O / 16) * ceil(C / 4), P), 192 threads.
constexpr int kWgRows = 4, kWgCols = 64, kWgOB = 16, kWgCB = 4;

__global__ void __launch_bounds__(192) k_conv_wgrad(const float *__restrict__ gz, const float *__restrict__ x,
                                                    float *partial, int B, int C, int O, int H, int Wd) {
  constexpr int K = kNetKT * kNetKX;
  // output-gradient tile, one padded block per channel: consecutive channels
  // start 4 banks apart, so the 16-byte reads of 8 lanes hit 32 distinct banks
  constexpr int GO = kWgRows * kWgCols + 4;
  constexpr int XR = kWgRows + kNetKT - 1, XC = kWgCols + kNetKX - 1 + 1;
  __shared__ __align__(16) float sg[kWgOB * GO];
  __shared__ float sx[kWgCB][XR][XC];
  const int ncb = (C + kWgCB - 1) / kWgCB;
  const int ob = (blockIdx.x / ncb) * kWgOB, cb = (blockIdx.x % ncb) * kWgCB;
  const int P = gridDim.y, p = blockIdx.y;
  const int ol = threadIdx.x % kWgOB, cl = (threadIdx.x / kWgOB) % kWgCB, i = threadIdx.x / (kWgOB * kWgCB);
  const int tilesT = (H + kWgRows - 1) / kWgRows, tilesX = (Wd + kWgCols - 1) / kWgCols;
  const long long tiles = (long long)B * tilesT * tilesX;
  float acc[kNetKX];
#pragma unroll
  for (int j = 0; j < kNetKX; ++j) acc[j] = 0.f;
  for (long long tile = p; tile < tiles; tile += P) {
    const int b = (int)(tile / ((long long)tilesT * tilesX));
    const int t0 = (int)((tile / tilesX) % tilesT) * kWgRows, s0 = (int)(tile % tilesX) * kWgCols;
    for (int e = threadIdx.x; e < kWgOB * kWgRows * kWgCols; e += blockDim.x) {
      const int o = e / (kWgRows * kWgCols), r = (e / kWgCols) % kWgRows, col = e % kWgCols;
      const int t = t0 + r, sp = s0 + col;
      float v = 0.f;
      if (ob + o < O && t < H && sp < Wd) v = gz[(((long long)b * O + ob + o) * H + t) * Wd + sp];
      sg[o * GO + r * kWgCols + col] = v;
    }
    for (int e = threadIdx.x; e < kWgCB * XR * XC; e += blockDim.x) {
      const int c = e / (XR * XC), r = (e / XC) % XR, col = e % XC;
      const int t = t0 + r - kNetKT / 2, sp = s0 + col - kNetKX / 2;
      float v = 0.f;
      if (cb + c < C && t >= 0 && t < H && sp >= 0 && sp < Wd) v = x[(((long long)b * C + cb + c) * H + t) * Wd + sp];
      sx[c][r][col] = v;
    }
    __syncthreads();
    if (i < kNetKT) {
#pragma unroll 1
      for (int r = 0; r < kWgRows; ++r) {
#pragma unroll 1
        for (int s = 0; s < kWgCols; s += 8) {
          const float4 g0 = *reinterpret_cast<const float4 *>(&sg[ol * GO + r * kWgCols + s]);
          const float4 g1 = *reinterpret_cast<const float4 *>(&sg[ol * GO + r * kWgCols + s + 4]);
          const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
          float xv[8 + kNetKX - 1];
#pragma unroll
          for (int k = 0; k < 8 + kNetKX - 1; ++k) xv[k] = sx[cl][r + i][s + k];
#pragma unroll
          for (int j = 0; j < kNetKX; ++j)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[j] = fmaf(g[k], xv[k + j], acc[j]);
        }
      }
    }
    __syncthreads();
  }
  if (i < kNetKT && ob + ol < O && cb + cl < C) {
    float *dst = partial + (((long long)p * O + ob + ol) * C + cb + cl) * K + i * kNetKX;
#pragma unroll
    for (int j = 0; j < kNetKX; ++j) dst[j] = acc[j];
  }
}

// gW[e] = sum_{p < P} partial[p][e] in order (e < O * C * 21)
__global__ void k_wgrad_reduce(const float *__restrict__ partial, int P, long long n, float *gW) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < P; ++q) s += partial[(long long)q * n + e];
    gW[e] = s;
  }
}

// bias gradient partials: partial[o * G + g] = sum over chunk g of gz[., o, ., .]
// (grid (O, G), 256 threads, fixed order); k_bias_reduce finishes
__global__ void k_bias_partial(const float *__restrict__ gz, int B, int O, long long TX, float *partial) {
  const int o = blockIdx.x, G = gridDim.y;
  const long long per = (long long)B * TX;
  float acc = 0.f;
  for (long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x; e < per; e += (long long)G * blockDim.x) {
    const long long b = e / TX, t = e % TX;
    acc += gz[(b * O + o) * TX + t];
  }
  __shared__ float red[8];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(kFull, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) s += red[q];
    partial[(long long)o * G + blockIdx.y] = s;
  }
}

__global__ void k_bias_reduce(const float *__restrict__ partial, int G, int O, float *gb) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  float s = 0.f;
  for (int q = 0; q < G; ++q) s += partial[(long long)o * G + q];
  gb[o] = s;
}

// Residual-metric loss: d[i] = scale[c] (y[i] - t[i]) in FP64, c = (i / TX) % C
// the channel of entry i (scale null: 1)
__global__ void k_metric_diff(const float *__restrict__ y, const float *__restrict__ t,
                              const float *__restrict__ scale, long long TX, int C, long long n, double *d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double sc = scale ? (double)scale[(i / TX) % C] : 1.0;
    d[i] = sc * ((double)y[i] - (double)t[i]);
  }
}

// g[i] = scale[c] * mul * a[i] (rounded to FP32), c as in k_metric_diff
__global__ void k_metric_grad(const double *__restrict__ a, const float *__restrict__ scale, long long TX, int C,
                              long long n, double mul, float *g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double sc = scale ? (double)scale[(i / TX) % C] : 1.0;
    g[i] = (float)(sc * mul * a[i]);
  }
}

// loss[0] = sum[0] * inv_n (FP32)
__global__ void k_metric_loss(const double *__restrict__ sum, double inv_n, float *loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) loss[0] = (float)(sum[0] * inv_n);
}

// loss partials of mean((y - t)^2) and g = 2 (y - t) / n
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, float *g, long long n, float *partial) {
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    g[i] = 2.f * d / (float)n;
    acc = fmaf(d, d, acc);
  }
  __shared__ float red[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(kFull, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials(const float *__restrict__ partial, int G, float scale, float *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < G; ++i) s += partial[i];
    out[0] = s * scale;
  }
}

// Adam (Kingma and Ba 2015) with bias correction
__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_f32_to_bf16(const float *__restrict__ x, __nv_bfloat16 *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

__global__ void k_bf16_to_f32(const __nv_bfloat16 *__restrict__ x, float *y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(x[i]);
}

// dst[k] = src[idx[k]] for rows of `row` floats (a shuffled minibatch)
__global__ void k_gather_rows(const float *__restrict__ src, const int *__restrict__ idx, int rows, long long row,
                              float *dst) {
  const long long total = (long long)rows * row;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / row, e = i % row;
    dst[i] = src[(long long)idx[k] * row + e];
  }
}

// dst[k] = src[idx[k]] / scale[channel] (per-channel normalised minibatch; rows of
// C x TX floats, channel = (e / TX) % C)
__global__ void k_gather_rows_scaled(const float *__restrict__ src, const int *__restrict__ idx, int rows,
                                     long long row, long long TX, int C, const float *__restrict__ scale,
                                     float *dst) {
  const long long total = (long long)rows * row;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / row, e = i % row;
    dst[i] = src[(long long)idx[k] * row + e] / scale[(int)((e / TX) % C)];
  }
}

// per-channel sums of squares of `count` samples (C x TX each): partial[c][blockIdx.y]
// in FP64, fixed order; grid (C, G)
__global__ void k_channel_sumsq(const float *__restrict__ x, long long count, long long TX, int C, double *partial) {
  const int c = blockIdx.x, G = gridDim.y;
  double acc = 0.0;
  const long long per = count * TX;
  for (long long i = blockIdx.y * (long long)blockDim.x + threadIdx.x; i < per; i += (long long)G * blockDim.x) {
    const long long k = i / TX, t = i % TX;
    const double v = x[(k * C + c) * TX + t];
    acc += v * v;
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(kFull, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];
    partial[(long long)c * G + blockIdx.y] = s;
  }
}

// scale[c] = sqrt(mean square) of channel c (1 where the channel is zero)
__global__ void k_channel_rms(const double *__restrict__ partial, int G, double n, int C, float *scale) {
  const int c = threadIdx.x;
  if (c >= C) return;
  double s = 0.0;
  for (int i = 0; i < G; ++i) s += partial[(long long)c * G + i];
  const double r = sqrt(s / n);
  scale[c] = r > 0.0 ? (float)r : 1.f;
}

// Move the first layer's input scaling and the last layer's output scaling
// into or out of the parameters: dir = +1 maps the parameters of net(x) to
// those of the normalised net' (x' = x / sx per input channel, y' = y / sy per
// output channel): W0[:, c] *= sx[c], (W3, b3)[o] /= sy[o]; dir = -1 undoes it.
__global__ void k_net_fold(float *params, const float *__restrict__ sx, const float *__restrict__ sy, int dir) {
  constexpr int K = kNetKT * kNetKX;
  const long long n0 = (long long)net_ch(1) * net_ch(0) * K;
  const long long o3 = net_layer_offset(kNetLayers - 1);
  const long long n3 = (long long)net_ch(kNetLayers) * net_ch(kNetLayers - 1) * K;
  const long long nb3 = net_ch(kNetLayers);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0 + n3 + nb3;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < n0) {
      const int c = (int)((i / K) % net_ch(0));
      params[i] = dir > 0 ? params[i] * sx[c] : params[i] / sx[c];
    } else {
      const long long j = i - n0;
      const int o = j < n3 ? (int)(j / ((long long)net_ch(kNetLayers - 1) * K)) : (int)(j - n3);
      params[o3 + j] = dir > 0 ? params[o3 + j] / sy[o] : params[o3 + j] * sy[o];
    }
  }
}

// coarse residual (FP64) -> network input (storage T): x = r / rms(r) with
// rms(r) = ||r|| / sqrt(n) (scal[1] = 1 / ||r||), so that x has unit mean square
template <typename T>
__global__ void k_net_input(const double *__restrict__ r, const double *__restrict__ scal, T *x, long long n) {
  const double inv = scal[1] * sqrt((double)n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = from_f<T>((float)(r[i] * inv));
}

// network output (storage T) -> coarse correction (FP64), scaled back by rms(r) = ||r|| / sqrt(n) (scal[0] = ||r||)
template <typename T>
__global__ void k_net_output(const T *__restrict__ y, const double *__restrict__ scal, double *e, long long n) {
  const double nr = scal[0] / sqrt((double)n);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    e[i] = (double)to_f(y[i]) * nr;
}

}  // namespace pintmg
