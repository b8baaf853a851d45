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
// y = z (last layer) or leaky(z).  One thread per output element, FP32
// accumulation; x, W, y in storage type T (float or bf16), z in FP32 when kept.
template <typename T>
__global__ void k_conv_fwd(const T *__restrict__ x, const T *__restrict__ W, const T *__restrict__ bias, T *y,
                           float *z, int B, int C, int O, int H, int Wd, int act) {
  const long long total = (long long)B * O * H * Wd;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(idx % Wd);
    const int t = (int)((idx / Wd) % H);
    const int o = (int)((idx / ((long long)Wd * H)) % O);
    const int b = (int)(idx / ((long long)Wd * H * O));
    float acc = to_f(bias[o]);
    for (int c = 0; c < C; ++c) {
      const T *xc = x + ((long long)b * C + c) * H * Wd;
      const T *wc = W + ((long long)o * C + c) * kNetKT * kNetKX;
#pragma unroll
      for (int i = 0; i < kNetKT; ++i) {
        const int tt = t + i - kNetKT / 2;
        if (tt < 0 || tt >= H) continue;
#pragma unroll
        for (int j = 0; j < kNetKX; ++j) {
          const int ss = s + j - kNetKX / 2;
          if (ss < 0 || ss >= Wd) continue;
          acc = fmaf(to_f(wc[i * kNetKX + j]), to_f(xc[(long long)tt * Wd + ss]), acc);
        }
      }
    }
    if (z) z[idx] = acc;
    y[idx] = from_f<T>(act ? (acc > 0.f ? acc : kNetSlope * acc) : acc);
  }
}

// g *= leaky'(z) elementwise (gradient through the activation)
__global__ void k_leaky_bwd(float *g, const float *__restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(z[i] > 0.f)) g[i] *= kNetSlope;
}

// gx[b,c,t,s] = sum_{o,i,j} W[o,c,i,j] gz[b,o,t-i+1,s-j+3]
__global__ void k_conv_bwd_data(const float *__restrict__ gz, const float *__restrict__ W, float *gx, int B, int C,
                                int O, int H, int Wd) {
  const long long total = (long long)B * C * H * Wd;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(idx % Wd);
    const int t = (int)((idx / Wd) % H);
    const int c = (int)((idx / ((long long)Wd * H)) % C);
    const int b = (int)(idx / ((long long)Wd * H * C));
    float acc = 0.f;
    for (int o = 0; o < O; ++o) {
      const float *go = gz + ((long long)b * O + o) * H * Wd;
      const float *wc = W + ((long long)o * C + c) * kNetKT * kNetKX;
#pragma unroll
      for (int i = 0; i < kNetKT; ++i) {
        const int tt = t - i + kNetKT / 2;
        if (tt < 0 || tt >= H) continue;
#pragma unroll
        for (int j = 0; j < kNetKX; ++j) {
          const int ss = s - j + kNetKX / 2;
          if (ss < 0 || ss >= Wd) continue;
          acc = fmaf(wc[i * kNetKX + j], go[(long long)tt * Wd + ss], acc);
        }
      }
    }
    gx[idx] = acc;
  }
}

// gW[o,c,i,j] = sum_{b,t,s} gz[b,o,t,s] x[b,c,t+i-1,s+j-3] and gb[o] = sum gz[b,o,.,.]:
// one CTA per (o, c) with the 21 taps (and the bias for c == 0) reduced in a
// fixed order (deterministic).
__global__ void __launch_bounds__(256) k_conv_bwd_weights(const float *__restrict__ gz, const float *__restrict__ x,
                                                          float *gW, float *gb, int B, int C, int O, int H, int Wd) {
  const int o = blockIdx.x / C, c = blockIdx.x % C;
  constexpr int K = kNetKT * kNetKX;
  float acc[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) acc[k] = 0.f;
  const long long pos = (long long)B * H * Wd;
  for (long long p = threadIdx.x; p < pos; p += blockDim.x) {
    const int s = (int)(p % Wd);
    const int t = (int)((p / Wd) % H);
    const int b = (int)(p / ((long long)Wd * H));
    const float g = gz[(((long long)b * O + o) * H + t) * Wd + s];
    const float *xc = x + ((long long)b * C + c) * H * Wd;
#pragma unroll
    for (int i = 0; i < kNetKT; ++i) {
      const int tt = t + i - kNetKT / 2;
#pragma unroll
      for (int j = 0; j < kNetKX; ++j) {
        const int ss = s + j - kNetKX / 2;
        const float xv = (tt >= 0 && tt < H && ss >= 0 && ss < Wd) ? xc[(long long)tt * Wd + ss] : 0.f;
        acc[i * kNetKX + j] = fmaf(g, xv, acc[i * kNetKX + j]);
      }
    }
    acc[K] += g;
  }
  __shared__ float red[K + 1][8];
  const int w = threadIdx.x / kWarp, ln = threadIdx.x & (kWarp - 1);
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    float v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
    if (ln == 0) red[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x <= K) {
    float sum = 0.f;
    for (int i = 0; i < (int)(blockDim.x / kWarp); ++i) sum += red[threadIdx.x][i];
    if (threadIdx.x < K)
      gW[((long long)o * C + c) * K + threadIdx.x] = sum;
    else if (c == 0)
      gb[o] = sum;
  }
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
