// The coarse network's BF16 convolutions on the fifth-generation tensor cores:
// tcgen05.mma with the accumulators in tensor memory (TMEM), the weights
// staged by a bulk asynchronous copy (cp.async.bulk), completion tracked by
// mbarriers whose every wait is bounded.
//
// A layer y[o][t][s] = bias[o] + sum_{c,i,j} W[o][c][i][j] x[c][t+i-1][s+j-3]
// is an implicit GEMM: D[m][o] = sum_k A[m][k] B[o][k] with m a position and
// k = (tap (i, j), input channel).  A CTA owns kTcRows time rows of kTcM = 128
// consecutive positions (space s0 .. s0 + 127) of one sample and computes, per
// row, 21 taps x CB channel blocks of one MMA each: M = 128, N = the output
// channels padded to 16 or 32, K = 16 channels (kind::f16, BF16 operands, FP32
// accumulation), the row's accumulator a TMEM block of 128 lanes x N columns.
//
// Shared-memory operands in the canonical K-major layout without swizzle: a
// "core matrix" is 8 rows of 16 bytes (8 BF16 values of K) stored
// contiguously; the descriptor gives the byte stride between core matrices
// along K (leading byte offset) and along M or N (stride byte offset).
//  * Input: plane (cb, half) holds input channels cb*16 + half*8 .. +7 of
//    every staged position, 16 bytes per position, positions of a staged row
//    consecutive, kTcRows + 2 rows.  The A operand of tap (i, j) is the 128
//    staged positions of row (row + i) starting at column j + 1 (the staged
//    columns begin 4 left of s0): core matrices 128 bytes apart along M, one
//    plane apart along K.  A tap is a shift of the start address, so no
//    im2col copy is made.  The layers' activations are stored with the
//    channels innermost ([B][T][X][Cp], Cp = 16 for the network's input with
//    channels 5..15 zero, 32 between layers), so a plane is one box of a
//    tiled TMA copy (cp.async.bulk.tensor, 8 channels x 136 positions x 6
//    rows, zero-filled outside the layer); the last layer writes [B][O][T][X].
//  * Weights: tile (tap, cb) holds [half][n] rows of 16 bytes, N rows per half:
//    core matrices 128 bytes apart along N, 16 N bytes apart along K.  The
//    whole layer's tiles are an image (k_conv_tc_image, once per parameter
//    change) that one thread copies with cp.async.bulk.
//
// Instruction descriptor (kind::f16): bits 4-5 D format (1 = FP32), 7-9 A
// format and 10-12 B format (1 = BF16), 15 and 16 transpose A and B (0 =
// K-major), 17-22 N / 8, 24-28 M / 16.  Shared-memory descriptor: bits 0-13
// start address / 16, 16-29 leading byte offset / 16, 32-45 stride byte
// offset / 16, 46-47 descriptor version (1), 61-63 layout (0 = no swizzle).
#pragma once
#include <cuda.h>

#include "common.cuh"
#include "learned_kernels.cuh"
#include "pair_kernels.cuh"

namespace pintmg {

constexpr int kTcM = 128;                        // positions per MMA tile (one time row)
constexpr int kTcRows = 4;                       // time rows per CTA
constexpr int kTcThreads = 256;                  // 8 warps: staging; warps w and w + 4 share TMEM lanes
constexpr int kTcSR = kTcRows + kNetKT - 1;      // staged input rows
constexpr int kTcSP = kTcM + 8;                  // staged positions per row: s0 - 4 .. s0 + 131
constexpr int kTcChunk = 4096;                   // bytes per bulk copy of the weight image

__host__ __device__ constexpr int tc_n(int O) { return O <= 16 ? 16 : 32; }
__host__ __device__ constexpr int tc_plane() { return kTcSR * kTcSP * 16; }
__host__ __device__ constexpr int tc_a_bytes(int CB) { return CB * 2 * tc_plane(); }
__host__ __device__ constexpr int tc_tile_bytes(int N) { return 2 * N * 16; }
__host__ __device__ constexpr int tc_img_bytes(int CB, int N) { return kNetKT * kNetKX * CB * tc_tile_bytes(N); }
__host__ __device__ constexpr int tc_smem(int CB, int N) { return tc_a_bytes(CB) + tc_img_bytes(CB, N) + 32; }
// (CB, N) of layer l and the offset of its image in a buffer of all four (BF16 values)
__host__ __device__ constexpr int tc_cb(int l) { return net_ch(l) <= 16 ? 1 : 2; }
__host__ __device__ constexpr int tc_nl(int l) { return tc_n(net_ch(l + 1)); }
__host__ __device__ constexpr long long tc_img_offset(int l) {
  return l == 0 ? 0 : tc_img_offset(l - 1) + tc_img_bytes(tc_cb(l - 1), tc_nl(l - 1)) / 2;
}
constexpr long long kTcImgValues = tc_img_offset(kNetLayers);

__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long tc_sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// The layer's weights as k_conv_tc's tiles: img[((tap * CB + cb) * 2 + half) * N + n][u] =
// W[n][cb * 16 + half * 8 + u][tap] (zero beyond C input or O output channels).
template <int CB, int N>
__global__ void k_conv_tc_image(const __nv_bfloat16 *__restrict__ W, int C, int O, __nv_bfloat16 *img) {
  constexpr int K = kNetKT * kNetKX;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * CB * 2 * N * 8; e += gridDim.x * blockDim.x) {
    const int u = e % 8, n = (e / 8) % N, half = (e / (8 * N)) % 2, cb = (e / (16 * N)) % CB, tap = e / (16 * N * CB);
    const int c = cb * 16 + half * 8 + u;
    img[e] = (n < O && c < C) ? W[((long long)n * C + c) * K + tap] : __float2bfloat16(0.f);
  }
}

// One layer: the input, [B][H][Wd][16 CB] BF16 behind the tensor map xmap
// (dims channels, Wd, H, B; box 8 x kTcSP x kTcSR x 1), to y: [B][H][Wd][N]
// with the channels innermost (kCiOut) or [B][O][H][Wd]; BF16, bias and the
// leaky rectifier (act) in the epilogue.  Grid (ceil(Wd / 128), ceil(H / 4),
// B), kTcThreads threads, tc_smem(CB, N) bytes of dynamic shared memory.  A
// wait that runs out (2 s) sets err[0]; the CTA then waits once more (bounded)
// for its copies and MMAs, skips its output and frees its TMEM.
template <int CB, int N, bool kCiOut>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(const __grid_constant__ CUtensorMap xmap,
                                                        const __nv_bfloat16 *__restrict__ img,
                                                        const __nv_bfloat16 *__restrict__ bias, __nv_bfloat16 *y,
                                                        int O, int H, int Wd, int act, int *err) {
  constexpr int PLANE = tc_plane(), A_BYTES = tc_a_bytes(CB), IMG = tc_img_bytes(CB, N), TILE = tc_tile_bytes(N);
  constexpr int COLS = kTcRows * N;  // TMEM columns: a power of two >= 32 (64 or 128)
  static_assert(COLS == 64 || COLS == 128, "TMEM allocation must be a power of two of at least 32 columns");
  static_assert(IMG % 16 == 0 && PLANE % 16 == 0, "bulk copies and core matrices need 16-byte units");
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  unsigned char *sa = tc_smem_raw, *sb = tc_smem_raw + A_BYTES;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(sb + IMG);  // [0] weights, [1] MMAs
  unsigned *tslot = reinterpret_cast<unsigned *>(bar + 2);
  const int b = blockIdx.z, t0 = blockIdx.y * kTcRows, s0 = blockIdx.x * kTcM;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {  // TMEM for the CTA's kTcRows accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;
  if (threadIdx.x == 0) {  // the weight image (chunks of kTcChunk bytes) and the input planes, one barrier
    mbar_expect_tx(bar, IMG + CB * 2 * PLANE);
    for (int off = 0; off < IMG; off += kTcChunk) {
      const unsigned n = (unsigned)min(kTcChunk, IMG - off);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
              smem_addr(sb + off)),
          "l"(reinterpret_cast<const unsigned char *>(img) + off), "r"(n), "r"(smem_addr(bar))
          : "memory");
    }
    // plane pl: channels 8 pl .. 8 pl + 7 of rows t0 - 1 .. t0 + kTcRows, positions s0 - 4 .. s0 + 131
    // (the innermost coordinate, 8 pl channels, is a multiple of 16 bytes)
    for (int pl = 0; pl < CB * 2; ++pl)
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
          "%5}], [%6];\n" ::"r"(smem_addr(sa + pl * PLANE)),
          "l"(reinterpret_cast<unsigned long long>(&xmap)), "r"(8 * pl), "r"(s0 - 4), "r"(t0 - kNetKT / 2), "r"(b),
          "r"(smem_addr(bar))
          : "memory");
  }
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    ok = mbar_wait(bar, 0) ? 1 : 0;
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      constexpr unsigned ID = tc_idesc(kTcM, N);
      for (int row = 0; row < kTcRows; ++row) {
        int k = 0;
        for (int tap = 0; tap < kNetKT * kNetKX; ++tap) {
          const int i = tap / kNetKX, j = tap % kNetKX;
#pragma unroll
          for (int cb = 0; cb < CB; ++cb, ++k) {
            const unsigned a = smem_addr(sa + cb * 2 * PLANE + ((row + i) * kTcSP + j + 1) * 16);
            const unsigned bb = smem_addr(sb + (tap * CB + cb) * TILE);
            const unsigned long long ad = tc_sdesc(a, PLANE, 128), bd = tc_sdesc(bb, N * 16, 128);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + row * N),
                "l"(ad), "l"(bd), "r"(ID), "r"(k)
                : "memory");
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(bar + 1))
                   : "memory");
    } else {
      atomicExch(err, 1);
      mbar_wait(bar, 0);  // let the copies land before the CTA's shared memory is released (bounded)
    }
  }
  ok = __syncthreads_and(ok);
  if (ok) {
    const bool done = __all_sync(0xffffffffu, mbar_wait(bar + 1, 0));
    if (!done) {
      if (lane == 0) atomicExch(err, 1);
      if (threadIdx.x == 0) mbar_wait(bar + 1, 0);  // once more (bounded) before the TMEM is freed
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int q = warp & 3;  // the TMEM lanes (positions) 32 q .. 32 q + 31 this warp may read
      const int sp = s0 + q * 32 + lane;
      for (int row = warp >> 2; row < kTcRows; row += kTcThreads / 128) {
        unsigned v[N];
        const unsigned addr = tmem + ((unsigned)(q * 32) << 16) + row * N;
        if constexpr (N == 32) {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
              "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                "=r"(v[30]), "=r"(v[31])
              : "r"(addr));
        } else {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(addr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        const int t = t0 + row;
        if (t < H && sp < Wd) {
          if constexpr (kCiOut) {  // the position's N channels, 16 bytes at a time
            uint4 *dst = reinterpret_cast<uint4 *>(y + (((long long)b * H + t) * Wd + sp) * N);
#pragma unroll
            for (int q8 = 0; q8 < N / 8; ++q8) {
              __align__(16) __nv_bfloat16 out[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int o = q8 * 8 + u;
                float val = __uint_as_float(v[o]) + (bias && o < O ? __bfloat162float(bias[o]) : 0.f);
                if (act) val = val > 0.f ? val : kNetSlope * val;
                out[u] = __float2bfloat16(o < O ? val : 0.f);
              }
              dst[q8] = *reinterpret_cast<const uint4 *>(out);
            }
          } else {
#pragma unroll
            for (int o = 0; o < N; ++o) {
              if (o >= O) break;
              float val = __uint_as_float(v[o]) + (bias ? __bfloat162float(bias[o]) : 0.f);
              if (act) val = val > 0.f ? val : kNetSlope * val;
              y[(((long long)b * O + o) * H + t) * Wd + sp] = __float2bfloat16(val);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(COLS) : "memory");
}

// network input with the channels innermost and padded: x [B][5][H][Wd] FP32 ->
// xc [B][H][Wd][16] BF16 (channels 5..15 zero)
__global__ void k_f32_to_bf16_ci(const float *__restrict__ x, __nv_bfloat16 *xc, int B, long long HW) {
  const long long n = (long long)B * HW;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / HW, pos = i % HW;
    __align__(16) __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = c < 5 ? __float2bfloat16(x[(b * 5 + c) * HW + pos]) : __float2bfloat16(0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(xc + i * 16);
    dst[0] = reinterpret_cast<const uint4 *>(v)[0];
    dst[1] = reinterpret_cast<const uint4 *>(v)[1];
  }
}

// the coarse residual scaled by 1 / rms(r) (scal[1] = 1 / ||r||; n = 5 H Wd entries in the
// type-major layout, a (5, H, Wd) tensor) as the network's input with the channels innermost
__global__ void k_net_input_ci(const double *__restrict__ r, const double *__restrict__ scal, __nv_bfloat16 *xc,
                               long long HW) {
  const double inv = scal[1] * sqrt(5.0 * (double)HW);
  for (long long pos = blockIdx.x * (long long)blockDim.x + threadIdx.x; pos < HW;
       pos += (long long)gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = c < 5 ? __float2bfloat16((float)(r[c * HW + pos] * inv)) : __float2bfloat16(0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(xc + pos * 16);
    dst[0] = reinterpret_cast<const uint4 *>(v)[0];
    dst[1] = reinterpret_cast<const uint4 *>(v)[1];
  }
}

}  // namespace pintmg
