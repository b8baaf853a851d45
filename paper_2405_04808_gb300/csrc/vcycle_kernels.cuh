// V-cycle kernels: block solve (Jacobi / SGS passes), residual + restriction,
// prolongation, operator apply and the serial SGS chains.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace pintmg {

// ---------------------------------------------------------------------------
// Local augmented solve D_j y = r of time block j (Thm 1), by the Schur
// complement of the identity block:
//   v = -r_mu;  S lambda = N r_u + Z r_z + V v - r_lambda,  S = N N^T + Z Z^T
//   u = r_u - N^T lambda;  z = r_z - Z^T lambda;  mu = v + V^T lambda - r_v
// (block 0 has no v, mu; block n has only v = -r_mu, mu = v - r_v).

// The coefficients of one time block (tridiagonal layout): bands of N, V, Z,
// the LDL^T factor of S and the chunk-scan compositions, in global or shared memory.
// (bands stored as CT, the factor and scan compositions as T)
template <typename T, typename CT = T>
struct TriBlock {
  const CT *N, *V, *Z;
  const T *fac, *scan;
};

template <typename T, typename CT>
__device__ __forceinline__ TriBlock<T, CT> tri_block(const LevelView<T, CT> &L, int j) {
  return {L.N + j * L.sN, L.V + j * L.sV, L.Z + j * L.sZ, L.fac + j * L.sFac, L.scan + (long long)j * kScanPerBlock};
}

// kappa != 0: V = kappa Z, so Z r_z + V v = Z (r_z + kappa v) and
// Z^T lambda, V^T lambda come from one product (the same values up to rounding).
template <typename T, int C, typename CT>
__device__ __forceinline__ void local_solve_tri(const TriBlock<T, CT> &Bk, int n, int p, int j,
                                                const T (&ru)[C], const T (&rz)[C], const T (&rl)[C],
                                                const T (&rv)[C], const T (&rm)[C],
                                                T (&u)[C], T (&z)[C], T (&l)[C], T (&v)[C], T (&m)[C],
                                                int ln, T kappa = T(0)) {
  if (j == n) {
#pragma unroll
    for (int e = 0; e < C; ++e) {
      v[e] = -rm[e];
      m[e] = v[e] - rv[e];
    }
    return;
  }
  const CT *N = Bk.N, *V = Bk.V, *Z = Bk.Z;
  const T *fac = Bk.fac, *scan = Bk.scan;
  T rhs[C];
  tri_mv<T, C, false>(rhs, N, ru, p, ln, T(1));
  if (j >= 1) {
#pragma unroll
    for (int e = 0; e < C; ++e) v[e] = -rm[e];
  }
  if (kappa != T(0) && j >= 1) {
    T w[C];
#pragma unroll
    for (int e = 0; e < C; ++e) w[e] = fma(kappa, v[e], rz[e]);
    tri_mv<T, C, true>(rhs, Z, w, p, ln, T(1));
#pragma unroll
    for (int e = 0; e < C; ++e) rhs[e] -= rl[e];
  } else {
    tri_mv<T, C, true>(rhs, Z, rz, p, ln, T(1));
#pragma unroll
    for (int e = 0; e < C; ++e) rhs[e] -= rl[e];
    if (j >= 1) tri_mv<T, C, true>(rhs, V, v, p, ln, T(1));
  }
  penta_solve<T, C>(l, rhs, fac, scan, p, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) u[e] = ru[e];
  tri_mtv<T, C, true>(u, N, l, p, ln, T(-1));
  if (kappa != T(0)) {
    T t[C];
    tri_mtv<T, C, false>(t, Z, l, p, ln, T(1));
#pragma unroll
    for (int e = 0; e < C; ++e) z[e] = rz[e] - t[e];
    if (j >= 1) {
#pragma unroll
      for (int e = 0; e < C; ++e) m[e] = fma(kappa, t[e], v[e] - rv[e]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < C; ++e) z[e] = rz[e];
    tri_mtv<T, C, true>(z, Z, l, p, ln, T(-1));
    if (j >= 1) {
#pragma unroll
      for (int e = 0; e < C; ++e) m[e] = v[e] - rv[e];
      tri_mtv<T, C, true>(m, V, l, p, ln, T(1));
    }
  }
}

template <typename T>
__device__ __forceinline__ void local_solve_dense(const LevelView<T> &L, int j,
                                                  const T *ru, const T *rz, const T *rl,
                                                  const T *rv, const T *rm,
                                                  T *u, T *z, T *l, T *v, T *m) {
  const int n = L.n, p = L.p, q = L.q;
  if (j == n) {
    for (int i = 0; i < p; ++i) {
      v[i] = -rm[i];
      m[i] = v[i] - rv[i];
    }
    return;
  }
  const T *N = L.N + j * L.sN, *V = L.V + j * L.sV, *Z = L.Z + j * L.sZ;
  const T *fac = L.fac + j * L.sFac;
  T rhs[kDenseMax];
  dn_mv<T>(rhs, N, ru, p, p, T(1), false);
  dn_mv<T>(rhs, Z, rz, p, q, T(1), true);
  for (int i = 0; i < p; ++i) rhs[i] -= rl[i];
  if (j >= 1) {
    for (int i = 0; i < p; ++i) v[i] = -rm[i];
    dn_mv<T>(rhs, V, v, p, p, T(1), true);
  }
  dn_chol_solve<T>(l, rhs, fac, p);
  for (int i = 0; i < p; ++i) u[i] = ru[i];
  for (int i = 0; i < q; ++i) z[i] = rz[i];
  dn_mtv<T>(u, N, l, p, p, T(-1), true);
  dn_mtv<T>(z, Z, l, p, q, T(-1), true);
  if (j >= 1) {
    for (int i = 0; i < p; ++i) m[i] = v[i] - rv[i];
    dn_mtv<T>(m, V, l, p, p, T(1), true);
  }
}

// ---------------------------------------------------------------------------
// out = D^-1 (r - C y), where C carries the couplings of A~ between blocks
// (the identity entries of L and L^T, Fig. 5): block j's mu_{j-1} row sees
// u_{j-1} (cplU) and its u_j row sees mu_j (cplM).  Either may be null (zero).
// With cplU = y.u, cplM = y.m this is one block-Jacobi sweep (Eq. jacobi-aj).
// omega != 1 (an option, not the paper's sweep) relaxes it:
// out = yold + omega (D^-1(...) - yold), yold null meaning 0.

template <typename T, int C>
__device__ __forceinline__ void relax_chunk(T (&x)[C], const T *yold, int len, int ln, T omega) {
  if (yold) {
    T o[C];
    chunk_load<T, C>(o, yold, len, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) x[e] = fma(omega, x[e] - o[e], o[e]);
  } else {
#pragma unroll
    for (int e = 0; e < C; ++e) x[e] *= omega;
  }
}

// 16-byte asynchronous copies global -> shared (cp.async, L2 only); the
// warp's lanes split `count` elements of T (count * sizeof(T) a multiple of 16,
// both addresses 16-byte aligned)
template <typename T>
__device__ __forceinline__ void stage16(T *dst, const T *src, int count, int ln) {
  const int chunks = count * (int)sizeof(T) / 16;
  const char *s = reinterpret_cast<const char *>(src);
  char *d = reinterpret_cast<char *>(dst);
  for (int c = ln; c < chunks; c += kWarp) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(d + 16 * c));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(s + 16 * c) : "memory");
  }
}

// shared memory of a staged block solve: per warp 12 p + kScanPerBlock values
template <typename T>
__host__ __device__ constexpr int tri_stage_elems(int p) { return 12 * p + kScanPerBlock; }

// kStage: each warp first copies its block's coefficients (bands of N, V, Z,
// factor, scan compositions: 12 p + 1280 values) into shared memory with
// cp.async, overlapping that one round trip with the loads of the right-hand
// side; the solve then reads them from shared memory.  Dynamic shared memory:
// 4 * tri_stage_elems(p) values of T.  Requires 3 p * sizeof(T) to be a multiple
// of 16 and 16-byte aligned coefficient arrays (checked on the host).
// PF > 0: p == PF == 32 C is known at compile time (every lane's chunk is full,
// so the bounds tests fold away).
template <typename T, int C, bool kStage = false, int PF = 0, typename CT = T>
__global__ void __launch_bounds__(128) k_block_solve_tri(LevelView<T, CT> L, const T *__restrict__ r,
                                                         const T *cplU, const T *cplM, T *out,
                                                         const T *yold, T omega, int j0 = 0, int j1 = -1) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int j = j0 + (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;  // blocks [j0, j1) (all: j1 < 0)
  const int n = L.n, p = PF ? PF : L.p, q = PF ? PF : L.q;
  if (j > n || (j1 >= 0 && j >= j1)) return;
  TriBlock<T, CT> Bk{};
  if (j < n) Bk = tri_block(L, j);
  if (kStage && j < n) {
    // bands at T offsets 0, 3p, 6p (as CT: a BF16 band fills the first half of its slot)
    extern __shared__ __align__(16) unsigned char tri_smem[];
    T *base = reinterpret_cast<T *>(tri_smem) + (threadIdx.x / kWarp) * tri_stage_elems<T>(p);
    stage16(reinterpret_cast<CT *>(base), Bk.N, 3 * p, ln);
    stage16(reinterpret_cast<CT *>(base + 3 * p), Bk.V, 3 * p, ln);
    stage16(reinterpret_cast<CT *>(base + 6 * p), Bk.Z, 3 * p, ln);
    stage16(base + 9 * p, Bk.fac, 3 * p, ln);
    stage16(base + 12 * p, Bk.scan, kScanPerBlock, ln);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    Bk = {reinterpret_cast<const CT *>(base), reinterpret_cast<const CT *>(base + 3 * p),
          reinterpret_cast<const CT *>(base + 6 * p), base + 9 * p, base + 12 * p};
  }
  Vec<const T> R = make_cvec(r, n, p, q);
  Vec<T> Y = make_vec(out, n, p, q);
  T ru[C], rz[C], rl[C], rv[C], rm[C];
  T u[C], z[C], l[C], v[C], m[C];
#pragma unroll
  for (int e = 0; e < C; ++e) { ru[e] = rz[e] = rl[e] = rv[e] = rm[e] = T(0); }
  if (j < n) {
    chunk_load<T, C>(ru, R.u + (long long)j * p, p, ln);
    chunk_load<T, C>(rz, R.z + (long long)j * q, q, ln);
    chunk_load<T, C>(rl, R.l + (long long)j * p, p, ln);
    if (cplM) {
      T c[C];
      chunk_load<T, C>(c, cplM + (long long)j * p, p, ln);
#pragma unroll
      for (int e = 0; e < C; ++e) ru[e] -= c[e];
    }
  }
  if (j >= 1) {
    chunk_load<T, C>(rv, R.v + (long long)(j - 1) * p, p, ln);
    chunk_load<T, C>(rm, R.m + (long long)(j - 1) * p, p, ln);
    if (cplU) {
      T c[C];
      chunk_load<T, C>(c, cplU + (long long)(j - 1) * p, p, ln);
#pragma unroll
      for (int e = 0; e < C; ++e) rm[e] -= c[e];
    }
  }
  if (kStage && j < n) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
  }
  local_solve_tri<T, C>(Bk, n, p, j, ru, rz, rl, rv, rm, u, z, l, v, m, ln, L.kappa);
  if (omega != T(1)) {
    Vec<const T> Yo = make_cvec(yold ? yold : r, n, p, q);
    if (j < n) {
      relax_chunk<T, C>(u, yold ? Yo.u + (long long)j * p : nullptr, p, ln, omega);
      relax_chunk<T, C>(z, yold ? Yo.z + (long long)j * q : nullptr, q, ln, omega);
      relax_chunk<T, C>(l, yold ? Yo.l + (long long)j * p : nullptr, p, ln, omega);
    }
    if (j >= 1) {
      relax_chunk<T, C>(v, yold ? Yo.v + (long long)(j - 1) * p : nullptr, p, ln, omega);
      relax_chunk<T, C>(m, yold ? Yo.m + (long long)(j - 1) * p : nullptr, p, ln, omega);
    }
  }
  if (j < n) {
    chunk_store<T, C>(Y.u + (long long)j * p, u, p, ln);
    chunk_store<T, C>(Y.z + (long long)j * q, z, q, ln);
    chunk_store<T, C>(Y.l + (long long)j * p, l, p, ln);
  }
  if (j >= 1) {
    chunk_store<T, C>(Y.v + (long long)(j - 1) * p, v, p, ln);
    chunk_store<T, C>(Y.m + (long long)(j - 1) * p, m, p, ln);
  }
}

// Tridiagonal blocks too large for one warp's registers (p > 128; one warp
// holds p / 32 values per lane and vector, 16 at p = 512, and the one-warp
// solve then runs at 255 registers, 8 warps per SM): the local solve of
// k_block_solve_tri in three launches with the same arithmetic, entry for
// entry, so the results are bitwise those of the one-warp kernel:
//   k_bs_rhs:   rhs = N r_u + Z (r_z + kappa v) - r_lambda (or N r_u + Z r_z -
//               r_lambda + V v), a thread per entry (neighbours read directly);
//   k_bs_penta: S lambda = rhs by the warp's chunked pentadiagonal solve
//               (penta_solve, p / 32 values per lane, nothing else live);
//   k_bs_out:   u, z, mu (and v) from lambda, relaxation, a thread per entry.
// rhs and lambda pass through L.ws_rhs and L.ws_lam ((n + 1) x p values).
// Blocks [j0, j1) (all: j1 < 0), couplings and relaxation as k_block_solve_tri.

// r_u - cplM and v = -(r_mu - cplU) of block j at entry k (0 outside [0, p))
template <typename T>
__device__ __forceinline__ T bs_ru(const Vec<const T> &R, const T *cplM, int j, int k, int p) {
  if (k < 0 || k >= p) return T(0);
  T v = R.u[(long long)j * p + k];
  if (cplM) v -= cplM[(long long)j * p + k];
  return v;
}
template <typename T>
__device__ __forceinline__ T bs_v(const Vec<const T> &R, const T *cplU, int j, int k, int p) {
  if (k < 0 || k >= p) return T(0);
  T rm = R.m[(long long)(j - 1) * p + k];
  if (cplU) rm -= cplU[(long long)(j - 1) * p + k];
  return -rm;
}
// (A x)_i and (A^T x)_i of a tridiagonal band A (3 rows of p), as tri_mv / tri_mtv form them
template <typename T, typename CT>
__device__ __forceinline__ T bs_mv(const CT *A, int i, int p, T xm, T x, T xp) {
  return fma(T(coef(A[i])), xm, fma(T(coef(A[p + i])), x, T(coef(A[2 * p + i])) * xp));
}
template <typename T, typename CT>
__device__ __forceinline__ T bs_mtv(const CT *A, int i, int p, T xm, T x, T xp) {
  const T up = (i > 0) ? T(coef(A[2 * p + i - 1])) : T(0);
  const T lo = (i + 1 < p) ? T(coef(A[i + 1])) : T(0);
  return fma(up, xm, fma(T(coef(A[p + i])), x, lo * xp));
}

template <typename T, typename CT>
__global__ void __launch_bounds__(256) k_bs_rhs(LevelView<T, CT> L, const T *__restrict__ r, const T *cplU,
                                                const T *cplM, int j0, int j1) {
  const int n = L.n, p = L.p, q = L.q;
  const int jend = (j1 < 0 ? n + 1 : j1) < n ? (j1 < 0 ? n + 1 : j1) : n;  // block n has no lambda
  const long long total = (long long)(jend - j0) * p;
  const Vec<const T> R = make_cvec(r, n, p, q);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = j0 + (int)(idx / p), i = (int)(idx % p);
    const CT *N = L.N + j * L.sN, *V = L.V + j * L.sV, *Z = L.Z + j * L.sZ;
    const T *rz = R.z + (long long)j * q;
    auto rzk = [&](int k) { return (k < 0 || k >= p) ? T(0) : rz[k]; };
    T rhs = bs_mv<T>(N, i, p, bs_ru(R, cplM, j, i - 1, p), bs_ru(R, cplM, j, i, p), bs_ru(R, cplM, j, i + 1, p));
    const T rl = R.l[(long long)j * p + i];
    if (L.kappa != T(0) && j >= 1) {
      auto wk = [&](int k) { return (k < 0 || k >= p) ? T(0) : fma(L.kappa, bs_v(R, cplU, j, k, p), rz[k]); };
      rhs = fma(T(1), bs_mv<T>(Z, i, p, wk(i - 1), wk(i), wk(i + 1)), rhs);
      rhs -= rl;
    } else {
      rhs = fma(T(1), bs_mv<T>(Z, i, p, rzk(i - 1), rzk(i), rzk(i + 1)), rhs);
      rhs -= rl;
      if (j >= 1)
        rhs = fma(T(1), bs_mv<T>(V, i, p, bs_v(R, cplU, j, i - 1, p), bs_v(R, cplU, j, i, p),
                                 bs_v(R, cplU, j, i + 1, p)),
                  rhs);
    }
    L.ws_rhs[(long long)j * p + i] = rhs;
  }
}

template <typename T, int C, typename CT>
__global__ void __launch_bounds__(128, 4) k_bs_penta(LevelView<T, CT> L, int j0, int j1) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int j = j0 + (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int n = L.n, p = L.p;
  if (j >= n || (j1 >= 0 && j >= j1)) return;
  T rhs[C], l[C];
  chunk_load<T, C>(rhs, L.ws_rhs + (long long)j * p, p, ln);
  penta_solve<T, C>(l, rhs, L.fac + j * L.sFac, L.scan + (long long)j * kScanPerBlock, p, ln);
  chunk_store<T, C>(L.ws_lam + (long long)j * p, l, p, ln);
}

template <typename T, typename CT>
__global__ void __launch_bounds__(256) k_bs_out(LevelView<T, CT> L, const T *__restrict__ r, const T *cplU,
                                                const T *cplM, T *out, const T *yold, T omega, int j0, int j1) {
  const int n = L.n, p = L.p, q = L.q;
  const int jend = j1 < 0 ? n + 1 : j1;
  const long long total = (long long)(jend - j0) * p;
  const Vec<const T> R = make_cvec(r, n, p, q);
  const Vec<T> Y = make_vec(out, n, p, q);
  const Vec<const T> Yo = make_cvec(yold ? yold : r, n, p, q);
  auto relax = [&](T x, const T *old, long long at) {
    if (omega == T(1)) return x;
    if (yold) {
      const T o = old[at];
      return fma(omega, x - o, o);
    }
    return x * omega;
  };
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = j0 + (int)(idx / p), i = (int)(idx % p);
    const long long at = (long long)j * p + i, atm = (long long)(j - 1) * p + i;
    if (j == n) {  // the last block holds v, mu of step n - 1 only
      const T v = bs_v(R, cplU, j, i, p);
      const T m = v - R.v[atm];
      Y.v[atm] = relax(v, Yo.v, atm);
      Y.m[atm] = relax(m, Yo.m, atm);
      continue;
    }
    const CT *N = L.N + j * L.sN, *V = L.V + j * L.sV, *Z = L.Z + j * L.sZ;
    const T *lam = L.ws_lam + (long long)j * p;
    const T lm = i > 0 ? lam[i - 1] : T(0), l0 = lam[i], lp = i + 1 < p ? lam[i + 1] : T(0);
    const T rz = R.z[(long long)j * q + i];
    const T u = fma(T(-1), bs_mtv<T>(N, i, p, lm, l0, lp), bs_ru(R, cplM, j, i, p));
    T z, m = T(0), v = T(0);
    if (j >= 1) v = bs_v(R, cplU, j, i, p);
    if (L.kappa != T(0)) {
      const T t = T(1) * bs_mtv<T>(Z, i, p, lm, l0, lp);
      z = rz - t;
      if (j >= 1) m = fma(L.kappa, t, v - R.v[atm]);
    } else {
      z = fma(T(-1), bs_mtv<T>(Z, i, p, lm, l0, lp), rz);
      if (j >= 1) {
        m = v - R.v[atm];
        m = fma(T(1), bs_mtv<T>(V, i, p, lm, l0, lp), m);
      }
    }
    Y.u[at] = relax(u, Yo.u, at);
    Y.z[(long long)j * q + i] = relax(z, Yo.z, (long long)j * q + i);
    Y.l[at] = relax(l0, Yo.l, at);
    if (j >= 1) {
      Y.v[atm] = relax(v, Yo.v, atm);
      Y.m[atm] = relax(m, Yo.m, atm);
    }
  }
}

// Two warps per time block (the same arithmetic split in two, for levels
// whose blocks do not fill the GPU): warp 0 forms N r_u, warp 1 Z r_z + V v -
// r_lambda; their sum goes through shared memory to warp 0, which solves the
// pentadiagonal system and returns lambda; then warp 0 forms u = r_u - N^T
// lambda and warp 1 z = r_z - Z^T lambda and mu = v + V^T lambda - r_v.  Each
// warp stages the coefficients it reads (cp.async) next to its loads.  A CTA
// of 128 threads holds two blocks; per block tri_pair_elems(p) values of
// dynamic shared memory.  Named barriers (id 1 + pair) join a block's warps.
template <typename T>
__host__ __device__ constexpr int tri_pair_elems(int p) { return 12 * p + kScanPerBlock + 2 * p; }

__device__ __forceinline__ void pair_barrier(int id) { asm volatile("bar.sync %0, 64;\n" ::"r"(id) : "memory"); }

template <typename T, int C, int PF = 0, typename CT = T>
__global__ void __launch_bounds__(128) k_block_solve_tri2(LevelView<T, CT> L, const T *__restrict__ r,
                                                          const T *cplU, const T *cplM, T *out,
                                                          const T *yold, T omega, int j0 = 0, int j1 = -1) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int w = threadIdx.x / kWarp, pair = w >> 1, role = w & 1;
  const int j = j0 + blockIdx.x * 2 + pair;  // blocks [j0, j1) (all: j1 < 0)
  const int n = L.n, p = PF ? PF : L.p, q = PF ? PF : L.q;
  if (j > n || (j1 >= 0 && j >= j1)) return;
  extern __shared__ __align__(16) unsigned char tri2_smem[];
  T *base = reinterpret_cast<T *>(tri2_smem) + pair * tri_pair_elems<T>(p);
  T *xch = base + 12 * p + kScanPerBlock;  // rhs part from warp 1, then lambda from warp 0
  Vec<const T> R = make_cvec(r, n, p, q);
  Vec<T> Y = make_vec(out, n, p, q);
  Vec<const T> Yo = make_cvec(yold ? yold : r, n, p, q);
  if (j == n) {  // last block: v = -r_mu, mu = v - r_v (warp 1 alone, no barrier)
    if (role == 1) {
      T rv[C], rm[C], v[C], m[C];
      chunk_load<T, C>(rv, R.v + (long long)(j - 1) * p, p, ln);
      chunk_load<T, C>(rm, R.m + (long long)(j - 1) * p, p, ln);
      if (cplU) {
        T c[C];
        chunk_load<T, C>(c, cplU + (long long)(j - 1) * p, p, ln);
#pragma unroll
        for (int e = 0; e < C; ++e) rm[e] -= c[e];
      }
#pragma unroll
      for (int e = 0; e < C; ++e) {
        v[e] = -rm[e];
        m[e] = v[e] - rv[e];
      }
      if (omega != T(1)) {
        relax_chunk<T, C>(v, yold ? Yo.v + (long long)(j - 1) * p : nullptr, p, ln, omega);
        relax_chunk<T, C>(m, yold ? Yo.m + (long long)(j - 1) * p : nullptr, p, ln, omega);
      }
      chunk_store<T, C>(Y.v + (long long)(j - 1) * p, v, p, ln);
      chunk_store<T, C>(Y.m + (long long)(j - 1) * p, m, p, ln);
    }
    return;
  }
  const TriBlock<T, CT> G = tri_block(L, j);
  if (role == 0) {
    stage16(reinterpret_cast<CT *>(base), G.N, 3 * p, ln);
    stage16(base + 9 * p, G.fac, 3 * p, ln);
    stage16(base + 12 * p, G.scan, kScanPerBlock, ln);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    T ru[C], rl[C], rhs[C], l[C];
    chunk_load<T, C>(ru, R.u + (long long)j * p, p, ln);
    chunk_load<T, C>(rl, R.l + (long long)j * p, p, ln);
    if (cplM) {
      T c[C];
      chunk_load<T, C>(c, cplM + (long long)j * p, p, ln);
#pragma unroll
      for (int e = 0; e < C; ++e) ru[e] -= c[e];
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const CT *N = reinterpret_cast<const CT *>(base);
    const T *fac = base + 9 * p, *scan = base + 12 * p;
    tri_mv<T, C, false>(rhs, N, ru, p, ln, T(1));
    pair_barrier(1 + pair);  // warp 1's part is in xch
    T part[C];
    chunk_load<T, C>(part, xch, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) rhs[e] += part[e];
    penta_solve<T, C>(l, rhs, fac, scan, p, ln);
    pair_barrier(1 + pair);  // warp 1 has read xch: reuse it for lambda
    chunk_store<T, C>(xch, l, p, ln);
    pair_barrier(1 + pair);
    T u[C];
#pragma unroll
    for (int e = 0; e < C; ++e) u[e] = ru[e];
    tri_mtv<T, C, true>(u, N, l, p, ln, T(-1));
    if (omega != T(1)) {
      relax_chunk<T, C>(u, yold ? Yo.u + (long long)j * p : nullptr, p, ln, omega);
      relax_chunk<T, C>(l, yold ? Yo.l + (long long)j * p : nullptr, p, ln, omega);
    }
    chunk_store<T, C>(Y.u + (long long)j * p, u, p, ln);
    chunk_store<T, C>(Y.l + (long long)j * p, l, p, ln);
  } else {
    stage16(reinterpret_cast<CT *>(base + 3 * p), G.V, 3 * p, ln);
    stage16(reinterpret_cast<CT *>(base + 6 * p), G.Z, 3 * p, ln);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    T rz[C], rl[C], rv[C], rm[C], v[C], part[C];
    chunk_load<T, C>(rz, R.z + (long long)j * q, q, ln);
    chunk_load<T, C>(rl, R.l + (long long)j * p, p, ln);
    if (j >= 1) {
      chunk_load<T, C>(rv, R.v + (long long)(j - 1) * p, p, ln);
      chunk_load<T, C>(rm, R.m + (long long)(j - 1) * p, p, ln);
      if (cplU) {
        T c[C];
        chunk_load<T, C>(c, cplU + (long long)(j - 1) * p, p, ln);
#pragma unroll
        for (int e = 0; e < C; ++e) rm[e] -= c[e];
      }
#pragma unroll
      for (int e = 0; e < C; ++e) v[e] = -rm[e];
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const CT *V = reinterpret_cast<const CT *>(base + 3 * p), *Z = reinterpret_cast<const CT *>(base + 6 * p);
    const T kappa = L.kappa;
    if (kappa != T(0) && j >= 1) {  // V = kappa Z: one product
      T wz[C];
#pragma unroll
      for (int e = 0; e < C; ++e) wz[e] = fma(kappa, v[e], rz[e]);
      tri_mv<T, C, false>(part, Z, wz, p, ln, T(1));
#pragma unroll
      for (int e = 0; e < C; ++e) part[e] -= rl[e];
    } else {
      tri_mv<T, C, false>(part, Z, rz, p, ln, T(1));
#pragma unroll
      for (int e = 0; e < C; ++e) part[e] -= rl[e];
      if (j >= 1) tri_mv<T, C, true>(part, V, v, p, ln, T(1));
    }
    chunk_store<T, C>(xch, part, p, ln);
    pair_barrier(1 + pair);
    pair_barrier(1 + pair);  // warp 0 has read the part
    pair_barrier(1 + pair);  // lambda is in xch
    T l[C], z[C], t[C];
    chunk_load<T, C>(l, xch, p, ln);
    if (kappa != T(0)) {
      tri_mtv<T, C, false>(t, Z, l, p, ln, T(1));
#pragma unroll
      for (int e = 0; e < C; ++e) z[e] = rz[e] - t[e];
    } else {
#pragma unroll
      for (int e = 0; e < C; ++e) z[e] = rz[e];
      tri_mtv<T, C, true>(z, Z, l, p, ln, T(-1));
    }
    if (omega != T(1)) relax_chunk<T, C>(z, yold ? Yo.z + (long long)j * q : nullptr, q, ln, omega);
    chunk_store<T, C>(Y.z + (long long)j * q, z, q, ln);
    if (j >= 1) {
      T m[C];
      if (kappa != T(0)) {
#pragma unroll
        for (int e = 0; e < C; ++e) m[e] = fma(kappa, t[e], v[e] - rv[e]);
      } else {
#pragma unroll
        for (int e = 0; e < C; ++e) m[e] = v[e] - rv[e];
        tri_mtv<T, C, true>(m, V, l, p, ln, T(1));
      }
      if (omega != T(1)) {
        relax_chunk<T, C>(v, yold ? Yo.v + (long long)(j - 1) * p : nullptr, p, ln, omega);
        relax_chunk<T, C>(m, yold ? Yo.m + (long long)(j - 1) * p : nullptr, p, ln, omega);
      }
      chunk_store<T, C>(Y.v + (long long)(j - 1) * p, v, p, ln);
      chunk_store<T, C>(Y.m + (long long)(j - 1) * p, m, p, ln);
    }
  }
}

// ---------------------------------------------------------------------------
// Several block-Jacobi sweeps of one level in one launch (two warps per time
// block, as k_block_solve_tri2).  Each warp pair owns one block for all
// sweeps: the block's coefficients are staged into shared memory once, its
// right-hand side and its iterate stay in registers, and only the couplings
// cross blocks: after sweep k a block publishes u_j (warp 0) and mu_{j-1}
// (warp 1) into a double-buffered exchange array and raises a per-block
// counter; sweep k + 1 of block j waits for the counters of blocks j - 1 (u)
// and j + 1 (mu).  Counters only grow (every block of a level ends a launch at
// the same count, which is where the next launch starts), so nothing resets
// them between launches.  The launch must be cooperative (every CTA resident
// at once); a wait gives up after kSweepWaitNs, sets err[0] and the kernel
// finishes without further waits (results void, the solve reports a timeout).
// Same arithmetic in the same order as `sweeps` launches of k_block_solve_tri2:
// bitwise-equal results.  y0 null: start from y = 0; else from y0 (out != y0).

constexpr unsigned long long kSweepWaitNs = 2000000000ull;  // 2 s

template <typename T>
struct SweepXchg {
  T *xu;         // [2][n + 1][p]: u_j published by block j after sweep k (slot k & 1)
  T *xm;         // [2][n + 1][p]: mu_{j-1} published by block j
  unsigned *fu;  // [n + 1] sweeps completed by block j's warp 0 (its u published)
  unsigned *fm;  // [n + 1] sweeps completed by block j's warp 1 (its mu published)
  int *err;      // set when a wait runs out
  int stall;     // failure-detection tests only: block 0 never publishes its u (a wait on it runs out)
};

__device__ __forceinline__ unsigned long long sweep_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// every lane polls the counter until it reaches `target` (acquire); false when
// err[0] is set or the wait runs out (then err[0] is set)
__device__ __forceinline__ bool sweep_wait(const unsigned *flag, unsigned target, int *err) {
  const unsigned long long t0 = sweep_clock_ns();
  for (unsigned it = 1;; ++it) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(flag) : "memory");
    if ((int)(v - target) >= 0) return true;
    if (*(volatile int *)err) return false;
    if ((it & 15u) == 0 && sweep_clock_ns() - t0 > kSweepWaitNs) {
      atomicOr(err, 1);
      return false;
    }
    __nanosleep(32);
  }
}

// the warp's stores are made visible device-wide, then lane 0 raises the counter (release)
__device__ __forceinline__ void sweep_publish(unsigned *flag, unsigned value, int ln) {
  __threadfence();
  __syncwarp();
  if (ln == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(flag), "r"(value) : "memory");
}

template <typename T, int C>
__device__ __forceinline__ void relax_regs(T (&x)[C], const T (&o)[C], T omega) {
#pragma unroll
  for (int e = 0; e < C; ++e) x[e] = fma(omega, x[e] - o[e], o[e]);
}

template <typename T, int C>
__device__ __forceinline__ void load_cg(T (&x)[C], const T *src, int p, int ln) {
#pragma unroll
  for (int e = 0; e < C; ++e) {
    const int i = ln * C + e;
    x[e] = (i < p) ? __ldcg(src + i) : T(0);
  }
}

template <typename T, int C, int PF = 0>
__global__ void __launch_bounds__(128) k_sweeps_tri2(LevelView<T> L, const T *__restrict__ r, const T *y0, T *out,
                                                     int sweeps, T omega, SweepXchg<T> X) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int w = threadIdx.x / kWarp, pair = w >> 1, role = w & 1;
  const int j = blockIdx.x * 2 + pair;
  const int n = L.n, p = PF ? PF : L.p, q = PF ? PF : L.q;
  if (j > n) return;
  const long long np1p = (long long)(n + 1) * p;
  extern __shared__ __align__(16) unsigned char sw2_smem[];
  T *base = reinterpret_cast<T *>(sw2_smem) + pair * tri_pair_elems<T>(p);
  T *xch = base + 12 * p + kScanPerBlock;
  Vec<const T> R = make_cvec(r, n, p, q);
  Vec<T> Y = make_vec(out, n, p, q);
  Vec<const T> Y0 = make_cvec(y0 ? y0 : r, n, p, q);
  const bool relax = omega != T(1);
  bool live = true;  // false once a wait has given up: no further waits
  if (role == 1 && j == n) {  // last block: v = -(r_mu - u_{n-1}), mu = v - r_v
    const unsigned s0 = *(volatile unsigned *)&X.fm[j];
    T rv[C], rm[C], v[C], m[C], vo[C], mo[C];
    chunk_load<T, C>(rv, R.v + (long long)(j - 1) * p, p, ln);
    chunk_load<T, C>(rm, R.m + (long long)(j - 1) * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) vo[e] = mo[e] = T(0);
    if (y0) {
      chunk_load<T, C>(vo, Y0.v + (long long)(j - 1) * p, p, ln);
      chunk_load<T, C>(mo, Y0.m + (long long)(j - 1) * p, p, ln);
    }
    for (int k = 0; k < sweeps; ++k) {
      T c[C];
      if (k == 0) {
        if (y0) chunk_load<T, C>(c, Y0.u + (long long)(j - 1) * p, p, ln);
      } else {
        if (live) live = sweep_wait(&X.fu[j - 1], s0 + k, X.err);
        load_cg<T, C>(c, X.xu + ((k - 1) & 1) * np1p + (long long)(j - 1) * p, p, ln);
      }
#pragma unroll
      for (int e = 0; e < C; ++e) {
        v[e] = (k == 0 && !y0) ? -rm[e] : -(rm[e] - c[e]);
        m[e] = v[e] - rv[e];
      }
      if (relax) {
        relax_regs<T, C>(v, vo, omega);
        relax_regs<T, C>(m, mo, omega);
      }
#pragma unroll
      for (int e = 0; e < C; ++e) { vo[e] = v[e]; mo[e] = m[e]; }
      if (k + 1 < sweeps) {
        chunk_store<T, C>(X.xm + (k & 1) * np1p + (long long)j * p, m, p, ln);
        sweep_publish(&X.fm[j], s0 + k + 1, ln);
      }
    }
    chunk_store<T, C>(Y.v + (long long)(j - 1) * p, vo, p, ln);
    chunk_store<T, C>(Y.m + (long long)(j - 1) * p, mo, p, ln);
    // the counter still advances by `sweeps` so that every block ends the launch at the same count
    sweep_publish(&X.fm[j], s0 + sweeps, ln);
    return;
  }
  if (j == n) return;  // warp 0 of the last block has nothing to do
  const TriBlock<T> G = tri_block(L, j);
  if (role == 0) {
    const unsigned s0 = *(volatile unsigned *)&X.fu[j];
    stage16(base, G.N, 3 * p, ln);
    stage16(base + 9 * p, G.fac, 3 * p, ln);
    stage16(base + 12 * p, G.scan, kScanPerBlock, ln);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    T ru[C], rl[C], uo[C], lo[C];
    chunk_load<T, C>(ru, R.u + (long long)j * p, p, ln);
    chunk_load<T, C>(rl, R.l + (long long)j * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) uo[e] = lo[e] = T(0);
    if (y0) {
      chunk_load<T, C>(uo, Y0.u + (long long)j * p, p, ln);
      chunk_load<T, C>(lo, Y0.l + (long long)j * p, p, ln);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const T *N = base, *fac = base + 9 * p, *scan = base + 12 * p;
    for (int k = 0; k < sweeps; ++k) {
      T ruk[C];
      if (k == 0 && !y0) {
#pragma unroll
        for (int e = 0; e < C; ++e) ruk[e] = ru[e];
      } else {
        T c[C];
        if (k == 0) {
          chunk_load<T, C>(c, Y0.m + (long long)j * p, p, ln);
        } else {
          if (live) live = sweep_wait(&X.fm[j + 1], s0 + k, X.err);
          load_cg<T, C>(c, X.xm + ((k - 1) & 1) * np1p + (long long)(j + 1) * p, p, ln);
        }
#pragma unroll
        for (int e = 0; e < C; ++e) ruk[e] = ru[e] - c[e];
      }
      T rhs[C], l[C], u[C];
      tri_mv<T, C, false>(rhs, N, ruk, p, ln, T(1));
      pair_barrier(1 + pair);  // warp 1's part is in xch
      T part[C];
      chunk_load<T, C>(part, xch, p, ln);
#pragma unroll
      for (int e = 0; e < C; ++e) rhs[e] += part[e];
      penta_solve<T, C>(l, rhs, fac, scan, p, ln);
      pair_barrier(1 + pair);  // warp 1 has read xch: reuse it for lambda
      chunk_store<T, C>(xch, l, p, ln);
      pair_barrier(1 + pair);
#pragma unroll
      for (int e = 0; e < C; ++e) u[e] = ruk[e];
      tri_mtv<T, C, true>(u, N, l, p, ln, T(-1));
      if (relax) {
        relax_regs<T, C>(u, uo, omega);
        relax_regs<T, C>(l, lo, omega);
      }
#pragma unroll
      for (int e = 0; e < C; ++e) { uo[e] = u[e]; lo[e] = l[e]; }
      const bool mute = X.stall && j == 0;
      if (k + 1 < sweeps && !mute) {
        chunk_store<T, C>(X.xu + (k & 1) * np1p + (long long)j * p, u, p, ln);
        sweep_publish(&X.fu[j], s0 + k + 1, ln);
      }
    }
    chunk_store<T, C>(Y.u + (long long)j * p, uo, p, ln);
    chunk_store<T, C>(Y.l + (long long)j * p, lo, p, ln);
    if (!(X.stall && j == 0)) sweep_publish(&X.fu[j], s0 + sweeps, ln);
  } else {
    const unsigned s0 = *(volatile unsigned *)&X.fm[j];
    stage16(base + 3 * p, G.V, 3 * p, ln);
    stage16(base + 6 * p, G.Z, 3 * p, ln);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    T rz[C], rl[C], rv[C], rm[C], zo[C], vo[C], mo[C];
    chunk_load<T, C>(rz, R.z + (long long)j * q, q, ln);
    chunk_load<T, C>(rl, R.l + (long long)j * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) { rv[e] = rm[e] = zo[e] = vo[e] = mo[e] = T(0); }
    if (j >= 1) {
      chunk_load<T, C>(rv, R.v + (long long)(j - 1) * p, p, ln);
      chunk_load<T, C>(rm, R.m + (long long)(j - 1) * p, p, ln);
    }
    if (y0) {
      chunk_load<T, C>(zo, Y0.z + (long long)j * q, q, ln);
      if (j >= 1) {
        chunk_load<T, C>(vo, Y0.v + (long long)(j - 1) * p, p, ln);
        chunk_load<T, C>(mo, Y0.m + (long long)(j - 1) * p, p, ln);
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const T *V = base + 3 * p, *Z = base + 6 * p;
    const T kappa = L.kappa;
    for (int k = 0; k < sweeps; ++k) {
      T v[C], part[C];
      if (j >= 1) {
        if (k == 0 && !y0) {
#pragma unroll
          for (int e = 0; e < C; ++e) v[e] = -rm[e];
        } else {
          T c[C];
          if (k == 0) {
            chunk_load<T, C>(c, Y0.u + (long long)(j - 1) * p, p, ln);
          } else {
            if (live) live = sweep_wait(&X.fu[j - 1], s0 + k, X.err);
            load_cg<T, C>(c, X.xu + ((k - 1) & 1) * np1p + (long long)(j - 1) * p, p, ln);
          }
#pragma unroll
          for (int e = 0; e < C; ++e) v[e] = -(rm[e] - c[e]);
        }
      }
      if (kappa != T(0) && j >= 1) {  // V = kappa Z: one product
        T wz[C];
#pragma unroll
        for (int e = 0; e < C; ++e) wz[e] = fma(kappa, v[e], rz[e]);
        tri_mv<T, C, false>(part, Z, wz, p, ln, T(1));
#pragma unroll
        for (int e = 0; e < C; ++e) part[e] -= rl[e];
      } else {
        tri_mv<T, C, false>(part, Z, rz, p, ln, T(1));
#pragma unroll
        for (int e = 0; e < C; ++e) part[e] -= rl[e];
        if (j >= 1) tri_mv<T, C, true>(part, V, v, p, ln, T(1));
      }
      chunk_store<T, C>(xch, part, p, ln);
      pair_barrier(1 + pair);
      pair_barrier(1 + pair);  // warp 0 has read the part
      pair_barrier(1 + pair);  // lambda is in xch
      T l[C], z[C], t[C];
      chunk_load<T, C>(l, xch, p, ln);
      if (kappa != T(0)) {
        tri_mtv<T, C, false>(t, Z, l, p, ln, T(1));
#pragma unroll
        for (int e = 0; e < C; ++e) z[e] = rz[e] - t[e];
      } else {
#pragma unroll
        for (int e = 0; e < C; ++e) z[e] = rz[e];
        tri_mtv<T, C, true>(z, Z, l, p, ln, T(-1));
      }
      if (relax) relax_regs<T, C>(z, zo, omega);
#pragma unroll
      for (int e = 0; e < C; ++e) zo[e] = z[e];
      if (j >= 1) {
        T m[C];
        if (kappa != T(0)) {
#pragma unroll
          for (int e = 0; e < C; ++e) m[e] = fma(kappa, t[e], v[e] - rv[e]);
        } else {
#pragma unroll
          for (int e = 0; e < C; ++e) m[e] = v[e] - rv[e];
          tri_mtv<T, C, true>(m, V, l, p, ln, T(1));
        }
        if (relax) {
          relax_regs<T, C>(v, vo, omega);
          relax_regs<T, C>(m, mo, omega);
        }
#pragma unroll
        for (int e = 0; e < C; ++e) { vo[e] = v[e]; mo[e] = m[e]; }
        if (k + 1 < sweeps) {
          chunk_store<T, C>(X.xm + (k & 1) * np1p + (long long)j * p, m, p, ln);
          sweep_publish(&X.fm[j], s0 + k + 1, ln);
        }
      }
    }
    chunk_store<T, C>(Y.z + (long long)j * q, zo, q, ln);
    if (j >= 1) {
      chunk_store<T, C>(Y.v + (long long)(j - 1) * p, vo, p, ln);
      chunk_store<T, C>(Y.m + (long long)(j - 1) * p, mo, p, ln);
    }
    sweep_publish(&X.fm[j], s0 + sweeps, ln);
  }
}

// Dense blocks with p, q <= 32 (kDenseWarpMax): one warp per time block, lane i
// holding entry i of every vector; the same Schur-complement solve as
// local_solve_dense, products by broadcasts, S^-1 by column substitutions.
template <typename T>
__global__ void __launch_bounds__(128) k_block_solve_dw(LevelView<T> L, const T *__restrict__ r,
                                                        const T *cplU, const T *cplM, T *out,
                                                        const T *yold, T omega, int j0 = 0, int j1 = -1) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int j = j0 + (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;  // blocks [j0, j1) (all: j1 < 0)
  const int n = L.n, p = L.p, q = L.q;
  if (j > n || (j1 >= 0 && j >= j1)) return;
  Vec<const T> R = make_cvec(r, n, p, q);
  Vec<T> Y = make_vec(out, n, p, q);
  Vec<const T> Yo = make_cvec(yold ? yold : r, n, p, q);
  const bool relax = omega != T(1);
  auto rlx = [&](T x, const T *o, int len) {
    if (!relax) return x;
    const T old = (yold && ln < len) ? o[ln] : T(0);
    return yold ? fma(omega, x - old, old) : omega * x;
  };
  T ru = 0, rz = 0, rl = 0, rv = 0, rm = 0, v = 0;
  if (j < n) {
    ru = dw_load(R.u + (long long)j * p, p, ln);
    rz = dw_load(R.z + (long long)j * q, q, ln);
    rl = dw_load(R.l + (long long)j * p, p, ln);
    if (cplM) ru -= dw_load(cplM + (long long)j * p, p, ln);
  }
  if (j >= 1) {
    rv = dw_load(R.v + (long long)(j - 1) * p, p, ln);
    rm = dw_load(R.m + (long long)(j - 1) * p, p, ln);
    if (cplU) rm -= dw_load(cplU + (long long)(j - 1) * p, p, ln);
    v = -rm;
  }
  if (j == n) {
    const T m = v - rv;
    if (ln < p) {
      Y.v[(long long)(j - 1) * p + ln] = rlx(v, Yo.v + (long long)(j - 1) * p, p);
      Y.m[(long long)(j - 1) * p + ln] = rlx(m, Yo.m + (long long)(j - 1) * p, p);
    }
    return;
  }
  const T *N = L.N + j * L.sN, *V = L.V + j * L.sV, *Z = L.Z + j * L.sZ, *fac = L.fac + j * L.sFac;
  T rhs = dw_mv(N, ru, p, p, ln) + dw_mv(Z, rz, p, q, ln) - rl;
  if (j >= 1) rhs += dw_mv(V, v, p, p, ln);
  if (ln >= p) rhs = T(0);
  const T l = dw_chol_solve(fac, rhs, p, ln);
  const T u = ru - dw_mtv(N, l, p, p, ln);
  const T z = rz - dw_mtv(Z, l, p, q, ln);
  if (ln < p) {
    Y.u[(long long)j * p + ln] = rlx(u, Yo.u + (long long)j * p, p);
    Y.l[(long long)j * p + ln] = rlx(l, Yo.l + (long long)j * p, p);
  }
  if (ln < q) Y.z[(long long)j * q + ln] = rlx(z, Yo.z + (long long)j * q, q);
  if (j >= 1) {
    const T m = v - rv + dw_mtv(V, l, p, p, ln);
    if (ln < p) {
      Y.v[(long long)(j - 1) * p + ln] = rlx(v, Yo.v + (long long)(j - 1) * p, p);
      Y.m[(long long)(j - 1) * p + ln] = rlx(m, Yo.m + (long long)(j - 1) * p, p);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_block_solve_dense(LevelView<T> L, const T *__restrict__ r,
                                                           const T *cplU, const T *cplM, T *out,
                                                           const T *yold, T omega, int j0 = 0, int j1 = -1) {
  const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;  // blocks [j0, j1) (all: j1 < 0)
  const int n = L.n, p = L.p, q = L.q;
  if (j > n || (j1 >= 0 && j >= j1)) return;
  Vec<const T> R = make_cvec(r, n, p, q);
  Vec<T> Y = make_vec(out, n, p, q);
  T ru[kDenseMax] = {}, rz[kDenseMax] = {}, rl[kDenseMax] = {}, rv[kDenseMax] = {}, rm[kDenseMax] = {};
  T u[kDenseMax], z[kDenseMax], l[kDenseMax], v[kDenseMax], m[kDenseMax];
  if (j < n) {
    for (int i = 0; i < p; ++i) {
      ru[i] = R.u[(long long)j * p + i];
      rl[i] = R.l[(long long)j * p + i];
      if (cplM) ru[i] -= cplM[(long long)j * p + i];
    }
    for (int i = 0; i < q; ++i) rz[i] = R.z[(long long)j * q + i];
  }
  if (j >= 1) {
    for (int i = 0; i < p; ++i) {
      rv[i] = R.v[(long long)(j - 1) * p + i];
      rm[i] = R.m[(long long)(j - 1) * p + i];
      if (cplU) rm[i] -= cplU[(long long)(j - 1) * p + i];
    }
  }
  local_solve_dense<T>(L, j, ru, rz, rl, rv, rm, u, z, l, v, m);
  if (omega != T(1)) {
    Vec<const T> Yo = make_cvec(yold ? yold : r, n, p, q);
    auto relax = [&](T *x, const T *o, int len) {
      for (int i = 0; i < len; ++i) x[i] = yold ? fma(omega, x[i] - o[i], o[i]) : omega * x[i];
    };
    if (j < n) {
      relax(u, Yo.u + (long long)j * p, p);
      relax(z, Yo.z + (long long)j * q, q);
      relax(l, Yo.l + (long long)j * p, p);
    }
    if (j >= 1) {
      relax(v, Yo.v + (long long)(j - 1) * p, p);
      relax(m, Yo.m + (long long)(j - 1) * p, p);
    }
  }
  if (j < n) {
    for (int i = 0; i < p; ++i) {
      Y.u[(long long)j * p + i] = u[i];
      Y.l[(long long)j * p + i] = l[i];
    }
    for (int i = 0; i < q; ++i) Y.z[(long long)j * q + i] = z[i];
  }
  if (j >= 1) {
    for (int i = 0; i < p; ++i) {
      Y.v[(long long)(j - 1) * p + i] = v[i];
      Y.m[(long long)(j - 1) * p + i] = m[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Rows of A~ x for step t (Fig. 4 rows, in the type-major layout):
//   u_t:      u_t + N_t^T l_t + m_t
//   v_t:      v_t + V_{t+1}^T l_{t+1} - m_t          (no V term for t = n-1)
//   z_t:      z_t + Z_t^T l_t
//   lambda_t: V_t v_{t-1} + N_t u_t + Z_t z_t       (no V term for t = 0)
//   mu_t:     u_t - v_t

// out = b - A~ x  (b non-null)  or  out = A~ x  (b null), all five types.
// xcopy (optional, whole level only): x is also stored into basis slot
// xcopy + (xcopy_idx[0] + xcopy_shift) * n (4p + q), each step by its warp
template <typename T>
__device__ __forceinline__ T *copy_slot(T *xcopy, const int *xcopy_idx, int xcopy_shift, int n, int p, int q) {
  return xcopy ? xcopy + (long long)(xcopy_idx[0] + xcopy_shift) * ((long long)n * (4 * p + q)) : nullptr;
}

template <typename T, int C, typename CT = T>
__global__ void __launch_bounds__(128) k_apply_tri(LevelView<T, CT> L, const T *__restrict__ x,
                                                   const T *__restrict__ b, T *out, const int *guard = nullptr,
                                                   int j0 = 0, int j1 = -1, T *xcopy = nullptr,
                                                   const int *xcopy_idx = nullptr, int xcopy_shift = 0) {
  if (guard && *guard == 0) return;
  const int ln = threadIdx.x & (kWarp - 1);
  const int n = L.n, p = L.p, q = L.q;
  // the rows of time blocks [j0, j1) (all: j1 < 0): u, z, lambda rows of steps [j0, j1), v, mu rows of
  // steps [j0 - 1, j1 - 1); a warp per step t from max(j0 - 1, 0)
  const int t = max(j0 - 1, 0) + (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int tend = j1 < 0 ? n : min(j1, n);
  if (t >= tend) return;
  const bool own_uzl = t >= j0, own_vm = t + 1 >= j0 && (j1 < 0 || t + 1 < j1);
  Vec<const T> X = make_cvec(x, n, p, q);
  Vec<T> O = make_vec(out, n, p, q);
  const CT *N = L.N + t * L.sN, *Z = L.Z + t * L.sZ, *Vt = L.V + t * L.sV;
  T xu[C], xv[C], xz[C], xl[C], xm[C], acc[C];
  chunk_load<T, C>(xu, X.u + (long long)t * p, p, ln);
  chunk_load<T, C>(xv, X.v + (long long)t * p, p, ln);
  chunk_load<T, C>(xz, X.z + (long long)t * q, q, ln);
  chunk_load<T, C>(xl, X.l + (long long)t * p, p, ln);
  chunk_load<T, C>(xm, X.m + (long long)t * p, p, ln);
  if (T *cp = copy_slot(xcopy, xcopy_idx, xcopy_shift, n, p, q)) {
    Vec<T> Cv = make_vec(cp, n, p, q);
    chunk_store<T, C>(Cv.u + (long long)t * p, xu, p, ln);
    chunk_store<T, C>(Cv.v + (long long)t * p, xv, p, ln);
    chunk_store<T, C>(Cv.z + (long long)t * q, xz, q, ln);
    chunk_store<T, C>(Cv.l + (long long)t * p, xl, p, ln);
    chunk_store<T, C>(Cv.m + (long long)t * p, xm, p, ln);
  }
  const T sgn = b ? T(-1) : T(1);
  Vec<const T> B = make_cvec(b ? b : x, n, p, q);
  // u row
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = xu[e] + xm[e];
  tri_mtv<T, C, true>(acc, N, xl, p, ln, T(1));
  {
    T o[C];
    if (b) chunk_load<T, C>(o, B.u + (long long)t * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) o[e] = b ? fma(sgn, acc[e], o[e]) : acc[e];
    if (own_uzl) chunk_store<T, C>(O.u + (long long)t * p, o, p, ln);
  }
  // v row
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = xv[e] - xm[e];
  if (t + 1 < n) {
    T xl1[C];
    chunk_load<T, C>(xl1, X.l + (long long)(t + 1) * p, p, ln);
    tri_mtv<T, C, true>(acc, L.V + (t + 1) * L.sV, xl1, p, ln, T(1));
  }
  {
    T o[C];
    if (b) chunk_load<T, C>(o, B.v + (long long)t * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) o[e] = b ? fma(sgn, acc[e], o[e]) : acc[e];
    if (own_vm) chunk_store<T, C>(O.v + (long long)t * p, o, p, ln);
  }
  // z row
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = xz[e];
  tri_mtv<T, C, true>(acc, Z, xl, p, ln, T(1));
  {
    T o[C];
    if (b) chunk_load<T, C>(o, B.z + (long long)t * q, q, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) o[e] = b ? fma(sgn, acc[e], o[e]) : acc[e];
    if (own_uzl) chunk_store<T, C>(O.z + (long long)t * q, o, q, ln);
  }
  // lambda row
  tri_mv<T, C, false>(acc, N, xu, p, ln, T(1));
  tri_mv<T, C, true>(acc, Z, xz, p, ln, T(1));
  if (t >= 1) {
    T xv0[C];
    chunk_load<T, C>(xv0, X.v + (long long)(t - 1) * p, p, ln);
    tri_mv<T, C, true>(acc, Vt, xv0, p, ln, T(1));
  }
  {
    T o[C];
    if (b) chunk_load<T, C>(o, B.l + (long long)t * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) o[e] = b ? fma(sgn, acc[e], o[e]) : acc[e];
    if (own_uzl) chunk_store<T, C>(O.l + (long long)t * p, o, p, ln);
  }
  // mu row
  {
    T o[C];
    if (b) chunk_load<T, C>(o, B.m + (long long)t * p, p, ln);
#pragma unroll
    for (int e = 0; e < C; ++e) o[e] = b ? fma(sgn, xu[e] - xv[e], o[e]) : xu[e] - xv[e];
    if (own_vm) chunk_store<T, C>(O.m + (long long)t * p, o, p, ln);
  }
}

// k_apply_tri for blocks too large for one warp's registers (p > 128): a
// thread per (step, entry) forms the five rows of that entry with the same
// operations as k_apply_tri (bitwise the same results); arguments as there.
template <typename T, typename CT>
__global__ void __launch_bounds__(256) k_apply_ent(LevelView<T, CT> L, const T *__restrict__ x,
                                                   const T *__restrict__ b, T *out, const int *guard = nullptr,
                                                   int j0 = 0, int j1 = -1, T *xcopy = nullptr,
                                                   const int *xcopy_idx = nullptr, int xcopy_shift = 0) {
  if (guard && *guard == 0) return;
  const int n = L.n, p = L.p, q = L.q;
  const int t0 = max(j0 - 1, 0), tend = j1 < 0 ? n : min(j1, n);
  const long long total = (long long)(tend - t0) * p;
  const Vec<const T> X = make_cvec(x, n, p, q);
  const Vec<T> O = make_vec(out, n, p, q);
  const T sgn = b ? T(-1) : T(1);
  const Vec<const T> B = make_cvec(b ? b : x, n, p, q);
  T *cp = copy_slot(xcopy, xcopy_idx, xcopy_shift, n, p, q);
  const Vec<T> Cv = make_vec(cp ? cp : out, n, p, q);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int t = t0 + (int)(idx / p), i = (int)(idx % p);
    const bool own_uzl = t >= j0, own_vm = t + 1 >= j0 && (j1 < 0 || t + 1 < j1);
    const CT *N = L.N + t * L.sN, *Z = L.Z + t * L.sZ, *Vt = L.V + t * L.sV;
    const long long at = (long long)t * p + i;
    auto ld = [&](const T *v, long long base, int k) { return (k < 0 || k >= p) ? T(0) : v[base + k]; };
    const long long bt = (long long)t * p;
    const T xu = X.u[at], xv = X.v[at], xz = X.z[(long long)t * q + i], xl = X.l[at], xm = X.m[at];
    if (cp) {
      Cv.u[at] = xu;
      Cv.v[at] = xv;
      Cv.z[(long long)t * q + i] = xz;
      Cv.l[at] = xl;
      Cv.m[at] = xm;
    }
    const T xlm = ld(X.l, bt, i - 1), xlp = ld(X.l, bt, i + 1);
    auto emit = [&](T *o, const T *bb, long long a, T acc) { o[a] = b ? fma(sgn, acc, bb[a]) : acc; };
    // u row
    {
      T acc = xu + xm;
      acc = fma(T(1), bs_mtv<T>(N, i, p, xlm, xl, xlp), acc);
      if (own_uzl) emit(O.u, B.u, at, acc);
    }
    // v row
    {
      T acc = xv - xm;
      if (t + 1 < n) {
        const long long b1 = (long long)(t + 1) * p;
        acc = fma(T(1), bs_mtv<T>(L.V + (t + 1) * L.sV, i, p, ld(X.l, b1, i - 1), X.l[b1 + i], ld(X.l, b1, i + 1)),
                  acc);
      }
      if (own_vm) emit(O.v, B.v, at, acc);
    }
    // z row
    {
      const T acc = fma(T(1), bs_mtv<T>(Z, i, p, xlm, xl, xlp), xz);
      if (own_uzl) emit(O.z, B.z, (long long)t * q + i, acc);
    }
    // lambda row
    {
      const long long bz = (long long)t * q;
      T acc = T(1) * bs_mv<T>(N, i, p, ld(X.u, bt, i - 1), xu, ld(X.u, bt, i + 1));
      acc = fma(T(1), bs_mv<T>(Z, i, p, ld(X.z, bz, i - 1), xz, ld(X.z, bz, i + 1)), acc);
      if (t >= 1) {
        const long long b0 = (long long)(t - 1) * p;
        acc = fma(T(1), bs_mv<T>(Vt, i, p, ld(X.v, b0, i - 1), X.v[b0 + i], ld(X.v, b0, i + 1)), acc);
      }
      if (own_uzl) emit(O.l, B.l, at, acc);
    }
    // mu row
    if (own_vm) emit(O.m, B.m, at, xu - xv);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_apply_dense(LevelView<T> L, const T *__restrict__ x,
                                                     const T *__restrict__ b, T *out, const int *guard = nullptr,
                                                     int j0 = 0, int j1 = -1, T *xcopy = nullptr,
                                                     const int *xcopy_idx = nullptr, int xcopy_shift = 0) {
  if (guard && *guard == 0) return;
  const int n = L.n, p = L.p, q = L.q;
  const int t = max(j0 - 1, 0) + blockIdx.x * blockDim.x + threadIdx.x;  // as k_apply_tri
  const int tend = j1 < 0 ? n : min(j1, n);
  if (t >= tend) return;
  const bool own_uzl = t >= j0, own_vm = t + 1 >= j0 && (j1 < 0 || t + 1 < j1);
  Vec<const T> X = make_cvec(x, n, p, q);
  Vec<T> O = make_vec(out, n, p, q);
  Vec<const T> B = make_cvec(b ? b : x, n, p, q);
  const T *N = L.N + t * L.sN, *Z = L.Z + t * L.sZ;
  const T sgn = b ? T(-1) : T(1);
  const T *xu = X.u + (long long)t * p, *xv = X.v + (long long)t * p, *xz = X.z + (long long)t * q;
  const T *xl = X.l + (long long)t * p, *xm = X.m + (long long)t * p;
  if (T *cp = copy_slot(xcopy, xcopy_idx, xcopy_shift, n, p, q)) {
    Vec<T> Cv = make_vec(cp, n, p, q);
    for (int i = 0; i < p; ++i) {
      Cv.u[(long long)t * p + i] = xu[i];
      Cv.v[(long long)t * p + i] = xv[i];
      Cv.l[(long long)t * p + i] = xl[i];
      Cv.m[(long long)t * p + i] = xm[i];
    }
    for (int i = 0; i < q; ++i) Cv.z[(long long)t * q + i] = xz[i];
  }
  T acc[kDenseMax];
  // u row
  for (int i = 0; i < p; ++i) acc[i] = xu[i] + xm[i];
  dn_mtv<T>(acc, N, xl, p, p, T(1), true);
  if (own_uzl)
    for (int i = 0; i < p; ++i)
      O.u[(long long)t * p + i] = b ? fma(sgn, acc[i], B.u[(long long)t * p + i]) : acc[i];
  // v row
  for (int i = 0; i < p; ++i) acc[i] = xv[i] - xm[i];
  if (t + 1 < n) dn_mtv<T>(acc, L.V + (t + 1) * L.sV, X.l + (long long)(t + 1) * p, p, p, T(1), true);
  if (own_vm)
    for (int i = 0; i < p; ++i)
      O.v[(long long)t * p + i] = b ? fma(sgn, acc[i], B.v[(long long)t * p + i]) : acc[i];
  // z row
  for (int i = 0; i < q; ++i) acc[i] = xz[i];
  dn_mtv<T>(acc, Z, xl, p, q, T(1), true);
  if (own_uzl)
    for (int i = 0; i < q; ++i)
      O.z[(long long)t * q + i] = b ? fma(sgn, acc[i], B.z[(long long)t * q + i]) : acc[i];
  // lambda row
  dn_mv<T>(acc, N, xu, p, p, T(1), false);
  dn_mv<T>(acc, Z, xz, p, q, T(1), true);
  if (t >= 1) dn_mv<T>(acc, L.V + t * L.sV, X.v + (long long)(t - 1) * p, p, p, T(1), true);
  if (own_uzl)
    for (int i = 0; i < p; ++i)
      O.l[(long long)t * p + i] = b ? fma(sgn, acc[i], B.l[(long long)t * p + i]) : acc[i];
  // mu row
  if (own_vm)
    for (int i = 0; i < p; ++i) {
      T d = xu[i] - xv[i];
      O.m[(long long)t * p + i] = b ? fma(sgn, d, B.m[(long long)t * p + i]) : d;
    }
}

// out = b - A~ x (b non-null) or A~ x on the rows of blocks [j0, j1), dense
// blocks up to 32: one warp per step (as k_apply_dense's rows)
template <typename T>
__global__ void __launch_bounds__(128) k_apply_dw(LevelView<T> L, const T *__restrict__ x, const T *__restrict__ b,
                                                  T *out, const int *guard = nullptr, int j0 = 0, int j1 = -1,
                                                  T *xcopy = nullptr, const int *xcopy_idx = nullptr,
                                                  int xcopy_shift = 0) {
  if (guard && *guard == 0) return;
  const int ln = threadIdx.x & (kWarp - 1);
  const int n = L.n, p = L.p, q = L.q;
  const int t = max(j0 - 1, 0) + (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int tend = j1 < 0 ? n : min(j1, n);
  if (t >= tend) return;
  const bool own_uzl = t >= j0, own_vm = t + 1 >= j0 && (j1 < 0 || t + 1 < j1);
  Vec<const T> X = make_cvec(x, n, p, q);
  Vec<T> O = make_vec(out, n, p, q);
  Vec<const T> B = make_cvec(b ? b : x, n, p, q);
  const T *N = L.N + t * L.sN, *Z = L.Z + t * L.sZ;
  const T xu = dw_load(X.u + (long long)t * p, p, ln), xv = dw_load(X.v + (long long)t * p, p, ln);
  const T xz = dw_load(X.z + (long long)t * q, q, ln), xl = dw_load(X.l + (long long)t * p, p, ln);
  const T xm = dw_load(X.m + (long long)t * p, p, ln);
  if (T *cp = copy_slot(xcopy, xcopy_idx, xcopy_shift, n, p, q)) {
    Vec<T> Cv = make_vec(cp, n, p, q);
    if (ln < p) {
      Cv.u[(long long)t * p + ln] = xu;
      Cv.v[(long long)t * p + ln] = xv;
      Cv.l[(long long)t * p + ln] = xl;
      Cv.m[(long long)t * p + ln] = xm;
    }
    if (ln < q) Cv.z[(long long)t * q + ln] = xz;
  }
  auto put = [&](T *dst, const T *bsrc, T row, int len) {
    if (ln < len) dst[ln] = b ? bsrc[ln] - row : row;
  };
  const T ru = xu + xm + dw_mtv(N, xl, p, p, ln);
  T rv = xv - xm;
  if (t + 1 < n) rv += dw_mtv(L.V + (t + 1) * L.sV, dw_load(X.l + (long long)(t + 1) * p, p, ln), p, p, ln);
  const T rz = xz + dw_mtv(Z, xl, p, q, ln);
  T rl = dw_mv(N, xu, p, p, ln) + dw_mv(Z, xz, p, q, ln);
  if (t >= 1) rl += dw_mv(L.V + t * L.sV, dw_load(X.v + (long long)(t - 1) * p, p, ln), p, p, ln);
  const T rmu = xu - xv;
  if (own_uzl) {
    put(O.u + (long long)t * p, B.u + (long long)t * p, ru, p);
    put(O.z + (long long)t * q, B.z + (long long)t * q, rz, q);
    put(O.l + (long long)t * p, B.l + (long long)t * p, rl, p);
  }
  if (own_vm) {
    put(O.v + (long long)t * p, B.v + (long long)t * p, rv, p);
    put(O.m + (long long)t * p, B.m + (long long)t * p, rmu, p);
  }
}

// residual restricted by the variable formulas (as k_residual_restrict_dense), dense blocks up to 32:
// one warp per coarse step
template <typename T>
__global__ void __launch_bounds__(128) k_residual_restrict_dw(LevelView<T> L, const T *__restrict__ y,
                                                              const T *__restrict__ b, T *rc) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int K = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int n = L.n, p = L.p, q = L.q, nc = n / 2;
  if (K >= nc) return;
  const int t0 = 2 * K, t1 = 2 * K + 1;
  Vec<const T> Y = make_cvec(y, n, p, q);
  Vec<const T> B = make_cvec(b, n, p, q);
  Vec<T> R = make_vec(rc, nc, p, q);
  const T *N0 = L.N + t0 * L.sN, *Z0 = L.Z + t0 * L.sZ, *Z1 = L.Z + t1 * L.sZ;
  const T yu = dw_load(Y.u + (long long)t0 * p, p, ln), yv = dw_load(Y.v + (long long)t0 * p, p, ln);
  const T yz = dw_load(Y.z + (long long)t0 * q, q, ln), yl = dw_load(Y.l + (long long)t0 * p, p, ln);
  const T ym = dw_load(Y.m + (long long)t0 * p, p, ln);
  const T yl1 = dw_load(Y.l + (long long)t1 * p, p, ln), yz1 = dw_load(Y.z + (long long)t1 * q, q, ln);
  const T ru = yu + ym + dw_mtv(N0, yl, p, p, ln);
  T rl = dw_mv(N0, yu, p, p, ln) + dw_mv(Z0, yz, p, q, ln);
  if (t0 >= 1) rl += dw_mv(L.V + t0 * L.sV, dw_load(Y.v + (long long)(t0 - 1) * p, p, ln), p, p, ln);
  const T rz0 = yz + dw_mtv(Z0, yl, p, q, ln), rz1 = yz1 + dw_mtv(Z1, yl1, p, q, ln);
  const T rv = yv - ym + dw_mtv(L.V + t1 * L.sV, yl1, p, p, ln);
  if (ln < p) {
    R.u[(long long)K * p + ln] = B.u[(long long)t0 * p + ln] - ru;
    R.m[(long long)K * p + ln] = B.m[(long long)t0 * p + ln] - (yu - yv);
    R.l[(long long)K * p + ln] = B.l[(long long)t0 * p + ln] - rl;
    R.v[(long long)K * p + ln] = B.v[(long long)t0 * p + ln] - rv;
  }
  if (ln < q)
    R.z[(long long)K * q + ln] = T(0.5) * ((B.z[(long long)t0 * q + ln] - rz0) + (B.z[(long long)t1 * q + ln] - rz1));
}

// ---------------------------------------------------------------------------
// Residual restricted to the coarse grid (Alg. 1, Sec. 5.3.1):
//   rc_x[K] = r_x[2K]                     (x = u, v, lambda, mu: injection)
//   rc_z[K] = (r_z[2K] + r_z[2K+1]) / 2   (control: average)
// with r = b - A~ y evaluated only at the rows it needs.

template <typename T, int C, typename CT = T>
__global__ void __launch_bounds__(128) k_residual_restrict_tri(LevelView<T, CT> L, const T *__restrict__ y,
                                                               const T *__restrict__ b, T *rc) {
  const int ln = threadIdx.x & (kWarp - 1);
  const int K = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int n = L.n, p = L.p, q = L.q, nc = n / 2;
  if (K >= nc) return;
  const int t0 = 2 * K, t1 = 2 * K + 1;
  Vec<const T> Y = make_cvec(y, n, p, q);
  Vec<const T> B = make_cvec(b, n, p, q);
  Vec<T> R = make_vec(rc, nc, p, q);
  const CT *N0 = L.N + t0 * L.sN, *Z0 = L.Z + t0 * L.sZ, *Z1 = L.Z + t1 * L.sZ;
  T yu[C], yv[C], yz[C], yl[C], ym[C], acc[C], o[C];
  chunk_load<T, C>(yu, Y.u + (long long)t0 * p, p, ln);
  chunk_load<T, C>(yv, Y.v + (long long)t0 * p, p, ln);
  chunk_load<T, C>(yz, Y.z + (long long)t0 * q, q, ln);
  chunk_load<T, C>(yl, Y.l + (long long)t0 * p, p, ln);
  chunk_load<T, C>(ym, Y.m + (long long)t0 * p, p, ln);
  // u row at t0
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = yu[e] + ym[e];
  tri_mtv<T, C, true>(acc, N0, yl, p, ln, T(1));
  chunk_load<T, C>(o, B.u + (long long)t0 * p, p, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) o[e] -= acc[e];
  chunk_store<T, C>(R.u + (long long)K * p, o, p, ln);
  // mu row at t0
  chunk_load<T, C>(o, B.m + (long long)t0 * p, p, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) o[e] -= yu[e] - yv[e];
  chunk_store<T, C>(R.m + (long long)K * p, o, p, ln);
  // lambda row at t0
  tri_mv<T, C, false>(acc, N0, yu, p, ln, T(1));
  tri_mv<T, C, true>(acc, Z0, yz, p, ln, T(1));
  if (t0 >= 1) {
    T yv0[C];
    chunk_load<T, C>(yv0, Y.v + (long long)(t0 - 1) * p, p, ln);
    tri_mv<T, C, true>(acc, L.V + t0 * L.sV, yv0, p, ln, T(1));
  }
  chunk_load<T, C>(o, B.l + (long long)t0 * p, p, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) o[e] -= acc[e];
  chunk_store<T, C>(R.l + (long long)K * p, o, p, ln);
  // z rows at t0 and t1, averaged
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = yz[e];
  tri_mtv<T, C, true>(acc, Z0, yl, p, ln, T(1));
  chunk_load<T, C>(o, B.z + (long long)t0 * q, q, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) o[e] -= acc[e];
  T yl1[C], yz1[C], b1[C];
  chunk_load<T, C>(yl1, Y.l + (long long)t1 * p, p, ln);
  chunk_load<T, C>(yz1, Y.z + (long long)t1 * q, q, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = yz1[e];
  tri_mtv<T, C, true>(acc, Z1, yl1, p, ln, T(1));
  chunk_load<T, C>(b1, B.z + (long long)t1 * q, q, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) o[e] = T(0.5) * (o[e] + (b1[e] - acc[e]));
  chunk_store<T, C>(R.z + (long long)K * q, o, q, ln);
  // v row at t0: v + V_{t0+1}^T l_{t0+1} - mu   (t0 + 1 = t1 <= n - 1)
#pragma unroll
  for (int e = 0; e < C; ++e) acc[e] = yv[e] - ym[e];
  tri_mtv<T, C, true>(acc, L.V + t1 * L.sV, yl1, p, ln, T(1));
  chunk_load<T, C>(o, B.v + (long long)t0 * p, p, ln);
#pragma unroll
  for (int e = 0; e < C; ++e) o[e] -= acc[e];
  chunk_store<T, C>(R.v + (long long)K * p, o, p, ln);
}

template <typename T>
__global__ void __launch_bounds__(128) k_residual_restrict_dense(LevelView<T> L, const T *__restrict__ y,
                                                                 const T *__restrict__ b, T *rc) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = L.n, p = L.p, q = L.q, nc = n / 2;
  if (K >= nc) return;
  const int t0 = 2 * K, t1 = 2 * K + 1;
  Vec<const T> Y = make_cvec(y, n, p, q);
  Vec<const T> B = make_cvec(b, n, p, q);
  Vec<T> R = make_vec(rc, nc, p, q);
  const T *N0 = L.N + t0 * L.sN, *Z0 = L.Z + t0 * L.sZ, *Z1 = L.Z + t1 * L.sZ;
  const T *yu = Y.u + (long long)t0 * p, *yv = Y.v + (long long)t0 * p, *yz = Y.z + (long long)t0 * q;
  const T *yl = Y.l + (long long)t0 * p, *ym = Y.m + (long long)t0 * p;
  const T *yl1 = Y.l + (long long)t1 * p, *yz1 = Y.z + (long long)t1 * q;
  T acc[kDenseMax], acc1[kDenseMax];
  for (int i = 0; i < p; ++i) acc[i] = yu[i] + ym[i];
  dn_mtv<T>(acc, N0, yl, p, p, T(1), true);
  for (int i = 0; i < p; ++i) R.u[(long long)K * p + i] = B.u[(long long)t0 * p + i] - acc[i];
  for (int i = 0; i < p; ++i) R.m[(long long)K * p + i] = B.m[(long long)t0 * p + i] - (yu[i] - yv[i]);
  dn_mv<T>(acc, N0, yu, p, p, T(1), false);
  dn_mv<T>(acc, Z0, yz, p, q, T(1), true);
  if (t0 >= 1) dn_mv<T>(acc, L.V + t0 * L.sV, Y.v + (long long)(t0 - 1) * p, p, p, T(1), true);
  for (int i = 0; i < p; ++i) R.l[(long long)K * p + i] = B.l[(long long)t0 * p + i] - acc[i];
  for (int i = 0; i < q; ++i) acc[i] = yz[i];
  dn_mtv<T>(acc, Z0, yl, p, q, T(1), true);
  for (int i = 0; i < q; ++i) acc1[i] = yz1[i];
  dn_mtv<T>(acc1, Z1, yl1, p, q, T(1), true);
  for (int i = 0; i < q; ++i)
    R.z[(long long)K * q + i] = T(0.5) * ((B.z[(long long)t0 * q + i] - acc[i]) +
                                          (B.z[(long long)t1 * q + i] - acc1[i]));
  for (int i = 0; i < p; ++i) acc[i] = yv[i] - ym[i];
  dn_mtv<T>(acc, L.V + t1 * L.sV, yl1, p, p, T(1), true);
  for (int i = 0; i < p; ++i) R.v[(long long)K * p + i] = B.v[(long long)t0 * p + i] - acc[i];
}

// ---------------------------------------------------------------------------
// Transfers between a level and the next coarser one (Sec. 5.3.1), in the
// type-major layout.  Each CTA works on whole coarse time steps: with
// tpk = transfer_threads(w) threads per step, thread e of a step handles
// access e, e + tpk, ... of the step's w = (4p + q) / VW vector accesses (the
// five types decoded by comparisons, 32-bit offsets within a type), so a warp
// reads and writes contiguous runs of one type and no thread divides a 64-bit
// index.
//
// Ownership of a vector entry by a range of time blocks [j0, j1) (j1 < 0: all):
// block j holds u, z, lambda of step j and v, mu of step j - 1.
__device__ __forceinline__ bool coarse_owned(bool vm, int K, int K0, int K1) {
  const int blk = vm ? K + 1 : K;
  return blk >= K0 && (K1 < 0 || blk < K1);
}

// entry e (< 4p + q) of a time step: its type (0 u, 1 v, 2 z, 3 lambda, 4 mu)
// and its index i within the type
__device__ __forceinline__ int entry_type(int e, int p, int q, int &i) {
  if (e < p) { i = e; return 0; }
  if (e < 2 * p) { i = e - p; return 1; }
  if (e < 2 * p + q) { i = e - 2 * p; return 2; }
  if (e < 3 * p + q) { i = e - 2 * p - q; return 3; }
  i = e - 3 * p - q;
  return 4;
}

// offset of type ty's block in a type-major vector of n steps
// (u 0, v np, z 2np, lambda 2np + nq, mu 3np + nq)
__device__ __forceinline__ long long type_offset(int ty, int n, int p, int q) {
  const long long np = (long long)n * p;
  return ty < 3 ? ty * np : 2 * np + (long long)n * q + (ty - 3) * np;
}

// threads per coarse step of the transfer kernels for steps of w vector
// accesses: one warp-multiple covering them, at most the CTA (256 threads)
inline __host__ __device__ int transfer_threads(int w) {
  const int t = (w + 31) / 32 * 32;
  return t < 256 ? t : 256;
}

// VW consecutive entries of one type as one access: VW = 2 loads and stores
// pairs (16 bytes in FP64), which needs p and q even and vectors aligned to a
// pair (pairs then never straddle two types); VW = 1 is the scalar form.  The
// arithmetic is per entry either way.
template <typename T, int VW>
struct TVec;
template <>
struct TVec<double, 1> { typedef double type; };
template <>
struct TVec<float, 1> { typedef float type; };
template <>
struct TVec<double, 2> { typedef double2 type; };
template <>
struct TVec<float, 2> { typedef float2 type; };

template <typename T, int VW>
__device__ __forceinline__ typename TVec<T, VW>::type tv_load(const T *p) {
  return *reinterpret_cast<const typename TVec<T, VW>::type *>(p);
}
template <typename T, int VW>
__device__ __forceinline__ void tv_store(T *p, typename TVec<T, VW>::type v) {
  *reinterpret_cast<typename TVec<T, VW>::type *>(p) = v;
}
// entry k of a vector access
__device__ __forceinline__ double &tv_at(double &v, int) { return v; }
__device__ __forceinline__ float &tv_at(float &v, int) { return v; }
__device__ __forceinline__ double &tv_at(double2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float &tv_at(float2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ double tv_at(const double &v, int) { return v; }
__device__ __forceinline__ float tv_at(const float &v, int) { return v; }
__device__ __forceinline__ double tv_at(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float tv_at(const float2 &v, int k) { return k == 0 ? v.x : v.y; }

// y += P e: u, v, lambda, mu linear (x_f[2K] = e[K], x_f[2K+1] = (e[K] +
// e[K+1]) / 2, the last odd point by end_rule: e[K] for 0, e[K] / 2 for 1);
// z piecewise constant (x_f[2K] = x_f[2K+1] = e[K]).  (j0, j1): add only to
// the entries of fine time blocks [j0, j1); j1 < 0: every entry.  n is even.
template <typename T, int VW = 1>
__global__ void __launch_bounds__(256) k_prolong_add(T *y, const T *__restrict__ e, int n, int p, int q,
                                                     int end_rule, int j0 = 0, int j1 = -1) {
  const int nc = n / 2, w = (4 * p + q) / VW, tpk = transfer_threads(w), kpb = blockDim.x / tpk;
  const int sub = threadIdx.x / tpk, lane = threadIdx.x - sub * tpk;
  if (sub >= kpb) return;
  for (int K = blockIdx.x * kpb + sub; K < nc; K += gridDim.x * kpb) {
    for (int ent = lane; ent < w; ent += tpk) {
      int i;
      const int ty = entry_type(ent * VW, p, q, i);
      const int width = ty == 2 ? q : p;
      const bool vm = ty == 1 || ty == 4;
      const T *ec = e + type_offset(ty, nc, p, q) + i;
      T *yf = y + type_offset(ty, n, p, q) + i;
      const auto e0 = tv_load<T, VW>(ec + (long long)K * width);
      if (coarse_owned(vm, 2 * K, j0, j1)) {
        T *dst = yf + (long long)(2 * K) * width;
        auto a = tv_load<T, VW>(dst);
#pragma unroll
        for (int k = 0; k < VW; ++k) tv_at(a, k) += tv_at(e0, k);
        tv_store<T, VW>(dst, a);
      }
      if (coarse_owned(vm, 2 * K + 1, j0, j1)) {
        typename TVec<T, VW>::type e1 = e0;
        const bool interior = ty != 2 && K + 1 < nc;
        if (interior) e1 = tv_load<T, VW>(ec + (long long)(K + 1) * width);
        T *dst = yf + (long long)(2 * K + 1) * width;
        auto a = tv_load<T, VW>(dst);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
          T add;
          if (ty == 2) add = tv_at(e0, k);
          else if (interior) add = T(0.5) * (tv_at(e0, k) + tv_at(e1, k));
          else add = end_rule == 0 ? tv_at(e0, k) : T(0.5) * tv_at(e0, k);
          tv_at(a, k) += add;
        }
        tv_store<T, VW>(dst, a);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Residual restriction by the transpose of the interpolation, R = P^T (the
// residual is a dual vector: it lives in the rows of A~).  With k_prolong_add's
// P, per coarse step K (0-based, nc = n / 2):
//   u, v, lambda, mu:  rc[K] = r[2K] + w r[2K+1] + (K >= 1 ? r[2K-1] / 2 : 0),
//                      w = 1/2, except at K = nc - 1 where w is the end rule's
//                      weight (1 for end_rule 0, 1/2 for end_rule 1)
//   z:                 rc[K] = r[2K] + r[2K+1]
// r is the full fine residual b - A~ y (k_apply_*).  (K0, K1): write only the
// entries of coarse time blocks [K0, K1).
template <typename T, int VW = 1>
__global__ void __launch_bounds__(256) k_restrict_transpose(const T *__restrict__ r, T *__restrict__ rc, int n,
                                                            int p, int q, int end_rule, int K0 = 0, int K1 = -1) {
  const int nc = n / 2, w = (4 * p + q) / VW, tpk = transfer_threads(w), kpb = blockDim.x / tpk;
  const int sub = threadIdx.x / tpk, lane = threadIdx.x - sub * tpk;
  if (sub >= kpb) return;
  for (int K = blockIdx.x * kpb + sub; K < nc; K += gridDim.x * kpb) {
    const T wr = (K + 1 < nc || end_rule != 0) ? T(0.5) : T(1);
    for (int ent = lane; ent < w; ent += tpk) {
      int i;
      const int ty = entry_type(ent * VW, p, q, i);
      if (!coarse_owned(ty == 1 || ty == 4, K, K0, K1)) continue;
      const int width = ty == 2 ? q : p;
      const T *rf = r + type_offset(ty, n, p, q) + i;
      const auto r0 = tv_load<T, VW>(rf + (long long)(2 * K) * width);
      const auto r1 = tv_load<T, VW>(rf + (long long)(2 * K + 1) * width);
      typename TVec<T, VW>::type acc;
      if (ty == 2) {
#pragma unroll
        for (int k = 0; k < VW; ++k) tv_at(acc, k) = tv_at(r0, k) + tv_at(r1, k);
      } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) tv_at(acc, k) = fma(wr, tv_at(r1, k), tv_at(r0, k));
        if (K >= 1) {
          const auto rm = tv_load<T, VW>(rf + (long long)(2 * K - 1) * width);
#pragma unroll
          for (int k = 0; k < VW; ++k) tv_at(acc, k) = fma(T(0.5), tv_at(rm, k), tv_at(acc, k));
        }
      }
      tv_store<T, VW>(rc + type_offset(ty, nc, p, q) + (long long)K * width + i, acc);
    }
  }
}

// Restriction of a given fine residual by the variable formulas of Sec. 5.3.1
// (injection at fine step 2K, average of z over 2K, 2K + 1), for the time-range
// entry points (the V-cycle itself fuses it with the residual:
// k_residual_restrict_*).  (K0, K1) as k_restrict_transpose.
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_inject(const T *__restrict__ r, T *__restrict__ rc, int n, int p,
                                                         int q, int K0, int K1) {
  const int nc = n / 2, w = 4 * p + q, tpk = transfer_threads(w), kpb = blockDim.x / tpk;
  const int sub = threadIdx.x / tpk, lane = threadIdx.x - sub * tpk;
  if (sub >= kpb) return;
  for (int K = blockIdx.x * kpb + sub; K < nc; K += gridDim.x * kpb) {
    for (int ent = lane; ent < w; ent += tpk) {
      int i;
      const int ty = entry_type(ent, p, q, i);
      if (!coarse_owned(ty == 1 || ty == 4, K, K0, K1)) continue;
      const int width = ty == 2 ? q : p;
      const T *rf = r + type_offset(ty, n, p, q) + i;
      const T r0 = rf[(long long)(2 * K) * width];
      rc[type_offset(ty, nc, p, q) + (long long)K * width + i] =
          ty == 2 ? T(0.5) * (r0 + rf[(long long)(2 * K + 1) * width]) : r0;
    }
  }
}

// ---------------------------------------------------------------------------
// SGS (Sec. 5.3.4) as two serial affine chains on the coarsest grid.  With
// w = (D + L)^-1 r and y = (D + L^T)^-1 D w, only u(w) carries the forward
// dependence and only mu(y) the backward one:
//   u_j  = uhat_j - Cu_j u_{j-1},      Cu_j = N_j^T S_j^-1 V_j   (j = 1..n-1)
//   mu_{j-1} = muhat_{j-1} - Em_j mu_j, Em_j = V_j^T S_j^-1 N_j  (j = n-1..1)
// where uhat, muhat come from independent local solves.  One CTA walks the
// chain; thread i owns row i, the previous link's vector lives in shared memory.
template <typename T>
__global__ void k_chain_forward(const T *__restrict__ Cu, const T *__restrict__ uhat, T *uout,
                                int n, int p) {
  extern __shared__ unsigned char smem_raw[];
  T *prev = reinterpret_cast<T *>(smem_raw);
  const int i = threadIdx.x;
  if (i < p) {
    T v0 = uhat[i];
    uout[i] = v0;
    prev[i] = v0;
  }
  __syncthreads();
  for (int j = 1; j < n; ++j) {
    T acc = T(0);
    if (i < p) {
      const T *row = Cu + ((long long)j * p + i) * p;
      acc = uhat[(long long)j * p + i];
      for (int k = 0; k < p; ++k) acc = fma(-row[k], prev[k], acc);
    }
    __syncthreads();
    if (i < p) {
      prev[i] = acc;
      uout[(long long)j * p + i] = acc;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_chain_backward(const T *__restrict__ Em, const T *__restrict__ muhat, T *mout,
                                 int n, int p) {
  extern __shared__ unsigned char smem_raw[];
  T *prev = reinterpret_cast<T *>(smem_raw);
  const int i = threadIdx.x;
  if (i < p) {
    T v0 = muhat[(long long)(n - 1) * p + i];
    mout[(long long)(n - 1) * p + i] = v0;
    prev[i] = v0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 1; --j) {
    T acc = T(0);
    if (i < p) {
      const T *row = Em + ((long long)j * p + i) * p;
      acc = muhat[(long long)(j - 1) * p + i];
      for (int k = 0; k < p; ++k) acc = fma(-row[k], prev[k], acc);
    }
    __syncthreads();
    if (i < p) {
      prev[i] = acc;
      mout[(long long)(j - 1) * p + i] = acc;
    }
    __syncthreads();
  }
}

}  // namespace pintmg

namespace pintmg {

// ---------------------------------------------------------------------------
// The same SGS chains spread over a thread-block cluster of S CTAs (one per
// SM).  Link j computes x_j = xhat_j - G_j x_{j-1} (p x p dense G_j, row-major)
// with CTA c owning rows [c R, c R + R), R = ceil(p / S).  Within a CTA, TPR
// threads share a row: each takes p / TPR consecutive columns (coalesced row
// loads), partial sums are combined with warp shuffles, and the row owner
// writes the new entry into every CTA's copy of x (distributed shared memory,
// double-buffered).  One cluster barrier per link publishes x_j.  The cluster
// barrier is the hardware barrier.cluster (all CTAs of a cluster are
// co-scheduled), reached the same number of times by every thread.
// Columns are interleaved over the TPR threads of a row so that each load
// instruction reads TPR consecutive entries of the row.
// kForward: links j = 1..n-1 on x = u; otherwise links j = n-1..1 on x = mu
// (x_{j-1} = xhat_{j-1} - G_j x_j).
// seg_len < n: each cluster (index blockIdx.x / S) runs one segment of seg_len
// chain positions from a zero incoming state (its first entry is xhat's); the
// segments are joined afterwards by k_seg_fix.  seg_len = n: the whole chain.
template <typename T, bool kForward, int K>
__global__ void k_chain_cluster(const T *__restrict__ G, const T *__restrict__ xhat, T *xout, int n, int p,
                                int rows_per_cta, int tpr, int seg_len) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);  // [2][p]
  const int S = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const int pos0 = (int)(blockIdx.x / S) * seg_len;                 // first chain position of this segment
  const int pos1 = pos0 + seg_len < n ? pos0 + seg_len : n;        // one past its last
  const int tid = threadIdx.x;
  const int row_local = tid / tpr, part = tid % tpr;
  const int row = c * rows_per_cta + row_local;
  const bool owner = (row_local < rows_per_cta) && (row < p);
  // this thread's K columns (part, part + tpr, ...) of its row for one link,
  // and the row's entry of xhat: loaded one link ahead
  T g[K];
  T xh = T(0);
  auto load_link = [&](int step) {
    if (step >= pos1 || !owner) return;
    const int j = kForward ? step : n - step;
    const long long dst = kForward ? j : (long long)(j - 1);
    const T *gr = G + ((long long)j * p + row) * p;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int k = part + i * tpr;
      g[i] = (k < p) ? gr[k] : T(0);
    }
    xh = xhat[dst * p + row];
  };
  const long long first = kForward ? pos0 : (long long)(n - 1 - pos0);
  for (int i = tid; i < p; i += blockDim.x) buf[i] = xhat[first * p + i];
  if (c == 0)
    for (int i = tid; i < p; i += blockDim.x) xout[first * p + i] = xhat[first * p + i];
#pragma unroll
  for (int i = 0; i < K; ++i) g[i] = T(0);
  load_link(pos0 + 1);
  cluster.sync();
  int cur = 0;
  for (int step = pos0 + 1; step < pos1; ++step) {
    const int j = kForward ? step : n - step;
    const long long dst = kForward ? j : (long long)(j - 1);
    const T *xv = buf + cur * p;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int k = part + i * tpr;
      if (k < p) acc = fma(g[i], xv[k], acc);
    }
    // combine the tpr partial sums of a row (lanes of a row are contiguous, tpr divides 32)
    for (int o = tpr >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o, tpr);
    const int nxt = cur ^ 1;
    if (owner && part == 0) {
      const T v = xh - acc;
      xout[dst * p + row] = v;
      for (int r = 0; r < S; ++r) {
        T *remote = cluster.map_shared_rank(buf, r);
        remote[nxt * p + row] = v;
      }
    }
    // publish x_j; the next link's loads do not depend on it and overlap the barrier
    auto token = cluster.barrier_arrive();
    load_link(step + 1);
    cluster.barrier_wait(std::move(token));
    cur = nxt;
  }
}

}  // namespace pintmg

namespace pintmg {

// ---------------------------------------------------------------------------
// Segmented chain, joining step.  After the segments' local chains (zero
// incoming state), position i of segment c >= 1 (positions [c L, c L + L))
// becomes x_i = y_i + Q_i x_{cL-1}, with Q_i = A_i ... A_{cL} (setup, column-
// major p x p per position) and x_{cL-1} the true last entry of segment c-1.
// only_seg >= 1: update only the last position of that segment (the serial
// pass over segment ends; grid (1, p / rows)); only_seg = 0: every position of
// segments >= 1 except their last (grid (n, p / rows)).  In place; rows /
// parts as in k_scan_round.  reverse: position i is stored at index n-1-i.
template <typename T>
__global__ void k_seg_fix(const T *__restrict__ Q, T *x, int n, int p, int L, int only_seg, int reverse, int parts,
                          int rows) {
  extern __shared__ unsigned char smem_raw[];
  T *src = reinterpret_cast<T *>(smem_raw);
  T *part_sum = src + p;  // [parts][rows]
  const int r0 = blockIdx.y * rows;
  int i = blockIdx.x;
  if (only_seg > 0) i = (only_seg + 1) * L - 1 < n - 1 ? (only_seg + 1) * L - 1 : n - 1;  // that segment's last
  const int c = i / L;
  if (c == 0 || i >= n) return;
  const int last = (c + 1) * L - 1 < n - 1 ? (c + 1) * L - 1 : n - 1;
  if (only_seg == 0 && i == last) return;
  const long long si = reverse ? (long long)(n - 1 - i) : i;
  const int j = c * L - 1;
  const long long sj = reverse ? (long long)(n - 1 - j) : j;
  for (int r = threadIdx.x; r < p; r += blockDim.x) src[r] = x[sj * p + r];
  __syncthreads();
  const T *Qi = Q + (long long)i * p * p + r0;
  const int r = threadIdx.x % rows, part = threadIdx.x / rows;
  if (part < parts) {
    const int k0 = part * p / parts, k1 = (part + 1) * p / parts;
    T acc = T(0);
#pragma unroll 8
    for (int k = k0; k < k1; ++k) acc = fma(Qi[(long long)k * p + r], src[k], acc);
    part_sum[part * rows + r] = acc;
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < rows; rr += blockDim.x) {
    T acc = x[si * p + r0 + rr];
    for (int q = 0; q < parts; ++q) acc += part_sum[q * rows + rr];
    x[si * p + r0 + rr] = acc;
  }
}

// ---------------------------------------------------------------------------
// SGS chains as a parallel scan in time.  A chain x_i = xhat_i + A_i x_{i-1}
// (i = 1..n-1, x_0 = xhat_0) is a linear recurrence; with the prefix products
// P^(d)_i = A_i A_{i-1} ... A_{i-2^d+1} (precomputed at setup, column-major
// p x p), a Kogge-Stone scan runs ceil(log2 n) rounds of
//     x_i <- x_i + P^(d)_i x_{i-2^d}      (i >= 2^d; others copied)
// each a batched GEMV over every time step at once.  Element i is stored at
// position i (forward chain) or n-1-i (backward chain, reverse = 1).
// CTA (i, slice) computes `rows` rows of step i (all p rows when rows = p;
// slices of 32 rows spread a round over more CTAs than there are steps, which
// balances the SMs when n is a few hundred); threads (r, part) with
// r = tid mod rows share row r over `parts` column slices (coalesced
// column-major loads, more loads in flight), the source vector x_{i-2^d} and
// the slice sums are staged in shared memory.  Grid: (n, p / rows).
template <typename T>
__global__ void k_scan_round(const T *__restrict__ Pd, const T *__restrict__ xin, T *xout, int n, int p,
                             int shift, int reverse, int parts, int rows) {
  extern __shared__ unsigned char smem_raw[];
  T *src = reinterpret_cast<T *>(smem_raw);
  T *part_sum = src + p;  // [parts][rows]
  const int i = blockIdx.x, r0 = blockIdx.y * rows;
  const long long si = reverse ? (long long)(n - 1 - i) : i;
  if (i < shift) {
    for (int r = threadIdx.x; r < rows; r += blockDim.x) xout[si * p + r0 + r] = xin[si * p + r0 + r];
    return;
  }
  const long long sj = reverse ? (long long)(n - 1 - (i - shift)) : (long long)(i - shift);
  for (int r = threadIdx.x; r < p; r += blockDim.x) src[r] = xin[sj * p + r];
  __syncthreads();
  const T *P = Pd + (long long)i * p * p + r0;
  const int r = threadIdx.x % rows, part = threadIdx.x / rows;
  if (part < parts) {
    const int k0 = part * p / parts, k1 = (part + 1) * p / parts;
    T acc = T(0);
#pragma unroll 8
    for (int k = k0; k < k1; ++k) acc = fma(P[(long long)k * p + r], src[k], acc);
    part_sum[part * rows + r] = acc;
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < rows; rr += blockDim.x) {
    T acc = xin[si * p + r0 + rr];
    for (int q = 0; q < parts; ++q) acc += part_sum[q * rows + rr];
    xout[si * p + r0 + rr] = acc;
  }
}

}  // namespace pintmg
