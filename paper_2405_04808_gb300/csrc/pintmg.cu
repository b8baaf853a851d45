// Host side of the pintmg C ABI (include/pintmg.h): hierarchy setup, the
// V-cycle of Alg. 1, the coarse GMRES with SGS (Sec. 5.3.4) and the outer
// flexible GMRES (Saad 1993).  Every arithmetic step runs in the kernels of
// vcycle_kernels.cuh, setup_kernels.cuh and krylov_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "krylov_kernels.cuh"
#include "learned_kernels.cuh"
#include "pair_kernels.cuh"
#include "setup_kernels.cuh"
#include "tc_kernels.cuh"
#include "vcycle_kernels.cuh"

using namespace pintmg;

namespace {

thread_local char g_last_cuda_error[256] = "";

struct CudaFail {
  cudaError_t err;
};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
    throw CudaFail{e};
  }
}

inline void ck_launch() { ck(cudaGetLastError()); }

inline int grid_for(long long work, int threads, int cap = 4 * 152) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// CTAs of 256 threads for a transfer kernel over nc coarse steps of w vector
// accesses (transfer_threads(w) threads per step)
inline int transfer_grid(int nc, int w) {
  const int kpb = 256 / transfer_threads(w);
  const long long g = ((long long)nc + kpb - 1) / kpb;
  return (int)std::max(1LL, std::min(g, 1LL << 20));
}

// the transfer kernels move entry pairs (VW = 2) when p and q are even and
// both vectors are aligned to a pair
template <typename T>
bool transfer_pairs(int p, int q, const void *a, const void *b) {
  return p % 2 == 0 && q % 2 == 0 &&
         ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) % (2 * sizeof(T))) == 0;
}

// y += P e on a level of n (even) steps from e on the next coarser one; (j0, j1) as k_prolong_add
template <typename T>
void launch_prolong(const T *e, T *y, int n, int p, int q, int end_rule, cudaStream_t s, int j0 = 0, int j1 = -1) {
  if (transfer_pairs<T>(p, q, e, y))
    k_prolong_add<T, 2><<<transfer_grid(n / 2, (4 * p + q) / 2), 256, 0, s>>>(y, e, n, p, q, end_rule, j0, j1);
  else
    k_prolong_add<T, 1><<<transfer_grid(n / 2, 4 * p + q), 256, 0, s>>>(y, e, n, p, q, end_rule, j0, j1);
}

// rc = P^T r; (K0, K1) as k_restrict_transpose
template <typename T>
void launch_restrict_transpose(const T *r, T *rc, int n, int p, int q, int end_rule, cudaStream_t s, int K0 = 0,
                               int K1 = -1) {
  if (transfer_pairs<T>(p, q, r, rc))
    k_restrict_transpose<T, 2><<<transfer_grid(n / 2, (4 * p + q) / 2), 256, 0, s>>>(r, rc, n, p, q, end_rule, K0,
                                                                                   K1);
  else
    k_restrict_transpose<T, 1><<<transfer_grid(n / 2, 4 * p + q), 256, 0, s>>>(r, rc, n, p, q, end_rule, K0, K1);
}

// one device allocation, freed by the handle
struct DevMem {
  std::vector<void *> ptrs;
  template <typename T>
  T *alloc(size_t count) {
    void *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
      throw std::bad_alloc();
    }
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
  void release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

template <typename T>
struct LevelData {
  LevelView<T> view{};
  T *Cu = nullptr, *Em = nullptr;  // coarsest level only
  // coarsest level: prefix products of the SGS chains for the parallel scan
  // (empty when the budget below is exceeded; the cluster chain is used then)
  std::vector<T *> scanF, scanB;
  T *scan_tmp = nullptr;
  // coarsest level: in-segment products Q of the segmented SGS chains (null when not formed)
  T *segF = nullptr, *segB = nullptr;
  int seg_len = 0;
  T *b = nullptr, *y = nullptr, *tmp = nullptr;
  T *chainU = nullptr, *chainM = nullptr, *sgs_w = nullptr;
  // smoothing levels whose blocks fit on the GPU at once: all sweeps of a
  // pre- or post-smoothing in one cooperative launch (k_sweeps_tri2)
  bool persist = false;
  SweepXchg<T> sx{};
  // MG_PRECISION_BF16_BANDS, smoothing levels: the view with the N, V, Z bands in BF16
  bool bands16 = false;
  LevelView<T, __nv_bfloat16> vh{};
};

struct Level {
  int n = 0;
  double dt = 0;
  long long len = 0;
  LevelData<double> d;
  LevelData<float> f;
};

}  // namespace

// The learned coarse correction's network (weights, optimiser state, workspaces).
struct mg_net {
  float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *partial = nullptr, *loss = nullptr;
  __nv_bfloat16 *params_bf16 = nullptr;
  __nv_bfloat16 *wimg = nullptr;  // per-layer weight images of the tensor-core convolutions (mma.sync)
  __nv_bfloat16 *timg = nullptr;  // the same for the tcgen05 convolutions
  int *tc_err = nullptr;          // a bounded wait of a tcgen05 convolution ran out (standalone forward)
  bool bf16_valid = false;
  int step = 0;              // Adam's step count (bias correction)
  long long updates = 0;     // optimiser steps ever taken by this network
  // training workspace: layer outputs h[l] (l = 1..4; h[0] is the caller's input),
  // pre-activations z[l] (l = 0..2), gradient ping-pong g0/g1, a gathered minibatch
  float *h[kNetLayers + 1] = {}, *z[kNetLayers] = {}, *g0 = nullptr, *g1 = nullptr, *bx = nullptr, *by = nullptr;
  long long ws_elems = 0;  // per sample: 32 * T * X
  int ws_batch = 0;
  // standalone inference workspace (mg_net_forward): ping-pong activations and a BF16 copy of x/y
  void *ia = nullptr, *ib = nullptr, *ic = nullptr;
  long long inf_bytes = 0;
  float *wt = nullptr;                 // flipped, transposed weights of one layer (input gradient)
  float *wpart = nullptr, *bpart = nullptr;  // weight / bias gradient partial sums
  float *sx = nullptr, *sy = nullptr;  // per-channel input / target scales of a normalised training run
  double *spart = nullptr;             // their partial sums
  int *order = nullptr;  // minibatch gather indices (device)
  int order_cap = 0;
  // residual-metric loss (mg_net_set_metric): the coarse operator of this handle (not owned)
  // and the loss's FP64 workspace (two minibatch-sized vectors, then partial sums and the total)
  mg_handle *metric = nullptr;
  double *mws = nullptr;
  long long mws_n = 0;
  DevMem mem, ws;        // mem: fixed buffers; ws: workspaces (reallocated when they grow)
};

struct mg_handle {
  mg_options opts{};
  int layout = 0, n = 0, p = 0, q = 0, C = 1;
  double theta = 0, gamma = 0;
  std::vector<Level> lv;
  DevMem mem;
  // coarse GMRES (FP64) workspace
  int cmax = 0;
  double *cV = nullptr, *cZ = nullptr, *cw = nullptr, *cr = nullptr, *cy = nullptr;
  // fine FGMRES (FP64) workspace, grown on demand
  int fm = 0;
  double *fV = nullptr, *fZ = nullptr, *fw = nullptr, *fr = nullptr;
  double *fx_stage = nullptr, *fb_stage = nullptr;
  std::vector<void *> fmem;
  // Arnoldi state of the outer FGMRES (kf) and of the coarse GMRES (kc): the
  // coarse solve runs inside every outer iteration, so they never share.
  struct Krylov {
    double *h = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *ycoef = nullptr,
           *scal = nullptr, *nrm2 = nullptr;
  } kf, kc;
  double *partial = nullptr;  // dot-product partial sums (used transiently)
  int *flag = nullptr;
  double *host_scal = nullptr;  // pinned, 4 doubles
  int ldh = 0;
  int G = 304;                  // CTAs of the dot-product kernels
  // counters of the last solve
  int vcycles = 0, coarse_iters = 0;
  int use_cluster = 1;  // SGS chains on a thread-block cluster (tridiagonal layout)
  int use_scan = 1;     // SGS chains as a parallel scan with precomputed prefix products
  int use_seg = 1;      // SGS chains as concurrent segment chains joined by batched products
  int dot_vb = 8;       // basis vectors per CTA of the blocked dot products (4, 8 or 16; same arithmetic)
  int stage_tri = 1;    // block solves read their coefficients from shared memory (staged by cp.async)
  int pair_tri = 1;     // levels with few blocks: two warps per block
  int split_bs = 1;     // p > 128: the block solve in three launches (PINTMG_SPLIT_BS=0: one warp per block)
  // per level (keyed by its number of time steps): the block-solve mapping the autotuner
  // chose, 1 = one warp per block, 2 = two warps per block; absent: the size rule
  std::map<int, int> bs_map;
  int pair_basis = 0;   // the FGMRES basis as FP32 pairs with compensated dot products (MG_BASIS_PAIR)
  int dcgs2 = 0;        // ... orthogonalised by delayed reorthogonalisation (MG_BASIS_PAIR_DCGS2)
  double *fu = nullptr;   // DCGS2: FP64 copy of the tentative basis vector (unnormalised)
  double *dcg = nullptr;  // DCGS2: coefficients, pending Hessenberg column, scalars (kDc* offsets)
  int pair_stall = 0;   // failure-detection tests: the streamed multi-dot issues no copies (its waits run out)
  int device = -1;      // the CUDA device current at mg_setup; every device buffer of the handle lives there
  int persist_sweeps = 0;  // smoothing levels that fit on the GPU run all their sweeps in one launch
                           // (off by default: no faster than one launch per sweep in a captured solve)
  int sweep_stall = 0;     // failure-detection tests: the multi-sweep kernel's block 0 publishes nothing
  int fuse_copies = 1;     // captured solves: the preconditioner input and Z_j copies ride on other kernels
  int fuse_reduce = 1;     // Krylov reductions and the Arnoldi column in the last CTA of their kernels:
                           // 0 never, 1 the Arnoldi column and dot products of <= 16 vectors, 2 always
  unsigned *ticket = nullptr;  // [0] multi-dot, [1] second axpy: CTAs finished (reset by the last one)
  // optional per-category kernel timing (CUDA events on the launch stream)
  int prof = 0;
  long long launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[16] = {};
  long long prof_count[16] = {};
  double work_bytes[16] = {}, work_flops[16] = {};  // algorithmic work of the timed launches
  // graph-captured solves (device_loops): device-resident loop state, fixed
  // preconditioner input/output slots, capture streams and the cached graph
  int capturing = 0;
  KState *kst_f = nullptr, *kst_c = nullptr;
  double *vin = nullptr, *zout = nullptr, *cvin = nullptr, *czout = nullptr;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  struct GraphKey {
    const double *b = nullptr;
    double *x = nullptr;
    double rtol = -1.0;
    int maxit = 0, restart = 0, gen = -1;
  } gkey;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long g_init = 0, g_body = 0, g_coarse = 0;  // kernel launches per region of the graph
  // learned coarse correction: network (not owned), admission threshold on the
  // residual reduction, workspaces, counters; recording of (r, y) coarse pairs
  mg_net *net = nullptr;
  double admit = 0.5;
  int net_bf16 = 1;
  void *net_x = nullptr, *net_a = nullptr, *net_b = nullptr;  // network input/output and ping-pong activations
  double *net_e = nullptr, *net_r = nullptr;
  int *net_flag = nullptr;         // [0] admitted (graph mode), [1] admitted count
  int coarse_learned = 0;          // coarse solves answered by the network in the last solve (host loops)
  float *rec_r = nullptr, *rec_y = nullptr;
  int rec_max = 0, rec_count = 0;
  int gen = 0;  // bumped when a change invalidates captured graphs (attach/detach of a network)
};

namespace {

// kernel categories reported by mg_profile_read
enum Cat { CAT_BLOCK_SOLVE = 0, CAT_APPLY, CAT_RESTRICT, CAT_PROLONG, CAT_CHAIN, CAT_DOT, CAT_AXPY, CAT_SMALL,
           CAT_CONVERT, CAT_SETUP, CAT_NET, CAT_PAIR_DOT, CAT_PAIR_AXPY, CAT_COUNT };
const char *kCatNames[CAT_COUNT] = {"block_solve", "apply", "residual_restrict", "prolong_add", "sgs_chain",
                                    "multidot", "axpy_scale", "arnoldi_scalar", "convert", "setup", "net_coarse",
                                    "pair_dot", "pair_axpy"};

cudaEvent_t take_event(mg_handle *h) {
  if (h->ev_pool.empty()) {
    cudaEvent_t e;
    ck(cudaEventCreate(&e));
    return e;
  }
  cudaEvent_t e = h->ev_pool.back();
  h->ev_pool.pop_back();
  return e;
}

// RAII bracket around one kernel launch: counts it and, when profiling, times it
struct Bracket {
  mg_handle *h;
  int cat;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Bracket(mg_handle *h_, int cat_, cudaStream_t s_, double bytes = 0.0, double flops = 0.0)
      : h(h_), cat(cat_), s(s_) {
    h->launches++;
    if (!h->capturing && ((h->prof >> cat) & 1)) {
      h->work_bytes[cat] += bytes;
      h->work_flops[cat] += flops;
      a = take_event(h);
      b = take_event(h);
      ck(cudaEventRecord(a, s));
    }
  }
  ~Bracket() noexcept(false) {
    if (a) {
      ck(cudaEventRecord(b, s));
      h->ev_pending.push_back({cat, {a, b}});
    }
  }
};

void harvest(mg_handle *h) {
  for (auto &pe : h->ev_pending) {
    ck(cudaEventSynchronize(pe.second.second));
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, pe.second.first, pe.second.second));
    h->prof_ms[pe.first] += ms;
    h->prof_count[pe.first] += 1;
    h->ev_pool.push_back(pe.second.first);
    h->ev_pool.push_back(pe.second.second);
  }
  h->ev_pending.clear();
}

// ---------------------------------------------------------------------------
// Launch helpers (templated on the V-cycle precision)

// the staged block solve applies: tridiagonal, p <= 128 (4 entries per lane), 16-byte
// aligned coefficient arrays and block strides
template <typename T, typename CT>
bool tri_stage_ok(const LevelView<T, CT> &L) {
  const auto al = [](const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0; };
  return L.layout == MG_LAYOUT_TRIDIAG && L.p <= 4 * kWarp && (3 * (size_t)L.p * sizeof(T)) % 16 == 0 &&
         (3 * (size_t)L.p * sizeof(CT)) % 16 == 0 && al(L.N) && al(L.V) && al(L.Z) && al(L.fac) && al(L.scan);
}

// levels with at most this many blocks take the two-warps-per-block solve
constexpr int kPairMaxBlocks = 4096;

// dynamic shared memory limits of the staged block solves, once per device, outside capture
void tri_stage_prepare() {
  static unsigned done = 0;
  int dev = 0;
  ck(cudaGetDevice(&dev));
  if (dev < 32 && (done >> dev) & 1u) return;
  const int bd = 4 * tri_stage_elems<double>(4 * kWarp) * (int)sizeof(double);
  const int bf = 4 * tri_stage_elems<float>(4 * kWarp) * (int)sizeof(float);
  ck(cudaFuncSetAttribute(k_block_solve_tri<double, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bd));
  ck(cudaFuncSetAttribute(k_block_solve_tri<double, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bd));
  ck(cudaFuncSetAttribute(k_block_solve_tri<double, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bd));
  ck(cudaFuncSetAttribute(k_block_solve_tri<double, 4, true, 4 * kWarp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          bd));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 4, true, 4 * kWarp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  const int pd = 2 * tri_pair_elems<double>(4 * kWarp) * (int)sizeof(double);
  const int pf = 2 * tri_pair_elems<float>(4 * kWarp) * (int)sizeof(float);
  ck(cudaFuncSetAttribute(k_block_solve_tri2<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pd));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pd));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pd));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<double, 4, 4 * kWarp>, cudaFuncAttributeMaxDynamicSharedMemorySize, pd));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 4, 4 * kWarp>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  // the same with BF16 bands (MG_PRECISION_BF16_BANDS): the same shared-memory slots
  using B16 = __nv_bfloat16;
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 1, true, 0, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 2, true, 0, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 4, true, 0, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri<float, 4, true, 4 * kWarp, B16>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, bf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 1, 0, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 2, 0, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 4, 0, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, pf));
  ck(cudaFuncSetAttribute(k_block_solve_tri2<float, 4, 4 * kWarp, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          pf));
  if (dev < 32) done |= 1u << dev;
}

template <typename T, typename CT = T>
void launch_block_solve(mg_handle *h, const LevelView<T, CT> &L, const T *r, const T *cplU, const T *cplM,
                        T *out, cudaStream_t s, const T *yold = nullptr, T omega = T(1), int j0 = 0,
                        int j1 = -1) {
  // blocks [j0, j1) of the level (all: j1 < 0)
  const int nb = (j1 < 0 ? L.n + 1 : j1) - j0;
  // per block: read r (4p+q), couplings (2p), N, V, Z (9p tridiagonal / 2p^2+pq dense), factor
  // (3p / p^2), old iterate if relaxed (4p+q); write 4p+q.  Flops: 45p (tridiagonal).
  const double w = 4.0 * L.p + L.q, p_ = L.p;
  const double coef = L.layout == MG_LAYOUT_TRIDIAG ? 9.0 * p_ * sizeof(CT) + 3.0 * p_ * sizeof(T)
                                                    : (3.0 * p_ * p_ + p_ * L.q) * sizeof(T);
  const double per_block = sizeof(T) * (2.0 * w + 2.0 * p_ + (omega != T(1) && yold ? w : 0.0)) + coef;
  const double fl = L.layout == MG_LAYOUT_TRIDIAG ? 45.0 * p_ : 2.0 * (3.0 * p_ * p_ + 2.0 * p_ * L.q + p_ * p_);
  Bracket br(h, CAT_BLOCK_SOLVE, s, per_block * nb, fl * nb);
  if (L.layout == MG_LAYOUT_DENSE) {
    if constexpr (std::is_same<T, CT>::value) {
      if (L.p > kDenseMax || L.q > kDenseMax)  // a warp per block
        k_block_solve_dw<T><<<(nb + 3) / 4, 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1);
      else
        k_block_solve_dense<T><<<grid_for(nb, 128, 1 << 30), 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0,
                                                                          j1);
    }
  } else {
    const int blocks = (nb + 3) / 4;
    const size_t smem = 4 * (size_t)tri_stage_elems<T>(L.p) * sizeof(T);
    const auto tuned = h->bs_map.find(L.n);
    const bool pair = tuned != h->bs_map.end() ? tuned->second == 2 : L.n + 1 <= kPairMaxBlocks;
    if (h->pair_tri && tri_stage_ok(L) && pair) {  // two warps per block
      const int pblocks = (nb + 1) / 2;
      const size_t psmem = 2 * (size_t)tri_pair_elems<T>(L.p) * sizeof(T);
      if (L.p == 4 * kWarp && L.q == L.p) {
        k_block_solve_tri2<T, 4, 4 * kWarp, CT><<<pblocks, 128, psmem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1);
      } else {
        switch (h->C) {
          case 1: k_block_solve_tri2<T, 1, 0, CT><<<pblocks, 128, psmem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
          case 2: k_block_solve_tri2<T, 2, 0, CT><<<pblocks, 128, psmem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
          default: k_block_solve_tri2<T, 4, 0, CT><<<pblocks, 128, psmem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
        }
      }
      ck_launch();
      return;
    }
    if (h->stage_tri && tri_stage_ok(L)) {  // coefficients staged in shared memory (p <= 128)
      if (L.p == 4 * kWarp && L.q == L.p) {  // full chunks: p known at compile time
        k_block_solve_tri<T, 4, true, 4 * kWarp, CT><<<blocks, 128, smem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1);
        ck_launch();
        return;
      }
      switch (h->C) {
        case 1: k_block_solve_tri<T, 1, true, 0, CT><<<blocks, 128, smem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
        case 2: k_block_solve_tri<T, 2, true, 0, CT><<<blocks, 128, smem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
        default: k_block_solve_tri<T, 4, true, 0, CT><<<blocks, 128, smem, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
      }
      ck_launch();
      return;
    }
    if (L.ws_rhs && h->split_bs) {  // large blocks: right-hand sides, pentadiagonal solves, outputs
      const long long ent = (long long)nb * L.p;
      const int g = grid_for(ent, 256, 1 << 20);
      k_bs_rhs<T, CT><<<g, 256, 0, s>>>(L, r, cplU, cplM, j0, j1);
      ck_launch();
      switch (h->C) {
        case 8: k_bs_penta<T, 8, CT><<<blocks, 128, 0, s>>>(L, j0, j1); break;
        default: k_bs_penta<T, 16, CT><<<blocks, 128, 0, s>>>(L, j0, j1); break;
      }
      ck_launch();
      k_bs_out<T, CT><<<g, 256, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1);
      ck_launch();
      return;
    }
    switch (h->C) {
      case 1: k_block_solve_tri<T, 1, false, 0, CT><<<blocks, 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
      case 2: k_block_solve_tri<T, 2, false, 0, CT><<<blocks, 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
      case 4: k_block_solve_tri<T, 4, false, 0, CT><<<blocks, 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
      case 8: k_block_solve_tri<T, 8, false, 0, CT><<<blocks, 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
      default: k_block_solve_tri<T, 16, false, 0, CT><<<blocks, 128, 0, s>>>(L, r, cplU, cplM, out, yold, omega, j0, j1); break;
    }
  }
  ck_launch();
}

template <typename T, typename CT = T>
void launch_apply(mg_handle *h, const LevelView<T, CT> &L, const T *x, const T *b, T *out, cudaStream_t s,
                  int j0 = 0, int j1 = -1, T *xcopy = nullptr, const int *xidx = nullptr, int xshift = 0) {
  // rows of blocks [j0, j1) (all: j1 < 0): a warp (thread) per step from max(j0 - 1, 0)
  const int steps = (j1 < 0 ? L.n : std::min(j1, L.n)) - std::max(j0 - 1, 0);
  if (steps <= 0) return;
  const double w = 4.0 * L.p + L.q;
  const double coef = L.layout == MG_LAYOUT_TRIDIAG ? 9.0 * L.p * sizeof(CT) / sizeof(T)
                                                    : 2.0 * L.p * L.p + L.p * L.q;
  Bracket br(h, CAT_APPLY, s, sizeof(T) * (L.n * ((b ? 3.0 : 2.0) * w + coef)),
             L.layout == MG_LAYOUT_TRIDIAG ? 2.0 * 18.0 * L.p * L.n : 4.0 * L.n * (2.0 * L.p * L.p + L.p * L.q));
  if (L.layout == MG_LAYOUT_DENSE) {
    if constexpr (std::is_same<T, CT>::value) {
      if (L.p > kDenseMax || L.q > kDenseMax)
        k_apply_dw<T><<<(steps + 3) / 4, 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift);
      else
        k_apply_dense<T><<<grid_for(steps, 128, 1 << 30), 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift);
    }
  } else if (L.p > 4 * kWarp && h->split_bs) {  // large blocks: a thread per (step, entry)
    k_apply_ent<T, CT><<<grid_for((long long)steps * L.p, 256, 1 << 20), 256, 0, s>>>(L, x, b, out, nullptr, j0, j1,
                                                                                    xcopy, xidx, xshift);
  } else {
    const int blocks = (steps + 3) / 4;
    switch (h->C) {
      case 1: k_apply_tri<T, 1, CT><<<blocks, 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift); break;
      case 2: k_apply_tri<T, 2, CT><<<blocks, 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift); break;
      case 4: k_apply_tri<T, 4, CT><<<blocks, 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift); break;
      case 8: k_apply_tri<T, 8, CT><<<blocks, 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift); break;
      default: k_apply_tri<T, 16, CT><<<blocks, 128, 0, s>>>(L, x, b, out, nullptr, j0, j1, xcopy, xidx, xshift); break;
    }
  }
  ck_launch();
}

// the multi-sweep kernel for this level's shape (p <= 128, two warps per block)
template <typename T>
void *sweeps_kernel(const LevelView<T> &L, int C) {
  if (L.p == 4 * kWarp && L.q == L.p) return reinterpret_cast<void *>(k_sweeps_tri2<T, 4, 4 * kWarp>);
  if (C == 1) return reinterpret_cast<void *>(k_sweeps_tri2<T, 1>);
  if (C == 2) return reinterpret_cast<void *>(k_sweeps_tri2<T, 2>);
  return reinterpret_cast<void *>(k_sweeps_tri2<T, 4>);
}

// Can every block of this smoothing level be resident at once (cooperative
// launch of k_sweeps_tri2)?  If so, allocate its coupling exchange.
template <typename T>
void prepare_sweeps(mg_handle *h, Level &lev, LevelData<T> &d, cudaStream_t s) {
  const LevelView<T> &L = d.view;
  if (!h->persist_sweeps || !h->pair_tri || L.layout != MG_LAYOUT_TRIDIAG || !tri_stage_ok(L) || h->C > 4 ||
      L.n + 1 > kPairMaxBlocks)
    return;
  int dev = 0, coop = 0, sms = 0;
  ck(cudaGetDevice(&dev));
  ck(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop) return;
  void *kern = sweeps_kernel(L, h->C);
  const size_t smem = 2 * (size_t)tri_pair_elems<T>(L.p) * sizeof(T);
  ck(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
  const long long grid = (L.n + 2) / 2;
  if ((long long)per_sm * sms < grid) return;
  const size_t xlen = 2 * (size_t)(L.n + 1) * L.p;
  d.sx.xu = h->mem.alloc<T>(xlen);
  d.sx.xm = h->mem.alloc<T>(xlen);
  d.sx.fu = h->mem.alloc<unsigned>((size_t)(L.n + 1));
  d.sx.fm = h->mem.alloc<unsigned>((size_t)(L.n + 1));
  ck(cudaMemsetAsync(d.sx.fu, 0, (size_t)(L.n + 1) * sizeof(unsigned), s));
  ck(cudaMemsetAsync(d.sx.fm, 0, (size_t)(L.n + 1) * sizeof(unsigned), s));
  d.sx.err = h->flag + 2;  // the solve's timeout flag
  d.sx.stall = h->sweep_stall;
  d.persist = true;
}

// `sweeps` block-Jacobi sweeps of a level in one cooperative launch: from y = 0
// (y0 null) or from y0, result in out (!= y0)
template <typename T>
void launch_sweeps(mg_handle *h, LevelData<T> &d, const T *r, const T *y0, T *out, int sweeps, T omega,
                   cudaStream_t s) {
  const LevelView<T> &L = d.view;
  // per block and launch: coefficients (12 p) and r (4p + q) once, y0 (4p + q) if given, y out (4p + q);
  // per sweep the two published couplings and the two read (4p).  Flops: 45 p per block and sweep
  const double w = 4.0 * L.p + L.q, p_ = L.p;
  const double per_block = sizeof(T) * (12.0 * p_ + (y0 ? 3.0 : 2.0) * w + 4.0 * p_ * (sweeps - 1));
  Bracket br(h, CAT_BLOCK_SOLVE, s, per_block * (L.n + 1), 45.0 * p_ * (L.n + 1) * sweeps);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((L.n + 2) / 2), 1, 1);
  cfg.blockDim = dim3(128, 1, 1);
  cfg.dynamicSmemBytes = 2 * (size_t)tri_pair_elems<T>(L.p) * sizeof(T);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (L.p == 4 * kWarp && L.q == L.p) {
    ck(cudaLaunchKernelEx(&cfg, k_sweeps_tri2<T, 4, 4 * kWarp>, L, r, y0, out, sweeps, omega, d.sx));
  } else if (h->C == 1) {
    ck(cudaLaunchKernelEx(&cfg, k_sweeps_tri2<T, 1>, L, r, y0, out, sweeps, omega, d.sx));
  } else if (h->C == 2) {
    ck(cudaLaunchKernelEx(&cfg, k_sweeps_tri2<T, 2>, L, r, y0, out, sweeps, omega, d.sx));
  } else {
    ck(cudaLaunchKernelEx(&cfg, k_sweeps_tri2<T, 4>, L, r, y0, out, sweeps, omega, d.sx));
  }
  ck_launch();
}

template <typename T, typename CT = T>
void launch_residual_restrict(mg_handle *h, const LevelView<T, CT> &L, const T *y, const T *b, T *rc,
                              cudaStream_t s) {
  const double w = 4.0 * L.p + L.q;
  Bracket br(h, CAT_RESTRICT, s,
             (L.n / 2) * (sizeof(T) * (2.0 * (w + L.q) + w + 3.0 * L.p) + sizeof(CT) * 9.0 * L.p), 0.0);
  const int nc = L.n / 2;
  if (L.layout == MG_LAYOUT_DENSE) {
    if constexpr (std::is_same<T, CT>::value) {
      if (L.p > kDenseMax || L.q > kDenseMax)
        k_residual_restrict_dw<T><<<(nc + 3) / 4, 128, 0, s>>>(L, y, b, rc);
      else
        k_residual_restrict_dense<T><<<grid_for(nc, 128, 1 << 30), 128, 0, s>>>(L, y, b, rc);
    }
  } else {
    const int blocks = (nc + 3) / 4;
    switch (h->C) {
      case 1: k_residual_restrict_tri<T, 1, CT><<<blocks, 128, 0, s>>>(L, y, b, rc); break;
      case 2: k_residual_restrict_tri<T, 2, CT><<<blocks, 128, 0, s>>>(L, y, b, rc); break;
      case 4: k_residual_restrict_tri<T, 4, CT><<<blocks, 128, 0, s>>>(L, y, b, rc); break;
      case 8: k_residual_restrict_tri<T, 8, CT><<<blocks, 128, 0, s>>>(L, y, b, rc); break;
      default: k_residual_restrict_tri<T, 16, CT><<<blocks, 128, 0, s>>>(L, y, b, rc); break;
    }
  }
  ck_launch();
}

template <typename T>
LevelData<T> &ldata(Level &L);
template <>
LevelData<double> &ldata<double>(Level &L) { return L.d; }
template <>
LevelData<float> &ldata<float>(Level &L) { return L.f; }

// ---------------------------------------------------------------------------
// Dot products (FP64), fixed reduction order

// 16-byte paired loads are possible: even lengths and strides, aligned bases
inline bool pair_ok(const void *a, const void *b, long long len, long long ld) {
  return len % 2 == 0 && ld % 2 == 0 && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

// m_dev (optional): the vector count lives on the device; m is then its
// upper bound (grid size) and the kernels read the actual count.
void multidot(mg_handle *h, const double *V, long long ldv, int m, const double *w, long long len, double *out,
              int accumulate, cudaStream_t s, const int *gate = nullptr, const int *m_dev = nullptr) {
  const int VB = h->dot_vb;
  const int items = ((m + VB - 1) / VB) * dot_parts(m, VB, len);
  const int grid = std::min(items, kDotGridCap);
  const bool pair = pair_ok(V, w, len, ldv);
  // fused: the last CTA reduces the partial sums into out (no second launch).  One CTA
  // summing many vectors' partials takes longer than a separate parallel reduction,
  // so by default only short ones are fused (m is the host's bound on the count)
  const bool fuse = h->fuse_reduce >= 2 || (h->fuse_reduce == 1 && m <= 16);
  unsigned *tk = fuse ? h->ticket : nullptr;
  {
    // algorithmic: read the m vectors and w once, 2 m len flops
    Bracket br(h, CAT_DOT, s, 8.0 * (m + (V == w ? 0 : 1)) * len, 2.0 * m * len);
#define PINTMG_DOT(VBV)                                                                                      \
  do {                                                                                                       \
    if (pair)                                                                                                \
      k_multidot_blocked<VBV, true><<<grid, kDotThreads, 0, s>>>(V, ldv, m, w, len, h->partial, gate, m_dev,  \
                                                                  tk, out, accumulate);                      \
    else                                                                                                     \
      k_multidot_blocked<VBV, false><<<grid, kDotThreads, 0, s>>>(V, ldv, m, w, len, h->partial, gate, m_dev, \
                                                                   tk, out, accumulate);                     \
  } while (0)
    if (VB == 4)
      PINTMG_DOT(4);
    else if (VB == 16)
      PINTMG_DOT(16);
    else
      PINTMG_DOT(8);
#undef PINTMG_DOT
    ck_launch();
  }
  if (!tk) {
    Bracket br(h, CAT_SMALL, s);
    k_reduce_partials<<<(m + 3) / 4, 128, 0, s>>>(h->partial, 0, m, out, accumulate, gate, m_dev, VB, len);
    ck_launch();
  }
}

void multi_axpy(mg_handle *h, double *y, const double *X, long long ldx, const double *c, int m, double sign,
                long long len, cudaStream_t s, const int *gate = nullptr, const int *m_dev = nullptr) {
  Bracket br(h, CAT_AXPY, s, 8.0 * (m + 2) * len, 2.0 * m * len);
  if (pair_ok(y, X, len, ldx))
    k_multi_axpy<true><<<grid_for(len / 2, 256, kDotGridCap), 256, 0, s>>>(y, X, ldx, c, m, sign, len, gate, m_dev);
  else
    k_multi_axpy<false><<<grid_for(len, 256, kDotGridCap), 256, 0, s>>>(y, X, ldx, c, m, sign, len, gate, m_dev);
  ck_launch();
}

void read_scal(mg_handle *h, const mg_handle::Krylov &K, cudaStream_t s) {
  ck(cudaMemcpyAsync(h->host_scal, K.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
}

// Classical Gram-Schmidt twice (CGS2) of w against V_0..V_j: h (j+1) and
// |w|^2 (nrm2, accumulated inside the second axpy) on the device.
// (m_dev: the count j + 1 lives on the device, j is then its upper bound - 1)
// the TMA-streamed multi-dot kernel of the pair basis: 8 vectors per item,
// 3 stages, 2 CTAs per SM
constexpr int kPairVB = 8, kPairNS = 3, kPairCtas = 2;
// layout of h->dcg: update coefficients s and t, the pending Hessenberg column, the step's scalars
constexpr int kDcC1 = 0, kDcC2 = 512, kDcHp = 1024, kDcS = 1600, kDcLen = 2048;
// the two-right-hand-side pass (DCGS2): 2 stages so that 2 CTAs per SM fit (3 stages at 1 CTA per SM
// measured 0.37 of HBM against 0.58)
constexpr int kPairNS2 = 2, kPairCtas2 = 2;
void pair_prepare() {
  static unsigned done = 0;
  int dev = 0;
  ck(cudaGetDevice(&dev));
  if (dev < 32 && (done >> dev) & 1u) return;
  ck(cudaFuncSetAttribute(k_multidot_pair_tma<kPairVB, kPairNS, kPairCtas>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_tma_smem<kPairVB, kPairNS>()));
  ck(cudaFuncSetAttribute(k_multidot_pair_tma<kPairVB, kPairNS2, kPairCtas2, 2>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_tma_smem<kPairVB, kPairNS2, 2>()));
  if (dev < 32) done |= 1u << dev;
}

// out = Vp^T w over the m pair vectors (out[i] for i < m), fixed order
void multidot_pair(mg_handle *h, const float2 *Vp, long long ldv, int m, const double *w, long long len, double *out,
                   cudaStream_t s, const int *m_dev = nullptr, const int *gate = nullptr) {
  const int items = ((m + kPairVB - 1) / kPairVB) * dot_parts(m, kPairVB, len);
  const int grid = std::min(items, kPairCtas * 152);
  {
    Bracket br(h, CAT_PAIR_DOT, s, 8.0 * (m + 1) * len, 2.0 * m * len);
    k_multidot_pair_tma<kPairVB, kPairNS, kPairCtas><<<grid, kPairTmaThreads, pair_tma_smem<kPairVB, kPairNS>(), s>>>(
        Vp, ldv, m, w, len, h->partial, gate, m_dev, h->flag + 2, h->pair_stall);
    ck_launch();
  }
  {
    Bracket br(h, CAT_SMALL, s);
    k_reduce_partials<<<(m + 3) / 4, 128, 0, s>>>(h->partial, 0, m, out, 0, gate, m_dev, kPairVB, len);
    ck_launch();
  }
}

// DCGS2's pass over the m final pair vectors: out[i] = V_i . u, out[m + i] = V_i . w (fixed order)
void multidot2_pair(mg_handle *h, const float2 *Vp, long long ldv, int m, const double *u, const double *w,
                    long long len, double *out, cudaStream_t s, const int *m_dev = nullptr) {
  const int items = std::max(1, ((m + kPairVB - 1) / kPairVB) * dot_parts(m, kPairVB, len));
  const int grid = std::min(items, kPairCtas2 * 152);
  {
    Bracket br(h, CAT_PAIR_DOT, s, 8.0 * (m + 2) * len, 4.0 * m * len);
    k_multidot_pair_tma<kPairVB, kPairNS2, kPairCtas2, 2>
        <<<grid, kPairTmaThreads, pair_tma_smem<kPairVB, kPairNS2, 2>(), s>>>(
            Vp, ldv, m, u, len, h->partial, nullptr, m_dev, h->flag + 2, h->pair_stall, w);
    ck_launch();
  }
  {
    Bracket br(h, CAT_SMALL, s);
    k_reduce_partials<<<(2 * m + 3) / 4 + 1, 128, 0, s>>>(h->partial, 0, m, out, 0, nullptr, m_dev, kPairVB, len, 2);
    ck_launch();
  }
}

// DCGS2's update pass (k_multi_axpy2_pair) over the m final pair vectors
void multi_axpy2_pair(mg_handle *h, float2 *Vp, long long len, int m, double *u, const double *w, double *dcg,
                      cudaStream_t s, const int *m_dev = nullptr, const int *gate = nullptr) {
  const int G = grid_for(len / 2, kDotThreads, kDotGridCap);
  Bracket br(h, CAT_PAIR_AXPY, s, 8.0 * (m + 4) * len, 4.0 * m * len);
  k_multi_axpy2_pair<<<G, kDotThreads, 0, s>>>(Vp, len, dcg + kDcC1, dcg + kDcC2, m, u, w, len, dcg + kDcS,
                                               h->partial, h->ticket + 2, gate, m_dev);
  ck_launch();
}

// CGS2 against the basis V (FP64) or Vp (pairs, when not null): K.h = the
// coefficients, K.nrm2 = ||w||^2 of the orthogonalised w.  With step (and the
// fused reductions on), the last CTA of the second axpy also forms the
// Arnoldi column j (index j_dev on the device if given): returns true, and
// the caller launches no k_arnoldi_step.
bool orthogonalise(mg_handle *h, mg_handle::Krylov &K, const double *V, long long len, int j, double *w,
                   cudaStream_t s, const int *m_dev = nullptr, const float2 *Vp = nullptr, bool step = false,
                   const int *j_dev = nullptr) {
  const int m = j + 1;
  const bool tail = step && h->fuse_reduce;
  ArnoldiTail at{};
  if (tail)
    at = ArnoldiTail{h->ticket + 1, K.h, K.h + 512, K.nrm2, K.H, K.cs, K.sn, K.g, K.scal, h->ldh, j, j_dev};
  if (Vp) {
    const int G = grid_for(len / 2, kDotThreads, kDotGridCap);
    multidot_pair(h, Vp, len, m, w, len, K.h, s, m_dev);
    {
      Bracket br(h, CAT_PAIR_AXPY, s, 8.0 * (m + 2) * len, 2.0 * m * len);
      k_multi_axpy_pair<false><<<G, kDotThreads, 0, s>>>(w, Vp, len, K.h, m, -1.0, len, nullptr, nullptr, m_dev);
      ck_launch();
    }
    multidot_pair(h, Vp, len, m, w, len, K.h + 512, s, m_dev);
    {
      Bracket br(h, CAT_PAIR_AXPY, s, 8.0 * (m + 2) * len, 2.0 * (m + 1) * len);
      k_multi_axpy_pair<true><<<G, kDotThreads, 0, s>>>(w, Vp, len, K.h + 512, m, -1.0, len, h->partial, nullptr,
                                                         m_dev, at);
      ck_launch();
    }
  } else {
    multidot(h, V, len, m, w, len, K.h, 0, s, nullptr, m_dev);
    multi_axpy(h, w, V, len, K.h, m, -1.0, len, s, nullptr, m_dev);
    multidot(h, V, len, m, w, len, K.h + 512, 0, s, nullptr, m_dev);
    const bool pair = pair_ok(w, V, len, len);
    const int G = pair ? grid_for(len / 2, kDotThreads, kDotGridCap) : grid_for(len, kDotThreads, kDotGridCap);
    {
      Bracket br(h, CAT_AXPY, s, 8.0 * (m + 2) * len, 2.0 * (m + 1) * len);
      if (pair)
        k_multi_axpy_norm<true><<<G, kDotThreads, 0, s>>>(w, V, len, K.h + 512, m, len, h->partial, m_dev, at);
      else
        k_multi_axpy_norm<false><<<G, kDotThreads, 0, s>>>(w, V, len, K.h + 512, m, len, h->partial, m_dev, at);
      ck_launch();
    }
    if (tail) return true;
    {
      Bracket br(h, CAT_SMALL, s);
      k_reduce_partials<<<1, 128, 0, s>>>(h->partial, G, 1, K.nrm2, 0);
      ck_launch();
    }
    {
      Bracket br(h, CAT_SMALL, s);
      k_add_inplace<<<(m + 127) / 128, 128, 0, s>>>(K.h, K.h + 512, m, nullptr, m_dev);
      ck_launch();
    }
    return false;
  }
  if (tail) return true;
  const int G = grid_for(len / 2, kDotThreads, kDotGridCap);
  {
    Bracket br(h, CAT_SMALL, s);
    k_reduce_partials<<<1, 128, 0, s>>>(h->partial, G, 1, K.nrm2, 0);
    ck_launch();
  }
  {
    Bracket br(h, CAT_SMALL, s);
    k_add_inplace<<<(m + 127) / 128, 128, 0, s>>>(K.h, K.h + 512, m, nullptr, m_dev);
    ck_launch();
  }
  return false;
}

// ||x|| into K.scal[0], 1/||x|| into K.scal[1]
void norm_into(mg_handle *h, mg_handle::Krylov &K, const double *x, long long len, cudaStream_t s) {
  multidot(h, x, len, 1, x, len, K.nrm2, 0, s);
  {
    Bracket br(h, CAT_SMALL, s);
    k_norm_from_sq<<<1, 1, 0, s>>>(K.nrm2, K.scal);
    ck_launch();
  }
}

// Arnoldi step with the index j on the device (st->j, st->m1): no read-back
void arnoldi_step_dev(mg_handle *h, mg_handle::Krylov &K, KState *st, int jmax, double *V, long long len, double *w,
                      cudaStream_t s, float2 *Vp = nullptr, double *also = nullptr) {
  if (!orthogonalise(h, K, V, len, jmax, w, s, &st->m1, Vp, true, &st->j)) {
    Bracket br(h, CAT_SMALL, s);
    k_arnoldi_step<<<1, kWarp, 0, s>>>(0, K.h, K.nrm2, K.H, h->ldh, K.cs, K.sn, K.g, K.scal, &st->j);
    ck_launch();
  }
  {
    Bracket br(h, CAT_AXPY, s);
    if (Vp)
      k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp, w, K.scal + 1, len, &st->j, 1, nullptr, also);
    else
      k_scale<<<grid_for(len, 256), 256, 0, s>>>(V, w, K.scal + 1, len, &st->j, 1, nullptr, also);
    ck_launch();
  }
}

// Add a WHILE conditional node after the work captured so far on stream s and
// capture its body on stream bs; the body must set the condition (handle hdl).
template <class Body>
void add_while(mg_handle *h, cudaStream_t s, cudaGraphConditionalHandle hdl, cudaStream_t bs, Body &&body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  ck(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams params = {};
  params.type = cudaGraphNodeTypeConditional;
  params.conditional.handle = hdl;
  params.conditional.type = cudaGraphCondTypeWhile;
  params.conditional.size = 1;
  cudaGraphNode_t node;
  ck(cudaGraphAddNode(&node, g, deps, nullptr, nd, &params));
  cudaGraph_t bodyg = params.conditional.phGraph_out[0];
  ck(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  body(bs);
  cudaGraph_t tmp = nullptr;
  ck(cudaStreamEndCapture(bs, &tmp));
  ck(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
}

// conditional handle for a node of the graph being captured on stream s
cudaGraphConditionalHandle new_handle(cudaStream_t s) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  ck(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle hdl;
  ck(cudaGraphConditionalHandleCreate(&hdl, g, 0, 0));
  return hdl;
}

// one Arnoldi step on basis V (column stride len): w = A z_j already in w
void arnoldi_step(mg_handle *h, mg_handle::Krylov &K, double *V, long long len, int j, double *w, cudaStream_t s,
                  float2 *Vp = nullptr) {
  if (!orthogonalise(h, K, V, len, j, w, s, nullptr, Vp, true)) {
    Bracket br(h, CAT_SMALL, s);
    k_arnoldi_step<<<1, kWarp, 0, s>>>(j, K.h, K.nrm2, K.H, h->ldh, K.cs, K.sn, K.g, K.scal);
    ck_launch();
  }
  {
    Bracket br(h, CAT_AXPY, s);
    if (Vp)
      k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp + (long long)(j + 1) * len, w, K.scal + 1, len);
    else
      k_scale<<<grid_for(len, 256), 256, 0, s>>>(V + (long long)(j + 1) * len, w, K.scal + 1, len);
    ck_launch();
  }
  read_scal(h, K, s);
}

template <typename T>
void convert(mg_handle *h, const double *x, T *y, long long len, cudaStream_t s);
template <>
void convert<double>(mg_handle *h, const double *x, double *y, long long len, cudaStream_t s) {
  if (x != y) ck(cudaMemcpyAsync(y, x, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
}
template <>
void convert<float>(mg_handle *h, const double *x, float *y, long long len, cudaStream_t s) {
  {
    Bracket br(h, CAT_CONVERT, s);
    k_to_float<<<grid_for(len, 256), 256, 0, s>>>(x, y, len);
    ck_launch();
  }
}
template <typename T>
void convert_back(mg_handle *h, const T *x, double *y, long long len, cudaStream_t s);
template <>
void convert_back<double>(mg_handle *h, const double *x, double *y, long long len, cudaStream_t s) {
  if (x != y) ck(cudaMemcpyAsync(y, x, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
}
template <>
void convert_back<float>(mg_handle *h, const float *x, double *y, long long len, cudaStream_t s) {
  {
    Bracket br(h, CAT_CONVERT, s);
    k_to_double<<<grid_for(len, 256), 256, 0, s>>>(x, y, len);
    ck_launch();
  }
}

// One SGS chain on a thread-block cluster (tridiagonal layout, p >= 32).
// Returns false if the device refuses the cluster launch.
template <typename T, bool kForward, int K>
cudaError_t launch_chain_cluster_k(int S, const T *G, const T *xhat, T *xout, int n, int p, cudaStream_t s,
                                   int seg_len) {
  const int tpr = 16;
  const int rows = (p + S - 1) / S;
  const int threads = ((rows * tpr + 31) / 32) * 32;
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  auto kern = k_chain_cluster<T, kForward, K>;
  if (S > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S * ((n + seg_len - 1) / seg_len), 1, 1);  // one cluster per segment
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 2 * (size_t)p * sizeof(T);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, G, xhat, xout, n, p, rows, tpr, seg_len);
}

// One SGS chain on a thread-block cluster (tridiagonal layout, 32 <= p <= 512):
// 16 threads per row, K = ceil(p / 16) columns per thread.  Returns false if
// the device refuses the cluster launch.
template <typename T, bool kForward>
bool launch_chain_cluster(mg_handle *h, const T *G, const T *xhat, T *xout, int n, int p, cudaStream_t s,
                          int seg_len = 0) {
  const int kneed = (p + 15) / 16;
  if (seg_len <= 0) seg_len = n;
  for (int S : {16, 8}) {
    cudaError_t e;
    if (kneed <= 2) e = launch_chain_cluster_k<T, kForward, 2>(S, G, xhat, xout, n, p, s, seg_len);
    else if (kneed <= 4) e = launch_chain_cluster_k<T, kForward, 4>(S, G, xhat, xout, n, p, s, seg_len);
    else if (kneed <= 8) e = launch_chain_cluster_k<T, kForward, 8>(S, G, xhat, xout, n, p, s, seg_len);
    else if (kneed <= 16) e = launch_chain_cluster_k<T, kForward, 16>(S, G, xhat, xout, n, p, s, seg_len);
    else e = launch_chain_cluster_k<T, kForward, 32>(S, G, xhat, xout, n, p, s, seg_len);
    if (e == cudaSuccess) return true;
    cudaGetLastError();
  }
  return false;
}

// One SGS chain as a parallel scan (k_scan_round): ceil(log2 n) batched GEMVs.
template <typename T>
void run_scan(mg_handle *h, const std::vector<T *> &P, const T *xhat, T *out, T *tmp, int n, int p, int reverse,
              cudaStream_t s) {
  // algorithmic: per round, the prefix products of the steps that update
  // (n - 2^d of them, p^2 each) plus two vector passes; 2 p^2 flops per update
  double bytes = 0.0, flops = 0.0;
  for (int d = 0; d < (int)P.size(); ++d) {
    const double upd = std::max(0, n - (1 << d));
    bytes += sizeof(T) * (upd * (double)p * p + 2.0 * n * p);
    flops += 2.0 * upd * (double)p * p;
  }
  Bracket br(h, CAT_CHAIN, s, bytes, flops);
  const int R = (int)P.size();
  if (R == 0) {
    ck(cudaMemcpyAsync(out, xhat, (size_t)n * p * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return;
  }
  // rows per CTA: slices of 32 rows when p is a multiple of 32 and n would leave
  // SMs idle, else all p; parts column slices per row: the largest power of two
  // with parts * rows <= 512 (256 for slices) and at least 8 columns per slice
  const int rows = (p % 32 == 0 && p >= 64 && n < 4 * 152) ? 32 : p;
  const int max_threads = rows < p ? 256 : 512;
  int parts = 1;
  while (parts * 2 * rows <= max_threads && p / (parts * 2) >= 8) parts *= 2;
  const int threads = std::max(parts * rows, 32);
  const size_t shm = (size_t)p * sizeof(T) + (size_t)parts * rows * sizeof(T);
  const dim3 grid(n, p / rows);
  const T *in = xhat;
  for (int d = 0; d < R; ++d) {
    T *dst = ((R - 1 - d) % 2 == 0) ? out : tmp;
    k_scan_round<T><<<grid, threads, shm, s>>>(P[d], in, dst, n, p, 1 << d, reverse, parts, rows);
    ck_launch();
    in = dst;
  }
}

// One SGS chain as concurrent segment chains (one thread-block cluster per
// segment of seg_len positions, from a zero incoming state) joined by the
// in-segment products Q: a serial pass over the segment ends, then every other
// position in one batched GEMV.  Returns false if the cluster launch is refused.
template <typename T, bool kForward>
bool run_seg(mg_handle *h, const T *G, const T *Q, int seg_len, const T *xhat, T *out, int n, int p,
             cudaStream_t s) {
  if (!launch_chain_cluster<T, kForward>(h, G, xhat, out, n, p, s, seg_len)) return false;
  ck_launch();
  const int rows = p % 32 == 0 ? 32 : p;
  int parts = 1;
  while (parts * 2 * rows <= 256 && p / (parts * 2) >= 8) parts *= 2;
  const int threads = std::max(parts * rows, 32);
  const size_t shm = (size_t)p * sizeof(T) + (size_t)parts * rows * sizeof(T);
  const int nseg = (n + seg_len - 1) / seg_len;
  for (int c = 1; c < nseg; ++c) {  // the true last entry of every segment, in order
    k_seg_fix<T><<<dim3(1, p / rows), threads, shm, s>>>(Q, out, n, p, seg_len, c, kForward ? 0 : 1, parts, rows);
    ck_launch();
  }
  k_seg_fix<T><<<dim3(n, p / rows), threads, shm, s>>>(Q, out, n, p, seg_len, 0, kForward ? 0 : 1, parts, rows);
  ck_launch();
  return true;
}

// ---------------------------------------------------------------------------
// The coarse preconditioner on the coarsest level (precision T):
// SGS y = [(D+L) D^-1 (D+L^T)]^-1 r, or one of Table 1's alternatives.

template <typename T>
void sgs_apply(mg_handle *h, Level &lev, const T *r, T *y, cudaStream_t s) {
  LevelData<T> &d = ldata<T>(lev);
  const int n = lev.n, p = h->p;
  const int kind = h->opts.coarse_precond;
  if (kind == MG_COARSE_JACOBI) {  // D^-1 r
    launch_block_solve<T>(h, d.view, r, nullptr, nullptr, y, s);
    return;
  }
  const int threads = std::max(32, ((p + 31) / 32) * 32);
  const size_t shm = (size_t)p * sizeof(T);
  const bool cluster = h->layout == MG_LAYOUT_TRIDIAG && p >= 32 && h->use_cluster;
  const bool scan = h->use_scan && (n == 1 || !d.scanF.empty());
  const bool seg = !scan && h->use_seg && d.segF != nullptr;
  const bool forward = kind != MG_COARSE_BGS;
  // algorithmic work of a segmented chain: the serial links plus the joining products
  const double seg_bytes = (double)sizeof(T) * 2.0 * n * ((double)p * p + 2.0 * p), seg_flops = 4.0 * n * p * p;
  if (forward) {
    // w = D^-1 r; forward chain u_j = uhat_j - Cu_j u_{j-1}
    launch_block_solve<T>(h, d.view, r, nullptr, nullptr, d.sgs_w, s);
    bool done = false;
    if (scan) {
      run_scan<T>(h, d.scanF, make_vec(d.sgs_w, n, p, h->q).u, d.chainU, d.scan_tmp, n, p, 0, s);
      done = true;
    } else if (seg) {
      Bracket br(h, CAT_CHAIN, s, seg_bytes, seg_flops);
      done = run_seg<T, true>(h, d.Cu, d.segF, d.seg_len, make_vec(d.sgs_w, n, p, h->q).u, d.chainU, n, p, s);
    }
    if (!done && n >= 1) {
      // algorithmic: one p x p link matrix read and applied per step
      Bracket br(h, CAT_CHAIN, s, (double)sizeof(T) * n * ((double)p * p + 2.0 * p), 2.0 * n * p * p);
      if (!cluster || !launch_chain_cluster<T, true>(h, d.Cu, make_vec(d.sgs_w, n, p, h->q).u, d.chainU, n, p, s)) {
        k_chain_forward<T><<<1, threads, shm, s>>>(d.Cu, make_vec(d.sgs_w, n, p, h->q).u, d.chainU, n, p);
      }
      ck_launch();
    }
    if (kind == MG_COARSE_FGS) {  // w = (D + L)^-1 r
      launch_block_solve<T>(h, d.view, r, d.chainU, nullptr, y, s);
      return;
    }
  }
  // yhat = D^-1 (r - L w) (SGS) or D^-1 r (backward Gauss-Seidel alone):
  // only mu(yhat) is needed by the backward chain
  const T *fwd = forward ? d.chainU : nullptr;
  launch_block_solve<T>(h, d.view, r, fwd, nullptr, d.sgs_w, s);
  bool done = false;
  if (scan) {
    run_scan<T>(h, d.scanB, make_vec(d.sgs_w, n, p, h->q).m, d.chainM, d.scan_tmp, n, p, 1, s);
    done = true;
  } else if (seg) {
    Bracket br(h, CAT_CHAIN, s, seg_bytes, seg_flops);
    done = run_seg<T, false>(h, d.Em, d.segB, d.seg_len, make_vec(d.sgs_w, n, p, h->q).m, d.chainM, n, p, s);
  }
  if (!done && n >= 1) {
    Bracket br(h, CAT_CHAIN, s, (double)sizeof(T) * n * ((double)p * p + 2.0 * p), 2.0 * n * p * p);
    if (!cluster || !launch_chain_cluster<T, false>(h, d.Em, make_vec(d.sgs_w, n, p, h->q).m, d.chainM, n, p, s)) {
      k_chain_backward<T><<<1, threads, shm, s>>>(d.Em, make_vec(d.sgs_w, n, p, h->q).m, d.chainM, n, p);
    }
    ck_launch();
  }
  // y = D^-1 (r - L w - L^T y)
  launch_block_solve<T>(h, d.view, r, fwd, d.chainM, y, s);
}

// precondition a coarse FP64 vector with SGS in precision T
template <typename T>
void sgs_fp64(mg_handle *h, Level &lev, const double *r, double *y, cudaStream_t s);
template <>
void sgs_fp64<double>(mg_handle *h, Level &lev, const double *r, double *y, cudaStream_t s) {
  sgs_apply<double>(h, lev, r, y, s);
}
template <>
void sgs_fp64<float>(mg_handle *h, Level &lev, const double *r, double *y, cudaStream_t s) {
  if (h->opts.precision == MG_PRECISION_FP32_SMOOTH) {  // the coarse solve stays FP64
    sgs_apply<double>(h, lev, r, y, s);
    return;
  }
  LevelData<float> &d = lev.f;
  convert<float>(h, r, d.b, lev.len, s);
  sgs_apply<float>(h, lev, d.b, d.y, s);
  convert_back<float>(h, d.y, y, lev.len, s);
}

// ---------------------------------------------------------------------------
// Learned coarse correction: network forward pass and the admission test

// one convolution layer (k_conv_tiled): 16 output channels per CTA, or 8 for narrow layers
template <typename T>
void launch_conv(const T *x, const T *W, const T *bias, T *y, float *z, int B, int C, int O, int H, int Wd, int act,
                 cudaStream_t s) {
  const int OB = O > 8 ? 16 : 8;
  const dim3 grid((Wd + kConvTX - 1) / kConvTX, (H + kConvTT - 1) / kConvTT, B * ((O + OB - 1) / OB));
  if (OB == 16)
    k_conv_tiled<T, 16><<<grid, 256, 0, s>>>(x, W, bias, y, z, B, C, O, H, Wd, act);
  else
    k_conv_tiled<T, 8><<<grid, 256, 0, s>>>(x, W, bias, y, z, B, C, O, H, Wd, act);
  ck_launch();
}

// BF16 layers on the tensor cores (k_conv_mma): 16-channel input blocks, 8-channel output tiles
// the kernels' dynamic shared memory limits (above the default 48 KB), once per
// device; called outside stream capture (network creation and attachment)
void conv_mma_prepare() {
  static unsigned done = 0;
  int dev = 0;
  ck(cudaGetDevice(&dev));
  if (dev < 32 && (done >> dev) & 1u) return;
  ck(cudaFuncSetAttribute(k_conv_mma<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_mma_smem(1, 4)));
  ck(cudaFuncSetAttribute(k_conv_mma<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_mma_smem(2, 1)));
  ck(cudaFuncSetAttribute(k_conv_mma<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, conv_mma_smem(2, 4)));
  ck(cudaFuncSetAttribute(k_conv_tc<1, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(1, 32)));
  ck(cudaFuncSetAttribute(k_conv_tc<2, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(2, 32)));
  ck(cudaFuncSetAttribute(k_conv_tc<2, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(2, 16)));
  if (dev < 32) done |= 1u << dev;
}

// BF16 inference layers on tcgen05 (default) or, with PINTMG_CONV_MMA=1, on mma.sync
bool conv_use_tc() {
  static const bool tc = [] {
    const char *e = std::getenv("PINTMG_CONV_MMA");
    return !(e && e[0] == '1');
  }();
  return tc;
}

// cuTensorMapEncodeTiled, resolved from the driver once (no link against libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// tensor map of a network activation [B][H][Wd][Cp] (BF16, channels innermost) for k_conv_tc's
// input planes: boxes of 8 channels x kTcSP positions x kTcSR rows x 1 sample, zero fill outside
CUtensorMap tc_input_map(const __nv_bfloat16 *x, int Cp, int B, int H, int Wd) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "cuTensorMapEncodeTiled is not available");
    throw CudaFail{cudaErrorNotSupported};
  }
  CUtensorMap m;
  const cuuint64_t dims[4] = {(cuuint64_t)Cp, (cuuint64_t)Wd, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)Cp * 2, (cuuint64_t)Wd * Cp * 2, (cuuint64_t)H * Wd * Cp * 2};
  const cuuint32_t box[4] = {8, (cuuint32_t)kTcSP, (cuuint32_t)kTcSR, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(x), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    throw CudaFail{cudaErrorInvalidValue};
  }
  return m;
}

// layer l of the network in BF16 on tcgen05 (weights from the layer's image): x [B][H][Wd][16 CB]
// (channels innermost), y channels innermost [B][H][Wd][32] for the hidden layers, [B][5][H][Wd] for
// the last; err: the wait flag
void launch_conv_tc(const __nv_bfloat16 *timg_all, int l, const __nv_bfloat16 *x, const __nv_bfloat16 *bias,
                    __nv_bfloat16 *y, int B, int H, int Wd, int act, int *err, cudaStream_t s) {
  const __nv_bfloat16 *img = timg_all + tc_img_offset(l);
  const int O = net_ch(l + 1);
  const dim3 grid((Wd + kTcM - 1) / kTcM, (H + kTcRows - 1) / kTcRows, B);
  const int cb = tc_cb(l), n = tc_nl(l);
  const CUtensorMap xm = tc_input_map(x, 16 * cb, B, H, Wd);
  if (cb == 1 && n == 32)
    k_conv_tc<1, 32, true><<<grid, kTcThreads, tc_smem(1, 32), s>>>(xm, img, bias, y, O, H, Wd, act, err);
  else if (cb == 2 && n == 16)
    k_conv_tc<2, 16, false><<<grid, kTcThreads, tc_smem(2, 16), s>>>(xm, img, bias, y, O, H, Wd, act, err);
  else
    k_conv_tc<2, 32, true><<<grid, kTcThreads, tc_smem(2, 32), s>>>(xm, img, bias, y, O, H, Wd, act, err);
  ck_launch();
}

template <int CB, int NT>
void launch_conv_mma_t(const __nv_bfloat16 *x, const __nv_bfloat16 *wimg, const __nv_bfloat16 *bias,
                       __nv_bfloat16 *y, int B, int C, int O, int H, int Wd, int act, cudaStream_t s) {
  constexpr int smem = conv_mma_smem(CB, NT);
  const dim3 grid((Wd + kMmaCols - 1) / kMmaCols, (H + kMmaRows - 1) / kMmaRows, B);
  k_conv_mma<CB, NT><<<grid, 128, smem, s>>>(x, wimg, bias, y, B, C, O, H, Wd, act);
  ck_launch();
}

// layer l of the network in BF16 on the tensor cores (weights from the layer's image)
void launch_conv_mma(const __nv_bfloat16 *wimg_all, int l, const __nv_bfloat16 *x, const __nv_bfloat16 *bias,
                     __nv_bfloat16 *y, int B, int H, int Wd, int act, cudaStream_t s) {
  const __nv_bfloat16 *wimg = wimg_all + conv_mma_wimg_offset(l);
  const int C = net_ch(l), O = net_ch(l + 1);
  const int cb = conv_mma_cb(l), nt = conv_mma_nt(l);
  if (cb == 1 && nt == 4)
    launch_conv_mma_t<1, 4>(x, wimg, bias, y, B, C, O, H, Wd, act, s);
  else if (cb == 2 && nt == 1)
    launch_conv_mma_t<2, 1>(x, wimg, bias, y, B, C, O, H, Wd, act, s);
  else
    launch_conv_mma_t<2, 4>(x, wimg, bias, y, B, C, O, H, Wd, act, s);
}

// The network's forward pass in storage type T (inference): x -> y through
// ping-pong buffers (x == y allowed).  h (may be NULL) counts and times the launches.
template <typename T>
void net_forward_storage(mg_handle *h, const mg_net *net, const T *x, int B, int H, int Wd, T *y, T *bufA, T *bufB,
                         cudaStream_t s) {
  constexpr bool kBf16 = std::is_same<T, __nv_bfloat16>::value;
  const T *params = kBf16 ? reinterpret_cast<const T *>(net->params_bf16) : reinterpret_cast<const T *>(net->params);
  const T *in = x;
  for (int l = 0; l < kNetLayers; ++l) {
    T *out = (l == kNetLayers - 1) ? y : ((l % 2 == 0) ? bufA : bufB);
    const T *W = params + net_layer_offset(l);
    const T *bias = W + (long long)net_ch(l + 1) * net_ch(l) * kNetKT * kNetKX;
    const long long n = (long long)B * net_ch(l + 1) * H * Wd;
    const double flops = 2.0 * n * net_ch(l) * kNetKT * kNetKX;
    const int act = l < kNetLayers - 1;
    auto run = [&] {
      if constexpr (kBf16) {
        if (conv_use_tc())
          launch_conv_tc(net->timg, l, in, bias, out, B, H, Wd, act, h ? h->flag + 2 : net->tc_err, s);
        else
          launch_conv_mma(net->wimg, l, in, bias, out, B, H, Wd, act, s);
      } else
        launch_conv<T>(in, W, bias, out, nullptr, B, net_ch(l), net_ch(l + 1), H, Wd, act, s);
    };
    if (h) {
      Bracket br(h, CAT_NET, s, (double)sizeof(T) * (n + (double)B * net_ch(l) * H * Wd), flops);
      run();
    } else {
      run();
    }
    in = out;
  }
}

void net_refresh_bf16(mg_net *net, cudaStream_t s) {
  if (net->bf16_valid) return;
  k_f32_to_bf16<<<grid_for(kNetParams, 256), 256, 0, s>>>(net->params, net->params_bf16, kNetParams);
  ck_launch();
  for (int l = 0; l < kNetLayers; ++l) {  // the tensor-core kernels' weight images
    const __nv_bfloat16 *W = net->params_bf16 + net_layer_offset(l);
    __nv_bfloat16 *img = net->wimg + conv_mma_wimg_offset(l);
    const int cb = conv_mma_cb(l), nt = conv_mma_nt(l);
    const int n = conv_mma_wimg(cb, nt);
    if (cb == 1 && nt == 4)
      k_conv_mma_image<1, 4><<<grid_for(n, 256), 256, 0, s>>>(W, net_ch(l), net_ch(l + 1), img);
    else if (cb == 2 && nt == 1)
      k_conv_mma_image<2, 1><<<grid_for(n, 256), 256, 0, s>>>(W, net_ch(l), net_ch(l + 1), img);
    else
      k_conv_mma_image<2, 4><<<grid_for(n, 256), 256, 0, s>>>(W, net_ch(l), net_ch(l + 1), img);
    ck_launch();
    __nv_bfloat16 *timg = net->timg + tc_img_offset(l);
    const int tn = tc_img_bytes(tc_cb(l), tc_nl(l)) / 2;
    if (tc_cb(l) == 1 && tc_nl(l) == 32)
      k_conv_tc_image<1, 32><<<grid_for(tn, 256), 256, 0, s>>>(W, net_ch(l), net_ch(l + 1), timg);
    else if (tc_cb(l) == 2 && tc_nl(l) == 16)
      k_conv_tc_image<2, 16><<<grid_for(tn, 256), 256, 0, s>>>(W, net_ch(l), net_ch(l + 1), timg);
    else
      k_conv_tc_image<2, 32><<<grid_for(tn, 256), 256, 0, s>>>(W, net_ch(l), net_ch(l + 1), timg);
    ck_launch();
  }
  net->bf16_valid = true;
}

// e = rms(r) net(r / rms(r)) on the coarse level, rms(r) = ||r|| / sqrt(len) (K.scal holds ||r||, 1/||r||)
void net_coarse_proposal(mg_handle *h, Level &lev, const mg_handle::Krylov &K, cudaStream_t s) {
  mg_net *net = h->net;
  const long long len = lev.len;
  const int H = lev.n, Wd = h->p;
  if (h->net_bf16) {
    if (!h->capturing) net_refresh_bf16(net, s);
    using B16 = __nv_bfloat16;
    B16 *xin = static_cast<B16 *>(h->net_x), *a = static_cast<B16 *>(h->net_a), *b = static_cast<B16 *>(h->net_b);
    {
      Bracket br(h, CAT_NET, s);
      if (conv_use_tc())  // the tcgen05 layers read their input with the channels innermost
        k_net_input_ci<<<grid_for((long long)H * Wd, 256), 256, 0, s>>>(h->cr, K.scal, xin, (long long)H * Wd);
      else
        k_net_input<B16><<<grid_for(len, 256), 256, 0, s>>>(h->cr, K.scal, xin, len);
      ck_launch();
    }
    net_forward_storage<B16>(h, net, xin, 1, H, Wd, xin, a, b, s);
    {
      Bracket br(h, CAT_NET, s);
      k_net_output<B16><<<grid_for(len, 256), 256, 0, s>>>(xin, K.scal, h->net_e, len);
      ck_launch();
    }
  } else {
    float *xin = static_cast<float *>(h->net_x), *a = static_cast<float *>(h->net_a),
          *b = static_cast<float *>(h->net_b);
    {
      Bracket br(h, CAT_NET, s);
      k_net_input<float><<<grid_for(len, 256), 256, 0, s>>>(h->cr, K.scal, xin, len);
      ck_launch();
    }
    net_forward_storage<float>(h, net, xin, 1, H, Wd, xin, a, b, s);
    {
      Bracket br(h, CAT_NET, s);
      k_net_output<float><<<grid_for(len, 256), 256, 0, s>>>(xin, K.scal, h->net_e, len);
      ck_launch();
    }
  }
}

// Coarse solve inside a captured graph: the same GMRES with its loop as a
// WHILE node whose condition the step-control kernel sets on the device.
template <typename T>
void coarse_solve_graph(mg_handle *h, const T *r_in, T *y_out, cudaStream_t s) {
  Level &lev = h->lv.back();
  const long long len = lev.len;
  const mg_options &o = h->opts;
  mg_handle::Krylov &K = h->kc;
  KState *st = h->kst_c;
  const bool fixed = o.coarse_fixed_iters > 0;
  const int limit = fixed ? std::min(o.coarse_fixed_iters, h->cmax) : o.coarse_maxit;
  convert_back<T>(h, r_in, h->cr, len, s);
  norm_into(h, K, h->cr, len, s);
  if (h->net) {  // the network's proposal, admitted if it reduces the residual enough
    net_coarse_proposal(h, lev, K, s);
    launch_apply<double>(h, lev.d.view, h->net_e, h->cr, h->net_r, s);
    multidot(h, h->net_r, len, 1, h->net_r, len, K.nrm2 + 3, 0, s);
    Bracket br(h, CAT_SMALL, s);
    k_net_admit<<<1, 1, 0, s>>>(K.nrm2 + 3, K.scal, h->admit, h->net_flag);
    ck_launch();
  }
  const cudaGraphConditionalHandle hdl = new_handle(s);
  {
    Bracket br(h, CAT_SMALL, s);
    k_ctl_start<<<1, 1, 0, s>>>(st, K.scal, fixed ? -1.0 : o.coarse_rtol, hdl, h->net ? h->net_flag : nullptr);
    ck_launch();
  }
  const bool fc = h->fuse_copies;  // the input and Z_j copies ride on the basis write and the product
  {
    Bracket br(h, CAT_AXPY, s);
    k_scale<<<grid_for(len, 256), 256, 0, s>>>(h->cV, h->cr, K.scal + 1, len, nullptr, 0, nullptr,
                                                fc ? h->cvin : nullptr);
    ck_launch();
  }
  {
    Bracket br(h, CAT_SMALL, s);
    k_arnoldi_init<<<1, 128, 0, s>>>(K.scal, K.g, h->cmax);
    ck_launch();
  }
  ck(cudaMemsetAsync(h->cy, 0, len * sizeof(double), s));
  const long long before = h->launches;
  add_while(h, s, hdl, h->cap[2], [&](cudaStream_t bs) {
    if (!fc) {
      Bracket br(h, CAT_SMALL, bs);
      k_copy_indexed<<<grid_for(len, 256), 256, 0, bs>>>(h->cvin, h->cV, len, &st->j, 0);
      ck_launch();
    }
    sgs_fp64<T>(h, lev, h->cvin, h->czout, bs);
    if (!fc) {
      Bracket br(h, CAT_SMALL, bs);
      k_copy_indexed<<<grid_for(len, 256), 256, 0, bs>>>(h->cZ, h->czout, len, &st->j, 1);
      ck_launch();
    }
    launch_apply<double>(h, lev.d.view, h->czout, nullptr, h->cw, bs, 0, -1, fc ? h->cZ : nullptr, &st->j, 0);
    arnoldi_step_dev(h, K, st, limit - 1, h->cV, len, h->cw, bs, nullptr, fc ? h->cvin : nullptr);
    {
      Bracket br(h, CAT_SMALL, bs);
      k_ctl_step<<<1, 1, 0, bs>>>(st, K.scal, limit, limit, 1, hdl);
      ck_launch();
    }
  });
  h->g_coarse = h->launches - before;
  h->launches = before;
  {
    Bracket br(h, CAT_SMALL, s);
    k_backsolve<<<1, 256, (size_t)limit * sizeof(double), s>>>(0, K.H, h->ldh, K.g, K.ycoef, &st->kcount);
    ck_launch();
  }
  multi_axpy(h, h->cy, h->cZ, len, K.ycoef, limit, 1.0, len, s, nullptr, &st->kcount);
  if (h->net) {
    Bracket br(h, CAT_SMALL, s);
    k_copy_if<<<grid_for(len, 256), 256, 0, s>>>(h->cy, h->net_e, len, h->net_flag);
    ck_launch();
  }
  convert<T>(h, h->cy, y_out, len, s);
}

// Coarse solve (Sec. 5.3.4): GMRES, right-preconditioned by SGS, x0 = 0,
// FP64 Arnoldi; y (precision T) = approximate A_c^-1 r.
template <typename T>
void coarse_solve(mg_handle *h, const T *r_in, T *y_out, cudaStream_t s) {
  if (h->capturing) {
    coarse_solve_graph<T>(h, r_in, y_out, s);
    return;
  }
  Level &lev = h->lv.back();
  const long long len = lev.len;
  const mg_options &o = h->opts;
  mg_handle::Krylov &K = h->kc;
  convert_back<T>(h, r_in, h->cr, len, s);
  norm_into(h, K, h->cr, len, s);
  read_scal(h, K, s);
  const double beta = h->host_scal[0];
  if (!(beta > 0.0)) {
    ck(cudaMemsetAsync(y_out, 0, len * sizeof(T), s));
    return;
  }
  if (h->net) {  // the network's proposal, admitted if it reduces the residual enough
    net_coarse_proposal(h, lev, K, s);
    launch_apply<double>(h, lev.d.view, h->net_e, h->cr, h->net_r, s);
    multidot(h, h->net_r, len, 1, h->net_r, len, K.nrm2 + 3, 0, s);
    double rr = 0.0;
    ck(cudaMemcpyAsync(&rr, K.nrm2 + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    if (std::sqrt(rr) <= h->admit * beta) {
      h->coarse_learned++;
      convert<T>(h, h->net_e, y_out, len, s);
      return;
    }
  }
  const int limit = o.coarse_fixed_iters > 0 ? std::min(o.coarse_fixed_iters, h->cmax) : o.coarse_maxit;
  {
    Bracket br(h, CAT_AXPY, s);
    k_scale<<<grid_for(len, 256), 256, 0, s>>>(h->cV, h->cr, K.scal + 1, len);
    ck_launch();
  }
  {
    Bracket br(h, CAT_SMALL, s);
    k_arnoldi_init<<<1, 128, 0, s>>>(K.scal, K.g, h->cmax);
    ck_launch();
  }
  int k = 0;
  for (int j = 0; j < limit; ++j) {
    double *vj = h->cV + (long long)j * len, *zj = h->cZ + (long long)j * len;
    sgs_fp64<T>(h, lev, vj, zj, s);
    launch_apply<double>(h, lev.d.view, zj, nullptr, h->cw, s);
    arnoldi_step(h, K, h->cV, len, j, h->cw, s);
    k = j + 1;
    const double est = h->host_scal[0], hj1 = h->host_scal[2];
    if (!std::isfinite(est) || !std::isfinite(hj1)) break;
    if (hj1 == 0.0) break;
    if (o.coarse_fixed_iters <= 0 && est <= o.coarse_rtol * beta) break;
  }
  h->coarse_iters += k;
  {
    Bracket br(h, CAT_SMALL, s);
    k_backsolve<<<1, 256, (size_t)k * sizeof(double), s>>>(k, K.H, h->ldh, K.g, K.ycoef);
    ck_launch();
  }
  ck(cudaMemsetAsync(h->cy, 0, len * sizeof(double), s));
  multi_axpy(h, h->cy, h->cZ, len, K.ycoef, k, 1.0, len, s);
  if (h->rec_r && h->rec_count < h->rec_max) {  // training pair of the plain method, scaled by 1/rms(r)
    Bracket br(h, CAT_SMALL, s);
    k_record_pair<<<grid_for(len, 256), 256, 0, s>>>(h->cr, h->cy, std::sqrt((double)len) / beta, h->rec_r + (long long)h->rec_count * len,
                                                     h->rec_y + (long long)h->rec_count * len, len);
    ck_launch();
    h->rec_count++;
  }
  convert<T>(h, h->cy, y_out, len, s);
}

// V-cycle from y = 0 on level l (Alg. 1 generalised): b, y in precision T
template <typename T>
void vcycle(mg_handle *h, int l, const T *b, T *y_out, cudaStream_t s);

// one smoothing level of the V-cycle; `view` is the level's coefficients as
// the smoother and residual read them (FP64 / FP32, or FP32 with BF16 bands)
template <typename T, typename VIEW>
void vcycle_level(mg_handle *h, int l, const VIEW &view, const T *b, T *y_out, cudaStream_t s) {
  Level &lev = h->lv[l];
  LevelData<T> &d = ldata<T>(lev);
  const mg_options &o = h->opts;
  constexpr bool kPlain = std::is_same<VIEW, LevelView<T>>::value;  // the multi-sweep kernel reads T bands
  const bool persist = kPlain && d.persist;
  T *y = y_out, *t = d.tmp;
  if (o.nu_pre == 0) {
    ck(cudaMemsetAsync(y, 0, lev.len * sizeof(T), s));
  } else if (persist) {
    launch_sweeps<T>(h, d, b, nullptr, y, o.nu_pre, (T)o.omega, s);  // all pre-sweeps, from y = 0
  } else {
    const T om = (T)o.omega;
    launch_block_solve<T>(h, view, b, nullptr, nullptr, y, s, nullptr, om);  // first sweep from y = 0
    for (int k = 1; k < o.nu_pre; ++k) {
      Vec<T> Y = make_vec(y, lev.n, h->p, h->q);
      launch_block_solve<T>(h, view, b, Y.u, Y.m, t, s, y, om);
      std::swap(y, t);
    }
  }
  LevelData<T> &dn = ldata<T>(h->lv[l + 1]);
  if (o.restrict_rule == MG_RESTRICT_TRANSPOSE) {
    launch_apply<T>(h, view, y, b, t, s);  // full fine residual into the free sweep buffer
    const double w = 4.0 * h->p + h->q;
    Bracket br(h, CAT_RESTRICT, s, sizeof(T) * (lev.n / 2) * w * 3.0, 0.0);
    launch_restrict_transpose<T>(t, dn.b, lev.n, h->p, h->q, o.end_rule, s);
    ck_launch();
  } else {
    launch_residual_restrict<T>(h, view, y, b, dn.b, s);
  }
  vcycle<T>(h, l + 1, dn.b, dn.y, s);
  {
    Bracket br(h, CAT_PROLONG, s);
    launch_prolong<T>(dn.y, y, lev.n, h->p, h->q, o.end_rule, s);
    ck_launch();
  }
  if (persist && o.nu_post > 0) {
    launch_sweeps<T>(h, d, b, y, t, o.nu_post, (T)o.omega, s);  // all post-sweeps, from y
    std::swap(y, t);
  } else {
    for (int k = 0; k < o.nu_post; ++k) {
      Vec<T> Y = make_vec(y, lev.n, h->p, h->q);
      launch_block_solve<T>(h, view, b, Y.u, Y.m, t, s, y, (T)o.omega);
      std::swap(y, t);
    }
  }
  if (y != y_out) ck(cudaMemcpyAsync(y_out, y, lev.len * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

template <typename T>
void vcycle(mg_handle *h, int l, const T *b, T *y_out, cudaStream_t s) {
  const int last = (int)h->lv.size() - 1;
  if (l == last) {
    coarse_solve<T>(h, b, y_out, s);
    return;
  }
  LevelData<T> &d = ldata<T>(h->lv[l]);
  if constexpr (std::is_same<T, float>::value) {
    if (d.bands16) {  // MG_PRECISION_BF16_BANDS: this level's bands are read as BF16
      vcycle_level<T>(h, l, d.vh, b, y_out, s);
      return;
    }
  }
  vcycle_level<T>(h, l, d.view, b, y_out, s);
}

// z = M^-1 v on FP64 fine vectors
void precondition(mg_handle *h, const double *v, double *z, cudaStream_t s) {
  h->vcycles++;
  if (h->opts.precision != MG_PRECISION_FP64) {
    Level &f = h->lv[0];
    convert<float>(h, v, f.f.b, f.len, s);
    vcycle<float>(h, 0, f.f.b, f.f.y, s);
    convert_back<float>(h, f.f.y, z, f.len, s);
  } else {
    vcycle<double>(h, 0, v, z, s);
  }
}

// ---------------------------------------------------------------------------
// Setup helpers

template <typename T>
void alloc_level_vectors(mg_handle *h, Level &lev, LevelData<T> &d, bool is_last, bool is_first, cudaStream_t s) {
  const long long len = lev.len;
  if (!is_last) prepare_sweeps<T>(h, lev, d, s);
  d.tmp = h->mem.alloc<T>(len);
  if (h->layout == MG_LAYOUT_TRIDIAG && h->p > 4 * kWarp) {  // the three-launch block solve's workspaces
    const size_t ws = (size_t)(lev.n + 1) * h->p;
    d.view.ws_rhs = h->mem.alloc<T>(ws);
    d.view.ws_lam = h->mem.alloc<T>(ws);
    d.vh.ws_rhs = d.view.ws_rhs;
    d.vh.ws_lam = d.view.ws_lam;
  }
  if (!is_first || sizeof(T) == sizeof(float)) {
    d.b = h->mem.alloc<T>(len);
    d.y = h->mem.alloc<T>(len);
  }
  if (is_last) {
    d.chainU = h->mem.alloc<T>((size_t)std::max(lev.n, 1) * h->p);
    d.chainM = h->mem.alloc<T>((size_t)std::max(lev.n, 1) * h->p);
    d.sgs_w = h->mem.alloc<T>(len);
  }
}

__nv_bfloat16 *to_bf16_copy(mg_handle *h, const float *x, long long len, cudaStream_t s) {
  __nv_bfloat16 *y = h->mem.alloc<__nv_bfloat16>(len);
  {
    Bracket br(h, CAT_CONVERT, s);
    k_to_bf16<<<grid_for(len, 256), 256, 0, s>>>(x, y, len);
    ck_launch();
  }
  return y;
}

float *to_float_copy(mg_handle *h, const double *x, long long len, cudaStream_t s) {
  float *y = h->mem.alloc<float>(len);
  {
    Bracket br(h, CAT_CONVERT, s);
    k_to_float<<<grid_for(len, 256), 256, 0, s>>>(x, y, len);
    ck_launch();
  }
  return y;
}

bool host_finite(const double *x, long long len) {
  for (long long i = 0; i < len; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

void ensure_fgmres_space(mg_handle *h, int m, cudaStream_t s) {
  if (m <= h->fm) return;
  ck(cudaStreamSynchronize(s));
  if (h->gexec) {  // a captured solve refers to the old basis
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  for (void *p : h->fmem) cudaFree(p);
  h->fmem.clear();
  h->fm = 0;
  const long long len = h->lv[0].len;
  auto grab = [&](size_t count) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
      throw std::bad_alloc();
    }
    h->fmem.push_back(p);
    return static_cast<double *>(p);
  };
  h->fV = grab((size_t)(m + 1) * len);
  h->fZ = grab((size_t)m * len);
  if (h->dcgs2) {
    h->fu = grab((size_t)len);
    h->dcg = grab((size_t)kDcLen);
  }
  h->fm = m;
}

// out = b - A x on the finest level when the gate is open (a kernel that returns at once otherwise)
void launch_apply_gated(mg_handle *h, const double *x, const double *b, double *out, const int *gate, cudaStream_t bs) {
  Bracket br(h, CAT_APPLY, bs);
  const LevelView<double> &L = h->lv[0].d.view;
  if (L.layout == MG_LAYOUT_DENSE && (L.p > kDenseMax || L.q > kDenseMax)) {
    k_apply_dw<double><<<(L.n + 3) / 4, 128, 0, bs>>>(L, x, b, out, gate);
  } else if (L.layout == MG_LAYOUT_DENSE) {
    k_apply_dense<double><<<grid_for(L.n, 128, 1 << 30), 128, 0, bs>>>(L, x, b, out, gate);
  } else if (L.p > 4 * kWarp && h->split_bs) {
    k_apply_ent<double, double><<<grid_for((long long)L.n * L.p, 256, 1 << 20), 256, 0, bs>>>(L, x, b, out, gate);
  } else {
    const int blocks = (L.n + 3) / 4;
    switch (h->C) {
      case 1: k_apply_tri<double, 1><<<blocks, 128, 0, bs>>>(L, x, b, out, gate); break;
      case 2: k_apply_tri<double, 2><<<blocks, 128, 0, bs>>>(L, x, b, out, gate); break;
      case 4: k_apply_tri<double, 4><<<blocks, 128, 0, bs>>>(L, x, b, out, gate); break;
      case 8: k_apply_tri<double, 8><<<blocks, 128, 0, bs>>>(L, x, b, out, gate); break;
      default: k_apply_tri<double, 16><<<blocks, 128, 0, bs>>>(L, x, b, out, gate); break;
    }
  }
  ck_launch();
}

// Capture one complete fgmres_solve (device-side loops) for fixed b, x:
//   init:  NaN test of b, ||b||, x = 0, v_0 = b / ||b||, g = (||b||, 0...)
//   WHILE (not done):                                 [condition set on the device]
//     v_j -> vin; z = V-cycle(vin) (coarse GMRES = nested WHILE); z -> Z_j
//     w = A z; CGS2 against V_0..V_j; Givens; v_{j+1} = w / h_{j+1,j}; step control
//     if the cycle closes: y = R^-1 g; x += Z y;  if not done: restart from b - A x
//   final: r = b - A x, ||r|| (the true residual)
// Issue the whole solve on stream s, which must be capturing.
void capture_solve(mg_handle *h, cudaStream_t s, const double *b, double *x, double rtol, int maxit, int m) {
  const long long len = h->lv[0].len;
  mg_handle::Krylov &K = h->kf;
  KState *st = h->kst_f;
  {
    h->launches = 0;
    ck(cudaMemsetAsync(h->flag + 1, 0, 2 * sizeof(int), s));
    {
      Bracket br(h, CAT_SMALL, s);
      k_check_finite<<<grid_for(len, 256), 256, 0, s>>>(b, len, h->flag + 1);
      ck_launch();
    }
    ck(cudaMemsetAsync(x, 0, len * sizeof(double), s));
    norm_into(h, K, b, len, s);
    float2 *Vp = h->pair_basis ? reinterpret_cast<float2 *>(h->fV) : nullptr;
    const cudaGraphConditionalHandle hdl = new_handle(s);
    {
      Bracket br(h, CAT_SMALL, s);
      k_ctl_start<<<1, 1, 0, s>>>(st, K.scal, rtol, hdl);
      ck_launch();
    }
    {
      Bracket br(h, CAT_AXPY, s);
      // fused copies: the basis vector is also written to the preconditioner's input slot
      double *vin_also = h->fuse_copies ? h->vin : nullptr;
      if (Vp)
        k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp, b, K.scal + 1, len, nullptr, 0, nullptr, vin_also);
      else
        k_scale<<<grid_for(len, 256), 256, 0, s>>>(h->fV, b, K.scal + 1, len, nullptr, 0, nullptr, vin_also);
      ck_launch();
    }
    {
      Bracket br(h, CAT_SMALL, s);
      k_arnoldi_init<<<1, 128, 0, s>>>(K.scal, K.g, m);
      ck_launch();
    }
    const long long n_init = h->launches;
    h->launches = 0;
    long long n_coarse = 0;
    add_while(h, s, hdl, h->cap[1], [&](cudaStream_t bs) {
      const bool fc = h->fuse_copies;  // the input and Z_j copies ride on the basis write and the product
      if (!fc) {
        Bracket br(h, CAT_SMALL, bs);
        if (Vp)
          k_join_basis<<<grid_for(len, 256), 256, 0, bs>>>(h->vin, Vp, len, &st->j);
        else
          k_copy_indexed<<<grid_for(len, 256), 256, 0, bs>>>(h->vin, h->fV, len, &st->j, 0);
        ck_launch();
      }
      const long long before = h->launches;
      precondition(h, h->vin, h->zout, bs);
      n_coarse = h->g_coarse;
      (void)before;
      if (!fc) {
        Bracket br(h, CAT_SMALL, bs);
        k_copy_indexed<<<grid_for(len, 256), 256, 0, bs>>>(h->fZ, h->zout, len, &st->j, 1);
        ck_launch();
      }
      launch_apply<double>(h, h->lv[0].d.view, h->zout, nullptr, h->fw, bs, 0, -1, fc ? h->fZ : nullptr, &st->j,
                           0);
      arnoldi_step_dev(h, K, st, m - 1, h->fV, len, h->fw, bs, Vp, fc ? h->vin : nullptr);
      {
        Bracket br(h, CAT_SMALL, bs);
        k_ctl_step<<<1, 1, 0, bs>>>(st, K.scal, m, maxit, 0, hdl);
        ck_launch();
      }
      // close the cycle (guarded by st->cycle_end) and restart if needed (st->restart)
      {
        Bracket br(h, CAT_SMALL, bs);
        k_backsolve<<<1, 256, (size_t)m * sizeof(double), bs>>>(0, K.H, h->ldh, K.g, K.ycoef, &st->kcount,
                                                                 &st->cycle_end);
        ck_launch();
      }
      multi_axpy(h, x, h->fZ, len, K.ycoef, m, 1.0, len, bs, &st->cycle_end, &st->kcount);
      launch_apply_gated(h, x, b, h->fr, &st->restart, bs);
      multidot(h, h->fr, len, 1, h->fr, len, K.nrm2, 0, bs, &st->restart);
      {
        Bracket br(h, CAT_SMALL, bs);
        k_norm_from_sq<<<1, 1, 0, bs>>>(K.nrm2, K.scal, &st->restart);
        ck_launch();
      }
      {
        Bracket br(h, CAT_AXPY, bs);
        if (Vp)
          k_split_basis<<<grid_for(len, 256), 256, 0, bs>>>(Vp, h->fr, K.scal + 1, len, nullptr, 0, &st->restart,
                                                            h->fuse_copies ? h->vin : nullptr);
        else
          k_scale<<<grid_for(len, 256), 256, 0, bs>>>(h->fV, h->fr, K.scal + 1, len, nullptr, 0, &st->restart,
                                                      h->fuse_copies ? h->vin : nullptr);
        ck_launch();
      }
      {
        Bracket br(h, CAT_SMALL, bs);
        k_arnoldi_init<<<1, 128, 0, bs>>>(K.scal, K.g, m, &st->restart);
        ck_launch();
      }
      {
        Bracket br(h, CAT_SMALL, bs);
        k_ctl_continue<<<1, 1, 0, bs>>>(st, hdl);
        ck_launch();
      }
    });
    const long long n_body = h->launches;
    h->launches = 0;
    launch_apply<double>(h, h->lv[0].d.view, x, b, h->fr, s);
    norm_into(h, K, h->fr, len, s);
    h->g_init = n_init + h->launches;
    h->g_body = n_body;
    h->g_coarse = n_coarse;
  }
}

// The graph of a DCGS2 solve (pair basis): as capture_solve, with the loop
// body of one DCGS2 step (section comment of k_multi_axpy2_pair):
//   v~_j -> vin (written with the previous step's split); z = V-cycle(vin); w = A z (and Z_j = z);
//   V^T [u, w] over the j final vectors and u . w; k_dcgs2_coef (column j - 1 finished and
//   rotated, the step's coefficients); k_dcgs2_ctl (a finished column that converged ends the
//   cycle; else the update pass runs and, on the cycle's last step, the closing pass follows);
//   [go] the update pass (final V_j, u = w', ||u||) and v~_{j+1} = u / ||u|| -> slot j + 1, vin;
//   [close] V^T u and column j - 1; then, as in capture_solve, the guarded cycle end
//   (least squares, x update) and restart (true residual, u = r, v~_0 = r / ||r||).
void capture_solve_dcgs2(mg_handle *h, cudaStream_t s, const double *b, double *x, double rtol, int maxit, int m) {
  const long long len = h->lv[0].len;
  mg_handle::Krylov &K = h->kf;
  KState *st = h->kst_f;
  float2 *Vp = reinterpret_cast<float2 *>(h->fV);
  double *dc = h->dcg + kDcS;
  h->launches = 0;
  ck(cudaMemsetAsync(h->flag + 1, 0, 2 * sizeof(int), s));
  {
    Bracket br(h, CAT_SMALL, s);
    k_check_finite<<<grid_for(len, 256), 256, 0, s>>>(b, len, h->flag + 1);
    ck_launch();
  }
  ck(cudaMemsetAsync(x, 0, len * sizeof(double), s));
  norm_into(h, K, b, len, s);
  const cudaGraphConditionalHandle hdl = new_handle(s);
  {
    Bracket br(h, CAT_SMALL, s);
    k_ctl_start<<<1, 1, 0, s>>>(st, K.scal, rtol, hdl);
    ck_launch();
    k_dcgs2_start<<<1, 32, 0, s>>>(K.scal, dc);
    ck_launch();
    k_copy_gated<<<grid_for(len, 256), 256, 0, s>>>(h->fu, b, len, nullptr);
    ck_launch();
  }
  {
    Bracket br(h, CAT_AXPY, s);
    k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp, b, dc, len, nullptr, 0, nullptr, h->vin);
    ck_launch();
  }
  {
    Bracket br(h, CAT_SMALL, s);
    k_arnoldi_init<<<1, 128, 0, s>>>(K.scal, K.g, m);
    ck_launch();
  }
  const long long n_init = h->launches;
  h->launches = 0;
  long long n_coarse = 0;
  add_while(h, s, hdl, h->cap[1], [&](cudaStream_t bs) {
    precondition(h, h->vin, h->zout, bs);
    n_coarse = h->g_coarse;
    launch_apply<double>(h, h->lv[0].d.view, h->zout, nullptr, h->fw, bs, 0, -1, h->fZ, &st->j, 0);
    multidot2_pair(h, Vp, len, m, h->fu, h->fw, len, K.h, bs, &st->j);
    multidot(h, h->fu, len, 1, h->fw, len, dc + 4, 0, bs);
    {
      Bracket br(h, CAT_SMALL, bs);
      k_dcgs2_coef<<<1, 32, 0, bs>>>(0, &st->j, K.h, dc, h->dcg + kDcC1, h->dcg + kDcC2, h->dcg + kDcHp, K.H,
                                     h->ldh, K.cs, K.sn, K.g, K.scal, 0);
      ck_launch();
      k_dcgs2_ctl<<<1, 1, 0, bs>>>(st, K.scal, m, maxit);
      ck_launch();
    }
    multi_axpy2_pair(h, Vp, len, m, h->fu, h->fw, h->dcg, bs, &st->j, &st->go);
    {
      Bracket br(h, CAT_AXPY, bs);
      k_split_basis<<<grid_for(len, 256), 256, 0, bs>>>(Vp, h->fu, dc, len, &st->j, 1, &st->go, h->vin);
      ck_launch();
    }
    {
      Bracket br(h, CAT_SMALL, bs);
      k_dcgs2_adv<<<1, 1, 0, bs>>>(st);
      ck_launch();
    }
    multidot_pair(h, Vp, len, m, h->fu, len, K.h, bs, &st->j, &st->close);
    {
      Bracket br(h, CAT_SMALL, bs);
      k_dcgs2_coef<<<1, 32, 0, bs>>>(0, &st->j, K.h, dc, h->dcg + kDcC1, h->dcg + kDcC2, h->dcg + kDcHp, K.H,
                                     h->ldh, K.cs, K.sn, K.g, K.scal, 1, &st->close);
      ck_launch();
      k_dcgs2_closed<<<1, 1, 0, bs>>>(st, K.scal, maxit);
      ck_launch();
    }
    {
      Bracket br(h, CAT_SMALL, bs);
      k_backsolve<<<1, 256, (size_t)m * sizeof(double), bs>>>(0, K.H, h->ldh, K.g, K.ycoef, &st->kcount,
                                                               &st->cycle_end);
      ck_launch();
    }
    multi_axpy(h, x, h->fZ, len, K.ycoef, m, 1.0, len, bs, &st->cycle_end, &st->kcount);
    launch_apply_gated(h, x, b, h->fr, &st->restart, bs);
    multidot(h, h->fr, len, 1, h->fr, len, K.nrm2, 0, bs, &st->restart);
    {
      Bracket br(h, CAT_SMALL, bs);
      k_norm_from_sq<<<1, 1, 0, bs>>>(K.nrm2, K.scal, &st->restart);
      ck_launch();
      k_dcgs2_start<<<1, 32, 0, bs>>>(K.scal, dc, &st->restart);
      ck_launch();
      k_copy_gated<<<grid_for(len, 256), 256, 0, bs>>>(h->fu, h->fr, len, &st->restart);
      ck_launch();
    }
    {
      Bracket br(h, CAT_AXPY, bs);
      k_split_basis<<<grid_for(len, 256), 256, 0, bs>>>(Vp, h->fr, dc, len, nullptr, 0, &st->restart, h->vin);
      ck_launch();
    }
    {
      Bracket br(h, CAT_SMALL, bs);
      k_arnoldi_init<<<1, 128, 0, bs>>>(K.scal, K.g, m, &st->restart);
      ck_launch();
      k_ctl_continue<<<1, 1, 0, bs>>>(st, hdl);
      ck_launch();
    }
  });
  const long long n_body = h->launches;
  h->launches = 0;
  launch_apply<double>(h, h->lv[0].d.view, x, b, h->fr, s);
  norm_into(h, K, h->fr, len, s);
  h->g_init = n_init + h->launches;
  h->g_body = n_body;
  h->g_coarse = n_coarse;
}

void build_solve_graph(mg_handle *h, const double *b, double *x, double rtol, int maxit, int m) {
  cudaStream_t s = h->cap[0];
  const long long saved = h->launches;
  h->capturing = 1;
  cudaGraph_t graph = nullptr;
  ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  try {
    if (h->dcgs2)
      capture_solve_dcgs2(h, s, b, x, rtol, maxit, m);
    else
      capture_solve(h, s, b, x, rtol, maxit, m);
    ck(cudaStreamEndCapture(s, &graph));
  } catch (...) {
    cudaStreamEndCapture(s, &graph);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    h->capturing = 0;
    h->launches = saved;
    throw;
  }
  h->capturing = 0;
  h->launches = saved;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph = graph;
  h->gexec = nullptr;
  ck(cudaGraphInstantiate(&h->gexec, graph, 0));
  h->gkey.b = b;
  h->gkey.x = x;
  h->gkey.rtol = rtol;
  h->gkey.maxit = maxit;
  h->gkey.restart = m;
  h->gkey.gen = h->gen;
}

// workspace of a solve with restart m (grown on demand)
void prepare_solve(mg_handle *h, int m, cudaStream_t s) {
  ensure_fgmres_space(h, m, s);
  // a solve that stopped early (a timed-out wait) may have left a count behind
  ck(cudaMemsetAsync(h->ticket, 0, 4 * sizeof(unsigned), s));
  if (!h->fw) {
    const long long len = h->lv[0].len;
    h->fw = h->mem.alloc<double>(len);
    h->fr = h->mem.alloc<double>(len);
    h->fx_stage = h->mem.alloc<double>(len);
    h->fb_stage = h->mem.alloc<double>(len);
  }
  h->coarse_learned = 0;
  if (h->net) {
    if (h->net_bf16) net_refresh_bf16(h->net, s);
    ck(cudaMemsetAsync(h->net_flag, 0, 2 * sizeof(int), s));
  }
}

// the graph of a batch of solves (one branch per system), cached per host thread
struct BatchGraph {
  std::vector<mg_handle *> hs;
  std::vector<const double *> b;
  std::vector<double *> x;
  std::vector<int> gen;
  double rtol = -1.0;
  int maxit = 0, restart = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t root = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  ~BatchGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : joins) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (root) cudaStreamDestroy(root);
  }
};
thread_local BatchGraph g_batch;

bool is_device_pointer(const void *p) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ===========================================================================
// Arithmetic-rate probe (measurement support): every thread runs kProbeChains
// independent FMA chains a <- a * b + c for `iters` steps and stores their sum,
// so the work cannot be removed; 2 * kProbeChains * iters flops per thread.
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(T *sink, int iters, T b, T c) {
  T a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  }
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) acc += a[k];
  sink[blockIdx.x * (long long)blockDim.x + threadIdx.x] = acc;
}

// ===========================================================================
// C ABI

extern "C" {

void mg_default_options(mg_options *o) {
  if (!o) return;
  o->levels = 2;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->coarse_rtol = 1e-3;
  o->coarse_maxit = 50;
  o->coarse_fixed_iters = 0;
  o->end_rule = 0;
  o->precision = MG_PRECISION_FP64;
  o->omega = 1.0;
  o->coarse_precond = MG_COARSE_SGS;
  o->device_loops = 1;
  o->krylov_basis = MG_BASIS_FP64;
  o->restrict_rule = MG_RESTRICT_INJECT;
}

const char *mg_status_string(int st) {
  switch (st) {
    case MG_OK: return "ok";
    case MG_NOT_CONVERGED: return "not converged within maxit";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_SINGULAR: return "singular local Schur complement (N_k not invertible)";
    case MG_ERR_BREAKDOWN: return "Arnoldi breakdown (non-finite Hessenberg entry)";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_OOM: return "device out of memory";
    case MG_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case MG_ERR_NONFINITE: return "NaN or Inf in the input";
    case MG_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char *mg_last_cuda_error(void) { return g_last_cuda_error; }

long long mg_vector_length(const mg_handle *h) { return h ? h->lv[0].len : 0; }

long long mg_launch_count(const mg_handle *h) { return h ? h->launches : 0; }

int mg_graph_launches(const mg_handle *h, long long *fixed, long long *per_iter, long long *per_coarse_iter) {
  const bool ok = h && h->graph;
  if (fixed) *fixed = ok ? h->g_init : 0;
  if (per_iter) *per_iter = ok ? h->g_body : 0;
  if (per_coarse_iter) *per_coarse_iter = ok ? h->g_coarse : 0;
  return ok ? MG_OK : MG_ERR_ARG;
}

int mg_probe_fma(int precision, int blocks, int iters, void *sink, void *stream) {
  if (blocks < 1 || blocks > (1 << 20) || iters < 1 || !sink) return MG_ERR_ARG;
  if (precision != MG_PRECISION_FP64 && precision != MG_PRECISION_FP32) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == MG_PRECISION_FP64)
    k_probe_fma<double><<<blocks, kProbeThreads, 0, s>>>(static_cast<double *>(sink), iters, 0.9999999, 1e-9);
  else
    k_probe_fma<float><<<blocks, kProbeThreads, 0, s>>>(static_cast<float *>(sink), iters, 0.9999999f, 1e-9f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

int mg_profile_enable(mg_handle *h, int enable) {
  if (!h) return MG_ERR_ARG;
  try {
    harvest(h);
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  }
  h->prof = enable;
  for (int c = 0; c < 16; ++c) {
    h->prof_ms[c] = 0.0;
    h->prof_count[c] = 0;
    h->work_bytes[c] = 0.0;
    h->work_flops[c] = 0.0;
  }
  return MG_OK;
}

int mg_profile_read(mg_handle *h, int max, const char **names, double *ms, long long *launches, double *bytes,
                    double *flops) {
  if (!h || max < 0) return MG_ERR_ARG;
  try {
    harvest(h);
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  }
  const int k = std::min<int>(max, CAT_COUNT);
  for (int c = 0; c < k; ++c) {
    if (names) names[c] = kCatNames[c];
    if (ms) ms[c] = h->prof_ms[c];
    if (launches) launches[c] = h->prof_count[c];
    if (bytes) bytes[c] = h->work_bytes[c];
    if (flops) flops[c] = h->work_flops[c];
  }
  return CAT_COUNT;
}

void mg_destroy(mg_handle *h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto &pe : h->ev_pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (cudaStream_t cs : h->cap)
    if (cs) cudaStreamDestroy(cs);
  h->mem.release();
  for (void *p : h->fmem) cudaFree(p);
  if (h->host_scal) cudaFreeHost(h->host_scal);
  delete h;
}

int mg_setup(const mg_problem *P, const mg_options *O, void *stream, mg_handle **out) {
  if (!out) return MG_ERR_ARG;
  *out = nullptr;
  if (!P || !O) return MG_ERR_ARG;
  g_last_cuda_error[0] = 0;
  const int n = P->n, p = P->p, q = P->q, layout = P->layout;
  if (n < 1 || p < 1 || q < 1) return MG_ERR_ARG;
  if (!(P->theta > 0.0 && P->theta <= 1.0) || !(P->gamma > 0.0)) return MG_ERR_ARG;
  if (layout != MG_LAYOUT_DENSE && layout != MG_LAYOUT_TRIDIAG) return MG_ERR_ARG;
  if (!P->M || !P->Ju_cur || !P->Ju_prev || !P->Jz_cur || !P->Jz_prev) return MG_ERR_ARG;
  if (O->levels < 1 || O->levels > 30 || O->nu_pre < 0 || O->nu_post < 0) return MG_ERR_ARG;
  if (O->coarse_maxit < 1 || O->coarse_maxit > 64 || O->coarse_fixed_iters < 0 || O->coarse_fixed_iters > 64)
    return MG_ERR_ARG;
  if (O->end_rule != 0 && O->end_rule != 1) return MG_ERR_ARG;
  if (O->precision != MG_PRECISION_FP64 && O->precision != MG_PRECISION_FP32 &&
      O->precision != MG_PRECISION_FP32_SMOOTH && O->precision != MG_PRECISION_BF16_BANDS)
    return MG_ERR_ARG;
  if (O->precision == MG_PRECISION_BF16_BANDS && layout != MG_LAYOUT_TRIDIAG) return MG_ERR_UNSUPPORTED;
  if (!(O->omega > 0.0 && O->omega <= 1.0)) return MG_ERR_ARG;
  if (O->coarse_precond < MG_COARSE_SGS || O->coarse_precond > MG_COARSE_BGS) return MG_ERR_ARG;
  if (O->device_loops != 0 && O->device_loops != 1) return MG_ERR_ARG;
  if (O->krylov_basis != MG_BASIS_FP64 && O->krylov_basis != MG_BASIS_PAIR && O->krylov_basis != MG_BASIS_PAIR_DCGS2)
    return MG_ERR_ARG;
  if (O->restrict_rule != MG_RESTRICT_INJECT && O->restrict_rule != MG_RESTRICT_TRANSPOSE) return MG_ERR_ARG;
  if (n % (1 << (O->levels - 1)) != 0) return MG_ERR_ARG;
  if (O->levels > 1 && P->separable != 1) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error,
                  "mg_setup: coarse levels need a separable problem (separable = 1)");
    return MG_ERR_ARG;
  }
  if (layout == MG_LAYOUT_TRIDIAG && q != p) return MG_ERR_ARG;
  if (layout == MG_LAYOUT_DENSE && (p > kDenseWarpMax || q > kDenseWarpMax)) return MG_ERR_UNSUPPORTED;
  if (layout == MG_LAYOUT_TRIDIAG && p > 32 * 16) return MG_ERR_UNSUPPORTED;

  const int msz = layout == MG_LAYOUT_DENSE ? p * p : 3 * p;
  const int zsz = layout == MG_LAYOUT_DENSE ? p * q : 3 * p;
  const long long nz = P->jz_const ? 1 : n;
  if (!host_finite(P->M, msz) || !host_finite(P->Ju_cur, (long long)n * msz) ||
      !host_finite(P->Ju_prev, (long long)n * msz) || !host_finite(P->Jz_cur, nz * zsz) ||
      !host_finite(P->Jz_prev, nz * zsz))
    return MG_ERR_NONFINITE;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mg_handle *h = new (std::nothrow) mg_handle();
  if (!h) return MG_ERR_OOM;
  h->opts = *O;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return MG_ERR_CUDA;
  }
  h->layout = layout;
  h->n = n;
  h->p = p;
  h->q = q;
  h->theta = P->theta;
  h->gamma = P->gamma;
  int C = 1;
  while (32 * C < p) C *= 2;
  h->C = C;
  // SGS chain implementation: "scan" (default), "cluster" or "serial"; the
  // environment variable PINTMG_SGS_CHAIN selects one (used by the tests)
  if (const char *e = std::getenv("PINTMG_SGS_CHAIN")) {
    if (std::strcmp(e, "cluster") == 0) h->use_scan = 0, h->use_seg = 0;
    if (std::strcmp(e, "serial") == 0) h->use_scan = 0, h->use_cluster = 0, h->use_seg = 0;
    if (std::strcmp(e, "segmented") == 0) h->use_scan = 0;
  }
  // PINTMG_STAGE_TRI=0 turns the shared-memory staging of the block solves off (tests)
  if (const char *e = std::getenv("PINTMG_STAGE_TRI")) h->stage_tri = std::atoi(e) != 0;
  // PINTMG_TRI_PAIR=0 keeps one warp per block on every level (tests)
  if (const char *e = std::getenv("PINTMG_TRI_PAIR")) h->pair_tri = std::atoi(e) != 0;
  if (const char *e = std::getenv("PINTMG_SPLIT_BS")) h->split_bs = std::atoi(e) != 0;
  // PINTMG_FUSE_COPIES=0: captured solves copy the preconditioner's input and output in kernels of their own
  if (const char *e = std::getenv("PINTMG_FUSE_COPIES")) h->fuse_copies = std::atoi(e) != 0;
  // PINTMG_FUSE_REDUCE=0 reduces dot products and forms the Arnoldi column in separate launches,
  // 2 fuses every dot product's reduction (tests, measurements); 1 is the default
  if (const char *e = std::getenv("PINTMG_FUSE_REDUCE")) h->fuse_reduce = std::min(2, std::max(0, std::atoi(e)));
  // PINTMG_PERSIST=1 runs each smoothing of a level that fits on the GPU as one cooperative
  // launch (k_sweeps_tri2); 0 (the default) launches every block-Jacobi sweep separately
  if (const char *e = std::getenv("PINTMG_PERSIST")) h->persist_sweeps = std::atoi(e) != 0;
  // PINTMG_TEST_SWEEP_STALL=1 (tests of the bounded waits): the multi-sweep kernel's
  // block 0 never publishes its coupling, so block 1's wait runs out (2 s) and the
  // solve returns MG_ERR_TIMEOUT; the handle stays unusable for solves afterwards
  if (const char *e = std::getenv("PINTMG_TEST_SWEEP_STALL")) h->sweep_stall = std::atoi(e) != 0;
  // PINTMG_TEST_PAIR_STALL=1 (tests of the bounded waits): the pair multi-dot's
  // producer issues nothing, so its consumers give up after 2 s and the solve
  // returns MG_ERR_TIMEOUT
  if (const char *e = std::getenv("PINTMG_TEST_PAIR_STALL")) h->pair_stall = std::min(2, std::max(0, std::atoi(e)));
  // dot-product blocking (4, 8 or 16 basis vectors per CTA; bitwise the same
  // results): PINTMG_DOT_VB overrides the default (used by the tests)
  if (const char *e = std::getenv("PINTMG_DOT_VB")) {
    const int vb = std::atoi(e);
    if (vb == 4 || vb == 8 || vb == 16) h->dot_vb = vb;
  }
  int status = MG_OK;
  try {
    ck(cudaMallocHost(&h->host_scal, 4 * sizeof(double)));
    tri_stage_prepare();
    // the pair basis streams two entries per 16-byte load: even vector lengths only
    h->pair_basis = (O->krylov_basis == MG_BASIS_PAIR || O->krylov_basis == MG_BASIS_PAIR_DCGS2) &&
                    ((long long)n * (4 * p + q)) % 2 == 0;
    h->dcgs2 = h->pair_basis && O->krylov_basis == MG_BASIS_PAIR_DCGS2;
    if (h->pair_basis) pair_prepare();
    // raw data on the device (FP64)
    double *dM = h->mem.alloc<double>(msz);
    double *dJuc = h->mem.alloc<double>((size_t)n * msz);
    double *dJup = h->mem.alloc<double>((size_t)n * msz);
    double *dJzc = h->mem.alloc<double>((size_t)nz * zsz);
    double *dJzp = h->mem.alloc<double>((size_t)nz * zsz);
    ck(cudaMemcpyAsync(dM, P->M, msz * sizeof(double), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dJuc, P->Ju_cur, (size_t)n * msz * sizeof(double), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dJup, P->Ju_prev, (size_t)n * msz * sizeof(double), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dJzc, P->Jz_cur, (size_t)nz * zsz * sizeof(double), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dJzp, P->Jz_prev, (size_t)nz * zsz * sizeof(double), cudaMemcpyHostToDevice, s));
    h->flag = h->mem.alloc<int>(4);
    ck(cudaMemsetAsync(h->flag, 0, 4 * sizeof(int), s));
    h->ticket = h->mem.alloc<unsigned>(4);
    ck(cudaMemsetAsync(h->ticket, 0, 4 * sizeof(unsigned), s));

    // index maps per level (injection reading of the coarse linearisation points)
    std::vector<int> cur(n), prev(n);
    for (int t = 0; t < n; ++t) cur[t] = prev[t] = t;
    const int L = O->levels;
    h->lv.resize(L);
    std::vector<int *> idx_dev;
    // theta = 1 and a constant d_z f = c M (tridiagonal layout): on every level
    // V = -M / dt and Z = -c M / gamma, so V = kappa Z with kappa = gamma / (c dt)
    double prop_c = 0.0;
    if (layout == MG_LAYOUT_TRIDIAG && P->theta == 1.0 && P->jz_const) {
      int i0 = -1;
      for (int i = 0; i < msz; ++i)
        if (P->M[i] != 0.0) {
          i0 = i;
          break;
        }
      if (i0 >= 0) {
        const double c = P->Jz_cur[i0] / P->M[i0];
        bool ok = c != 0.0 && std::isfinite(c);
        for (int i = 0; ok && i < msz; ++i)
          ok = std::fabs(P->Jz_cur[i] - c * P->M[i]) <= 1e-15 * std::fabs(c * P->M[i]);
        if (ok) prop_c = c;
      }
    }
    double dt = 1.0 / n;
    int nl = n;
    for (int l = 0; l < L; ++l) {
      Level &lev = h->lv[l];
      lev.n = nl;
      lev.dt = dt;
      lev.len = (long long)nl * (4 * p + q);
      int *dcur = h->mem.alloc<int>(nl), *dprev = h->mem.alloc<int>(nl);
      ck(cudaMemcpyAsync(dcur, cur.data(), nl * sizeof(int), cudaMemcpyHostToDevice, s));
      ck(cudaMemcpyAsync(dprev, prev.data(), nl * sizeof(int), cudaMemcpyHostToDevice, s));
      // the host vectors must outlive the async copies
      ck(cudaStreamSynchronize(s));
      double *N = h->mem.alloc<double>((size_t)nl * msz);
      double *V = h->mem.alloc<double>((size_t)nl * msz);
      double *Z = h->mem.alloc<double>((size_t)nl * zsz);
      const long long work = (long long)nl * (2 * msz + zsz);
      k_form_blocks<<<grid_for(work, 256, 1 << 20), 256, 0, s>>>(
          nl, msz, zsz, layout == MG_LAYOUT_TRIDIAG ? p : 0, P->theta, dt, P->gamma, dM, dJuc, dJup, dJzc, dJzp,
          P->jz_const, dcur, dprev, N, V, Z);
      ck_launch();
      LevelView<double> &v = lev.d.view;
      v.n = nl;
      v.p = p;
      v.q = q;
      v.layout = layout;
      v.N = N;
      v.V = V;
      v.Z = Z;
      v.sN = msz;
      v.sV = msz;
      v.sZ = zsz;
      v.kappa = prop_c != 0.0 ? P->gamma / (prop_c * dt) : 0.0;
      if (layout == MG_LAYOUT_TRIDIAG) {
        double *fac = h->mem.alloc<double>((size_t)nl * 3 * p);
        double *scan = h->mem.alloc<double>((size_t)nl * kScanPerBlock);
        k_factor_tri<<<grid_for(nl, 64, 1 << 20), 64, 0, s>>>(nl, p, C, N, msz, Z, zsz, fac, scan, h->flag);
        ck_launch();
        v.fac = fac;
        v.sFac = 3 * p;
        v.scan = scan;
      } else {
        double *fac = h->mem.alloc<double>((size_t)nl * p * p);
        if (p > kDenseMax || q > kDenseMax)
          k_factor_dw<<<(nl + 3) / 4, 128, 0, s>>>(nl, p, q, N, msz, Z, zsz, fac, h->flag);
        else
          k_factor_dense<<<grid_for(nl, 64, 1 << 20), 64, 0, s>>>(nl, p, q, N, msz, Z, zsz, fac, h->flag);
        ck_launch();
        v.fac = fac;
        v.sFac = (long long)p * p;
        v.scan = nullptr;
      }
      if (l == L - 1) {
        lev.d.Cu = h->mem.alloc<double>((size_t)nl * p * p);
        lev.d.Em = h->mem.alloc<double>((size_t)nl * p * p);
        if (nl > 1) {
          if (layout == MG_LAYOUT_TRIDIAG) {
            const long long warps = (long long)(nl - 1) * p;
            const int blocks = (int)((warps + 3) / 4);
            switch (C) {
              case 1: k_chain_mats_tri<1><<<blocks, 128, 0, s>>>(v, lev.d.Cu, lev.d.Em); break;
              case 2: k_chain_mats_tri<2><<<blocks, 128, 0, s>>>(v, lev.d.Cu, lev.d.Em); break;
              case 4: k_chain_mats_tri<4><<<blocks, 128, 0, s>>>(v, lev.d.Cu, lev.d.Em); break;
              case 8: k_chain_mats_tri<8><<<blocks, 128, 0, s>>>(v, lev.d.Cu, lev.d.Em); break;
              default: k_chain_mats_tri<16><<<blocks, 128, 0, s>>>(v, lev.d.Cu, lev.d.Em); break;
            }
          } else {
            if (p > kDenseMax || q > kDenseMax)
              k_chain_mats_dw<<<(nl - 1 + 3) / 4, 128, 0, s>>>(v, lev.d.Cu, lev.d.Em);
            else
              k_chain_mats_dense<<<grid_for(nl - 1, 64, 1 << 20), 64, 0, s>>>(v, lev.d.Cu, lev.d.Em);
          }
          ck_launch();
        }
        // prefix products for the parallel-scan SGS chains (budget: 8 GiB in FP64)
        int R = 0;
        while ((1 << R) < nl) ++R;
        const double bytes = 2.0 * R * (double)nl * p * p * sizeof(double);
        if (nl > 1 && bytes <= 8.0 * (1 << 30)) {
          for (int dir = 0; dir < 2; ++dir) {
            std::vector<double *> &Pv = dir == 0 ? lev.d.scanF : lev.d.scanB;
            for (int dd = 0; dd < R; ++dd) Pv.push_back(h->mem.alloc<double>((size_t)nl * p * p));
            k_scan_init<<<grid_for((long long)nl * p * p, 256, 1 << 20), 256, 0, s>>>(
                dir == 0 ? lev.d.Cu : lev.d.Em, Pv[0], nl, p, dir);
            ck_launch();
            for (int dd = 0; dd + 1 < R; ++dd) {
              const int shift = 1 << dd;
              if (nl - 2 * shift <= 0) continue;
              dim3 grid((p + 31) / 32, (p + 31) / 32, nl - 2 * shift);
              k_scan_products<<<grid, 256, 0, s>>>(Pv[dd], Pv[dd + 1], nl, p, shift);
              ck_launch();
            }
          }
          lev.d.scan_tmp = h->mem.alloc<double>((size_t)nl * p);
        }
        // segmented chains: in-segment products Q (one p x p per position, 2 n p^2 values in
        // all), up to 16 segments of >= 16 steps.  They serve when the full scan does not
        // fit, and as a candidate of the autotuner (mg_autotune) when it does
        const double seg_bytes = 2.0 * (double)nl * p * p * sizeof(double);
        if (layout == MG_LAYOUT_TRIDIAG && p >= 32 && nl >= 32 && seg_bytes <= 8.0 * (1 << 30)) {
          const int nseg = std::min(16, nl / 16);
          const int L = (nl + nseg - 1) / nseg;
          lev.d.seg_len = L;
          lev.d.segF = h->mem.alloc<double>((size_t)nl * p * p);
          lev.d.segB = h->mem.alloc<double>((size_t)nl * p * p);
          const dim3 grid((p + 31) / 32, (p + 31) / 32, nseg - 1);
          for (int t = 0; t < L; ++t) {
            k_seg_products<<<grid, 256, 0, s>>>(lev.d.Cu, lev.d.segF, nl, p, L, t, 0);
            ck_launch();
            k_seg_products<<<grid, 256, 0, s>>>(lev.d.Em, lev.d.segB, nl, p, L, t, 1);
            ck_launch();
          }
        }
      }
      alloc_level_vectors<double>(h, lev, lev.d, l == L - 1, l == 0, s);
      if (O->precision != MG_PRECISION_FP64) {
        LevelView<float> &f = lev.f.view;
        f.n = nl;
        f.p = p;
        f.q = q;
        f.layout = layout;
        f.N = to_float_copy(h, N, (long long)nl * msz, s);
        f.V = to_float_copy(h, V, (long long)nl * msz, s);
        f.Z = to_float_copy(h, Z, (long long)nl * zsz, s);
        f.sN = v.sN;
        f.sV = v.sV;
        f.sZ = v.sZ;
        f.kappa = (float)v.kappa;
        f.fac = to_float_copy(h, v.fac, (long long)nl * v.sFac, s);
        f.sFac = v.sFac;
        f.scan = layout == MG_LAYOUT_TRIDIAG ? to_float_copy(h, v.scan, (long long)nl * kScanPerBlock, s)
                                             : nullptr;
        if (O->precision == MG_PRECISION_BF16_BANDS && l < L - 1) {
          // smoothing levels read their N, V, Z bands as BF16 (rounded from the FP32 copies);
          // the factor, the scan compositions and the coarsest level stay FP32
          LevelView<float, __nv_bfloat16> &vh = lev.f.vh;
          vh.n = nl;
          vh.p = p;
          vh.q = q;
          vh.layout = layout;
          vh.N = to_bf16_copy(h, f.N, (long long)nl * msz, s);
          vh.V = to_bf16_copy(h, f.V, (long long)nl * msz, s);
          vh.Z = to_bf16_copy(h, f.Z, (long long)nl * zsz, s);
          vh.sN = f.sN;
          vh.sV = f.sV;
          vh.sZ = f.sZ;
          vh.kappa = 0.0f;  // the rounded V is no longer a multiple of the rounded Z: both are read
          // the local factor of the rounded blocks (FP64, then FP32), so that each sweep solves
          // the rounded D_k exactly up to FP32 rounding
          double *Nr = h->mem.alloc<double>((size_t)nl * msz), *Zr = h->mem.alloc<double>((size_t)nl * zsz);
          {
            Bracket br(h, CAT_CONVERT, s);
            k_bf16_to_double<<<grid_for((long long)nl * msz, 256), 256, 0, s>>>(vh.N, Nr, (long long)nl * msz);
            ck_launch();
          }
          {
            Bracket br(h, CAT_CONVERT, s);
            k_bf16_to_double<<<grid_for((long long)nl * zsz, 256), 256, 0, s>>>(vh.Z, Zr, (long long)nl * zsz);
            ck_launch();
          }
          double *facr = h->mem.alloc<double>((size_t)nl * 3 * p);
          double *scanr = h->mem.alloc<double>((size_t)nl * kScanPerBlock);
          k_factor_tri<<<grid_for(nl, 64, 1 << 20), 64, 0, s>>>(nl, p, C, Nr, msz, Zr, zsz, facr, scanr, h->flag);
          ck_launch();
          vh.fac = to_float_copy(h, facr, (long long)nl * 3 * p, s);
          vh.sFac = 3 * p;
          vh.scan = to_float_copy(h, scanr, (long long)nl * kScanPerBlock, s);
          lev.f.bands16 = true;
        }
        if (l == L - 1) {
          lev.f.Cu = to_float_copy(h, lev.d.Cu, (long long)nl * p * p, s);
          lev.f.Em = to_float_copy(h, lev.d.Em, (long long)nl * p * p, s);
          for (double *P : lev.d.scanF) lev.f.scanF.push_back(to_float_copy(h, P, (long long)nl * p * p, s));
          for (double *P : lev.d.scanB) lev.f.scanB.push_back(to_float_copy(h, P, (long long)nl * p * p, s));
          if (lev.d.segF) {
            lev.f.segF = to_float_copy(h, lev.d.segF, (long long)nl * p * p, s);
            lev.f.segB = to_float_copy(h, lev.d.segB, (long long)nl * p * p, s);
            lev.f.seg_len = lev.d.seg_len;
          }
          if (lev.d.scan_tmp) lev.f.scan_tmp = h->mem.alloc<float>((size_t)nl * p);
        }
        alloc_level_vectors<float>(h, lev, lev.f, l == L - 1, l == 0, s);
      }
      // next level's maps: coarse K <- fine 2K (current), max(2K-1, 0) (previous)
      if (l + 1 < L) {
        const int nc = nl / 2;
        std::vector<int> c2(nc), p2(nc);
        for (int K = 0; K < nc; ++K) {
          c2[K] = cur[2 * K];
          p2[K] = prev[std::max(2 * K - 1, 0)];
        }
        cur.swap(c2);
        prev.swap(p2);
        nl = nc;
        dt *= 2.0;
      }
    }
    // coarse GMRES workspace
    Level &cl = h->lv.back();
    h->cmax = std::max(O->coarse_maxit, O->coarse_fixed_iters);
    h->cV = h->mem.alloc<double>((size_t)(h->cmax + 1) * cl.len);
    h->cZ = h->mem.alloc<double>((size_t)h->cmax * cl.len);
    h->cw = h->mem.alloc<double>(cl.len);
    h->cr = h->mem.alloc<double>(cl.len);
    h->cy = h->mem.alloc<double>(cl.len);
    // small buffers (sized for restarts up to 512)
    h->ldh = 513;
    h->partial = h->mem.alloc<double>((size_t)h->G * 512);
    for (mg_handle::Krylov *K : {&h->kf, &h->kc}) {
      K->h = h->mem.alloc<double>(1024);
      K->H = h->mem.alloc<double>((size_t)h->ldh * 512);
      K->cs = h->mem.alloc<double>(512);
      K->sn = h->mem.alloc<double>(512);
      K->g = h->mem.alloc<double>(513);
      K->ycoef = h->mem.alloc<double>(512);
      K->scal = h->mem.alloc<double>(8);
      K->nrm2 = h->mem.alloc<double>(8);
    }
    // graph-captured solves: loop states, fixed preconditioner slots, capture streams
    h->kst_f = h->mem.alloc<KState>(1);
    h->kst_c = h->mem.alloc<KState>(1);
    ck(cudaMemsetAsync(h->kst_f, 0, sizeof(KState), s));
    ck(cudaMemsetAsync(h->kst_c, 0, sizeof(KState), s));
    h->vin = h->mem.alloc<double>(h->lv[0].len);
    h->zout = h->mem.alloc<double>(h->lv[0].len);
    h->cvin = h->mem.alloc<double>(cl.len);
    h->czout = h->mem.alloc<double>(cl.len);
    for (cudaStream_t &cs : h->cap) ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int flag = 0;
    ck(cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    if (flag) status = MG_ERR_SINGULAR;
  } catch (const CudaFail &) {
    status = MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    status = MG_ERR_OOM;
  }
  if (status != MG_OK) {
    mg_destroy(h);
    return status;
  }
  *out = h;
  return MG_OK;
}

int mg_vcycle(mg_handle *h, const double *r, double *y, void *stream) {
  if (!h || !r || !y || r == y) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int tmo = 0;
  try {
    ck(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), s));
    precondition(h, r, y, s);
    ck(cudaMemcpyAsync(&tmo, h->flag + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    return MG_ERR_OOM;
  }
  return tmo ? MG_ERR_TIMEOUT : MG_OK;
}

int fgmres_solve(mg_handle *h, const double *b_in, double *x_out, double rtol, int maxit, int restart,
                 mg_solve_info *info, void *stream) {
  if (!h || !b_in || !x_out || maxit < 1 || restart < 1 || restart > 512 || !(rtol >= 0.0)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long len = h->lv[0].len;
  int status = MG_OK;
  h->vcycles = 0;
  h->coarse_iters = 0;
  int total = 0;
  double est_rel = 1.0, true_rel = 0.0;
  try {
    const int m = std::min(restart, maxit);
    prepare_solve(h, m, s);
    const bool b_dev = is_device_pointer(b_in), x_dev = is_device_pointer(x_out);
    const double *b = b_in;
    if (!b_dev) {
      ck(cudaMemcpyAsync(h->fb_stage, b_in, len * sizeof(double), cudaMemcpyHostToDevice, s));
      b = h->fb_stage;
    }
    double *x = x_dev ? x_out : h->fx_stage;
    if (h->opts.device_loops) {
      // one CUDA graph per solve: loops on the device, one read-back at the end
      if (!h->gexec || h->gkey.b != b || h->gkey.x != x || h->gkey.rtol != rtol || h->gkey.maxit != maxit ||
          h->gkey.restart != m || h->gkey.gen != h->gen) {
        ck(cudaStreamSynchronize(s));
        build_solve_graph(h, b, x, rtol, maxit, m);
      }
      KState before_c{};
      ck(cudaMemcpyAsync(&before_c, h->kst_c, sizeof(KState), cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      ck(cudaGraphLaunch(h->gexec, s));
      KState fs{}, cs{};
      int bad[2] = {0, 0};
      ck(cudaMemcpyAsync(&fs, h->kst_f, sizeof(KState), cudaMemcpyDeviceToHost, s));
      ck(cudaMemcpyAsync(&cs, h->kst_c, sizeof(KState), cudaMemcpyDeviceToHost, s));
      ck(cudaMemcpyAsync(bad, h->flag + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      ck(cudaMemcpyAsync(h->host_scal, h->kf.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (h->net) ck(cudaMemcpyAsync(&h->coarse_learned, h->net_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
      if (!x_dev) ck(cudaMemcpyAsync(x_out, x, len * sizeof(double), cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      total = fs.total;
      h->vcycles = fs.total;
      h->coarse_iters = (int)(cs.iters_all - before_c.iters_all);
      h->launches += h->g_init + h->g_body * (h->dcgs2 ? fs.bodies : fs.total) +
                     h->g_coarse * (cs.iters_all - before_c.iters_all);
      if (bad[0]) throw 1;
      const double bnorm = fs.bnorm;
      if (bnorm > 0.0) {
        true_rel = h->host_scal[0] / bnorm;
        est_rel = fs.est / bnorm;
        if (fs.breakdown) status = MG_ERR_BREAKDOWN;
        else if (!fs.converged) status = MG_NOT_CONVERGED;
        if (bad[1]) status = MG_ERR_TIMEOUT;
      } else {
        est_rel = 0.0;
        true_rel = 0.0;
      }
    } else {
    ck(cudaMemsetAsync(h->flag + 1, 0, 2 * sizeof(int), s));
    {
      Bracket br(h, CAT_SMALL, s);
      k_check_finite<<<grid_for(len, 256), 256, 0, s>>>(b, len, h->flag + 1);
      ck_launch();
    }
    float2 *Vp = h->pair_basis ? reinterpret_cast<float2 *>(h->fV) : nullptr;
    int bad = 0;
    ck(cudaMemcpyAsync(&bad, h->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    mg_handle::Krylov &K = h->kf;
    norm_into(h, K, b, len, s);
    read_scal(h, K, s);
    if (bad) throw 1;
    const double bnorm = h->host_scal[0];
    ck(cudaMemsetAsync(x, 0, len * sizeof(double), s));
    if (bnorm > 0.0) {
      const double *r = b;
      bool done = false;
      while (!done && total < maxit && h->dcgs2) {
        // DCGS2 cycle (pair basis): slot 0 = r / ||r|| is the tentative v_0, u = r, eta = ||r||
        double *dc = h->dcg + kDcS;
        norm_into(h, K, r, len, s);
        {
          Bracket br(h, CAT_SMALL, s);
          k_dcgs2_start<<<1, 32, 0, s>>>(K.scal, dc);
          ck_launch();
        }
        ck(cudaMemcpyAsync(h->fu, r, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
        {
          Bracket br(h, CAT_AXPY, s);
          k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp, r, dc, len);
          ck_launch();
        }
        {
          Bracket br(h, CAT_SMALL, s);
          k_arnoldi_init<<<1, 128, 0, s>>>(K.scal, K.g, m);
          ck_launch();
        }
        const int mm = std::min(m, maxit - total);
        int k = 0;
        bool lag_closed = false;  // the cycle ended at a column finished by a step (no closing pass)
        for (int j = 0; j < mm; ++j) {
          double *zj = h->fZ + (long long)j * len;
          {
            Bracket br(h, CAT_SMALL, s);
            k_join_basis<<<grid_for(len, 256), 256, 0, s>>>(h->vin, Vp + (long long)j * len, len);
            ck_launch();
          }
          precondition(h, h->vin, zj, s);
          launch_apply<double>(h, h->lv[0].d.view, zj, nullptr, h->fw, s);
          multidot2_pair(h, Vp, len, j, h->fu, h->fw, len, K.h, s);
          multidot(h, h->fu, len, 1, h->fw, len, dc + 4, 0, s);
          {
            Bracket br(h, CAT_SMALL, s);
            k_dcgs2_coef<<<1, 32, 0, s>>>(j, nullptr, K.h, dc, h->dcg + kDcC1, h->dcg + kDcC2, h->dcg + kDcHp, K.H,
                                          h->ldh, K.cs, K.sn, K.g, K.scal, 0);
            ck_launch();
          }
          if (j >= 1) {  // column j - 1 is final: its residual estimate
            read_scal(h, K, s);
            k = j;
            const double est = h->host_scal[0], hj1 = h->host_scal[2];
            if (!std::isfinite(est) || !std::isfinite(hj1)) {
              status = MG_ERR_BREAKDOWN;
              done = true;
              lag_closed = true;
              break;
            }
            est_rel = est / bnorm;
            if (est <= rtol * bnorm || hj1 == 0.0) {
              done = true;
              lag_closed = true;
              break;
            }
          }
          multi_axpy2_pair(h, Vp, len, j, h->fu, h->fw, h->dcg, s);
          {
            Bracket br(h, CAT_AXPY, s);
            k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp + (long long)(j + 1) * len, h->fu, dc, len);
            ck_launch();
          }
        }
        if (status != MG_OK) break;
        if (!lag_closed) {  // finish the last column: one pass of V^T u
          k = mm;
          multidot_pair(h, Vp, len, k, h->fu, len, K.h, s);
          {
            Bracket br(h, CAT_SMALL, s);
            k_dcgs2_coef<<<1, 32, 0, s>>>(k, nullptr, K.h, dc, h->dcg + kDcC1, h->dcg + kDcC2, h->dcg + kDcHp,
                                          K.H, h->ldh, K.cs, K.sn, K.g, K.scal, 1);
            ck_launch();
          }
          read_scal(h, K, s);
          const double est = h->host_scal[0], hj1 = h->host_scal[2];
          if (!std::isfinite(est) || !std::isfinite(hj1)) {
            status = MG_ERR_BREAKDOWN;
            break;
          }
          est_rel = est / bnorm;
          if (est <= rtol * bnorm || hj1 == 0.0) done = true;
        }
        total += k;
        if (total >= maxit) done = true;
        {
          Bracket br(h, CAT_SMALL, s);
          k_backsolve<<<1, 256, (size_t)k * sizeof(double), s>>>(k, K.H, h->ldh, K.g, K.ycoef);
          ck_launch();
        }
        multi_axpy(h, x, h->fZ, len, K.ycoef, k, 1.0, len, s);
        if (!done) {
          launch_apply<double>(h, h->lv[0].d.view, x, b, h->fr, s);
          r = h->fr;
        }
      }
      while (!done && total < maxit && !h->dcgs2) {
        // beta = ||r||, v_0 = r / beta
        norm_into(h, K, r, len, s);
        {
          Bracket br(h, CAT_AXPY, s);
          if (Vp)
            k_split_basis<<<grid_for(len, 256), 256, 0, s>>>(Vp, r, K.scal + 1, len);
          else
            k_scale<<<grid_for(len, 256), 256, 0, s>>>(h->fV, r, K.scal + 1, len);
          ck_launch();
        }
        {
          Bracket br(h, CAT_SMALL, s);
          k_arnoldi_init<<<1, 128, 0, s>>>(K.scal, K.g, m);
          ck_launch();
        }
        const int mm = std::min(m, maxit - total);
        int k = 0;
        for (int j = 0; j < mm; ++j) {
          double *vj = h->fV + (long long)j * len, *zj = h->fZ + (long long)j * len;
          if (Vp) {
            Bracket br(h, CAT_SMALL, s);
            k_join_basis<<<grid_for(len, 256), 256, 0, s>>>(h->vin, Vp + (long long)j * len, len);
            ck_launch();
            vj = h->vin;
          }
          precondition(h, vj, zj, s);
          launch_apply<double>(h, h->lv[0].d.view, zj, nullptr, h->fw, s);
          arnoldi_step(h, K, h->fV, len, j, h->fw, s, Vp);
          k = j + 1;
          total++;
          const double est = h->host_scal[0], hj1 = h->host_scal[2];
          if (!std::isfinite(est) || !std::isfinite(hj1)) {
            status = MG_ERR_BREAKDOWN;
            done = true;
            break;
          }
          est_rel = est / bnorm;
          if (est <= rtol * bnorm || hj1 == 0.0) {
            done = true;
            break;
          }
        }
        if (status != MG_OK) break;
        {
          Bracket br(h, CAT_SMALL, s);
          k_backsolve<<<1, 256, (size_t)k * sizeof(double), s>>>(k, K.H, h->ldh, K.g, K.ycoef);
          ck_launch();
        }
        multi_axpy(h, x, h->fZ, len, K.ycoef, k, 1.0, len, s);
        if (!done && total < maxit) {
          launch_apply<double>(h, h->lv[0].d.view, x, b, h->fr, s);
          r = h->fr;
        }
      }
      // true residual (FP64)
      launch_apply<double>(h, h->lv[0].d.view, x, b, h->fr, s);
      norm_into(h, K, h->fr, len, s);
      read_scal(h, K, s);
      true_rel = h->host_scal[0] / bnorm;
      if (status == MG_OK && est_rel > rtol) status = MG_NOT_CONVERGED;
      int tmo = 0;  // a streamed multi-dot's wait ran out (pair basis)
      ck(cudaMemcpyAsync(&tmo, h->flag + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      if (tmo) status = MG_ERR_TIMEOUT;
    } else {
      est_rel = 0.0;
    }
    if (!x_dev) ck(cudaMemcpyAsync(x_out, x, len * sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    }
    harvest(h);
  } catch (const CudaFail &) {
    status = MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    status = MG_ERR_OOM;
  } catch (int) {
    status = MG_ERR_NONFINITE;
  }
  if (info) {
    info->status = status;
    info->iters = total;
    info->vcycles = h->vcycles;
    info->coarse_iters = h->coarse_iters;
    info->relres = est_rel;
    info->true_relres = true_rel;
    info->coarse_learned = h->coarse_learned;
  }
  return status;
}

}  // extern "C"

// ===========================================================================
// Many systems in one graph launch.

extern "C" int fgmres_solve_batched(mg_handle *const *hs, int count, const double *const *b, double *const *x,
                                    double rtol, int maxit, int restart, mg_solve_info *infos, void *stream) {
  if (!hs || !b || !x || count < 1 || maxit < 1 || restart < 1 || restart > 512 || !(rtol >= 0.0)) return MG_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b[i] || !x[i]) return MG_ERR_ARG;
    if (!is_device_pointer(b[i]) || !is_device_pointer(x[i])) return MG_ERR_ARG;
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) return MG_ERR_ARG;  // each system needs its own handle (workspaces)
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BatchGraph &bg = g_batch;
  const int m = std::min(restart, maxit);
  int worst = MG_OK;
  try {
    for (int i = 0; i < count; ++i) prepare_solve(hs[i], m, s);
    bool same = bg.exec && (int)bg.hs.size() == count && bg.rtol == rtol && bg.maxit == maxit && bg.restart == m;
    for (int i = 0; same && i < count; ++i) same = bg.hs[i] == hs[i] && bg.b[i] == b[i] && bg.x[i] == x[i];
    for (int i = 0; same && i < count; ++i) same = hs[i]->fm >= m && bg.gen[i] == hs[i]->gen;
    if (!same) {
      ck(cudaStreamSynchronize(s));
      if (bg.exec) cudaGraphExecDestroy(bg.exec);
      if (bg.graph) cudaGraphDestroy(bg.graph);
      bg.exec = nullptr;
      bg.graph = nullptr;
      if (!bg.root) ck(cudaStreamCreateWithFlags(&bg.root, cudaStreamNonBlocking));
      if (!bg.fork) ck(cudaEventCreateWithFlags(&bg.fork, cudaEventDisableTiming));
      while ((int)bg.joins.size() < count) {
        cudaEvent_t e;
        ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        bg.joins.push_back(e);
      }
      // root -> fork into one branch per system (its own capture stream) -> join
      ck(cudaStreamBeginCapture(bg.root, cudaStreamCaptureModeRelaxed));
      try {
        ck(cudaEventRecord(bg.fork, bg.root));
        for (int i = 0; i < count; ++i) {
          mg_handle *h = hs[i];
          ck(cudaStreamWaitEvent(h->cap[0], bg.fork, 0));
          const long long saved = h->launches;
          h->capturing = 1;
          try {
            capture_solve(h, h->cap[0], b[i], x[i], rtol, maxit, m);
          } catch (...) {
            h->capturing = 0;
            h->launches = saved;
            throw;
          }
          h->capturing = 0;
          h->launches = saved;
          ck(cudaEventRecord(bg.joins[i], h->cap[0]));
          ck(cudaStreamWaitEvent(bg.root, bg.joins[i], 0));
        }
        ck(cudaStreamEndCapture(bg.root, &bg.graph));
      } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(bg.root, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
      }
      ck(cudaGraphInstantiate(&bg.exec, bg.graph, 0));
      bg.hs.assign(hs, hs + count);
      bg.b.assign(b, b + count);
      bg.x.assign(x, x + count);
      bg.gen.resize(count);
      for (int i = 0; i < count; ++i) bg.gen[i] = hs[i]->gen;
      bg.rtol = rtol;
      bg.maxit = maxit;
      bg.restart = m;
      // a single solve of these handles must recapture its own graph: the
      // batch capture reused their capture state
      for (int i = 0; i < count; ++i) hs[i]->gkey.b = nullptr;
    }
    std::vector<KState> before(count), fs(count), cs(count);
    std::vector<int> bad(2 * (size_t)count), learned(count, 0);
    std::vector<double> tr(4 * (size_t)count);
    for (int i = 0; i < count; ++i)
      ck(cudaMemcpyAsync(&before[i], hs[i]->kst_c, sizeof(KState), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    ck(cudaGraphLaunch(bg.exec, s));
    for (int i = 0; i < count; ++i) {
      ck(cudaMemcpyAsync(&fs[i], hs[i]->kst_f, sizeof(KState), cudaMemcpyDeviceToHost, s));
      ck(cudaMemcpyAsync(&cs[i], hs[i]->kst_c, sizeof(KState), cudaMemcpyDeviceToHost, s));
      ck(cudaMemcpyAsync(&bad[2 * (size_t)i], hs[i]->flag + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      ck(cudaMemcpyAsync(&tr[4 * (size_t)i], hs[i]->kf.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (hs[i]->net) ck(cudaMemcpyAsync(&learned[i], hs[i]->net_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    ck(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) {
      mg_handle *h = hs[i];
      const long long citers = cs[i].iters_all - before[i].iters_all;
      h->launches += h->g_init + h->g_body * fs[i].total + h->g_coarse * citers;
      int st = MG_OK;
      double est_rel = 0.0, true_rel = 0.0;
      if (bad[2 * (size_t)i]) {
        st = MG_ERR_NONFINITE;
      } else if (fs[i].bnorm > 0.0) {
        true_rel = tr[4 * (size_t)i] / fs[i].bnorm;
        est_rel = fs[i].est / fs[i].bnorm;
        if (fs[i].breakdown) st = MG_ERR_BREAKDOWN;
        else if (!fs[i].converged) st = MG_NOT_CONVERGED;
      }
      if (bad[2 * (size_t)i + 1]) st = MG_ERR_TIMEOUT;
      if (infos) {
        infos[i].status = st;
        infos[i].iters = fs[i].total;
        infos[i].vcycles = fs[i].total;
        infos[i].coarse_iters = (int)citers;
        infos[i].relres = est_rel;
        infos[i].true_relres = true_rel;
        infos[i].coarse_learned = learned[i];
      }
      if (st < 0 && (worst >= 0 || st < worst)) worst = st;
      else if (st == MG_NOT_CONVERGED && worst == MG_OK) worst = st;
    }
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    return MG_ERR_OOM;
  }
  return worst;
}

// ===========================================================================
// Time-range operations: the V-cycle's steps on a contiguous range of time
// blocks of one level, for a cycle sharded across processes by time (each
// process owns a range of blocks on every level and exchanges the couplings
// at the range ends; the paper's block-Jacobi sweep parallelises trivially in
// time, Sec. 5.3.2).  Vectors are full level-length FP64 device vectors in the
// type-major layout; only the entries the call names are read or written.

namespace {

// the FP64 view of a level, or null
const LevelView<double> *range_view(mg_handle *h, int level) {
  if (!h || level < 0 || level >= (int)h->lv.size()) return nullptr;
  return &h->lv[level].d.view;
}

bool range_ok(const LevelView<double> &L, int j0, int j1) { return j0 >= 0 && j1 > j0 && j1 <= L.n + 1; }

int range_status() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

}  // namespace

extern "C" int mg_level_info(const mg_handle *h, int level, int *n, long long *len) {
  if (!h || level < 0 || level >= (int)h->lv.size()) return MG_ERR_ARG;
  if (n) *n = h->lv[level].n;
  if (len) *len = h->lv[level].len;
  return MG_OK;
}

extern "C" int mg_range_sweep(mg_handle *h, int level, int j0, int j1, const double *r, const double *yold,
                              double *y, void *stream) {
  const LevelView<double> *L = range_view(h, level);
  if (!L || level == (int)h->lv.size() - 1 || !r || !y || y == yold || !range_ok(*L, j0, j1)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double om = h->opts.omega;
  Vec<const double> Y = make_cvec(yold ? yold : r, L->n, h->p, h->q);
  const double *cu = yold ? Y.u : nullptr, *cm = yold ? Y.m : nullptr;
  try {
    // the V-cycle's own kernel choice for this level, restricted to the range: the same bits per block
    launch_block_solve<double>(h, *L, r, cu, cm, y, s, yold, om, j0, j1);
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  }
  return range_status();
}

extern "C" int mg_range_residual(mg_handle *h, int level, int j0, int j1, const double *y, const double *b,
                                 double *r, void *stream) {
  const LevelView<double> *L = range_view(h, level);
  if (!L || !y || !r || y == r || !range_ok(*L, j0, j1)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    launch_apply<double>(h, *L, y, b, r, s, j0, j1);  // b null: r = A y
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  }
  return range_status();
}

extern "C" int mg_range_restrict(mg_handle *h, int level, int j0, int j1, const double *r, double *rc,
                                 void *stream) {
  const LevelView<double> *L = range_view(h, level);
  if (!L || level == (int)h->lv.size() - 1 || !r || !rc || !range_ok(*L, j0, j1) || (j0 & 1)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K0 = j0 / 2, K1 = (j1 + 1) / 2;
  h->launches++;
  if (h->opts.restrict_rule == MG_RESTRICT_TRANSPOSE)
    launch_restrict_transpose<double>(r, rc, L->n, h->p, h->q, h->opts.end_rule, s, K0, K1);
  else
    k_restrict_inject<double><<<transfer_grid(L->n / 2, 4 * h->p + h->q), 256, 0, s>>>(r, rc, L->n, h->p, h->q, K0,
                                                                                      K1);
  return range_status();
}

extern "C" int mg_range_prolong(mg_handle *h, int level, int j0, int j1, const double *ec, double *y,
                                void *stream) {
  const LevelView<double> *L = range_view(h, level);
  if (!L || level == (int)h->lv.size() - 1 || !ec || !y || !range_ok(*L, j0, j1)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->launches++;
  launch_prolong<double>(ec, y, L->n, h->p, h->q, h->opts.end_rule, s, j0, j1);
  return range_status();
}

extern "C" int mg_coarse_solve(mg_handle *h, const double *rc, double *yc, void *stream) {
  if (!h || !rc || !yc || rc == yc) return MG_ERR_ARG;
  if (h->opts.precision != MG_PRECISION_FP64) return MG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    coarse_solve<double>(h, rc, yc, s);
    ck(cudaStreamSynchronize(s));
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    return MG_ERR_OOM;
  }
  return MG_OK;
}

namespace {
// The entries of blocks [j0, j1) of a level in its type-major vector: one
// contiguous run per type, in storage order u, v, z, lambda, mu (block j holds
// u_j, z_j, lambda_j for j < n and v_{j-1}, mu_{j-1} for j >= 1).
struct RangeRuns {
  long long off[5], len[5];
};
RangeRuns range_runs(const LevelView<double> &L, int j0, int j1) {
  const long long n = L.n, p = L.p, q = L.q;
  const long long a = j0, su = std::max<long long>(std::min<long long>(j1, n) - a, 0);    // steps of u, z, lambda
  const long long c = std::max(j0, 1) - 1, sv = std::max<long long>((long long)j1 - 1 - c, 0);  // of v, mu
  return RangeRuns{{a * p, n * p + c * p, 2 * n * p + a * q, 2 * n * p + n * q + a * p, 3 * n * p + n * q + c * p},
                   {su * p, sv * p, su * q, su * p, sv * p}};
}

bool range_vecs_ok(mg_handle *h, int level, int j0, int j1, int k, long long ldv) {
  const LevelView<double> *L = range_view(h, level);
  return L && range_ok(*L, j0, j1) && k >= 1 && k <= 512 && ldv >= h->lv[level].len;
}
}  // namespace

extern "C" int mg_range_dots(mg_handle *h, int level, int j0, int j1, const double *V, long long ldv, int k,
                             const double *w, double *out, void *stream) {
  if (!V || !w || !out || !range_vecs_ok(h, level, j0, j1, k, ldv)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const RangeRuns R = range_runs(h->lv[level].d.view, j0, j1);
  try {
    int accumulate = 0;  // runs summed in storage order, each by the solve's blocked multi-dot
    for (int t = 0; t < 5; ++t)
      if (R.len[t]) {
        multidot(h, V + R.off[t], ldv, k, w + R.off[t], R.len[t], out, accumulate, s);
        accumulate = 1;
      }
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  }
  return range_status();
}

extern "C" int mg_range_axpy(mg_handle *h, int level, int j0, int j1, const double *V, long long ldv, int k,
                             const double *c, double sign, double *w, void *stream) {
  if (!V || !c || !w || !range_vecs_ok(h, level, j0, j1, k, ldv)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const RangeRuns R = range_runs(h->lv[level].d.view, j0, j1);
  try {
    for (int t = 0; t < 5; ++t)
      if (R.len[t]) multi_axpy(h, w + R.off[t], V + R.off[t], ldv, c, k, sign, R.len[t], s);
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  }
  return range_status();
}

extern "C" int mg_range_scale(mg_handle *h, int level, int j0, int j1, const double *x, const double *a, double *y,
                              void *stream) {
  const LevelView<double> *L = range_view(h, level);
  if (!L || !x || !a || !y || !range_ok(*L, j0, j1)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const RangeRuns R = range_runs(*L, j0, j1);
  for (int t = 0; t < 5; ++t)
    if (R.len[t]) {
      h->launches++;
      k_scale<<<grid_for(R.len[t], 256), 256, 0, s>>>(y + R.off[t], x + R.off[t], a, R.len[t]);
    }
  return range_status();
}

// ===========================================================================
// Residual check that allocates nothing.
//
// Some callers must not allocate device memory when they check a solution:
// code that runs while a framework's caching allocator owns the device pool,
// a real-time loop with a fixed memory budget, or an outer optimisation loop
// that tests its stopping rule between captured work.  fgmres_solve grows its
// workspace on first use, so it cannot serve them.  This entry point computes
// the FP64 true residual of any x for an existing handle with its scratch (the
// residual vector and the reduction partial sums) in one file-scope device
// array of fixed size, shared by every call of the process on that device.

namespace {

constexpr long long kNoAllocMaxLen = 1LL << 20;      // longest vector n (4p+q) accepted
constexpr int kNoAllocPartials = 2 * 304;             // two dot products, <= 304 CTAs each
constexpr int kMaxDevices = 64;

// residual vector, then partial sums, then the two reduced squares
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxLen + kNoAllocPartials + 8];

double *g_noalloc_ptr[kMaxDevices] = {};

__global__ void k_noalloc_finish(const double *sums, double *out) {
  const double rn = sqrt(sums[0]), bn = sqrt(sums[1]);
  out[0] = rn;
  out[1] = bn > 0.0 ? rn / bn : 0.0;
}

}  // namespace

extern "C" int mg_true_residual_noalloc(mg_handle *h, const double *b, const double *x, double *out, void *stream) {
  if (!h || !b || !x || !out) return MG_ERR_ARG;
  const long long len = h->lv[0].len;
  if (len > kNoAllocMaxLen) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error,
                  "mg_true_residual_noalloc: vector length %lld exceeds the fixed scratch of %lld doubles", len,
                  kNoAllocMaxLen);
    return MG_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  if (dev != h->device) {  // the handle's buffers live on another device: launching here would fault
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error,
                  "mg_true_residual_noalloc: device %d is current, the handle was set up on device %d", dev,
                  h->device);
    return MG_ERR_ARG;
  }
  if (!g_noalloc_ptr[dev]) {  // first call on this device: resolve the array's device address
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  double *r = g_noalloc_ptr[dev];
  double *partial = r + kNoAllocMaxLen;
  double *sums = partial + kNoAllocPartials;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const LevelView<double> &L = h->lv[0].d.view;
  // r = b - A x (every entry written)
  if (L.layout == MG_LAYOUT_DENSE && (L.p > kDenseMax || L.q > kDenseMax)) {
    k_apply_dw<double><<<(L.n + 3) / 4, 128, 0, s>>>(L, x, b, r);
  } else if (L.layout == MG_LAYOUT_DENSE) {
    k_apply_dense<double><<<grid_for(L.n, 128, 1 << 30), 128, 0, s>>>(L, x, b, r);
  } else {
    const int blocks = (L.n + 3) / 4;
    switch (h->C) {
      case 1: k_apply_tri<double, 1><<<blocks, 128, 0, s>>>(L, x, b, r); break;
      case 2: k_apply_tri<double, 2><<<blocks, 128, 0, s>>>(L, x, b, r); break;
      case 4: k_apply_tri<double, 4><<<blocks, 128, 0, s>>>(L, x, b, r); break;
      case 8: k_apply_tri<double, 8><<<blocks, 128, 0, s>>>(L, x, b, r); break;
      default: k_apply_tri<double, 16><<<blocks, 128, 0, s>>>(L, x, b, r); break;
    }
  }
  // ||r||^2 and ||b||^2 with the library's fixed-order reductions (each CTA
  // overwrites its partial slot; nothing carries over between calls)
  const int G = (int)std::max<long long>(1, std::min<long long>(304, (len + kDotThreads - 1) / kDotThreads));
  k_multidot_partial<<<dim3(G, 1), kDotThreads, 0, s>>>(r, len, r, len, partial);
  k_reduce_partials<<<1, 128, 0, s>>>(partial, G, 1, sums, 0);
  k_multidot_partial<<<dim3(G, 1), kDotThreads, 0, s>>>(b, len, b, len, partial + 304);
  k_reduce_partials<<<1, 128, 0, s>>>(partial + 304, G, 1, sums + 1, 0);
  k_noalloc_finish<<<1, 1, 0, s>>>(sums, out);
  h->launches += 6;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

// ===========================================================================
// Learned coarse-grid correction: the network object, its training, and its
// use as the coarse solve of a handle's V-cycles.

namespace {

constexpr int kLossPartials = 1024;
constexpr int kNetMaxBatch = 32767;  // grid z of the convolution launches (batch x output-channel blocks)
constexpr int kNetMaxT = 65535 * 4;  // grid y of the tensor-core convolution (4 rows per CTA)
constexpr int kScaleParts = 64;
constexpr int kWgSlices = 64;   // position slices of the weight gradient (partial sums)
constexpr int kBiasParts = 64;

// per-channel root mean square of `count` samples of 5 x TX floats
void channel_rms(mg_net *net, const float *x, int count, long long TX, float *scale, cudaStream_t s) {
  const int C = net_ch(0);
  k_channel_sumsq<<<dim3(C, kScaleParts), 256, 0, s>>>(x, count, TX, C, net->spart);
  ck_launch();
  k_channel_rms<<<1, 32, 0, s>>>(net->spart, kScaleParts, (double)count * TX, C, scale);
  ck_launch();
}

// training workspace for `batch` samples of T x X (grown on demand)
void net_ensure_train(mg_net *net, int batch, long long TX, int minibatches) {
  const long long need = (long long)batch * 32 * TX;
  if (need <= net->ws_elems && minibatches <= net->ws_batch) return;
  ck(cudaDeviceSynchronize());
  net->ws.release();
  net->ws_elems = 0;
  net->ws_batch = 0;
  const long long cap = need;
  for (int l = 1; l < kNetLayers; ++l) net->h[l] = net->ws.alloc<float>((size_t)cap);
  net->h[kNetLayers] = net->ws.alloc<float>((size_t)cap);
  for (int l = 0; l < kNetLayers - 1; ++l) net->z[l] = net->ws.alloc<float>((size_t)cap);
  net->g0 = net->ws.alloc<float>((size_t)cap);
  net->g1 = net->ws.alloc<float>((size_t)cap);
  net->bx = net->ws.alloc<float>((size_t)cap);
  net->by = net->ws.alloc<float>((size_t)cap);
  net->loss = net->ws.alloc<float>((size_t)std::max(1, minibatches));
  net->ws_elems = cap;
  net->ws_batch = std::max(1, minibatches);
}

// Residual-metric loss of the output net->h[4] (B samples of the coarse
// level's 5 x T x X entries, the type-major layout of its vectors):
//   d_b = scale (out_b - target_b),  L = sum_b ||A_c d_b||^2 / n,
// n = B 5 T X, A_c the coarse operator of net->metric (FP64, the library's
// own product), and dL/dout_b = scale 2 A_c^T A_c d_b / n into net->g0
// (A_c is symmetric: the lifted augmented matrix).  scale (per channel) may be
// null.
constexpr int kMetricParts = 304;
void net_metric_loss(mg_net *net, const float *target, int B, long long TX, const float *scale, float *loss_dev,
                     cudaStream_t s) {
  mg_handle *hm = net->metric;
  const Level &cl = hm->lv.back();
  const LevelView<double> &L = cl.d.view;
  const long long len = cl.len, n = (long long)B * len;
  if (n > net->mws_n) {
    ck(cudaStreamSynchronize(s));
    if (net->mws) cudaFree(net->mws);
    net->mws = nullptr;
    net->mws_n = 0;
    cudaError_t e = cudaMalloc(&net->mws, (size_t)(2 * n + kMetricParts + 1) * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    net->mws_n = n;
  }
  double *d = net->mws, *u = d + n, *part = u + n, *sum = part + kMetricParts;
  const int C = net_ch(kNetLayers);
  const int gg = grid_for(n, 256, 1 << 20);
  k_metric_diff<<<gg, 256, 0, s>>>(net->h[kNetLayers], target, scale, TX, C, n, d);
  ck_launch();
  for (int b = 0; b < B; ++b) launch_apply<double>(hm, L, d + b * len, nullptr, u + b * len, s);
  const int G = (int)std::max<long long>(1, std::min<long long>(kMetricParts, (n + kDotThreads - 1) / kDotThreads));
  k_multidot_partial<<<dim3(G, 1), kDotThreads, 0, s>>>(u, n, u, n, part);
  ck_launch();
  k_reduce_partials<<<1, 128, 0, s>>>(part, G, 1, sum, 0);
  ck_launch();
  k_metric_loss<<<1, 1, 0, s>>>(sum, 1.0 / (double)n, loss_dev);
  ck_launch();
  for (int b = 0; b < B; ++b) launch_apply<double>(hm, L, u + b * len, nullptr, d + b * len, s);
  k_metric_grad<<<gg, 256, 0, s>>>(d, scale, TX, C, n, 2.0 / (double)n, net->g0);
  ck_launch();
}

// forward (keeping every layer's output and pre-activation), the loss into
// loss_dev[0] (mean squared error, or the residual metric when the network has
// one; mscale: the metric's per-channel scale of the output, may be null),
// backward into net->grad
void net_loss_grad_dev(mg_net *net, const float *x, const float *target, int B, int T, int X, float *loss_dev,
                       cudaStream_t s, const float *mscale = nullptr) {
  const long long TX = (long long)T * X;
  const float *in = x;
  for (int l = 0; l < kNetLayers; ++l) {
    const float *W = net->params + net_layer_offset(l);
    const float *bias = W + (long long)net_ch(l + 1) * net_ch(l) * kNetKT * kNetKX;
    const long long n = (long long)B * net_ch(l + 1) * TX;
    const bool act = l < kNetLayers - 1;
    (void)n;
    launch_conv<float>(in, W, bias, net->h[l + 1], act ? net->z[l] : nullptr, B, net_ch(l), net_ch(l + 1), T, X, act,
                       s);
    in = net->h[l + 1];
  }
  if (net->metric) {
    net_metric_loss(net, target, B, TX, mscale, loss_dev, s);
  } else {
    const long long nout = (long long)B * net_ch(kNetLayers) * TX;
    const int G = grid_for(nout, 256, kLossPartials);
    k_mse<<<G, 256, 0, s>>>(net->h[kNetLayers], target, net->g0, nout, net->partial);
    ck_launch();
    k_sum_partials<<<1, 32, 0, s>>>(net->partial, G, 1.0f / (float)nout, loss_dev);
    ck_launch();
  }
  float *g = net->g0, *other = net->g1;
  for (int l = kNetLayers - 1; l >= 0; --l) {
    const int C = net_ch(l), O = net_ch(l + 1);
    if (l < kNetLayers - 1) {
      const long long n = (long long)B * O * TX;
      k_leaky_bwd<<<grid_for(n, 256, 1 << 20), 256, 0, s>>>(g, net->z[l], n);
      ck_launch();
    }
    const float *hin = l == 0 ? x : net->h[l];
    float *gW = net->grad + net_layer_offset(l);
    float *gb = gW + (long long)O * C * kNetKT * kNetKX;
    {
      const int ncb = (C + kWgCB - 1) / kWgCB, nob = (O + kWgOB - 1) / kWgOB;
      const int P = std::min(kWgSlices, std::max(1, 608 / (ncb * nob)));
      k_conv_wgrad<<<dim3(nob * ncb, P), 192, 0, s>>>(g, hin, net->wpart, B, C, O, T, X);
      ck_launch();
      const long long nw = (long long)O * C * kNetKT * kNetKX;
      k_wgrad_reduce<<<grid_for(nw, 256), 256, 0, s>>>(net->wpart, P, nw, gW);
      ck_launch();
      k_bias_partial<<<dim3(O, kBiasParts), 256, 0, s>>>(g, B, O, TX, net->bpart);
      ck_launch();
      k_bias_reduce<<<1, 32, 0, s>>>(net->bpart, kBiasParts, O, gb);
      ck_launch();
    }
    if (l > 0) {  // gradient of the layer's input: the convolution with the flipped, transposed weights
      const float *W = net->params + net_layer_offset(l);
      k_flip_transpose<<<grid_for((long long)O * C * kNetKT * kNetKX, 256), 256, 0, s>>>(W, net->wt, C, O);
      ck_launch();
      launch_conv<float>(g, net->wt, nullptr, other, nullptr, B, O, C, T, X, 0, s);
      std::swap(g, other);
    }
  }
}

void net_adam(mg_net *net, float lr, float b1, float b2, float eps, cudaStream_t s) {
  net->step++;
  net->updates++;
  const double c1 = 1.0 - std::pow((double)b1, net->step), c2 = 1.0 - std::pow((double)b2, net->step);
  k_adam<<<grid_for(kNetParams, 256), 256, 0, s>>>(net->params, net->grad, net->m, net->v, kNetParams, lr, b1, b2,
                                                   eps, (float)c1, (float)c2);
  ck_launch();
  net->bf16_valid = false;
}

// splitmix64 (Steele, Lea and Flood 2014)
struct SplitMix64 {
  unsigned long long x;
  unsigned long long next() {
    unsigned long long z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
};

template <typename F>
int net_guard(F &&f) {
  try {
    f();
  } catch (const CudaFail &) {
    return MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    return MG_ERR_OOM;
  }
  return MG_OK;
}

}  // namespace

extern "C" {

long long mg_net_param_count(void) { return kNetParams; }

void mg_net_destroy(mg_net *net) {
  if (!net) return;
  cudaDeviceSynchronize();
  net->ws.release();
  net->mem.release();
  for (void *p : {net->ia, net->ib, net->ic, static_cast<void *>(net->order), static_cast<void *>(net->mws)})
    if (p) cudaFree(p);
  delete net;
}

int mg_net_create(const float *init_params, mg_net **out) {
  if (!init_params || !out) return MG_ERR_ARG;
  *out = nullptr;
  mg_net *net = new (std::nothrow) mg_net();
  if (!net) return MG_ERR_OOM;
  const int st = net_guard([&] {
    net->params = net->mem.alloc<float>(kNetParams);
    net->grad = net->mem.alloc<float>(kNetParams);
    net->m = net->mem.alloc<float>(kNetParams);
    net->v = net->mem.alloc<float>(kNetParams);
    net->partial = net->mem.alloc<float>(kLossPartials);
    net->params_bf16 = net->mem.alloc<__nv_bfloat16>(kNetParams);
    net->wimg = net->mem.alloc<__nv_bfloat16>(kConvMmaWimg);
    net->timg = net->mem.alloc<__nv_bfloat16>(kTcImgValues);
    net->tc_err = net->mem.alloc<int>(1);
    ck(cudaMemset(net->tc_err, 0, sizeof(int)));
    net->wt = net->mem.alloc<float>((size_t)32 * 32 * kNetKT * kNetKX);
    net->wpart = net->mem.alloc<float>((size_t)kWgSlices * 32 * 32 * kNetKT * kNetKX);
    net->bpart = net->mem.alloc<float>((size_t)32 * kBiasParts);
    net->sx = net->mem.alloc<float>(8);
    net->sy = net->mem.alloc<float>(8);
    net->spart = net->mem.alloc<double>((size_t)8 * kScaleParts);
    ck(cudaMemcpy(net->params, init_params, kNetParams * sizeof(float), cudaMemcpyHostToDevice));
    ck(cudaMemset(net->grad, 0, kNetParams * sizeof(float)));
    ck(cudaMemset(net->m, 0, kNetParams * sizeof(float)));
    ck(cudaMemset(net->v, 0, kNetParams * sizeof(float)));
    conv_mma_prepare();
  });
  if (st != MG_OK) {
    mg_net_destroy(net);
    return st;
  }
  *out = net;
  return MG_OK;
}

int mg_net_set_params(mg_net *net, const float *params) {
  if (!net || !params) return MG_ERR_ARG;
  return net_guard([&] {
    ck(cudaDeviceSynchronize());
    ck(cudaMemcpy(net->params, params, kNetParams * sizeof(float), cudaMemcpyHostToDevice));
    net->bf16_valid = false;
  });
}

int mg_net_get_params(const mg_net *net, float *params) {
  if (!net || !params) return MG_ERR_ARG;
  return net_guard([&] {
    ck(cudaDeviceSynchronize());
    ck(cudaMemcpy(params, net->params, kNetParams * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

int mg_net_get_grad(const mg_net *net, float *grad) {
  if (!net || !grad) return MG_ERR_ARG;
  return net_guard([&] {
    ck(cudaDeviceSynchronize());
    ck(cudaMemcpy(grad, net->grad, kNetParams * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

int mg_net_forward(mg_net *net, const float *x, int batch, int T, int X, float *y, int bf16, void *stream) {
  if (!net || !x || !y || batch < 1 || batch > kNetMaxBatch || T < 1 || T > kNetMaxT || X < 1 ||
      (bf16 != 0 && bf16 != 1))
    return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long TX = (long long)T * X;
  const int st = net_guard([&] {
    const long long bytes = (long long)batch * 32 * TX * (long long)sizeof(float);
    if (bytes > net->inf_bytes) {
      ck(cudaStreamSynchronize(s));
      for (void *p : {net->ia, net->ib, net->ic})
        if (p) cudaFree(p);
      net->ia = net->ib = net->ic = nullptr;
      net->inf_bytes = 0;
      for (void **p : {&net->ia, &net->ib, &net->ic}) {
        cudaError_t e = cudaMalloc(p, (size_t)bytes);
        if (e != cudaSuccess) {
          cudaGetLastError();
          std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
          throw std::bad_alloc();
        }
      }
      net->inf_bytes = bytes;
    }
    const long long nio = (long long)batch * net_ch(0) * TX;
    if (bf16) {
      net_refresh_bf16(net, s);
      using B16 = __nv_bfloat16;
      B16 *c = static_cast<B16 *>(net->ic);
      if (conv_use_tc())  // the tcgen05 layers read their input with the channels innermost
        k_f32_to_bf16_ci<<<grid_for((long long)batch * TX, 256), 256, 0, s>>>(x, c, batch, TX);
      else
        k_f32_to_bf16<<<grid_for(nio, 256), 256, 0, s>>>(x, c, nio);
      ck_launch();
      net_forward_storage<B16>(nullptr, net, c, batch, T, X, c, static_cast<B16 *>(net->ia),
                               static_cast<B16 *>(net->ib), s);
      k_bf16_to_f32<<<grid_for(nio, 256), 256, 0, s>>>(c, y, nio);
      ck_launch();
    } else {
      net_forward_storage<float>(nullptr, net, x, batch, T, X, y, static_cast<float *>(net->ia),
                                 static_cast<float *>(net->ib), s);
    }
  });
  if (st != MG_OK || !bf16 || !conv_use_tc()) return st;
  // a tcgen05 layer whose bounded wait ran out: the output is void (the flag is cleared for the next call)
  int tmo = 0;
  if (cudaMemcpyAsync(&tmo, net->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MG_ERR_CUDA;
  if (!tmo) return MG_OK;
  cudaMemsetAsync(net->tc_err, 0, sizeof(int), s);
  return MG_ERR_TIMEOUT;
}

// the samples' shape is the metric handle's coarse level (or there is no metric)
static bool metric_shape_ok(const mg_net *net, int T, int X) {
  return !net->metric || (net->metric->lv.back().n == T && net->metric->p == X);
}

int mg_net_set_metric(mg_net *net, mg_handle *h) {
  if (!net) return MG_ERR_ARG;
  if (h && (h->q != h->p || h->opts.precision != MG_PRECISION_FP64)) return MG_ERR_UNSUPPORTED;
  net->metric = h;
  return MG_OK;
}

int mg_net_loss_grad(mg_net *net, const float *x, const float *target, int batch, int T, int X, float *loss,
                     void *stream) {
  if (!net || !x || !target || !loss || batch < 1 || batch > kNetMaxBatch || T < 1 || T > kNetMaxT || X < 1)
    return MG_ERR_ARG;
  if (!metric_shape_ok(net, T, X)) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return net_guard([&] {
    net_ensure_train(net, batch, (long long)T * X, 1);
    net_loss_grad_dev(net, x, target, batch, T, X, net->loss, s);
    ck(cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
  });
}

int mg_net_adam_step(mg_net *net, float lr, float beta1, float beta2, float eps, void *stream) {
  if (!net || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return MG_ERR_ARG;
  return net_guard([&] { net_adam(net, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)); });
}

int mg_net_train(mg_net *net, const float *x_all, const float *y_all, int count, int T, int X, int batch, int epochs,
                 float lr, unsigned long long seed, int normalize, float *epoch_loss, void *stream) {
  if (!net || !x_all || !y_all || count < 1 || T < 1 || T > kNetMaxT || X < 1 || batch < 1 || batch > kNetMaxBatch ||
      epochs < 0 ||
      !(lr > 0.f) ||
      (normalize != 0 && normalize != 1) || !metric_shape_ok(net, T, X))
    return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long TX = (long long)T * X, row = (long long)net_ch(0) * TX;
  const int B = std::min(batch, count);
  const int nmb = (count + B - 1) / B;
  return net_guard([&] {
    net_ensure_train(net, B, TX, nmb);
    if (net->order_cap < count) {
      ck(cudaStreamSynchronize(s));
      if (net->order) cudaFree(net->order);
      net->order = nullptr;
      net->order_cap = 0;
      cudaError_t e = cudaMalloc(&net->order, (size_t)count * sizeof(int));
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw std::bad_alloc();
      }
      net->order_cap = count;
    }
    const int C = net_ch(0);
    const int fold_grid = grid_for(net_layer_params(0) + net_layer_params(kNetLayers - 1), 256);
    if (normalize) {  // train the normalised network x / sx -> y / sy from a fresh optimiser state
      channel_rms(net, x_all, count, TX, net->sx, s);
      channel_rms(net, y_all, count, TX, net->sy, s);
      if (net->updates > 0) {  // a trained network keeps its function; a fresh one starts as the normalised one
        k_net_fold<<<fold_grid, 256, 0, s>>>(net->params, net->sx, net->sy, +1);
        ck_launch();
      }
      ck(cudaMemsetAsync(net->m, 0, kNetParams * sizeof(float), s));
      ck(cudaMemsetAsync(net->v, 0, kNetParams * sizeof(float), s));
      net->step = 0;
    }
    SplitMix64 rng{seed};
    std::vector<int> order(count);
    std::vector<float> losses(nmb);
    for (int e = 0; e < epochs; ++e) {
      // Fisher-Yates shuffle of the sample order
      for (int i = 0; i < count; ++i) order[i] = i;
      for (int i = count - 1; i > 0; --i) std::swap(order[i], order[(int)(rng.next() % (unsigned long long)(i + 1))]);
      ck(cudaMemcpyAsync(net->order, order.data(), (size_t)count * sizeof(int), cudaMemcpyHostToDevice, s));
      for (int k = 0; k < nmb; ++k) {
        const int b0 = k * B, nb = std::min(B, count - b0);
        const int gg = grid_for((long long)nb * row, 256, 1 << 20);
        if (normalize) {
          k_gather_rows_scaled<<<gg, 256, 0, s>>>(x_all, net->order + b0, nb, row, TX, C, net->sx, net->bx);
          ck_launch();
          k_gather_rows_scaled<<<gg, 256, 0, s>>>(y_all, net->order + b0, nb, row, TX, C, net->sy, net->by);
          ck_launch();
        } else {
          k_gather_rows<<<gg, 256, 0, s>>>(x_all, net->order + b0, nb, row, net->bx);
          ck_launch();
          k_gather_rows<<<gg, 256, 0, s>>>(y_all, net->order + b0, nb, row, net->by);
          ck_launch();
        }
        // normalised training: the metric measures the error of the unnormalised output (times sy)
        net_loss_grad_dev(net, net->bx, net->by, nb, T, X, net->loss + k, s, normalize ? net->sy : nullptr);
        net_adam(net, lr, 0.9f, 0.999f, 1e-8f, s);
      }
      ck(cudaMemcpyAsync(losses.data(), net->loss, (size_t)nmb * sizeof(float), cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));  // also keeps `order` alive until its copy has run
      if (epoch_loss) {
        double sum = 0.0;
        for (float l : losses) sum += l;
        epoch_loss[e] = (float)(sum / nmb);
      }
    }
    if (normalize) {  // back to the network of the unnormalised data
      k_net_fold<<<fold_grid, 256, 0, s>>>(net->params, net->sx, net->sy, -1);
      ck_launch();
      net->bf16_valid = false;
      ck(cudaStreamSynchronize(s));
    }
  });
}

int mg_coarse_shape(const mg_handle *h, int *T, int *X) {
  if (!h || !T || !X) return MG_ERR_ARG;
  *T = h->lv.back().n;
  *X = h->p;
  return MG_OK;
}

int mg_attach_coarse_net(mg_handle *h, mg_net *net, double admit, int bf16) {
  if (!h) return MG_ERR_ARG;
  if (!net) {
    if (h->net) {
      h->net = nullptr;
      h->gen++;
    }
    return MG_OK;
  }
  if (!(admit > 0.0 && admit < 1.0) || (bf16 != 0 && bf16 != 1)) return MG_ERR_ARG;
  if (h->q != h->p || h->lv.back().n > kNetMaxT) return MG_ERR_UNSUPPORTED;
  return net_guard([&] {
    conv_mma_prepare();
    const Level &cl = h->lv.back();
    if (!h->net_e) {
      const long long TX = (long long)cl.n * h->p;
      h->net_x = h->mem.alloc<float>((size_t)8 * TX);  // 5 FP32 channels, or 16 BF16 channels innermost
      h->net_a = h->mem.alloc<float>((size_t)32 * TX);
      h->net_b = h->mem.alloc<float>((size_t)32 * TX);
      h->net_e = h->mem.alloc<double>(cl.len);
      h->net_r = h->mem.alloc<double>(cl.len);
      h->net_flag = h->mem.alloc<int>(2);
      ck(cudaMemset(h->net_flag, 0, 2 * sizeof(int)));
    }
    h->net = net;
    h->admit = admit;
    h->net_bf16 = bf16;
    h->gen++;
  });
}

int mg_record_coarse(mg_handle *h, float *r, float *y, int max_pairs) {
  if (!h) return MG_ERR_ARG;
  if (!r || !y || max_pairs < 1) {
    h->rec_r = h->rec_y = nullptr;
    h->rec_max = 0;
    return MG_OK;
  }
  if (h->opts.device_loops) return MG_ERR_UNSUPPORTED;
  h->rec_r = r;
  h->rec_y = y;
  h->rec_max = max_pairs;
  h->rec_count = 0;
  return MG_OK;
}

int mg_recorded_pairs(const mg_handle *h) { return h ? h->rec_count : MG_ERR_ARG; }

}  // extern "C"

// ===========================================================================
// Autotuner: picks, per problem shape, the fastest SGS chain evaluation
// (parallel scan, thread-block-cluster chain or single-CTA chain; equal up to
// rounding) and the basis-vector blocking of the dot products (4, 8 or 16 per
// CTA; bitwise the same results) by timing them on the handle's own levels.
// Choices are cached for the process by shape.

namespace {

struct TuneChoice {
  int chain = 0;   // 0 scan, 1 cluster, 2 single CTA, 3 segmented
  int dot_vb = 8;
  std::vector<std::pair<int, int>> bs;  // (level steps, block-solve mapping 1 or 2) of the smoothing levels
  float ms_chain[4] = {-1.f, -1.f, -1.f, -1.f};
  float ms_dot[3] = {-1.f, -1.f, -1.f};  // VB 4, 8, 16
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, TuneChoice> g_tune_cache;

template <typename F>
float time_min(cudaStream_t s, int reps, F &&f) {
  cudaEvent_t a, b;
  ck(cudaEventCreate(&a));
  ck(cudaEventCreate(&b));
  f();  // warm-up
  float best = 1e30f;
  for (int i = 0; i < reps; ++i) {
    ck(cudaEventRecord(a, s));
    f();
    ck(cudaEventRecord(b, s));
    ck(cudaEventSynchronize(b));
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

template <typename T>
void tune_chain(mg_handle *h, Level &lev, TuneChoice &c, cudaStream_t s) {
  LevelData<T> &d = ldata<T>(lev);
  const bool has_scan = lev.n == 1 || !d.scanF.empty();
  const bool has_cluster = h->layout == MG_LAYOUT_TRIDIAG && h->p >= 32;
  const bool has_seg = d.segF != nullptr;
  // input: the level's scratch vector (zeroed); output: its y vector, or the coarse
  // GMRES's preconditioner slot on a single-level FP64 handle (no y there)
  T *in = d.tmp;
  T *out = d.y ? d.y : reinterpret_cast<T *>(h->czout);
  ck(cudaMemsetAsync(in, 0, lev.len * sizeof(T), s));
  const int save_scan = h->use_scan, save_cluster = h->use_cluster, save_seg = h->use_seg;
  for (int k = 0; k < 4; ++k) {
    if ((k == 0 && !has_scan) || (k == 1 && !has_cluster) || (k == 3 && (!has_seg || !has_cluster))) continue;
    h->use_scan = k == 0;
    h->use_cluster = k == 1 || k == 3;
    h->use_seg = k == 3;
    c.ms_chain[k] = time_min(s, 3, [&] { sgs_apply<T>(h, lev, in, out, s); });
  }
  h->use_scan = save_scan;
  h->use_cluster = save_cluster;
  h->use_seg = save_seg;
  int best = -1;
  for (int k = 0; k < 4; ++k)
    if (c.ms_chain[k] >= 0.f && (best < 0 || c.ms_chain[k] < c.ms_chain[best])) best = k;
  c.chain = best < 0 ? 2 : best;
}

// one block-Jacobi sweep of level `lev` (zero data in `scratch`, at least 3 level
// vectors of T) with one and with two warps per block, where both apply (tridiagonal
// blocks staged in shared memory); returns the faster mapping, or 0
template <typename T>
int tune_block_map(mg_handle *h, Level &lev, void *scratch, cudaStream_t s) {
  const LevelView<T> &L = ldata<T>(lev).view;
  if (L.layout != MG_LAYOUT_TRIDIAG || !h->pair_tri || !tri_stage_ok(L)) return 0;
  T *r = static_cast<T *>(scratch), *y = r + lev.len, *out = y + lev.len;
  ck(cudaMemsetAsync(r, 0, 2 * lev.len * sizeof(T), s));
  Vec<T> Y = make_vec(y, lev.n, h->p, h->q);
  float ms[2];
  for (int k = 0; k < 2; ++k) {
    h->bs_map[lev.n] = k + 1;
    ms[k] = time_min(s, 5, [&] { launch_block_solve<T>(h, L, r, Y.u, Y.m, out, s); });
  }
  h->bs_map.erase(lev.n);
  return ms[1] < ms[0] ? 2 : 1;
}

}  // namespace

extern "C" int mg_block_mapping(const mg_handle *h, int level) {
  if (!h || level < 0 || level >= (int)h->lv.size()) return MG_ERR_ARG;
  const int n = h->lv[level].n;
  const auto it = h->bs_map.find(n);
  if (it != h->bs_map.end()) return it->second;
  const LevelView<double> &L = h->lv[level].d.view;
  if (h->layout != MG_LAYOUT_TRIDIAG) return 1;
  return (h->pair_tri && n + 1 <= kPairMaxBlocks && L.p <= 4 * kWarp) ? 2 : 1;
}

extern "C" int mg_autotune(mg_handle *h, int *chain, int *dot_vb, void *stream) {
  if (!h) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto key = std::make_tuple(h->layout, h->lv.back().n, h->p, h->q, h->lv[0].n, h->opts.precision);
  TuneChoice c;
  bool hit = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c = it->second;
      hit = true;
    }
  }
  const bool env_chain = std::getenv("PINTMG_SGS_CHAIN") != nullptr;  // a forced chain is kept
  const long long saved = h->launches;
  const int saved_prof = h->prof;
  h->prof = 0;
  int status = MG_OK;
  double *tmp = nullptr;
  try {
    if (!hit) {
      Level &cl = h->lv.back();
      if (!env_chain) {
        if (h->opts.precision == MG_PRECISION_FP32 || h->opts.precision == MG_PRECISION_BF16_BANDS)
          // the coarse SGS runs in FP32 only in these modes
          tune_chain<float>(h, cl, c, s);
        else
          tune_chain<double>(h, cl, c, s);
      }
      // dot products at the fine level's own length against 16, 64, 128 and 240 basis
      // vectors (a spread of Arnoldi indices; fewer where 2 GiB of scratch does not hold
      // them), summed, for VB = 4, 8, 16: the partition and the occupancy both depend on
      // the length and the count
      const long long tl = h->lv[0].len;
      const int kM = (int)std::max<long long>(16, std::min<long long>(240, (1LL << 28) / tl - 1));
      cudaError_t e = cudaMalloc(&tmp, (size_t)(kM + 1) * tl * sizeof(double));
      if (e != cudaSuccess) {
        cudaGetLastError();
        tmp = nullptr;
        throw std::bad_alloc();
      }
      ck(cudaMemsetAsync(tmp, 0, (size_t)(kM + 1) * tl * sizeof(double), s));
      const int save_vb = h->dot_vb;
      const int vbs[3] = {4, 8, 16};
      const int ms[4] = {16, 64, 128, 240};
      int best = 1;
      for (int k = 0; k < 3; ++k) {
        h->dot_vb = vbs[k];
        c.ms_dot[k] = 0.f;
        for (int mm : ms) {
          const int m = std::min(mm, kM);
          c.ms_dot[k] += time_min(s, 3, [&] { multidot(h, tmp, tl, m, tmp + (long long)kM * tl, tl, h->kf.h, 0, s); });
        }
        if (c.ms_dot[k] < c.ms_dot[best]) best = k;
      }
      h->dot_vb = save_vb;
      c.dot_vb = vbs[best];
      // block-solve mapping of every smoothing level (the sweeps' kernel)
      const bool f32 = h->opts.precision == MG_PRECISION_FP32 || h->opts.precision == MG_PRECISION_FP32_SMOOTH;
      for (size_t l = 0; l + 1 < h->lv.size(); ++l) {
        if (h->opts.precision == MG_PRECISION_BF16_BANDS) break;  // the BF16-band view keeps the size rule
        const int m = f32 ? tune_block_map<float>(h, h->lv[l], tmp, s) : tune_block_map<double>(h, h->lv[l], tmp, s);
        if (m) c.bs.emplace_back(h->lv[l].n, m);
      }
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = c;
    }
    if (!env_chain) {
      h->use_scan = c.chain == 0;
      h->use_cluster = c.chain == 1 || c.chain == 3;
      h->use_seg = c.chain == 3;
    }
    h->dot_vb = c.dot_vb;
    for (const auto &kv : c.bs) h->bs_map[kv.first] = kv.second;
    h->gen++;  // captured graphs used the previous choices
  } catch (const CudaFail &) {
    status = MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    status = MG_ERR_OOM;
  }
  if (tmp) cudaFree(tmp);
  h->launches = saved;
  h->prof = saved_prof;
  if (status == MG_OK) {
    if (chain) *chain = env_chain ? (h->use_scan ? 0 : (h->use_seg ? 3 : (h->use_cluster ? 1 : 2))) : c.chain;
    if (dot_vb) *dot_vb = c.dot_vb;
  }
  return status;
}

// ===========================================================================
// Spectral radius of the block-Jacobi iteration (Table 2) by power iteration

extern "C" int mg_jacobi_radius(mg_handle *h, int level, int iters, double *rho, void *stream) {
  if (!h || !rho || level < 0 || level >= (int)h->lv.size() || iters < 8) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Level &lev = h->lv[level];
  const long long len = lev.len;
  const LevelView<double> &L = lev.d.view;
  double *buf = nullptr;
  int status = MG_OK;
  try {
    // x, y, a zero right-hand side, |y|^2 and the log accumulator
    cudaError_t e = cudaMalloc(&buf, (3 * (size_t)len + 8) * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      buf = nullptr;
      throw std::bad_alloc();
    }
    double *x = buf, *y = buf + len, *zero = buf + 2 * len, *nrm2 = buf + 3 * len, *acc = nrm2 + 4;
    ck(cudaMemsetAsync(zero, 0, (len + 8) * sizeof(double), s));
    k_power_start<<<grid_for(len, 256), 256, 0, s>>>(x, len);
    ck_launch();
    const Vec<double> X = make_vec(x, L.n, L.p, L.q);
    for (int k = 0; k < iters; ++k) {
      // y = D^-1 (0 - (L + L^T) x) = (I - D^-1 A) x: one undamped sweep from x with a zero right-hand side
      launch_block_solve<double>(h, L, zero, X.u, X.m, y, s);
      multidot(h, y, len, 1, y, len, nrm2, 0, s);
      k_power_step<<<grid_for(len, 256), 256, 0, s>>>(y, x, len, nrm2, acc, k >= iters / 2);
      ck_launch();
    }
    double a[2] = {0.0, 0.0};
    ck(cudaMemcpyAsync(a, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    *rho = a[1] > 0.0 ? std::exp(a[0] / a[1]) : 0.0;
  } catch (const CudaFail &) {
    status = MG_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    status = MG_ERR_OOM;
  }
  if (buf) {
    cudaStreamSynchronize(s);
    cudaFree(buf);
  }
  return status;
}
