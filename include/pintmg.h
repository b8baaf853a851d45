/*
 * pintmg.h - C ABI of the GB300 parallel-in-time multigrid solver for
 * augmented systems (Vuchkov, Cyr, Javeed, Ridzal, arXiv 2405.04808).
 *
 * The library solves A x = b with A = [[I, B^T], [B, 0]] (Eq. augsys-aj),
 * where B = dF~ is the scaled Jacobian of the theta-method constraint with
 * virtual interface variables (Eq. theta2-aj, Sec. 4.1 and Sec. 5.1), by
 * flexible GMRES (Saad 1993; Sec. 5.3.4 and Sec. 6) preconditioned with a
 * multigrid V-cycle in time (Alg. 1): block-Jacobi smoothing (Eq. jacobi-aj),
 * linear interpolation / injection in time (Sec. 5.3.1) and a coarse solve by
 * GMRES right-preconditioned with symmetric block Gauss-Seidel (Sec. 5.3.4).
 *
 * Vectors (both host and device) are type-major as in Fig. 4:
 *   [u_1..u_n | v_1..v_n | z_1..z_n | lambda_1..lambda_n | mu_1..mu_n],
 * each step contiguous (p entries, q for z), n (4p + q) doubles in all, in the
 * scaled Euclidean coordinates of Sec. 4.1.
 *
 * Errors: every entry point returns an mg_status code; nothing aborts, traps
 * or throws.  One kernel waits on the device: the streamed multi-dot of the
 * FP32-pair Krylov basis (MG_BASIS_PAIR) polls shared-memory barriers for its
 * copies, at most 2 s per wait (%globaltimer); a wait that runs out ends the
 * kernel, after its issued copies have landed, and the solve returns
 * MG_ERR_TIMEOUT.  No other kernel waits on anything.
 * Threading: one handle is used by one host thread and one stream at a time.
 */
#ifndef PINTMG_H
#define PINTMG_H

#ifdef __cplusplus
extern "C" {
#endif

#define PINTMG_ABI_VERSION 2

typedef enum {
  MG_OK = 0,
  MG_NOT_CONVERGED = 1,   /* ran to maxit; outputs hold the last iterate */
  MG_ERR_ARG = -1,        /* invalid sizes, options or null pointers */
  MG_ERR_SINGULAR = -2,   /* a local Schur complement S_k had a non-positive pivot (Thm 1: N_k singular) */
  MG_ERR_BREAKDOWN = -3,  /* Arnoldi produced a non-finite Hessenberg entry */
  MG_ERR_CUDA = -4,       /* a CUDA runtime call failed; mg_last_cuda_error() names it */
  MG_ERR_OOM = -5,        /* device allocation failed */
  MG_ERR_TIMEOUT = -6,    /* a bounded device-side wait ran out (the copy pipeline of a streaming kernel);
                             the solve's outputs are not valid */
  MG_ERR_NONFINITE = -7,  /* NaN or Inf in the problem data or right-hand side */
  MG_ERR_UNSUPPORTED = -8 /* a valid request this build does not implement (e.g. p too large for the dense layout) */
} mg_status;

typedef enum {
  MG_LAYOUT_DENSE = 0,   /* blocks stored dense, row-major; p <= 32, q <= 32 (a thread per time block up to 4,
                            a warp per time block beyond) */
  MG_LAYOUT_TRIDIAG = 1  /* q == p, every p x p block tridiagonal (band rows, below) */
} mg_layout;

typedef enum {
  MG_PRECISION_FP64 = 0,        /* the plain method: every step in FP64 */
  MG_PRECISION_FP32 = 1,        /* V-cycle (smoother, transfers, SGS) in FP32; FGMRES, coarse GMRES and true
                                   residual in FP64 */
  MG_PRECISION_FP32_SMOOTH = 2, /* smoother and transfers in FP32; the coarse solve (GMRES and its SGS), FGMRES
                                   and true residual in FP64 */
  MG_PRECISION_BF16_BANDS = 3   /* as MG_PRECISION_FP32, with the N, V, Z~ bands of every level but the coarsest
                                   stored in BF16 (rounded to nearest from their FP32 values) and every product
                                   formed in FP32: half the bytes of those bands per sweep and residual.  The
                                   local factor, the coarsest level and the FGMRES operator keep their precision.
                                   Tridiagonal layout only (else MG_ERR_UNSUPPORTED) */
} mg_precision;

/*
 * Storage of the FGMRES Krylov basis v_0..v_m (the vectors CGS2 orthogonalises
 * against, Sec. 5.3.4 / Saad 1993).  The preconditioned vectors z_j, the
 * solution and the true residual stay FP64 in both modes.
 */
typedef enum {
  MG_BASIS_FP64 = 0,  /* FP64 vectors; dot products and axpys in FP64 (the default) */
  MG_BASIS_PAIR = 1,  /* each entry as two FP32 values hi + lo (the FP64 value rounded to ~48 bits, 8 bytes);
                         dot products and axpys against the basis in compensated FP32 arithmetic (error-free
                         products and sums of Ogita, Rump and Oishi's Dot2) with FP64 reductions; on GB300,
                         whose FP64 rate bounds the FP64 kernels, these kernels run about 1.5x faster (the C2
                         solve 1.2x).  Requires an even vector length n (4p+q), else the FP64 basis is used.
                         Its streamed dot products wait on shared-memory barriers for at most 2 s each; a
                         wait that runs out makes the solve return MG_ERR_TIMEOUT */
  MG_BASIS_PAIR_DCGS2 = 2 /* the pair basis orthogonalised by delayed reorthogonalisation (DCGS2, Bielich et
                         al. 2022): at step j one pass over the basis forms V^T u and V^T w (u: the previous
                         step's vector, not yet reorthogonalised) and one pass writes the final V_j and the
                         projected w, half of classical Gram-Schmidt twice's four passes; column j - 1 of the
                         Hessenberg matrix is completed, rotated and tested one step late, so a converging
                         cycle runs one more preconditioner application, and a cycle that ends full runs one
                         more dot-product pass.  Requires what MG_BASIS_PAIR requires, else the FP64 basis
                         (with classical Gram-Schmidt twice) is used */
} mg_krylov_basis;

/*
 * Problem data (Eq. blocks-aj and Sec. 5.1).  All pointers are HOST memory,
 * read during mg_setup only, owned by the caller.
 *
 * Index t = 0..n-1 is the paper's step k = t + 1.  Raw Jacobians are taken at
 * physical (unscaled) points:
 *   Ju_cur[t]  = d_u f(u_{t+1}, z_{t+1}),   Ju_prev[t] = d_u f(v_t, z_{t+1})
 *   Jz_cur[t]  = d_z f(u_{t+1}, z_{t+1}),   Jz_prev[t] = d_z f(v_t, z_{t+1})
 * (v_0 = the initial state).  The library forms, per grid level,
 *   N_k  = dt^-1 [ M - theta dt Ju_cur ],   V_k = dt^-1 [ -M - (1-theta) dt Ju_prev ],
 *   Z~_k = -(theta Jz_cur + (1-theta) Jz_prev) / gamma.
 * Coarse levels are rediscretised at 2 dt with the Jacobians of fine step
 * 2K-1 (current) and 2K-2 (previous) in the paper's 1-based count; this is
 * exact when d_u f does not depend on z and f is affine in z, which the
 * caller asserts with `separable`.
 *
 * MG_LAYOUT_DENSE:   M is p*p, Ju_* are n*p*p, Jz_* are n*p*q (row-major blocks).
 * MG_LAYOUT_TRIDIAG: every p x p tridiagonal matrix is 3*p doubles,
 *                    band[0][i] = A[i][i-1] (band[0][0] ignored),
 *                    band[1][i] = A[i][i],
 *                    band[2][i] = A[i][i+1] (band[2][p-1] ignored);
 *                    M is 3*p, Ju_* and Jz_* are n*3*p.
 * jz_const != 0: Jz_cur and Jz_prev each hold ONE block used at every step.
 */
typedef struct {
  int layout;        /* mg_layout */
  int n, p, q;       /* time steps, states, controls */
  double theta;      /* theta-method weight, 0 < theta <= 1 (Eq. theta-aj) */
  double gamma;      /* control scale factor gamma > 0 (Sec. 4.1, Sec. 5.3.3) */
  int jz_const;
  const double *M;
  const double *Ju_cur, *Ju_prev, *Jz_cur, *Jz_prev;
  int separable;     /* 1: d_u f does not depend on z and f is affine in z (both of Sec. 6's problems).  The
                        coarse levels are rediscretised from the fine Jacobians (above), which is exact only
                        then; levels > 1 with separable = 0 are rejected with MG_ERR_ARG (levels = 1, GMRES
                        with SGS alone, needs no coarse operator and accepts either value) */
} mg_problem;

/* Block fixed-point iterations of Sec. 5.3.4 / Table 1, one step from zero,
 * as the right preconditioner of the coarse GMRES (with levels = 1: of GMRES
 * on the whole system, the paper's serial baseline of Sec. 6.3). */
typedef enum {
  MG_COARSE_SGS = 0,     /* [(D + L) D^-1 (D + L^T)]^-1, the paper's coarse solver */
  MG_COARSE_JACOBI = 1,  /* D^-1 */
  MG_COARSE_FGS = 2,     /* (D + L)^-1 */
  MG_COARSE_BGS = 3      /* (D + L^T)^-1 */
} mg_coarse_precond;

/*
 * Restriction of the residual in the V-cycle (Alg. 1, step 2; Sec. 5.3.1).
 * The paper states its transfers for the variables: linear interpolation and
 * injection at fine step 2k-1 for u, v, lambda, mu; piecewise-constant
 * interpolation and averaging for z.  The residual it restricts is a dual
 * vector (the rows of A~).
 */
typedef enum {
  MG_RESTRICT_INJECT = 0,    /* the variable formulas applied to the residual: r^c_k = r_{2k-1} (u, v, lambda,
                                mu), (r_{2k-1} + r_{2k}) / 2 (z) */
  MG_RESTRICT_TRANSPOSE = 1  /* the transpose of the interpolation, R = P^T: r^c_k = r_{2k-1} + (r_{2k-2} +
                                r_{2k}) / 2 (u, v, lambda, mu; the last coarse step takes r_{2k} with the end
                                rule's weight), r_{2k-1} + r_{2k} (z).  With a weighted sweep (omega = 2/3) the
                                iteration counts grow logarithmically in n as in Tables 3-4; with omega = 1
                                neither rule does, because the undamped sweep never damps modes that
                                alternate from step to step */
} mg_restrict_rule;

typedef struct {
  int levels;             /* V-cycle levels Lv >= 1; n must be divisible by 2^(Lv-1); Lv = 1 is SGS-GMRES alone */
  int nu_pre, nu_post;    /* block-Jacobi sweeps before / after the coarse correction (>= 0) */
  double coarse_rtol;     /* coarse GMRES relative tolerance (the paper uses 1e-3) */
  int coarse_maxit;       /* coarse GMRES iteration cap (1..64) */
  int coarse_fixed_iters; /* > 0: run exactly this many coarse GMRES iterations, ignoring coarse_rtol */
  int end_rule;           /* last fine point of linear interpolation: 0 repeats the last coarse value, 1 uses 0 */
  int precision;          /* mg_precision */
  double omega;           /* block-Jacobi relaxation weight, 0 < omega <= 1; the paper's sweep (Eq. jacobi-aj) is omega = 1 */
  int coarse_precond;     /* mg_coarse_precond: preconditioner of the coarse GMRES (the paper's is SGS) */
  int device_loops;       /* 1: each fgmres_solve runs as one CUDA graph whose FGMRES and coarse-GMRES loops are
                             conditional nodes decided on the device (one host read-back per solve);
                             0: loops driven from the host (a few scalars read back per iteration).
                             Same arithmetic either way. */
  int krylov_basis;       /* mg_krylov_basis of the FGMRES basis */
  int restrict_rule;      /* mg_restrict_rule: how the V-cycle restricts the residual (Alg. 1, step 2) */
} mg_options;

typedef struct {
  int status;             /* mg_status of this solve */
  int iters;              /* FGMRES iterations taken */
  int vcycles;            /* preconditioner applications */
  int coarse_iters;       /* coarse GMRES iterations summed over all V-cycles */
  double relres;          /* Arnoldi estimate ||b - A x|| / ||b|| at exit */
  double true_relres;     /* recomputed ||b - A x|| / ||b|| at exit (FP64) */
  int coarse_learned;     /* coarse solves answered by an attached network (mg_attach_coarse_net), else 0 */
} mg_solve_info;

typedef struct mg_handle mg_handle;  /* opaque; owns every device buffer */

/* Fill *opts with the defaults: levels 2, 1/1 sweeps, coarse 1e-3 / 50, tolerance mode, end rule 0, FP64,
 * omega 1, SGS coarse preconditioner, device loops, FP64 basis, injection of the residual. */
void mg_default_options(mg_options *opts);

/*
 * Build the hierarchy: scaled blocks on every level and their local
 * Schur-complement factors (Thm 1), all on the device, on `stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  Host data are
 * copied; the caller may free them on return.  On success *out owns all
 * device memory until mg_destroy.  Returns MG_ERR_ARG, MG_ERR_NONFINITE,
 * MG_ERR_SINGULAR, MG_ERR_OOM, MG_ERR_UNSUPPORTED or MG_ERR_CUDA on failure,
 * leaving *out NULL.
 */
int mg_setup(const mg_problem *prob, const mg_options *opts, void *stream, mg_handle **out);

/*
 * One V-cycle (Alg. 1 generalised to Lv levels, starting from y = 0):
 * y = M^-1 r.  r and y are DEVICE pointers to type-major vectors of n (4p+q)
 * doubles; they must not overlap.  Asynchronous on `stream` except for the
 * coarse GMRES convergence tests, which read a few scalars back.
 */
int mg_vcycle(mg_handle *h, const double *r, double *y, void *stream);

/*
 * Solve A x = b by FGMRES(restart) from x0 = 0, preconditioned by the
 * V-cycle, until ||b - A x|| / ||b|| <= rtol (Arnoldi estimate) or maxit
 * iterations.  b and x may be HOST or DEVICE pointers (detected per call);
 * host buffers are staged through the handle's device memory on `stream`.
 * info (may be NULL) receives the counters and the FP64 true residual.
 * Returns MG_OK, MG_NOT_CONVERGED, MG_ERR_NONFINITE (b has NaN/Inf),
 * MG_ERR_BREAKDOWN, MG_ERR_TIMEOUT, MG_ERR_ARG or MG_ERR_CUDA.  Synchronises
 * `stream`.
 */
int fgmres_solve(mg_handle *h, const double *b, double *x, double rtol, int maxit, int restart,
                 mg_solve_info *info, void *stream);

/*
 * Solve `count` independent systems (each with its own handle, so sizes,
 * layouts and options may differ) in ONE CUDA graph launch: every system is
 * a branch of the graph with its own device-side FGMRES and coarse-GMRES
 * loops, so the branches run concurrently and the host reads back once for
 * the whole batch.  b[i], x[i] are DEVICE pointers; the graph is built on the
 * first call and reused while the handles, vectors, rtol, maxit and restart
 * stay the same (one cached batch graph per host thread).  infos (may be
 * NULL) receives count entries with each solve's status.  Returns the most
 * severe status: an error code if any solve failed, else MG_NOT_CONVERGED if
 * any did not converge, else MG_OK.  Synchronises `stream`.
 */
int fgmres_solve_batched(mg_handle *const *hs, int count, const double *const *b, double *const *x, double rtol,
                         int maxit, int restart, mg_solve_info *infos, void *stream);

/* Sizes of a handle: the vector length n (4p+q) and the number of levels. */
long long mg_vector_length(const mg_handle *h);

/*
 * Measurement support (no counterpart in the paper).  mg_launch_count returns
 * the number of kernels the handle has launched since mg_setup returned.
 * mg_profile_enable(h, mask) brackets every later kernel launch of the
 * handle whose category bit is set in `mask` (bit c = the c-th category of
 * mg_profile_read; 0 turns timing off) with a pair of CUDA events on its
 * stream, and resets the per-category sums;
 * mg_profile_read synchronises those events and fills up to `max` entries of
 * names (static strings), ms (summed kernel time), launches (count), bytes and
 * flops (the algorithmic memory traffic and floating-point operations of the
 * timed launches: each launch adds the bytes its kernel must move at least,
 * every input and output touched once, and the flops its arithmetic needs)
 * per kernel category; any output pointer may be NULL.  It returns the number
 * of categories or a negative status.
 */
long long mg_launch_count(const mg_handle *h);

/*
 * Kernel launches of the handle's captured single-system solve graph
 * (options.device_loops), as recorded when the graph was last built by
 * fgmres_solve: *fixed = the launches outside the loops (start and final
 * residual), *per_iter = one pass of the FGMRES WHILE body (preconditioner,
 * operator product, Gram-Schmidt, step control, guarded restart block),
 * counting the coarse-grid GMRES loop inside each V-cycle as absent, and
 * *per_coarse_iter = one pass of the coarse GMRES WHILE body.  Any output
 * pointer may be NULL.  Returns MG_OK, or MG_ERR_ARG when h is NULL or no
 * graph has been built yet (all outputs then set to 0).
 */
int mg_graph_launches(const mg_handle *h, long long *fixed, long long *per_iter, long long *per_coarse_iter);

/*
 * Arithmetic-rate probe (measurement support, no counterpart in the paper):
 * launches `blocks` CTAs of 256 threads on `stream`, each thread running 8
 * independent fused multiply-add chains of `iters` steps in FP64
 * (precision = MG_PRECISION_FP64) or FP32 (MG_PRECISION_FP32), then writing
 * one value per thread to `sink` (a DEVICE buffer of blocks * 256 elements of
 * that type, owned by the caller).  The launch does 2 * 8 * iters * blocks *
 * 256 floating-point operations; timing it with events on `stream` gives the
 * FMA rate the FP64 (or FP32) kernels' rooflines are measured against.
 * Asynchronous; returns MG_ERR_ARG for bad arguments, MG_ERR_CUDA if the
 * launch fails.
 */
int mg_probe_fma(int precision, int blocks, int iters, void *sink, void *stream);
int mg_profile_enable(mg_handle *h, int mask);
int mg_profile_read(mg_handle *h, int max, const char **names, double *ms, long long *launches, double *bytes,
                    double *flops);

/*
 * Time-range operations, for a V-cycle sharded across processes by time
 * (each process owns a contiguous range of time blocks on every level and
 * exchanges the couplings at the range ends; Sec. 5.3.2: the block-Jacobi
 * sweep parallelises trivially in time, and the residual and the transfers
 * of Sec. 5.3.1 couple neighbouring steps only).  Time block j = 0..n_l of
 * level l holds u_j, z_j, lambda_j (j < n_l) and v_{j-1}, mu_{j-1} (j >= 1).
 * Every vector is a full level-length FP64 DEVICE vector (mg_level_info), type
 * major as above; only the entries named below are read or written, so each
 * process may leave the rest unset.  FP64 levels of the handle (its
 * precision option is ignored); the handle's omega, restriction rule and end
 * rule apply.  Asynchronous on `stream` (mg_coarse_solve synchronises);
 * MG_ERR_ARG for a bad level, range or pointer, MG_ERR_CUDA if a launch fails.
 *
 * mg_level_info: n_l (time steps) and the vector length n_l (4p + q).
 * mg_range_sweep: one block-Jacobi sweep (Eq. jacobi-aj) of blocks [j0, j1)
 *   of a smoothing level (not the coarsest): y = D^-1 (r - C yold) on those
 *   blocks, relaxed by omega; yold NULL sweeps from y = 0.  Reads r and yold
 *   of the blocks and the couplings u_{j0-1} (block j0 - 1) and mu_{j1-1}
 *   (block j1) of yold.  y must not alias yold.
 * mg_range_residual: r = b - A~ y on the rows of blocks [j0, j1); reads y on
 *   the blocks and u_{j0-1}, mu_{j1-1}.  b NULL: r = A~ y (the operator
 *   product of the Arnoldi step).  r must not alias y.
 * mg_range_restrict: the restricted residual (Alg. 1, step 2, by the handle's
 *   restriction rule) on the coarse blocks [j0 / 2, (j1 + 1) / 2) of level + 1
 *   (j0 even); reads the fine residual r on blocks [j0 - 2, j1).
 * mg_range_prolong: y += P e (Sec. 5.3.1) on blocks [j0, j1) of the level;
 *   reads the coarse correction e on coarse blocks [j0 / 2, (j1 + 1) / 2 + 1).
 * mg_coarse_solve: the coarsest level's solve of the V-cycle (GMRES with SGS,
 *   the handle's coarse options) on a full coarse vector; FP64 handles only
 *   (else MG_ERR_UNSUPPORTED); synchronises `stream`.
 *
 * The vector work of an FGMRES around the sharded cycle (the outer solver of
 * Sec. 6): every process forms its share of the Gram-Schmidt dot products
 * over its own entries (the entries of blocks [j0, j1), as above) and the
 * processes sum the shares (an allreduce of k values), then every process
 * updates its own entries.  V is k vectors of the level's length at a stride
 * of ldv >= the length doubles; 1 <= k <= 512; coefficient and result arrays
 * are DEVICE arrays of k doubles.  These calls use the handle's reduction
 * scratch: do not overlap them with another call on the same handle.
 * mg_range_dots: out[i] = sum over the entries e of blocks [j0, j1) of
 *   V_i[e] w[e], i < k (per type run a fixed-order blocked sum, the runs
 *   added in storage order; V may be w for a squared norm).
 * mg_range_axpy: w[e] += sign * sum_{i < k} c[i] V_i[e] on those entries
 *   (each entry's sum over i in order).
 * mg_range_scale: y[e] = a[0] x[e] on those entries (a: one DEVICE double;
 *   y may be x).
 */
int mg_level_info(const mg_handle *h, int level, int *n, long long *len);
int mg_range_sweep(mg_handle *h, int level, int j0, int j1, const double *r, const double *yold, double *y,
                   void *stream);
int mg_range_residual(mg_handle *h, int level, int j0, int j1, const double *y, const double *b, double *r,
                      void *stream);
int mg_range_restrict(mg_handle *h, int level, int j0, int j1, const double *r, double *rc, void *stream);
int mg_range_prolong(mg_handle *h, int level, int j0, int j1, const double *ec, double *y, void *stream);
int mg_coarse_solve(mg_handle *h, const double *rc, double *yc, void *stream);
int mg_range_dots(mg_handle *h, int level, int j0, int j1, const double *V, long long ldv, int k, const double *w,
                  double *out, void *stream);
int mg_range_axpy(mg_handle *h, int level, int j0, int j1, const double *V, long long ldv, int k, const double *c,
                  double sign, double *w, void *stream);
int mg_range_scale(mg_handle *h, int level, int j0, int j1, const double *x, const double *a, double *y,
                   void *stream);

/*
 * True residual without allocating (the paper has no counterpart).  For
 * callers that must not allocate device memory when they check a solution
 * (a framework's caching allocator owns the device pool, a real-time loop
 * with a fixed memory budget, an outer optimisation loop testing its stopping
 * rule), computes on `stream`, asynchronously:
 *   out[0] = ||b - A x||_2,   out[1] = ||b - A x||_2 / ||b||_2  (0 if b = 0)
 * with the same FP64 residual kernel as fgmres_solve's reported true
 * residual and fixed-order reductions (a different partition of the sums,
 * so the two agree to rounding, not bitwise).  b, x and out (2 doubles) are DEVICE pointers owned by the
 * caller.  It calls no cudaMalloc, cudaFree or allocating library routine:
 * its scratch (residual vector, reduction partials) is one file-scope device
 * array of 2^20 + 616 doubles (about 8 MiB), held by every GPU that loads the
 * library until the process exits.  Vectors longer than 2^20 doubles are
 * rejected with MG_ERR_ARG (mg_last_cuda_error() says why).  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The device current at the
 * call must be the one the handle was set up on (else MG_ERR_ARG, with
 * mg_last_cuda_error() naming both).  Every call overwrites the
 * same array, so calls that overlap on the GPU (other streams, other host
 * threads) race; serialise them.
 */
int mg_true_residual_noalloc(mg_handle *h, const double *b, const double *x, double *out, void *stream);

/*
 * Learned coarse-grid correction.  A small network proposes the coarse solve
 * of the V-cycle (the step the paper does with GMRES preconditioned by SGS,
 * Sec. 5.3.4); the paper has no network, this is an extension.  Fixed
 * architecture: four 2-D convolutions over (time, space) with 3 x 7 kernels
 * and zero "same" padding, channels 5 -> 32 -> 32 -> 32 -> 5, leaky rectifier
 * (slope 0.1) after the first three; mg_net_param_count() = 49,829 FP32
 * parameters, flat, layer by layer, each layer's weights W[o][c][i][j]
 * (i: time tap, j: space tap) followed by its biases.  A tensor is NCHW
 * (batch, channel, T, X), FP32, contiguous; a coarse type-major vector
 * (u, v, z, lambda, mu, each n_c x p) is exactly one (5, n_c, p) sample.
 *
 * mg_net_create copies `init_params` (HOST, mg_net_param_count() floats) and
 * allocates the parameters, the gradient and Adam's moments on the current
 * device.  mg_net_set_params / mg_net_get_params / mg_net_get_grad copy
 * HOST <-> device and synchronise.  mg_net_forward runs the network on x
 * (DEVICE, batch x 5 x T x X) into y (DEVICE, same shape; x == y allowed):
 * bf16 = 0 in FP32, bf16 = 1 with parameters and activations stored in BF16
 * and FP32 accumulation.  mg_net_loss_grad computes L = mean((net(x) -
 * target)^2) in FP32, writes *loss (HOST) and leaves dL/dparams in the
 * network's gradient buffer (synchronises `stream`).  mg_net_adam_step takes
 * one Adam step (Kingma and Ba 2015, bias-corrected) from that gradient.
 * mg_net_train runs `epochs` passes of minibatch Adam (lr, betas 0.9 and
 * 0.999, eps 1e-8) over `count` samples (x_all, y_all: DEVICE, count x 5 x T
 * x X), the sample order reshuffled every epoch from `seed` (splitmix64
 * Fisher-Yates); epoch_loss (HOST, may be NULL) receives each epoch's mean
 * minibatch loss.  normalize = 1 trains in per-channel normalised
 * coordinates: with sx, sy the root mean squares of x_all's and y_all's five
 * channels, training runs on (x / sx, y / sy) from zero Adam moments and at
 * the end the scalings are folded into the parameters (first layer's weights
 * divided by sx of their input channel, last layer's weights and biases times
 * sy of their output channel), so the result maps x to y.  A network that has
 * taken optimiser steps before is first mapped to normalised coordinates (the
 * inverse fold: same function); a fresh network's parameters are taken as
 * the normalised network's initial parameters.  Losses are then those of the
 * normalised targets.  Workspaces grow on demand
 * (about 8 x batch x 32 x T x X floats for training).  Errors: MG_ERR_ARG for
 * bad sizes (batch 1..32767, T 1..262140) or NULL pointers, MG_ERR_OOM, MG_ERR_CUDA.
 */
typedef struct mg_net mg_net;  /* opaque; owns its device buffers */
long long mg_net_param_count(void);
int mg_net_create(const float *init_params, mg_net **out);
int mg_net_set_params(mg_net *net, const float *params);
int mg_net_get_params(const mg_net *net, float *params);
int mg_net_get_grad(const mg_net *net, float *grad);
int mg_net_forward(mg_net *net, const float *x, int batch, int T, int X, float *y, int bf16, void *stream);
int mg_net_loss_grad(mg_net *net, const float *x, const float *target, int batch, int T, int X, float *loss,
                     void *stream);
/*
 * Residual-metric loss (an extension; the paper trains no network).  A coarse
 * proposal e is admitted by its residual ||r - A_c e|| (mg_attach_coarse_net),
 * which the mean squared error of e against the coarse solution y does not
 * control: A_c amplifies some error components far more than others.  After
 * mg_net_set_metric(net, h), mg_net_loss_grad and mg_net_train minimise
 *   L = sum_b ||A_c d_b||^2 / n,   d_b = s (net(x_b) - y_b),   n = batch 5 T X,
 * with A_c the coarsest-level operator of h (FP64, the library's own product;
 * it is symmetric), d_b in the type-major coarse layout of the samples, s = 1
 * in mg_net_loss_grad and the targets' per-channel scales sy in a normalised
 * mg_net_train (so L measures the unnormalised error); for y = A_c^-1 r this
 * is the mean squared residual of the proposals.  The samples' T and X must
 * be h's coarse shape (mg_coarse_shape; MG_ERR_ARG otherwise).  h is not owned
 * and must outlive its use; h = NULL restores the mean squared error.  Needs
 * an FP64 handle with q == p (MG_ERR_UNSUPPORTED otherwise).  Trained on the
 * metric of one system, the network may serve other systems of similar
 * operators: the admission test always uses the solved system's own A_c.
 */
int mg_net_set_metric(mg_net *net, mg_handle *h);
int mg_net_adam_step(mg_net *net, float lr, float beta1, float beta2, float eps, void *stream);
int mg_net_train(mg_net *net, const float *x_all, const float *y_all, int count, int T, int X, int batch,
                 int epochs, float lr, unsigned long long seed, int normalize, float *epoch_loss, void *stream);
void mg_net_destroy(mg_net *net);

/*
 * Use `net` (not owned; keep it alive while attached, NULL detaches) as the
 * coarse solve of h's V-cycles: with r the coarse residual (N entries) and
 * rms(r) = ||r|| / sqrt(N), the proposal is
 *   e = rms(r) net(r / rms(r))   (BF16 inference if bf16 = 1, else FP32),
 * and it is admitted when ||r - A_c e|| <= admit ||r|| (FP64 residual on the
 * coarse level); otherwise the coarse GMRES with SGS runs as without the
 * network, so it both measures the proposal and is the fallback.  FGMRES accepts the
 * resulting variable preconditioner.  Needs q == p and at most 262,140 coarse
 * steps (MG_ERR_UNSUPPORTED otherwise) and 0 < admit < 1.  Several handles
 * may share one network.  Parameter updates reach later solves (BF16 copies
 * are refreshed at the start of each fgmres_solve).
 *
 * mg_record_coarse(h, r, y, max_pairs) makes later host-driven solves
 * (options.device_loops = 0) record each coarse GMRES solve as a training
 * pair (r / rms(r), y / rms(r)) in FP32 into r, y (DEVICE, caller-owned,
 * max_pairs x 5 x n_c x p floats each) until max_pairs are stored; NULL
 * stops recording.  mg_recorded_pairs returns the number stored.  Returns
 * MG_ERR_UNSUPPORTED for device-loop handles.
 */
int mg_attach_coarse_net(mg_handle *h, mg_net *net, double admit, int bf16);
int mg_record_coarse(mg_handle *h, float *r, float *y, int max_pairs);
int mg_recorded_pairs(const mg_handle *h);
/* Coarse level shape (time steps n_c, space p) of a handle: the network's T and X. */
int mg_coarse_shape(const mg_handle *h, int *T, int *X);

/*
 * Autotuner (no counterpart in the paper).  Times, on h's own levels and on
 * `stream`, the candidate evaluations of the coarse SGS chains (parallel scan
 * with prefix products when they were formed, the 16-CTA cluster chain for
 * the tridiagonal layout with p >= 32, the single-CTA chain, and the
 * segmented chain when its in-segment products were formed: equal up to
 * rounding) and the dot-product blocking (4, 8 or 16 basis vectors per CTA:
 * bitwise equal), and makes the fastest ones h's choice.  Results are cached
 * for the process by (layout, coarse n, p, q, fine n, precision), so later
 * handles of the same shape take the cached choice without timing.  A chain
 * forced by the environment (PINTMG_SGS_CHAIN) is kept.  *chain (0 scan,
 * 1 cluster, 2 single CTA, 3 segmented) and *dot_vb (may be NULL) report the choice.
 * Allocates a temporary of (m + 1) x n(4p+q) doubles, m = 240 basis vectors or
 * fewer (at least 16) so that it stays near 2 GiB; synchronises
 * `stream`; invalidates h's captured graphs.
 */
int mg_autotune(mg_handle *h, int *chain, int *dot_vb, void *stream);
/*
 * Block-solve mapping of level `level` (0 = finest) as its sweeps launch it: 1 =
 * one warp per time block, 2 = two warps per time block (the split solve for
 * levels whose blocks alone do not fill the GPU).  mg_autotune times both on
 * every smoothing level where both apply and keeps the faster (the results
 * differ in rounding only: the two warps sum the right-hand side's parts in
 * another order); before that, or where only one applies, the size rule
 * decides (two warps up to 4096 blocks with p <= 128).  Returns the mapping,
 * or MG_ERR_ARG for a bad handle or level.
 */
int mg_block_mapping(const mg_handle *h, int level);

/*
 * Spectral radius of the undamped block-Jacobi iteration I - D^-1 A~ on level
 * `level` (0 = finest), the quantity of Table 2, by power iteration on the
 * device: `iters` sweeps (>= 8) of the smoother with a zero right-hand side
 * from a fixed start vector, each normalised; *rho = the geometric mean of the
 * norm ratios over the second half (robust to complex or +- pairs of dominant
 * eigenvalues).  FP64.  Allocates 3 level vectors for the call; synchronises.
 */
int mg_jacobi_radius(mg_handle *h, int level, int iters, double *rho, void *stream);

/* Release every device buffer of the handle.  NULL is accepted. */
void mg_destroy(mg_handle *h);

/* Static text for a status code. */
const char *mg_status_string(int status);

/* Name of the last CUDA error seen by this thread's library calls ("" if none). */
const char *mg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PINTMG_H */
