/*
 * tlr_mdd.h -- C ABI of the GB300 (sm_103a) library for reciprocity-aware
 * tile low-rank (TLR) multidimensional deconvolution, arXiv 2412.14973.
 *
 * One handle holds one frequency's problem (eq. 2): D(w), U(w) in C^{ns x nr},
 * unknown Green's function X = X^T in C^{nr x nr}.  The library reorders the
 * receivers along a Hilbert curve (eq. 10-14), normalises by alpha
 * (Hyper-parameter selection section), parametrises X_h by tiles (eq. 6-9) and
 * evaluates the operator, its adjoint, the misfit (eq. 17a), the factor
 * gradients (eq. 25-27) and the ADMM / L-BFGS solve (eq. 18-24) on the GPU.
 *
 * Conventions (all entry points):
 *   - Return 0 (TLR_OK) on success, a negative TLR_ERR_* code otherwise; no
 *     C++ exception crosses this boundary.  tlr_mdd_last_error() explains the
 *     last failure on a handle (or the last handle-less failure with NULL).
 *   - Complex numbers are complex64: interleaved (re, im) float pairs.
 *   - All matrices are row-major.  "Receiver-major" matrices have one row per
 *     receiver in Hilbert order (a = 0..nr-1) and one column per source.
 *   - Buffers passed in are owned by the caller and are device pointers unless
 *     a flag says host; the library never keeps a caller pointer past the call.
 *     The library owns its reordered data panels and its workspace.
 *   - Work is enqueued on the handle's stream; a call returns once its work is
 *     enqueued, except where a result is written to host memory (then it
 *     synchronises the stream first).
 *   - stream arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).
 */
#ifndef TLR_MDD_H
#define TLR_MDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TLR_OK               0
#define TLR_ERR_ARG         -1  /* NULL or out-of-range argument */
#define TLR_ERR_SHAPE       -2  /* nr % tile != 0 (or tile sizes not summing to nr), nx*ny != nr,
                                   rank outside [0, min(d_i, d_j)] */
#define TLR_ERR_UNSUPPORTED -3  /* a valid option this build does not implement */
#define TLR_ERR_NOMEM       -4  /* device allocation failed */
#define TLR_ERR_CUDA        -5  /* a CUDA runtime call failed */
#define TLR_ERR_NONFINITE   -6  /* NaN / Inf met in data or solver state */
#define TLR_ERR_TIMEOUT     -7  /* a bounded device wait gave up */
#define TLR_ERR_STATE       -8  /* call out of order (e.g. destroyed handle) */

/* ---- precision of the complex contractions ---- */
#define TLR_PREC_FP32   0  /* FP32 SIMT (CUDA cores), FP32 accumulation */
#define TLR_PREC_BF16X3 1  /* tcgen05 tensor cores: BF16 hi/lo split (3 products), 4M complex, FP32 accumulation */
#define TLR_PREC_TF32   2  /* tcgen05 tensor cores: operands rounded to TF32 (RN, ties away; 10 mantissa bits),
                              4M complex, FP32 accumulation.  The dense adjoint (tlr_mdd_adjoint) and the
                              benchmark solver of a TF32 handle compute in BF16x3. */

/* ---- diagonal tile representation (eq. 6 / eq. 7) ---- */
#define TLR_DIAG_RULE     0  /* dense iff k_ii >= d_i/4 (d_i: the tile size) */
#define TLR_DIAG_LOWRANK  1  /* every X_ii = Q_ii Q_ii^T */
#define TLR_DIAG_DENSE    2  /* every X_ii = P Z_ii = (Z_ii + Z_ii^T)/2 */
#define TLR_DIAG_PER_TILE 3  /* diag_dense[i] != 0 -> dense */

/* ---- reciprocity constraint (Receivers re-ordering / eq. 9) ---- */
#define TLR_RECIP_SYMMETRIC 0  /* X = X^T, super-diagonal tiles are plain transposes */
#define TLR_RECIP_NONE      1  /* general TLR X (the form the reciprocity reduction starts from,
                                  Tile Low-rank MDD section): every tile free, X_ij = L_ij R_ij^T
                                  for all i != j, X_ii = L_ii R_ii^T or dense Z_ii (no
                                  symmetrisation); the model is still D-hat X = U-hat */

/* ---- where a buffer lives ---- */
#define TLR_MEM_DEVICE 0
#define TLR_MEM_HOST   1

typedef struct tlr_mdd_s tlr_mdd_t;

/* Problem description (Theory section, eq. 2; Tile Low-rank MDD section). */
typedef struct {
    int64_t nr;              /* receivers (= virtual sources); X is nr x nr */
    int64_t ns;              /* sources (rows of D and U) */
    int32_t nx, ny;          /* receiver grid, natural index r = y*nx + x; nx*ny == nr.
                                Ignored when perm != NULL. */
    const int32_t* perm;     /* optional HOST array [nr]: perm[a] = natural index of the
                                receiver at position a (overrides the Hilbert order) */
    int32_t tile;            /* tile size b; nr % b == 0 (uniform partition, N = nr/b).
                                Ignored when tiles != NULL. */
    int32_t rank;            /* uniform rank k of every tile, used when ranks == NULL */
    const int32_t* ranks;    /* optional HOST array [N + N(N-1)/2]: the N diagonal
                                ranks, then the sub-diagonal pair ranks in stacking
                                order (column j ascending, row i > j ascending).
                                TLR_RECIP_NONE: [N + N(N-1)], the ordered pairs (i, j),
                                i != j, column j ascending, row i ascending.  Tile (i, j)
                                takes 0 <= k <= min(d_i, d_j). */
    int32_t diag_mode;       /* TLR_DIAG_* */
    const uint8_t* diag_dense; /* HOST [N], used with TLR_DIAG_PER_TILE */
    int32_t reciprocity;     /* TLR_RECIP_* */
    int32_t precision;       /* TLR_PREC_* */
    double alpha;            /* normalisation; 0 -> max_{s,r} |D[s,r]| of this D */
    int32_t input_memory;    /* TLR_MEM_* for D and U passed to tlr_mdd_create */
    int32_t ntiles;          /* N when tiles != NULL, else ignored */
    const int32_t* tiles;    /* optional HOST array [ntiles]: the tile sizes d_i >= 1
                                (block i = the d_i receivers after those of blocks
                                < i in Hilbert order), sum d_i == nr.  The paper's
                                partition is uniform but need not be (Tile Low-rank MDD
                                section); NULL -> N = nr/tile tiles of size tile. */
} tlr_mdd_desc_t;

/* Solver options (ADMM solver section; values the paper leaves open are
 * defaults of this library: rho = 1, 2 ADMM iterations per lambda stage,
 * 5 L-BFGS iterations per x-update, memory 10). */
typedef struct {
    double lam0;             /* first lambda (paper: 10) */
    double decay;            /* lambda_{s+1} = decay * lambda_s (paper: 0.1) */
    int32_t stages;          /* lambda stages (paper: 3) */
    int32_t admm_iters;      /* ADMM iterations per stage */
    int32_t lbfgs_iters;     /* L-BFGS iterations per x-update */
    int32_t memory;          /* L-BFGS memory m (1..32) */
    double rho;              /* ADMM penalty rho > 0 */
    int32_t theta_memory;    /* TLR_MEM_* of theta_inout */
    int32_t flags;           /* TLR_SOLVE_* bits, 0 by default */
} tlr_mdd_solve_opts_t;

/* Checkpoint / resume (the paper has none).  The L-BFGS memory is cleared at
 * every x-update, so the solver's state at an ADMM-iteration boundary is
 * theta, z and u.  TLR_SOLVE_RESUME: start from the handle's z, u (left by
 * the previous solve on the handle, or set with tlr_mdd_set_state) instead of
 * z = theta, u = 0.  TLR_SOLVE_REFRESH: recompute the residual and the factor
 * products from theta at every x-update after the first of the call (one
 * extra forward product and gradient per ADMM iteration) instead of carrying
 * the in-place updates; with it a solve split at ADMM-iteration boundaries
 * reproduces the uninterrupted solve bit for bit.  To continue a schedule at
 * lambda stage s, pass lam0 * decay^s (exactly) as lam0 and the remaining
 * stages; to split inside a stage, run its ADMM iterations in two calls. */
#define TLR_SOLVE_RESUME  1
#define TLR_SOLVE_REFRESH 2

#define TLR_MAX_HIST 1024
typedef struct {
    int32_t iters;           /* L-BFGS steps taken */
    int32_t restarts;        /* steps where the memory was cleared (no descent) */
    int32_t status;          /* TLR_OK or TLR_ERR_NONFINITE */
    int32_t n_hist;
    double f_hist[TLR_MAX_HIST]; /* data misfit f (eq. 17a) after each L-BFGS step */
    double f0;               /* f at the starting point */
    double gpu_ms;           /* device time of the solve (CUDA events) */
} tlr_mdd_stats_t;

/* Fill *d with defaults (SYMMETRIC, FP32, RULE, alpha = 0, device inputs). */
void tlr_mdd_desc_init(tlr_mdd_desc_t* d);
/* Fill *o with the paper's schedule (lam0 10, decay 0.1, 3 stages) and the
 * library defaults above. */
void tlr_mdd_solve_opts_init(tlr_mdd_solve_opts_t* o);

/* Number of complex entries of the stacked unknown theta = (Z-bar, L-bar, R-bar)
 * (Tile Low-rank MDD section) for this description. */
int tlr_mdd_theta_size(const tlr_mdd_desc_t* d, int64_t* n_theta);

/* Offsets (complex entries) of each block of theta, written to HOST arrays:
 * off_diag[N] (Q_ii d_i x k_ii, or Z_ii d_i x d_i), off_l[P] (L_ij, d_i x k_ij)
 * and off_r[P] (R_ij, d_j x k_ij), P = N(N-1)/2, pair order as for ranks; d_i
 * = b for a uniform partition.  Layout: all diagonal blocks in i order, then
 * L-bar, then R-bar; every block row-major.  R_ij is stored as the d_j x k
 * matrix whose transpose is the paper's k x d_j factor: X_ij = L_ij R_ij^T,
 * X_ji = R_ij L_ij^T.  dense_out[N] (HOST, may be NULL) receives the resolved
 * diagonal representation.  TLR_RECIP_NONE: P = N(N-1) ordered pairs (order as
 * for ranks), X_ij = L_ij R_ij^T for each (L_ij d_i x k, R_ij d_j x k); a
 * low-rank diagonal block is L_ii (d_i x k_ii) at off_diag[i] followed by R_ii
 * (d_i x k_ii), X_ii = L_ii R_ii^T; a dense one is Z_ii with X_ii = Z_ii. */
int tlr_mdd_theta_layout(const tlr_mdd_desc_t* d, int64_t* off_diag, int64_t* off_l,
                         int64_t* off_r, uint8_t* dense_out);

/* Device bytes the library allocates for a handle with this description
 * (data panels + workspace), for admission control. */
int64_t tlr_mdd_workspace_bytes(const tlr_mdd_desc_t* d);

/* Hilbert order of an nx x ny receiver grid, computed on the GPU (eq. 10):
 * perm_dev[a] = natural index (y*nx + x) of the a-th receiver along the curve
 * drawn on the smallest power-of-two square holding the grid.  perm_dev is a
 * DEVICE int32 array [nx*ny].  Bit-exact. */
int tlr_mdd_hilbert_perm(int32_t nx, int32_t ny, int32_t* perm_dev, void* stream);

/* Create a handle: validates *d, computes the receiver order, alpha, and the
 * receiver-major panels Dfrak[a, s] = D[s, perm[a]] / alpha and
 * Ufrak[a, s] = U[s, perm[a]] / alpha (eq. 14; normalisation; each part is one
 * IEEE FP32 division by alpha rounded to FP32), then allocates
 * the workspace.  D, U: complex64 [ns x nr] row-major (the paper's layout),
 * device or host per d->input_memory; they are not referenced after the call
 * returns.  On failure *h is NULL. */
int tlr_mdd_create(tlr_mdd_t** h, const tlr_mdd_desc_t* d, const void* D, const void* U,
                   void* stream);

/* New data for an existing handle (same shapes): recomputes alpha (when
 * desc.alpha == 0) and the panels Dfrak, Ufrak from D, U exactly as
 * tlr_mdd_create does, reusing the handle's workspace and its recorded solve.
 * D, U: complex64 ns x nr row-major, device or host per input_memory
 * (TLR_MEM_*); host inputs are copied on the handle's stream.  Synchronises
 * only when alpha is computed. */
int tlr_mdd_set_data(tlr_mdd_t* h, const void* D, const void* U, int32_t input_memory);

/* Y = X_h Dfrak (receiver-major, Hilbert order), nr x ns complex64 DEVICE.
 * X_h = C(theta) by eq. (6)-(9), (15); theta DEVICE complex64 [n_theta]. */
int tlr_mdd_apply(tlr_mdd_t* h, const void* theta, void* Y);

/* G = V Dfrak^H, nr x nr complex64 DEVICE, for V nr x ns complex64 DEVICE.
 * With V = X_h Dfrak - Ufrak this is W^T, W = D^H (D X - U) (Derivatives
 * paragraph); W' = G + G^T. */
int tlr_mdd_adjoint(tlr_mdd_t* h, const void* V, void* G);

/* f = 0.5 ||D-hat C(theta) - U-hat||_F^2 (eq. 17a) and its factor gradients
 * (eq. 25-27) stacked like theta in grad (DEVICE complex64 [n_theta]); the
 * convention is grad = df/dRe(theta) + i df/dIm(theta).  f: HOST double
 * (the call synchronises the stream), or NULL. */
int tlr_mdd_grad(tlr_mdd_t* h, const void* theta, void* grad, double* f);

/* ADMM with an L-BFGS x-update and exact line search (eq. 18-24), lambda
 * continuation (lam0, decay, stages).  theta_inout: complex64 [n_theta],
 * device or host per opts->theta_memory; it is the start point on entry and
 * the x-iterate on return.  stats: HOST, may be NULL.  Synchronises. */
int tlr_mdd_solve(tlr_mdd_t* h, void* theta_inout, const tlr_mdd_solve_opts_t* opts,
                  tlr_mdd_stats_t* stats);

/* Asynchronous form of tlr_mdd_solve: enqueues the whole solve on the
 * handle's stream and returns.  theta_inout (device or host per
 * opts->theta_memory) must stay valid and untouched until the solve has
 * finished.  The launch sequence is recorded once into a CUDA graph per
 * handle and solver options and replayed afterwards: a handle's first solve
 * with given options runs as plain launches, the second records the graph,
 * later ones replay it (TLR_MDD_LAZY_GRAPH=0 records on the first; set
 * TLR_MDD_GRAPHS=0, or use the NULL stream, for plain launches only).
 * One solve may be pending per handle; handles on different streams run
 * concurrently. */
int tlr_mdd_solve_async(tlr_mdd_t* h, void* theta_inout, const tlr_mdd_solve_opts_t* opts);
/* 1 if the handle's pending solve (if any) has finished, 0 if it is still
 * running, a negative code on error.  Never blocks. */
int tlr_mdd_solve_query(tlr_mdd_t* h);
/* Waits for the pending solve, fills stats (HOST, may be NULL) and returns its
 * status (TLR_ERR_NONFINITE, TLR_ERR_TIMEOUT, ...). */
int tlr_mdd_solve_wait(tlr_mdd_t* h, tlr_mdd_stats_t* stats);

/* Benchmark solver of eq. (4) (least-squares preconditioned MDD) on the
 * handle's data: min_Z 0.5 ||D-hat P Z - U-hat||_F^2 + lambda ||Z||_F^2 with
 * P Z = (Z + Z^T)/2, solved by conjugate gradients on its normal equations
 * P(D-hat^H D-hat P(Z)) + 2 lambda Z = P(D-hat^H U-hat) (real inner product
 * Re tr(A^H B)) from Z = 0, for at most `iters` iterations, stopping once
 * ||residual|| <= tol ||right-hand side||.  The iterates are symmetric, so
 * the result X = P Z = Z is written to X: DEVICE complex64 nr x nr, Hilbert
 * order (like X_h), row-major.  D-hat^H D-hat is formed once; every
 * iteration is one nr x nr x nr complex product in the handle's precision.
 * Work memory (6 nr^2 complex64, plus packed operands on the tensor-core
 * path) is allocated on the handle's stream and released before return; the
 * call synchronises.  lambda < 0 or non-finite, iters < 0, tol < 0, X NULL:
 * TLR_ERR_ARG; a pending solve on the handle: TLR_ERR_STATE.
 * stats (HOST, may be NULL): iterations taken, final ||r|| / ||b||, device
 * time of the whole call. */
typedef struct {
    int32_t iters;
    int32_t status;
    double rel_res;
    double gpu_ms;
} tlr_mdd_bench_stats_t;
int tlr_mdd_benchmark_solve(tlr_mdd_t* h, double lambda, int32_t iters, double tol, void* X,
                            tlr_mdd_bench_stats_t* stats);

/* Tile rank rule of the hyper-parameter selection (Examples section, steps
 * 1-3): the lower tiles of the nr x nr matrix X (DEVICE complex64, row-major;
 * e.g. the benchmark solution in Hilbert order) in b x b tiles, their
 * singular values (one-sided Jacobi SVD per tile on the GPU), v0 = the
 * largest singular value over all tiles, and per tile the numerical rank
 * k = #{sigma >= eps v0} (a tile with none below the threshold is full rank).
 * ranks: HOST int32 [N (N + 1) / 2] in the descriptor's order (N diagonal
 * tiles, then the pairs in the stacking order of tlr_mdd_theta_layout).
 * entries (HOST, may be NULL): complex entries of the factors, sum over pairs
 * of k (d_i + d_j) plus, per diagonal tile, b k, or b^2 where 4 k >= b (the
 * diagonal rule); the entry count ratio is nr^2 / entries.  v0: HOST, may
 * be NULL.  b <= 512 and nr % b == 0 (else TLR_ERR_SHAPE), 0 < eps <= 1.
 * Allocates its work (about nr^2 / 2 complex64) on `stream`; synchronises. */
int tlr_mdd_tile_ranks(const void* X, int64_t nr, int64_t b, double eps, int32_t* ranks, int64_t* entries,
                       double* v0, void* stream);

/* Tile size selection: among the candidate tile sizes (HOST int64 [ncand];
 * those that do not divide nr or exceed 512 are skipped) the one whose rank
 * rule gives the fewest factor entries (the largest entry count ratio); the
 * first candidate wins ties.  best_b, best_entries: HOST. */
int tlr_mdd_choose_tile(const void* X, int64_t nr, const int64_t* candidates, int32_t ncand, double eps,
                        int64_t* best_b, int64_t* best_entries, void* stream);

/* Warm start (hyper-parameter selection and initialisation section) for the
 * handle's layout from X (DEVICE complex64 nr x nr, Hilbert order, e.g. the
 * benchmark solution): for each stored tile (i, j) with rank k (reciprocal
 * form: i > j; TLR_RECIP_NONE: every i != j) the truncated SVD
 * X_ij ~ U_k Sigma_k V_k^H gives L = U_k Sigma_k^1/2 and R = conj(V_k)
 * Sigma_k^1/2 (so L R^T = U_k Sigma_k V_k^H); a low-rank diagonal tile gets,
 * in the reciprocal form, the Takagi form Q = conj(V_k) E_k Sigma_k^1/2,
 * E = diag(V^T U)^1/2, whose Q Q^T is the same truncation (the Q Q^T = X_ii
 * initialisation), and L_ii, R_ii as any tile in the general form; a dense
 * diagonal tile gets Z = X_ii.  Equal or unequal tiles.
 * theta: DEVICE complex64 [n_theta].  Needs every tile <= 512.  Allocates its
 * work (2 d_max^2 complex64 per low-rank tile) on the handle's stream;
 * synchronises. */
int tlr_mdd_warm_start(tlr_mdd_t* h, const void* X, void* theta);

/* Failure detection: every barrier wait in the tensor-core contraction
 * kernels is bounded (2 s of the GPU's global timer, or earlier once another
 * CTA of the launch has given up); a wait that runs out records
 * TLR_ERR_TIMEOUT for the host and the kernel returns, leaving the context
 * usable.  This self-test runs that wait on an mbarrier that nothing arrives
 * at, with the limit limit_ns (0 < limit_ns <= 1e10): *status (HOST) receives
 * TLR_ERR_TIMEOUT and *waited_ms (HOST, may be NULL) the time the wait took.
 * Returns TLR_OK when the kernel ran; synchronises the stream. */
int tlr_mdd_wait_selftest(int64_t limit_ns, int32_t* status, double* waited_ms, void* stream);

/* Solver state for checkpoint / resume: z and u of the ADMM split (eq.
 * 22-24, scaled dual), DEVICE complex64 [n_theta] each in theta's stacking
 * order.  get: copies the handle's current z, u out (after a solve on the
 * handle); set: loads them for a following solve with TLR_SOLVE_RESUME.
 * Both run on the handle's stream and synchronise. */
int tlr_mdd_get_state(tlr_mdd_t* h, void* z, void* u);
int tlr_mdd_set_state(tlr_mdd_t* h, const void* z, const void* u);

/* Time <-> frequency stacks (Numerical Examples: the separated wavefields are
 * transformed to the frequency domain and the MDD solved per frequency; the
 * Green's function returns to time-offset gathers by the inverse transform).
 * Traces are trace-major: x_t DEVICE float [ntr][nt] (for data tr = s nr + r,
 * for X tr = a nr + b).  Stacks are frequency-major: X_w DEVICE complex64
 * [nf][ntr], so frequency f is one row-major panel (ns x nr for D and U,
 * nr x nr for X).  time_to_freq: X_w[f][tr] = sum_t x_t[tr][t]
 * exp(-2 pi i (f0 + f) t / nt), the bins f0 .. f0 + nf - 1 of the real DFT
 * (f0 + nf <= nt / 2 + 1).  freq_to_time: the inverse real DFT of the band
 * (bins outside it zero, the imaginary parts of bins 0 and nt/2 ignored), with
 * the factor 1 / nt, so freq_to_time(time_to_freq(x)) = x when the band is the
 * whole spectrum.  Real FFTs by cuFFT over chunks of traces (work memory about
 * 256 MB plus cuFFT's own, allocated and released per call); synchronises.
 * Invalid sizes: TLR_ERR_ARG. */
int tlr_mdd_time_to_freq(const float* x_t, int64_t ntr, int64_t nt, int64_t f0, int64_t nf, void* X_w,
                         void* stream);
int tlr_mdd_freq_to_time(const void* X_w, int64_t ntr, int64_t nt, int64_t f0, int64_t nf, float* x_t,
                         void* stream);
/* alpha = max |D(omega)| over a whole stack (n complex64 values, DEVICE): the
 * normalisation of the hyper-parameter section, to pass as desc.alpha to every
 * frequency of the stack.  alpha: HOST.  Synchronises. */
int tlr_mdd_stack_alpha(const void* D_w, int64_t n, double* alpha, void* stream);

/* X = S X_h S^T in natural receiver order (eq. 11), nr x nr complex64 DEVICE. */
int tlr_mdd_unpermute_dense(tlr_mdd_t* h, const void* theta, void* X);

/* Copies of the handle's receiver order (HOST int32 [nr]), alpha (HOST) and,
 * if Dt / Ut are non-NULL, its panels (DEVICE complex64 [nr x ns]). */
int tlr_mdd_get_data(tlr_mdd_t* h, int32_t* perm_host, double* alpha, void* Dt, void* Ut);

/* The handle's stream (as passed to create, or last set). */
void* tlr_mdd_stream(const tlr_mdd_t* h);

/* Moves the handle to another stream (of the same device): later calls enqueue
 * there; the handle's workspace, data panels and recorded solve stay.  Waits
 * for the work already enqueued on the old stream.  A pending solve:
 * TLR_ERR_STATE.  Used by a server that keeps finished handles for reuse by
 * later requests of the same shape on whichever slot is free. */
int tlr_mdd_set_stream(tlr_mdd_t* h, void* stream);

/* ---- allocation-free dense adjoint ----
 * G = V Dt^H (nr x nr) for receiver-major V and Dt (nr x ns), all complex64
 * DEVICE buffers owned by the caller; FP32 CUDA-core arithmetic, the same
 * kernels as tlr_mdd_adjoint.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- a process that
 * hands all device memory to its own pool allocator (an allocation from this
 * library would fail or fragment that pool), or a latency-critical path on
 * which an allocation call may synchronise the device.  It allocates nothing
 * and needs no handle: its split-K scratch is one fixed device array of
 * TLR_NOALLOC_SCRATCH_BYTES inside the library, held on every GPU that loads
 * the library until the process exits.  Sizes: nr * nr * 8 bytes must fit in
 * TLR_NOALLOC_SCRATCH_BYTES - 256 (nr <= 1448); larger nr returns
 * TLR_ERR_SHAPE before any work is enqueued.  V, Dt, G and the stream must
 * belong to the current device (managed memory is accepted); a pointer on
 * another device, or a host pointer, returns TLR_ERR_ARG.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use this entry point on a device
 * after cudaDeviceReset (the kept address then belongs to a destroyed
 * context).  Every call shares the one array and it keeps the last call's
 * contents (each call overwrites all it reads): calls that overlap on the GPU
 * -- other streams, other host threads -- race on it.  While diagnostics
 * timing is on (tlr_mdd_timing_enable) the launch is timed in the "project"
 * class like tlr_mdd_adjoint.  Synchronises the stream before returning. */
#define TLR_NOALLOC_SCRATCH_BYTES (16u << 20)
int tlr_mdd_adjoint_noalloc(const void* V, const void* Dt, int64_t nr, int64_t ns, void* G, void* stream);

/* ---- diagnostics (process-wide, not part of the method) ----
 * While enabled, every contraction kernel launch is bracketed by CUDA events
 * on the stream it is launched on; tlr_mdd_timing_read() waits for those
 * events and returns, per class, the summed device time (ms), the algorithmic
 * flops (8 real flops per complex multiply-add) and the launch count.
 * Classes: 0 compress (T = F^T Dfrak, V = F^H Rf), 1 expand (Y = F T~ + P Z
 * Dfrak and the line-search products), 2 project (gradient split-K partials
 * and the dense adjoint).  tlr_mdd_launch_count() is the number of kernels
 * this library has launched since load (all classes and helpers). */
#define TLR_NCLASS 3
void tlr_mdd_timing_enable(int on);
void tlr_mdd_timing_reset(void);
int tlr_mdd_timing_read(double* ms, double* flops, int64_t* launches, int nclass);
int64_t tlr_mdd_launch_count(void);

/* ---- batched solve (serving; the paper solves frequencies one by one) ----
 * A batch runs the solves of n handles (1 <= n <= 64, tensor-core precision
 * with packed operands, one precision for all, any sizes) in lockstep: every
 * member's own kernels run on a stream of the batch's, and each contraction
 * of an L-BFGS step (compress, expand, projection) is ONE launch over the
 * output tiles of every member, so requests of different sizes share the
 * GPU's waves.  Each member's result is bit for bit its result alone (the
 * same K chunks reach the same accumulators; every reduction has a fixed
 * order).  create: validates, creates the batch's streams and events and its
 * merged launch tables (device memory from the workspace pool), synchronises
 * `stream`.  solve_async: thetas[m] (device or host per opts->theta_memory,
 * n_theta of member m) is member m's start point and receives its solution;
 * the same options for every member; enqueued on `stream` (plain launches,
 * no graph); thetas must stay valid until the wait.  query: 1 done, 0
 * running.  wait: stats (HOST array [n], may be NULL) as for a single solve,
 * gpu_ms the whole batch's device time; returns TLR_ERR_TIMEOUT if a merged
 * contraction timed out, TLR_ERR_NONFINITE if a member met a non-finite
 * value.  A member must not be used otherwise while a batched solve is
 * pending; destroy does not destroy the members. */
typedef struct tlr_mdd_batch_s tlr_mdd_batch_t;
int tlr_mdd_batch_create(tlr_mdd_batch_t** b, tlr_mdd_t* const* hs, int32_t n, void* stream);
int tlr_mdd_batch_solve_async(tlr_mdd_batch_t* b, void* const* thetas, const tlr_mdd_solve_opts_t* opts);
int tlr_mdd_batch_query(tlr_mdd_batch_t* b);
int tlr_mdd_batch_wait(tlr_mdd_batch_t* b, tlr_mdd_stats_t* stats);
int tlr_mdd_batch_destroy(tlr_mdd_batch_t* b);

/* Workspace pool (the paper has no counterpart).  Every handle's device
 * workspace comes from one stream-ordered memory pool per device owned by the
 * library, which keeps the memory of destroyed handles reserved for the next
 * handle (creating and destroying handles per frequency or per request maps
 * no fresh device memory).  tlr_mdd_trim_pool releases the current device's
 * reserve down to keep_bytes (memory of live handles is never released) and
 * writes the bytes still reserved to *reserved (HOST, may be NULL).  Call it
 * once the device's memory is wanted elsewhere.  keep_bytes < 0: TLR_ERR_ARG. */
int tlr_mdd_trim_pool(int64_t keep_bytes, int64_t* reserved);

/* Launch shape of the memory-bound passes (the paper has no counterpart).
 * The fused update-and-pack kernels of the tensor-core path (the step of T
 * with its packings, the residual step with its packings) are launched at
 * the device's greatest stream priority, so that where solves on several
 * streams share the GPU their CTAs run beside other streams' contraction
 * CTAs.  tlr_mdd_set_pass_ctas caps the CTAs of one such launch (each walks
 * tiles until all are done; 0: one CTA per tile, the initial value unless the
 * environment variable TLR_MDD_PASS_CTAS gives another), process-wide, for
 * launches made and graphs recorded after the call; the previous cap goes to
 * *previous (HOST, may be NULL).  Results do not depend on the cap (every
 * tile's arithmetic and its partial sums are the same).  ctas < 0:
 * TLR_ERR_ARG. */
int tlr_mdd_set_pass_ctas(int64_t ctas, int64_t* previous);

const char* tlr_mdd_last_error(const tlr_mdd_t* h);
int tlr_mdd_destroy(tlr_mdd_t* h);

#ifdef __cplusplus
}
#endif
#endif /* TLR_MDD_H */
