// Internal declarations shared by the translation units of libtlr_mdd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/tlr_mdd.h"

namespace tlr {

typedef float2 cf;  // complex64, interleaved

// number of kernels this library has launched (diagnostics)
extern std::atomic<long long> g_launches;
inline void counted(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Launch priority of the memory-bound passes (operand packs, the fused
// update-and-pack kernels): the device's greatest stream priority, so that
// where solves on several streams share the GPU, their CTAs are dispatched
// ahead of pending contraction CTAs as an SM's resources free up and run
// beside the contraction CTAs already there.  The environment variable
// TLR_MDD_PASS_PRIORITY=0 launches them at their stream's priority.
int pass_priority();

// Cap on the CTAs of a fused update-and-pack launch (0: one CTA per tile).
constexpr long long kPassCtasDefault = 0;
long long pass_cap();
void set_pass_cap(long long ctas);

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pass(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = pass_priority();
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---------------------------------------------------------------------------
// Grouped complex GEMM descriptors (FP32 SIMT and tensor-core paths).
//
// One problem computes C[m, n] (M x N) = sum over terms t of
//   sum_k opA_t[m, k] * opB_t[k, n]
// with, per term,
//   A element (m, k) at A[k * lda + m]  (KM mode) or A[m * lda + k] (MK mode),
//   B element (k, n) at B[row(k) * ldb + n] (KN mode) or B[row(n) * ldb + k]
//   (NK mode), row(r) = g ? g[r] : r  (a row gather),
//   and the imaginary parts of A / B multiplied by sa / sb (+1 or -1: conj).
// ---------------------------------------------------------------------------
struct GTerm {
    const cf* A;
    const cf* B;
    const int* g;
    long long lda, ldb;
    int K;
    float sa, sb;
};

constexpr int kMaxTerms = 3;

struct GProb {
    GTerm t[kMaxTerms];
    int nt;
    int M, N;
    cf* C;          // output (or partial buffer base for split-K)
    const cf* S;    // subtrahend for EPI_SUB (same indexing as C)
    long long ldc;
};

// EPI_PACKNK (packed tensor-core path only): row m of the product is written in
// the packed BF16-plane format as row rowptr[m] of an NK-packed B operand
// (16 columns = one 16-deep chunk of that operand), not as FP32.
enum Epi { EPI_STORE = 0, EPI_SUB = 1, EPI_ACCUM = 2, EPI_PARTIAL = 3, EPI_PACKNK = 4 };
enum AMode { A_KM = 0, A_MK = 1 };
enum BMode { B_KN = 0, B_NK = 1 };

// ---------------------------------------------------------------------------
// Packed-operand tensor-core path (k_gemm_tcp.cu).
// Packed tile formats (one tile = 128 rows x 16 k = 16 KB in both):
//   kFmtBF16X3: four BF16 planes (Re hi, Re lo, Im hi, Im lo), x = hi + lo;
//   kFmtTF32:   two planes (Re, Im) of FP32 words rounded to TF32 (RN, ties away).
constexpr int kFmtBF16X3 = 0, kFmtTF32 = 1;
inline int pack_fmt(int precision) { return precision == TLR_PREC_TF32 ? kFmtTF32 : kFmtBF16X3; }
inline bool tensor_core(int precision) { return precision == TLR_PREC_BF16X3 || precision == TLR_PREC_TF32; }
// One pack job writes one operand in a packed tile format; element
// (r, k) of the logical operand is src[row(r) * ld + k] when kcontig, else
// src[krow(k) * ld + r]; row(r) = g_row ? g_row[r] : r, krow likewise with g_k;
// the imaginary part is multiplied by sgn.
struct PackJob {
    const cf* src;
    long long ld;
    const int* g_row;
    const int* g_k;
    int kcontig;
    float sgn;
    int R, K, TR;
    void* dst;
    int fmt;   // kFmt*
};
// row-tile heights of packed A (M) and B (N) operands: the GEMM tile's M and N
constexpr int kPackTRA = 128, kPackTRB = 128;
// rows per CTA of the fused update-and-pack kernels (tpack, rstep): 16 rows x
// 128 columns keep their shared memory at 16.5 KB, so one of their CTAs fits
// beside the two GEMM CTAs an SM holds (2 x 97 KB) and they overlap
// contractions of other streams; the tiles of rstep need 16 | d_i for every tile
constexpr int kFuseRows = 16;
struct PTerm {
    const void* A;   // packed A of this problem (TR = kPackTRA), all row blocks
    const void* B;   // packed B of this problem (TR = kPackTRB)
    int K;
};
struct PProb {
    PTerm t[kMaxTerms];
    int nt;
    int M, N;
    cf* C;
    const cf* S;
    long long ldc;
    char* const* rowptr;   // EPI_PACKNK: per output row, its first 16-byte group in the packed operand
};

// One problem-and-split slice of a launch whose problems have their own split
// (the persistent kernel's z index through a map): K chunk `chunk` of
// `kchunk` (0: the whole K), split-K partial at element offset part_off of C.
struct ZItem {
    int prob, chunk, kchunk, pad;
    long long part_off;
};
struct TPackTile;
struct GemmLaunch {
    GProb* d_probs = nullptr;   // device copy
    int nprob = 0;
    int maxM = 0, maxN = 0, maxK = 0;
    int nsplit = 1;
    int kchunk = 0;             // per-split K range (multiple of the K tile)
    long long part_stride = 0;  // elements between split-K partial slabs
    int amode = 0, bmode = 0, epi = 0;
    double flops = 0.0;         // algorithmic flops of one launch (8 per complex MAC)
    int cls = 0;                // diagnostics class (0 compress, 1 expand, 2 project)
    int prec = 0;               // TLR_PREC_FP32 (SIMT), TLR_PREC_BF16X3 or TLR_PREC_TF32 (tcgen05)
    bool persistent = false;    // packed path: the persistent, double-buffered kernel
    const ZItem* d_zmap = nullptr;   // persistent only: per-slice problem, split and partial offset
    int nz = 0;                      // slices in d_zmap (replaces nprob x nsplit)
    int* err = nullptr;         // device error word (tensor-core path: bounded-wait timeouts)
    // packed tensor-core path: problems on packed operands and the packs to run first
    PProb* d_pprobs = nullptr;
    PackJob* d_jobs = nullptr;
    int njobs = 0;
    long long max_items = 0;
    // gathered KN packs of a product matrix (rows of gpack_src, ns columns)
    // written by tpack's packing phase (no update) before the other packs
    const TPackTile* d_gpack = nullptr;
    int n_gpack = 0;
    cf* gpack_src = nullptr;
    int gpack_ns = 0;
};
// One row tile of the fused factor-product update (tpack): rows k0 .. k0+nk-1 (nk <= kFuseRows)
// of block i's gathered products T~_i (T~_i[k] = T[g[k]]), with the packed
// destinations of that block: T~_i as a B operand with rows = ns and k = the
// factor index (KN), and conj(T~_i) as a B operand with rows = the factor
// index and k = ns (NK).
struct TPackTile {
    const int* g;   // block i's gather, indexed by k (0 .. K_i - 1)
    int k0, nk, Ki;
    void* kn;       // packed T~_i (KN), base of block i's buffer
    void* nk_dst;   // packed conj(T~_i) (NK), base of block i's buffer
    int fmt;        // kFmt*
};
// T[r] += alpha T_p[r] (FP32 fmaf, alpha read on the device; alpha == nullptr
// or *alpha == 0: no update) for every row reached through the tiles (each
// row of T exactly once), then both packed forms of the updated rows (the NK
// form only for tiles with nk_dst != nullptr).
cudaError_t tpack(const TPackTile* d_tiles, int ntiles, cf* T, const cf* Tp, const double* alpha, int ns,
                  cudaStream_t st);
// Fused residual step of the tensor-core path: R += a A1 + a^2 A2 (FP32, the
// same arithmetic as the plain residual step; a read on the device), with R
// read from and written back to its packed forms only (the FP32 R of the
// forward product is read when alpha == nullptr: packing, no update); the
// per-tile partial of ||R||^2 (16 x 128 tiles; two-sum per thread, FP64
// across the CTA) into part[tile] when part != nullptr, whatever the grid,
// and R in both packed forms: block i's rows
// as an A operand with k = ns (MK, mk[i]) and as a B operand with rows = ns
// and k = the receiver (KN, kn[i]).  Blocks of
// b rows (roff == nullptr) or block i = rows roff[i] .. roff[i+1]-1 (DEVICE
// [nblk + 1]); every block size a multiple of kFuseRows.  rstep_ctas gives the
// number of tiles (and partials).
long long rstep_ctas(int nr, int ns);
// The six line-search inner products with R read from its KN packing (kn[i],
// as rstep writes it), over rstep's tiles: part[blk * 6 + k], kRedBlocks
// partials (a fixed grid, so the sums are reproducible).
cudaError_t dots6_packed(char* const* kn, const cf* A1, const cf* A2, int nr, int ns, int b, double* part,
                         cudaStream_t st, const long long* roff, int nblk, int fmt);
cudaError_t rstep(cf* R, const cf* A1, const cf* A2, const double* alpha, int nr, int ns, int b, char* const* kn,
                  char* const* mk, double* part, cudaStream_t st, const long long* roff, int nblk, int fmt);
// Benchmark solver of eq. (4) (k_cg.cu): the symmetrising pass
// out = P(y) + s2 p (with partials of <p, out> when part != nullptr; p may be
// nullptr: out = P(y)), the start (x = 0, r = p = b with b in r on entry),
// and the CG tail of one iteration (alpha, step, beta, direction) on device
// scalars sc[8] (slots in k_cg.cu: rr, <p,Ap>, alpha, beta, ||b||^2, done,
// iterations).  cg_partials(n) = partial slots needed.
int cg_partials(int n);
cudaError_t cg_sym(const cf* y, const cf* p, float s2, cf* out, int n, double* part, cudaStream_t st);
cudaError_t cg_start(cf* x, cf* r, cf* p, int n, double* part, double* sc, cudaStream_t st);
cudaError_t cg_iteration_tail(cf* x, cf* r, cf* p, const cf* Ap, int n, double tol, double* part, double* sc,
                              cudaStream_t st);
// Tile SVDs (k_svd.cu) for the rank rule and the warm start.  tile_svd: one
// one-sided Jacobi SVD per listed tile (rows r0 .. r0+m-1, columns c0 ..
// c0+n-1 of the row-major X; trans: the SVD of its transpose, for n > m),
// m, n <= bmax <= 512, work = tile_svd_work_bytes(ntiles, bmax, vec);
// sig[t bmax ..] the decreasing singular values (as many as the columns the
// sweeps work on) then -1, order[t bmax + q] the column of the q-th (may be
// nullptr), sweeps[t] sweeps used (may be nullptr).  rank_rule (equal tiles,
// bmax = b): v0 = max sigma, ranks[t] = #{sigma >= eps v0}.  warm_fill: the
// warm-start factors (kinds: 0 low-rank tile L, R; 1 low-rank diagonal Q by
// the Takagi form; 2 dense Z = tile) written into theta at the given offsets.
struct SvdTile {
    int r0, c0, m, n, trans;
};
struct WarmTile {
    int r0, c0, m, n;       // the tile of X: rows r0.., columns c0.., m x n
    int kind, k;
    long long offL, offR;   // theta offsets (R unused for kinds 1 and 2)
    int svd;                // index of the tile's SVD (-1 for dense)
    int trans;              // that SVD ran on the transpose
};
size_t tile_svd_work_bytes(int ntiles, int b, bool vec);
cudaError_t tile_svd(const cf* X, long long ldx, const SvdTile* tiles, int ntiles, int bmax, cf* work, bool vec,
                     int max_sweeps, float tol, float* sig, int* order, int* sweeps, cudaStream_t st);
cudaError_t rank_rule(const float* sig, int ntiles, int b, double eps, int* ranks, double* v0, cudaStream_t st);
cudaError_t warm_fill(const cf* X, long long ldx, const WarmTile* wt, int nt, int bmax, const cf* work,
                      const float* sig, const int* order, cf* theta, cudaStream_t st);
// Time <-> frequency stack (fourier.cu): forward: x_t_in [ntr][nt] real ->
// X_out [nf][ntr], the bins f0 .. f0 + nf - 1 of the unnormalised real DFT;
// inverse: X_in [nf][ntr] (band, zero elsewhere) -> x_t_out [ntr][nt] with
// the 1 / nt factor.  Synchronises (returns a TLR_* code, message in err).
int fft_stack(bool forward, const float* x_t_in, const cf* X_in, long long ntr, long long nt, long long f0,
              long long nf, cf* X_out, float* x_t_out, cudaStream_t st, std::string& err);
// bytes of one operand (R rows x K) in the packed tile format with TR-row tiles;
// pack_operands: max_items = (largest padded row count << 32) | largest k-group count
long long packed_bytes(long long R, long long K, int TR);
cudaError_t pack_operands(const PackJob* d_jobs, int njobs, long long max_items, cudaStream_t st);
cudaError_t gemm_tcp_prepare();
// Bounded-wait self-test: one thread waits, with the contraction kernels'
// wait, on an mbarrier that nothing arrives at; after limit_ns the wait gives
// up and *status (DEVICE, zero on entry) becomes TLR_ERR_TIMEOUT, *waited_ns
// (DEVICE) the time it waited.
cudaError_t wait_selftest(int* status, unsigned long long limit_ns, unsigned long long* waited_ns, cudaStream_t st);
cudaError_t gemm_tcp(const GemmLaunch& L, cudaStream_t st);

// SIMT path (k_gemm_simt.cu)
cudaError_t gemm_simt(const GemmLaunch& L, cudaStream_t st);
// tcgen05 path (k_gemm_tc.cu): BF16x3 split, 3M complex, FP32 accumulation in TMEM
cudaError_t gemm_tc(const GemmLaunch& L, cudaStream_t st);
// one-time kernel attributes (shared-memory size), outside any stream capture
cudaError_t gemm_tc_prepare();
inline cudaError_t gemm_any(const GemmLaunch& L, cudaStream_t st) {
    if (!tensor_core(L.prec)) return gemm_simt(L, st);
    if (!L.d_pprobs) return gemm_tc(L, st);
    cudaError_t e = cudaSuccess;
    if (L.n_gpack) e = tpack(L.d_gpack, L.n_gpack, L.gpack_src, nullptr, nullptr, L.gpack_ns, st);
    if (e == cudaSuccess) e = pack_operands(L.d_jobs, L.njobs, L.max_items, st);
    return e == cudaSuccess ? gemm_tcp(L, st) : e;
}
// One grouped contraction through gemm_any, bracketed by CUDA events on its
// stream while the diagnostics timing (tlr_mdd_timing_enable) is on (api.cu).
cudaError_t run_gemm(const GemmLaunch& L, cudaStream_t st);

// ---------------------------------------------------------------------------
// data kernels (k_data.cu)
// ---------------------------------------------------------------------------
cudaError_t hilbert_perm(int nx, int ny, int32_t* perm, int32_t* scratch_keys, cudaStream_t st);
// max |D|^2 over n complex entries -> *out (device double), deterministic
cudaError_t max_abs2(const cf* D, long long n, double* partial, int nblk, double* out, cudaStream_t st);
// Dt[a, s] = D[s, perm[a]] / alpha for D ns x nr row-major; alpha read from device
cudaError_t permute_normalise(const cf* D, long long ns, long long nr, const int32_t* perm,
                              const double* alpha_dev, cf* Dt, cudaStream_t st);
// Per-tile description for dense assembly: tiles 0..N-1 are the diagonal
// (off_l = theta offset of Q_ii or Z_ii, off_r = off_l for Q), then the
// sub-diagonal pairs in stacking order (off_l = L_ij, off_r = R_ij).
struct AsmTile {
    long long off_l, off_r;
    int k;
    int dense;
};
// roff: nullptr for N tiles of size b, else DEVICE [N + 1] block row offsets
// (roff[N] = nr) of a non-uniform partition
cudaError_t assemble_dense(const cf* theta, long long nr, long long b, int N, const AsmTile* tiles, cf* Xh,
                           cudaStream_t st, int general = 0, const long long* roff = nullptr);
// X[perm[a], perm[c]] = Xh[a, c]
cudaError_t unpermute_dense(const cf* Xh, long long nr, const int32_t* perm, cf* X, cudaStream_t st);

// ---------------------------------------------------------------------------
// theta-space and reduction kernels (k_vec.cu)
// ---------------------------------------------------------------------------
constexpr int kRedBlocks = 608;   // 4 x 152 SMs: fixed grid -> fixed summation order
constexpr int kRedThreads = 256;

// theta (paper stacking) <-> panel vector (block-major factor panels + dense tiles)
struct PanelMap {
    const long long* colsrc;   // [Ktot] theta offset of row 0 of this panel column
    const int* colstride;      // [Ktot] row stride in theta (rank of the factor)
    const long long* colpan;   // [Ktot] panel offset of row 0 of this column
    const int* panstride;      // [Ktot] row stride in the panel (K of its block)
    const int* colrows;        // [Ktot] rows of this column's block (its tile size d_i)
    const long long* zsrc;     // [ndense] theta offset of each dense tile
    const long long* zoff;     // [ndense] offset of each dense tile after zbase
    const int* zdim;           // [ndense] size d_i of each dense tile
    long long Ktot, b, ndense, zbase;  // b = the largest tile size; zbase = low-rank panel entries
};
cudaError_t theta_to_panel(const PanelMap& m, const cf* theta, cf* pan, cudaStream_t st);
cudaError_t panel_to_theta(const PanelMap& m, const cf* pan, cf* theta, cudaStream_t st);
// Dense tiles of a panel vector: ndense tiles of size b stored one after the
// other (zoff == nullptr), or tile t of size zdim[t] at zoff[t] (DEVICE arrays;
// b is then the largest size).
// Zs = (Z + Z^T)/2 for every dense tile (general != 0: Zs = Z^T, the general
// form's dense tiles); Zs has the same tile offsets.
cudaError_t sym_dense(const cf* pan, long long zbase, long long ndense, long long b, cf* Zs, cudaStream_t st,
                      int general = 0, const long long* zoff = nullptr, const int* zdim = nullptr);
// grad[e] = sum_c part[c * stride + e] (LR part), dense tiles symmetrised: (G + G^T)/2
// (general != 0: G^T, the general form's dense tiles)
cudaError_t reduce_grad(const cf* part, int nsplit, long long stride, long long nlr, long long ndense,
                        long long b, cf* grad, cudaStream_t st, int general = 0, const long long* zoff = nullptr,
                        const int* zdim = nullptr);

// partial FP64 real dot sums over float arrays (2 per complex) -> part[kRedBlocks]
cudaError_t dot_part(const float* a, const float* b, long long n2, double* part, cudaStream_t st);
// out[k] = sum_{blk} part[blk * stride + k], k < cnt, one block, fixed order
cudaError_t finalize(const double* part, int nblk, int stride, int cnt, double* out, cudaStream_t st);
// six partials of the line-search inner products over Rf, A1, A2 (n complex)
cudaError_t dots6_part(const cf* R, const cf* A1, const cf* A2, long long n, double* part, cudaStream_t st);
// elementwise step: R += a A1 + a^2 A2 (n complex); alpha read from device
cudaError_t step_residual(cf* R, const cf* A1, const cf* A2, long long n, const double* alpha, cudaStream_t st);
// x += a * y over n2 floats, a = alpha[0] (device)
cudaError_t axpy_dev(float* x, const float* y, long long n2, const double* alpha, cudaStream_t st);


}  // namespace tlr
