// theta-space and reduction kernels: the layout maps between the stacked
// unknown (Z-bar, L-bar, R-bar) and the block panels, the gradient split-K
// reduction with the dense-tile symmetrisation (eq. 26), FP64 inner products,
// the exact line search on the quartic phi(alpha), and the L-BFGS direction
// (compact form) / ADMM updates (eq. 19-24) with every scalar kept on the device.
//
// All reductions run on a fixed grid (kRedBlocks x kRedThreads) and sum their
// per-block partials in a fixed order, so results are bitwise reproducible.
#include "internal.h"
#include "solver_dev.h"
#include "reduce.h"

namespace tlr {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// Sum of part[i * stride + k] over i < nblk by warp 0 in a fixed order; every
// block that calls this obtains the same value.  Result broadcast via shared.
__device__ __forceinline__ double sum_partials(const double* part, int nblk, int stride, int k, double* sh1) {
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nblk; i += 32) v += part[(long long)i * stride + k];
        v = warp_sum(v);
        if (threadIdx.x == 0) sh1[0] = v;
    }
    __syncthreads();
    const double r = sh1[0];
    __syncthreads();
    return r;
}

#define GRID_STRIDE(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// layout maps
// ---------------------------------------------------------------------------
__global__ void k_theta_to_panel(PanelMap m, const cf* __restrict__ th, cf* __restrict__ pan) {
    const long long nlr = m.Ktot * m.b;
    GRID_STRIDE(e, nlr) {
        const long long g = e % m.Ktot, a = e / m.Ktot;
        if (a < m.colrows[g]) pan[m.colpan[g] + a * m.panstride[g]] = th[m.colsrc[g] + a * m.colstride[g]];
    }
    const long long bb = m.b * m.b;
    GRID_STRIDE(e, m.ndense * bb) {
        const long long t = e / bb, r = (e % bb) / m.b, c = e % m.b, n = m.zdim[t];
        if (r < n && c < n) pan[m.zbase + m.zoff[t] + r * n + c] = th[m.zsrc[t] + r * n + c];
    }
}

__global__ void k_panel_to_theta(PanelMap m, const cf* __restrict__ pan, cf* __restrict__ th) {
    const long long nlr = m.Ktot * m.b;
    GRID_STRIDE(e, nlr) {
        const long long g = e % m.Ktot, a = e / m.Ktot;
        if (a < m.colrows[g]) th[m.colsrc[g] + a * m.colstride[g]] = pan[m.colpan[g] + a * m.panstride[g]];
    }
    const long long bb = m.b * m.b;
    GRID_STRIDE(e, m.ndense * bb) {
        const long long t = e / bb, r = (e % bb) / m.b, c = e % m.b, n = m.zdim[t];
        if (r < n && c < n) th[m.zsrc[t] + r * n + c] = pan[m.zbase + m.zoff[t] + r * n + c];
    }
}

cudaError_t theta_to_panel(const PanelMap& m, const cf* theta, cf* pan, cudaStream_t st) {
    (void)launch_pass(k_theta_to_panel, dim3(1024), dim3(256), st, m, theta, pan);
    counted(1);
    return cudaGetLastError();
}
cudaError_t panel_to_theta(const PanelMap& m, const cf* pan, cf* theta, cudaStream_t st) {
    (void)launch_pass(k_panel_to_theta, dim3(1024), dim3(256), st, m, pan, theta);
    counted(1);
    return cudaGetLastError();
}

// Dense tile t of a panel-ordered region: (offset, size) from the per-tile
// tables, or the t-th of equal tiles of size b.
__device__ __forceinline__ bool dense_tile(long long e, long long b, const long long* zoff, const int* zdim,
                                           long long& base, long long& n, long long& r, long long& c) {
    const long long bb = b * b, t = e / bb;
    r = (e % bb) / b;
    c = e % b;
    if (!zoff) {
        base = t * bb;
        n = b;
        return true;
    }
    base = zoff[t];
    n = zdim[t];
    return r < n && c < n;
}

// Zs = (Z + Z^T)/2 (reciprocal form: the symmetrisation preconditioner P of
// eq. 7, X_ii = P Z_ii) or Z^T (general form: row block i of Y = X^T Dfrak
// takes X_ii^T)
__global__ void k_sym_dense(const cf* __restrict__ pan, long long zbase, long long ndense, long long b,
                            cf* __restrict__ Zs, int general, const long long* __restrict__ zoff,
                            const int* __restrict__ zdim) {
    GRID_STRIDE(e, ndense * b * b) {
        long long base, n, r, c;
        if (!dense_tile(e, b, zoff, zdim, base, n, r, c)) continue;
        const cf u = pan[zbase + base + r * n + c];
        const cf v = pan[zbase + base + c * n + r];
        Zs[base + r * n + c] = general ? v : make_float2(0.5f * (u.x + v.x), 0.5f * (u.y + v.y));
    }
}

cudaError_t sym_dense(const cf* pan, long long zbase, long long ndense, long long b, cf* Zs, cudaStream_t st,
                      int general, const long long* zoff, const int* zdim) {
    if (ndense == 0) return cudaSuccess;
    (void)launch_pass(k_sym_dense, dim3(512), dim3(256), st, pan, zbase, ndense, b, Zs, general, zoff, zdim);
    counted(1);
    return cudaGetLastError();
}

// grad = sum of split-K partials (FP64, fixed order); dense tiles: (G + G^T)/2
// (reciprocal form) or G^T (general form)
__global__ void k_reduce_grad(const cf* __restrict__ part, int nsplit, long long stride, long long nlr,
                              long long ndense, long long b, cf* __restrict__ grad, int general,
                              const long long* __restrict__ zoff, const int* __restrict__ zdim) {
    GRID_STRIDE(e, nlr) {
        Acc x, y;
        for (int c = 0; c < nsplit; ++c) {
            const cf v = part[c * stride + e];
            x.add(v.x);
            y.add(v.y);
        }
        grad[e] = make_float2((float)x.val(), (float)y.val());
    }
    GRID_STRIDE(e, ndense * b * b) {
        long long base, n, r, q;
        if (!dense_tile(e, b, zoff, zdim, base, n, r, q)) continue;
        const long long e1 = nlr + base + r * n + q, e2 = nlr + base + q * n + r;
        Acc x, y;
        for (int c = 0; c < nsplit; ++c) {
            const cf v = part[c * stride + e2];
            if (!general) {
                const cf u = part[c * stride + e1];
                x.add(u.x);
                y.add(u.y);
            }
            x.add(v.x);
            y.add(v.y);
        }
        const double s = general ? 1.0 : 0.5;
        grad[e1] = make_float2((float)(s * x.val()), (float)(s * y.val()));
    }
}

cudaError_t reduce_grad(const cf* part, int nsplit, long long stride, long long nlr, long long ndense,
                        long long b, cf* grad, cudaStream_t st, int general, const long long* zoff,
                        const int* zdim) {
    (void)launch_pass(k_reduce_grad, dim3(1024), dim3(256), st, part, nsplit, stride, nlr, ndense, b, grad, general,
                      zoff, zdim);
    counted(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 inner products
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads) k_dot_part(const float* __restrict__ a, const float* __restrict__ b,
                                                         long long n2, double* part) {
    __shared__ double sh[32];
    Acc s;
    GRID_STRIDE(i, n2) s.add(a[i] * b[i]);
    const double r = block_sum(s.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

cudaError_t dot_part(const float* a, const float* b, long long n2, double* part, cudaStream_t st) {
    (void)launch_pass(k_dot_part, dim3(kRedBlocks), dim3(kRedThreads), st, a, b, n2, part);
    counted(1);
    return cudaGetLastError();
}

__global__ void k_finalize(const double* part, int nblk, int stride, int cnt, double* out) {
    __shared__ double sh1[1];
    for (int k = 0; k < cnt; ++k) {
        const double v = sum_partials(part, nblk, stride, k, sh1);
        if (threadIdx.x == 0) out[k] = v;
    }
}

cudaError_t finalize(const double* part, int nblk, int stride, int cnt, double* out, cudaStream_t st) {
    (void)launch_pass(k_finalize, dim3(1), dim3(32), st, part, nblk, stride, cnt, out);
    counted(1);
    return cudaGetLastError();
}

// Re<R,R>, Re<R,A1>, Re<R,A2>, Re<A1,A1>, Re<A1,A2>, Re<A2,A2>  -> part[blk*6 + k]
// (two complex values per 16-byte load when n is even; the buffers start
// 256-byte aligned)
__device__ __forceinline__ void dots6_add(Acc* s, float rx, float ry, float ax, float ay, float cx, float cy) {
    s[0].add(fmaf(rx, rx, ry * ry));
    s[1].add(fmaf(rx, ax, ry * ay));
    s[2].add(fmaf(rx, cx, ry * cy));
    s[3].add(fmaf(ax, ax, ay * ay));
    s[4].add(fmaf(ax, cx, ay * cy));
    s[5].add(fmaf(cx, cx, cy * cy));
}

// the six products of one complex element added to t (plain FP32: a group of
// up to four elements is summed like this before one compensated add, so
// the group's rounding is of the order of the products' own)
__device__ __forceinline__ void dots6_group(float* t, float rx, float ry, float ax, float ay, float cx, float cy) {
    t[0] += fmaf(rx, rx, ry * ry);
    t[1] += fmaf(rx, ax, ry * ay);
    t[2] += fmaf(rx, cx, ry * cy);
    t[3] += fmaf(ax, ax, ay * ay);
    t[4] += fmaf(ax, cx, ay * cy);
    t[5] += fmaf(cx, cx, cy * cy);
}

__global__ void __launch_bounds__(kRedThreads) k_dots6(const cf* __restrict__ R, const cf* __restrict__ A1,
                                                      const cf* __restrict__ A2, long long n, double* part) {
    __shared__ double sh[32];
    Acc s[6];
    if ((n & 1) == 0) {
        const float4* R4 = reinterpret_cast<const float4*>(R);
        const float4* A4 = reinterpret_cast<const float4*>(A1);
        const float4* C4 = reinterpret_cast<const float4*>(A2);
        const long long n4 = n >> 1, stride = (long long)gridDim.x * blockDim.x;
        long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        for (; i + stride < n4; i += 2 * stride) {   // two 16-byte loads of each array in flight
            const float4 r = R4[i], a = A4[i], c = C4[i];
            const float4 r2 = R4[i + stride], a2 = A4[i + stride], c2 = C4[i + stride];
            float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            dots6_group(t, r.x, r.y, a.x, a.y, c.x, c.y);
            dots6_group(t, r.z, r.w, a.z, a.w, c.z, c.w);
            dots6_group(t, r2.x, r2.y, a2.x, a2.y, c2.x, c2.y);
            dots6_group(t, r2.z, r2.w, a2.z, a2.w, c2.z, c2.w);
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k].add(t[k]);
        }
        if (i < n4) {
            const float4 r = R4[i], a = A4[i], c = C4[i];
            float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            dots6_group(t, r.x, r.y, a.x, a.y, c.x, c.y);
            dots6_group(t, r.z, r.w, a.z, a.w, c.z, c.w);
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k].add(t[k]);
        }
    } else {
        GRID_STRIDE(i, n) {
            const cf r = R[i], a = A1[i], c = A2[i];
            dots6_add(s, r.x, r.y, a.x, a.y, c.x, c.y);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = block_sum(s[k].val(), sh);
        if (threadIdx.x == 0) part[blockIdx.x * 6 + k] = v;
    }
}

cudaError_t dots6_part(const cf* R, const cf* A1, const cf* A2, long long n, double* part, cudaStream_t st) {
    (void)launch_pass(k_dots6, dim3(kRedBlocks), dim3(kRedThreads), st, R, A1, A2, n, part);
    counted(1);
    return cudaGetLastError();
}

// R += a A1 + a^2 A2 ; partial of ||R_new||^2 -> part[blk]
__global__ void __launch_bounds__(kRedThreads) k_step_residual(cf* __restrict__ R, const cf* __restrict__ A1,
                                                              const cf* __restrict__ A2, long long n,
                                                              const double* __restrict__ alpha, double* part) {
    __shared__ double sh[32];
    const float a = (float)alpha[0];
    const float a2 = (float)(alpha[0] * alpha[0]);
    Acc s;
    GRID_STRIDE(i, n) {
        cf r = R[i];
        if (a != 0.f) {
            const cf u = A1[i], w = A2[i];
            r.x = fmaf(a2, w.x, fmaf(a, u.x, r.x));
            r.y = fmaf(a2, w.y, fmaf(a, u.y, r.y));
            R[i] = r;
        }
        s.add(fmaf(r.x, r.x, r.y * r.y));
    }
    const double t = block_sum(s.val(), sh);
    if (part && threadIdx.x == 0) part[blockIdx.x] = t;
}

cudaError_t step_residual(cf* R, const cf* A1, const cf* A2, long long n, const double* alpha, cudaStream_t st) {
    (void)launch_pass(k_step_residual, dim3(kRedBlocks), dim3(kRedThreads), st, R, A1, A2, n, alpha, nullptr);
    counted(1);
    return cudaGetLastError();
}

__global__ void k_axpy_dev(float* __restrict__ x, const float* __restrict__ y, long long n2,
                           const double* __restrict__ alpha) {
    const float a = (float)alpha[0];
    if (a == 0.f) return;
    GRID_STRIDE(i, n2) x[i] = fmaf(a, y[i], x[i]);
}

cudaError_t axpy_dev(float* x, const float* y, long long n2, const double* alpha, cudaStream_t st) {
    (void)launch_pass(k_axpy_dev, dim3(1024), dim3(256), st, x, y, n2, alpha);
    counted(1);
    return cudaGetLastError();
}

// ===========================================================================
// Solver kernels (L-BFGS two-loop recursion, exact line search, ADMM).
// ===========================================================================

// f = 0.5 ||R||^2 from a fresh norm pass: part[blk] -> sc[SC_F]
__global__ void __launch_bounds__(kRedThreads) k_norm_part(const cf* __restrict__ R, long long n, double* part) {
    __shared__ double sh[32];
    Acc s;
    GRID_STRIDE(i, n) {
        const cf r = R[i];
        s.add(fmaf(r.x, r.x, r.y * r.y));
    }
    const double t = block_sum(s.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// g = gf + rho (x - v); history cleared (start of an x-update)
__global__ void k_xupdate_start(SolverDev S, double rho) {
    const float r = (float)rho;
    GRID_STRIDE(i, S.n2) S.g[i] = S.gf[i] + r * (S.x[i] - S.v[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) S.ints[SI_CNT] = 0;
}

__device__ __forceinline__ int ring_idx(const SolverDev& S, int j) {
    // j-th newest pair (0 = newest)
    const int R = S.ring;
    return ((S.ints[SI_NEWEST] - j) % R + R) % R;
}

// L-BFGS direction d = -H g in the compact form of the inverse BFGS update
// (Byrd, Nocedal and Schnabel 1994): with the k stored pairs ordered oldest
// first, S = [s_1 .. s_k], Y = [y_1 .. y_k], R = triu(S^T Y), D = diag(S^T Y),
// H0 = gamma I and gamma = <s,y>/<y,y> of the newest pair,
//   H g = gamma g + S a - gamma Y u,  u = R^-1 S^T g,
//   a = R^-T ((D + gamma Y^T Y) u - gamma Y^T g).
// This is the matrix the two-loop recursion applies, evaluated in three
// steps: the inner products (passes over groups of pairs; they also fill the
// newest pair's row and column of S^T Y and Y^T Y, which are kept by slot),
// the small FP64 triangular solves in one block, and one combination pass.

// partials per block: for pair j of the group, <s_j,g>, <y_j,g>, <s_j,y_n>,
// <s_n,y_j>, <y_j,y_n> (n = the newest pair).  Per-thread sums are plain FP32
// multiply-adds (a thread sums n2 / (kRedBlocks kRedThreads) terms, a few
// dozen at these sizes), combined in FP64 across threads and blocks: these
// products only set the direction's coefficients, whose rounding the exact
// line search and the descent test absorb.
// 128 threads of <= 128 registers: a CTA fits beside the two GEMM CTAs of an SM
constexpr int kLbThreads = 128;
__global__ void __launch_bounds__(kLbThreads, 4) k_lb_dots(SolverDev S, int j0) {
    __shared__ double sh[32];
    const int cnt = S.ints[SI_CNT];
    if (j0 >= cnt) return;
    const int jc = min(kLbGroup, cnt - j0);
    const float* sp[kLbGroup];
    const float* yp[kLbGroup];
#pragma unroll
    for (int jj = 0; jj < kLbGroup; ++jj) {
        const int idx = ring_idx(S, jj < jc ? j0 + jj : j0);
        sp[jj] = S.sh + (long long)idx * S.n2;
        yp[jj] = S.yh + (long long)idx * S.n2;
    }
    const int nw = ring_idx(S, 0);
    const float* sn = S.sh + (long long)nw * S.n2;
    const float* yn = S.yh + (long long)nw * S.n2;
    float acc[kLbGroup][5];
#pragma unroll
    for (int jj = 0; jj < kLbGroup; ++jj)
#pragma unroll
        for (int t = 0; t < 5; ++t) acc[jj][t] = 0.f;
    float gg = 0.f;   // <g, g> for the descent test (first group only)
    GRID_STRIDE(i, S.n2) {
        const float gi = S.g[i], sni = sn[i], yni = yn[i];
        gg = fmaf(gi, gi, gg);
#pragma unroll
        for (int jj = 0; jj < kLbGroup; ++jj) {
            if (jj < jc) {
                const float s = sp[jj][i], y = yp[jj][i];
                acc[jj][0] = fmaf(s, gi, acc[jj][0]);
                acc[jj][1] = fmaf(y, gi, acc[jj][1]);
                acc[jj][2] = fmaf(s, yni, acc[jj][2]);
                acc[jj][3] = fmaf(sni, y, acc[jj][3]);
                acc[jj][4] = fmaf(y, yni, acc[jj][4]);
            }
        }
    }
    double* out = S.lbpart + (long long)(j0 / kLbGroup) * kRedBlocks * (5 * kLbGroup) +
                  (long long)blockIdx.x * (5 * kLbGroup);
#pragma unroll
    for (int jj = 0; jj < kLbGroup; ++jj) {
        if (jj >= jc) break;
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const double r = block_sum((double)acc[jj][t], sh);
            if (threadIdx.x == 0) out[jj * 5 + t] = r;
        }
    }
    if (j0 == 0) {
        const double r = block_sum((double)gg, sh);
        if (threadIdx.x == 0) S.lbpart[kLbGGOff + blockIdx.x] = r;
    }
}

// One block: finalise the partials (warp per value, fixed order), update the
// newest pair's row / column of S^T Y and Y^T Y, then (thread 0) the
// triangular solves; coefficients to acoef, gamma to sc[SC_GAMMA].
// single-block finalisers on the solve's critical path: 256 threads sum the
// partial slabs (fixed order per thread, then the block tree); at 256 threads
// (56 registers at most) a finaliser fits on an SM beside two contraction
// CTAs, so with several solves in flight it never waits for a free SM
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads) k_lb_solve(SolverDev S) {
    __shared__ double val[32 * 5 + 1];
    __shared__ double Rm[32 * 33];
    __shared__ double Ym[32 * 33];
    __shared__ double p[32], q[32], u[32], t[32];
    const int cnt = S.ints[SI_CNT];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int nval = cnt > 0 ? 5 * cnt + 1 : 0;   // the last value is <g, g>
    for (int v = w; v < nval; v += kFinThreads / 32) {
        const double* base;
        long long stride;
        if (v == 5 * cnt) {
            base = S.lbpart + kLbGGOff;
            stride = 1;
        } else {
            const int j = v / 5, kind = v % 5;
            base = S.lbpart + (long long)(j / kLbGroup) * kRedBlocks * (5 * kLbGroup) + (j % kLbGroup) * 5 + kind;
            stride = 5 * kLbGroup;
        }
        double a = 0.0;
        for (int b = l; b < kRedBlocks; b += 32) a += base[(long long)b * stride];
        a = warp_sum(a);
        if (l == 0) val[v] = a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    S.ints[SI_RFLAG] = 0;
    if (cnt == 0) {
        // d = -g, a descent direction unless g = 0 (which the line search meets)
        S.sc[SC_GAMMA] = 1.0;
        return;
    }
    const int R = S.ring;
    const int nw = ring_idx(S, 0);
    for (int j = 0; j < cnt; ++j) {
        const int a = ring_idx(S, j);
        S.SYm[a * R + nw] = val[j * 5 + 2];
        S.SYm[nw * R + a] = val[j * 5 + 3];
        S.YYm[a * R + nw] = val[j * 5 + 4];
        S.YYm[nw * R + a] = val[j * 5 + 4];
    }
    // oldest first: position i holds the (cnt - 1 - i)-th newest pair
    const int k = cnt;
    for (int i = 0; i < k; ++i) {
        const int si = ring_idx(S, k - 1 - i);
        p[i] = val[(k - 1 - i) * 5 + 0];
        q[i] = val[(k - 1 - i) * 5 + 1];
        for (int j = 0; j < k; ++j) {
            const int sj = ring_idx(S, k - 1 - j);
            Rm[i * 33 + j] = S.SYm[si * R + sj];
            Ym[i * 33 + j] = S.YYm[si * R + sj];
        }
    }
    const double gamma = Rm[(k - 1) * 33 + (k - 1)] / Ym[(k - 1) * 33 + (k - 1)];
    // u = R^-1 p (R upper triangular)
    for (int i = k - 1; i >= 0; --i) {
        double a = p[i];
        for (int j = i + 1; j < k; ++j) a -= Rm[i * 33 + j] * u[j];
        u[i] = a / Rm[i * 33 + i];
    }
    // t = D u + gamma Y^T Y u - gamma q
    for (int i = 0; i < k; ++i) {
        double a = Rm[i * 33 + i] * u[i] - gamma * q[i];
        for (int j = 0; j < k; ++j) a += gamma * Ym[i * 33 + j] * u[j];
        t[i] = a;
    }
    // a = R^-T t (R^T lower triangular), written over t
    for (int i = 0; i < k; ++i) {
        double a = t[i];
        for (int j = 0; j < i; ++j) a -= Rm[j * 33 + i] * t[j];
        t[i] = a / Rm[i * 33 + i];
    }
    // descent test: <g, d> = -(gamma <g,g> + sum_i a_i <s_i,g> - gamma sum_i u_i <y_i,g>)
    double gd = gamma * val[5 * k];
    for (int i = 0; i < k; ++i) gd += t[i] * p[i] - gamma * u[i] * q[i];
    gd = -gd;
    if (!(gd < 0.0)) {
        // not a descent direction: clear the memory and take d = -g in this
        // same iteration (the restart of L-BFGS)
        S.ints[SI_CNT] = 0;
        S.ints[SI_RESTARTS] += 1;
        S.ints[SI_RFLAG] = 1;
        S.sc[SC_GAMMA] = 1.0;
        return;
    }
    for (int i = 0; i < k; ++i) {
        const int j = k - 1 - i;   // j-th newest
        S.acoef[j] = t[i];
        S.acoef[32 + j] = -gamma * u[i];
    }
    S.sc[SC_GAMMA] = gamma;
}

// d = -(gamma g + sum_j a_j s_j + sum_j c_j y_j); four floats per thread and
// four pairs per step in flight (the vectors start 16-byte aligned when n2 is
// a multiple of 4, else a scalar loop)
__global__ void __launch_bounds__(256) k_lb_dir(SolverDev S) {
    __shared__ float cs[32], cy[32];
    __shared__ const float* ps[32];
    __shared__ const float* py[32];
    const int cnt = S.ints[SI_CNT];
    if (threadIdx.x < cnt) {
        const int idx = ring_idx(S, threadIdx.x);
        cs[threadIdx.x] = (float)S.acoef[threadIdx.x];
        cy[threadIdx.x] = (float)S.acoef[32 + threadIdx.x];
        ps[threadIdx.x] = S.sh + (long long)idx * S.n2;
        py[threadIdx.x] = S.yh + (long long)idx * S.n2;
    }
    __syncthreads();
    const float gamma = (float)S.sc[SC_GAMMA];
    if ((S.n2 & 3) == 0) {
        const long long n4 = S.n2 >> 2;
        const float4* g4 = reinterpret_cast<const float4*>(S.g);
        float4* d4 = reinterpret_cast<float4*>(S.d);
        GRID_STRIDE(i, n4) {
            const float4 gv = g4[i];
            float4 r = make_float4(gamma * gv.x, gamma * gv.y, gamma * gv.z, gamma * gv.w);
            int j = 0;
            for (; j + 4 <= cnt; j += 4) {
                float4 sv[4], yv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    sv[u] = reinterpret_cast<const float4*>(ps[j + u])[i];
                    yv[u] = reinterpret_cast<const float4*>(py[j + u])[i];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float a = cs[j + u], c = cy[j + u];
                    r.x = fmaf(c, yv[u].x, fmaf(a, sv[u].x, r.x));
                    r.y = fmaf(c, yv[u].y, fmaf(a, sv[u].y, r.y));
                    r.z = fmaf(c, yv[u].z, fmaf(a, sv[u].z, r.z));
                    r.w = fmaf(c, yv[u].w, fmaf(a, sv[u].w, r.w));
                }
            }
            for (; j < cnt; ++j) {
                const float4 sv = reinterpret_cast<const float4*>(ps[j])[i];
                const float4 yv = reinterpret_cast<const float4*>(py[j])[i];
                const float a = cs[j], c = cy[j];
                r.x = fmaf(c, yv.x, fmaf(a, sv.x, r.x));
                r.y = fmaf(c, yv.y, fmaf(a, sv.y, r.y));
                r.z = fmaf(c, yv.z, fmaf(a, sv.z, r.z));
                r.w = fmaf(c, yv.w, fmaf(a, sv.w, r.w));
            }
            d4[i] = make_float4(-r.x, -r.y, -r.z, -r.w);
        }
    } else {
        GRID_STRIDE(i, S.n2) {
            float r = gamma * S.g[i];
            for (int j = 0; j < cnt; ++j) r = fmaf(cy[j], py[j][i], fmaf(cs[j], ps[j][i], r));
            S.d[i] = -r;
        }
    }
}

// theta-space line-search inner products: <x - v, x - v>, <x - v, d>, <d, d>
__global__ void __launch_bounds__(kRedThreads) k_dots3(SolverDev S, double* part) {
    __shared__ double sh[32];
    Acc s0, s1, s2;
    GRID_STRIDE(i, S.n2) {
        const float w = S.x[i] - S.v[i];
        const float d = S.d[i];
        s0.add(w * w);
        s1.add(w * d);
        s2.add(d * d);
    }
    double r;
    r = block_sum(s0.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 3 + 0] = r;
    r = block_sum(s1.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 3 + 1] = r;
    r = block_sum(s2.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 3 + 2] = r;
}

__device__ double quartic_val(const double* c, double a) {
    return c[0] + a * (c[1] + a * (c[2] + a * (c[3] + a * c[4])));
}

__device__ void consider(const double* c, double a, double& best_a, double& best_v, bool& have) {
    // two Newton polishes on phi'
    for (int it = 0; it < 2; ++it) {
        const double d1 = c[1] + a * (2 * c[2] + a * (3 * c[3] + a * 4 * c[4]));
        const double d2 = 2 * c[2] + a * (6 * c[3] + a * 12 * c[4]);
        if (d2 != 0.0) a -= d1 / d2;
    }
    if (!(a > 0.0) || !isfinite(a)) return;
    const double v = quartic_val(c, a);
    if (!have || v < best_v || (v == best_v && a < best_a)) {
        have = true;
        best_a = a;
        best_v = v;
    }
}

// Minimiser over a > 0 of the quartic: real roots of phi'(a) =
// 4 c4 a^3 + 3 c3 a^2 + 2 c2 a + c1 in closed form (depressed cubic:
// trigonometric form for three real roots, Cardano otherwise), polished.
__device__ bool quartic_argmin(const double* c, double* out) {
    double best_a = 0.0, best_v = 0.0;
    bool have = false;
    const double A = 4 * c[4], B = 3 * c[3], C = 2 * c[2], D = c[1];
    if (A != 0.0) {
        const double p = B / A, q = C / A, r = D / A;
        const double P = q - p * p / 3.0;
        const double Q = 2.0 * p * p * p / 27.0 - p * q / 3.0 + r;
        const double disc = 0.25 * Q * Q + P * P * P / 27.0;
        const double sh = -p / 3.0;
        if (disc > 0.0) {
            const double sq = sqrt(disc);
            const double t = cbrt(-0.5 * Q + sq) + cbrt(-0.5 * Q - sq);
            consider(c, t + sh, best_a, best_v, have);
        } else if (P == 0.0) {
            consider(c, cbrt(-Q) + sh, best_a, best_v, have);
        } else {
            const double m = 2.0 * sqrt(-P / 3.0);
            double arg = 3.0 * Q / (P * m);
            arg = fmin(1.0, fmax(-1.0, arg));
            const double th = acos(arg) / 3.0;
            const double tpi = 2.0943951023931954923;  // 2 pi / 3
            for (int k = 0; k < 3; ++k) consider(c, m * cos(th - tpi * k) + sh, best_a, best_v, have);
        }
    } else if (B != 0.0) {
        const double dsc = C * C - 4 * B * D;
        if (dsc >= 0.0) {
            const double s = sqrt(dsc);
            consider(c, (-C + s) / (2 * B), best_a, best_v, have);
            consider(c, (-C - s) / (2 * B), best_a, best_v, have);
        }
    } else if (C != 0.0) {
        consider(c, -D / C, best_a, best_v, have);
    }
    *out = best_a;
    return have;
}

// One thread: finalise the 6 + 3 inner products, form phi's coefficients,
// check descent, pick alpha; alpha = 0 and a memory reset when no step.
__global__ void __launch_bounds__(kFinThreads) k_line_search(SolverDev S, const double* part6, int nb6,
                                                             const double* part3, double rho) {
    __shared__ double sh[32];
    double d6[6], d3[3];
    for (int k = 0; k < 6; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nb6; i += blockDim.x) v += part6[i * 6 + k];
        d6[k] = block_sum(v, sh);
    }
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) v += part3[i * 3 + k];
        d3[k] = block_sum(v, sh);
    }
    if (threadIdx.x != 0) return;
    double c[5];
    c[0] = 0.5 * d6[0] + 0.5 * rho * d3[0];
    c[1] = d6[1] + rho * d3[1];
    c[2] = 0.5 * d6[3] + d6[2] + 0.5 * rho * d3[2];
    c[3] = d6[4];
    c[4] = 0.5 * d6[5];
    for (int k = 0; k < 5; ++k) S.sc[SC_C0 + k] = c[k];
    double a = 0.0;
    bool ok = false;
    if (c[1] < 0.0) ok = quartic_argmin(c, &a);
    if (!ok) {
        // no minimiser on a > 0 along d: no step, memory cleared; counted as a
        // restart unless the direction test already counted this iteration
        a = 0.0;
        S.ints[SI_CNT] = 0;
        if (!S.ints[SI_RFLAG]) S.ints[SI_RESTARTS] += 1;
    }
    bool finite = isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]) && isfinite(c[3]) && isfinite(c[4]);
    if (!finite) {
        a = 0.0;
        S.ints[SI_STATUS] = TLR_ERR_NONFINITE;
    }
    S.sc[SC_ALPHA] = a;
}

// x += a d ; s_free = a d
__global__ void k_step_theta(SolverDev S) {
    const double ad = S.sc[SC_ALPHA];
    const float a = (float)ad;
    const int R = S.ring;
    const int fr = (S.ints[SI_NEWEST] + 1) % R;
    float* s = S.sh + (long long)fr * S.n2;
    GRID_STRIDE(i, S.n2) {
        const float st = a * S.d[i];
        s[i] = st;
        S.x[i] += st;
    }
}

// y_free = (gf + rho (x - v)) - g ; g <- gf + rho (x - v); partials ss, sy, yy
__global__ void __launch_bounds__(kRedThreads) k_pair_prep(SolverDev S, double rho, double* part) {
    __shared__ double sh[32];
    const float r = (float)rho;
    const int R = S.ring;
    const int fr = (S.ints[SI_NEWEST] + 1) % R;
    const float* s = S.sh + (long long)fr * S.n2;
    float* y = S.yh + (long long)fr * S.n2;
    Acc ss, sy, yy;
    GRID_STRIDE(i, S.n2) {
        const float gn = S.gf[i] + r * (S.x[i] - S.v[i]);
        const float yi = gn - S.g[i];
        y[i] = yi;
        S.g[i] = gn;
        const float si = s[i];
        ss.add(si * si);
        sy.add(si * yi);
        yy.add(yi * yi);
    }
    double t;
    t = block_sum(ss.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 3 + 0] = t;
    t = block_sum(sy.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 3 + 1] = t;
    t = block_sum(yy.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x * 3 + 2] = t;
}

// one thread: accept the pair (s, y) when alpha > 0 and <s,y> > 1e-12 |s||y|;
// record f = 0.5 ||R||^2 from the nf residual-norm partials.
__global__ void __launch_bounds__(kFinThreads) k_pair_accept(SolverDev S, const double* part3, const double* partf,
                                                             int nf) {
    __shared__ double sh[32];
    double v[4];
    for (int k = 0; k < 3; ++k) {
        double a = 0.0;
        for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) a += part3[i * 3 + k];
        v[k] = block_sum(a, sh);
    }
    {
        // the residual-norm partials can number tens of thousands (one per
        // fused residual-step CTA): four independent sums per thread in a
        // fixed order keep the loads in flight
        const int bd = blockDim.x;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int i = threadIdx.x;
        for (; i + 3 * bd < nf; i += 4 * bd) {
            a0 += partf[i];
            a1 += partf[i + bd];
            a2 += partf[i + 2 * bd];
            a3 += partf[i + 3 * bd];
        }
        for (; i < nf; i += bd) a0 += partf[i];
        v[3] = block_sum((a0 + a1) + (a2 + a3), sh);
    }
    if (threadIdx.x != 0) return;
    const double ss = v[0], sy = v[1], yy = v[2], rr = v[3];
    const double f = 0.5 * rr;
    S.sc[SC_F] = f;
    const int it = S.ints[SI_ITERS];
    if (it < TLR_MAX_HIST) S.fhist[it] = f;
    S.ints[SI_ITERS] = it + 1;
    if (!isfinite(f)) S.ints[SI_STATUS] = TLR_ERR_NONFINITE;
    if (S.sc[SC_ALPHA] > 0.0 && sy > 1e-12 * sqrt(ss * yy)) {
        const int R = S.ring;
        const int fr = (S.ints[SI_NEWEST] + 1) % R;
        S.ints[SI_NEWEST] = fr;
        S.ints[SI_CNT] = min(S.ints[SI_CNT] + 1, S.m);
        S.rho_h[fr] = 1.0 / sy;
        S.sy_h[fr] = sy;
        S.yy_h[fr] = yy;
    }
}

// ADMM z- and dual updates (eq. 23, 24 in scaled form) and v = z - u
__global__ void k_admm_zu(SolverDev S, double lam, double rho) {
    const float den = (float)(1.0 / (1.0 + 2.0 * lam / rho));
    GRID_STRIDE(i, S.n2) {
        const float x = S.x[i], u = S.u[i];
        const float z = (x + u) * den;
        const float un = u + x - z;
        S.z[i] = z;
        S.u[i] = un;
        S.v[i] = z - un;
    }
}

// start of the solve: z = x, u = 0, v = x, counters cleared
__global__ void k_admm_init(SolverDev S) {
    GRID_STRIDE(i, S.n2) {
        const float x = S.x[i];
        S.z[i] = x;
        S.u[i] = 0.f;
        S.v[i] = x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.ints[SI_CNT] = 0;
        S.ints[SI_NEWEST] = 0;
        S.ints[SI_ITERS] = 0;
        S.ints[SI_RESTARTS] = 0;
        S.ints[SI_STATUS] = 0;
        S.ints[SI_RFLAG] = 0;
    }
}

// resumed solve: v = z - u from the stored split; counters cleared
__global__ void k_admm_resume(SolverDev S) {
    GRID_STRIDE(i, S.n2) S.v[i] = S.z[i] - S.u[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.ints[SI_CNT] = 0;
        S.ints[SI_NEWEST] = 0;
        S.ints[SI_ITERS] = 0;
        S.ints[SI_RESTARTS] = 0;
        S.ints[SI_STATUS] = 0;
        S.ints[SI_RFLAG] = 0;
    }
}

// record f0 = 0.5 ||R||^2
__global__ void k_record_f0(SolverDev S, const double* partf) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double rr = 0;
    for (int i = 0; i < kRedBlocks; ++i) rr += partf[i];
    S.sc[SC_F0] = 0.5 * rr;
    S.sc[SC_F] = 0.5 * rr;
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
cudaError_t sv_norm_part(const cf* R, long long n, double* part, cudaStream_t st) {
    (void)launch_pass(k_norm_part, dim3(kRedBlocks), dim3(kRedThreads), st, R, n, part);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_record_f0(const SolverDev& S, const double* partf, cudaStream_t st) {
    (void)launch_pass(k_record_f0, dim3(1), dim3(32), st, S, partf);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_admm_init(const SolverDev& S, cudaStream_t st) {
    (void)launch_pass(k_admm_init, dim3(1024), dim3(256), st, S);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_admm_resume(const SolverDev& S, cudaStream_t st) {
    (void)launch_pass(k_admm_resume, dim3(1024), dim3(256), st, S);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_xupdate_start(const SolverDev& S, double rho, cudaStream_t st) {
    (void)launch_pass(k_xupdate_start, dim3(1024), dim3(256), st, S, rho);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_direction(const SolverDev& S, cudaStream_t st) {
    for (int j0 = 0; j0 < S.m; j0 += kLbGroup) {
        (void)launch_pass(k_lb_dots, dim3(kRedBlocks), dim3(kLbThreads), st, S, j0);
        counted(1);
    }
    (void)launch_pass(k_lb_solve, dim3(1), dim3(kFinThreads), st, S);
    counted(1);
    (void)launch_pass(k_lb_dir, dim3(1024), dim3(256), st, S);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_dots3(const SolverDev& S, double* part, cudaStream_t st) {
    (void)launch_pass(k_dots3, dim3(kRedBlocks), dim3(kRedThreads), st, S, part);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_line_search(const SolverDev& S, const double* part6, int nb6, const double* part3, double rho,
                           cudaStream_t st) {
    (void)launch_pass(k_line_search, dim3(1), dim3(kFinThreads), st, S, part6, nb6, part3, rho);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_step_residual(cf* R, const cf* A1, const cf* A2, long long n, const double* alpha,
                             double* partf, cudaStream_t st) {
    (void)launch_pass(k_step_residual, dim3(kRedBlocks), dim3(kRedThreads), st, R, A1, A2, n, alpha, partf);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_step_theta(const SolverDev& S, cudaStream_t st) {
    (void)launch_pass(k_step_theta, dim3(1024), dim3(256), st, S);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_pair_prep(const SolverDev& S, double rho, double* part, cudaStream_t st) {
    (void)launch_pass(k_pair_prep, dim3(kRedBlocks), dim3(kRedThreads), st, S, rho, part);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_pair_accept(const SolverDev& S, const double* part3, const double* partf, int nf, cudaStream_t st) {
    (void)launch_pass(k_pair_accept, dim3(1), dim3(kFinThreads), st, S, part3, partf, nf);
    counted(1);
    return cudaGetLastError();
}
cudaError_t sv_admm_zu(const SolverDev& S, double lam, double rho, cudaStream_t st) {
    (void)launch_pass(k_admm_zu, dim3(1024), dim3(256), st, S, lam, rho);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
