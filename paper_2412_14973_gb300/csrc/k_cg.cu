// Benchmark solver of eq. (4): conjugate gradients on the normal equations
//   P(G P(Z)) + 2 lambda Z = P(D-hat^H U-hat),  G = D-hat^H D-hat,
// P Z = (Z + Z^T)/2, with the real inner product Re tr(A^H B).  From Z = 0
// every iterate, residual and direction is exactly symmetric (the right-hand
// side is, and each update is elementwise symmetric), so P(p) = p and one
// iteration is y = G p (a dense GEMM, launched by the caller) plus the passes
// here: Ap = P(y) + 2 lambda p with <p, Ap>, the step, and the new direction.
// Scalars live on the device (FP64); reductions run on fixed grids and sum in
// a fixed order.
#include "internal.h"
#include "reduce.h"

namespace tlr {

namespace {

constexpr int CG_T = 32;   // transpose tile

enum CgSlot { CG_RR = 0, CG_PAP, CG_ALPHA, CG_BETA, CG_BN, CG_DONE, CG_ITERS, CG_COUNT };

__device__ __forceinline__ double sum_fixed(const double* part, int n, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    return block_sum(v, sh);
}

// out = P(y) + s2 * p (s2 = 2 lambda), or out = P(y) if p == nullptr;
// partial <p, out> per block when part != nullptr.  32 x 32 tiles: the tile
// and its mirror are read through shared memory, both coalesced.
__global__ void __launch_bounds__(256) k_cg_sym(const cf* __restrict__ y, const cf* __restrict__ p, float s2,
                                                cf* __restrict__ out, int n, double* __restrict__ part) {
    __shared__ cf t[CG_T][CG_T + 1];
    __shared__ double sh[32];
    const int bx = blockIdx.x * CG_T, by = blockIdx.y * CG_T;   // out tile rows by.., cols bx..
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;     // 8 rows per pass
    // mirror tile: y[bx + r][by + c] -> t[c][r]
    for (int r = ty; r < CG_T; r += 8) {
        const int a = bx + r, b = by + tx;
        t[tx][r] = (a < n && b < n) ? y[(long long)a * n + b] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    Acc acc;
    for (int r = ty; r < CG_T; r += 8) {
        const int a = by + r, b = bx + tx;
        if (a < n && b < n) {
            const long long o = (long long)a * n + b;
            const cf u = y[o], v = t[r][tx];
            cf w = make_float2(0.5f * (u.x + v.x), 0.5f * (u.y + v.y));
            if (p) {
                const cf q = p[o];
                w.x = fmaf(s2, q.x, w.x);
                w.y = fmaf(s2, q.y, w.y);
                if (part) acc.add(fmaf(q.x, w.x, q.y * w.y));
            }
            out[o] = w;
        }
    }
    if (part) {
        const double s = block_sum(acc.val(), sh);
        if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// one block: sc[CG_RR] = sc[CG_BN] = ||r||^2 from partials; iteration count 0
__global__ void __launch_bounds__(kRedThreads) k_cg_init(const double* part, int np, double* sc) {
    __shared__ double sh[32];
    const double rr = sum_fixed(part, np, sh);
    if (threadIdx.x == 0) {
        sc[CG_RR] = rr;
        sc[CG_BN] = rr;
        sc[CG_DONE] = rr > 0.0 ? 0.0 : 1.0;
        sc[CG_ITERS] = 0.0;
    }
}

// one block: alpha = rr / <p, Ap>, 0 once converged (or a non-positive curvature)
__global__ void __launch_bounds__(kRedThreads) k_cg_alpha(const double* part, int np, double* sc) {
    __shared__ double sh[32];
    const double pap = sum_fixed(part, np, sh);
    if (threadIdx.x == 0) {
        sc[CG_PAP] = pap;
        const bool go = sc[CG_DONE] == 0.0 && pap > 0.0 && isfinite(pap);
        sc[CG_ALPHA] = go ? sc[CG_RR] / pap : 0.0;
        if (!go) sc[CG_DONE] = 1.0;
    }
}

// x += alpha p ; r -= alpha Ap ; partial ||r||^2
__global__ void __launch_bounds__(kRedThreads) k_cg_step(cf* __restrict__ x, cf* __restrict__ r,
                                                         const cf* __restrict__ p, const cf* __restrict__ Ap,
                                                         long long n2, const double* __restrict__ sc,
                                                         double* __restrict__ part) {
    __shared__ double sh[32];
    const float a = (float)sc[CG_ALPHA];
    Acc acc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        cf ri = r[i];
        if (a != 0.f) {
            const cf pi = p[i], qi = Ap[i];
            cf xi = x[i];
            xi.x = fmaf(a, pi.x, xi.x);
            xi.y = fmaf(a, pi.y, xi.y);
            ri.x = fmaf(-a, qi.x, ri.x);
            ri.y = fmaf(-a, qi.y, ri.y);
            x[i] = xi;
            r[i] = ri;
        }
        acc.add(fmaf(ri.x, ri.x, ri.y * ri.y));
    }
    const double s = block_sum(acc.val(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// one block: beta = rr_new / rr, convergence test ||r|| <= tol ||b||
__global__ void __launch_bounds__(kRedThreads) k_cg_beta(const double* part, int np, double tol, double* sc) {
    __shared__ double sh[32];
    const double rn = sum_fixed(part, np, sh);
    if (threadIdx.x == 0) {
        if (sc[CG_ALPHA] != 0.0) {
            sc[CG_BETA] = rn / sc[CG_RR];
            sc[CG_RR] = rn;
            sc[CG_ITERS] += 1.0;
            if (!(rn > tol * tol * sc[CG_BN])) sc[CG_DONE] = 1.0;
        } else {
            sc[CG_BETA] = 0.0;
        }
    }
}

// p = r + beta p (skipped once converged)
__global__ void k_cg_dir(cf* __restrict__ p, const cf* __restrict__ r, long long n2, const double* __restrict__ sc) {
    if (sc[CG_DONE] != 0.0 && sc[CG_ALPHA] == 0.0) return;
    const float b = (float)sc[CG_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        const cf ri = r[i];
        cf pi = p[i];
        pi.x = fmaf(b, pi.x, ri.x);
        pi.y = fmaf(b, pi.y, ri.y);
        p[i] = pi;
    }
}

}  // namespace

int cg_partials(int n) {
    const int t = (n + CG_T - 1) / CG_T;
    return std::max(t * t, kRedBlocks);
}

cudaError_t cg_sym(const cf* y, const cf* p, float s2, cf* out, int n, double* part, cudaStream_t st) {
    const int t = (n + CG_T - 1) / CG_T;
    k_cg_sym<<<dim3(t, t), 256, 0, st>>>(y, p, s2, out, n, part);
    counted(1);
    return cudaGetLastError();
}

// start: x = 0, r = p = b (r holds b on entry), sc cleared, rr = ||b||^2
cudaError_t cg_start(cf* x, cf* r, cf* p, int n, double* part, double* sc, cudaStream_t st) {
    const long long n2 = (long long)n * n;
    cudaError_t e = cudaMemsetAsync(x, 0, n2 * sizeof(cf), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, r, n2 * sizeof(cf), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, 8 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_cg_step<<<kRedBlocks, kRedThreads, 0, st>>>(x, r, p, p, n2, sc, part);   // alpha = 0: norm only
    counted(1);
    k_cg_init<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t cg_iteration_tail(cf* x, cf* r, cf* p, const cf* Ap, int n, double tol, double* part, double* sc,
                              cudaStream_t st) {
    const int t = (n + CG_T - 1) / CG_T;
    const long long n2 = (long long)n * n;
    k_cg_alpha<<<1, kRedThreads, 0, st>>>(part, t * t, sc);
    counted(1);
    k_cg_step<<<kRedBlocks, kRedThreads, 0, st>>>(x, r, p, Ap, n2, sc, part);
    counted(1);
    k_cg_beta<<<1, kRedThreads, 0, st>>>(part, kRedBlocks, tol, sc);
    counted(1);
    k_cg_dir<<<1024, 256, 0, st>>>(p, r, n2, sc);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
