// Tile singular value decompositions for the hyper-parameter selection and
// warm start (the tile rank rule and the SVD / Takagi initialisation).
//
// One CTA per m x n tile of a dense nr x nr matrix (row-major): one-sided
// (Hestenes) Jacobi on the tile's n columns, complex FP32.  A sweep visits
// every column pair once in round-robin order (n - 1 rounds of n/2 disjoint
// pairs, one warp per pair); a pair (p, q) with Gram entries alpha = |a_p|^2,
// beta = |a_q|^2, gamma = a_p^H a_q is made orthogonal by the unitary
// [a_p, a_q e^{-i phi}] [[c, s], [-s, c]], phi = arg gamma, t = s / c the
// smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2 |gamma|);
// V accumulates the same column operations.  Sweeps stop once every pair has
// |gamma| <= tol sqrt(alpha beta) (or after max_sweeps): then
// A_0 = U Sigma V^H with sigma_c = |a_c| and u_c = a_c / sigma_c (columns that
// end at zero, n - m of them at least when n > m, have sigma_c = 0).
#include "internal.h"

namespace tlr {

namespace {

constexpr int SVD_THREADS = 1024;   // 32 warps: the pairs of a round run in parallel

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// player at position m of round r (circle method; position 0 is fixed)
__device__ __forceinline__ int player(int m, int r, int nb) { return m == 0 ? 0 : ((m - 1 + r) % (nb - 1)) + 1; }

__global__ void __launch_bounds__(SVD_THREADS) k_tile_svd(const cf* __restrict__ X, long long ldx,
                                                          const SvdTile* __restrict__ tiles, int bmax,
                                                          cf* __restrict__ work, int want_vec, int max_sweeps,
                                                          float tol, float* __restrict__ sig,
                                                          int* __restrict__ order, int* __restrict__ sweeps_out) {
    const int t = blockIdx.x;
    const SvdTile tg = tiles[t];
    // the matrix the sweeps work on: the tile (m x n) or its transpose
    const int m = tg.trans ? tg.n : tg.m, n = tg.trans ? tg.m : tg.n, nb = n + (n & 1);
    const long long slot = (long long)bmax * bmax;
    cf* A = work + (long long)t * (want_vec ? 2 : 1) * slot;   // column-major m x n
    cf* V = A + slot;                                          // column-major n x n
    __shared__ unsigned int smax;
    __shared__ float snorm[512];
    // load the tile (reads coalesced along the rows of X), V = I
    for (long long e = threadIdx.x; e < (long long)m * n; e += blockDim.x) {
        if (tg.trans) {
            const int r = (int)(e % m), c = (int)(e / m);   // A[r][c] = X tile[c][r]
            A[(long long)c * m + r] = X[((long long)tg.r0 + c) * ldx + (long long)tg.c0 + r];
        } else {
            const int r = (int)(e / n), c = (int)(e % n);
            A[(long long)c * m + r] = X[((long long)tg.r0 + r) * ldx + (long long)tg.c0 + c];
        }
    }
    if (want_vec)
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x)
            V[e] = make_float2((e / n) == (e % n) ? 1.f : 0.f, 0.f);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    int sw = 0;
    for (; sw < max_sweeps; ++sw) {
        if (threadIdx.x == 0) smax = 0u;
        __syncthreads();
        for (int r = 0; r < nb - 1; ++r) {
            for (int k = warp; k < nb / 2; k += nwarp) {
                const int p = player(k, r, nb), q = player(nb - 1 - k, r, nb);
                if (p >= n || q >= n) continue;   // the dummy player of an odd n
                cf* ap = A + (long long)p * m;
                cf* aq = A + (long long)q * m;
                float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
                for (int i = lane; i < m; i += 32) {
                    const cf x = ap[i], y = aq[i];
                    al = fmaf(x.x, x.x, fmaf(x.y, x.y, al));
                    be = fmaf(y.x, y.x, fmaf(y.y, y.y, be));
                    gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));    // Re(conj(x) y)
                    gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));   // Im(conj(x) y)
                }
                al = warp_sumf(al);
                be = warp_sumf(be);
                gr = warp_sumf(gr);
                gi = warp_sumf(gi);
                const float g = sqrtf(gr * gr + gi * gi);
                if (!(al > 0.f) || !(be > 0.f) || !(g > tol * sqrtf(al) * sqrtf(be))) continue;
                if (lane == 0) atomicMax(&smax, __float_as_uint(g / (sqrtf(al) * sqrtf(be))));
                const float zeta = (be - al) / (2.f * g);
                const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                const float c = rsqrtf(1.f + tt * tt), s = c * tt;
                const float er = gr / g, ei = -gi / g;   // e^{-i phi}
                for (int i = lane; i < m; i += 32) {
                    const cf x = ap[i], y = aq[i];
                    const cf yb = make_float2(y.x * er - y.y * ei, y.x * ei + y.y * er);
                    ap[i] = make_float2(c * x.x - s * yb.x, c * x.y - s * yb.y);
                    aq[i] = make_float2(s * x.x + c * yb.x, s * x.y + c * yb.y);
                }
                if (want_vec) {
                    cf* vp = V + (long long)p * n;
                    cf* vq = V + (long long)q * n;
                    for (int i = lane; i < n; i += 32) {
                        const cf x = vp[i], y = vq[i];
                        const cf yb = make_float2(y.x * er - y.y * ei, y.x * ei + y.y * er);
                        vp[i] = make_float2(c * x.x - s * yb.x, c * x.y - s * yb.y);
                        vq[i] = make_float2(s * x.x + c * yb.x, s * x.y + c * yb.y);
                    }
                }
            }
            __syncthreads();
        }
        if (__uint_as_float(smax) <= tol) {
            ++sw;
            break;
        }
        __syncthreads();
    }
    // sigma_c = |a_c|, then the order of decreasing sigma (ties by column);
    // slots n .. bmax-1 get sigma = -1 (below every threshold)
    for (int c = warp; c < n; c += nwarp) {
        const cf* ac = A + (long long)c * m;
        float s2 = 0.f;
        for (int i = lane; i < m; i += 32) s2 = fmaf(ac[i].x, ac[i].x, fmaf(ac[i].y, ac[i].y, s2));
        s2 = warp_sumf(s2);
        if (lane == 0) snorm[c] = sqrtf(s2);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const float v = snorm[c];
        int rk = 0;
        for (int c2 = 0; c2 < n; ++c2) {
            const float w = snorm[c2];
            rk += (w > v) || (w == v && c2 < c);
        }
        sig[(long long)t * bmax + rk] = v;
        if (order) order[(long long)t * bmax + rk] = c;
    }
    for (int c = n + threadIdx.x; c < bmax; c += blockDim.x) {
        sig[(long long)t * bmax + c] = -1.f;
        if (order) order[(long long)t * bmax + c] = 0;
    }
    if (threadIdx.x == 0 && sweeps_out) sweeps_out[t] = sw;
}

// one block: v0 = max sigma over all tiles; rank of tile t = #{sigma >= eps v0}
__global__ void k_rank_rule(const float* __restrict__ sig, int ntiles, int b, double eps, int* __restrict__ ranks,
                            double* __restrict__ v0_out) {
    __shared__ float smx[32];
    float m = 0.f;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) m = fmaxf(m, sig[(long long)t * b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) smx[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? smx[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) smx[0] = m;
    }
    __syncthreads();
    const double v0 = smx[0];
    const float thr = (float)(eps * v0);
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int k = 0;
        while (k < b && sig[(long long)t * b + k] >= thr) ++k;
        ranks[t] = k;
    }
    if (threadIdx.x == 0) *v0_out = v0;
}

// Warm-start factors from tile SVDs (one CTA per tile, one thread per column
// q < k of the factor, rows in a loop):
//   low-rank tile (kind 0, m x n): L = U_k Sigma_k^1/2 (m x k), R = conj(V_k)
//     Sigma_k^1/2 (n x k), so L R^T = U_k Sigma_k V_k^H;
//   low-rank diagonal of the reciprocal form (kind 1, square): Q = conj(V_k)
//     E_k Sigma_k^1/2 with E = diag(V^T U)^1/2 (Takagi form of the symmetric
//     tile), Q Q^T = U_k Sigma_k V_k^H;
//   dense diagonal (kind 2): Z = the m x m tile itself (no SVD).
//   A tile whose SVD ran on its transpose (trans: T^T = U' Sigma V'^H) has
//   U = conj(V'), V = conj(U'): L = conj(V'_k) Sigma^1/2, R = U'_k Sigma^1/2.
__global__ void k_warm_fill(const cf* __restrict__ X, long long ldx, const WarmTile* __restrict__ wt, int bmax,
                            const cf* __restrict__ work, const float* __restrict__ sig,
                            const int* __restrict__ order, cf* __restrict__ theta) {
    const WarmTile w = wt[blockIdx.x];
    const int m = w.m, n = w.n;
    const int jm = w.trans ? n : m, jn = w.trans ? m : n;   // the SVD's rows and columns
    if (w.kind == 2) {
        for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
            const int r = (int)(e / m), c = (int)(e % m);
            theta[w.offL + e] = X[((long long)w.r0 + r) * ldx + (long long)w.c0 + c];
        }
        return;
    }
    const long long slot = (long long)bmax * bmax;
    const cf* A = work + (long long)w.svd * 2 * slot;   // column-major jm x jn
    const cf* V = A + slot;                             // column-major jn x jn
    for (int q = threadIdx.x; q < w.k; q += blockDim.x) {
        const int c = order[(long long)w.svd * bmax + q];
        const float s = sig[(long long)w.svd * bmax + q];
        const float rs = sqrtf(s), inv = s > 0.f ? 1.f / s : 0.f;
        const cf* ac = A + (long long)c * jm;
        const cf* vc = V + (long long)c * jn;
        if (w.kind == 0) {
            // u_c = a_c / s (jm rows), v_c (jn rows)
            cf* Lq = theta + w.offL + q;
            cf* Rq = theta + w.offR + q;
            if (!w.trans) {
                for (int r = 0; r < m; ++r) Lq[(long long)r * w.k] = make_float2(ac[r].x * inv * rs, ac[r].y * inv * rs);
                for (int r = 0; r < n; ++r) Rq[(long long)r * w.k] = make_float2(vc[r].x * rs, -vc[r].y * rs);
            } else {
                for (int r = 0; r < m; ++r) Lq[(long long)r * w.k] = make_float2(vc[r].x * rs, -vc[r].y * rs);
                for (int r = 0; r < n; ++r) Rq[(long long)r * w.k] = make_float2(ac[r].x * inv * rs, ac[r].y * inv * rs);
            }
        } else {
            // d = sum_r V[r] U[r] (U = a_c / s): the phase pair of the Takagi form
            float dr = 0.f, di = 0.f;
            for (int r = 0; r < m; ++r) {
                const cf u = ac[r], v = vc[r];
                dr = fmaf(v.x, u.x, fmaf(-v.y, u.y, dr));
                di = fmaf(v.x, u.y, fmaf(v.y, u.x, di));
            }
            const float ph = 0.5f * atan2f(di, dr);
            const float er = cosf(ph), ei = sinf(ph);
            for (int r = 0; r < m; ++r) {
                const cf v = vc[r];
                // conj(v) e^{i ph} sqrt(s)
                const float xr = v.x * er + v.y * ei, xi = v.x * ei - v.y * er;
                theta[w.offL + (long long)r * w.k + q] = make_float2(xr * rs, xi * rs);
            }
        }
    }
}

}  // namespace

size_t tile_svd_work_bytes(int ntiles, int b, bool vec) { return (size_t)ntiles * (vec ? 2 : 1) * b * b * sizeof(cf); }

cudaError_t tile_svd(const cf* X, long long ldx, const SvdTile* tiles, int ntiles, int bmax, cf* work, bool vec,
                     int max_sweeps, float tol, float* sig, int* order, int* sweeps, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    if (bmax < 1 || bmax > 512) return cudaErrorInvalidValue;
    k_tile_svd<<<ntiles, SVD_THREADS, 0, st>>>(X, ldx, tiles, bmax, work, vec ? 1 : 0, max_sweeps, tol, sig, order,
                                               sweeps);
    counted(1);
    return cudaGetLastError();
}

cudaError_t rank_rule(const float* sig, int ntiles, int b, double eps, int* ranks, double* v0, cudaStream_t st) {
    k_rank_rule<<<1, 256, 0, st>>>(sig, ntiles, b, eps, ranks, v0);
    counted(1);
    return cudaGetLastError();
}

cudaError_t warm_fill(const cf* X, long long ldx, const WarmTile* wt, int nt, int bmax, const cf* work,
                      const float* sig, const int* order, cf* theta, cudaStream_t st) {
    if (nt == 0) return cudaSuccess;
    k_warm_fill<<<nt, 128, 0, st>>>(X, ldx, wt, bmax, work, sig, order, theta);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
