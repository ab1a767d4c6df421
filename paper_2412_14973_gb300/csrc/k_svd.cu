// Tile singular value decompositions for the hyper-parameter selection and
// warm start (the tile rank rule and the SVD / Takagi initialisation).
//
// One CTA per b x b tile of a dense nr x nr matrix (row-major): one-sided
// (Hestenes) Jacobi on the tile's columns, complex FP32.  A sweep visits every
// column pair once in round-robin order (b - 1 rounds of b/2 disjoint pairs,
// one warp per pair); a pair (p, q) with Gram entries alpha = |a_p|^2,
// beta = |a_q|^2, gamma = a_p^H a_q is made orthogonal by the unitary
// [a_p, a_q e^{-i phi}] [[c, s], [-s, c]], phi = arg gamma, t = s / c the
// smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2 |gamma|);
// V accumulates the same column operations.  Sweeps stop once every pair has
// |gamma| <= tol sqrt(alpha beta) (or after max_sweeps): then
// A_0 = U Sigma V^H with sigma_c = |a_c| and u_c = a_c / sigma_c.
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
                                                          const int2* __restrict__ tiles, int b, int nb,
                                                          cf* __restrict__ work, int want_vec, int max_sweeps,
                                                          float tol, float* __restrict__ sig,
                                                          int* __restrict__ order, int* __restrict__ sweeps_out) {
    const int t = blockIdx.x;
    const int2 ij = tiles[t];
    const long long bb = (long long)b * b;
    cf* A = work + (long long)t * (want_vec ? 2 : 1) * bb;   // column-major b x b
    cf* V = A + bb;
    __shared__ unsigned int smax;
    __shared__ float snorm[512];
    // load the tile (coalesced along its rows), V = I
    for (long long e = threadIdx.x; e < bb; e += blockDim.x) {
        const int r = (int)(e / b), c = (int)(e % b);
        A[(long long)c * b + r] = X[((long long)ij.x * b + r) * ldx + (long long)ij.y * b + c];
        if (want_vec) V[e] = make_float2((e / b) == (e % b) ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    int sw = 0;
    for (; sw < max_sweeps; ++sw) {
        if (threadIdx.x == 0) smax = 0u;
        __syncthreads();
        for (int r = 0; r < nb - 1; ++r) {
            for (int k = warp; k < nb / 2; k += nwarp) {
                const int p = player(k, r, nb), q = player(nb - 1 - k, r, nb);
                if (p >= b || q >= b) continue;   // the dummy player of an odd b
                cf* ap = A + (long long)p * b;
                cf* aq = A + (long long)q * b;
                float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
                for (int i = lane; i < b; i += 32) {
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
                for (int i = lane; i < b; i += 32) {
                    const cf x = ap[i], y = aq[i];
                    const cf yb = make_float2(y.x * er - y.y * ei, y.x * ei + y.y * er);
                    ap[i] = make_float2(c * x.x - s * yb.x, c * x.y - s * yb.y);
                    aq[i] = make_float2(s * x.x + c * yb.x, s * x.y + c * yb.y);
                }
                if (want_vec) {
                    cf* vp = V + (long long)p * b;
                    cf* vq = V + (long long)q * b;
                    for (int i = lane; i < b; i += 32) {
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
    // sigma_c = |a_c|, then the order of decreasing sigma (ties by column)
    for (int c = warp; c < b; c += nwarp) {
        const cf* ac = A + (long long)c * b;
        float s2 = 0.f;
        for (int i = lane; i < b; i += 32) s2 = fmaf(ac[i].x, ac[i].x, fmaf(ac[i].y, ac[i].y, s2));
        s2 = warp_sumf(s2);
        if (lane == 0) snorm[c] = sqrtf(s2);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        const float v = snorm[c];
        int rk = 0;
        for (int c2 = 0; c2 < b; ++c2) {
            const float w = snorm[c2];
            rk += (w > v) || (w == v && c2 < c);
        }
        sig[(long long)t * b + rk] = v;
        if (order) order[(long long)t * b + rk] = c;
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
//   off-diagonal (kind 0): L = U_k Sigma_k^1/2, R = conj(V_k) Sigma_k^1/2, so
//     L R^T = U_k Sigma_k V_k^H;
//   low-rank diagonal (kind 1): Q = conj(V_k) E_k Sigma_k^1/2 with
//     E = diag(V^T U)^1/2 (Takagi form of the symmetric tile), Q Q^T = U_k Sigma_k V_k^H;
//   dense diagonal (kind 2): Z = the tile itself (no SVD).
__global__ void k_warm_fill(const cf* __restrict__ X, long long ldx, const WarmTile* __restrict__ wt, int b,
                            const cf* __restrict__ work, const float* __restrict__ sig,
                            const int* __restrict__ order, cf* __restrict__ theta) {
    const WarmTile w = wt[blockIdx.x];
    const long long bb = (long long)b * b;
    if (w.kind == 2) {
        for (long long e = threadIdx.x; e < bb; e += blockDim.x) {
            const int r = (int)(e / b), c = (int)(e % b);
            theta[w.offL + e] = X[((long long)w.i * b + r) * ldx + (long long)w.i * b + c];
        }
        return;
    }
    const cf* A = work + (long long)w.svd * 2 * bb;
    const cf* V = A + bb;
    for (int q = threadIdx.x; q < w.k; q += blockDim.x) {
        const int c = order[(long long)w.svd * b + q];
        const float s = sig[(long long)w.svd * b + q];
        const float rs = sqrtf(s), inv = s > 0.f ? 1.f / s : 0.f;
        const cf* ac = A + (long long)c * b;
        const cf* vc = V + (long long)c * b;
        if (w.kind == 0) {
            for (int r = 0; r < b; ++r) {
                const cf u = ac[r], v = vc[r];
                theta[w.offL + (long long)r * w.k + q] = make_float2(u.x * inv * rs, u.y * inv * rs);
                theta[w.offR + (long long)r * w.k + q] = make_float2(v.x * rs, -v.y * rs);
            }
        } else {
            // d = sum_r V[r] U[r] (U = a_c / s): the phase pair of the Takagi form
            float dr = 0.f, di = 0.f;
            for (int r = 0; r < b; ++r) {
                const cf u = ac[r], v = vc[r];
                dr = fmaf(v.x, u.x, fmaf(-v.y, u.y, dr));
                di = fmaf(v.x, u.y, fmaf(v.y, u.x, di));
            }
            const float ph = 0.5f * atan2f(di, dr);
            const float er = cosf(ph), ei = sinf(ph);
            for (int r = 0; r < b; ++r) {
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

cudaError_t tile_svd(const cf* X, long long ldx, const int2* tiles, int ntiles, int b, cf* work, bool vec,
                     int max_sweeps, float tol, float* sig, int* order, int* sweeps, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    if (b < 1 || b > 512) return cudaErrorInvalidValue;
    const int nb = b + (b & 1);
    k_tile_svd<<<ntiles, SVD_THREADS, 0, st>>>(X, ldx, tiles, b, nb, work, vec ? 1 : 0, max_sweeps, tol, sig, order,
                                               sweeps);
    counted(1);
    return cudaGetLastError();
}

cudaError_t rank_rule(const float* sig, int ntiles, int b, double eps, int* ranks, double* v0, cudaStream_t st) {
    k_rank_rule<<<1, 256, 0, st>>>(sig, ntiles, b, eps, ranks, v0);
    counted(1);
    return cudaGetLastError();
}

cudaError_t warm_fill(const cf* X, long long ldx, const WarmTile* wt, int nt, int b, const cf* work, const float* sig,
                      const int* order, cf* theta, cudaStream_t st) {
    if (nt == 0) return cudaSuccess;
    k_warm_fill<<<nt, 128, 0, st>>>(X, ldx, wt, b, work, sig, order, theta);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
