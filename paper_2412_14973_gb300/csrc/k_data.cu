// Data-preparation kernels: Hilbert receiver order (eq. 10), normalisation
// alpha (Hyper-parameter selection section), receiver-major reordered panels
// (eq. 14) and the natural-order back-mapping X = S X_h S^T (eq. 11).
#include "internal.h"

namespace tlr {

// Distance of cell (x, y) along the Hilbert curve on an n x n square (n a
// power of two): quadrant (rx, ry) at level s contributes s*s*((3 rx) ^ ry)
// cells visited before it; the coordinates are then reflected / swapped so the
// sub-square is walked in the base orientation (0,0),(0,1),(1,1),(1,0).
__device__ __forceinline__ long long hilbert_d(long long n, long long x, long long y) {
    long long d = 0;
    for (long long s = n >> 1; s > 0; s >>= 1) {
        const int rx = (x & s) ? 1 : 0;
        const int ry = (y & s) ? 1 : 0;
        d += s * s * (long long)((3 * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            const long long t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// slot[key(r)] = r for every receiver; slot is n*n, pre-filled with -1.
__global__ void k_hilbert_scatter(int nx, int ny, long long n, int32_t* slot) {
    const long long nr = (long long)nx * ny;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
         r += (long long)gridDim.x * blockDim.x) {
        const long long x = r % nx, y = r / nx;
        slot[hilbert_d(n, x, y)] = (int32_t)r;
    }
}

__global__ void k_fill_i32(int32_t* p, long long n, int32_t v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Stable compaction of the occupied slots in key order, one block of 1024
// threads: perm[a] = receiver with the a-th smallest key.
__global__ void __launch_bounds__(1024) k_hilbert_compact(const int32_t* slot, long long nslot, int32_t* perm) {
    __shared__ long long cnt[1024];
    const int t = threadIdx.x;
    const long long per = (nslot + 1023) / 1024;
    const long long lo = t * per, hi = min(nslot, lo + per);
    long long c = 0;
    for (long long i = lo; i < hi; ++i) c += (slot[i] >= 0);
    cnt[t] = c;
    __syncthreads();
    // inclusive Hillis-Steele scan
    for (int off = 1; off < 1024; off <<= 1) {
        long long v = (t >= off) ? cnt[t - off] : 0;
        __syncthreads();
        cnt[t] += v;
        __syncthreads();
    }
    long long pos = cnt[t] - c;
    for (long long i = lo; i < hi; ++i)
        if (slot[i] >= 0) perm[pos++] = slot[i];
}

cudaError_t hilbert_perm(int nx, int ny, int32_t* perm, int32_t* slot, cudaStream_t st) {
    long long n = 1;
    while (n < nx || n < ny) n <<= 1;
    const long long nslot = n * n;
    k_fill_i32<<<256, 256, 0, st>>>(slot, nslot, -1);
    counted(1);
    k_hilbert_scatter<<<256, 256, 0, st>>>(nx, ny, n, slot);
    counted(1);
    k_hilbert_compact<<<1, 1024, 0, st>>>(slot, nslot, perm);
    counted(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// alpha = max |D| : per-block maxima of re^2 + im^2 in FP64, then one block.
// ---------------------------------------------------------------------------
__global__ void k_max_abs2_part(const cf* __restrict__ D, long long n, double* part) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cf v = D[i];
        const double a = (double)v.x * v.x + (double)v.y * v.y;
        m = a > m ? a : m;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_max_final_sqrt(const double* part, int nblk, double* out) {
    __shared__ double sh[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) m = fmax(m, part[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(sh[0]);
}

cudaError_t max_abs2(const cf* D, long long n, double* part, int nblk, double* out, cudaStream_t st) {
    k_max_abs2_part<<<nblk, 256, 0, st>>>(D, n, part);
    counted(1);
    k_max_final_sqrt<<<1, 256, 0, st>>>(part, nblk, out);
    counted(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dt[a, s] = RN32(D[s, perm[a]] / RN32(alpha)).  Walks D in natural receiver order so both
// the read (a row segment of D) and the write (a row segment of Dt, at row
// inv[r]) are 256-byte contiguous; a 32 x 32 tile is transposed in shared memory.
// ---------------------------------------------------------------------------
__global__ void k_inverse_perm(const int32_t* perm, long long n, int32_t* inv) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        inv[perm[a]] = (int32_t)a;
}

__global__ void __launch_bounds__(256) k_permute_normalise(const cf* __restrict__ D, long long ns, long long nr,
                                                            const int32_t* __restrict__ inv,
                                                            const double* __restrict__ alpha_dev,
                                                            cf* __restrict__ Dt) {
    __shared__ cf tile[32][33];
    const long long r0 = (long long)blockIdx.x * 32, s0 = (long long)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    // one IEEE FP32 division by alpha rounded to FP32: Dt = RN(D / RN(alpha))
    const float alpha = (float)alpha_dev[0];
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const long long s = s0 + ty + j, r = r0 + tx;
        cf v = make_float2(0.f, 0.f);
        if (s < ns && r < nr) v = D[s * nr + r];
        tile[ty + j][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const long long r = r0 + ty + j, s = s0 + tx;
        if (r < nr && s < ns) {
            const cf v = tile[tx][ty + j];
            cf o;
            o.x = __fdiv_rn(v.x, alpha);
            o.y = __fdiv_rn(v.y, alpha);
            Dt[(long long)inv[r] * ns + s] = o;
        }
    }
}

cudaError_t permute_normalise(const cf* D, long long ns, long long nr, const int32_t* perm,
                              const double* alpha_dev, cf* Dt, cudaStream_t st) {
    // The perm buffer holds 2*nr slots: perm[0..nr) then its inverse.
    int32_t* inv = const_cast<int32_t*>(perm) + nr;
    k_inverse_perm<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(perm, nr, inv);
    counted(1);
    dim3 grid((unsigned)((nr + 31) / 32), (unsigned)((ns + 31) / 32));
    k_permute_normalise<<<grid, dim3(32, 8), 0, st>>>(D, ns, nr, inv, alpha_dev, Dt);
    counted(1);
    return cudaGetLastError();
}

// Block of row r: r / b for equal tiles, else the largest i with roff[i] <= r.
__device__ __forceinline__ int block_of(long long r, long long b, const long long* roff, int N) {
    if (!roff) return (int)(r / b);
    int lo = 0, hi = N - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (roff[mid] <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// X_h = C(theta) assembled entry by entry from the stacked unknown (eq. 6-9,
// 15).  An entry of a super-diagonal tile evaluates exactly the expression of
// its mirror in the sub-diagonal tile (same products, same order), so the
// result is bitwise symmetric, as X_ji = X_ij^T demands.
// General form (general != 0): the tiles are listed row-major (i N + j) and
// every entry is its own tile's L R^T (or Z entry), without mirroring.
// roff == nullptr: N tiles of size b; else block i covers rows roff[i] ..
// roff[i + 1] - 1.
__global__ void k_assemble(const cf* __restrict__ th, long long nr, long long b, int N, const AsmTile* __restrict__ t,
                           cf* __restrict__ Xh, int general, const long long* __restrict__ roff) {
    const long long n2 = nr * nr;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2;
         e += (long long)gridDim.x * blockDim.x) {
        long long r = e / nr, c = e % nr;
        int i = block_of(r, b, roff, N), j = block_of(c, b, roff, N);
        if (general) {
            const AsmTile& a = t[i * N + j];
            const long long rr = r - (roff ? roff[i] : i * b), cc = c - (roff ? roff[j] : j * b);
            const long long di = roff ? roff[i + 1] - roff[i] : b;
            float x = 0.f, y = 0.f;
            if (i == j && a.dense) {
                const cf u = th[a.off_l + rr * di + cc];
                x = u.x;
                y = u.y;
            } else {
                const cf* L = th + a.off_l + rr * a.k;
                const cf* R = th + a.off_r + cc * a.k;
                for (int q = 0; q < a.k; ++q) {
                    const cf l = L[q], m = R[q];
                    x = fmaf(l.x, m.x, fmaf(-l.y, m.y, x));
                    y = fmaf(l.x, m.y, fmaf(l.y, m.x, y));
                }
            }
            Xh[e] = make_float2(x, y);
            continue;
        }
        if (i < j) {  // mirror into the sub-diagonal tile
            const long long tr = r;
            r = c;
            c = tr;
            const int ti = i;
            i = j;
            j = ti;
        }
        long long rr = r - (roff ? roff[i] : i * b), cc = c - (roff ? roff[j] : j * b);
        if (i == j && rr > cc) {  // low-rank diagonal: evaluate the upper triangle's entry
            const long long t2 = rr;
            rr = cc;
            cc = t2;
        }
        const AsmTile& a = t[i == j ? i : N + (j * N - j * (j + 1) / 2 + (i - j - 1))];
        float x = 0.f, y = 0.f;
        if (i == j && a.dense) {
            const long long di = roff ? roff[i + 1] - roff[i] : b;
            const cf u = th[a.off_l + rr * di + cc], v = th[a.off_l + cc * di + rr];
            x = 0.5f * (u.x + v.x);
            y = 0.5f * (u.y + v.y);
        } else {
            const cf* L = th + a.off_l + rr * a.k;
            const cf* R = th + a.off_r + cc * a.k;
            for (int q = 0; q < a.k; ++q) {
                const cf l = L[q], m = R[q];
                x = fmaf(l.x, m.x, fmaf(-l.y, m.y, x));
                y = fmaf(l.x, m.y, fmaf(l.y, m.x, y));
            }
        }
        Xh[e] = make_float2(x, y);
    }
}

cudaError_t assemble_dense(const cf* theta, long long nr, long long b, int N, const AsmTile* tiles, cf* Xh,
                           cudaStream_t st, int general, const long long* roff) {
    k_assemble<<<1024, 256, 0, st>>>(theta, nr, b, N, tiles, Xh, general, roff);
    counted(1);
    return cudaGetLastError();
}

// X[r, q] = Xh[inv[r], inv[q]]  (X = S X_h S^T)
__global__ void k_unpermute(const cf* __restrict__ Xh, long long nr, const int32_t* __restrict__ inv,
                            cf* __restrict__ X) {
    const long long n2 = nr * nr;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / nr, q = e % nr;
        X[e] = Xh[(long long)inv[r] * nr + inv[q]];
    }
}

cudaError_t unpermute_dense(const cf* Xh, long long nr, const int32_t* perm, cf* X, cudaStream_t st) {
    const int32_t* inv = perm + nr;
    k_unpermute<<<1024, 256, 0, st>>>(Xh, nr, inv, X);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
