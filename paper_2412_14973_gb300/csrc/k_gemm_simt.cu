// FP32 SIMT grouped complex GEMM (CUDA cores): the plain-precision path for
// the TLR contractions -- compress T = F^T Dfrak, expand Y = F T~ (+ P Z Dfrak),
// the factor-gradient projections (eq. 25-27) and the dense adjoint
// G = V Dfrak^H.  Every product is complex, 4 real FMAs per complex MAC,
// FP32 accumulation; split-K partials are reduced elsewhere in a fixed order.
#include "internal.h"

namespace tlr {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int TM = 4, TN = 4;  // per-thread complex outputs (16 x 16 threads)

template <int AM>
__device__ __forceinline__ void load_a(cf (*As)[BM + 2], const GTerm& t, int M, int m0, int k0, int kend) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
        const int e = tid + r * NT;
        int mm, kk;
        if (AM == A_KM) {
            kk = e / BM;
            mm = e % BM;
        } else {
            mm = e / BK;
            kk = e % BK;
        }
        const int m = m0 + mm, k = k0 + kk;
        cf v = make_float2(0.f, 0.f);
        if (m < M && k < kend) {
            v = (AM == A_KM) ? t.A[(long long)k * t.lda + m] : t.A[(long long)m * t.lda + k];
            v.y *= t.sa;
        }
        As[kk][mm] = v;
    }
}

template <int BMD>
__device__ __forceinline__ void load_b(cf (*Bs)[BN + 2], const GTerm& t, int N, int n0, int k0, int kend) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
        const int e = tid + r * NT;
        int nn, kk;
        if (BMD == B_KN) {
            kk = e / BN;
            nn = e % BN;
        } else {
            nn = e / BK;
            kk = e % BK;
        }
        const int n = n0 + nn, k = k0 + kk;
        cf v = make_float2(0.f, 0.f);
        if (n < N && k < kend) {
            if (BMD == B_KN) {
                const long long row = t.g ? t.g[k] : k;
                v = t.B[row * t.ldb + n];
            } else {
                const long long row = t.g ? t.g[n] : n;
                v = t.B[row * t.ldb + k];
            }
            v.y *= t.sb;
        }
        Bs[kk][nn] = v;
    }
}

template <int AM, int BMD>
__global__ void __launch_bounds__(NT) k_cgemm_simt(const GProb* __restrict__ probs, int nsplit, int kchunk,
                                                   int epi, long long part_stride) {
    const int prob = blockIdx.z / nsplit, chunk = blockIdx.z % nsplit;
    const GProb& P = probs[prob];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= P.M || n0 >= P.N) return;

    __shared__ __align__(16) cf As[BK][BM + 2];
    __shared__ __align__(16) cf Bs[BK][BN + 2];

    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int ti = 0; ti < P.nt; ++ti) {
        const GTerm& t = P.t[ti];
        int kb = 0, ke = t.K;
        if (nsplit > 1) {
            kb = chunk * kchunk;
            ke = min(t.K, kb + kchunk);
        }
        for (int k0 = kb; k0 < ke; k0 += BK) {
            load_a<AM>(As, t, P.M, m0, k0, ke);
            load_b<BMD>(Bs, t, P.N, n0, k0, ke);
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float2 a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
                        acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
                        acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
                        acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
                    }
            }
            __syncthreads();
        }
    }

    cf* C = P.C + (epi == EPI_PARTIAL ? chunk * part_stride : 0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty * TM + i;
        if (m >= P.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx * TN + j;
            if (n >= P.N) continue;
            const long long o = (long long)m * P.ldc + n;
            cf v = acc[i][j];
            if (epi == EPI_SUB) {
                const cf s = P.S[o];
                v.x -= s.x;
                v.y -= s.y;
            } else if (epi == EPI_ACCUM) {
                const cf c = C[o];
                v.x += c.x;
                v.y += c.y;
            }
            C[o] = v;
        }
    }
}

}  // namespace

cudaError_t gemm_simt(const GemmLaunch& L, cudaStream_t st) {
    if (L.nprob == 0 || L.maxM == 0 || L.maxN == 0) return cudaSuccess;
    dim3 grid((L.maxN + BN - 1) / BN, (L.maxM + BM - 1) / BM, L.nprob * L.nsplit);
    const int kchunk = L.nsplit > 1 ? L.kchunk : 0;
#define TLR_LAUNCH(AMv, BMv)                                                                           \
    do {                                                                                               \
        k_cgemm_simt<AMv, BMv><<<grid, NT, 0, st>>>(L.d_probs, L.nsplit, kchunk, L.epi, L.part_stride); \
        counted(1);                                                                                    \
    } while (0)
    if (L.amode == A_KM && L.bmode == B_KN)
        TLR_LAUNCH(A_KM, B_KN);
    else if (L.amode == A_MK && L.bmode == B_KN)
        TLR_LAUNCH(A_MK, B_KN);
    else if (L.amode == A_MK && L.bmode == B_NK)
        TLR_LAUNCH(A_MK, B_NK);
    else
        return cudaErrorInvalidValue;
#undef TLR_LAUNCH
    return cudaGetLastError();
}

}  // namespace tlr
