// Tensor-core (tcgen05, sm_103a) grouped complex GEMM for the TLR contractions,
// same problem tables as the FP32 SIMT path (compress, expand, projection,
// adjoint).
//
// Arithmetic.  Every complex product C = A B is formed with three real
// products (3M): P1 = Ar Br, P2 = Ai Bi, P3 = (Ar + Ai)(Br + Bi), then
// Cr = P1 - P2, Ci = P3 - P1 - P2.  Every real product X Y runs in BF16 with
// a hi/lo split of both operands (x = hi + lo, hi = RN_bf16(x),
// lo = RN_bf16(x - hi)) and three tensor-core products hi*hi + hi*lo + lo*hi,
// all accumulated in FP32 in tensor memory (TMEM).  The dropped lo*lo term is
// below 2^-16 of |x||y|.
//
// Data movement.  A CTA owns one 128 x 128 output tile.  For each K chunk of
// 32 complex elements its 256 threads load the A and B sub-tiles from global
// memory (applying the row gather and the conjugation of the problem table),
// split them into six BF16 planes each (Re, Im, Re+Im; hi and lo) and store
// them in shared memory in the canonical K-major, no-swizzle layout of the
// tensor core: 8-row x 16-byte core matrices, 128 B apart along K (LBO) and
// 512 B apart along M/N (SBO).  One thread issues the 18 MMAs of the chunk
// (2 K-steps x 3 products x 3 split terms) and commits them to the stage's
// mbarrier; the other threads meanwhile fill the other stage.  Accumulators:
// P1, P2, P3 at TMEM columns 0, 128, 256 (512 columns allocated; one CTA per
// SM by shared-memory size).  The epilogue reads TMEM with tcgen05.ld and
// combines 3M.
//
// Every mbarrier wait is bounded; on timeout the CTA records TLR_ERR_TIMEOUT
// in the error word, stops issuing work, waits (bounded) for what it issued,
// frees its TMEM and exits.
#include <cuda_bf16.h>

#include "internal.h"

namespace tlr {

namespace {

constexpr int TM = 128, TN = 128, KC = 32, NTHR = 256, NSTAGE = 2;
constexpr int PLANE = TM * KC * 2;                  // bytes of one BF16 plane (128 rows x 32 k)
constexpr int STAGE = 12 * PLANE;                   // 6 A planes + 6 B planes = 96 KB
constexpr int SMEM_BYTES = NSTAGE * STAGE + 256;    // + barriers and the TMEM address
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_LIMIT = 1LL << 22;

// instruction descriptor: D f32, A bf16, B bf16, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
    d |= (uint64_t)(512u >> 4) << 32;   // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;             // descriptor version
    return d;                           // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem), "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// split 8 complex values into the six BF16 planes and store 16 B per plane
__device__ __forceinline__ void split_store(const float2 (&v)[8], char* plane0, int off) {
    uint32_t w[6][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        float x[3][2];
        x[0][0] = v[j].x;
        x[0][1] = v[j + 1].x;
        x[1][0] = v[j].y;
        x[1][1] = v[j + 1].y;
        x[2][0] = v[j].x + v[j].y;
        x[2][1] = v[j + 1].x + v[j + 1].y;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const __nv_bfloat162 hi = __floats2bfloat162_rn(x[p][0], x[p][1]);
            const float2 hf = __bfloat1622float2(hi);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(x[p][0] - hf.x, x[p][1] - hf.y);
            w[2 * p][j >> 1] = *reinterpret_cast<const uint32_t*>(&hi);
            w[2 * p + 1][j >> 1] = *reinterpret_cast<const uint32_t*>(&lo);
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        *reinterpret_cast<uint4*>(plane0 + q * PLANE + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// byte offset of (row r, k-group kg) in a K-major no-swizzle plane
__device__ __forceinline__ int core_off(int r, int kg) { return ((r >> 3) * (KC / 8) + kg) * 128 + (r & 7) * 16; }

template <int AM>
__device__ __forceinline__ void stage_a(char* st, const GTerm& t, int M, int m0, int k0, int kend) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int id = threadIdx.x + it * NTHR;
        const int r = id & (TM - 1), kg = id >> 7;
        const int m = m0 + r;
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + kg * 8 + j;
            float2 x = make_float2(0.f, 0.f);
            if (m < M && k < kend) {
                x = (AM == A_KM) ? t.A[(long long)k * t.lda + m] : t.A[(long long)m * t.lda + k];
                x.y *= t.sa;
            }
            v[j] = x;
        }
        split_store(v, st, core_off(r, kg));
    }
}

template <int BMD>
__device__ __forceinline__ void stage_b(char* st, const GTerm& t, int N, int n0, int k0, int kend) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int id = threadIdx.x + it * NTHR;
        const int r = id & (TN - 1), kg = id >> 7;
        const int n = n0 + r;
        float2 v[8];
        long long rowN = 0;
        if (BMD == B_NK && n < N) rowN = t.g ? t.g[n] : n;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + kg * 8 + j;
            float2 x = make_float2(0.f, 0.f);
            if (n < N && k < kend) {
                if (BMD == B_KN) {
                    const long long row = t.g ? t.g[k] : k;
                    x = t.B[row * t.ldb + n];
                } else {
                    x = t.B[rowN * t.ldb + k];
                }
                x.y *= t.sb;
            }
            v[j] = x;
        }
        split_store(v, st + 6 * PLANE, core_off(r, kg));
    }
}

template <int AM, int BMD>
__global__ void __launch_bounds__(NTHR, 1) k_cgemm_tc(const GProb* __restrict__ probs, int nsplit, int kchunk,
                                                      int epi, long long part_stride, int* err) {
    extern __shared__ __align__(1024) char smem[];
    const int prob = blockIdx.z / nsplit, chunk = blockIdx.z % nsplit;
    const GProb& P = probs[prob];
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    if (m0 >= P.M || n0 >= P.N) return;

    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + NSTAGE * STAGE + 64);
    int* abort_flag = reinterpret_cast<int*>(smem + NSTAGE * STAGE + 128);
    const int warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // flatten (term, k chunk) pairs
    int c = 0;  // chunks issued
    bool started = false;
    for (int ti = 0; ti < P.nt; ++ti) {
        const GTerm& t = P.t[ti];
        int kb = 0, ke = t.K;
        if (nsplit > 1) {
            kb = chunk * kchunk;
            ke = min(t.K, kb + kchunk);
        }
        for (int k0 = kb; k0 < ke; k0 += KC, ++c) {
            const int s = c & 1;
            char* st = smem + s * STAGE;
            if (c >= NSTAGE) {
                if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)(((c - NSTAGE) >> 1) & 1))) *abort_flag = 1;
            }
            __syncthreads();
            if (*abort_flag) break;
            stage_a<AM>(st, t, P.M, m0, k0, ke);
            stage_b<BMD>(st, t, P.N, n0, k0, ke);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(st), b0 = a0 + 6 * PLANE;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
                    for (int p = 0; p < 3; ++p) {
                        const uint32_t d = tmem + p * 128;
                        const uint32_t ah = a0 + (2 * p) * PLANE + ks * 256, al = ah + PLANE;
                        const uint32_t bh = b0 + (2 * p) * PLANE + ks * 256, bl = bh + PLANE;
                        mma_bf16(d, sdesc(ah), sdesc(bh), started ? 1u : 0u);
                        mma_bf16(d, sdesc(ah), sdesc(bl), 1u);
                        mma_bf16(d, sdesc(al), sdesc(bh), 1u);
                    }
                    started = true;
                }
                mma_commit(smem_u32(&bars[s]));
            }
            started = true;
        }
        if (*abort_flag) break;
    }

    // wait for the last commit of every stage still in flight
    bool ok = true;
    for (int cc = (c > NSTAGE ? c - NSTAGE : 0); cc < c; ++cc) {
        if (!mbar_wait(smem_u32(&bars[cc & 1]), (uint32_t)((cc >> 1) & 1))) ok = false;
    }
    if (!ok || *abort_flag) {
        if (threadIdx.x == 0) atomicExch(err, TLR_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();

    if (ok && !*abort_flag) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, columns half (w / 4)
        const int lg = warp & 3, ch = warp >> 2;
        const int m = m0 + lg * 32 + (threadIdx.x & 31);
        cf* C = P.C + (epi == EPI_PARTIAL ? chunk * part_stride : 0);
        const uint32_t lane_addr = tmem + ((uint32_t)(lg * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) {
            const int col = ch * 64 + cb * 16;
            float p1[16], p2[16], p3[16];
            if (c > 0) {
                tmem_ld16(lane_addr + col, p1);
                tmem_ld16(lane_addr + 128 + col, p2);
                tmem_ld16(lane_addr + 256 + col, p3);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) p1[j] = p2[j] = p3[j] = 0.f;
            }
            if (m < P.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + col + j;
                    if (n >= P.N) break;
                    const long long o = (long long)m * P.ldc + n;
                    cf v = make_float2(p1[j] - p2[j], p3[j] - p1[j] - p2[j]);
                    if (epi == EPI_SUB) {
                        const cf sv = P.S[o];
                        v.x -= sv.x;
                        v.y -= sv.y;
                    } else if (epi == EPI_ACCUM) {
                        const cf cv = C[o];
                        v.x += cv.x;
                        v.y += cv.y;
                    }
                    C[o] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

template <int AM, int BMD>
cudaError_t launch_tc(const GemmLaunch& L, dim3 grid, int kchunk, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc<AM, BMD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_cgemm_tc<AM, BMD><<<grid, NTHR, SMEM_BYTES, st>>>(L.d_probs, L.nsplit, kchunk, L.epi, L.part_stride, L.err);
    counted(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_tc(const GemmLaunch& L, cudaStream_t st) {
    if (L.nprob == 0 || L.maxM == 0 || L.maxN == 0) return cudaSuccess;
    if (!L.err) return cudaErrorInvalidValue;
    dim3 grid((L.maxN + TN - 1) / TN, (L.maxM + TM - 1) / TM, L.nprob * L.nsplit);
    const int kchunk = L.nsplit > 1 ? L.kchunk : 0;
    if (L.amode == A_KM && L.bmode == B_KN) return launch_tc<A_KM, B_KN>(L, grid, kchunk, st);
    if (L.amode == A_MK && L.bmode == B_KN) return launch_tc<A_MK, B_KN>(L, grid, kchunk, st);
    if (L.amode == A_MK && L.bmode == B_NK) return launch_tc<A_MK, B_NK>(L, grid, kchunk, st);
    return cudaErrorInvalidValue;
}

}  // namespace tlr
