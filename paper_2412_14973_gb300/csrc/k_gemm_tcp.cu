// Tensor-core GEMM on pre-packed operands, and the pack kernel that makes them.
//
// Packed format ("P-format") of an operand with R rows (the M or N index) and
// K columns (the contraction index): tiles of TR = 128 rows x 16 k; tile
// (rb, kc) starts at byte
// (rb * nkc + kc) * 4 * TR * 32 and holds four BF16 planes (Re hi, Re lo,
// Im hi, Im lo; x = hi + lo with hi = RN_bf16(x), lo = RN_bf16(x - hi)), each
// in the tensor core's canonical K-major, no-swizzle layout (8-row x 16-byte
// core matrices, 128 B apart along K, 256 B apart along rows).  Elements
// outside R x K are zero.  The pack applies the row gather and the
// conjugation of the operand, so a tile is exactly what a stage of the GEMM
// needs and is moved with one cp.async.bulk copy.
//
// The GEMM (4M complex products, 128 x 128 tile, 12 MMAs per 16-deep chunk)
// has one thread issuing the bulk copies of the A and B tiles of each chunk
// into a 3-stage ring with a transaction-count mbarrier,
// one thread issuing the MMAs, and eight warps for the epilogue.  Every wait
// is bounded (2 s of %globaltimer, grid-wide abort word).
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "reduce.h"

namespace tlr {

namespace {

// 128 x 128 tiles, 3 stages: about 97 KB of shared memory and 256 TMEM columns
// per CTA, so two CTAs share an SM and one's epilogue and set-up run while the
// other's MMAs keep the tensor core busy.
constexpr int TM = kPackTRA, TN = kPackTRB, KC = 16;
static_assert(TM == 128 && (TN == 128 || TN == 256), "tile shapes of the MMA and epilogue");
constexpr int NSTAGE = TN == 128 ? 3 : 4;
constexpr int CTAS_PER_SM = TN == 128 ? 2 : 1;
constexpr int TILE_A = 4 * TM * KC * 2;             // 16 KB
constexpr int TILE_B = 4 * TN * KC * 2;             // 16 KB (TN 128)
constexpr int STAGE = TILE_A + TILE_B;              // 32 KB (TN 128)
constexpr int CTRL_OFF = NSTAGE * STAGE;
constexpr int SMEM_BYTES = CTRL_OFF + 256 + 256;    // barriers etc. + problem descriptor
constexpr int NTHR = 320;                           // warps 0-7 epilogue, 8 copies, 9 MMAs
constexpr int WCOPY = 8, WMMA = 9;
constexpr uint32_t TMEM_COLS = 2 * TN;              // Cr at column 0, Ci at column TN
static_assert(CTAS_PER_SM * TMEM_COLS <= 512, "TMEM columns of the CTAs sharing an SM");
static_assert(8 * 32 * 17 * 8 <= NSTAGE * STAGE, "epilogue staging fits in the operand ring");
constexpr unsigned long long WAIT_NS = 2000000000ull;

constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* err,
                                          unsigned long long limit_ns = WAIT_NS) {
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u && (*err != 0 || now_ns() - t0 > limit_ns)) return false;
    }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
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

__device__ __forceinline__ int core_off(int r, int kg) { return ((r >> 3) * 2 + kg) * 128 + (r & 7) * 16; }

// ---------------------------------------------------------------------------
// pack
// ---------------------------------------------------------------------------
// One CTA packs 256 consecutive (padded) rows of one job over PACK_KG k-groups
// of 8: thread = row, so the strided source reads (k-major sources) and the
// 16-byte tile writes are both coalesced across a warp; row-contiguous
// sources are read 16 bytes at a time.  All index arithmetic is 32-bit and
// TR is a power of two.
constexpr int PACK_KG = 2;

__global__ void __launch_bounds__(256) k_pack(const PackJob* __restrict__ jobs) {
    const PackJob& J = jobs[blockIdx.y];
    const int nkc = (J.K + KC - 1) / KC;
    const int nrb = (J.R + J.TR - 1) / J.TR;
    const int r = blockIdx.x * 256 + threadIdx.x;
    if (r >= nrb * J.TR) return;
    const int kg_end = min(2 * nkc, (int)(blockIdx.z + 1) * PACK_KG);
    const int trs = 31 - __clz(J.TR);              // log2(TR)
    const int rb = r >> trs, rr = r & (J.TR - 1);
    const bool rv = r < J.R;
    const cf* rowp = nullptr;
    bool vec = false;
    if (rv && J.kcontig) {
        const long long row = J.g_row ? J.g_row[r] : r;
        rowp = J.src + row * J.ld;
        vec = ((reinterpret_cast<uintptr_t>(rowp) & 15) == 0);
    }
    const int plane = J.TR * KC * 2;
    char* const base = reinterpret_cast<char*>(J.dst) + (size_t)rb * nkc * 4 * plane;
    for (int kg2 = blockIdx.z * PACK_KG; kg2 < kg_end; ++kg2) {
        const int kc = kg2 >> 1, kg = kg2 & 1;
        const int k0 = kc * KC + kg * 8;
        float2 v[8];
        if (rv && J.kcontig && vec && k0 + 8 <= J.K) {
            const float4* q = reinterpret_cast<const float4*>(rowp + k0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 t = q[j];
                v[2 * j] = make_float2(t.x, t.y * J.sgn);
                v[2 * j + 1] = make_float2(t.z, t.w * J.sgn);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = k0 + j;
                float2 x = make_float2(0.f, 0.f);
                if (rv && k < J.K) {
                    if (J.kcontig) {
                        x = rowp[k];
                    } else {
                        const long long kr = J.g_k ? J.g_k[k] : k;
                        x = J.src[kr * J.ld + r];
                    }
                    x.y *= J.sgn;
                }
                v[j] = x;
            }
        }
        uint32_t w[4][4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const float x[2][2] = {{v[j].x, v[j + 1].x}, {v[j].y, v[j + 1].y}};
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const __nv_bfloat162 hi = __floats2bfloat162_rn(x[p][0], x[p][1]);
                const float2 hf = __bfloat1622float2(hi);
                const __nv_bfloat162 lo = __floats2bfloat162_rn(x[p][0] - hf.x, x[p][1] - hf.y);
                w[2 * p][j >> 1] = *reinterpret_cast<const uint32_t*>(&hi);
                w[2 * p + 1][j >> 1] = *reinterpret_cast<const uint32_t*>(&lo);
            }
        }
        char* tile = base + (size_t)kc * 4 * plane + core_off(rr, kg);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(tile + q * plane) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

// ---------------------------------------------------------------------------
// tpack: fused update of the factor products and both of their packings
// ---------------------------------------------------------------------------
// A CTA takes one row tile (TP_K rows of one block's gathered T~_i) and 128
// columns (n).  Phase 1 either reads the TP_K source rows of T coalesced
// along n (packing only: alpha == nullptr), or, for the update, reads the
// tile's current values from its own KN packing (one 16 KB packed tile: the
// carried products live in packed form between forward products, each
// update re-rounding them to the hi + lo pair) and the rows of T_p, applies
// T += alpha T_p; it keeps the tile in shared memory; phase 2 writes the KN
// packing (thread = (n, k-group of 8)); phase 3 the conjugated NK packing
// (thread = (k, n-group of 8), lanes along k).  Padding of the packed buffers
// (k >= K_i, rows >= ns) is zero from the buffer's creation and is never
// written.
constexpr int TP_K = kFuseRows, TP_N = 128, TP_LD = TP_N + 1;
constexpr int TP_KS = TP_K == 16 ? 4 : 5;   // log2(TP_K)
static_assert(kPackTRB == 128 && KC == 16 && (TP_K == 16 || TP_K == 32),
              "tpack writes 128-row, 16-deep B tiles, 16 or 32 rows per CTA");

__device__ __forceinline__ void split_store(char* dst, int plane, const float2* v, float sgn) {
    uint32_t w[4][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        const float x[2][2] = {{v[j].x, v[j + 1].x}, {v[j].y * sgn, v[j + 1].y * sgn}};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const __nv_bfloat162 hi = __floats2bfloat162_rn(x[p][0], x[p][1]);
            const float2 hf = __bfloat1622float2(hi);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(x[p][0] - hf.x, x[p][1] - hf.y);
            w[2 * p][j >> 1] = *reinterpret_cast<const uint32_t*>(&hi);
            w[2 * p + 1][j >> 1] = *reinterpret_cast<const uint32_t*>(&lo);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(dst + q * plane) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// The 8 complex values of k-group kg of one row of a 16-deep packed tile
// (src = the row's 16-byte group in plane 0): hi + lo of each part, the
// BF16 halves widened by moving their bits into the high half of an FP32 word.
__device__ __forceinline__ void unpack8(const char* src, float2* v) {
    constexpr int plane = 128 * 16 * 2;
    uint4 w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = *reinterpret_cast<const uint4*>(src + q * plane);
    const uint32_t* wr = reinterpret_cast<const uint32_t*>(&w[0]);
    const uint32_t* wl = reinterpret_cast<const uint32_t*>(&w[1]);
    const uint32_t* wi = reinterpret_cast<const uint32_t*>(&w[2]);
    const uint32_t* wm = reinterpret_cast<const uint32_t*>(&w[3]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t sh = (j & 1) * 16;
        v[j] = make_float2(__uint_as_float(((wr[j >> 1] >> sh) & 0xffffu) << 16) +
                               __uint_as_float(((wl[j >> 1] >> sh) & 0xffffu) << 16),
                           __uint_as_float(((wi[j >> 1] >> sh) & 0xffffu) << 16) +
                               __uint_as_float(((wm[j >> 1] >> sh) & 0xffffu) << 16));
    }
}

__global__ void __launch_bounds__(256) k_tpack(const TPackTile* __restrict__ tiles, cf* __restrict__ T,
                                               const cf* __restrict__ Tp, const double* __restrict__ alpha,
                                               int ns) {
    __shared__ float2 s[TP_K * TP_LD];
    const TPackTile& P = tiles[blockIdx.y];
    const int n0 = blockIdx.x * TP_N;
    const int nk = P.nk;
    const float a = alpha ? (float)alpha[0] : 0.f;
    constexpr int plane = 128 * 16 * 2;   // bytes of one BF16 plane of a 128 x 16 tile
    // phase 1 (source row indices staged first; four rows per thread in flight)
    __shared__ long long srow[TP_K];
    if (threadIdx.x < nk) srow[threadIdx.x] = (long long)P.g[P.k0 + threadIdx.x] * ns;
    __syncthreads();
    if (alpha) {
        // thread = (n, k-group of 8): four 16-byte loads (one per BF16 plane)
        // give 8 complex values of the tile, then the 8 rows of T_p at n
        static_assert(TP_K == 16, "the update reads one 16-deep packed tile");
        const int n = threadIdx.x & (TP_N - 1), kg = threadIdx.x >> 7;
        const int nkcK = (P.Ki + 15) >> 4;
        const char* src = reinterpret_cast<const char*>(P.kn) +
                          ((long long)(n0 >> 7) * nkcK + (P.k0 >> 4)) * 4 * plane + core_off(n, kg);
        float2 v[8];
        unpack8(src, v);
        const bool nv = n0 + n < ns;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int kk = kg * 8 + j;
            float2 t = v[j];
            if (kk < nk && nv && a != 0.f) {
                const float2 d = Tp[srow[kk] + n0 + n];
                t.x = fmaf(a, d.x, t.x);
                t.y = fmaf(a, d.y, t.y);
            }
            s[kk * TP_LD + n] = kk < nk ? t : make_float2(0.f, 0.f);
        }
    } else {
        const int n = threadIdx.x & (TP_N - 1), kq = threadIdx.x >> 7;
        const bool nv = n0 + n < ns;
#pragma unroll 1
        for (int kb = kq; kb < TP_K; kb += 8) {
            float2 t[4], d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int kk = kb + 2 * u;
                t[u] = d[u] = make_float2(0.f, 0.f);
                if (kk < nk && nv) {
                    const long long o = srow[kk] + n0 + n;
                    t[u] = T[o];
                    if (a != 0.f) d[u] = Tp[o];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int kk = kb + 2 * u;
                if (kk >= nk) continue;
                s[kk * TP_LD + n] = t[u];
            }
        }
    }
    __syncthreads();
    // phase 2: KN, rows n, k = factor index; nk rows of this tile in k-groups of 8
    {
        const int nkcK = (P.Ki + 15) >> 4;
        const int ngrp = (nk + 7) >> 3;
        for (int it = threadIdx.x; it < TP_N * ngrp; it += blockDim.x) {
            const int n = it & (TP_N - 1), kg = it >> 7;
            if (n0 + n >= ns) continue;
            float2 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int kk = kg * 8 + j;
                v[j] = kk < nk ? s[kk * TP_LD + n] : make_float2(0.f, 0.f);
            }
            const int k = P.k0 + kg * 8;   // multiple of 8
            const int nn = n0 + n;
            char* dst = reinterpret_cast<char*>(P.kn) + ((long long)(nn >> 7) * nkcK + (k >> 4)) * 4 * plane +
                        core_off(nn & 127, (k >> 3) & 1);
            split_store(dst, plane, v, 1.f);
        }
    }
    // phase 3: NK, rows = factor index, k = n; conjugated
    if (P.nk_dst) {
        const int nkcN = (ns + 15) >> 4;
        // lanes take consecutive rows: conflict-free shared reads, and 16-byte
        // stores 16 bytes apart in the packed tile
        for (int it = threadIdx.x; it < TP_K * (TP_N / 8); it += blockDim.x) {
            const int kk = it & (TP_K - 1), ng = it >> TP_KS;
            const int nb = n0 + ng * 8;
            if (kk >= nk || nb >= ns) continue;
            float2 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = nb + j < ns ? s[kk * TP_LD + ng * 8 + j] : make_float2(0.f, 0.f);
            const int r = P.k0 + kk;
            char* dst = reinterpret_cast<char*>(P.nk_dst) + ((long long)(r >> 7) * nkcN + (nb >> 4)) * 4 * plane +
                        core_off(r & 127, (nb >> 3) & 1);
            split_store(dst, plane, v, -1.f);
        }
    }
}

// ---------------------------------------------------------------------------
// rstep: fused residual step and both packings of the residual
// ---------------------------------------------------------------------------
// A CTA takes TP_K receiver rows (inside one block, every block a multiple of
// TP_K) and 128 columns: phase 1 either reads the FP32 rows of R left by a
// forward product (packing only), or, for the step, reads the tile from R's
// own KN packing (the residual is carried in packed form between forward
// products) with A1, A2 coalesced along n and applies it; it accumulates
// ||R||^2 and keeps the tile in shared memory; phase 2 writes the MK packing
// (rows = receivers, lanes along rows); phase 3 the KN packing (rows = n,
// k = receiver, lanes along n).

// Block of the 16-row residual tile starting at row r0: r0 / b for equal
// tiles, else the largest i with roff[i] <= r0 (every roff[i] is a multiple
// of TP_K, so the tile lies in it); rl0 = its first row in the block, bK =
// the block's size.
struct RTile {
    int blk, rl0, bK;
};
__device__ __forceinline__ RTile rtile(int r0, int b, const long long* roff, int nblk) {
    RTile t;
    if (roff) {
        int lo = 0, hi = nblk - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (roff[mid] <= r0)
                lo = mid;
            else
                hi = mid - 1;
        }
        t.blk = lo;
        t.rl0 = r0 - (int)roff[lo];
        t.bK = (int)(roff[lo + 1] - roff[lo]);
    } else {
        t.blk = r0 / b;
        t.rl0 = r0 - t.blk * b;
        t.bK = b;
    }
    return t;
}

__global__ void __launch_bounds__(256) k_rstep(cf* __restrict__ R, const cf* __restrict__ A1,
                                               const cf* __restrict__ A2, const double* __restrict__ alpha, int ns,
                                               int b, char* const* __restrict__ kn, char* const* __restrict__ mk,
                                               double* __restrict__ part, const long long* __restrict__ roff,
                                               int nblk) {
    __shared__ float2 s[TP_K * TP_LD];
    __shared__ double sh[32];
    constexpr int plane = 128 * 16 * 2;
    const int n0 = blockIdx.x * TP_N, r0 = blockIdx.y * TP_K;
    const RTile tl = rtile(r0, b, roff, nblk);
    const int blk = tl.blk, rl0 = tl.rl0, bK = tl.bK;
    const float a = alpha ? (float)alpha[0] : 0.f;
    const float a2 = alpha ? (float)(alpha[0] * alpha[0]) : 0.f;
    Acc acc;
    if (alpha) {
        // the step: the tile's current values from its own KN packing (one
        // 16-deep packed tile; thread = (n, k-group of 8)), then A1, A2
        const int n = threadIdx.x & (TP_N - 1), kg = threadIdx.x >> 7;
        const bool nv = n0 + n < ns;
        float2 v[8];
        unpack8(kn[blk] + ((long long)(n0 >> 7) * (bK >> 4) + (rl0 >> 4)) * 4 * plane + core_off(n, kg), v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int kk = kg * 8 + j;
            float2 r = v[j];
            if (nv) {
                if (a != 0.f) {
                    const long long o = (long long)(r0 + kk) * ns + n0 + n;
                    const float2 u = A1[o], w = A2[o];
                    r.x = fmaf(a2, w.x, fmaf(a, u.x, r.x));
                    r.y = fmaf(a2, w.y, fmaf(a, u.y, r.y));
                }
                acc.add(fmaf(r.x, r.x, r.y * r.y));
            }
            s[kk * TP_LD + n] = r;
        }
    } else {
        // packing only (after a forward product): the FP32 rows of R
        const int n = threadIdx.x & (TP_N - 1), kq = threadIdx.x >> 7;
        const bool nv = n0 + n < ns;
#pragma unroll 1
        for (int kb = kq; kb < TP_K; kb += 8) {
            float2 r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                r[q] = make_float2(0.f, 0.f);
                if (nv) r[q] = R[(long long)(r0 + kb + 2 * q) * ns + n0 + n];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = kb + 2 * q;
                if (nv) acc.add(fmaf(r[q].x, r[q].x, r[q].y * r[q].y));
                s[kk * TP_LD + n] = r[q];
            }
        }
    }
    if (part) {
        const double t = block_sum(acc.val(), sh);   // includes the __syncthreads phase 2 needs
        if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
    } else {
        __syncthreads();
    }
    // phase 2: MK, rows = receivers of block blk, k = n
    {
        const int nkcN = (ns + 15) >> 4;
        char* const base = mk[blk];
        for (int it = threadIdx.x; it < TP_K * (TP_N / 8); it += blockDim.x) {
            const int kk = it & (TP_K - 1), ng = it >> TP_KS;
            const int nb = n0 + ng * 8;
            if (nb >= ns) continue;
            float2 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = nb + j < ns ? s[kk * TP_LD + ng * 8 + j] : make_float2(0.f, 0.f);
            const int rl = rl0 + kk;
            char* dst = base + ((long long)(rl >> 7) * nkcN + (nb >> 4)) * 4 * plane + core_off(rl & 127, (nb >> 3) & 1);
            split_store(dst, plane, v, 1.f);
        }
    }
    // phase 3: KN, rows = n, k = receiver of block blk
    {
        const int nkcK = bK >> 4;
        char* const base = kn[blk];
        for (int it = threadIdx.x; it < TP_N * (TP_K / 8); it += blockDim.x) {
            const int n = it & (TP_N - 1), kg = it >> 7;
            const int nn = n0 + n;
            if (nn >= ns) continue;
            float2 v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = s[(kg * 8 + j) * TP_LD + n];
            const int k = rl0 + kg * 8;
            char* dst = base + ((long long)(nn >> 7) * nkcK + (k >> 4)) * 4 * plane + core_off(nn & 127, (k >> 3) & 1);
            split_store(dst, plane, v, 1.f);
        }
    }
}

// The six line-search inner products Re<R,R>, Re<R,A1>, Re<R,A2>, Re<A1,A1>,
// Re<A1,A2>, Re<A2,A2> over rstep's 16-row x 128-column tiles, with R read
// from its KN packing (the form it is carried in between forward products)
// and A1, A2 in FP32; products of four elements summed in FP32 before each
// compensated add.  A fixed grid walks the tiles in a fixed order and leaves
// one partial per dot and CTA (few partials for the one-block finaliser).
__global__ void __launch_bounds__(256) k_dots6p(char* const* __restrict__ kn, const cf* __restrict__ A1,
                                                const cf* __restrict__ A2, int ns, int nr, int b,
                                                const long long* __restrict__ roff, int nblk,
                                                double* __restrict__ part) {
    __shared__ double sh[32];
    constexpr int plane = 128 * 16 * 2;
    const int gx = (ns + TP_N - 1) / TP_N;
    const long long ntiles = (long long)gx * (nr / TP_K);
    const int n = threadIdx.x & (TP_N - 1), kg = threadIdx.x >> 7;
    Acc acc[6];
    for (long long tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const int n0 = (int)(tt % gx) * TP_N, r0 = (int)(tt / gx) * TP_K;
        if (n0 + n >= ns) continue;
        const RTile tl = rtile(r0, b, roff, nblk);
        float2 v[8];
        unpack8(kn[tl.blk] + ((long long)(n0 >> 7) * (tl.bK >> 4) + (tl.rl0 >> 4)) * 4 * plane + core_off(n, kg), v);
        float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long long o = (long long)(r0 + kg * 8 + j) * ns + n0 + n;
            const float2 r = v[j], x = A1[o], c = A2[o];
            g[0] += fmaf(r.x, r.x, r.y * r.y);
            g[1] += fmaf(r.x, x.x, r.y * x.y);
            g[2] += fmaf(r.x, c.x, r.y * c.y);
            g[3] += fmaf(x.x, x.x, x.y * x.y);
            g[4] += fmaf(x.x, c.x, x.y * c.y);
            g[5] += fmaf(c.x, c.x, c.y * c.y);
            if ((j & 3) == 3) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    acc[k].add(g[k]);
                    g[k] = 0.f;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double t = block_sum(acc[k].val(), sh);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * 6 + k] = t;
    }
}

// ---------------------------------------------------------------------------
// GEMM on packed operands
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHR, CTAS_PER_SM) k_cgemm_tcp(const PProb* __restrict__ probs, int nsplit, int kchunk,
                                                       int epi, long long part_stride, int* err) {
    extern __shared__ __align__(1024) char smem[];
    const int prob = blockIdx.z / nsplit, chunk = blockIdx.z % nsplit;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    {
        const PProb& Pg = probs[prob];
        if (m0 >= Pg.M || n0 >= Pg.N) return;
        if (*(volatile int*)err != 0) return;
    }
    PProb& P = *reinterpret_cast<PProb*>(smem + CTRL_OFF + 256);
    static_assert(sizeof(PProb) <= 256, "descriptor slot");
    {
        const int* src = reinterpret_cast<const int*>(&probs[prob]);
        int* dst = reinterpret_cast<int*>(&P);
        for (int i = threadIdx.x; i < (int)(sizeof(PProb) / 4); i += blockDim.x) dst[i] = src[i];
    }
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + CTRL_OFF);
    uint64_t* empty = full + NSTAGE;
    uint64_t* done = empty + NSTAGE;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == WMMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // the chunk list: per term, K chunks [kb, ke) of 16 (kb a multiple of 16)
    int C = 0;
    for (int ti = 0; ti < P.nt; ++ti) {
        int kb = 0, ke = P.t[ti].K;
        if (nsplit > 1) {
            kb = chunk * kchunk;
            ke = min(P.t[ti].K, kb + kchunk);
        }
        if (ke > kb) C += (ke - kb + KC - 1) / KC;
    }

    if (warp == WCOPY && lane == 0) {
        // ---------------- bulk copies ----------------
        int c = 0;
        for (int ti = 0; ti < P.nt && !*abort_flag; ++ti) {
            const PTerm& t = P.t[ti];
            int kb = 0, ke = t.K;
            if (nsplit > 1) {
                kb = chunk * kchunk;
                ke = min(t.K, kb + kchunk);
            }
            const int nkcA = (t.K + KC - 1) / KC, nkcB = nkcA;
            const char* abase = reinterpret_cast<const char*>(t.A) + (long long)(m0 / TM) * nkcA * TILE_A;
            const char* bbase = reinterpret_cast<const char*>(t.B) + (long long)(n0 / TN) * nkcB * TILE_B;
            for (int k0 = kb; k0 < ke; k0 += KC, ++c) {
                const int s = c % NSTAGE;
                if (c >= NSTAGE) {
                    if (!mbar_wait(smem_u32(&empty[s]), (uint32_t)(((c / NSTAGE) - 1) & 1), err)) {
                        *abort_flag = 1;
                        break;
                    }
                }
                const uint32_t fb = smem_u32(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE)
                             : "memory");
                const int kc = k0 / KC;
                const uint32_t dst = smem_u32(smem + s * STAGE);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                    "l"(abase + (long long)kc * TILE_A), "r"(TILE_A), "r"(fb)
                    : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        dst + TILE_A),
                    "l"(bbase + (long long)kc * TILE_B), "r"(TILE_B), "r"(fb)
                    : "memory");
            }
        }
    } else if (warp == WMMA && lane == 0) {
        // ---------------- MMA issuer ----------------
        for (int c = 0; c < C; ++c) {
            const int s = c % NSTAGE;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((c / NSTAGE) & 1), err)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + TILE_A;
            constexpr int PA = TILE_A / 4, PB = TILE_B / 4;
            const uint64_t arh = sdesc(a0), arl = sdesc(a0 + PA), aih = sdesc(a0 + 2 * PA), ail = sdesc(a0 + 3 * PA);
            const uint64_t brh = sdesc(b0), brl = sdesc(b0 + PB), bih = sdesc(b0 + 2 * PB), bil = sdesc(b0 + 3 * PB);
            const uint32_t dr = tmem, di = tmem + TN;
            const uint32_t first = c > 0 ? 1u : 0u;
            mma_bf16(dr, arh, brh, IDESC, first);
            mma_bf16(dr, arh, brl, IDESC, 1u);
            mma_bf16(dr, arl, brh, IDESC, 1u);
            mma_bf16(dr, aih, bih, IDESC_NEG_A, 1u);
            mma_bf16(dr, aih, bil, IDESC_NEG_A, 1u);
            mma_bf16(dr, ail, bih, IDESC_NEG_A, 1u);
            mma_bf16(di, arh, bih, IDESC, first);
            mma_bf16(di, arh, bil, IDESC, 1u);
            mma_bf16(di, arl, bih, IDESC, 1u);
            mma_bf16(di, aih, brh, IDESC, 1u);
            mma_bf16(di, aih, brl, IDESC, 1u);
            mma_bf16(di, ail, brh, IDESC, 1u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    }

    // ---------------- epilogue (warps 0-7) ----------------
    // warp w reads TMEM lanes 32 (w % 4) .. +31 and columns [TN/2 (w / 4), +TN/2)
    bool ok = true;
    if (warp < 8 && C > 0) ok = mbar_wait(smem_u32(done), 0u, err);
    if (!ok || *abort_flag) {
        if (threadIdx.x == 0 || !ok) atomicExch(err, TLR_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 8 && ok && !*abort_flag && epi == EPI_PACKNK) {
        // Row m goes to one row of a packed NK operand: 16 columns are one
        // 16-deep chunk there (two 16-byte groups per BF16 plane).  Lanes hold
        // consecutive rows, which are 16 bytes apart in the packed tile.
        const int lg = warp & 3, ch = warp >> 2;
        const uint32_t lane_addr = tmem + ((uint32_t)(lg * 32) << 16);
        const int m = m0 + lg * 32 + lane;
        constexpr int plane = 128 * 16 * 2;
#pragma unroll 1
        for (int cb = 0; cb < TN / 32; ++cb) {
            const int col = ch * (TN / 2) + cb * 16;
            if (n0 + col >= P.N) break;
            float pr[16], pi[16];
            if (C > 0) {
                tmem_ld16(lane_addr + col, pr);
                tmem_ld16(lane_addr + TN + col, pi);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) pr[j] = pi[j] = 0.f;
            }
            if (m < P.M) {
                const int n = n0 + col;
                float2 v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = n + j < P.N ? make_float2(pr[j], pi[j]) : make_float2(0.f, 0.f);
                char* d = P.rowptr[m] + (long long)(n >> 4) * 4 * plane;
                split_store(d, plane, v, 1.f);
                split_store(d + 128, plane, v + 8, 1.f);
            }
        }
    } else if (warp < 8 && ok && !*abort_flag) {
        // Each warp drains 32 rows x 16 columns at a time: tcgen05.ld gives a
        // thread one row; the block is transposed through shared memory (the
        // operand ring is idle once the last MMA has completed) so that each
        // store instruction writes four full 128-byte row segments.
        const int lg = warp & 3, ch = warp >> 2;
        cf* Cp = P.C + (epi == EPI_PARTIAL ? chunk * part_stride : 0);
        const uint32_t lane_addr = tmem + ((uint32_t)(lg * 32) << 16);
        cf* stg = reinterpret_cast<cf*>(smem) + warp * (32 * 17);   // 32 rows x 16 (+1 pad)
        const int rsub = lane >> 3, q = lane & 7;                   // write phase: row group, 16-B chunk
#pragma unroll 1
        for (int cb = 0; cb < TN / 32; ++cb) {
            const int col = ch * (TN / 2) + cb * 16;
            if (n0 + col >= P.N) break;
            float pr[16], pi[16];
            if (C > 0) {
                tmem_ld16(lane_addr + col, pr);
                tmem_ld16(lane_addr + TN + col, pi);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) pr[j] = pi[j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = make_float2(pr[j], pi[j]);
            __syncwarp();
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                const int r = j2 * 4 + rsub;
                const int m = m0 + lg * 32 + r;
                const int n = n0 + col + 2 * q;
                if (m < P.M && n < P.N) {
                    const long long o = (long long)m * P.ldc + n;
                    cf v0 = stg[r * 17 + 2 * q], v1 = stg[r * 17 + 2 * q + 1];
                    const bool two = n + 1 < P.N;
                    if (epi == EPI_SUB) {
                        const cf s0 = P.S[o];
                        v0.x -= s0.x;
                        v0.y -= s0.y;
                        if (two) {
                            const cf s1 = P.S[o + 1];
                            v1.x -= s1.x;
                            v1.y -= s1.y;
                        }
                    } else if (epi == EPI_ACCUM) {
                        const cf c0 = Cp[o];
                        v0.x += c0.x;
                        v0.y += c0.y;
                        if (two) {
                            const cf c1 = Cp[o + 1];
                            v1.x += c1.x;
                            v1.y += c1.y;
                        }
                    }
                    if (two && ((reinterpret_cast<uintptr_t>(Cp + o) & 15) == 0)) {
                        *reinterpret_cast<float4*>(Cp + o) = make_float4(v0.x, v0.y, v1.x, v1.y);
                    } else {
                        Cp[o] = v0;
                        if (two) Cp[o + 1] = v1;
                    }
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == WMMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Self-test of the contraction kernels' bounded barrier wait: one thread
// waits on an mbarrier that nothing arrives at; the wait gives up after
// limit_ns and the kernel records TLR_ERR_TIMEOUT (and the nanoseconds it
// waited) for the host.
__global__ void k_wait_selftest(int* status, unsigned long long limit_ns, unsigned long long* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const unsigned long long t0 = now_ns();
    const bool ok = mbar_wait(b, 0u, status, limit_ns);
    *waited_ns = now_ns() - t0;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
    *status = ok ? TLR_OK : TLR_ERR_TIMEOUT;
}

}  // namespace

long long packed_bytes(long long R, long long K, int TR) {
    const long long nkc = (K + KC - 1) / KC, nrb = (R + TR - 1) / TR;
    return nrb * nkc * 4LL * TR * KC * 2;
}

// max_items encodes the largest job: (padded rows << 32) | k-groups
cudaError_t pack_operands(const PackJob* jobs, int njobs, long long max_items, cudaStream_t st) {
    if (njobs == 0 || max_items == 0) return cudaSuccess;
    const long long rows = max_items >> 32, kgs = max_items & 0xffffffffLL;
    dim3 grid((unsigned)((rows + 255) / 256), (unsigned)njobs, (unsigned)((kgs + PACK_KG - 1) / PACK_KG));
    k_pack<<<grid, 256, 0, st>>>(jobs);
    counted(1);
    return cudaGetLastError();
}

cudaError_t tpack(const TPackTile* d_tiles, int ntiles, cf* T, const cf* Tp, const double* alpha, int ns,
                  cudaStream_t st) {
    if (ntiles == 0 || ns == 0) return cudaSuccess;
    dim3 grid((unsigned)((ns + TP_N - 1) / TP_N), (unsigned)ntiles);
    k_tpack<<<grid, 256, 0, st>>>(d_tiles, T, Tp, alpha, ns);
    counted(1);
    return cudaGetLastError();
}

long long rstep_ctas(int nr, int ns) { return (long long)((ns + TP_N - 1) / TP_N) * (nr / TP_K); }

cudaError_t rstep(cf* R, const cf* A1, const cf* A2, const double* alpha, int nr, int ns, int b, char* const* kn,
                  char* const* mk, double* part, cudaStream_t st, const long long* roff, int nblk) {
    if (nr == 0 || ns == 0) return cudaSuccess;
    if (nr % TP_K != 0) return cudaErrorInvalidValue;
    if (!roff && (b <= 0 || b % TP_K != 0 || nr % b != 0)) return cudaErrorInvalidValue;
    if (roff && nblk <= 0) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((ns + TP_N - 1) / TP_N), (unsigned)(nr / TP_K));
    k_rstep<<<grid, 256, 0, st>>>(R, A1, A2, alpha, ns, b, kn, mk, part, roff, nblk);
    counted(1);
    return cudaGetLastError();
}

cudaError_t dots6_packed(char* const* kn, const cf* A1, const cf* A2, int nr, int ns, int b, double* part,
                         cudaStream_t st, const long long* roff, int nblk) {
    if (nr == 0 || ns == 0) return cudaSuccess;
    if (nr % TP_K != 0) return cudaErrorInvalidValue;
    if (!roff && (b <= 0 || b % TP_K != 0 || nr % b != 0)) return cudaErrorInvalidValue;
    if (roff && nblk <= 0) return cudaErrorInvalidValue;
    k_dots6p<<<kRedBlocks, 256, 0, st>>>(kn, A1, A2, ns, nr, b, roff, nblk, part);
    counted(1);
    return cudaGetLastError();
}

cudaError_t wait_selftest(int* status, unsigned long long limit_ns, unsigned long long* waited_ns,
                          cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(status, limit_ns, waited_ns);
    counted(1);
    return cudaGetLastError();
}

cudaError_t gemm_tcp_prepare() {
    return cudaFuncSetAttribute(k_cgemm_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t gemm_tcp(const GemmLaunch& L, cudaStream_t st) {
    if (L.nprob == 0 || L.maxM == 0 || L.maxN == 0) return cudaSuccess;
    if (!L.err || !L.d_pprobs) return cudaErrorInvalidValue;
    dim3 grid((L.maxN + TN - 1) / TN, (L.maxM + TM - 1) / TM, L.nprob * L.nsplit);
    const int kchunk = L.nsplit > 1 ? L.kchunk : 0;
    k_cgemm_tcp<<<grid, NTHR, SMEM_BYTES, st>>>(L.d_pprobs, L.nsplit, kchunk, L.epi, L.part_stride, L.err);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
