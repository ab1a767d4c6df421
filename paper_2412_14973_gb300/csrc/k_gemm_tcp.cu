// Tensor-core GEMM on pre-packed operands, and the pack kernel that makes them.
//
// Packed format ("P-format") of an operand with R rows (the M or N index) and
// K columns (the contraction index): tiles of TR = 128 rows x 16 k, 16 KB
// each; tile (rb, kc) starts at byte (rb * nkc + kc) * 16384.  Two formats:
//   BF16x3: four BF16 planes (Re hi, Re lo, Im hi, Im lo; x = hi + lo with
//     hi = RN_bf16(x), lo = RN_bf16(x - hi)) of 4 KB;
//   TF32: two planes (Re, Im) of 8 KB, FP32 words rounded to TF32 (RN, ties
//     away from zero: the low 13 mantissa bits zero, so the tensor core's
//     handling of them does not matter).
// Each plane is in the tensor core's canonical K-major, no-swizzle layout:
// 8-row x 16-byte core matrices, 128 B apart along K, 256 B (BF16, two per
// 16 k) or 512 B (TF32, four per 16 k) apart along rows.  Elements outside
// R x K are zero.  The pack applies the row gather and the conjugation of the
// operand, so a tile is exactly what a stage of the GEMM needs and is moved
// with one cp.async.bulk copy.
//
// The GEMM (4M complex products, 128 x 128 tile, 12 BF16 MMAs of K 16 or 8
// TF32 MMAs of K 8 per 16-deep chunk)
// has one thread issuing the bulk copies of the A and B tiles of each chunk
// into a 3-stage ring with a transaction-count mbarrier,
// one thread issuing the MMAs, and eight warps for the epilogue.  Every wait
// is bounded (2 s of %globaltimer, grid-wide abort word).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

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

// instruction descriptors: FP32 accumulator (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: 1 = BF16, 2 = TF32), N / 8 (bits 17-22), M / 16 (bits 24-28),
// bit 13 negates A
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);
constexpr uint32_t IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_TF32_NEG_A = IDESC_TF32 | (1u << 13);
constexpr int PK_TILE = 16384;   // bytes of one packed 128 x 16 tile (both formats)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major no-swizzle: leading byte offset
// 128 (core matrices adjacent along K), stride byte offset sbo (adjacent
// along M / N: 256 for the BF16 planes, 512 for the TF32 planes)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo = 256u) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
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

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
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

// byte offset of row r's first 16-byte group (k 0 .. 7 for BF16, k 0 .. 3
// for TF32) inside a packed tile's first plane
__device__ __forceinline__ int row_off(int fmt, int r) {
    return (r >> 3) * (fmt == kFmtTF32 ? 512 : 256) + (r & 7) * 16;
}

// TF32 bit pattern of x rounded to nearest, ties away from zero
__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// The 8 complex values of k-group kg (k = 8 kg .. 8 kg + 7) of one row of a
// packed tile, row = tile + row_off(fmt, r); the imaginary parts times sgn.
__device__ __forceinline__ void pk_store8(char* row, int fmt, int kg, const float2* v, float sgn) {
    if (fmt == kFmtTF32) {
        uint32_t re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            re[j] = tf32_rna(v[j].x);
            im[j] = tf32_rna(v[j].y * sgn);
        }
        char* p = row + kg * 256;
        *reinterpret_cast<uint4*>(p) = make_uint4(re[0], re[1], re[2], re[3]);
        *reinterpret_cast<uint4*>(p + 128) = make_uint4(re[4], re[5], re[6], re[7]);
        *reinterpret_cast<uint4*>(p + 8192) = make_uint4(im[0], im[1], im[2], im[3]);
        *reinterpret_cast<uint4*>(p + 8192 + 128) = make_uint4(im[4], im[5], im[6], im[7]);
        return;
    }
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
    char* dst = row + kg * 128;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(dst + q * 4096) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// The inverse: the 8 complex values of k-group kg of a packed row (BF16:
// hi + lo of each part, the BF16 halves widened by moving their bits into the
// high half of an FP32 word; TF32: the stored words).
__device__ __forceinline__ void pk_load8(const char* row, int fmt, int kg, float2* v) {
    if (fmt == kFmtTF32) {
        const char* p = row + kg * 256;
        const uint4 r0 = *reinterpret_cast<const uint4*>(p), r1 = *reinterpret_cast<const uint4*>(p + 128);
        const uint4 i0 = *reinterpret_cast<const uint4*>(p + 8192),
                    i1 = *reinterpret_cast<const uint4*>(p + 8192 + 128);
        const uint32_t re[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const uint32_t im[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
        return;
    }
    const char* src = row + kg * 128;
    uint4 w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = *reinterpret_cast<const uint4*>(src + q * 4096);
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
    if (J.TR != 128) return;   // both formats are laid out on 128-row tiles
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
        pk_store8(base + (size_t)kc * 4 * plane + row_off(J.fmt, rr), J.fmt, kg, v, 1.f);
    }
}

// ---------------------------------------------------------------------------
// tpack: fused update of the factor products and both of their packings
// ---------------------------------------------------------------------------
// A tile is TP_K = 16 rows of one block's gathered T~_i by 128 columns (n);
// thread = (n, k-group of 8).  A thread reads its 8 values either from the
// rows of T (packing only: alpha == nullptr; coalesced along n) or, for the
// update, from the tile's own KN packing (the carried products live in packed
// form between forward products, each update re-rounding them to the hi + lo
// pair) plus the rows of T_p, applying T += alpha T_p; it writes them back to
// the KN packing as they are (the same 8 k of row n), then an 8 x 8 transpose
// across each group of 8 lanes (warp shuffles) gives every lane 8
// consecutive n of one row k for the conjugated NK packing.  No shared
// memory: beside two contraction CTAs an SM then has room for as many pass
// CTAs as registers allow.  Padding of the packed buffers (k >= K_i, rows >=
// ns) is zero from the buffer's creation; whole padding groups are never
// written, and the padding inside a written group is written as zeros.
constexpr int TP_K = kFuseRows, TP_N = 128;
static_assert(kPackTRB == 128 && KC == 16 && TP_K == 16,
              "the passes take 16-deep, 128-row packed tiles with two k-groups of 8");

// 8 x 8 transpose across the 8 lanes of each aligned lane group: lane i holds
// a[j] = M[i][j] before and M[j][i] after (three butterfly exchanges).
__device__ __forceinline__ void transpose8(float2* a) {
    const int i = threadIdx.x & 7;
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
        const bool upper = (i & s) != 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j & s) continue;
            const float2 send = upper ? a[j] : a[j + s];
            float2 recv;
            recv.x = __shfl_xor_sync(0xffffffffu, send.x, s);
            recv.y = __shfl_xor_sync(0xffffffffu, send.y, s);
            if (upper)
                a[j] = recv;
            else
                a[j + s] = recv;
        }
    }
}

__global__ void __launch_bounds__(256) k_tpack(const TPackTile* __restrict__ tiles, cf* __restrict__ T,
                                               const cf* __restrict__ Tp, const double* __restrict__ alpha,
                                               int ns, int gx, long long ntiles) {
    const float a = alpha ? (float)alpha[0] : 0.f;
    constexpr int plane = 128 * 16 * 2;   // bytes of one BF16 plane of a 128 x 16 tile
    const int n = threadIdx.x & (TP_N - 1), kg = threadIdx.x >> 7;
    // tile tt = (row tile tt / gx, columns (tt % gx) * 128 ..): a capped grid
    // walks them in launch order
    for (long long tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const TPackTile& P = tiles[tt / gx];
        const int n0 = (int)(tt % gx) * TP_N;
        const int nk = P.nk;
        const int nkcK = (P.Ki + 15) >> 4;
        const bool nv = n0 + n < ns;
        float2 t[8];
        if (alpha) {
            // four 16-byte loads (one per BF16 plane) give the thread's 8
            // values of the tile, then the 8 rows of T_p at n
            const char* src = reinterpret_cast<const char*>(P.kn) +
                              ((long long)(n0 >> 7) * nkcK + (P.k0 >> 4)) * 4 * plane + row_off(P.fmt, n);
            pk_load8(src, P.fmt, kg, t);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int kk = kg * 8 + j;
                if (kk < nk && nv && a != 0.f) {
                    const float2 d = Tp[(long long)P.g[P.k0 + kk] * ns + n0 + n];
                    t[j].x = fmaf(a, d.x, t[j].x);
                    t[j].y = fmaf(a, d.y, t[j].y);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int kk = kg * 8 + j;
                t[j] = (kk < nk && nv) ? T[(long long)P.g[P.k0 + kk] * ns + n0 + n] : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (kg * 8 + j >= nk || !nv) t[j] = make_float2(0.f, 0.f);
        // KN: rows n, k = factor index (this thread's own 8 values)
        if (kg * 8 < nk && nv) {
            const int k = P.k0 + kg * 8;   // multiple of 8
            const int nn = n0 + n;
            char* dst = reinterpret_cast<char*>(P.kn) + ((long long)(nn >> 7) * nkcK + (k >> 4)) * 4 * plane +
                        row_off(P.fmt, nn & 127);
            pk_store8(dst, P.fmt, (k >> 3) & 1, t, 1.f);
        }
        // NK: rows = factor index, k = n; conjugated.  After the transpose
        // lane i of a group holds row kg * 8 + i at the group's 8 columns.
        if (P.nk_dst) {
            transpose8(t);
            const int kk = kg * 8 + (threadIdx.x & 7);
            const int nb = n0 + (n & ~7);
            if (kk < nk && nb < ns) {
                const int nkcN = (ns + 15) >> 4;
                const int r = P.k0 + kk;
                char* dst = reinterpret_cast<char*>(P.nk_dst) + ((long long)(r >> 7) * nkcN + (nb >> 4)) * 4 * plane +
                            row_off(P.fmt, r & 127);
                pk_store8(dst, P.fmt, (nb >> 3) & 1, t, -1.f);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// rstep: fused residual step and both packings of the residual
// ---------------------------------------------------------------------------
// A tile is TP_K = 16 receiver rows (inside one block, every block a
// multiple of TP_K) by 128 columns; thread = (n, k-group of 8 rows).  A
// thread reads its 8 values either from the FP32 rows of R left by a forward
// product (packing only), or, for the step, from R's own KN packing (the
// residual is carried in packed form between forward products) with A1, A2
// coalesced along n, and applies the step; it accumulates ||R||^2, writes its
// 8 values to the KN packing (rows = n, k = receiver) as they are, and after
// an 8 x 8 transpose across each group of 8 lanes, 8 consecutive n of one
// receiver row to the MK packing (rows = receivers, k = n).  No shared
// memory besides the block sum.

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
                                               int nblk, int fmt, int gx, long long ntiles) {
    __shared__ double sh[32];
    constexpr int plane = 128 * 16 * 2;
    const float a = alpha ? (float)alpha[0] : 0.f;
    const float a2 = alpha ? (float)(alpha[0] * alpha[0]) : 0.f;
    const int n = threadIdx.x & (TP_N - 1), kg = threadIdx.x >> 7;
    const int nkcN = (ns + 15) >> 4;
    // tile tt = (rows (tt / gx) * 16 .., columns (tt % gx) * 128 ..): a capped
    // grid walks them in launch order; tile tt's partial of ||R||^2 is part[tt]
    for (long long tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const int n0 = (int)(tt % gx) * TP_N, r0 = (int)(tt / gx) * TP_K;
        const RTile tl = rtile(r0, b, roff, nblk);
        const int blk = tl.blk, rl0 = tl.rl0, bK = tl.bK;
        const bool nv = n0 + n < ns;
        Acc acc;
        float2 r[8];
        if (alpha) {
            // the step: the thread's 8 values from the tile's KN packing (one
            // 16-deep packed tile), then A1, A2
            pk_load8(kn[blk] + ((long long)(n0 >> 7) * (bK >> 4) + (rl0 >> 4)) * 4 * plane + row_off(fmt, n), fmt,
                     kg, r);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (nv) {
                    if (a != 0.f) {
                        const long long o = (long long)(r0 + kg * 8 + j) * ns + n0 + n;
                        const float2 u = A1[o], w = A2[o];
                        r[j].x = fmaf(a2, w.x, fmaf(a, u.x, r[j].x));
                        r[j].y = fmaf(a2, w.y, fmaf(a, u.y, r[j].y));
                    }
                    acc.add(fmaf(r[j].x, r[j].x, r[j].y * r[j].y));
                }
            }
        } else {
            // packing only (after a forward product): the FP32 rows of R
#pragma unroll
            for (int j = 0; j < 8; ++j)
                r[j] = nv ? R[(long long)(r0 + kg * 8 + j) * ns + n0 + n] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (nv) acc.add(fmaf(r[j].x, r[j].x, r[j].y * r[j].y));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (!nv) r[j] = make_float2(0.f, 0.f);
        if (part) {
            const double t = block_sum(acc.val(), sh);
            if (threadIdx.x == 0) part[tt] = t;
        }
        // KN: rows = n, k = receiver of block blk (this thread's own 8 values)
        if (nv) {
            const int nn = n0 + n, k = rl0 + kg * 8;
            char* dst = kn[blk] + ((long long)(nn >> 7) * (bK >> 4) + (k >> 4)) * 4 * plane + row_off(fmt, nn & 127);
            pk_store8(dst, fmt, (k >> 3) & 1, r, 1.f);
        }
        // MK: rows = receivers of block blk, k = n.  After the transpose lane
        // i of a group holds receiver row kg * 8 + i at the group's 8 columns.
        transpose8(r);
        const int nb = n0 + (n & ~7);
        if (nb < ns) {
            const int rl = rl0 + kg * 8 + (threadIdx.x & 7);
            char* dst = mk[blk] + ((long long)(rl >> 7) * nkcN + (nb >> 4)) * 4 * plane + row_off(fmt, rl & 127);
            pk_store8(dst, fmt, (nb >> 3) & 1, r, 1.f);
        }
    }
}

// The six line-search inner products Re<R,R>, Re<R,A1>, Re<R,A2>, Re<A1,A1>,
// Re<A1,A2>, Re<A2,A2> over rstep's 16-row x 128-column tiles, with R read
// from its KN packing (the form it is carried in between forward products)
// and A1, A2 in FP32; products of four elements summed in FP32 before each
// compensated add.  A fixed grid walks the tiles in a fixed order and leaves
// one partial per dot and CTA (few partials for the one-block finaliser).
__global__ void __maxnreg__(48) k_dots6p(char* const* __restrict__ kn, const cf* __restrict__ A1,
                                                const cf* __restrict__ A2, int ns, int nr, int b,
                                                const long long* __restrict__ roff, int nblk,
                                                double* __restrict__ part, int fmt) {
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
        pk_load8(kn[tl.blk] + ((long long)(n0 >> 7) * (tl.bK >> 4) + (tl.rl0 >> 4)) * 4 * plane + row_off(fmt, n), fmt,
                 kg, v);
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
// Epilogue of one 128 x TN output tile (warps 0-7): warp w reads TMEM lanes
// 32 (w % 4) .. +31 and columns [TN/2 (w / 4), +TN/2) of the accumulator
// pair at tmem (Cr at column 0, Ci at column TN; zeros when !have, a tile
// without K chunks) and writes the tile to its destination: a packed NK
// operand (EPI_PACKNK), or rows of C (store, subtract S, accumulate, split-K
// partial) through the warp's 32 x 17 staging block stg in shared memory.
__device__ __forceinline__ void epi_drain(const PProb& P, int m0, int n0, long long part_off, int epi, int fmt,
                                          uint32_t tmem, bool have, cf* stg, int warp, int lane) {
    if (epi == EPI_PACKNK) {
        // Row m goes to one row of a packed NK operand: 16 columns are one
        // 16-deep chunk there (two k-groups of 8).  Lanes hold consecutive
        // rows, which are 16 bytes apart in the packed tile.
        const int lg = warp & 3, ch = warp >> 2;
        const uint32_t lane_addr = tmem + ((uint32_t)(lg * 32) << 16);
        const int m = m0 + lg * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < TN / 32; ++cb) {
            const int col = ch * (TN / 2) + cb * 16;
            if (n0 + col >= P.N) break;
            float pr[16], pi[16];
            if (have) {
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
                char* d = P.rowptr[m] + (long long)(n >> 4) * PK_TILE;
                pk_store8(d, fmt, 0, v, 1.f);
                pk_store8(d, fmt, 1, v + 8, 1.f);
            }
        }
        return;
    }
    // Each warp drains 32 rows x 16 columns at a time: tcgen05.ld gives a
    // thread one row; the block is transposed through shared memory so that
    // each store instruction writes four full 128-byte row segments.
    const int lg = warp & 3, ch = warp >> 2;
    cf* Cp = P.C + (epi == EPI_PARTIAL ? part_off : 0);
    const uint32_t lane_addr = tmem + ((uint32_t)(lg * 32) << 16);
    const int rsub = lane >> 3, q = lane & 7;   // write phase: row group, 16-B chunk
#pragma unroll 1
    for (int cb = 0; cb < TN / 32; ++cb) {
        const int col = ch * (TN / 2) + cb * 16;
        if (n0 + col >= P.N) break;
        float pr[16], pi[16];
        if (have) {
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

// Grid (M tiles, N tiles, problems x splits) with the M tile fastest in
// launch order (mfast): the CTAs that read the same B tile (all M tiles of an
// N tile) run together and the later ones find it in L2; (N, M, ...) when
// the N tiles exceed the grid's y limit.
__global__ void __launch_bounds__(NTHR, CTAS_PER_SM + 1) k_cgemm_tcp(const PProb* __restrict__ probs,
                                                       const ZItem* __restrict__ zmap, int nsplit, int kchunk,
                                                       int epi, long long part_stride, int* err, int fmt,
                                                       int mfast) {
    extern __shared__ __align__(1024) char smem[];
    // slice z: problem and split (uniform, or each problem its own through zmap)
    int prob, chunk;
    long long part_off;
    if (zmap) {
        const ZItem zi = zmap[blockIdx.z];
        prob = zi.prob;
        chunk = zi.chunk;
        kchunk = zi.kchunk;
        part_off = zi.part_off;
    } else {
        prob = blockIdx.z / nsplit;
        chunk = blockIdx.z % nsplit;
        kchunk = nsplit > 1 ? kchunk : 0;
        part_off = (long long)chunk * part_stride;
    }
    const int m0 = (mfast ? blockIdx.x : blockIdx.y) * TM, n0 = (mfast ? blockIdx.y : blockIdx.x) * TN;
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
        if (kchunk > 0) {
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
            if (kchunk > 0) {
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
            const uint32_t dr = tmem, di = tmem + TN;
            const uint32_t first = c > 0 ? 1u : 0u;
            if (fmt == kFmtTF32) {
                // planes Re, Im of 8 KB; K = 8 per MMA: two K steps 256 B apart
                constexpr int PA = TILE_A / 2, PB = TILE_B / 2;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint32_t o = ks * 256;
                    const uint64_t ar = sdesc(a0 + o, 512u), ai = sdesc(a0 + PA + o, 512u);
                    const uint64_t br = sdesc(b0 + o, 512u), bi = sdesc(b0 + PB + o, 512u);
                    const uint32_t acc = ks > 0 ? 1u : first;
                    mma_tf32(dr, ar, br, IDESC_TF32, acc);
                    mma_tf32(dr, ai, bi, IDESC_TF32_NEG_A, 1u);
                    mma_tf32(di, ar, bi, IDESC_TF32, acc);
                    mma_tf32(di, ai, br, IDESC_TF32, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
                continue;
            }
            constexpr int PA = TILE_A / 4, PB = TILE_B / 4;
            const uint64_t arh = sdesc(a0), arl = sdesc(a0 + PA), aih = sdesc(a0 + 2 * PA), ail = sdesc(a0 + 3 * PA);
            const uint64_t brh = sdesc(b0), brl = sdesc(b0 + PB), bih = sdesc(b0 + 2 * PB), bil = sdesc(b0 + 3 * PB);
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
    if (warp < 8 && ok && !*abort_flag)
        epi_drain(P, m0, n0, part_off, epi, fmt, tmem, C > 0,
                  reinterpret_cast<cf*>(smem) + warp * (32 * 17), warp, lane);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == WMMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Persistent form of the packed GEMM: one CTA per SM walks the launch's
// output tiles (item i = (y, x, z): M tile y fastest, then N tile x, then
// problem-and-split z; CTA c takes items c, c + grid, ...), with the copy
// thread streaming K chunks across tile boundaries through a 5-stage ring and
// two TMEM accumulator pairs (512 columns): the MMA thread fills one pair
// while the eight epilogue warps drain the other, so a tile's set-up,
// pipeline fill and epilogue overlap the next tile's MMAs.  Items outside
// their problem are skipped by every role alike; items without K chunks are
// written as zeros by the epilogue alone.  Every wait is bounded (2 s, or an
// abort by another role); before it returns, the copy thread waits (bounded)
// for its copies still in flight.
constexpr int P_NSTAGE = 5;
constexpr int P_STG_OFF = P_NSTAGE * STAGE;                 // 160 KB of operand ring
constexpr int P_CTRL_OFF = P_STG_OFF + 8 * 32 * 17 * 8;     // + 34 KB epilogue staging
constexpr int P_SMEM_BYTES = P_CTRL_OFF + 256;
constexpr uint32_t P_TMEM_COLS = 512;                       // two accumulator pairs of 2 x TN columns
static_assert(P_SMEM_BYTES <= 227 * 1024, "shared memory of the persistent GEMM");
static_assert(2 * 2 * TN <= (int)P_TMEM_COLS, "two accumulator pairs");

struct PItem {
    int prob, m0, n0, chunk, kchunk;   // kchunk 0: the whole K
    long long part_off;
};

// item i: M tile fastest (the items that share a B tile are adjacent), then
// N tile, then slice z (problem and split: z / nsplit, z % nsplit, or zmap[z])
__device__ __forceinline__ bool p_item(const PProb* probs, const ZItem* zmap, long long i, int nx, int ny,
                                       int nsplit, int kchunk, long long part_stride, PItem& it) {
    const long long xy = (long long)nx * ny;
    const int z = (int)(i / xy);
    const int r = (int)(i - (long long)z * xy);
    if (zmap) {
        const ZItem zi = zmap[z];
        it.prob = zi.prob;
        it.chunk = zi.chunk;
        it.kchunk = zi.kchunk;
        it.part_off = zi.part_off;
    } else {
        it.prob = z / nsplit;
        it.chunk = z - it.prob * nsplit;
        it.kchunk = nsplit > 1 ? kchunk : 0;
        it.part_off = (long long)it.chunk * part_stride;
    }
    it.m0 = (r % ny) * TM;
    it.n0 = (r / ny) * TN;
    const PProb& P = probs[it.prob];
    return it.m0 < P.M && it.n0 < P.N;
}

// the K range [kb, ke) of term t for an item
__device__ __forceinline__ void p_range(const PTerm& t, const PItem& it, int& kb, int& ke) {
    kb = 0;
    ke = t.K;
    if (it.kchunk > 0) {
        kb = it.chunk * it.kchunk;
        ke = min(t.K, kb + it.kchunk);
    }
}

// K chunks of one item (16-deep chunks over its terms)
__device__ __forceinline__ int p_chunks(const PProb& P, const PItem& it) {
    int C = 0;
    for (int ti = 0; ti < P.nt; ++ti) {
        int kb, ke;
        p_range(P.t[ti], it, kb, ke);
        if (ke > kb) C += (ke - kb + KC - 1) / KC;
    }
    return C;
}

__global__ void __launch_bounds__(NTHR, 1) k_cgemm_tcp_pers(const PProb* __restrict__ probs,
                                                            const ZItem* __restrict__ zmap, int nsplit, int kchunk,
                                                            int epi, long long part_stride, int* err, int fmt,
                                                            int nx, int ny, long long nitems) {
    extern __shared__ __align__(1024) char smem[];
    if (*(volatile int*)err != 0) return;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + P_CTRL_OFF);
    uint64_t* empty = full + P_NSTAGE;
    uint64_t* tfull = empty + P_NSTAGE;    // [2] accumulator pair ready for the epilogue
    uint64_t* tempty = tfull + 2;          // [2] accumulator pair drained (8 warp arrivals)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P_NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&tempty[b])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == WMMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(P_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == WCOPY && lane == 0) {
        // ---------------- bulk copies, across tiles ----------------
        long long c = 0;
        for (long long i = blockIdx.x; i < nitems && !*abort_flag; i += gridDim.x) {
            PItem it;
            if (!p_item(probs, zmap, i, nx, ny, nsplit, kchunk, part_stride, it)) continue;
            const PProb& P = probs[it.prob];
            for (int ti = 0; ti < P.nt && !*abort_flag; ++ti) {
                const PTerm& t = P.t[ti];
                int kb, ke;
                p_range(t, it, kb, ke);
                const int nkc = (t.K + KC - 1) / KC;
                const char* abase = reinterpret_cast<const char*>(t.A) + (long long)(it.m0 / TM) * nkc * TILE_A;
                const char* bbase = reinterpret_cast<const char*>(t.B) + (long long)(it.n0 / TN) * nkc * TILE_B;
                for (int k0 = kb; k0 < ke; k0 += KC, ++c) {
                    const int s = (int)(c % P_NSTAGE);
                    if (c >= P_NSTAGE &&
                        !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((c / P_NSTAGE) - 1) & 1), err)) {
                        *abort_flag = 1;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full[s]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE)
                                 : "memory");
                    const int kc = k0 / KC;
                    const uint32_t dst = smem_u32(smem + s * STAGE);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            dst),
                        "l"(abase + (long long)kc * TILE_A), "r"(TILE_A), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            dst + TILE_A),
                        "l"(bbase + (long long)kc * TILE_B), "r"(TILE_B), "r"(fb)
                        : "memory");
                }
            }
        }
        // copies still in flight land before the CTA's shared memory goes away
        for (long long j = c - 1; j >= 0 && j >= c - P_NSTAGE; --j) {
            const int s = (int)(j % P_NSTAGE);
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((j / P_NSTAGE) & 1), err)) *abort_flag = 1;
        }
    } else if (warp == WMMA && lane == 0) {
        // ---------------- MMA issuer ----------------
        long long c = 0, u = 0;
        for (long long i = blockIdx.x; i < nitems && !*abort_flag; i += gridDim.x) {
            PItem it;
            if (!p_item(probs, zmap, i, nx, ny, nsplit, kchunk, part_stride, it)) continue;
            const int C = p_chunks(probs[it.prob], it);
            if (C == 0) continue;
            const int ab = (int)(u & 1);
            if (u >= 2 && !mbar_wait(smem_u32(&tempty[ab]), (uint32_t)(((u >> 1) - 1) & 1), err)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dr = tmem + ab * 2 * TN, di = dr + TN;
            for (int k = 0; k < C; ++k, ++c) {
                const int s = (int)(c % P_NSTAGE);
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((c / P_NSTAGE) & 1), err)) {
                    *abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + TILE_A;
                const uint32_t first = k > 0 ? 1u : 0u;
                if (fmt == kFmtTF32) {
                    constexpr int PA = TILE_A / 2, PB = TILE_B / 2;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t o = ks * 256;
                        const uint64_t ar = sdesc(a0 + o, 512u), ai = sdesc(a0 + PA + o, 512u);
                        const uint64_t br = sdesc(b0 + o, 512u), bi = sdesc(b0 + PB + o, 512u);
                        const uint32_t acc = ks > 0 ? 1u : first;
                        mma_tf32(dr, ar, br, IDESC_TF32, acc);
                        mma_tf32(dr, ai, bi, IDESC_TF32_NEG_A, 1u);
                        mma_tf32(di, ar, bi, IDESC_TF32, acc);
                        mma_tf32(di, ai, br, IDESC_TF32, 1u);
                    }
                } else {
                    constexpr int PA = TILE_A / 4, PB = TILE_B / 4;
                    const uint64_t arh = sdesc(a0), arl = sdesc(a0 + PA), aih = sdesc(a0 + 2 * PA),
                                   ail = sdesc(a0 + 3 * PA);
                    const uint64_t brh = sdesc(b0), brl = sdesc(b0 + PB), bih = sdesc(b0 + 2 * PB),
                                   bil = sdesc(b0 + 3 * PB);
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
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
            }
            if (*abort_flag) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&tfull[ab]))
                         : "memory");
            ++u;
        }
    } else if (warp < 8) {
        // ---------------- epilogue, one accumulator pair at a time ----------------
        cf* stg = reinterpret_cast<cf*>(smem + P_STG_OFF) + warp * (32 * 17);
        long long u = 0;
        for (long long i = blockIdx.x; i < nitems && !*abort_flag; i += gridDim.x) {
            PItem it;
            if (!p_item(probs, zmap, i, nx, ny, nsplit, kchunk, part_stride, it)) continue;
            const PProb& P = probs[it.prob];
            const int C = p_chunks(P, it);
            if (C == 0) {
                epi_drain(P, it.m0, it.n0, it.part_off, epi, fmt, tmem, false, stg, warp, lane);
                continue;
            }
            const int ab = (int)(u & 1);
            if (!mbar_wait(smem_u32(&tfull[ab]), (uint32_t)((u >> 1) & 1), err)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epi_drain(P, it.m0, it.n0, it.part_off, epi, fmt, tmem + ab * 2 * TN, true, stg, warp, lane);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[ab])) : "memory");
            ++u;
        }
    }
    if (*abort_flag && threadIdx.x == 0) atomicExch(err, TLR_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == WMMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P_TMEM_COLS) : "memory");
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

// The passes' launch priority: the device's greatest, or their stream's with
// TLR_MDD_PASS_PRIORITY=0 (read once).  Measured on the nr = 9216 workload
// with 3 streams: 3.32 freq-solves/s against 3.26 at the stream's priority
// (both with the pass grid capped at 4 CTAs per SM), and 3.26 with the
// contractions at the greatest priority instead.
int pass_priority() {
    static const int prio = [] {
        const char* e = getenv("TLR_MDD_PASS_PRIORITY");
        if (e && atoi(e) == 0) return 0;
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        return greatest;
    }();
    return prio;
}

// CTAs of a fused update-and-pack launch over nt tiles: all of them, or at
// most the cap (a tile loop walks the rest), so that beside contractions of
// other streams the pass holds a bounded share of the SMs.  The cap starts
// from the environment variable TLR_MDD_PASS_CTAS (else kPassCtasDefault)
// and is set with tlr_mdd_set_pass_ctas.
namespace {
std::atomic<long long> g_pass_cap{-1};
}

long long pass_cap() {
    long long c = g_pass_cap.load(std::memory_order_relaxed);
    if (c < 0) {
        const char* e = getenv("TLR_MDD_PASS_CTAS");
        long long want = e ? std::max(0LL, atoll(e)) : kPassCtasDefault;
        long long expect = -1;
        g_pass_cap.compare_exchange_strong(expect, want);
        c = g_pass_cap.load(std::memory_order_relaxed);
    }
    return c;
}

void set_pass_cap(long long ctas) {
    pass_cap();   // the environment's value is consumed first, so a set is never overwritten
    g_pass_cap.store(std::max(0LL, ctas), std::memory_order_relaxed);
}

long long pass_grid(long long nt) {
    const long long cap = pass_cap();
    return cap > 0 ? std::min(nt, cap) : nt;
}

long long packed_bytes(long long R, long long K, int TR) {
    const long long nkc = (K + KC - 1) / KC, nrb = (R + TR - 1) / TR;
    return nrb * nkc * 4LL * TR * KC * 2;
}

// max_items encodes the largest job: (padded rows << 32) | k-groups
cudaError_t pack_operands(const PackJob* jobs, int njobs, long long max_items, cudaStream_t st) {
    if (njobs == 0 || max_items == 0) return cudaSuccess;
    const long long rows = max_items >> 32, kgs = max_items & 0xffffffffLL;
    dim3 grid((unsigned)((rows + 255) / 256), (unsigned)njobs, (unsigned)((kgs + PACK_KG - 1) / PACK_KG));
    const cudaError_t e = launch_pass(k_pack, grid, dim3(256), st, jobs);
    counted(1);
    return e;
}

cudaError_t tpack(const TPackTile* d_tiles, int ntiles, cf* T, const cf* Tp, const double* alpha, int ns,
                  cudaStream_t st) {
    if (ntiles == 0 || ns == 0) return cudaSuccess;
    const int gx = (ns + TP_N - 1) / TP_N;
    const long long nt = (long long)gx * ntiles;
    const cudaError_t e = launch_pass(k_tpack, dim3((unsigned)pass_grid(nt)), dim3(256), st, d_tiles, T, Tp, alpha, ns,
                                      gx, nt);
    counted(1);
    return e;
}

long long rstep_ctas(int nr, int ns) { return (long long)((ns + TP_N - 1) / TP_N) * (nr / TP_K); }

cudaError_t rstep(cf* R, const cf* A1, const cf* A2, const double* alpha, int nr, int ns, int b, char* const* kn,
                  char* const* mk, double* part, cudaStream_t st, const long long* roff, int nblk, int fmt) {
    if (nr == 0 || ns == 0) return cudaSuccess;
    if (nr % TP_K != 0) return cudaErrorInvalidValue;
    if (!roff && (b <= 0 || b % TP_K != 0 || nr % b != 0)) return cudaErrorInvalidValue;
    if (roff && nblk <= 0) return cudaErrorInvalidValue;
    const int gx = (ns + TP_N - 1) / TP_N;
    const long long nt = (long long)gx * (nr / TP_K);
    const cudaError_t e = launch_pass(k_rstep, dim3((unsigned)pass_grid(nt)), dim3(256), st, R, A1, A2, alpha, ns, b, kn,
                                      mk, part, roff, nblk, fmt, gx, nt);
    counted(1);
    return e;
}

cudaError_t dots6_packed(char* const* kn, const cf* A1, const cf* A2, int nr, int ns, int b, double* part,
                         cudaStream_t st, const long long* roff, int nblk, int fmt) {
    if (nr == 0 || ns == 0) return cudaSuccess;
    if (nr % TP_K != 0) return cudaErrorInvalidValue;
    if (!roff && (b <= 0 || b % TP_K != 0 || nr % b != 0)) return cudaErrorInvalidValue;
    if (roff && nblk <= 0) return cudaErrorInvalidValue;
    const cudaError_t e = launch_pass(k_dots6p, dim3(kRedBlocks), dim3(256), st, kn, A1, A2, ns, nr, b, roff, nblk,
                                      part, fmt);
    counted(1);
    return e;
}

cudaError_t wait_selftest(int* status, unsigned long long limit_ns, unsigned long long* waited_ns,
                          cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(status, limit_ns, waited_ns);
    counted(1);
    return cudaGetLastError();
}

cudaError_t gemm_tcp_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_cgemm_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cgemm_tcp_pers, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM_BYTES);
    return e;
}

cudaError_t gemm_tcp(const GemmLaunch& L, cudaStream_t st) {
    if (L.nprob == 0 || L.maxM == 0 || L.maxN == 0) return cudaSuccess;
    if (!L.err || !L.d_pprobs) return cudaErrorInvalidValue;
    const int kchunk = L.nsplit > 1 ? L.kchunk : 0;
    if (L.persistent) {
        const int nx = (L.maxN + TN - 1) / TN, ny = (L.maxM + TM - 1) / TM;
        const long long nz = L.d_zmap ? L.nz : (long long)L.nprob * L.nsplit;
        const long long nitems = (long long)nx * ny * nz;
        if (nitems == 0) return cudaSuccess;
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
        const unsigned g = (unsigned)std::min<long long>(sms, nitems);
        k_cgemm_tcp_pers<<<g, NTHR, P_SMEM_BYTES, st>>>(L.d_pprobs, L.d_zmap, L.nsplit, kchunk, L.epi,
                                                        L.part_stride, L.err, pack_fmt(L.prec), nx, ny, nitems);
        counted(1);
        return cudaGetLastError();
    }
    const unsigned mt = (unsigned)((L.maxM + TM - 1) / TM), nt = (unsigned)((L.maxN + TN - 1) / TN);
    const int mfast = nt <= 65535u ? 1 : 0;
    const unsigned nzs = (unsigned)(L.d_zmap ? L.nz : L.nprob * L.nsplit);
    if (nzs == 0) return cudaSuccess;
    dim3 grid(mfast ? mt : nt, mfast ? nt : mt, nzs);
    k_cgemm_tcp<<<grid, NTHR, SMEM_BYTES, st>>>(L.d_pprobs, L.d_zmap, L.nsplit, kchunk, L.epi, L.part_stride, L.err,
                                                 pack_fmt(L.prec), mfast);
    counted(1);
    return cudaGetLastError();
}

}  // namespace tlr
