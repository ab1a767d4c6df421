// Tensor-core (tcgen05, sm_103a) grouped complex GEMM for the TLR contractions,
// same problem tables as the FP32 SIMT path (compress, expand, projection,
// adjoint).
//
// Arithmetic.  Every complex product C = A B is formed from four real
// products (4M): Cr = Ar Br - Ai Bi, Ci = Ar Bi + Ai Br, accumulated in two
// FP32 TMEM accumulators (the subtraction is the MMA's negate-A flag).  Every
// real product X Y runs in BF16 with a hi/lo split of both operands
// (x = hi + lo, hi = RN_bf16(x), lo = RN_bf16(x - hi)) and three tensor-core
// products hi*hi + hi*lo + lo*hi.  The dropped lo*lo term is below 2^-16 of
// |x||y|.  4M rather than 3M: two accumulators of 256 columns fill the 512
// TMEM columns, so a CTA owns a 128 x 256 output tile and splits each A
// element once per 256 output columns and only two values (Re, Im) per
// complex element; the kernel is bound by that on-the-fly split, not by the
// 33% more MMAs of 4M.
//
// Data movement.  Warps 0-7 (producers) walk the K chunks of 16 complex
// elements: each thread copies one 8-element run of A and two of B from
// global memory into a raw FP32 shared-memory ring with cp.async (applying
// the row gather of the problem table; cp.async copies are not waited on by
// fences or barrier arrivals, so the next chunk stays in flight), then splits
// the chunk that has landed into four BF16 planes per operand (Re, Im; hi and
// lo) in the canonical K-major, no-swizzle layout of the tensor core (8-row x
// 16-byte core matrices, 128 B apart along K, 256 B apart along M/N) and
// arrives on the stage's "full" mbarrier.  Warp 8 waits for "full", issues
// the 12 MMAs of the chunk (M = 128, N = 256, K = 16) and commits them to the
// stage's "empty" mbarrier, which the producers wait on before reusing it.
// After a final commit the producer warps read TMEM with tcgen05.ld.
//
// Every mbarrier wait is bounded; on timeout the CTA records TLR_ERR_TIMEOUT
// in the error word, stops issuing work, waits (bounded) for what it issued,
// frees its TMEM and exits.
#include <cuda_bf16.h>

#include "internal.h"

namespace tlr {

namespace {

constexpr int TM = 128, TN = 256, KC = 16;          // tile and K chunk (complex elements)
constexpr int NPROD = 256;                          // producer threads (warps 0-7)
constexpr int NTHR = NPROD + 32;                    // + one MMA warp (warp 8)
constexpr int NSTAGE = 2;                           // BF16 operand stages read by the tensor core
constexpr int RSTAGE = 2;                           // raw FP32 stages filled by cp.async
constexpr int PLANE_A = TM * KC * 2;                // one BF16 plane of A (128 rows x 16 k) = 4 KB
constexpr int PLANE_B = TN * KC * 2;                // one BF16 plane of B (256 rows x 16 k) = 8 KB
constexpr int STAGE = 4 * PLANE_A + 4 * PLANE_B;    // Re/Im x hi/lo for A and B = 48 KB
constexpr int RAW_A = NPROD * 8 * 8;                // one 8-complex run of A per producer = 16 KB
constexpr int RAW = RAW_A + 2 * RAW_A;              // + two runs of B per producer = 48 KB
constexpr int RAW_OFF = NSTAGE * STAGE;
constexpr int IDX_CAP = 4096;                       // gather indices staged in shared memory
constexpr int CTRL = 256;                           // barriers, TMEM address, abort flag
constexpr int CTRL_OFF = RAW_OFF + RSTAGE * RAW;
constexpr int PROB_OFF = CTRL_OFF + CTRL;           // problem descriptor copy
constexpr int IDX_OFF = PROB_OFF + 256;
constexpr int SMEM_BYTES = IDX_OFF + IDX_CAP * 4;
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // a barrier wait gives up after 2 s
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");

// instruction descriptor: D f32, A bf16, B bf16, both K-major, N = 256, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);   // D += (-A) B

// shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 B; 128 B apart along K (leading byte offset), 256 B apart
// along M/N (stride byte offset: KC/8 = 2 core matrices per 8-row group)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;             // descriptor version
    return d;                           // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the given phase parity of an mbarrier: gives up after
// WAIT_NS of wall time, or at once when another CTA has already recorded an
// error in the launch's error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* err) {
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
        if ((it & 255u) == 255u && (*err != 0 || now_ns() - t0 > WAIT_NS)) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// split 8 complex values into the four BF16 planes (Re hi, Re lo, Im hi,
// Im lo) and store 16 B per plane; planes are ``plane`` bytes apart
__device__ __forceinline__ void split_store(const float2 (&v)[8], char* plane0, int plane, int off) {
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
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(plane0 + q * plane + off) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// byte offset of (row r, k-group kg) in a K-major no-swizzle plane
__device__ __forceinline__ int core_off(int r, int kg) { return ((r >> 3) * (KC / 8) + kg) * 128 + (r & 7) * 16; }

// Asynchronous 8-byte copy global -> shared with zero fill (src_size 0 or 8).
// cp.async copies are not waited on by fences or barrier arrivals, so the
// producers can keep several chunks in flight.
__device__ __forceinline__ void cp8(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}

// Raw stage layout: element j (0..7) of producer pid at [j][pid] for A, then
// the same for B; a warp reading element j touches 32 consecutive float2.
__device__ __forceinline__ uint32_t raw_a(uint32_t base, int j, int pid) { return base + (j * NPROD + pid) * 8; }
__device__ __forceinline__ uint32_t raw_b(uint32_t base, int it, int j, int pid) {
    return base + RAW_A + it * RAW_A + (j * NPROD + pid) * 8;
}

template <int AM>
__device__ __forceinline__ void issue_a(const GTerm& t, int M, int m0, int k0, int kend, int pid, uint32_t rb) {
    const int r = pid & (TM - 1), kg = pid >> 7;
    const int m = m0 + r, kb = k0 + kg * 8;
    const bool mv = m < M;
    const cf* base = t.A;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = kb + j;
        const bool v = mv && k < kend;
        const cf* src = v ? ((AM == A_MK) ? base + (long long)m * t.lda + k : base + (long long)k * t.lda + m) : base;
        cp8(raw_a(rb, j, pid), src, v);
    }
}

// gidx: the term's gather indices, offset so that gidx[k] (KN) or gidx[n]
// (NK) is the row; nullptr without a gather.
template <int BMD>
__device__ __forceinline__ void issue_b(const GTerm& t, const int* gidx, int N, int n0, int k0, int kend, int pid,
                                        uint32_t rb) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int id = pid + it * NPROD;
        const int r = id & (TN - 1), kg = id >> 8;
        const int n = n0 + r, kb = k0 + kg * 8;
        const bool nv = n < N;
        const cf* base = t.B;
        long long rowN = 0;
        if (BMD == B_NK && nv) rowN = gidx ? gidx[n] : n;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = kb + j;
            const bool v = nv && k < kend;
            const cf* src = base;
            if (v) {
                if (BMD == B_KN) {
                    const long long row = gidx ? gidx[k] : k;
                    src = base + row * t.ldb + n;
                } else {
                    src = base + rowN * t.ldb + k;
                }
            }
            cp8(raw_b(rb, it, j, pid), src, v);
        }
    }
}

// read one of this producer's raw runs back (slot 0: A, 1-2: B), apply the
// conjugation sign
__device__ __forceinline__ void read_raw(const char* smem, uint32_t off0, int pid, float sgn, int slot,
                                         float2 (&v)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t o = slot * RAW_A + (j * NPROD + pid) * 8;
        float2 x = *reinterpret_cast<const float2*>(smem + off0 + o);
        x.y *= sgn;
        v[j] = x;
    }
}

// The chunks of a problem: for each term, K range [kb, ke) cut in KC pieces.
struct ChunkIter {
    int ti, k0, kb, ke;
};

__device__ __forceinline__ void term_range(const GProb& P, int ti, int nsplit, int chunk, int kchunk, int& kb,
                                           int& ke) {
    kb = 0;
    ke = P.t[ti].K;
    if (nsplit > 1) {
        kb = chunk * kchunk;
        ke = min(P.t[ti].K, kb + kchunk);
    }
}

__device__ __forceinline__ int count_chunks(const GProb& P, int nsplit, int chunk, int kchunk) {
    int c = 0;
    for (int ti = 0; ti < P.nt; ++ti) {
        int kb, ke;
        term_range(P, ti, nsplit, chunk, kchunk, kb, ke);
        if (ke > kb) c += (ke - kb + KC - 1) / KC;
    }
    return c;
}

// first chunk at or after term ti (k0 = kb); ti == nt when exhausted
__device__ __forceinline__ void seek(const GProb& P, int nsplit, int chunk, int kchunk, ChunkIter& it) {
    while (it.ti < P.nt) {
        term_range(P, it.ti, nsplit, chunk, kchunk, it.kb, it.ke);
        if (it.ke > it.kb) {
            it.k0 = it.kb;
            return;
        }
        ++it.ti;
    }
}

__device__ __forceinline__ void advance(const GProb& P, int nsplit, int chunk, int kchunk, ChunkIter& it) {
    it.k0 += KC;
    if (it.k0 >= it.ke) {
        ++it.ti;
        seek(P, nsplit, chunk, kchunk, it);
    }
}

template <int AM, int BMD>
__global__ void __launch_bounds__(NTHR, 1) k_cgemm_tc(const GProb* __restrict__ probs, int nsplit, int kchunk,
                                                      int epi, long long part_stride, int* err) {
    extern __shared__ __align__(1024) char smem[];
    const int prob = blockIdx.z / nsplit, chunk = blockIdx.z % nsplit;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    {
        const GProb& Pg = probs[prob];
        if (m0 >= Pg.M || n0 >= Pg.N) return;
        if (*(volatile int*)err != 0) return;   // an earlier CTA gave up: do no more work
    }
    // descriptor and gather indices go to shared memory once, so the
    // producers' per-chunk loads are single, independent global loads
    GProb& P = *reinterpret_cast<GProb*>(smem + PROB_OFF);
    int* sidx = reinterpret_cast<int*>(smem + IDX_OFF);
    static_assert(sizeof(GProb) <= 256, "descriptor slot");
    {
        const int* src = reinterpret_cast<const int*>(&probs[prob]);
        int* dst = reinterpret_cast<int*>(&P);
        for (int i = threadIdx.x; i < (int)(sizeof(GProb) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    // per term: the staged indices (sidx + goff[ti])[j] = g[j], or read g from
    // global memory when they do not fit (gst[ti] false)
    int goff[kMaxTerms];
    bool gst[kMaxTerms];
    {
        int used = 0;
        for (int ti = 0; ti < P.nt; ++ti) {
            goff[ti] = 0;
            gst[ti] = false;
            const GTerm& t = P.t[ti];
            if (!t.g) continue;
            int lo, hi;
            if (BMD == B_KN) {
                term_range(P, ti, nsplit, chunk, kchunk, lo, hi);
            } else {
                lo = n0;
                hi = min(P.N, n0 + TN);
            }
            const int cnt = max(0, hi - lo);
            if (used + cnt <= IDX_CAP) {
                for (int i = threadIdx.x; i < cnt; i += blockDim.x) sidx[used + i] = t.g[lo + i];
                goff[ti] = used - lo;
                gst[ti] = true;
                used += cnt;
            }
        }
    }

    uint64_t* full = reinterpret_cast<uint64_t*>(smem + CTRL_OFF);
    uint64_t* empty = full + NSTAGE;
    uint64_t* done = empty + NSTAGE;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = count_chunks(P, nsplit, chunk, kchunk);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(NPROD / 32)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp < 8) {
        // ---------------- producers ----------------
        const int pid = threadIdx.x;
        const int r = pid & 127, kg = pid >> 7;
        const uint32_t raw0 = smem_u32(smem + RAW_OFF);
        ChunkIter it{0, 0, 0, 0};
        seek(P, nsplit, chunk, kchunk, it);
        ChunkIter nx = it;      // next chunk to issue
        ChunkIter cur = it;     // chunk being converted
        // prologue: chunks 0 .. RSTAGE-2 in flight
#pragma unroll
        for (int q = 0; q < RSTAGE - 1; ++q) {
            if (q < C) {
                const GTerm& t = P.t[nx.ti];
                const int* gi = t.g ? (gst[nx.ti] ? sidx + goff[nx.ti] : t.g) : nullptr;
                const uint32_t rb = raw0 + q * RAW;
                issue_a<AM>(t, P.M, m0, nx.k0, nx.ke, pid, rb);
                issue_b<BMD>(t, gi, P.N, n0, nx.k0, nx.ke, pid, rb);
                advance(P, nsplit, chunk, kchunk, nx);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        for (int c = 0; c < C; ++c) {
            // keep RSTAGE - 1 chunks in flight: issue chunk c + RSTAGE - 1
            if (c + RSTAGE - 1 < C) {
                const GTerm& t = P.t[nx.ti];
                const int* gi = t.g ? (gst[nx.ti] ? sidx + goff[nx.ti] : t.g) : nullptr;
                const uint32_t rb = raw0 + ((c + RSTAGE - 1) % RSTAGE) * RAW;
                issue_a<AM>(t, P.M, m0, nx.k0, nx.ke, pid, rb);
                issue_b<BMD>(t, gi, P.N, n0, nx.k0, nx.ke, pid, rb);
                advance(P, nsplit, chunk, kchunk, nx);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group %0;" ::"n"(RSTAGE - 1) : "memory");  // chunk c has landed
            const int s = c % NSTAGE;
            if (c >= NSTAGE) {
                if (!mbar_wait(smem_u32(&empty[s]), (uint32_t)(((c / NSTAGE) - 1) & 1), err)) *abort_flag = 1;
            }
            if (*abort_flag) break;
            const GTerm& t = P.t[cur.ti];
            const uint32_t roff = RAW_OFF + (c % RSTAGE) * RAW;
            float2 v[8];
            char* st = smem + s * STAGE;
            read_raw(smem, roff, pid, t.sa, 0, v);
            split_store(v, st, PLANE_A, core_off(r, kg));
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int id = pid + it * NPROD;
                read_raw(smem, roff, pid, t.sb, 1 + it, v);
                split_store(v, st + 4 * PLANE_A, PLANE_B, core_off(id & (TN - 1), id >> 8));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full[s]));
            advance(P, nsplit, chunk, kchunk, cur);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        for (int c = 0; c < C; ++c) {
            const int s = c % NSTAGE;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((c / NSTAGE) & 1), err)) {
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + 4 * PLANE_A;
            // planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo
            const uint64_t arh = sdesc(a0), arl = sdesc(a0 + PLANE_A), aih = sdesc(a0 + 2 * PLANE_A),
                           ail = sdesc(a0 + 3 * PLANE_A);
            const uint64_t brh = sdesc(b0), brl = sdesc(b0 + PLANE_B), bih = sdesc(b0 + 2 * PLANE_B),
                           bil = sdesc(b0 + 3 * PLANE_B);
            const uint32_t dr = tmem, di = tmem + 256;
            const uint32_t first = c > 0 ? 1u : 0u;
            // Cr += Ar Br - Ai Bi
            mma_bf16(dr, arh, brh, IDESC, first);
            mma_bf16(dr, arh, brl, IDESC, 1u);
            mma_bf16(dr, arl, brh, IDESC, 1u);
            mma_bf16(dr, aih, bih, IDESC_NEG_A, 1u);
            mma_bf16(dr, aih, bil, IDESC_NEG_A, 1u);
            mma_bf16(dr, ail, bih, IDESC_NEG_A, 1u);
            // Ci += Ar Bi + Ai Br
            mma_bf16(di, arh, bih, IDESC, first);
            mma_bf16(di, arh, bil, IDESC, 1u);
            mma_bf16(di, arl, bih, IDESC, 1u);
            mma_bf16(di, aih, brh, IDESC, 1u);
            mma_bf16(di, aih, brl, IDESC, 1u);
            mma_bf16(di, ail, brh, IDESC, 1u);
            mma_commit(smem_u32(&empty[s]));
        }
        mma_commit(smem_u32(done));   // arrives once every MMA issued above has completed
    }

    // ---------------- epilogue (producer warps) ----------------
    bool ok = true;
    if (warp < 8 && C > 0) ok = mbar_wait(smem_u32(done), 0u, err);
    if (!ok || *abort_flag) {
        if (threadIdx.x == 0 || !ok) atomicExch(err, TLR_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 8 && ok && !*abort_flag) {
        const int lg = warp & 3, ch = warp >> 2;
        const int m = m0 + lg * 32 + lane;
        cf* Cp = P.C + (epi == EPI_PARTIAL ? chunk * part_stride : 0);
        const uint32_t lane_addr = tmem + ((uint32_t)(lg * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < 8; ++cb) {
            const int col = ch * 128 + cb * 16;
            if (n0 + col >= P.N) break;
            float pr[16], pi[16];
            if (C > 0) {
                tmem_ld16(lane_addr + col, pr);
                tmem_ld16(lane_addr + 256 + col, pi);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) pr[j] = pi[j] = 0.f;
            }
            if (m < P.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + col + j;
                    if (n >= P.N) break;
                    const long long o = (long long)m * P.ldc + n;
                    cf v = make_float2(pr[j], pi[j]);
                    if (epi == EPI_SUB) {
                        const cf sv = P.S[o];
                        v.x -= sv.x;
                        v.y -= sv.y;
                    } else if (epi == EPI_ACCUM) {
                        const cf cv = Cp[o];
                        v.x += cv.x;
                        v.y += cv.y;
                    }
                    Cp[o] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8) {
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

cudaError_t gemm_tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc<A_KM, B_KN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cgemm_tc<A_MK, B_KN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cgemm_tc<A_MK, B_NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    return e;
}

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
