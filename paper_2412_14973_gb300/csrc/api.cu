// C ABI of libtlr_mdd: handle life cycle, the tile layout of the stacked
// unknown (Tile Low-rank MDD section), grouped-GEMM work tables and the
// device-resident ADMM / L-BFGS solve (eq. 18-24).
//
// Internal representation.  Every factor of the TLR parametrisation acts on
// exactly one block column of Dfrak in the forward product and on exactly one
// block row of Y, and for a symmetric X both are the same block: block i holds
//   F_i = [ Q_ii | L_ij (j < i) | R_ji (j > i) ]   (d_i x K_i, row-major panel)
// so that, with T_i = F_i^T Dfrak_i (compress) and T~ the rows of T taken at
// each column's partner factor (L_ij <-> R_ij, Q_ii <-> itself),
//   Y_i = X_h Dfrak |_i = F_i T~_i + P(Z_ii) Dfrak_i            (eq. 6-9, 15)
//   grad F_i = Rf_i T~_i^H + conj(Dfrak_i) V~_i^T,  V_i = F_i^H Rf_i (eq. 25-27)
//   grad Z_ii = (G_ii + G_ii^T) / 2,  G_ii = Rf_i Dfrak_i^H       (eq. 26)
// with Rf = Y - Ufrak the receiver-major residual.  The panel vector
// [F_0 .. F_{N-1} | dense Z tiles] is a permutation of theta.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "solver_dev.h"

#include <map>
#include <mutex>
#include <set>
#include <tuple>

using namespace tlr;

std::atomic<long long> tlr::g_launches{0};

namespace {

thread_local std::string g_last_error;
constexpr int kPersistDefault = 0;

// ---- workspace pool ----
// Handles take their device workspace from one stream-ordered memory pool per
// device owned by this library, created with no release threshold: memory a
// destroyed handle gives back stays reserved for the next handle instead of
// returning to the driver at the next synchronisation, so creating and
// destroying a handle per frequency (or per served request) maps no fresh
// device memory.  tlr_mdd_trim_pool() hands the reserve back.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};

cudaError_t ws_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps pr;
        memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.handleTypes = cudaMemHandleTypeNone;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t p = nullptr;
        e = cudaMemPoolCreate(&p, &pr);
        if (e != cudaSuccess) return e;
        unsigned long long thr = ~0ULL;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// stream-ordered allocation of handle workspace from the library's pool
cudaError_t ws_alloc(void** ptr, size_t bytes, cudaStream_t st) {
    cudaMemPool_t p = nullptr;
    cudaError_t e = ws_pool(&p);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(ptr, bytes, p, st);
}

// environment switch set to "0"
bool getenv_off(const char* name) {
    const char* e = getenv(name);
    return e && e[0] == '0';
}

// ---- diagnostics: CUDA-event timing of the contraction launches ----
struct TimedLaunch {
    int cls;
    double flops;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimedLaunch> g_pending;
std::vector<cudaEvent_t> g_evpool;
double g_ms[TLR_NCLASS] = {0}, g_fl[TLR_NCLASS] = {0};
long long g_nl[TLR_NCLASS] = {0};

cudaEvent_t ev_get() {
    if (!g_evpool.empty()) {
        cudaEvent_t e = g_evpool.back();
        g_evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// While a solve is being captured into a CUDA graph, timed launches are
// collected here (per handle) instead of in g_pending: their events are
// re-recorded at every replay and read after each one.
thread_local std::vector<TimedLaunch>* g_capture_sink = nullptr;

}  // namespace

// Contraction classes (bit 0 compress, 1 expand, 2 project) whose packed
// tensor-core launches use the persistent, double-buffered kernel; the
// environment variable TLR_MDD_PERSIST (a bit mask) overrides the default.
static int persist_classes() {
    const char* e = getenv("TLR_MDD_PERSIST");   // read when a handle's launches are planned
    return e ? (atoi(e) & 7) : kPersistDefault;
}

// launch one grouped contraction, timed when diagnostics are on
cudaError_t tlr::run_gemm(const GemmLaunch& L, cudaStream_t st) {
    if (L.nprob == 0) return cudaSuccess;
    if (!g_timing) return gemm_any(L, st);
    std::lock_guard<std::mutex> lk(g_tmu);
    TimedLaunch t{L.cls, L.flops, ev_get(), ev_get()};
    // inside a stream capture the events must become real event-record
    // nodes of the graph (external), so every replay records them
    const unsigned fl = g_capture_sink ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaError_t e = cudaEventRecordWithFlags(t.a, st, fl);
    if (e == cudaSuccess) e = gemm_any(L, st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(t.b, st, fl);
    if (g_capture_sink)
        g_capture_sink->push_back(t);
    else
        g_pending.push_back(t);
    return e;
}

namespace {

// add the device times of a replayed graph's timed launches to the totals
void account_replay(const std::vector<TimedLaunch>& v) {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (const auto& t : v) {
        float m = 0.f;
        if (cudaEventElapsedTime(&m, t.a, t.b) == cudaSuccess) {
            g_ms[t.cls] += m;
            g_fl[t.cls] += t.flops;
            g_nl[t.cls] += 1;
        } else {
            (void)cudaGetLastError();  // a diagnostic read never poisons later calls
        }
    }
}

struct HostStats {
    int ints[SI_COUNT + 2];
    double sc[SC_COUNT];
    double fhist[TLR_MAX_HIST];
};

struct GraphKey {
    double lam0 = -1, decay = 0, rho = 0;
    int stages = -1, admm = -1, lbfgs = -1, mem = -1, timing = -1, flags = -1;
    bool operator==(const GraphKey& o) const {
        return lam0 == o.lam0 && decay == o.decay && rho == o.rho && stages == o.stages && admm == o.admm &&
               lbfgs == o.lbfgs && mem == o.mem && timing == o.timing && flags == o.flags;
    }
};

struct Arena {
    char* base = nullptr;
    size_t used = 0;
    size_t cap = 0;
    template <class T>
    T* take(size_t n) {
        size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
        if (base == nullptr) {  // sizing pass
            used += bytes;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

// Panels.  Expand side (A): block i holds the factors that multiply the
// products T into row block i of Y (the right factors of the tiles X_ji);
// compress side (B): block j holds the factors that compress column block j
// of Dfrak (the left factors of the tiles X_ji).  In the reciprocal form the
// two sides are the same panel (Q_ii, L_ij for j < i, R_ji for j > i serve
// both); in the general form (reciprocity NONE) they are disjoint: A panels
// first, then B panels, in one panel vector.
struct Layout {
    int64_t nr = 0, ns = 0;
    int64_t b = 0;                 // tile size of a uniform partition, 0 for a non-uniform one
    int64_t dmax = 0;              // the largest tile size
    int N = 0, P = 0;              // P: stored pairs (N(N-1)/2 reciprocal, N(N-1) general)
    bool general = false;
    std::vector<int64_t> d, roff;  // tile sizes d_i; roff[i] = first row of block i (roff[N] = nr)
    std::vector<int> kd, kp;
    std::vector<uint8_t> dense;
    std::vector<int64_t> off_diag, off_l, off_r;   // general low-rank diagonal: L_ii at off_diag, R_ii after it
    int64_t ntheta = 0;
    // expand side (A): columns 0 .. Ktot-1
    std::vector<int> Kb;
    std::vector<int64_t> Koff;
    // compress side (B): columns 0 .. KtotB-1 (the rows of T)
    std::vector<int> KbB;
    std::vector<int64_t> KoffB;
    std::vector<int64_t> panA, panB;   // panel offset of block i's A / B panel
    std::vector<int> dslot;   // dense slot of block i or -1
    int64_t Ktot = 0, KtotB = 0, ncol = 0, nlr = 0, ndense = 0, nth = 0;
    // maps (host copies): partner[A column] = row of T (B column); partnerB[B column] = row of V (A column)
    std::vector<int> partner, partnerB, colstride, panstride, colrows, zdim;
    std::vector<long long> colsrc, colpan, zsrc, zoff;   // zoff[slot]: dense tile offset after the low-rank panels
};

int build_layout(const tlr_mdd_desc_t* d, Layout& L, std::string& err) {
    if (!d) {
        err = "desc is NULL";
        return TLR_ERR_ARG;
    }
    if (d->nr <= 0 || d->ns <= 0 || (!d->tiles && d->tile <= 0)) {
        err = "nr, ns and tile must be positive";
        return TLR_ERR_SHAPE;
    }
    if (d->nr > (int64_t)1 << 30 || d->ns > (int64_t)1 << 30) {
        err = "nr and ns must be below 2^30";
        return TLR_ERR_SHAPE;
    }
    if (d->tiles) {
        if (d->ntiles <= 0 || d->ntiles > d->nr) {
            err = "ntiles must lie in [1, nr]";
            return TLR_ERR_SHAPE;
        }
        int64_t sum = 0;
        for (int i = 0; i < d->ntiles; ++i) {
            if (d->tiles[i] <= 0) {
                err = "tile sizes must be positive";
                return TLR_ERR_SHAPE;
            }
            sum += d->tiles[i];
        }
        if (sum != d->nr) {
            err = "tile sizes must sum to nr";
            return TLR_ERR_SHAPE;
        }
    } else if (d->nr % d->tile != 0) {
        err = "tile must divide nr (uniform partition)";
        return TLR_ERR_SHAPE;
    }
    if (d->reciprocity != TLR_RECIP_SYMMETRIC && d->reciprocity != TLR_RECIP_NONE) {
        err = "unknown reciprocity mode";
        return TLR_ERR_ARG;
    }
    if (d->precision != TLR_PREC_FP32 && d->precision != TLR_PREC_BF16X3 && d->precision != TLR_PREC_TF32) {
        err = "unknown precision mode";
        return TLR_ERR_ARG;
    }
    L.nr = d->nr;
    L.ns = d->ns;
    L.N = d->tiles ? d->ntiles : (int)(d->nr / d->tile);
    L.d.assign(L.N, d->tiles ? 0 : d->tile);
    if (d->tiles)
        for (int i = 0; i < L.N; ++i) L.d[i] = d->tiles[i];
    L.roff.assign(L.N + 1, 0);
    for (int i = 0; i < L.N; ++i) L.roff[i + 1] = L.roff[i] + L.d[i];
    L.dmax = *std::max_element(L.d.begin(), L.d.end());
    L.b = std::all_of(L.d.begin(), L.d.end(), [&](int64_t x) { return x == L.d[0]; }) ? L.d[0] : 0;
    L.general = d->reciprocity == TLR_RECIP_NONE;
    L.P = L.general ? L.N * (L.N - 1) : L.N * (L.N - 1) / 2;
    const int N = L.N, P = L.P;
    // row / column block of every stored pair, in stacking order
    std::vector<int> prow(P), pcol(P);
    {
        int p = 0;
        for (int j = 0; j < N; ++j)
            for (int i = L.general ? 0 : j + 1; i < N; ++i) {
                if (i == j) continue;
                prow[p] = i;
                pcol[p] = j;
                ++p;
            }
    }
    L.kd.assign(N, d->rank);
    L.kp.assign(P, d->rank);
    if (d->ranks) {
        for (int i = 0; i < N; ++i) L.kd[i] = d->ranks[i];
        for (int p = 0; p < P; ++p) L.kp[p] = d->ranks[N + p];
    }
    for (int i = 0; i < N; ++i)
        if (L.kd[i] < 0 || L.kd[i] > L.d[i]) {
            err = "rank outside [0, tile]";
            return TLR_ERR_SHAPE;
        }
    for (int p = 0; p < P; ++p)
        if (L.kp[p] < 0 || L.kp[p] > std::min(L.d[prow[p]], L.d[pcol[p]])) {
            err = "rank outside [0, tile]";
            return TLR_ERR_SHAPE;
        }
    L.dense.assign(N, 0);
    for (int i = 0; i < N; ++i) {
        switch (d->diag_mode) {
            case TLR_DIAG_RULE: L.dense[i] = (4LL * L.kd[i] >= L.d[i]); break;
            case TLR_DIAG_LOWRANK: L.dense[i] = 0; break;
            case TLR_DIAG_DENSE: L.dense[i] = 1; break;
            case TLR_DIAG_PER_TILE:
                if (!d->diag_dense) {
                    err = "diag_dense is NULL with TLR_DIAG_PER_TILE";
                    return TLR_ERR_ARG;
                }
                L.dense[i] = d->diag_dense[i] != 0;
                break;
            default: err = "unknown diag_mode"; return TLR_ERR_ARG;
        }
    }
    // theta (paper stacking): diagonal blocks, then L-bar, then R-bar (general
    // form: the ordered pairs (i, j), i != j, column j outer, row i inner)
    // (L_ij: d_i x k, R_ij: d_j x k; diagonal blocks d_i x k or d_i x d_i)
    int64_t o = 0;
    L.off_diag.resize(N);
    for (int i = 0; i < N; ++i) {
        L.off_diag[i] = o;
        o += L.d[i] * (L.dense[i] ? L.d[i] : (L.general ? 2 : 1) * L.kd[i]);
    }
    L.off_l.resize(P);
    L.off_r.resize(P);
    for (int p = 0; p < P; ++p) {
        L.off_l[p] = o;
        o += L.d[prow[p]] * L.kp[p];
    }
    for (int p = 0; p < P; ++p) {
        L.off_r[p] = o;
        o += L.d[pcol[p]] * L.kp[p];
    }
    L.ntheta = o;

    // panels.  Factor lists per block: (theta offset, rank, partner factor id).
    struct Fac {
        int id;
        int64_t off;
        int k;
        int partner;
    };
    std::vector<std::vector<Fac>> blkA(N), blkB(N);
    if (!L.general) {
        // pair index p(i, j) = j N - j(j+1)/2 + (i - j - 1), i > j; factor ids:
        // Q_i -> i ; L_p -> N + p ; R_p -> N + P + p
        auto pidx = [N](int i, int j) { return j * N - j * (j + 1) / 2 + (i - j - 1); };
        for (int i = 0; i < N; ++i) {
            if (!L.dense[i] && L.kd[i] > 0) blkA[i].push_back({i, L.off_diag[i], L.kd[i], i});
            for (int j = 0; j < i; ++j) {
                const int p = pidx(i, j);
                if (L.kp[p] > 0) blkA[i].push_back({N + p, L.off_l[p], L.kp[p], N + P + p});
            }
            for (int j = i + 1; j < N; ++j) {
                const int p = pidx(j, i);
                if (L.kp[p] > 0) blkA[i].push_back({N + P + p, L.off_r[p], L.kp[p], N + p});
            }
        }
    } else {
        // ordered pair index of tile (r, c), r != c: c (N - 1) + r - (r > c); factor
        // ids: L of tile t -> t, R of tile t -> N^2 + t with t = r N + c.  Y = X^T Dfrak:
        // row block i of Y takes R_ji (A side of block i), column block j of Dfrak
        // is compressed by L_ji (B side of block j).
        auto op = [N](int r, int c) { return c * (N - 1) + r - (r > c ? 1 : 0); };
        const int NN = N * N;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const int t = j * N + i;   // tile (j, i)
                int k;
                int64_t offL, offR;
                if (i == j) {
                    if (L.dense[i] || L.kd[i] == 0) continue;
                    k = L.kd[i];
                    offL = L.off_diag[i];
                    offR = L.off_diag[i] + L.d[i] * k;
                } else {
                    const int q = op(j, i);
                    k = L.kp[q];
                    if (k == 0) continue;
                    offL = L.off_l[q];
                    offR = L.off_r[q];
                }
                blkA[i].push_back({NN + t, offR, k, t});
                blkB[j].push_back({t, offL, k, NN + t});
            }
    }
    // columns: A side first (0 .. Ktot-1), then B side (general form only)
    const int nid = L.general ? 2 * N * N : N + 2 * P;
    std::vector<int64_t> fac_col(nid, -1), fac_b(nid, -1);
    L.Kb.assign(N, 0);
    L.Koff.assign(N, 0);
    int64_t K = 0;
    for (int i = 0; i < N; ++i) {
        L.Koff[i] = K;
        for (auto& f : blkA[i]) {
            fac_col[f.id] = K + L.Kb[i];
            L.Kb[i] += f.k;
        }
        K += L.Kb[i];
    }
    L.Ktot = K;
    if (L.general) {
        L.KbB.assign(N, 0);
        L.KoffB.assign(N, 0);
        int64_t KB = 0;
        for (int j = 0; j < N; ++j) {
            L.KoffB[j] = KB;
            for (auto& f : blkB[j]) {
                fac_b[f.id] = KB + L.KbB[j];
                L.KbB[j] += f.k;
            }
            KB += L.KbB[j];
        }
        L.KtotB = KB;
    } else {
        L.KbB = L.Kb;
        L.KoffB = L.Koff;
        L.KtotB = L.Ktot;
    }
    L.ncol = L.general ? L.Ktot + L.KtotB : L.Ktot;
    // panel i: d_i x K_i row-major; A panels first, then (general form) B panels
    L.panA.assign(N, 0);
    L.panB.assign(N, 0);
    int64_t po = 0;
    for (int i = 0; i < N; ++i) {
        L.panA[i] = po;
        po += L.d[i] * L.Kb[i];
    }
    if (L.general)
        for (int j = 0; j < N; ++j) {
            L.panB[j] = po;
            po += L.d[j] * L.KbB[j];
        }
    else
        L.panB = L.panA;
    L.nlr = po;
    L.partner.resize(L.Ktot);
    L.partnerB.resize(L.KtotB);
    L.colsrc.resize(L.ncol);
    L.colstride.resize(L.ncol);
    L.colpan.resize(L.ncol);
    L.panstride.resize(L.ncol);
    L.colrows.resize(L.ncol);
    for (int i = 0; i < N; ++i) {
        int64_t c = 0;
        for (auto& f : blkA[i]) {
            for (int q = 0; q < f.k; ++q) {
                const int64_t g = L.Koff[i] + c + q;
                L.partner[g] = (int)((L.general ? fac_b[f.partner] : fac_col[f.partner]) + q);
                L.colsrc[g] = f.off + q;
                L.colstride[g] = f.k;
                L.colpan[g] = L.panA[i] + c + q;
                L.panstride[g] = L.Kb[i];
                L.colrows[g] = (int)L.d[i];
            }
            c += f.k;
        }
    }
    if (L.general) {
        for (int j = 0; j < N; ++j) {
            int64_t c = 0;
            for (auto& f : blkB[j]) {
                for (int q = 0; q < f.k; ++q) {
                    const int64_t g = L.KoffB[j] + c + q;
                    L.partnerB[g] = (int)(fac_col[f.partner] + q);
                    L.colsrc[L.Ktot + g] = f.off + q;
                    L.colstride[L.Ktot + g] = f.k;
                    L.colpan[L.Ktot + g] = L.panB[j] + c + q;
                    L.panstride[L.Ktot + g] = L.KbB[j];
                    L.colrows[L.Ktot + g] = (int)L.d[j];
                }
                c += f.k;
            }
        }
    } else {
        L.partnerB = L.partner;
    }
    L.dslot.assign(N, -1);
    int64_t zo = 0;
    for (int i = 0; i < N; ++i)
        if (L.dense[i]) {
            L.dslot[i] = (int)L.ndense++;
            L.zsrc.push_back(L.off_diag[i]);
            L.zoff.push_back(zo);
            L.zdim.push_back((int)L.d[i]);
            zo += L.d[i] * L.d[i];
        }
    L.nth = L.nlr + zo;
    if (L.nth != L.ntheta) {
        err = "internal: panel size differs from theta size";
        return TLR_ERR_STATE;
    }
    return TLR_OK;
}

int choose_split(long long tiles, long long K) {
    const long long target = 4LL * 152 * 2;
    long long s = (target + tiles - 1) / std::max(1LL, tiles);
    s = std::min(s, std::max(1LL, K / 256));
    s = std::max(1LL, std::min(s, 64LL));
    return (int)s;
}

}  // namespace

struct tlr_mdd_s {
    tlr_mdd_desc_t d{};
    cudaStream_t st = nullptr;
    Layout L;
    std::string err;
    // device arena
    char* arena = nullptr;
    size_t arena_bytes = 0;
    int32_t* perm = nullptr;   // 2 nr: perm, inverse
    double* scal = nullptr;    // [0] alpha
    double alpha = 0.0;
    cf *Dt = nullptr, *Ut = nullptr, *R = nullptr, *A1 = nullptr, *A2 = nullptr;
    cf *T = nullptr, *Tp = nullptr;   // Tp doubles as V
    cf *Zs = nullptr, *Zsd = nullptr;
    cf* part = nullptr;
    int nsplit = 1;
    int kchunk = 0;
    double* dpart = nullptr;   // reduction partial slabs
    int* d_partner = nullptr;    // [Ktot] row of T for each A column
    int* d_partnerB = nullptr;   // [KtotB] row of V for each B column (= d_partner when reciprocal)
    long long* d_roff = nullptr; // [N + 1] first row of each block
    PanelMap pm{};
    // theta-space vectors
    cf *x = nullptr, *z = nullptr, *u = nullptr, *v = nullptr, *g = nullptr, *gf = nullptr, *dd = nullptr,
       *q = nullptr;
    // solver small state
    double *rho_h = nullptr, *sy_h = nullptr, *yy_h = nullptr, *acoef = nullptr, *sc = nullptr, *fhist = nullptr;
    double *lbm = nullptr, *lbpart = nullptr;   // compact L-BFGS: S^T Y and Y^T Y by slot; partials
    int* ints = nullptr;
    // ring (allocated on first solve)
    float* ring = nullptr;
    int ring_m = 0;
    // GEMM tables
    GemmLaunch Lc_x, Lc_d, Lc_v, Le_fwd, Le_apply, Le_a1, Le_a2, Lp;
    char* tab_base = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // packed tensor-core path: packed operand storage, tables, static packs
    char* packed = nullptr;
    size_t packed_size = 0;
    char* tcp_tables = nullptr;
    PackJob* d_static_jobs = nullptr;
    int n_static_jobs = 0;
    long long static_items = 0;
    TPackTile* d_tpack = nullptr;      // fused update + packing of T (packs of T are not per-launch jobs)
    int n_tpack = 0;
    // fused residual step + packing of R (packs of R are not per-launch jobs when on)
    bool rstep_on = false;
    char** d_rkn = nullptr;            // [N] packed R_i (KN) for the residual compression
    char** d_rmk = nullptr;            // [N] packed R_i (MK) for the projection
    double* rpart = nullptr;           // per-CTA partials of ||R||^2
    long long n_rpart = 0;
    // asynchronous solve and its CUDA graph
    cf* th_io = nullptr;               // theta staging (stable address for the graph)
    HostStats* hstats = nullptr;       // pinned
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;       // kernel launches recorded in gexec
    int plain_solves = 0;              // solves enqueued as plain launches since the last recording
    GraphKey gkey;
    std::vector<TimedLaunch> gtimed;
    bool pending = false;
    bool pending_graph = false;
    void* pending_host_theta = nullptr;
};

#define FAIL(h, code, msg)                  \
    do {                                    \
        if (h) (h)->err = (msg);            \
        g_last_error = (msg);               \
        return (code);                      \
    } while (0)

#define CK(h, expr)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            std::string m_ = std::string(#expr) + ": " + cudaGetErrorString(e_);           \
            if (h) (h)->err = m_;                                                           \
            g_last_error = m_;                                                              \
            return e_ == cudaErrorMemoryAllocation ? TLR_ERR_NOMEM : TLR_ERR_CUDA;         \
        }                                                                                   \
    } while (0)

namespace {

// Lay out (or size, when a.base == nullptr) the handle's device arena.
void carve(tlr_mdd_s* h, Arena& a) {
    const Layout& L = h->L;
    // T has a row per B column; Tp holds T_p (B rows) or V (A rows)
    const size_t nrs = (size_t)L.nr * L.ns, kns = (size_t)std::max<int64_t>(1, L.KtotB) * L.ns;
    const size_t knsp = (size_t)std::max<int64_t>(1, std::max(L.Ktot, L.KtotB)) * L.ns;
    h->perm = a.take<int32_t>(2 * L.nr);
    h->scal = a.take<double>(16);
    h->Dt = a.take<cf>(nrs);
    h->Ut = a.take<cf>(nrs);
    h->R = a.take<cf>(nrs);
    h->A1 = a.take<cf>(nrs);
    h->A2 = a.take<cf>(nrs);
    h->T = a.take<cf>(kns);
    h->Tp = a.take<cf>(knsp);
    const size_t nz = std::max<size_t>(1, (size_t)(L.nth - L.nlr));
    h->Zs = a.take<cf>(nz);
    h->Zsd = a.take<cf>(nz);
    h->part = a.take<cf>((size_t)h->nsplit * L.nth);
    h->dpart = a.take<double>(16 * kRedBlocks);
    // the fused residual step works on 16-row tiles of one block each: every
    // tile size a multiple of 16
    h->n_rpart = std::all_of(L.d.begin(), L.d.end(), [](int64_t x) { return x % kFuseRows == 0; })
                     ? rstep_ctas((int)L.nr, (int)L.ns)
                     : 0;
    h->rpart = a.take<double>((size_t)std::max<long long>(1, h->n_rpart));
    const size_t K = std::max<int64_t>(1, L.ncol);
    h->d_partner = a.take<int>(std::max<int64_t>(1, L.general ? L.Ktot + L.KtotB : L.Ktot));
    h->d_partnerB = L.general ? h->d_partner + L.Ktot : h->d_partner;
    long long* colsrc = a.take<long long>(K);
    int* colstride = a.take<int>(K);
    long long* colpan = a.take<long long>(K);
    int* panstride = a.take<int>(K);
    int* colrows = a.take<int>(K);
    const size_t nd = std::max<int64_t>(1, L.ndense);
    long long* zsrc = a.take<long long>(nd);
    long long* zoff = a.take<long long>(nd);
    int* zdim = a.take<int>(nd);
    h->d_roff = a.take<long long>((size_t)L.N + 1);
    h->pm = PanelMap{colsrc, colstride, colpan, panstride, colrows, zsrc, zoff, zdim,
                     L.ncol, L.dmax, L.ndense, L.nlr};
    const size_t nth = std::max<int64_t>(1, L.nth);
    h->x = a.take<cf>(nth);
    h->z = a.take<cf>(nth);
    h->u = a.take<cf>(nth);
    h->v = a.take<cf>(nth);
    h->g = a.take<cf>(nth);
    h->gf = a.take<cf>(nth);
    h->dd = a.take<cf>(nth);
    h->q = a.take<cf>(nth);
    h->th_io = a.take<cf>(nth);
    h->rho_h = a.take<double>(64);
    h->sy_h = a.take<double>(64);
    h->yy_h = a.take<double>(64);
    h->acoef = a.take<double>(64);
    h->sc = a.take<double>(SC_COUNT + 8);
    h->ints = a.take<int>(SI_COUNT + 8);
    h->fhist = a.take<double>(TLR_MAX_HIST);
    h->lbm = a.take<double>(2 * 33 * 33);
    h->lbpart = a.take<double>((size_t)kLbPartDoubles);
    // GEMM tables: 8 slots of at most 3N + 1 problems each
    h->tab_base = reinterpret_cast<char*>(a.take<GProb>(3 * (size_t)L.N + 1));
    for (int t = 1; t < 8; ++t) a.take<GProb>(3 * (size_t)L.N + 1);
}

// Upper bound of the packed-operand storage of the tensor-core path (the
// distinct operands listed in build_tc; 1 KB alignment per operand).
long long packed_estimate(const Layout& L) {
    auto pb = [](long long R, long long K, int TR) { return (packed_bytes(R, K, TR) + 1023) & ~1023LL; };
    const long long ns = L.ns;
    long long t = 0;
    for (int i = 0; i < L.N; ++i) {
        const long long b = L.d[i];
        const long long Ki = std::max(L.Kb[i], L.KbB[i]);   // upper bound for both sides
        if (Ki > 0) {
            t += 3 * pb(Ki, b, kPackTRA) + 2 * pb(b, Ki, kPackTRA);     // F, conj F, F_d (KM); F, F_d (MK)
            t += 2 * pb(ns, Ki, kPackTRB) + 2 * pb(Ki, ns, kPackTRB);   // T~, T~_p (KN); conj T~, V~ (NK)
            t += pb(ns, b, kPackTRB);                              // Rf_i (KN)
        }
        if (Ki > 0 || L.dense[i]) t += pb(ns, b, kPackTRB) + 2 * pb(b, ns, kPackTRA);   // Dfrak_i (KN); Rf_i, conj Dfrak_i (MK)
        if (L.dense[i]) t += 2 * pb(b, b, kPackTRA) + pb(b, ns, kPackTRB);              // Zs, Zs_d; conj Dfrak_i (NK)
    }
    return t;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 152;
    }
    return n;
}

// Split of the contraction over ns in the gradient projection.  SIMT path:
// enough 64 x 64 tiles for a few waves.  Tensor-core path: the split s that
// minimises the modelled time ceil(tiles s / SMs) (ns / s + c0) of 128 x 128
// tiles, c0 = 128 standing for a tile's fixed cost (set-up, pipeline fill,
// epilogue) in units of contraction depth; this avoids a short last wave.
int split_for(const Layout& L, int prec) {
    if (tensor_core(prec)) {
        long long tiles = 0;
        for (int i = 0; i < L.N; ++i) {
            const long long b = L.d[i];
            tiles += ((b + kPackTRA - 1) / kPackTRA) * ((L.Kb[i] + kPackTRB - 1) / kPackTRB);
            if (L.general) tiles += ((b + kPackTRA - 1) / kPackTRA) * ((L.KbB[i] + kPackTRB - 1) / kPackTRB);
            if (L.dense[i]) tiles += ((b + kPackTRA - 1) / kPackTRA) * ((b + kPackTRB - 1) / kPackTRB);
        }
        tiles = std::max(1LL, tiles);
        const long long sms = sm_count(), smax = std::max(1LL, std::min(16LL, (long long)L.ns / 256));
        long long best = 1;
        double tbest = 1e300;
        for (long long sp = 1; sp <= smax; ++sp) {
            const double t = (double)((tiles * sp + sms - 1) / sms) * ((double)L.ns / sp + 128.0);
            if (t < tbest * 0.999) {
                tbest = t;
                best = sp;
            }
        }
        return (int)best;
    }
    long long tiles = 0;
    for (int i = 0; i < L.N; ++i) {
        const long long b = L.d[i];
        tiles += ((b + 63) / 64) * ((L.Kb[i] + 63) / 64);
        if (L.general) tiles += ((b + 63) / 64) * ((L.KbB[i] + 63) / 64);
        if (L.dense[i]) tiles += ((b + 63) / 64) * ((b + 63) / 64);
    }
    return choose_split(std::max(1LL, tiles), L.ns);
}

GTerm term(const cf* A, long long lda, const cf* B, long long ldb, const int* g, int K, bool conjA, bool conjB) {
    GTerm t;
    t.A = A;
    t.B = B;
    t.g = g;
    t.lda = lda;
    t.ldb = ldb;
    t.K = K;
    t.sa = conjA ? -1.f : 1.f;
    t.sb = conjB ? -1.f : 1.f;
    return t;
}

struct HostTable {
    GemmLaunch* G;
    std::vector<GProb> v;
};

// Build the grouped problems for every contraction of the handle and upload.
int build_tables(tlr_mdd_s* h, char* tab_base, std::vector<HostTable>* keep) {
    const Layout& L = h->L;
    const long long ns = L.ns;
    const size_t slot = ((sizeof(GProb) * (3 * (size_t)L.N + 1)) + 255) & ~size_t(255);
    int ti = 0;
    auto upload = [&](GemmLaunch& G, std::vector<GProb>& v, int am, int bm, int epi) -> int {
        GProb* dst = reinterpret_cast<GProb*>(tab_base + slot * ti++);
        G.d_probs = dst;
        G.nprob = (int)v.size();
        G.amode = am;
        G.bmode = bm;
        G.epi = epi;
        G.maxM = G.maxN = G.maxK = 0;
        G.flops = 0.0;
        for (auto& p : v) {
            G.maxM = std::max(G.maxM, p.M);
            G.maxN = std::max(G.maxN, p.N);
            for (int t = 0; t < p.nt; ++t) G.flops += 8.0 * p.M * (double)p.N * p.t[t].K;
        }
        G.cls = am == A_KM ? 0 : (bm == B_KN ? 1 : 2);
        G.prec = h->d.precision;
        G.persistent = tensor_core(G.prec) && ((persist_classes() >> G.cls) & 1);
        G.err = h->ints + SI_COUNT + 1;
        if (!v.empty()) {
            cudaError_t e = cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(GProb), cudaMemcpyHostToDevice, h->st);
            if (e != cudaSuccess) return -1;
        }
        if (keep) keep->push_back(HostTable{&G, v});
        return 0;
    };
    auto blank = []() {
        GProb p;
        memset(&p, 0, sizeof(p));
        return p;
    };
    const cf* X = h->x;
    const cf* Dd = h->dd;
    // compress: T_j = B_j^T Dfrak_j (src x), T_p (src d) over the B panels;
    // V_i = A_i^H Rf_i (into Tp) over the A panels
    for (int which = 0; which < 3; ++which) {
        std::vector<GProb> v;
        const bool aside = which == 2;
        for (int i = 0; i < L.N; ++i) {
            const int Ki = aside ? L.Kb[i] : L.KbB[i];
            if (Ki == 0) continue;
            GProb p = blank();
            const cf* src = which == 1 ? Dd : X;
            const cf* data = which == 2 ? h->R : h->Dt;
            cf* out = which == 0 ? h->T : h->Tp;
            p.t[0] = term(src + (aside ? L.panA[i] : L.panB[i]), Ki, data + L.roff[i] * ns, ns, nullptr, (int)L.d[i],
                          which == 2, false);
            p.nt = 1;
            p.M = Ki;
            p.N = (int)ns;
            p.C = out + (aside ? L.Koff[i] : L.KoffB[i]) * ns;
            p.ldc = ns;
            v.push_back(p);
        }
        GemmLaunch& G = which == 0 ? h->Lc_x : (which == 1 ? h->Lc_d : h->Lc_v);
        if (upload(G, v, A_KM, B_KN, EPI_STORE)) return -1;
    }
    // expand: forward residual (SUB Ufrak), plain apply (STORE), A1, A2.  The
    // line-search pair runs as one grouped launch, block i's A1 problem next to
    // its A2 problem (both read T~_p,i, which then comes from L2 the second
    // time): their tiles share the operand packs and one launch fills the last
    // wave better than two; Le_a2 stays empty.
    std::vector<GProb> a12;
    for (int which = 0; which < 4; ++which) {
        std::vector<GProb> v;
        for (int i = 0; i < L.N; ++i) {
            GProb p = blank();
            const int* gi = h->d_partner + L.Koff[i];
            const int Ki = L.Kb[i];
            const cf* Fi = X + L.panA[i];
            const cf* Fd = Dd + L.panA[i];
            const long long b = L.d[i];
            const cf* Di = h->Dt + L.roff[i] * ns;
            const long long zo = L.dense[i] ? L.zoff[L.dslot[i]] : 0;
            int nt = 0;
            if (which <= 1) {
                if (Ki > 0) p.t[nt++] = term(Fi, Ki, h->T, ns, gi, Ki, false, false);
                if (L.dense[i]) p.t[nt++] = term(h->Zs + zo, b, Di, ns, nullptr, (int)b, false, false);
            } else if (which == 2) {
                if (Ki > 0) {
                    p.t[nt++] = term(Fd, Ki, h->T, ns, gi, Ki, false, false);
                    p.t[nt++] = term(Fi, Ki, h->Tp, ns, gi, Ki, false, false);
                }
                if (L.dense[i]) p.t[nt++] = term(h->Zsd + zo, b, Di, ns, nullptr, (int)b, false, false);
            } else {
                if (Ki > 0) p.t[nt++] = term(Fd, Ki, h->Tp, ns, gi, Ki, false, false);
            }
            p.nt = nt;
            p.M = (int)b;
            p.N = (int)ns;
            cf* out = which <= 1 ? h->R : (which == 2 ? h->A1 : h->A2);
            p.C = out + L.roff[i] * ns;
            p.S = h->Ut + L.roff[i] * ns;
            p.ldc = ns;
            v.push_back(p);
        }
        if (which == 2) {
            a12 = v;
            continue;
        }
        if (which == 3) {
            std::vector<GProb> a1 = a12;
            a12.clear();
            for (size_t i = 0; i < v.size(); ++i) {
                a12.push_back(a1[i]);
                a12.push_back(v[i]);
            }
            std::vector<GProb> none;
            if (upload(h->Le_a1, a12, A_MK, B_KN, EPI_STORE)) return -1;
            if (upload(h->Le_a2, none, A_MK, B_KN, EPI_STORE)) return -1;
            continue;
        }
        GemmLaunch& G = which == 0 ? h->Le_fwd : h->Le_apply;
        if (upload(G, v, A_MK, B_KN, which == 0 ? EPI_SUB : EPI_STORE)) return -1;
    }
    // project: split-K partials of grad F_i and G_ii
    {
        std::vector<GProb> v;
        for (int i = 0; i < L.N; ++i) {
            const long long b = L.d[i];
            const cf* Ri = h->R + L.roff[i] * ns;
            const cf* Di = h->Dt + L.roff[i] * ns;
            if (!L.general && L.Kb[i] > 0) {
                // reciprocal: block i's panel takes both terms
                GProb p = blank();
                const int* gi = h->d_partner + L.Koff[i];
                p.t[0] = term(Ri, ns, h->T, ns, gi, (int)ns, false, true);
                p.t[1] = term(Di, ns, h->Tp, ns, gi, (int)ns, true, false);
                p.nt = 2;
                p.M = (int)b;
                p.N = L.Kb[i];
                p.C = h->part + L.panA[i];
                p.ldc = L.Kb[i];
                v.push_back(p);
            }
            if (L.general && L.Kb[i] > 0) {   // A panel i: Rf_i T~_i^H
                GProb p = blank();
                p.t[0] = term(Ri, ns, h->T, ns, h->d_partner + L.Koff[i], (int)ns, false, true);
                p.nt = 1;
                p.M = (int)b;
                p.N = L.Kb[i];
                p.C = h->part + L.panA[i];
                p.ldc = L.Kb[i];
                v.push_back(p);
            }
            if (L.general && L.KbB[i] > 0) {   // B panel i: conj(Dfrak_i) V~_i^T
                GProb p = blank();
                p.t[0] = term(Di, ns, h->Tp, ns, h->d_partnerB + L.KoffB[i], (int)ns, true, false);
                p.nt = 1;
                p.M = (int)b;
                p.N = L.KbB[i];
                p.C = h->part + L.panB[i];
                p.ldc = L.KbB[i];
                v.push_back(p);
            }
            if (L.dense[i]) {
                GProb p = blank();
                p.t[0] = term(Ri, ns, Di, ns, nullptr, (int)ns, false, true);
                p.nt = 1;
                p.M = (int)b;
                p.N = (int)b;
                p.C = h->part + L.nlr + L.zoff[L.dslot[i]];
                p.ldc = b;
                v.push_back(p);
            }
        }
        if (upload(h->Lp, v, A_MK, B_NK, EPI_PARTIAL)) return -1;
        h->Lp.nsplit = h->nsplit;
        h->Lp.kchunk = h->kchunk;
        h->Lp.part_stride = L.nth;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Packed tensor-core plan.  Every operand of every tensor-core contraction is
// written once per use into the packed BF16-plane tile format by a pack job
// that runs just before the contraction; identical operands (same source,
// layout, gather, conjugation and shape) share one packed buffer.  Operands
// read from the data panel Dfrak never change during a solve: they are packed
// once when the data are loaded.  The line-search pair A1 / A2 shares its
// packs (A2 packs nothing).  The two packings of the factor products T (KN for
// the expansions, conjugated NK for the projection) are written by tpack right
// after T is formed or updated, and the residual's two packings by the fused
// residual step (rstep), so no contraction packs them.
// ---------------------------------------------------------------------------
struct PackKey {
    const void* src;
    long long ld;
    const void* gr;
    const void* gk;
    int kcontig, R, K, TR;
    float sgn;
    bool operator<(const PackKey& o) const {
        return std::tie(src, ld, gr, gk, kcontig, R, K, TR, sgn) <
               std::tie(o.src, o.ld, o.gr, o.gk, o.kcontig, o.R, o.K, o.TR, o.sgn);
    }
};

int build_tc(tlr_mdd_s* h, std::vector<HostTable>& tabs) {
    const Layout& L = h->L;
    const char* dlo = reinterpret_cast<const char*>(h->Dt);
    const char* dhi = dlo + (size_t)L.nr * L.ns * sizeof(cf);
    std::map<PackKey, size_t> offs;   // key -> byte offset in the packed arena
    std::vector<std::pair<PackKey, size_t>> order;
    size_t total = 0;
    auto key_of = [](const GTerm& t, bool isA, int amode, int bmode, int R) {
        PackKey k{};
        if (isA) {
            k.src = t.A;
            k.ld = t.lda;
            k.kcontig = amode == A_MK;
            k.sgn = t.sa;
            k.TR = kPackTRA;
        } else {
            k.src = t.B;
            k.ld = t.ldb;
            k.kcontig = bmode == B_NK;
            if (k.kcontig)
                k.gr = t.g;
            else
                k.gk = t.g;
            k.sgn = t.sb;
            k.TR = kPackTRB;
        }
        k.R = R;
        k.K = t.K;
        return k;
    };
    auto place = [&](const PackKey& k) -> size_t {
        auto it = offs.find(k);
        if (it != offs.end()) return it->second;
        const size_t o = total;
        offs[k] = o;
        order.push_back({k, o});
        total += (size_t)((packed_bytes(k.R, k.K, k.TR) + 1023) & ~1023LL);
        return o;
    };
    // pass 1: storage
    for (auto& T : tabs)
        for (auto& p : T.v)
            for (int t = 0; t < p.nt; ++t) {
                place(key_of(p.t[t], true, T.G->amode, T.G->bmode, p.M));
                place(key_of(p.t[t], false, T.G->amode, T.G->bmode, p.N));
            }
    h->packed_size = total;
    CK(h, ws_alloc((void**)&h->packed, std::max<size_t>(total, 256), h->st));
    // padding rows and k-slots of every packed operand stay zero from here on
    CK(h, cudaMemsetAsync(h->packed, 0, std::max<size_t>(total, 256), h->st));
    auto job_of = [&](const PackKey& k, size_t off) {
        PackJob j;
        j.src = (const cf*)k.src;
        j.ld = k.ld;
        j.g_row = (const int*)k.gr;
        j.g_k = (const int*)k.gk;
        j.kcontig = k.kcontig;
        j.sgn = k.sgn;
        j.R = k.R;
        j.K = k.K;
        j.TR = k.TR;
        j.dst = h->packed + off;
        j.fmt = pack_fmt(h->d.precision);
        return j;
    };
    // (padded rows << 32) | k-groups of 8; the launch grid covers the maximum of each
    auto items_of = [](const PackKey& k) {
        const long long nkc = (k.K + 15) / 16, nrb = (k.R + k.TR - 1) / k.TR;
        return ((nrb * k.TR) << 32) | (nkc * 2);
    };
    auto merge = [](long long a, long long b) {
        return (std::max(a >> 32, b >> 32) << 32) | std::max(a & 0xffffffffLL, b & 0xffffffffLL);
    };
    auto is_static = [&](const PackKey& k) {
        const char* c = reinterpret_cast<const char*>(k.src);
        return c >= dlo && c < dhi;
    };
    // The projection reads V~_i (V's rows gathered by partner, NK) only in
    // packed form: the compression V = F^H Rf writes it there directly
    // (EPI_PACKNK), so V is never stored in FP32 and never packed by a job.
    // Row g of V is row k = partner[g] - Koff[i] of V~_i, i the block of partner[g].
    std::map<const void*, size_t> v_nk;   // gather of block i -> packed V~_i (NK)
    for (auto& ko : order)
        if (ko.first.src == (const void*)h->Tp && ko.first.kcontig == 1 && ko.first.sgn > 0)
            v_nk[ko.first.gr] = ko.second;
    // The residual's two packings (MK for the projection, KN for the residual
    // compression) come from the fused residual step when every tile size is a
    // multiple of kFuseRows and every block has both.
    const char* rlo = reinterpret_cast<const char*>(h->R);
    const char* rhi = rlo + (size_t)L.nr * L.ns * sizeof(cf);
    auto is_R = [&](const PackKey& k) {
        const char* c = reinterpret_cast<const char*>(k.src);
        return c >= rlo && c < rhi;
    };
    std::vector<char*> rkn(L.N, nullptr), rmk(L.N, nullptr);
    std::set<PackKey> rkeys;
    for (auto& ko : order) {
        const PackKey& k = ko.first;
        if (!is_R(k) || k.gr || k.gk || k.sgn < 0 || k.ld != L.ns) continue;
        const long long off = reinterpret_cast<const cf*>(k.src) - h->R;
        if (off % L.ns != 0) continue;
        const auto at = std::lower_bound(L.roff.begin(), L.roff.end() - 1, off / L.ns);
        if (at == L.roff.end() - 1 || *at != off / L.ns) continue;
        const long long blk = at - L.roff.begin(), db = L.d[blk];
        if (k.kcontig == 0 && k.R == L.ns && k.K == db) {
            rkn[blk] = h->packed + ko.second;
            rkeys.insert(k);
        }
        if (k.kcontig == 1 && k.R == db && k.K == L.ns) {
            rmk[blk] = h->packed + ko.second;
            rkeys.insert(k);
        }
    }
    bool rfuse = h->n_rpart > 0;
    for (int i = 0; i < L.N && rfuse; ++i)
        if (!rkn[i] || !rmk[i]) rfuse = false;
    std::vector<char*> rowptr;
    bool vpack = L.Ktot > 0;
    for (int j = 0; j < L.N && vpack; ++j)
        if (L.KbB[j] > 0 && !v_nk.count(h->d_partnerB + L.KoffB[j])) vpack = false;
    if (vpack) {
        constexpr long long plane = 128 * 16 * 2;
        const long long nkcN = (L.ns + 15) / 16;
        rowptr.resize(L.Ktot);
        for (int64_t gm = 0; gm < L.Ktot; ++gm) {
            // V row gm (A column) is read by B column partner[gm] of V~
            const int64_t pg = L.partner[gm];
            const int i = (int)(std::upper_bound(L.KoffB.begin(), L.KoffB.end(), pg) - L.KoffB.begin()) - 1;
            const int64_t k = pg - L.KoffB[i];
            // the row's first 16-byte group in its packed tile (row groups of
            // 8 are 256 B apart in the BF16 planes, 512 B in the TF32 planes)
            const long long rg = h->d.precision == TLR_PREC_TF32 ? 512 : 256;
            rowptr[gm] = h->packed + v_nk[h->d_partnerB + L.KoffB[i]] + (k >> 7) * nkcN * 4 * plane +
                         ((k & 127) >> 3) * rg + (k & 7) * 16;
        }
    }
    std::vector<std::pair<size_t, int64_t>> vfix;   // (problem index in Lc_v, Koff of its block)
    // pass 2: problems on packed operands and per-launch pack jobs
    std::vector<std::vector<PProb>> pp(tabs.size());
    std::vector<std::vector<PackJob>> jobs(tabs.size());
    std::vector<long long> maxit(tabs.size(), 0);
    std::vector<PackJob> sjobs;
    long long smax = 0;
    std::set<PackKey> static_done;
    std::set<PackKey> a1_keys;
    std::map<const void*, size_t> t_kn, t_nk;   // gather of block i -> packed T~_i (KN), conj T~_i (NK)
    std::map<const void*, std::pair<size_t, int>> tp_kn;   // gather of block i -> packed T~_p,i (KN), K_i
    auto is_T = [&](const PackKey& k) { return k.src == (const void*)h->T; };
    for (size_t ti = 0; ti < tabs.size(); ++ti) {
        auto& T = tabs[ti];
        std::set<PackKey> here;
        for (auto& p : T.v) {
            PProb q;
            memset(&q, 0, sizeof(q));
            q.nt = p.nt;
            q.M = p.M;
            q.N = p.N;
            q.C = p.C;
            q.S = p.S;
            q.ldc = p.ldc;
            for (int t = 0; t < p.nt; ++t) {
                const PackKey ka = key_of(p.t[t], true, T.G->amode, T.G->bmode, p.M);
                const PackKey kb = key_of(p.t[t], false, T.G->amode, T.G->bmode, p.N);
                q.t[t].A = h->packed + offs[ka];
                q.t[t].B = h->packed + offs[kb];
                q.t[t].K = p.t[t].K;
                for (const PackKey* k : {&ka, &kb}) {
                    if (vpack && k->src == (const void*)h->Tp && k->kcontig == 1) continue;   // written by Lc_v
                    if (T.G == &h->Le_a1 && k->src == (const void*)h->Tp && k->kcontig == 0 && k->gk &&
                        k->sgn > 0 && k->ld == L.ns && k->R == L.ns) {
                        tp_kn[k->gk] = std::make_pair(offs[*k], k->K);   // gathered pack of T_p (tpack)
                        continue;
                    }
                    if (rfuse && rkeys.count(*k)) continue;                                    // written by rstep
                    if (is_T(*k)) {
                        if (k->kcontig == 0 && k->sgn > 0)
                            t_kn[k->gk] = offs[*k];
                        else if (k->kcontig == 1 && k->sgn < 0)
                            t_nk[k->gr] = offs[*k];
                        else
                            FAIL(h, TLR_ERR_STATE, "internal: unexpected packing of T");
                        continue;
                    }
                    if (is_static(*k)) {
                        if (static_done.insert(*k).second) {
                            sjobs.push_back(job_of(*k, offs[*k]));
                            smax = merge(smax, items_of(*k));
                        }
                    } else if (here.insert(*k).second) {
                        if (T.G == &h->Le_a2 && a1_keys.count(*k)) continue;   // packed for A1 already
                        jobs[ti].push_back(job_of(*k, offs[*k]));
                        maxit[ti] = merge(maxit[ti], items_of(*k));
                    }
                }
            }
            if (vpack && T.G == &h->Lc_v) vfix.push_back({pp[ti].size(), (int64_t)((p.C - h->Tp) / L.ns)});
            pp[ti].push_back(q);
        }
        if (T.G == &h->Le_a1) a1_keys = here;
    }
    // upload: one allocation for all tables
    size_t bytes = 0;
    std::vector<size_t> po(tabs.size()), jo(tabs.size());
    for (size_t ti = 0; ti < tabs.size(); ++ti) {
        po[ti] = bytes;
        bytes += (pp[ti].size() * sizeof(PProb) + 255) & ~size_t(255);
        jo[ti] = bytes;
        bytes += (jobs[ti].size() * sizeof(PackJob) + 255) & ~size_t(255);
    }
    std::vector<TPackTile> tt;
    for (int i = 0; i < L.N; ++i) {
        const int Ki = L.Kb[i];
        if (Ki == 0) continue;
        const int* gi = h->d_partner + L.Koff[i];
        auto a = t_kn.find(gi), c = t_nk.find(gi);
        if (a == t_kn.end() || c == t_nk.end()) FAIL(h, TLR_ERR_STATE, "internal: T packing not planned");
        for (int k0 = 0; k0 < Ki; k0 += kFuseRows) {
            TPackTile t;
            t.g = gi;
            t.k0 = k0;
            t.nk = std::min(kFuseRows, Ki - k0);
            t.Ki = Ki;
            t.kn = h->packed + a->second;
            t.nk_dst = h->packed + c->second;
            t.fmt = pack_fmt(h->d.precision);
            tt.push_back(t);
        }
    }
    // the line-search expansion's gathered packs of T_p (KN only): tpack's
    // packing phase on 16-row tiles instead of per-element pack jobs
    std::vector<TPackTile> ttp;
    for (auto& kv : tp_kn) {
        const int Ki = kv.second.second;
        for (int k0 = 0; k0 < Ki; k0 += kFuseRows) {
            TPackTile t;
            t.g = (const int*)kv.first;
            t.k0 = k0;
            t.nk = std::min(kFuseRows, Ki - k0);
            t.Ki = Ki;
            t.kn = h->packed + kv.second.first;
            t.nk_dst = nullptr;
            t.fmt = pack_fmt(h->d.precision);
            ttp.push_back(t);
        }
    }
    const size_t tpo = bytes;
    bytes += (ttp.size() * sizeof(TPackTile) + 255) & ~size_t(255);
    const size_t so = bytes;
    bytes += (sjobs.size() * sizeof(PackJob) + 255) & ~size_t(255);
    const size_t to = bytes;
    bytes += (tt.size() * sizeof(TPackTile) + 255) & ~size_t(255);
    const size_t ro = bytes;
    bytes += (rowptr.size() * sizeof(char*) + 255) & ~size_t(255);
    const size_t rpo = bytes;
    bytes += (2 * (size_t)L.N * sizeof(char*) + 255) & ~size_t(255);
    CK(h, ws_alloc((void**)&h->tcp_tables, std::max<size_t>(bytes, 256), h->st));
    if (vpack) {
        char** d_rowptr = reinterpret_cast<char**>(h->tcp_tables + ro);
        CK(h, cudaMemcpyAsync(d_rowptr, rowptr.data(), rowptr.size() * sizeof(char*), cudaMemcpyHostToDevice, h->st));
        for (size_t ti = 0; ti < tabs.size(); ++ti)
            if (tabs[ti].G == &h->Lc_v) {
                for (auto& f : vfix) pp[ti][f.first].rowptr = d_rowptr + f.second;
                h->Lc_v.epi = EPI_PACKNK;
            }
    }
    for (size_t ti = 0; ti < tabs.size(); ++ti) {
        GemmLaunch& G = *tabs[ti].G;
        G.d_pprobs = reinterpret_cast<PProb*>(h->tcp_tables + po[ti]);
        G.d_jobs = reinterpret_cast<PackJob*>(h->tcp_tables + jo[ti]);
        G.njobs = (int)jobs[ti].size();
        G.max_items = maxit[ti];
        if (!pp[ti].empty())
            CK(h, cudaMemcpyAsync(G.d_pprobs, pp[ti].data(), pp[ti].size() * sizeof(PProb), cudaMemcpyHostToDevice,
                                  h->st));
        if (!jobs[ti].empty())
            CK(h, cudaMemcpyAsync(G.d_jobs, jobs[ti].data(), jobs[ti].size() * sizeof(PackJob),
                                  cudaMemcpyHostToDevice, h->st));
    }
    if (rfuse) {
        h->d_rkn = reinterpret_cast<char**>(h->tcp_tables + rpo);
        h->d_rmk = h->d_rkn + L.N;
        CK(h, cudaMemcpyAsync(h->d_rkn, rkn.data(), L.N * sizeof(char*), cudaMemcpyHostToDevice, h->st));
        CK(h, cudaMemcpyAsync(h->d_rmk, rmk.data(), L.N * sizeof(char*), cudaMemcpyHostToDevice, h->st));
        h->rstep_on = true;
    }
    if (!ttp.empty()) {
        TPackTile* d_ttp = reinterpret_cast<TPackTile*>(h->tcp_tables + tpo);
        CK(h, cudaMemcpyAsync(d_ttp, ttp.data(), ttp.size() * sizeof(TPackTile), cudaMemcpyHostToDevice, h->st));
        h->Le_a1.d_gpack = d_ttp;
        h->Le_a1.n_gpack = (int)ttp.size();
        h->Le_a1.gpack_src = h->Tp;
        h->Le_a1.gpack_ns = (int)L.ns;
    }
    h->d_tpack = reinterpret_cast<TPackTile*>(h->tcp_tables + to);
    h->n_tpack = (int)tt.size();
    if (!tt.empty())
        CK(h, cudaMemcpyAsync(h->d_tpack, tt.data(), tt.size() * sizeof(TPackTile), cudaMemcpyHostToDevice, h->st));
    h->d_static_jobs = reinterpret_cast<PackJob*>(h->tcp_tables + so);
    h->n_static_jobs = (int)sjobs.size();
    h->static_items = smax;
    if (!sjobs.empty())
        CK(h, cudaMemcpyAsync(h->d_static_jobs, sjobs.data(), sjobs.size() * sizeof(PackJob), cudaMemcpyHostToDevice,
                              h->st));
    CK(h, cudaStreamSynchronize(h->st));   // host vectors go out of scope
    return TLR_OK;
}

}  // namespace

// The data step of a request (eq. 14 and the normalisation): alpha, then the
// receiver-major panels Dfrak = D[:, perm]^T / alpha and Ufrak likewise.
static int load_data(tlr_mdd_s* h, const void* D, const void* U, int memory) {
    const Layout& L = h->L;
    const tlr_mdd_desc_t* d = &h->d;
    const cf* Dsrc = (const cf*)D;
    const cf* Usrc = (const cf*)U;
    const size_t nrs = (size_t)L.nr * L.ns;
    if (memory == TLR_MEM_HOST) {  // host inputs are staged through the residual / A1 buffers
        CK(h, cudaMemcpyAsync(h->R, D, nrs * sizeof(cf), cudaMemcpyHostToDevice, h->st));
        CK(h, cudaMemcpyAsync(h->A1, U, nrs * sizeof(cf), cudaMemcpyHostToDevice, h->st));
        Dsrc = h->R;
        Usrc = h->A1;
    }
    if (d->alpha > 0.0) {
        const double al = d->alpha;
        CK(h, cudaMemcpyAsync(h->scal, &al, sizeof(double), cudaMemcpyHostToDevice, h->st));
    } else {
        CK(h, max_abs2(Dsrc, (long long)nrs, h->dpart, kRedBlocks, h->scal, h->st));
    }
    CK(h, permute_normalise(Dsrc, L.ns, L.nr, h->perm, h->scal, h->Dt, h->st));
    CK(h, permute_normalise(Usrc, L.ns, L.nr, h->perm, h->scal, h->Ut, h->st));
    return TLR_OK;
}

// ===========================================================================
// entry points
// ===========================================================================
extern "C" {

void tlr_mdd_desc_init(tlr_mdd_desc_t* d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->diag_mode = TLR_DIAG_RULE;
    d->reciprocity = TLR_RECIP_SYMMETRIC;
    d->precision = TLR_PREC_FP32;
    d->input_memory = TLR_MEM_DEVICE;
}

void tlr_mdd_solve_opts_init(tlr_mdd_solve_opts_t* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->lam0 = 10.0;
    o->decay = 0.1;
    o->stages = 3;
    o->admm_iters = 2;
    o->lbfgs_iters = 5;
    o->memory = 10;
    o->rho = 1.0;
    o->theta_memory = TLR_MEM_DEVICE;
}

int tlr_mdd_theta_size(const tlr_mdd_desc_t* d, int64_t* n) {
    Layout L;
    std::string e;
    int rc = build_layout(d, L, e);
    if (rc) {
        g_last_error = e;
        return rc;
    }
    if (!n) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "n_theta is NULL");
    *n = L.ntheta;
    return TLR_OK;
}

int tlr_mdd_theta_layout(const tlr_mdd_desc_t* d, int64_t* off_diag, int64_t* off_l, int64_t* off_r,
                         uint8_t* dense_out) {
    Layout L;
    std::string e;
    int rc = build_layout(d, L, e);
    if (rc) {
        g_last_error = e;
        return rc;
    }
    if (off_diag) std::copy(L.off_diag.begin(), L.off_diag.end(), off_diag);
    if (off_l) std::copy(L.off_l.begin(), L.off_l.end(), off_l);
    if (off_r) std::copy(L.off_r.begin(), L.off_r.end(), off_r);
    if (dense_out) std::copy(L.dense.begin(), L.dense.end(), dense_out);
    return TLR_OK;
}

int64_t tlr_mdd_workspace_bytes(const tlr_mdd_desc_t* d) {
    tlr_mdd_s tmp;
    std::string e;
    if (build_layout(d, tmp.L, e)) return -1;
    tmp.nsplit = split_for(tmp.L, d->precision);
    Arena a;
    carve(&tmp, a);
    // plus the L-BFGS ring for the default memory (m = 10: 11 slots of s and y)
    int64_t total = (int64_t)a.used + (int64_t)2 * 11 * tmp.L.nth * (int64_t)sizeof(cf);
    if (tensor_core(d->precision)) total += packed_estimate(tmp.L);
    return total;
}

int tlr_mdd_hilbert_perm(int32_t nx, int32_t ny, int32_t* perm_dev, void* stream) {
    if (nx <= 0 || ny <= 0 || !perm_dev) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "bad grid or NULL perm");
    if (nx > 32768 || ny > 32768) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_SHAPE, "grid side above 32768");
    cudaStream_t st = (cudaStream_t)stream;
    long long n = 1;
    while (n < nx || n < ny) n <<= 1;
    int32_t* slot = nullptr;
    tlr_mdd_s* h = nullptr;
    CK(h, cudaMallocAsync((void**)&slot, (size_t)(n * n) * sizeof(int32_t), st));
    cudaError_t e = hilbert_perm(nx, ny, perm_dev, slot, st);
    cudaFreeAsync(slot, st);
    CK(h, e);
    return TLR_OK;
}

int tlr_mdd_create(tlr_mdd_t** out, const tlr_mdd_desc_t* d, const void* D, const void* U, void* stream) {
    if (!out) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "handle pointer is NULL");
    *out = nullptr;
    if (!d || !D || !U) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "desc, D or U is NULL");
    tlr_mdd_s* h = new tlr_mdd_s();
    h->d = *d;
    h->d.perm = nullptr;
    h->d.ranks = nullptr;
    h->d.diag_dense = nullptr;
    h->d.tiles = nullptr;
    h->st = (cudaStream_t)stream;
    int rc = build_layout(d, h->L, h->err);
    if (rc) {
        g_last_error = h->err;
        delete h;
        return rc;
    }
    const Layout& L = h->L;
    if (!d->perm && ((int64_t)d->nx * d->ny != d->nr || d->nx <= 0 || d->ny <= 0)) {
        g_last_error = "nx * ny must equal nr (or pass perm)";
        delete h;
        return TLR_ERR_SHAPE;
    }
    h->nsplit = split_for(L, d->precision);
    h->kchunk = (int)(((L.ns + h->nsplit - 1) / h->nsplit + 15) / 16 * 16);
    Arena a;
    carve(h, a);
    h->arena_bytes = a.used;
    auto fail = [&](int code) {
        g_last_error = h->err;
        if (h->packed) cudaFreeAsync(h->packed, h->st);
        if (h->tcp_tables) cudaFreeAsync(h->tcp_tables, h->st);
        if (h->arena) cudaFreeAsync(h->arena, h->st);
        delete h;
        return code;
    };
    {
        cudaError_t e = ws_alloc((void**)&h->arena, h->arena_bytes, h->st);
        if (e != cudaSuccess) {
            h->arena = nullptr;
            h->err = std::string("device allocation failed: ") + cudaGetErrorString(e);
            return fail(TLR_ERR_NOMEM);
        }
    }
    Arena b2;
    b2.base = h->arena;
    carve(h, b2);
#define CKF(expr)                                                                  \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            h->err = std::string(#expr) + ": " + cudaGetErrorString(e_);           \
            return fail(e_ == cudaErrorMemoryAllocation ? TLR_ERR_NOMEM : TLR_ERR_CUDA); \
        }                                                                          \
    } while (0)
    // receiver order
    if (d->perm) {
        std::vector<char> seen(L.nr, 0);
        for (int64_t a2 = 0; a2 < L.nr; ++a2) {
            const int32_t r = d->perm[a2];
            if (r < 0 || r >= L.nr || seen[r]) {
                h->err = "perm is not a permutation of 0..nr-1";
                return fail(TLR_ERR_ARG);
            }
            seen[r] = 1;
        }
        CKF(cudaMemcpyAsync(h->perm, d->perm, L.nr * sizeof(int32_t), cudaMemcpyHostToDevice, h->st));
    } else {
        long long n = 1;
        while (n < d->nx || n < d->ny) n <<= 1;
        int32_t* slot = nullptr;
        CKF(cudaMallocAsync((void**)&slot, (size_t)(n * n) * sizeof(int32_t), h->st));
        cudaError_t e = hilbert_perm(d->nx, d->ny, h->perm, slot, h->st);
        cudaFreeAsync(slot, h->st);
        CKF(e);
    }
    {
        int rc = load_data(h, D, U, d->input_memory);
        if (rc) {
            h->err = g_last_error;
            return fail(rc);
        }
    }
    // maps
    if (L.Ktot > 0)
        CKF(cudaMemcpyAsync(h->d_partner, L.partner.data(), L.Ktot * sizeof(int), cudaMemcpyHostToDevice, h->st));
    if (L.general && L.KtotB > 0)
        CKF(cudaMemcpyAsync(h->d_partnerB, L.partnerB.data(), L.KtotB * sizeof(int), cudaMemcpyHostToDevice, h->st));
    if (L.ncol > 0) {
        CKF(cudaMemcpyAsync((void*)h->pm.colsrc, L.colsrc.data(), L.ncol * sizeof(long long), cudaMemcpyHostToDevice, h->st));
        CKF(cudaMemcpyAsync((void*)h->pm.colstride, L.colstride.data(), L.ncol * sizeof(int), cudaMemcpyHostToDevice, h->st));
        CKF(cudaMemcpyAsync((void*)h->pm.colpan, L.colpan.data(), L.ncol * sizeof(long long), cudaMemcpyHostToDevice, h->st));
        CKF(cudaMemcpyAsync((void*)h->pm.panstride, L.panstride.data(), L.ncol * sizeof(int), cudaMemcpyHostToDevice, h->st));
        CKF(cudaMemcpyAsync((void*)h->pm.colrows, L.colrows.data(), L.ncol * sizeof(int), cudaMemcpyHostToDevice, h->st));
    }
    if (L.ndense > 0) {
        CKF(cudaMemcpyAsync((void*)h->pm.zsrc, L.zsrc.data(), L.ndense * sizeof(long long), cudaMemcpyHostToDevice, h->st));
        CKF(cudaMemcpyAsync((void*)h->pm.zoff, L.zoff.data(), L.ndense * sizeof(long long), cudaMemcpyHostToDevice, h->st));
        CKF(cudaMemcpyAsync((void*)h->pm.zdim, L.zdim.data(), L.ndense * sizeof(int), cudaMemcpyHostToDevice, h->st));
    }
    CKF(cudaMemcpyAsync(h->d_roff, L.roff.data(), (L.N + 1) * sizeof(long long), cudaMemcpyHostToDevice, h->st));
    // solver counters and the contraction kernels' error word start at zero
    CKF(cudaMemsetAsync(h->ints, 0, (SI_COUNT + 8) * sizeof(int), h->st));
    std::vector<HostTable> tabs;
    if (build_tables(h, h->tab_base, &tabs)) {
        h->err = "uploading GEMM tables failed";
        return fail(TLR_ERR_CUDA);
    }
    // packed operands: always for TF32 (the on-the-fly kernel splits to BF16x3
    // only); for BF16x3 unless TLR_MDD_PACKED=0 selects the on-the-fly kernel
    if (d->precision == TLR_PREC_TF32 || (d->precision == TLR_PREC_BF16X3 && !getenv_off("TLR_MDD_PACKED"))) {
        // every tensor-core contraction except the dense adjoint (allocated per call)
        int rc = build_tc(h, tabs);
        if (rc) return fail(rc);
        CKF(gemm_tcp_prepare());
        CKF(pack_operands(h->d_static_jobs, h->n_static_jobs, h->static_items, h->st));
    }
    CKF(cudaEventCreate(&h->ev0));
    CKF(cudaEventCreate(&h->ev1));
    CKF(cudaMallocHost((void**)&h->hstats, sizeof(HostStats)));
    if (tensor_core(d->precision)) CKF(gemm_tc_prepare());
    CKF(cudaStreamSynchronize(h->st));
    CKF(cudaMemcpy(&h->alpha, h->scal, sizeof(double), cudaMemcpyDeviceToHost));
#undef CKF
    *out = h;
    return TLR_OK;
}

int tlr_mdd_set_data(tlr_mdd_t* h, const void* D, const void* U, int32_t input_memory) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!D || !U) FAIL(h, TLR_ERR_ARG, "D or U is NULL");
    if (input_memory != TLR_MEM_DEVICE && input_memory != TLR_MEM_HOST) FAIL(h, TLR_ERR_ARG, "bad input_memory");
    if (h->pending) FAIL(h, TLR_ERR_STATE, "a solve is pending on this handle");
    int rc = load_data(h, D, U, input_memory);
    if (rc) return rc;
    if (h->n_static_jobs) CK(h, pack_operands(h->d_static_jobs, h->n_static_jobs, h->static_items, h->st));
    if (h->d.alpha <= 0.0) {
        CK(h, cudaMemcpyAsync(&h->alpha, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
    }
    return TLR_OK;
}

static int forward(tlr_mdd_s* h, bool plain_apply) {
    const Layout& L = h->L;
    CK(h, sym_dense(h->x, L.nlr, L.ndense, L.dmax, h->Zs, h->st, L.general, h->pm.zoff, h->pm.zdim));
    CK(h, run_gemm(h->Lc_x, h->st));
    if (h->n_tpack) CK(h, tpack(h->d_tpack, h->n_tpack, h->T, h->Tp, nullptr, (int)L.ns, h->st));
    CK(h, run_gemm(plain_apply ? h->Le_apply : h->Le_fwd, h->st));
    if (!plain_apply && h->rstep_on)
        CK(h, rstep(h->R, h->A1, h->A2, nullptr, (int)L.nr, (int)L.ns, (int)L.b, h->d_rkn, h->d_rmk, nullptr, h->st,
                    L.b > 0 ? nullptr : h->d_roff, L.N, pack_fmt(h->d.precision)));
    return TLR_OK;
}

static int gradient(tlr_mdd_s* h) {
    const Layout& L = h->L;
    CK(h, run_gemm(h->Lc_v, h->st));
    CK(h, run_gemm(h->Lp, h->st));
    CK(h, reduce_grad(h->part, h->nsplit, L.nth, L.nlr, L.ndense, L.dmax, h->gf, h->st, L.general, h->pm.zoff,
                      h->pm.zdim));
    return TLR_OK;
}

int tlr_mdd_apply(tlr_mdd_t* h, const void* theta, void* Y) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!theta || !Y) FAIL(h, TLR_ERR_ARG, "theta or Y is NULL");
    const Layout& L = h->L;
    CK(h, theta_to_panel(h->pm, (const cf*)theta, h->x, h->st));
    int rc = forward(h, true);
    if (rc) return rc;
    CK(h, cudaMemcpyAsync(Y, h->R, (size_t)L.nr * L.ns * sizeof(cf), cudaMemcpyDeviceToDevice, h->st));
    return TLR_OK;
}

int tlr_mdd_grad(tlr_mdd_t* h, const void* theta, void* grad, double* f) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!theta || !grad) FAIL(h, TLR_ERR_ARG, "theta or grad is NULL");
    const Layout& L = h->L;
    CK(h, theta_to_panel(h->pm, (const cf*)theta, h->x, h->st));
    int rc = forward(h, false);
    if (rc) return rc;
    rc = gradient(h);
    if (rc) return rc;
    CK(h, panel_to_theta(h->pm, h->gf, (cf*)grad, h->st));
    if (f) {
        CK(h, sv_norm_part(h->R, (long long)L.nr * L.ns, h->dpart, h->st));
        CK(h, finalize(h->dpart, kRedBlocks, 1, 1, h->scal + 1, h->st));
        double rr = 0;
        int werr = 0;
        CK(h, cudaMemcpyAsync(&rr, h->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaMemcpyAsync(&werr, h->ints + SI_COUNT + 1, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        if (werr != 0) {
            CK(h, cudaMemsetAsync(h->ints + SI_COUNT + 1, 0, sizeof(int), h->st));
            CK(h, cudaStreamSynchronize(h->st));
            FAIL(h, TLR_ERR_TIMEOUT, "a tensor-core contraction timed out on a barrier wait");
        }
        *f = 0.5 * rr;
    }
    return TLR_OK;
}

int tlr_mdd_adjoint(tlr_mdd_t* h, const void* V, void* G) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!V || !G) FAIL(h, TLR_ERR_ARG, "V or G is NULL");
    const Layout& L = h->L;
    const long long nr = L.nr, ns = L.ns;
    const long long tiles = ((nr + 63) / 64) * ((nr + 63) / 64);
    const int ns_split = choose_split(tiles, ns);
    GProb p;
    memset(&p, 0, sizeof(p));
    p.t[0] = term((const cf*)V, ns, h->Dt, ns, nullptr, (int)ns, false, true);
    p.nt = 1;
    p.M = (int)nr;
    p.N = (int)nr;
    p.ldc = nr;
    GProb* dp = nullptr;
    cf* part = nullptr;
    CK(h, cudaMallocAsync((void**)&dp, sizeof(GProb), h->st));
    if (ns_split > 1) {
        cudaError_t e = cudaMallocAsync((void**)&part, (size_t)ns_split * nr * nr * sizeof(cf), h->st);
        if (e != cudaSuccess) {
            cudaFreeAsync(dp, h->st);
            CK(h, e);
        }
        p.C = part;
    } else {
        p.C = (cf*)G;
    }
    GemmLaunch G1;
    G1.d_probs = dp;
    G1.nprob = 1;
    G1.maxM = G1.maxN = (int)nr;
    G1.amode = A_MK;
    G1.bmode = B_NK;
    G1.nsplit = ns_split;
    G1.kchunk = (int)(((ns + ns_split - 1) / ns_split + 15) / 16 * 16);
    G1.part_stride = nr * nr;
    G1.epi = ns_split > 1 ? EPI_PARTIAL : EPI_STORE;
    cudaError_t e = cudaMemcpyAsync(dp, &p, sizeof(GProb), cudaMemcpyHostToDevice, h->st);
    G1.flops = 8.0 * nr * (double)nr * ns;
    G1.cls = 2;
    G1.prec = tensor_core(h->d.precision) ? TLR_PREC_BF16X3 : TLR_PREC_FP32;   // operands split on the fly
    G1.err = h->ints + SI_COUNT + 1;
    if (e == cudaSuccess) e = run_gemm(G1, h->st);
    if (e == cudaSuccess && ns_split > 1) e = reduce_grad(part, ns_split, nr * nr, nr * nr, 0, 1, (cf*)G, h->st);
    if (part) cudaFreeAsync(part, h->st);
    cudaFreeAsync(dp, h->st);
    CK(h, e);
    CK(h, cudaStreamSynchronize(h->st));  // p lives on this stack frame
    return TLR_OK;
}

// Benchmark solver of eq. (4) on the handle's data: conjugate gradients on
// P(G P(Z)) + 2 lambda Z = P(D-hat^H U-hat) with G = D-hat^H D-hat formed once.
// In the receiver-major panels D-hat^H D-hat = conj(Dfrak) Dfrak^T and
// D-hat^H U-hat = conj(Dfrak) Ufrak^T.  The iterates stay exactly symmetric,
// so X = P(Z) = Z.
int tlr_mdd_benchmark_solve(tlr_mdd_t* h, double lambda, int32_t iters, double tol, void* X,
                            tlr_mdd_bench_stats_t* stats) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!X) FAIL(h, TLR_ERR_ARG, "X is NULL");
    if (!(lambda >= 0.0) || !std::isfinite(lambda) || iters < 0 || !(tol >= 0.0))
        FAIL(h, TLR_ERR_ARG, "lambda must be finite and >= 0, iters >= 0, tol >= 0");
    if (h->pending) FAIL(h, TLR_ERR_STATE, "a solve is pending on this handle");
    const Layout& L = h->L;
    const int n = (int)L.nr, ns = (int)L.ns;
    const size_t n2 = (size_t)n * n;
    const bool tc = tensor_core(h->d.precision);   // BF16x3 packed products for both tensor-core modes
    const int np = cg_partials(n);
    // work arrays: G, x, r, p, y, Ap; partials; scalars; tables; packed operands (tensor cores)
    const size_t pk = tc ? (size_t)std::max(packed_bytes(n, ns, kPackTRA), packed_bytes(n, n, kPackTRA)) : 0;
    const size_t tab = 4096;
    const size_t bytes = 6 * n2 * sizeof(cf) + (size_t)np * sizeof(double) + 64 + tab + 2 * pk + 16 * 256;
    char* buf = nullptr;
    CK(h, cudaMallocAsync((void**)&buf, bytes, h->st));
    Arena a;
    a.base = buf;
    cf* G = a.take<cf>(n2);
    cf* x = a.take<cf>(n2);
    cf* r = a.take<cf>(n2);
    cf* pv = a.take<cf>(n2);
    cf* y = a.take<cf>(n2);
    cf* Ap = a.take<cf>(n2);
    double* part = a.take<double>(np);
    double* sc = a.take<double>(8);
    char* tables = a.take<char>(tab);
    char* pkA = tc ? a.take<char>(pk) : nullptr;
    char* pkB = tc ? a.take<char>(pk) : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    auto blank = []() {
        GProb q;
        memset(&q, 0, sizeof(q));
        return q;
    };
    // three products: G = conj(D) D^T, Bm = conj(D) U^T, y = G p
    GemmLaunch GL[3];
    if (!tc) {
        GProb q[3] = {blank(), blank(), blank()};
        q[0].t[0] = term(h->Dt, ns, h->Dt, ns, nullptr, ns, true, false);
        q[1].t[0] = term(h->Dt, ns, h->Ut, ns, nullptr, ns, true, false);
        q[2].t[0] = term(G, n, pv, n, nullptr, n, false, false);
        cf* outs[3] = {G, y, y};
        for (int i = 0; i < 3; ++i) {
            q[i].nt = 1;
            q[i].M = q[i].N = n;
            q[i].C = outs[i];
            q[i].ldc = n;
        }
        GProb* dq = reinterpret_cast<GProb*>(tables);
        e = cudaMemcpyAsync(dq, q, sizeof(q), cudaMemcpyHostToDevice, h->st);
        for (int i = 0; i < 3; ++i) {
            GL[i].d_probs = dq + i;
            GL[i].nprob = 1;
            GL[i].maxM = GL[i].maxN = n;
            GL[i].maxK = i < 2 ? ns : n;
            GL[i].amode = A_MK;
            GL[i].bmode = i < 2 ? B_NK : B_KN;
            GL[i].epi = EPI_STORE;
            GL[i].prec = TLR_PREC_FP32;
            GL[i].err = h->ints + SI_COUNT + 1;
        }
    } else {
        // pack jobs: 0 conj(D) (A, MK) -> pkA; 1 D (B, rows n) -> pkB; 2 U (B) -> pkB;
        // 3 G (A, MK) -> pkA; 4 p (B; p is symmetric, so its rows serve) -> pkB
        PackJob J[5];
        const cf* src[5] = {h->Dt, h->Dt, h->Ut, G, pv};
        const int Ks[5] = {ns, ns, ns, n, n};
        for (int i = 0; i < 5; ++i) {
            J[i].src = src[i];
            J[i].ld = Ks[i];
            J[i].g_row = nullptr;
            J[i].g_k = nullptr;
            J[i].kcontig = 1;
            J[i].sgn = i == 0 ? -1.f : 1.f;
            J[i].R = n;
            J[i].K = Ks[i];
            J[i].TR = (i == 0 || i == 3) ? kPackTRA : kPackTRB;
            J[i].dst = (i == 0 || i == 3) ? (void*)pkA : (void*)pkB;
            J[i].fmt = kFmtBF16X3;
        }
        PProb q[3];
        memset(q, 0, sizeof(q));
        cf* outs[3] = {G, y, y};
        for (int i = 0; i < 3; ++i) {
            q[i].t[0].A = pkA;
            q[i].t[0].B = pkB;
            q[i].t[0].K = i < 2 ? ns : n;
            q[i].nt = 1;
            q[i].M = q[i].N = n;
            q[i].C = outs[i];
            q[i].ldc = n;
        }
        PProb* dq = reinterpret_cast<PProb*>(tables);
        PackJob* dj = reinterpret_cast<PackJob*>(tables + 1024);
        e = cudaMemcpyAsync(dq, q, sizeof(q), cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dj, J, sizeof(J), cudaMemcpyHostToDevice, h->st);
        auto items = [](long long R, long long K, int TR) {
            return (((R + TR - 1) / TR * TR) << 32) | ((K + 15) / 16 * 2);
        };
        const int first[3] = {0, 2, 4}, cnt[3] = {2, 1, 1};
        for (int i = 0; i < 3; ++i) {
            GL[i].d_pprobs = dq + i;
            GL[i].d_jobs = dj + first[i];
            GL[i].njobs = cnt[i];
            GL[i].max_items = items(n, i < 2 ? ns : n, kPackTRB);
            GL[i].nprob = 1;
            GL[i].maxM = GL[i].maxN = n;
            GL[i].maxK = i < 2 ? ns : n;
            GL[i].epi = EPI_STORE;
            GL[i].prec = TLR_PREC_BF16X3;
            GL[i].err = h->ints + SI_COUNT + 1;
        }
        static_assert(sizeof(PProb) * 3 <= 1024 && sizeof(PackJob) * 5 <= 3072, "table slots");
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->st);
    if (e == cudaSuccess) e = gemm_any(GL[0], h->st);                          // G
    if (e == cudaSuccess) e = gemm_any(GL[1], h->st);                          // Bm -> y
    if (e == cudaSuccess) e = cg_sym(y, nullptr, 0.f, r, n, nullptr, h->st);   // b = P(Bm) -> r
    if (e == cudaSuccess && tc) {                                              // G packed once, as A
        PackJob* dj = reinterpret_cast<PackJob*>(tables + 1024);
        e = pack_operands(dj + 3, 1, (((long long)(n + kPackTRA - 1) / kPackTRA * kPackTRA) << 32) | ((n + 15) / 16 * 2),
                          h->st);
    }
    if (e == cudaSuccess) e = cg_start(x, r, pv, n, part, sc, h->st);
    const float s2 = (float)(2.0 * lambda);
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        e = gemm_any(GL[2], h->st);                                            // y = G p
        if (e == cudaSuccess) e = cg_sym(y, pv, s2, Ap, n, part, h->st);       // Ap = P(y) + 2 lambda p
        if (e == cudaSuccess) e = cg_iteration_tail(x, r, pv, Ap, n, tol, part, sc, h->st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, x, n2 * sizeof(cf), cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->st);
    double hs[8] = {0};
    int werr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&werr, h->ints + SI_COUNT + 1, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    cudaFreeAsync(buf, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    CK(h, e);
    if (werr != 0) {
        CK(h, cudaMemsetAsync(h->ints + SI_COUNT + 1, 0, sizeof(int), h->st));
        CK(h, cudaStreamSynchronize(h->st));
        FAIL(h, TLR_ERR_TIMEOUT, "a tensor-core contraction timed out on a barrier wait");
    }
    // slots of k_cg.cu: rr 0, <p,Ap> 1, alpha 2, beta 3, ||b||^2 4, done 5, iterations 6
    const double rel = hs[4] > 0.0 ? std::sqrt(hs[0] / hs[4]) : 0.0;
    const int status = std::isfinite(hs[0]) ? TLR_OK : TLR_ERR_NONFINITE;
    if (stats) {
        stats->iters = (int32_t)hs[6];
        stats->status = status;
        stats->rel_res = rel;
        stats->gpu_ms = ms;
    }
    if (status != TLR_OK) FAIL(h, status, "non-finite value in the benchmark solver");
    return TLR_OK;
}

// Tile rank rule: the lower tiles (diagonal tiles, then the pairs in the
// stacking order) of X in b x b tiles, their singular values by the tile SVD,
// v0 = the largest of all, k = #{sigma >= eps v0}; entries = the number of
// complex entries of the factors with dense diagonals where 4 k >= b.
namespace {
int tile_ranks_impl(const cf* X, int64_t nr, int64_t b, double eps, std::vector<int32_t>& ranks, int64_t* entries,
                    double* v0, cudaStream_t st, std::string& err) {
    const int N = (int)(nr / b), P = N * (N - 1) / 2, nt = N + P;
    const int bi = (int)b;
    std::vector<SvdTile> tl(nt);
    for (int i = 0; i < N; ++i) tl[i] = SvdTile{i * bi, i * bi, bi, bi, 0};
    for (int j = 0; j < N; ++j)
        for (int i = j + 1; i < N; ++i) tl[N + j * N - j * (j + 1) / 2 + (i - j - 1)] = SvdTile{i * bi, j * bi, bi, bi, 0};
    Arena a;
    a.take<cf>(tile_svd_work_bytes(nt, (int)b, false) / sizeof(cf));
    a.take<float>((size_t)nt * b);
    a.take<SvdTile>(nt);
    a.take<int>(nt);
    a.take<double>(1);
    char* buf = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&buf, a.used, st);
    if (e != cudaSuccess) {
        err = std::string("tile ranks: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? TLR_ERR_NOMEM : TLR_ERR_CUDA;
    }
    Arena w;
    w.base = buf;
    cf* work = w.take<cf>(tile_svd_work_bytes(nt, (int)b, false) / sizeof(cf));
    float* sig = w.take<float>((size_t)nt * b);
    SvdTile* dtl = w.take<SvdTile>(nt);
    int* dr = w.take<int>(nt);
    double* dv0 = w.take<double>(1);
    ranks.assign(nt, 0);
    double hv0 = 0.0;
    e = cudaMemcpyAsync(dtl, tl.data(), nt * sizeof(SvdTile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = tile_svd(X, nr, dtl, nt, (int)b, work, false, 30, 1e-5f, sig, nullptr, nullptr, st);
    if (e == cudaSuccess) e = rank_rule(sig, nt, (int)b, eps, dr, dv0, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ranks.data(), dr, nt * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hv0, dv0, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        err = std::string("tile ranks: ") + cudaGetErrorString(e);
        return TLR_ERR_CUDA;
    }
    int64_t ent = 0;
    for (int i = 0; i < N; ++i) ent += 4LL * ranks[i] >= b ? b * b : b * ranks[i];
    for (int p = 0; p < P; ++p) ent += 2 * b * (int64_t)ranks[N + p];
    if (entries) *entries = ent;
    if (v0) *v0 = hv0;
    return TLR_OK;
}
}  // namespace

int tlr_mdd_tile_ranks(const void* X, int64_t nr, int64_t b, double eps, int32_t* ranks, int64_t* entries,
                       double* v0, void* stream) {
    tlr_mdd_s* h = nullptr;
    if (!X || !ranks) FAIL(h, TLR_ERR_ARG, "X or ranks is NULL");
    if (nr <= 0 || b <= 0 || b > 512 || nr % b != 0) FAIL(h, TLR_ERR_SHAPE, "need 0 < b <= 512 and nr % b == 0");
    if (!(eps > 0.0) || !(eps <= 1.0)) FAIL(h, TLR_ERR_ARG, "eps must lie in (0, 1]");
    std::vector<int32_t> r;
    std::string err;
    const int rc = tile_ranks_impl((const cf*)X, nr, b, eps, r, entries, v0, (cudaStream_t)stream, err);
    if (rc) FAIL(h, rc, err);
    std::copy(r.begin(), r.end(), ranks);
    return TLR_OK;
}

int tlr_mdd_choose_tile(const void* X, int64_t nr, const int64_t* candidates, int32_t ncand, double eps,
                        int64_t* best_b, int64_t* best_entries, void* stream) {
    tlr_mdd_s* h = nullptr;
    if (!X || !candidates || !best_b || ncand <= 0) FAIL(h, TLR_ERR_ARG, "X, candidates or best_b is NULL");
    if (!(eps > 0.0) || !(eps <= 1.0)) FAIL(h, TLR_ERR_ARG, "eps must lie in (0, 1]");
    int64_t bb = 0, be = 0;
    for (int c = 0; c < ncand; ++c) {
        const int64_t b = candidates[c];
        if (b <= 0 || b > 512 || nr % b != 0) continue;
        std::vector<int32_t> r;
        int64_t ent = 0;
        std::string err;
        const int rc = tile_ranks_impl((const cf*)X, nr, b, eps, r, &ent, nullptr, (cudaStream_t)stream, err);
        if (rc) FAIL(h, rc, err);
        if (bb == 0 || ent < be) {
            bb = b;
            be = ent;
        }
    }
    if (bb == 0) FAIL(h, TLR_ERR_SHAPE, "no candidate divides nr (with 0 < b <= 512)");
    *best_b = bb;
    if (best_entries) *best_entries = be;
    return TLR_OK;
}

// Warm start: the handle's layout decides each tile's form and rank; X is
// cut into tiles and each low-rank tile initialised from its truncated SVD
// (L = U Sigma^1/2, R = conj(V) Sigma^1/2; low-rank diagonals of the
// reciprocal form: the Takagi form Q with Q Q^T the rank-k truncation; of the
// general form: L, R as for any tile), dense diagonals copied.  Tiles of any
// sizes d_i <= 512; a wide tile's SVD runs on its transpose.
int tlr_mdd_warm_start(tlr_mdd_t* h, const void* X, void* theta) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!X || !theta) FAIL(h, TLR_ERR_ARG, "X or theta is NULL");
    const Layout& L = h->L;
    if (L.dmax > 512) FAIL(h, TLR_ERR_SHAPE, "warm start needs tiles <= 512");
    const int N = L.N;
    std::vector<SvdTile> tl;
    std::vector<WarmTile> wt;
    // a low-rank tile (i, j) with factors at offL (rows of block i) and offR (rows of block j)
    auto lowrank = [&](int i, int j, int k, long long offL, long long offR) {
        WarmTile w{};
        w.r0 = (int)L.roff[i];
        w.c0 = (int)L.roff[j];
        w.m = (int)L.d[i];
        w.n = (int)L.d[j];
        w.kind = 0;
        w.k = k;
        w.offL = offL;
        w.offR = offR;
        w.trans = w.n > w.m;
        w.svd = (int)tl.size();
        tl.push_back(SvdTile{w.r0, w.c0, w.m, w.n, w.trans});
        wt.push_back(w);
    };
    for (int i = 0; i < N; ++i) {
        const int di = (int)L.d[i];
        if (L.dense[i]) {
            WarmTile w{};
            w.r0 = w.c0 = (int)L.roff[i];
            w.m = w.n = di;
            w.kind = 2;
            w.k = di;
            w.offL = L.off_diag[i];
            w.svd = -1;
            wt.push_back(w);
        } else if (L.kd[i] > 0) {
            if (L.general) {
                lowrank(i, i, L.kd[i], L.off_diag[i], L.off_diag[i] + (long long)di * L.kd[i]);
            } else {
                WarmTile w{};
                w.r0 = w.c0 = (int)L.roff[i];
                w.m = w.n = di;
                w.kind = 1;
                w.k = L.kd[i];
                w.offL = L.off_diag[i];
                w.svd = (int)tl.size();
                tl.push_back(SvdTile{w.r0, w.c0, di, di, 0});
                wt.push_back(w);
            }
        }
    }
    // stored pairs in stacking order: (i, j), column j outer, row i inner
    // (reciprocal: i > j; general: every i != j)
    for (int p = 0, j = 0; j < N; ++j)
        for (int i = L.general ? 0 : j + 1; i < N; ++i) {
            if (i == j) continue;
            if (L.kp[p] > 0) lowrank(i, j, L.kp[p], L.off_l[p], L.off_r[p]);
            ++p;
        }
    const int nsvd = (int)tl.size(), nw = (int)wt.size();
    const int bmax = (int)L.dmax;
    Arena a;
    a.take<cf>(tile_svd_work_bytes(std::max(1, nsvd), bmax, true) / sizeof(cf));
    a.take<float>((size_t)std::max(1, nsvd) * bmax);
    a.take<int>((size_t)std::max(1, nsvd) * bmax);
    a.take<SvdTile>(std::max(1, nsvd));
    a.take<WarmTile>(std::max(1, nw));
    char* buf = nullptr;
    CK(h, cudaMallocAsync((void**)&buf, a.used, h->st));
    Arena w;
    w.base = buf;
    cf* work = w.take<cf>(tile_svd_work_bytes(std::max(1, nsvd), bmax, true) / sizeof(cf));
    float* sig = w.take<float>((size_t)std::max(1, nsvd) * bmax);
    int* ord = w.take<int>((size_t)std::max(1, nsvd) * bmax);
    SvdTile* dtl = w.take<SvdTile>(std::max(1, nsvd));
    WarmTile* dwt = w.take<WarmTile>(std::max(1, nw));
    cudaError_t e = cudaSuccess;
    if (nsvd) e = cudaMemcpyAsync(dtl, tl.data(), nsvd * sizeof(SvdTile), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess && nw) e = cudaMemcpyAsync(dwt, wt.data(), nw * sizeof(WarmTile), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
        e = tile_svd((const cf*)X, L.nr, dtl, nsvd, bmax, work, true, 30, 1e-5f, sig, ord, nullptr, h->st);
    if (e == cudaSuccess) e = warm_fill((const cf*)X, L.nr, dwt, nw, bmax, work, sig, ord, (cf*)theta, h->st);
    cudaFreeAsync(buf, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);   // the host tables above go out of scope
    CK(h, e);
    return TLR_OK;
}

int tlr_mdd_wait_selftest(int64_t limit_ns, int32_t* status, double* waited_ms, void* stream) {
    tlr_mdd_s* h = nullptr;
    if (!status) FAIL(h, TLR_ERR_ARG, "status is NULL");
    if (limit_ns <= 0 || limit_ns > 10000000000LL) FAIL(h, TLR_ERR_ARG, "limit_ns must lie in (0, 1e10]");
    const cudaStream_t st = (cudaStream_t)stream;
    char* buf = nullptr;
    CK(h, cudaMallocAsync((void**)&buf, 16, st));
    int* dst = reinterpret_cast<int*>(buf);
    unsigned long long* dw = reinterpret_cast<unsigned long long*>(buf + 8);
    int hs = 0;
    unsigned long long hw = 0;
    cudaError_t e = cudaMemsetAsync(buf, 0, 16, st);
    if (e == cudaSuccess) e = wait_selftest(dst, (unsigned long long)limit_ns, dw, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, dst, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hw, dw, sizeof(hw), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    CK(h, e);
    *status = hs;
    if (waited_ms) *waited_ms = (double)hw * 1e-6;
    return TLR_OK;
}

int tlr_mdd_get_state(tlr_mdd_t* h, void* z, void* u) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!z || !u) FAIL(h, TLR_ERR_ARG, "z or u is NULL");
    if (h->pending) FAIL(h, TLR_ERR_STATE, "a solve is pending on this handle");
    CK(h, panel_to_theta(h->pm, h->z, (cf*)z, h->st));
    CK(h, panel_to_theta(h->pm, h->u, (cf*)u, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return TLR_OK;
}

int tlr_mdd_set_state(tlr_mdd_t* h, const void* z, const void* u) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!z || !u) FAIL(h, TLR_ERR_ARG, "z or u is NULL");
    if (h->pending) FAIL(h, TLR_ERR_STATE, "a solve is pending on this handle");
    CK(h, theta_to_panel(h->pm, (const cf*)z, h->z, h->st));
    CK(h, theta_to_panel(h->pm, (const cf*)u, h->u, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return TLR_OK;
}

namespace {
int check_stack(long long ntr, long long nt, long long f0, long long nf, std::string& err) {
    if (ntr <= 0 || nt <= 0 || nt > 0x7fffffffLL || f0 < 0 || nf <= 0 || f0 + nf > nt / 2 + 1) {
        err = "need ntr > 0, 0 < nt < 2^31, f0 >= 0, nf > 0, f0 + nf <= nt / 2 + 1";
        return TLR_ERR_ARG;
    }
    return TLR_OK;
}
}  // namespace

int tlr_mdd_time_to_freq(const float* x_t, int64_t ntr, int64_t nt, int64_t f0, int64_t nf, void* X_w,
                         void* stream) {
    tlr_mdd_s* h = nullptr;
    if (!x_t || !X_w) FAIL(h, TLR_ERR_ARG, "x_t or X_w is NULL");
    std::string err;
    int rc = check_stack(ntr, nt, f0, nf, err);
    if (rc) FAIL(h, rc, err);
    rc = fft_stack(true, x_t, nullptr, ntr, nt, f0, nf, (cf*)X_w, nullptr, (cudaStream_t)stream, err);
    if (rc) FAIL(h, rc, err);
    return TLR_OK;
}

int tlr_mdd_freq_to_time(const void* X_w, int64_t ntr, int64_t nt, int64_t f0, int64_t nf, float* x_t,
                         void* stream) {
    tlr_mdd_s* h = nullptr;
    if (!x_t || !X_w) FAIL(h, TLR_ERR_ARG, "x_t or X_w is NULL");
    std::string err;
    int rc = check_stack(ntr, nt, f0, nf, err);
    if (rc) FAIL(h, rc, err);
    rc = fft_stack(false, nullptr, (const cf*)X_w, ntr, nt, f0, nf, nullptr, x_t, (cudaStream_t)stream, err);
    if (rc) FAIL(h, rc, err);
    return TLR_OK;
}

int tlr_mdd_stack_alpha(const void* D_w, int64_t n, double* alpha, void* stream) {
    tlr_mdd_s* h = nullptr;
    if (!D_w || !alpha || n <= 0) FAIL(h, TLR_ERR_ARG, "D_w or alpha is NULL, or n <= 0");
    cudaStream_t st = (cudaStream_t)stream;
    double* buf = nullptr;
    CK(h, cudaMallocAsync((void**)&buf, (kRedBlocks + 1) * sizeof(double), st));
    double a = 0.0;
    cudaError_t e = max_abs2((const cf*)D_w, n, buf + 1, kRedBlocks, buf, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&a, buf, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    CK(h, e);
    *alpha = a;
    return TLR_OK;
}

int tlr_mdd_unpermute_dense(tlr_mdd_t* h, const void* theta, void* X) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!theta || !X) FAIL(h, TLR_ERR_ARG, "theta or X is NULL");
    const Layout& L = h->L;
    const long long nr = L.nr;
    std::vector<AsmTile> tiles;
    if (!L.general) {
        tiles.resize(L.N + L.P);
        for (int i = 0; i < L.N; ++i)
            tiles[i] = AsmTile{L.off_diag[i], L.off_diag[i], L.dense[i] ? (int)L.d[i] : L.kd[i], (int)L.dense[i]};
        for (int p = 0; p < L.P; ++p) tiles[L.N + p] = AsmTile{L.off_l[p], L.off_r[p], L.kp[p], 0};
    } else {
        // every tile, row-major; ordered pair index of (i, j): j (N - 1) + i - (i > j)
        tiles.resize((size_t)L.N * L.N);
        for (int i = 0; i < L.N; ++i)
            for (int j = 0; j < L.N; ++j) {
                if (i == j) {
                    const int k = L.dense[i] ? (int)L.d[i] : L.kd[i];
                    tiles[i * L.N + j] = AsmTile{L.off_diag[i], L.off_diag[i] + (L.dense[i] ? 0 : L.d[i] * k), k,
                                                 (int)L.dense[i]};
                } else {
                    const int q = j * (L.N - 1) + i - (i > j ? 1 : 0);
                    tiles[i * L.N + j] = AsmTile{L.off_l[q], L.off_r[q], L.kp[q], 0};
                }
            }
    }
    cf* Xh = nullptr;
    AsmTile* dt = nullptr;
    CK(h, cudaMallocAsync((void**)&Xh, (size_t)nr * nr * sizeof(cf), h->st));
    cudaError_t e = cudaMallocAsync((void**)&dt, tiles.size() * sizeof(AsmTile), h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(AsmTile), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
        e = assemble_dense((const cf*)theta, nr, L.dmax, L.N, dt, Xh, h->st, L.general, L.b > 0 ? nullptr : h->d_roff);
    if (e == cudaSuccess) e = unpermute_dense(Xh, nr, h->perm, (cf*)X, h->st);
    if (dt) cudaFreeAsync(dt, h->st);
    cudaFreeAsync(Xh, h->st);
    CK(h, e);
    CK(h, cudaStreamSynchronize(h->st));
    return TLR_OK;
}

int tlr_mdd_get_data(tlr_mdd_t* h, int32_t* perm_host, double* alpha, void* Dt, void* Ut) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    const Layout& L = h->L;
    if (perm_host) CK(h, cudaMemcpyAsync(perm_host, h->perm, L.nr * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
    if (Dt) CK(h, cudaMemcpyAsync(Dt, h->Dt, (size_t)L.nr * L.ns * sizeof(cf), cudaMemcpyDeviceToDevice, h->st));
    if (Ut) CK(h, cudaMemcpyAsync(Ut, h->Ut, (size_t)L.nr * L.ns * sizeof(cf), cudaMemcpyDeviceToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (alpha) *alpha = h->alpha;
    return TLR_OK;
}

void tlr_mdd_timing_enable(int on) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = on != 0;
}

void tlr_mdd_timing_reset(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto& t : g_pending) {
        cudaEventSynchronize(t.b);
        g_evpool.push_back(t.a);
        g_evpool.push_back(t.b);
    }
    g_pending.clear();
    for (int c = 0; c < TLR_NCLASS; ++c) g_ms[c] = g_fl[c] = 0.0, g_nl[c] = 0;
}

int tlr_mdd_timing_read(double* ms, double* flops, int64_t* launches, int nclass) {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (auto& t : g_pending) {
        if (cudaEventSynchronize(t.b) != cudaSuccess) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_CUDA, "timing event failed");
        float m = 0.f;
        if (cudaEventElapsedTime(&m, t.a, t.b) != cudaSuccess) (void)cudaGetLastError();
        g_ms[t.cls] += m;
        g_fl[t.cls] += t.flops;
        g_nl[t.cls] += 1;
        g_evpool.push_back(t.a);
        g_evpool.push_back(t.b);
    }
    g_pending.clear();
    for (int c = 0; c < nclass && c < TLR_NCLASS; ++c) {
        if (ms) ms[c] = g_ms[c];
        if (flops) flops[c] = g_fl[c];
        if (launches) launches[c] = g_nl[c];
    }
    return TLR_OK;
}

int64_t tlr_mdd_launch_count(void) { return g_launches.load(); }

void* tlr_mdd_stream(const tlr_mdd_t* h) { return h ? (void*)h->st : nullptr; }

int tlr_mdd_set_stream(tlr_mdd_t* h, void* stream) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (h->pending) FAIL(h, TLR_ERR_STATE, "a solve is pending on this handle");
    if (stream == (void*)h->st) return TLR_OK;
    // work already enqueued on the old stream finishes before anything that
    // follows on the new one
    CK(h, cudaStreamSynchronize(h->st));
    h->st = (cudaStream_t)stream;
    return TLR_OK;
}

const char* tlr_mdd_last_error(const tlr_mdd_t* h) { return h ? h->err.c_str() : g_last_error.c_str(); }

int tlr_mdd_trim_pool(int64_t keep_bytes, int64_t* reserved) {
    if (keep_bytes < 0) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "keep_bytes must be >= 0");
    cudaMemPool_t p = nullptr;
    CK((tlr_mdd_s*)nullptr, ws_pool(&p));
    CK((tlr_mdd_s*)nullptr, cudaMemPoolTrimTo(p, (size_t)keep_bytes));
    if (reserved) {
        unsigned long long r = 0;
        CK((tlr_mdd_s*)nullptr, cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &r));
        *reserved = (int64_t)r;
    }
    return TLR_OK;
}

int tlr_mdd_set_pass_ctas(int64_t ctas, int64_t* previous) {
    if (ctas < 0) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "ctas must be >= 0");
    if (previous) *previous = (int64_t)pass_cap();
    set_pass_cap((long long)ctas);
    return TLR_OK;
}

int tlr_mdd_destroy(tlr_mdd_t* h) {
    if (!h) return TLR_ERR_ARG;
    if (h->pending) cudaEventSynchronize(h->ev1);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    for (auto& t : h->gtimed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (h->hstats) cudaFreeHost(h->hstats);
    if (h->ring) cudaFreeAsync(h->ring, h->st);
    if (h->packed) cudaFreeAsync(h->packed, h->st);
    if (h->tcp_tables) cudaFreeAsync(h->tcp_tables, h->st);
    if (h->arena) cudaFreeAsync(h->arena, h->st);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    cudaError_t e = cudaStreamSynchronize(h->st);
    delete h;
    return e == cudaSuccess ? TLR_OK : TLR_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
static int check_opts(tlr_mdd_s* h, const tlr_mdd_solve_opts_t* o) {
    if (o->memory < 1 || o->memory > 32) FAIL(h, TLR_ERR_ARG, "memory must lie in [1, 32]");
    if (!(o->rho > 0.0) || o->stages < 0 || o->admm_iters < 0 || o->lbfgs_iters < 0 || !(o->lam0 >= 0.0))
        FAIL(h, TLR_ERR_ARG, "invalid solver options");
    if (o->flags & ~(TLR_SOLVE_RESUME | TLR_SOLVE_REFRESH)) FAIL(h, TLR_ERR_ARG, "unknown solver flags");
    return TLR_OK;
}

// The whole solve as a fixed sequence of launches on h->st: theta is read from
// and written back to h->th_io; every decision lives in device memory.
// The device-side solver state of a handle for L-BFGS memory m.
static SolverDev solver_dev(tlr_mdd_s* h, int m) {
    const long long n2 = 2 * h->L.nth;
    SolverDev S;
    S.n2 = n2;
    S.m = m;
    S.ring = m + 1;
    S.x = (float*)h->x;
    S.z = (float*)h->z;
    S.u = (float*)h->u;
    S.v = (float*)h->v;
    S.g = (float*)h->g;
    S.gf = (float*)h->gf;
    S.d = (float*)h->dd;
    S.q = (float*)h->q;
    S.sh = h->ring;
    S.yh = h->ring + (size_t)S.ring * n2;
    S.rho_h = h->rho_h;
    S.sy_h = h->sy_h;
    S.yy_h = h->yy_h;
    S.acoef = h->acoef;
    S.SYm = h->lbm;
    S.YYm = h->lbm + 33 * 33;
    S.lbpart = h->lbpart;
    S.sc = h->sc;
    S.ints = h->ints;
    S.fhist = h->fhist;
    S.part = h->dpart;   // 2 slabs
    return S;
}

static int enqueue_solve(tlr_mdd_s* h, const tlr_mdd_solve_opts_t* o) {
    const Layout& L = h->L;
    const long long nrs = (long long)L.nr * L.ns;
    SolverDev S = solver_dev(h, o->memory);
    double* part6 = h->dpart + 2 * kRedBlocks;    // 6 slabs
    double* part3 = h->dpart + 8 * kRedBlocks;    // 3 slabs
    double* part3b = h->dpart + 11 * kRedBlocks;  // 3 slabs
    double* partf = h->dpart + 14 * kRedBlocks;   // 1 slab
    const double rho = o->rho;

    CK(h, theta_to_panel(h->pm, h->th_io, h->x, h->st));
    if (o->flags & TLR_SOLVE_RESUME)
        CK(h, sv_admm_resume(S, h->st));
    else
        CK(h, sv_admm_init(S, h->st));
    int rc = forward(h, false);
    if (rc) return rc;
    CK(h, sv_norm_part(h->R, nrs, partf, h->st));
    CK(h, sv_record_f0(S, partf, h->st));
    rc = gradient(h);
    if (rc) return rc;
    int xu = 0;   // x-updates of this call
    for (int s = 0; s < o->stages; ++s) {
        const double lam = o->lam0 * std::pow(o->decay, (double)s);
        for (int it = 0; it < o->admm_iters; ++it, ++xu) {
            if ((o->flags & TLR_SOLVE_REFRESH) && xu > 0) {
                // fresh residual, products and gradient at theta (what a resumed call starts from)
                rc = forward(h, false);
                if (rc) return rc;
                rc = gradient(h);
                if (rc) return rc;
            }
            CK(h, sv_xupdate_start(S, rho, h->st));
            for (int t = 0; t < o->lbfgs_iters; ++t) {
                CK(h, sv_direction(S, h->st));
                CK(h, run_gemm(h->Lc_d, h->st));
                CK(h, sym_dense(h->dd, L.nlr, L.ndense, L.dmax, h->Zsd, h->st, L.general, h->pm.zoff, h->pm.zdim));
                CK(h, run_gemm(h->Le_a1, h->st));
                CK(h, run_gemm(h->Le_a2, h->st));
                if (h->rstep_on) {
                    // the carried residual lives in its packed forms
                    CK(h, dots6_packed(h->d_rkn, h->A1, h->A2, (int)L.nr, (int)L.ns, (int)L.b, part6, h->st,
                                       L.b > 0 ? nullptr : h->d_roff, L.N, pack_fmt(h->d.precision)));
                    CK(h, sv_dots3(S, part3, h->st));
                    CK(h, sv_line_search(S, part6, kRedBlocks, part3, rho, h->st));
                } else {
                    CK(h, dots6_part(h->R, h->A1, h->A2, nrs, part6, h->st));
                    CK(h, sv_dots3(S, part3, h->st));
                    CK(h, sv_line_search(S, part6, kRedBlocks, part3, rho, h->st));
                }
                if (h->rstep_on)
                    CK(h, rstep(h->R, h->A1, h->A2, h->sc + SC_ALPHA, (int)L.nr, (int)L.ns, (int)L.b, h->d_rkn,
                                h->d_rmk, h->rpart, h->st, L.b > 0 ? nullptr : h->d_roff, L.N,
                                pack_fmt(h->d.precision)));
                else
                    CK(h, sv_step_residual(h->R, h->A1, h->A2, nrs, h->sc + SC_ALPHA, partf, h->st));
                if (h->n_tpack)
                    CK(h, tpack(h->d_tpack, h->n_tpack, h->T, h->Tp, h->sc + SC_ALPHA, (int)L.ns, h->st));
                else if (L.KtotB > 0)
                    CK(h, axpy_dev((float*)h->T, (const float*)h->Tp, 2LL * L.KtotB * L.ns, h->sc + SC_ALPHA, h->st));
                CK(h, sv_step_theta(S, h->st));
                rc = gradient(h);
                if (rc) return rc;
                CK(h, sv_pair_prep(S, rho, part3b, h->st));
                if (h->rstep_on)
                    CK(h, sv_pair_accept(S, part3b, h->rpart, (int)h->n_rpart, h->st));
                else
                    CK(h, sv_pair_accept(S, part3b, partf, kRedBlocks, h->st));
            }
            CK(h, sv_admm_zu(S, lam, rho, h->st));
        }
    }
    CK(h, panel_to_theta(h->pm, h->x, h->th_io, h->st));
    return TLR_OK;
}

static bool graphs_enabled(const tlr_mdd_s* h) {
    if (h->st == nullptr) return false;  // the legacy default stream cannot be captured
    const char* e = getenv("TLR_MDD_GRAPHS");
    return !(e && e[0] == '0');
}

// Everything between the staging copies; a CUDA graph replay when possible.
static int enqueue_body(tlr_mdd_s* h, const tlr_mdd_solve_opts_t* o) {
    const Layout& L = h->L;
    const long long n2 = 2 * L.nth;
    if (h->ring_m < o->memory) {  // ring of s / y vectors, m + 1 slots each
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        if (h->ring) cudaFreeAsync(h->ring, h->st);
        h->ring = nullptr;
        h->ring_m = 0;
        CK(h, ws_alloc((void**)&h->ring, (size_t)2 * (o->memory + 1) * n2 * sizeof(float), h->st));
        h->ring_m = o->memory;
    }
    h->pending_graph = false;
    if (!graphs_enabled(h)) return enqueue_solve(h, o);
    // A handle's first solve with given options runs as plain launches (a
    // recording and instantiation cost more host time than one enqueue, and a
    // handle used once, as most served requests are, never needs the graph);
    // the second records the graph that every later solve replays.
    const bool same = h->gexec && [&] {
        GraphKey k;
        k.lam0 = o->lam0;
        k.decay = o->decay;
        k.rho = o->rho;
        k.stages = o->stages;
        k.admm = o->admm_iters;
        k.lbfgs = o->lbfgs_iters;
        k.mem = o->memory;
        k.flags = o->flags;
        std::lock_guard<std::mutex> lk(g_tmu);
        k.timing = g_timing ? 1 : 0;
        return k == h->gkey;
    }();
    if (!same && h->plain_solves == 0 && !getenv_off("TLR_MDD_LAZY_GRAPH")) {
        h->plain_solves = 1;
        return enqueue_solve(h, o);
    }
    h->plain_solves = 0;
    GraphKey k;
    k.lam0 = o->lam0;
    k.decay = o->decay;
    k.rho = o->rho;
    k.stages = o->stages;
    k.admm = o->admm_iters;
    k.lbfgs = o->lbfgs_iters;
    k.mem = o->memory;
    k.flags = o->flags;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        k.timing = g_timing ? 1 : 0;
    }
    if (!h->gexec || !(k == h->gkey)) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        for (auto& t : h->gtimed) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        h->gtimed.clear();
        cudaGraph_t g = nullptr;
        CK(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
        g_capture_sink = &h->gtimed;
        const long long n_before = g_launches.load();
        int rc = enqueue_solve(h, o);
        h->graph_kernels = g_launches.load() - n_before;
        g_launches.fetch_sub(h->graph_kernels);   // recorded, not launched: counted at each replay
        g_capture_sink = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CK(h, e);
        // node priorities kept: the memory-bound passes run ahead of other
        // streams' pending contraction CTAs, as in plain launches
        e = cudaGraphInstantiate(&h->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        CK(h, e);
        h->gkey = k;
    }
    CK(h, cudaGraphLaunch(h->gexec, h->st));
    counted((int)h->graph_kernels);
    h->pending_graph = true;
    return TLR_OK;
}

int tlr_mdd_solve_async(tlr_mdd_t* h, void* theta_inout, const tlr_mdd_solve_opts_t* o) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!theta_inout || !o) FAIL(h, TLR_ERR_ARG, "theta or opts is NULL");
    if (h->pending) FAIL(h, TLR_ERR_STATE, "a solve is already pending on this handle");
    int rc = check_opts(h, o);
    if (rc) return rc;
    const size_t bytes = h->L.nth * sizeof(cf);
    const bool host = o->theta_memory == TLR_MEM_HOST;
    CK(h, cudaEventRecord(h->ev0, h->st));
    CK(h, cudaMemcpyAsync(h->th_io, theta_inout, bytes, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          h->st));
    rc = enqueue_body(h, o);
    if (rc) return rc;
    CK(h, cudaMemcpyAsync(theta_inout, h->th_io, bytes, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          h->st));
    CK(h, cudaMemcpyAsync(h->hstats->ints, h->ints, sizeof(h->hstats->ints), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(h->hstats->sc, h->sc, sizeof(h->hstats->sc), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(h->hstats->fhist, h->fhist, sizeof(h->hstats->fhist), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaEventRecord(h->ev1, h->st));
    h->pending = true;
    return TLR_OK;
}

int tlr_mdd_solve_query(tlr_mdd_t* h) {
    if (!h) return TLR_ERR_STATE;
    if (!h->pending) return 1;
    cudaError_t e = cudaEventQuery(h->ev1);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    h->err = cudaGetErrorString(e);
    return TLR_ERR_CUDA;
}

int tlr_mdd_solve_wait(tlr_mdd_t* h, tlr_mdd_stats_t* stats) {
    if (!h) FAIL(h, TLR_ERR_STATE, "handle is NULL");
    if (!h->pending) FAIL(h, TLR_ERR_STATE, "no solve is pending on this handle");
    h->pending = false;
    CK(h, cudaEventSynchronize(h->ev1));
    if (h->pending_graph && !h->gtimed.empty()) account_replay(h->gtimed);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) != cudaSuccess) (void)cudaGetLastError();
    const HostStats& hs = *h->hstats;
    if (stats) {
        stats->iters = hs.ints[SI_ITERS];
        stats->restarts = hs.ints[SI_RESTARTS];
        stats->status = hs.ints[SI_STATUS];
        stats->n_hist = std::min(hs.ints[SI_ITERS], TLR_MAX_HIST);
        memcpy(stats->f_hist, hs.fhist, sizeof(stats->f_hist));
        stats->f0 = hs.sc[SC_F0];
        stats->gpu_ms = ms;
    }
    if (hs.ints[SI_COUNT + 1] != 0) {
        // a tensor-core contraction gave up on a bounded wait: report and re-arm
        CK(h, cudaMemsetAsync(h->ints + SI_COUNT + 1, 0, sizeof(int), h->st));
        CK(h, cudaStreamSynchronize(h->st));
        FAIL(h, TLR_ERR_TIMEOUT, "a tensor-core contraction timed out on a barrier wait");
    }
    if (hs.ints[SI_STATUS] != 0) FAIL(h, TLR_ERR_NONFINITE, "non-finite value met during the solve");
    return TLR_OK;
}

int tlr_mdd_solve(tlr_mdd_t* h, void* theta_inout, const tlr_mdd_solve_opts_t* o, tlr_mdd_stats_t* stats) {
    int rc = tlr_mdd_solve_async(h, theta_inout, o);
    if (rc) return rc;
    return tlr_mdd_solve_wait(h, stats);
}

// ---------------------------------------------------------------------------
// batched solve: several handles in lockstep, each contraction one
// persistent launch over the tiles of every member
// ---------------------------------------------------------------------------
}  // extern "C"

struct tlr_mdd_batch_s {
    std::vector<tlr_mdd_s*> hs;
    cudaStream_t st = nullptr;            // merged contractions; the solve's start and end
    std::vector<cudaStream_t> ms;         // one per member: its own kernels
    std::vector<cudaEvent_t> evm;         // end of a member's phase
    cudaEvent_t evj = nullptr;            // end of a merged contraction
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    char* tables = nullptr;               // merged problem / job / slice tables and the error word
    int* err = nullptr;
    // merged launches (null d_pprobs: that kind runs per member)
    GemmLaunch Lc_x, Lc_d, Lc_v, Le_fwd, Le_a1, Lp;
    std::vector<void*> io;                // caller theta buffers of the pending solve
    int theta_memory = 0;
    bool pending = false;
    std::string err_msg;
};

namespace {

// One merged launch of contraction kind `kind` over every member: problem
// tables and pack jobs concatenated (device-to-device), one slice per
// member problem and split in a map.  Returns false when the members'
// launches of this kind differ in epilogue or format (they then run apart).
bool plan_merged(tlr_mdd_batch_s* b, GemmLaunch tlr_mdd_s::*kind, GemmLaunch& M, size_t& off, bool size_only,
                 cudaStream_t st, cudaError_t& e) {
    const GemmLaunch& G0 = b->hs[0]->*kind;
    int nprob = 0, njobs = 0, nz = 0;
    for (auto* h : b->hs) {
        const GemmLaunch& G = h->*kind;
        if (G.epi != G0.epi || pack_fmt(G.prec) != pack_fmt(G0.prec) || G.cls != G0.cls || !G.d_pprobs)
            return false;
        nprob += G.nprob;
        njobs += G.njobs;
        nz += G.nprob * G.nsplit;
    }
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t po = take(std::max<size_t>(1, nprob) * sizeof(PProb));
    const size_t jo = take(std::max<size_t>(1, njobs) * sizeof(PackJob));
    const size_t zo = take(std::max<size_t>(1, nz) * sizeof(ZItem));
    if (size_only) return true;
    M = GemmLaunch();
    M.d_pprobs = reinterpret_cast<PProb*>(b->tables + po);
    M.d_jobs = njobs ? reinterpret_cast<PackJob*>(b->tables + jo) : nullptr;
    M.d_zmap = reinterpret_cast<ZItem*>(b->tables + zo);
    M.nprob = nprob;
    M.njobs = njobs;
    M.nz = nz;
    M.nsplit = 1;
    M.epi = G0.epi;
    M.cls = G0.cls;
    M.prec = G0.prec;
    M.persistent = (persist_classes() >> G0.cls) & 1;
    M.err = b->err;
    std::vector<ZItem> zm;
    int pbase = 0, jbase = 0;
    for (auto* h : b->hs) {
        const GemmLaunch& G = h->*kind;
        M.maxM = std::max(M.maxM, G.maxM);
        M.maxN = std::max(M.maxN, G.maxN);
        M.maxK = std::max(M.maxK, G.maxK);
        M.flops += G.flops;
        M.max_items = std::max(M.max_items >> 32, G.max_items >> 32) << 32 |
                      std::max(M.max_items & 0xffffffffLL, G.max_items & 0xffffffffLL);
        if (G.nprob && e == cudaSuccess)
            e = cudaMemcpyAsync(M.d_pprobs + pbase, G.d_pprobs, G.nprob * sizeof(PProb), cudaMemcpyDeviceToDevice, st);
        if (G.njobs && e == cudaSuccess)
            e = cudaMemcpyAsync(M.d_jobs + jbase, G.d_jobs, G.njobs * sizeof(PackJob), cudaMemcpyDeviceToDevice, st);
        for (int p = 0; p < G.nprob; ++p)
            for (int c = 0; c < G.nsplit; ++c) {
                ZItem z;
                z.prob = pbase + p;
                z.chunk = c;
                z.kchunk = G.nsplit > 1 ? G.kchunk : 0;
                z.pad = 0;
                z.part_off = (long long)c * G.part_stride;
                zm.push_back(z);
            }
        pbase += G.nprob;
        jbase += G.njobs;
    }
    if (!zm.empty() && e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<ZItem*>(M.d_zmap), zm.data(), zm.size() * sizeof(ZItem), cudaMemcpyHostToDevice,
                            st);
    return true;
}

using BatchKinds = GemmLaunch tlr_mdd_s::*;
const BatchKinds kBatchKinds[6] = {&tlr_mdd_s::Lc_x, &tlr_mdd_s::Lc_d, &tlr_mdd_s::Lc_v,
                                    &tlr_mdd_s::Le_fwd, &tlr_mdd_s::Le_a1, &tlr_mdd_s::Lp};

GemmLaunch tlr_mdd_batch_s::* const kBatchMerged[6] = {&tlr_mdd_batch_s::Lc_x, &tlr_mdd_batch_s::Lc_d,
                                                       &tlr_mdd_batch_s::Lc_v, &tlr_mdd_batch_s::Le_fwd,
                                                       &tlr_mdd_batch_s::Le_a1, &tlr_mdd_batch_s::Lp};

#define BCK(expr)                                                              \
    do {                                                                       \
        cudaError_t e_ = (expr);                                               \
        if (e_ != cudaSuccess) {                                               \
            b->err_msg = std::string(#expr) + ": " + cudaGetErrorString(e_);   \
            g_last_error = b->err_msg;                                         \
            return TLR_ERR_CUDA;                                               \
        }                                                                      \
    } while (0)

// the merged stream waits for every member's stream / every member waits for it
int b_join(tlr_mdd_batch_s* b) {
    for (size_t m = 0; m < b->hs.size(); ++m) {
        BCK(cudaEventRecord(b->evm[m], b->ms[m]));
        BCK(cudaStreamWaitEvent(b->st, b->evm[m], 0));
    }
    return TLR_OK;
}
int b_fork(tlr_mdd_batch_s* b) {
    BCK(cudaEventRecord(b->evj, b->st));
    for (auto s : b->ms) BCK(cudaStreamWaitEvent(s, b->evj, 0));
    return TLR_OK;
}

// one contraction kind for every member: the merged launch on the merged
// stream (after the members' gathered packs on their own streams), or each
// member's own launch on its stream when the kinds could not be merged
int b_gemm(tlr_mdd_batch_s* b, int k) {
    GemmLaunch& M = b->*kBatchMerged[k];
    const BatchKinds kind = kBatchKinds[k];
    if (!M.d_pprobs) {
        for (size_t m = 0; m < b->hs.size(); ++m) BCK(run_gemm(b->hs[m]->*kind, b->ms[m]));
        return TLR_OK;
    }
    for (size_t m = 0; m < b->hs.size(); ++m) {
        const GemmLaunch& G = b->hs[m]->*kind;
        if (G.n_gpack) BCK(tpack(G.d_gpack, G.n_gpack, G.gpack_src, nullptr, nullptr, G.gpack_ns, b->ms[m]));
    }
    int rc = b_join(b);
    if (rc) return rc;
    if (M.njobs) BCK(pack_operands(M.d_jobs, M.njobs, M.max_items, b->st));
    GemmLaunch L = M;
    L.njobs = 0;   // packed above
    BCK(run_gemm(L, b->st));
    return b_fork(b);
}

int b_forward(tlr_mdd_batch_s* b) {
    for (size_t m = 0; m < b->hs.size(); ++m) {
        tlr_mdd_s* h = b->hs[m];
        const Layout& L = h->L;
        BCK(sym_dense(h->x, L.nlr, L.ndense, L.dmax, h->Zs, b->ms[m], L.general, h->pm.zoff, h->pm.zdim));
    }
    int rc = b_gemm(b, 0);   // Lc_x
    if (rc) return rc;
    for (size_t m = 0; m < b->hs.size(); ++m) {
        tlr_mdd_s* h = b->hs[m];
        if (h->n_tpack) BCK(tpack(h->d_tpack, h->n_tpack, h->T, h->Tp, nullptr, (int)h->L.ns, b->ms[m]));
    }
    rc = b_gemm(b, 3);   // Le_fwd
    if (rc) return rc;
    for (size_t m = 0; m < b->hs.size(); ++m) {
        tlr_mdd_s* h = b->hs[m];
        const Layout& L = h->L;
        if (h->rstep_on)
            BCK(rstep(h->R, h->A1, h->A2, nullptr, (int)L.nr, (int)L.ns, (int)L.b, h->d_rkn, h->d_rmk, nullptr,
                      b->ms[m], L.b > 0 ? nullptr : h->d_roff, L.N, pack_fmt(h->d.precision)));
    }
    return TLR_OK;
}

int b_gradient(tlr_mdd_batch_s* b) {
    int rc = b_gemm(b, 2);   // Lc_v
    if (rc) return rc;
    rc = b_gemm(b, 5);       // Lp
    if (rc) return rc;
    for (size_t m = 0; m < b->hs.size(); ++m) {
        tlr_mdd_s* h = b->hs[m];
        const Layout& L = h->L;
        BCK(reduce_grad(h->part, h->nsplit, L.nth, L.nlr, L.ndense, L.dmax, h->gf, b->ms[m], L.general, h->pm.zoff,
                        h->pm.zdim));
    }
    return TLR_OK;
}

// The lockstep solve: the same sequence as enqueue_solve for every member,
// its own kernels on its own stream, the contractions merged.
int b_enqueue(tlr_mdd_batch_s* b, const tlr_mdd_solve_opts_t* o) {
    const size_t n = b->hs.size();
    std::vector<SolverDev> S(n);
    for (size_t m = 0; m < n; ++m) S[m] = solver_dev(b->hs[m], o->memory);
    auto part = [&](size_t m, int slab) { return b->hs[m]->dpart + (size_t)slab * kRedBlocks; };
    const double rho = o->rho;
    for (size_t m = 0; m < n; ++m) {
        tlr_mdd_s* h = b->hs[m];
        BCK(theta_to_panel(h->pm, h->th_io, h->x, b->ms[m]));
        if (o->flags & TLR_SOLVE_RESUME)
            BCK(sv_admm_resume(S[m], b->ms[m]));
        else
            BCK(sv_admm_init(S[m], b->ms[m]));
    }
    int rc = b_forward(b);
    if (rc) return rc;
    for (size_t m = 0; m < n; ++m) {
        tlr_mdd_s* h = b->hs[m];
        BCK(sv_norm_part(h->R, (long long)h->L.nr * h->L.ns, part(m, 14), b->ms[m]));
        BCK(sv_record_f0(S[m], part(m, 14), b->ms[m]));
    }
    rc = b_gradient(b);
    if (rc) return rc;
    int xu = 0;
    for (int s = 0; s < o->stages; ++s) {
        const double lam = o->lam0 * std::pow(o->decay, (double)s);
        for (int it = 0; it < o->admm_iters; ++it, ++xu) {
            if ((o->flags & TLR_SOLVE_REFRESH) && xu > 0) {
                rc = b_forward(b);
                if (rc) return rc;
                rc = b_gradient(b);
                if (rc) return rc;
            }
            for (size_t m = 0; m < n; ++m) BCK(sv_xupdate_start(S[m], rho, b->ms[m]));
            for (int t = 0; t < o->lbfgs_iters; ++t) {
                for (size_t m = 0; m < n; ++m) BCK(sv_direction(S[m], b->ms[m]));
                rc = b_gemm(b, 1);   // Lc_d
                if (rc) return rc;
                for (size_t m = 0; m < n; ++m) {
                    tlr_mdd_s* h = b->hs[m];
                    const Layout& L = h->L;
                    BCK(sym_dense(h->dd, L.nlr, L.ndense, L.dmax, h->Zsd, b->ms[m], L.general, h->pm.zoff,
                                  h->pm.zdim));
                }
                rc = b_gemm(b, 4);   // Le_a1 (A1 and A2)
                if (rc) return rc;
                for (size_t m = 0; m < n; ++m) {
                    tlr_mdd_s* h = b->hs[m];
                    const Layout& L = h->L;
                    const long long nrs = (long long)L.nr * L.ns;
                    cudaStream_t st = b->ms[m];
                    if (h->rstep_on)
                        BCK(dots6_packed(h->d_rkn, h->A1, h->A2, (int)L.nr, (int)L.ns, (int)L.b, part(m, 2), st,
                                         L.b > 0 ? nullptr : h->d_roff, L.N, pack_fmt(h->d.precision)));
                    else
                        BCK(dots6_part(h->R, h->A1, h->A2, nrs, part(m, 2), st));
                    BCK(sv_dots3(S[m], part(m, 8), st));
                    BCK(sv_line_search(S[m], part(m, 2), kRedBlocks, part(m, 8), rho, st));
                    if (h->rstep_on)
                        BCK(rstep(h->R, h->A1, h->A2, h->sc + SC_ALPHA, (int)L.nr, (int)L.ns, (int)L.b, h->d_rkn,
                                  h->d_rmk, h->rpart, st, L.b > 0 ? nullptr : h->d_roff, L.N,
                                  pack_fmt(h->d.precision)));
                    else
                        BCK(sv_step_residual(h->R, h->A1, h->A2, nrs, h->sc + SC_ALPHA, part(m, 14), st));
                    if (h->n_tpack)
                        BCK(tpack(h->d_tpack, h->n_tpack, h->T, h->Tp, h->sc + SC_ALPHA, (int)L.ns, st));
                    else if (L.KtotB > 0)
                        BCK(axpy_dev((float*)h->T, (const float*)h->Tp, 2LL * L.KtotB * L.ns, h->sc + SC_ALPHA, st));
                    BCK(sv_step_theta(S[m], st));
                }
                rc = b_gradient(b);
                if (rc) return rc;
                for (size_t m = 0; m < n; ++m) {
                    tlr_mdd_s* h = b->hs[m];
                    BCK(sv_pair_prep(S[m], rho, part(m, 11), b->ms[m]));
                    if (h->rstep_on)
                        BCK(sv_pair_accept(S[m], part(m, 11), h->rpart, (int)h->n_rpart, b->ms[m]));
                    else
                        BCK(sv_pair_accept(S[m], part(m, 11), part(m, 14), kRedBlocks, b->ms[m]));
                }
            }
            for (size_t m = 0; m < n; ++m) BCK(sv_admm_zu(S[m], lam, rho, b->ms[m]));
        }
    }
    for (size_t m = 0; m < n; ++m) BCK(panel_to_theta(b->hs[m]->pm, b->hs[m]->x, b->hs[m]->th_io, b->ms[m]));
    return TLR_OK;
}

void b_free(tlr_mdd_batch_s* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    for (auto s : b->ms)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    for (auto e : b->evm)
        if (e) cudaEventDestroy(e);
    if (b->evj) cudaEventDestroy(b->evj);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->tables) {
        cudaFreeAsync(b->tables, b->st);
        cudaStreamSynchronize(b->st);
    }
    delete b;
}

}  // namespace

extern "C" {

int tlr_mdd_batch_create(tlr_mdd_batch_t** out, tlr_mdd_t* const* hs, int32_t n, void* stream) {
    if (!out) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "batch pointer is NULL");
    *out = nullptr;
    if (!hs || n < 1 || n > 64) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "a batch holds 1 to 64 handles");
    int fmt = -1;
    for (int i = 0; i < n; ++i) {
        tlr_mdd_s* h = hs[i];
        if (!h) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "NULL handle in the batch");
        if (h->pending) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_STATE, "a member has a pending solve");
        if (!h->packed) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_UNSUPPORTED, "batched solves need the packed tensor-core path");
        if (fmt >= 0 && pack_fmt(h->d.precision) != fmt)
            FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "members of a batch share one tensor-core precision");
        fmt = pack_fmt(h->d.precision);
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "a handle appears twice in the batch");
    }
    tlr_mdd_batch_s* b = new tlr_mdd_batch_s();
    b->hs.assign(hs, hs + n);
    b->st = (cudaStream_t)stream;
    auto fail = [&](int code, const char* msg) {
        g_last_error = msg;
        b_free(b);
        return code;
    };
    b->ms.assign(n, nullptr);
    b->evm.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        if (cudaStreamCreateWithFlags(&b->ms[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->evm[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(TLR_ERR_CUDA, "creating the batch's streams failed");
    }
    if (cudaEventCreateWithFlags(&b->evj, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
        return fail(TLR_ERR_CUDA, "creating the batch's events failed");
    // sizing pass, then the tables
    size_t off = 256;   // the error word first
    cudaError_t e = cudaSuccess;
    bool merged[6];
    for (int k = 0; k < 6; ++k) {
        GemmLaunch tmp;
        merged[k] = plan_merged(b, kBatchKinds[k], tmp, off, true, b->st, e);
    }
    if (ws_alloc((void**)&b->tables, off, b->st) != cudaSuccess) {
        b->tables = nullptr;
        return fail(TLR_ERR_NOMEM, "allocating the batch's tables failed");
    }
    b->err = reinterpret_cast<int*>(b->tables);
    e = cudaMemsetAsync(b->tables, 0, 256, b->st);
    off = 256;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        if (merged[k]) plan_merged(b, kBatchKinds[k], b->*kBatchMerged[k], off, false, b->st, e);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return fail(TLR_ERR_CUDA, cudaGetErrorString(e));
    *out = b;
    return TLR_OK;
}

int tlr_mdd_batch_solve_async(tlr_mdd_batch_t* b, void* const* thetas, const tlr_mdd_solve_opts_t* o) {
    if (!b) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_STATE, "batch is NULL");
    if (!thetas || !o) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "thetas or opts is NULL");
    if (b->pending) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_STATE, "a batched solve is already pending");
    const size_t n = b->hs.size();
    for (size_t m = 0; m < n; ++m) {
        if (!thetas[m]) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_ARG, "NULL theta in the batch");
        if (b->hs[m]->pending) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_STATE, "a member has a pending solve");
        int rc = check_opts(b->hs[m], o);
        if (rc) return rc;
    }
    const bool host = o->theta_memory == TLR_MEM_HOST;
    BCK(cudaEventRecord(b->ev0, b->st));
    int rc = b_fork(b);
    if (rc) return rc;
    for (size_t m = 0; m < n; ++m) {
        tlr_mdd_s* h = b->hs[m];
        const long long n2 = 2 * h->L.nth;
        if (h->ring_m < o->memory) {   // the member's ring of s / y vectors
            if (h->gexec) {
                cudaGraphExecDestroy(h->gexec);
                h->gexec = nullptr;
            }
            if (h->ring) cudaFreeAsync(h->ring, b->ms[m]);
            h->ring = nullptr;
            h->ring_m = 0;
            BCK(ws_alloc((void**)&h->ring, (size_t)2 * (o->memory + 1) * n2 * sizeof(float), b->ms[m]));
            h->ring_m = o->memory;
        }
        BCK(cudaMemcpyAsync(h->th_io, thetas[m], h->L.nth * sizeof(cf),
                            host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->ms[m]));
    }
    rc = b_enqueue(b, o);
    if (rc) return rc;
    for (size_t m = 0; m < n; ++m) {
        tlr_mdd_s* h = b->hs[m];
        cudaStream_t s = b->ms[m];
        BCK(cudaMemcpyAsync(thetas[m], h->th_io, h->L.nth * sizeof(cf),
                            host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        BCK(cudaMemcpyAsync(h->hstats->ints, h->ints, sizeof(h->hstats->ints), cudaMemcpyDeviceToHost, s));
        BCK(cudaMemcpyAsync(h->hstats->sc, h->sc, sizeof(h->hstats->sc), cudaMemcpyDeviceToHost, s));
        BCK(cudaMemcpyAsync(h->hstats->fhist, h->fhist, sizeof(h->hstats->fhist), cudaMemcpyDeviceToHost, s));
    }
    rc = b_join(b);
    if (rc) return rc;
    BCK(cudaEventRecord(b->ev1, b->st));
    b->pending = true;
    return TLR_OK;
}

int tlr_mdd_batch_query(tlr_mdd_batch_t* b) {
    if (!b) return TLR_ERR_STATE;
    if (!b->pending) return 1;
    cudaError_t e = cudaEventQuery(b->ev1);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return TLR_ERR_CUDA;
}

int tlr_mdd_batch_wait(tlr_mdd_batch_t* b, tlr_mdd_stats_t* stats) {
    if (!b) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_STATE, "batch is NULL");
    if (!b->pending) FAIL((tlr_mdd_s*)nullptr, TLR_ERR_STATE, "no batched solve is pending");
    b->pending = false;
    BCK(cudaEventSynchronize(b->ev1));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) != cudaSuccess) (void)cudaGetLastError();
    int werr = 0;
    BCK(cudaMemcpy(&werr, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    int worst = TLR_OK;
    for (size_t m = 0; m < b->hs.size(); ++m) {
        const HostStats& hs = *b->hs[m]->hstats;
        if (stats) {
            tlr_mdd_stats_t& s = stats[m];
            s.iters = hs.ints[SI_ITERS];
            s.restarts = hs.ints[SI_RESTARTS];
            s.status = hs.ints[SI_STATUS];
            s.n_hist = std::min(hs.ints[SI_ITERS], TLR_MAX_HIST);
            memcpy(s.f_hist, hs.fhist, sizeof(s.f_hist));
            s.f0 = hs.sc[SC_F0];
            s.gpu_ms = ms;
        }
        if (hs.ints[SI_STATUS] != 0) worst = TLR_ERR_NONFINITE;
    }
    if (werr != 0) {
        BCK(cudaMemset(b->err, 0, sizeof(int)));
        FAIL((tlr_mdd_s*)nullptr, TLR_ERR_TIMEOUT, "a tensor-core contraction timed out on a barrier wait");
    }
    if (worst) FAIL((tlr_mdd_s*)nullptr, worst, "non-finite value met during a member's solve");
    return TLR_OK;
}

int tlr_mdd_batch_destroy(tlr_mdd_batch_t* b) {
    if (!b) return TLR_ERR_ARG;
    b_free(b);
    return TLR_OK;
}

}  // extern "C"
