// Allocation-free variant of the dense adjoint G = V Dfrak^H.
//
// tlr_mdd_adjoint() reduces its split-K partial products in a buffer it
// allocates per call.  This variant keeps that scratch in one file-scope
// device array instead, so a caller that must not allocate device memory (its
// process hands all device memory to its own pool allocator, or it runs on a
// latency-critical path where an allocation call may synchronise the device)
// can still use the kernel.  The array is TLR_NOALLOC_SCRATCH_BYTES per GPU
// that loads the library and is held until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace tlr {
namespace {

constexpr size_t kScratchBytes = TLR_NOALLOC_SCRATCH_BYTES;
constexpr size_t kProbBytes = 256;  // problem descriptor slot at the start of the array

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on each device.  In host code the
// symbol's name is only a host-side stand-in, never a device address, so it
// is resolved with cudaGetSymbolAddress once per device, with that device
// current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// A buffer of this call must live on the current device (or be managed
// memory): the scratch array and the launch belong to that device.
bool on_current_device(const void* p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace tlr

using namespace tlr;

extern "C" int tlr_mdd_adjoint_noalloc(const void* V, const void* Dt, int64_t nr, int64_t ns, void* G,
                                       void* stream) {
    if (!V || !Dt || !G) return TLR_ERR_ARG;
    if (nr <= 0 || ns <= 0 || nr > (int64_t)1 << 30 || ns > (int64_t)1 << 30) return TLR_ERR_SHAPE;
    const size_t slab = (size_t)nr * (size_t)nr * sizeof(cf);
    if (slab > kScratchBytes - kProbBytes) return TLR_ERR_SHAPE;  // nr above the scratch limit
    if (!on_current_device(V) || !on_current_device(Dt) || !on_current_device(G)) return TLR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return TLR_ERR_CUDA;

    // split-K over ns into as many partial slabs as fit (deterministic reduction)
    const long long tiles = ((nr + 63) / 64) * ((nr + 63) / 64);
    long long want = (4LL * 152 * 2 + tiles - 1) / tiles;
    want = std::min(want, std::max(1LL, (long long)ns / 256));
    want = std::max(1LL, std::min(want, 64LL));
    const long long fit = (long long)((kScratchBytes - kProbBytes) / slab);
    const int nsplit = (int)std::max(1LL, std::min(want, fit));

    GProb p;
    memset(&p, 0, sizeof(p));
    p.t[0].A = (const cf*)V;
    p.t[0].lda = ns;
    p.t[0].B = (const cf*)Dt;
    p.t[0].ldb = ns;
    p.t[0].g = nullptr;
    p.t[0].K = (int)ns;
    p.t[0].sa = 1.f;
    p.t[0].sb = -1.f;  // conj(Dfrak)
    p.nt = 1;
    p.M = (int)nr;
    p.N = (int)nr;
    p.ldc = nr;
    cf* part = reinterpret_cast<cf*>(reinterpret_cast<char*>(base) + kProbBytes);
    p.C = part;
    static_assert(sizeof(GProb) <= kProbBytes, "descriptor slot too small");

    GemmLaunch L;
    L.d_probs = reinterpret_cast<GProb*>(base);
    L.nprob = 1;
    L.maxM = L.maxN = (int)nr;
    L.amode = A_MK;
    L.bmode = B_NK;
    L.nsplit = nsplit;
    L.kchunk = (int)(((ns + nsplit - 1) / nsplit + 15) / 16 * 16);
    L.part_stride = nr * nr;
    L.epi = EPI_PARTIAL;
    L.cls = 2;                                           // diagnostics class: project / adjoint
    L.flops = 8.0 * (double)nr * (double)nr * (double)ns;
    // Every partial slab is written in full by the GEMM before the reduction
    // reads it, so no part of the array has to start at zero.
    if (cudaMemcpyAsync(base, &p, sizeof(GProb), cudaMemcpyHostToDevice, st) != cudaSuccess) return TLR_ERR_CUDA;
    if (run_gemm(L, st) != cudaSuccess) return TLR_ERR_CUDA;
    if (reduce_grad(part, nsplit, nr * nr, nr * nr, 0, 1, (cf*)G, st) != cudaSuccess) return TLR_ERR_CUDA;
    // p lives on this stack frame; the copy above was staged before return,
    // but wait for the stream so the caller may reuse V, Dt and G at once.
    if (cudaStreamSynchronize(st) != cudaSuccess) return TLR_ERR_CUDA;
    return TLR_OK;
}
