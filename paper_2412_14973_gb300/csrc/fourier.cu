// Time <-> frequency pipeline of the examples: the wavefields are recorded in
// time, transformed to the frequency domain and solved one frequency at a
// time; the Green's function comes back to time (time-offset gathers) by the
// inverse transform over the solved band.
//
// Traces are stored trace-major, x_t[tr][t] (tr = s nr + r for data, a nr +
// b for X), nt samples each.  X(omega_k) = sum_t x(t) exp(-2 pi i k t / nt)
// (unnormalised), k = 0 .. nt/2; the inverse puts the band [f0, f0 + nf) back
// (zero elsewhere) and divides by nt.  The real FFTs are cuFFT plans over a
// chunk of traces; the band gather / scatter between the trace-major spectrum
// and the frequency-major stack (stack[f][tr], one ns x nr panel per
// frequency) are transposes through shared memory, coalesced on both sides.
#include <cufft.h>

#include <string>

#include "internal.h"

namespace tlr {

namespace {

constexpr int FT = 32;

// out[f][tr] = spec[tr][f0 + f] for one chunk of traces (tr0 .. tr0 + ntr_c)
__global__ void __launch_bounds__(256) k_band_gather(const cf* __restrict__ spec, long long ntr_c, int nh, int f0,
                                                     int nf, cf* __restrict__ out, long long ld_out) {
    __shared__ cf t[FT][FT + 1];
    const long long tr0 = (long long)blockIdx.x * FT;
    const int fb = blockIdx.y * FT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < FT; r += 8) {
        const long long tr = tr0 + r;
        const int f = fb + tx;
        t[r][tx] = (tr < ntr_c && f < nf) ? spec[tr * nh + f0 + f] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < FT; r += 8) {
        const int f = fb + r;
        const long long tr = tr0 + tx;
        if (f < nf && tr < ntr_c) out[(long long)f * ld_out + tr] = t[tx][r];
    }
}

// spec[tr][h] = in[h - f0][tr] inside the band, 0 outside, for one chunk
__global__ void __launch_bounds__(256) k_band_scatter(const cf* __restrict__ in, long long ld_in, long long ntr_c,
                                                      int nh, int f0, int nf, cf* __restrict__ spec) {
    __shared__ cf t[FT][FT + 1];
    const long long tr0 = (long long)blockIdx.x * FT;
    const int hb = blockIdx.y * FT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < FT; r += 8) {
        const int h = hb + r;
        const long long tr = tr0 + tx;
        const int f = h - f0;
        t[r][tx] = (tr < ntr_c && f >= 0 && f < nf) ? in[(long long)f * ld_in + tr] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < FT; r += 8) {
        const long long tr = tr0 + r;
        const int h = hb + tx;
        if (tr < ntr_c && h < nh) spec[tr * nh + h] = t[tx][r];
    }
}

__global__ void k_scale(float* x, long long n, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= s;
}

const char* cufft_msg(cufftResult r) {
    switch (r) {
        case CUFFT_SUCCESS: return "success";
        case CUFFT_ALLOC_FAILED: return "cuFFT allocation failed";
        case CUFFT_INVALID_VALUE: return "cuFFT invalid value";
        case CUFFT_EXEC_FAILED: return "cuFFT execution failed";
        case CUFFT_SETUP_FAILED: return "cuFFT setup failed";
        case CUFFT_INVALID_SIZE: return "cuFFT invalid size";
        default: return "cuFFT error";
    }
}

// traces per chunk: the chunk's real and complex buffers within ~256 MB
long long chunk_traces(long long ntr, long long nt) {
    const long long per = nt * 4 + (nt / 2 + 1) * 8;
    long long c = std::max(1LL, (256LL << 20) / per);
    return std::min(ntr, c);
}

}  // namespace

int fft_stack(bool forward, const float* x_t_in, const cf* X_in, long long ntr, long long nt, long long f0,
              long long nf, cf* X_out, float* x_t_out, cudaStream_t st, std::string& err) {
    const long long nh = nt / 2 + 1;
    const long long C = chunk_traces(ntr, nt);
    cf* spec = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&spec, (size_t)C * nh * sizeof(cf), st);
    if (e != cudaSuccess) {
        err = std::string("frequency stack: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? TLR_ERR_NOMEM : TLR_ERR_CUDA;
    }
    int rc = TLR_OK;
    cufftHandle plan = 0, plan_tail = 0;
    long long planned = 0, planned_tail = 0;
    for (long long tr0 = 0; tr0 < ntr && rc == TLR_OK; tr0 += C) {
        const long long c = std::min(C, ntr - tr0);
        cufftHandle* p = c == C ? &plan : &plan_tail;
        long long& have = c == C ? planned : planned_tail;
        if (have != c) {
            int n[1] = {(int)nt};
            const cufftResult r = cufftPlanMany(p, 1, n, nullptr, 1, (int)nt, nullptr, 1, (int)nh,
                                                forward ? CUFFT_R2C : CUFFT_C2R, (int)c);
            if (r != CUFFT_SUCCESS) {
                err = cufft_msg(r);
                rc = r == CUFFT_ALLOC_FAILED ? TLR_ERR_NOMEM : TLR_ERR_CUDA;
                break;
            }
            cufftSetStream(*p, st);
            have = c;
        }
        const dim3 grid((unsigned)((c + FT - 1) / FT), (unsigned)(((forward ? nf : nh) + FT - 1) / FT));
        cufftResult r;
        if (forward) {
            r = cufftExecR2C(*p, const_cast<float*>(x_t_in) + tr0 * nt, reinterpret_cast<cufftComplex*>(spec));
            if (r == CUFFT_SUCCESS) {
                k_band_gather<<<grid, 256, 0, st>>>(spec, c, (int)nh, (int)f0, (int)nf, X_out + tr0, ntr);
                counted(1);
            }
        } else {
            k_band_scatter<<<grid, 256, 0, st>>>(X_in + tr0, ntr, c, (int)nh, (int)f0, (int)nf, spec);
            counted(1);
            r = cufftExecC2R(*p, reinterpret_cast<cufftComplex*>(spec), x_t_out + tr0 * nt);
            if (r == CUFFT_SUCCESS) {
                k_scale<<<1024, 256, 0, st>>>(x_t_out + tr0 * nt, c * nt, 1.f / (float)nt);
                counted(1);
            }
        }
        if (r != CUFFT_SUCCESS) {
            err = cufft_msg(r);
            rc = TLR_ERR_CUDA;
        } else if ((e = cudaGetLastError()) != cudaSuccess) {
            err = cudaGetErrorString(e);
            rc = TLR_ERR_CUDA;
        }
    }
    if (e == cudaSuccess && rc == TLR_OK) e = cudaStreamSynchronize(st);   // plans are destroyed below
    if (e != cudaSuccess && rc == TLR_OK) {
        err = cudaGetErrorString(e);
        rc = TLR_ERR_CUDA;
    }
    if (plan) cufftDestroy(plan);
    if (plan_tail) cufftDestroy(plan_tail);
    cudaFreeAsync(spec, st);
    return rc;
}

}  // namespace tlr
