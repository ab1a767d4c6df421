// Device-side state of the ADMM / L-BFGS solver: every vector lives in the
// panel layout of the stacked unknown (2 * n floats), every scalar decision
// (step length, pair acceptance, memory reset) stays in device memory so the
// whole solve is a fixed sequence of launches with no host round trip.
#pragma once

#include "internal.h"

namespace tlr {

enum ScalarSlot { SC_ALPHA = 0, SC_F, SC_F0, SC_C0, SC_C1, SC_C2, SC_C3, SC_C4, SC_GAMMA, SC_COUNT };
// SI_RFLAG: 1 when this iteration's direction failed the descent test and was
// replaced by -g (the iteration already counts as a restart)
enum IntSlot { SI_CNT = 0, SI_NEWEST, SI_ITERS, SI_RESTARTS, SI_STATUS, SI_RFLAG, SI_COUNT };

// compact L-BFGS: pairs per inner-product pass, and the partial storage for
// the largest memory (32 pairs), followed by one slab of <g, g> partials
constexpr int kLbGroup = 10;
constexpr long long kLbGGOff = (long long)kRedBlocks * 5 * kLbGroup * ((32 + kLbGroup - 1) / kLbGroup);
constexpr long long kLbPartDoubles = kLbGGOff + kRedBlocks;

struct SolverDev {
    long long n2;        // floats per theta-space vector (2 * n_theta)
    int m;               // L-BFGS memory
    int ring;            // m + 1 slots: the slot after the newest is always free
    float *x, *z, *u, *v, *g, *gf, *d, *q;
    float *sh, *yh;      // ring of s and y vectors, ring * n2 floats each
    double* rho_h;       // [ring] 1 / <s, y>
    double* sy_h;        // [ring] <s, y>
    double* yy_h;        // [ring] <y, y>
    double* acoef;       // [64] direction coefficients: [j] of s_j, [32 + j] of y_j (j-th newest)
    double* SYm;         // [ring * ring] <s_a, y_b> by slot
    double* YYm;         // [ring * ring] <y_a, y_b> by slot
    double* lbpart;      // kRedBlocks * 5 * kLbGroup partials per group of pairs (direction inner products)
    double* sc;          // ScalarSlot values
    int* ints;           // IntSlot values
    double* fhist;       // [TLR_MAX_HIST]
    double* part;        // 2 * kRedBlocks partial slabs
};

cudaError_t sv_norm_part(const cf* R, long long n, double* part, cudaStream_t st);
cudaError_t sv_record_f0(const SolverDev& S, const double* partf, cudaStream_t st);
cudaError_t sv_admm_init(const SolverDev& S, cudaStream_t st);
cudaError_t sv_admm_resume(const SolverDev& S, cudaStream_t st);
cudaError_t sv_xupdate_start(const SolverDev& S, double rho, cudaStream_t st);
cudaError_t sv_direction(const SolverDev& S, cudaStream_t st);
cudaError_t sv_dots3(const SolverDev& S, double* part, cudaStream_t st);
// part6: nb6 blocks of 6 partial sums (kRedBlocks from dots6_part, or one per
// CTA of the packed-residual inner products)
cudaError_t sv_line_search(const SolverDev& S, const double* part6, int nb6, const double* part3, double rho,
                           cudaStream_t st);
cudaError_t sv_step_residual(cf* R, const cf* A1, const cf* A2, long long n, const double* alpha,
                             double* partf, cudaStream_t st);
cudaError_t sv_step_theta(const SolverDev& S, cudaStream_t st);
cudaError_t sv_pair_prep(const SolverDev& S, double rho, double* part, cudaStream_t st);
cudaError_t sv_pair_accept(const SolverDev& S, const double* part3, const double* partf, int nf, cudaStream_t st);
cudaError_t sv_admm_zu(const SolverDev& S, double lam, double rho, cudaStream_t st);

}  // namespace tlr
