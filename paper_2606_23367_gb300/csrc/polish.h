// polish.h -- FP64 polish / certification state.
#pragma once

#include "internal.h"

namespace prism {

constexpr int PMAXROWS = 24;   // working rows per polish: budget + held bands + cap

struct PolDev {
    int M = 0, N = 0, Npad = 0, K = 0, S = 0;
    const double* B64 = nullptr;
    const double* f64 = nullptr;
    const double* d64 = nullptr;
    const double* mu64 = nullptr;
    const float* B32 = nullptr;         // FP32 B (Npad x K)
    const float* B32p = nullptr;        // FP32 B zero-padded to 64 factors (Npad x 64)
    const double* Bn1 = nullptr;        // sum_k |B_ik| per asset (error bound of that product)
    const float* Bn1f = nullptr;        // its FP32 copy
    const float* mu32 = nullptr;
    const float* w0f = nullptr;         // FP32 copies of the per-entry data (M x Npad)
    const float* lof = nullptr;
    const float* upf = nullptr;
    const float* cf = nullptr;
    const int* sec_start = nullptr;
    const int* sector = nullptr;
    const double* w0 = nullptr;         // M x Npad
    const double* lo = nullptr;
    const double* up = nullptr;
    const double* c = nullptr;
    const int* pw_idx = nullptr;
    const double* pw_bp = nullptr;
    const double* pw_sl = nullptr;
    const double* pw_phi_lo = nullptr;  // phi at the left breakpoint of each PWL row
    const int* pw_nbp = nullptr;
    const double* band_lo = nullptr;    // M x S
    const double* band_hi = nullptr;
    const double* tau = nullptr;        // M (+inf = none)
    const double* flo = nullptr;        // M x K factor-exposure bounds, or null (no factor rows)
    const double* fhi = nullptr;
    const int* sflag = nullptr;         // M x K: factor rows the iterations hold at a bound
    int* wfac = nullptr;                // M x K working factor rows (+1 upper, -1 lower, 0 none)
    double* kappa = nullptr;            // M x K their multipliers (output)
    const float* z = nullptr;           // ADMM iterate, M x Npad
    const float* nu_f = nullptr;        // ADMM budget multiplier, M
    const float* eta_hi_f = nullptr;    // M x S
    const float* eta_lo_f = nullptr;
    const float* theta_f = nullptr;     // M
    int* skip = nullptr;                // M: 1 = leave this account alone
    const int* sel = nullptr;           // M: when set, only the accounts with sel[a] == gen
    int gen = 0;
    // state and scratch
    int8_t* st = nullptr;               // M x Npad entry state
    int* wband = nullptr;               // M x S working bands
    int* wcap = nullptr;                // M
    int* done = nullptr;                // M: 0 running, 1 certified, 2 failed
    int* Flist = nullptr;               // M x FMAX
    int* NZlist = nullptr;              // M x FMAX
    double* Fsig = nullptr;             // M x FMAX cap sign of each free entry
    double* Fdinv = nullptr;            // M x FMAX 1/d of each free entry
    double* Y = nullptr;                // M x FMAX x (PMAXROWS + 1)
    int FMAX = 0;
    double* fh64 = nullptr;             // M x 64: f .* (B' w) of the solved point
    float* fh32 = nullptr;              // M x K, its FP32 copy (operand of the product)
    double* quad = nullptr;             // M: w' B F B' w
    double* fhmax = nullptr;            // M: max_k |f_k h_k|
    int* ndep = nullptr;                // M: working rows dependent on the free set
    int* pending = nullptr;             // unused
    // outputs
    double* W = nullptr;                // M x Npad weights (FP64)
    double* nu = nullptr;               // M
    double* lam = nullptr;              // M x S
    double* theta = nullptr;            // M
    double* diag = nullptr;             // M x PRISM_NDIAG
    int* status = nullptr;              // M
    double dmin = 0.0;                  // smallest d_i of the universe: 2 Sigma >= 2 dmin I
    double tol_dual = 1e-11;
    double tol_primal = 1e-12;
};

size_t polish_smem_bytes();
void launch_classify(const PolDev& P, cudaStream_t st);
void launch_polish(const PolDev& P, int rounds, cudaStream_t st);
void launch_fallback(const PolDev& P, cudaStream_t st);
void launch_finish_status(const PolDev& P, double eps, cudaStream_t st);
// Per-entry active-set flags of the polished solution for the adjoint:
// bit 0 free; bit 1 fixed at an interior breakpoint (a kink of phi, moving with w0);
// bits 2-3 the cap row's coefficient (1: +1, 2: -1, 0: none).
void launch_adjoint_flags(const PolDev& P, uint8_t* flags, cudaStream_t st);
// The backward-pass state of a polished solve (adjoint.cu).
int make_backward_state(const prism_universe* uh, const PolDev& P, const int* status_dev, const int64_t* offsets_dev,
                        const int32_t* asset_idx_dev, int64_t nnz, cudaStream_t st, prism_state** out);

}  // namespace prism
