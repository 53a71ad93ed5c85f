// plain64.h -- the FP64 iteration kernel of PRISM_PLAIN_FP64 (plain64.cu).
#pragma once

#include "internal.h"

namespace prism {

struct P64Args {
    int M = 0, N = 0, Npad = 0, K = 0, S = 0;
    // universe, sorted positions, FP64
    const double* B = nullptr;          // Npad x K
    const double* f = nullptr;          // K
    const double* d = nullptr;          // Npad
    const double* mu = nullptr;         // Npad
    const int* sec_start = nullptr;     // S + 1
    const int* sector = nullptr;        // Npad (-1 = padding)
    // per entry (M x Npad), FP64
    const double *w0 = nullptr, *lo = nullptr, *up = nullptr, *c = nullptr;
    const int* pw_idx = nullptr;        // -1 = plain L1 entry
    const double* pw_bp = nullptr;      // n_pw x MAXBP
    const double* pw_sl = nullptr;      // n_pw x (MAXBP - 1)
    const int* pw_nbp = nullptr;
    const double *band_lo = nullptr, *band_hi = nullptr;   // M x S
    const double* tau = nullptr;        // M (+inf = no cap)
    const double *flo = nullptr, *fhi = nullptr;   // M x K factor-exposure bounds, or null
    int* sflag = nullptr;               // M x K: the iterations' factor rows at a bound (for the polish)
    const int* skip = nullptr;          // M: accounts the capacity test rejected
    // FP64 state (M x Npad), kept between calls of the same solve
    double *z = nullptr, *y = nullptr, *X = nullptr;
    double *rho_state = nullptr, *theta_state = nullptr;   // M
    double *s_state = nullptr, *ys_state = nullptr;        // M x K (factor-exposure block)
    // what the polish reads
    float* zf = nullptr;                // M x Npad
    float *nu_f = nullptr, *eta_hi_f = nullptr, *eta_lo_f = nullptr, *theta_f = nullptr;
    int *iters = nullptr, *active = nullptr, *status = nullptr;
    double alpha = 1.5, eps = 5e-4, rho0 = 3.0;
    int max_iter = 4000, min_iter = 20, adapt_every = 25;
    int resume = 0;                     // 1: continue from z, y, rho_state (a tighter second pass)
};

size_t p64_smem_bytes();
void launch_admm64(const P64Args& A, cudaStream_t st);

}  // namespace prism
