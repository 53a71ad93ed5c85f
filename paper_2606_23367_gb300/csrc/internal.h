// internal.h -- host/device data structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/prism.h"

namespace prism {

// Penalty grid: rho_j = RHO_MIN * 10^(j / RHO_PER_DECADE), j = 0 .. NRHO-1.
// The Woodbury capacitance (2F)^{-1} + B' Delta_j^{-1} B with Delta_j = diag(2d + rho_j)
// is precomputed for every grid point when the universe is created, so a
// per-account penalty change costs nothing but an index.
constexpr int NRHO = 33;
constexpr double RHO_MIN = 1e-4;
constexpr int RHO_PER_DECADE = 4;
inline double rho_of(int j) { return RHO_MIN * pow(10.0, double(j) / RHO_PER_DECADE); }

constexpr int KMAX = 64;     // largest factor count
constexpr int SMAX = 64;     // largest sector count
constexpr int MAXLOT = 4;    // lots per entry the prox keeps (more are rejected)
constexpr int MAXBP = MAXLOT + 3;   // breakpoints per entry: l, kinks (<= MAXLOT), w0, u

void set_error(const std::string& msg);

// A universe resident on one device, assets reordered so that each sector is
// a contiguous range (sorted position p <-> original asset perm[p]).
struct Universe {
    int device = 0;
    int N = 0, K = 0, S = 0, Npad = 0;
    std::vector<int> perm, inv_perm, sec_start;   // host copies
    int* d_inv_perm = nullptr;     // N: original asset -> sorted position
    int* d_perm = nullptr;         // N: sorted position -> original asset
    int* d_sec_start = nullptr;    // S+1
    int* d_sector = nullptr;       // Npad: sector of each sorted position (-1 = padding)
    // segments: the nonempty intersections of the 32-position quarters [32q, 32q + 32) with the
    // sector ranges, numbered in position order (so each sector's segments are consecutive)
    int nq = 0, nseg = 0;          // nq = Npad / 32
    int* d_qseg = nullptr;         // nq + 1: first segment of each quarter
    int* d_sseg = nullptr;         // S + 1: first segment of each sector
    double* d_B64 = nullptr;       // Npad x K (sorted, zero rows in padding)
    double* d_f64 = nullptr;       // K
    double* d_d64 = nullptr;       // Npad (1 in padding)
    double* d_mu64 = nullptr;      // Npad (0 in padding)
    double* d_Bn1 = nullptr;       // Npad: sum_k |B_ik|
    float* d_Bn1f = nullptr;       // Npad: its FP32 copy
    float* d_B32 = nullptr;        // Npad x K
    float* d_B32p = nullptr;       // Npad x 64 (factors zero-padded to 64, rows 256-byte aligned)
    float* d_f32 = nullptr;        // K
    float* d_d32 = nullptr;        // Npad
    float* d_mu32 = nullptr;       // Npad
    __nv_bfloat16* d_B16 = nullptr;   // Npad x K  (row-major, K contiguous)
    __nv_bfloat16* d_Bt16 = nullptr;  // K x Npad  (assets contiguous)
    __nv_bfloat16* d_B16p = nullptr;  // Npad x 64 (factors zero-padded to 64)
    __nv_bfloat16* d_Bt16p = nullptr; // 64 x Npad
    float* d_Cinv32 = nullptr;     // NRHO x K x K, capacitance inverses for FP32 B
    float* d_Cinv16 = nullptr;     // NRHO x K x K, for the BF16-rounded B
    // factor-exposure bounds (Eq. 1 rows B'w in [lo, hi]) split off as s = B'x with penalty rho:
    // the x-update then has capacitance (2F + rho I)^{-1} + B' Delta^{-1} B, and needs the Gram
    // matrices G_j = B' Delta_j^{-1} B themselves
    float* d_G32 = nullptr;        // NRHO x K x K, G_j for FP32 B
    float* d_G16 = nullptr;        // NRHO x K x K, G_j for the BF16-rounded B
    float* d_CinvF32 = nullptr;    // NRHO x K x K, ((2F + rho_j I)^{-1} + G_j)^{-1}, FP32 B
    float* d_CinvF16 = nullptr;    // the same for the BF16-rounded B
    double dmin = 0.0;             // smallest idiosyncratic variance d_i (strong convexity of the risk)
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
};

// Device workspace of one solve (grown on demand, kept by the universe's owner).
struct Workspace {
    size_t bytes = 0;
    std::vector<void*> blocks;
    void* alloc(size_t n);        // 256-byte aligned, zero-filled by the caller if needed
    void release();
};

// Per-account transition-cost description on the device (sorted layout, M x Npad).
struct BatchDev {
    int M = 0, Npad = 0;
    bool has_lots = false, has_cap = false;
    // FP64 per entry (polish / certification)
    double *w0 = nullptr, *lo = nullptr, *up = nullptr, *c = nullptr;
    // FP32 per entry (iterations)
    float *w0f = nullptr, *lof = nullptr, *upf = nullptr, *cf = nullptr;
    // piecewise-linear pieces for entries with lots: MAXBP breakpoints, MAXBP-1 slopes
    int* pw_idx = nullptr;         // M x Npad: -1 = plain L1 entry, else row in pw tables
    int n_pw = 0;
    double *pw_bp = nullptr, *pw_sl = nullptr;   // n_pw x MAXBP, n_pw x (MAXBP-1)
    float *pw_bpf = nullptr, *pw_slf = nullptr;
    int* pw_nbp = nullptr;         // n_pw
    double *band_lo = nullptr, *band_hi = nullptr;   // M x S
    float *band_lof = nullptr, *band_hif = nullptr;
    double* tau = nullptr;         // M
    float* tauf = nullptr;
    bool has_fac = false;          // some factor exposure has a finite bound
    double *flo = nullptr, *fhi = nullptr;    // M x K factor-exposure bounds (+-inf = none)
    float *flof = nullptr, *fhif = nullptr;
    int* member = nullptr;         // M x Npad: 1 if the entry belongs to the account
};

}  // namespace prism

struct prism_universe {
    prism::Universe u;
};

// What the backward pass needs of a polished solve: the identified active set and
// the ragged layout. Device buffers are owned by the state; the universe must outlive it.
struct prism_state {
    const prism_universe* uh = nullptr;
    int device = 0, M = 0, N = 0, Npad = 0, K = 0, S = 0;
    int64_t nnz = 0;
    int64_t* offsets = nullptr;       // M + 1
    int32_t* asset_idx = nullptr;     // nnz, or null for full-universe accounts
    double* W = nullptr;              // M x Npad polished weights (sorted layout)
    uint8_t* flags = nullptr;         // M x Npad active-set flags
    int* wband = nullptr;             // M x S working bands
    int* wcap = nullptr;              // M
    int* status = nullptr;            // M
    std::vector<void*> blocks;        // every device allocation above and the scratch below
    // backward scratch (allocated on first use)
    int fmax = 0;
    double *G = nullptr, *U = nullptr, *DW0 = nullptr, *Fh = nullptr, *Ft = nullptr, *Y = nullptr;
    int *Flist = nullptr, *NZlist = nullptr, *err = nullptr;
    double *out_dmu = nullptr, *out_dd = nullptr, *out_dB = nullptr, *out_dw0 = nullptr, *in_g = nullptr;
};
