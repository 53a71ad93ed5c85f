// solver.h -- device-side state of one batched solve and the kernel launchers.
#pragma once

#include "internal.h"

namespace prism {

// Everything the iteration kernels touch, passed by value to every kernel.
struct Dev {
    int M = 0, N = 0, Npad = 0, K = 0, S = 0;
    // universe (sorted order)
    const float* B32 = nullptr;
    const float* d32 = nullptr;
    const float* mu32 = nullptr;
    const int* sec_start = nullptr;
    const int* sector = nullptr;
    const __nv_bfloat16* B16 = nullptr;
    const __nv_bfloat16* Bt16 = nullptr;
    const __nv_bfloat16* B16p = nullptr;    // Npad x 64, factors zero-padded (tensor-core operand)
    const __nv_bfloat16* Bt16p = nullptr;   // 64 x Npad
    const float* Cinv = nullptr;        // NRHO x K x K for the mode's B
    // per-entry account data (M x Npad), FP32
    const float* w0 = nullptr;
    const float* lo = nullptr;
    const float* up = nullptr;
    const float* c = nullptr;
    const int* pw_idx = nullptr;        // -1 = plain L1 entry
    const float* pw_bp = nullptr;       // n_pw x MAXBP
    const float* pw_sl = nullptr;       // n_pw x (MAXBP-1)
    const int* pw_nbp = nullptr;
    const float* band_lo = nullptr;     // M x S
    const float* band_hi = nullptr;
    const float* tau = nullptr;         // M (inf = no cap)
    // ADMM state (M x Npad)
    float* z = nullptr;
    float* y = nullptr;
    float* X = nullptr;                 // Delta^{-1}(mu + rho z - y), FP32
    float* v = nullptr;                 // relaxed x plus scaled dual, input of the prox
    __nv_bfloat16* Xhi = nullptr;       // X split for the BF16 products: X ~ Xhi + Xlo
    __nv_bfloat16* Xlo = nullptr;
    float* Ppart = nullptr;             // nsplit x M x pstride partial B'X
    int pstride = 0;                    // row stride of Ppart: K (SIMT G2) or 64 (tensor-core G2)
    float* Q = nullptr;                 // M x K
    __nv_bfloat16* Qhi = nullptr;       // M x 64 split of Q (factors zero-padded)
    __nv_bfloat16* Qlo = nullptr;
    int nsplit = 1;
    int g2_sets = 0;                    // tile shape of the tensor-core G2 (0 = automatic)
    // per-account control
    int* rho_idx = nullptr;
    int* iters = nullptr;
    int* active = nullptr;
    int* status = nullptr;
    float* nu = nullptr;                // M warm start
    float* dnu = nullptr;               // M last change of nu (margin of the streaming prox)
    float* eta_hi = nullptr;            // M x S warm start / result
    float* eta_lo = nullptr;            // M x S
    float* theta = nullptr;             // M cap multiplier
    float* rp = nullptr;                // M residuals
    float* rd = nullptr;
    int* n_active = nullptr;            // [0] accounts still iterating, [1] pipeline error flags
    int* err = nullptr;                 // = n_active + 1
    float alpha = 1.6f;
    float eps_admm = 3e-4f;
    int min_iter = 20;
    int max_iter = 4000;
    int adapt_every = 25;
    bool bf16 = false;                  // X / Q split in BF16 for tensor-core products
    int raw_out = 0;                    // diagnostics: G4 writes B Q itself into v
    int stream_prox = 0;                // prox in the streaming form (no lots, no turnover cap)
    // the streaming pass fused into the tensor-core x-update (k_tc_xprox), finished per
    // account by k_prox_roots. Partials are indexed [row][account], rows as follows.
    int fused = 0;
    int uniform = 0;                    // every account has uniform l and c (lo_u, c_u not NaN)
    // the accounts [m0, m1) this launch works on (m1 = 0: all M); G2, G3 and the fused kernels
    // take it, so that two halves of a book can iterate as independent chains
    int m0 = 0, m1 = 0;
    int nq = 0, nseg = 0, nt = 0;       // quarters (32 positions), segments, asset tiles (128 positions)
    const int* qseg = nullptr;          // nq + 1: first segment of each quarter
    const int* sseg = nullptr;          // S + 1: first segment of each sector
    const float* lo_u = nullptr;        // M: l when equal over the account's positions, else NaN
    const float* c_u = nullptr;         // M: c when equal over its positions with u > l, else NaN
    float* SOp = nullptr;               // nseg x M: sum of l_i over the segment's entries pinned at L
                                        // (written only for accounts whose l differs over positions)
    float* Rt = nullptr;                // M x 5 x nt: residual maxima (rp, rd, nx, nz, ny) of the pinned
                                        // entries of each asset tile; rp is NaN when one was not finite
    unsigned* Cm = nullptr;             // M x nq: bit b of quarter q set = entry 32q + b not pinned at L
    unsigned long long* pcount = nullptr;   // profile mode: [0] candidates, [1] entries of the fused pass
    float* crec = nullptr;              // M x Npad x 8: (v, w0, u, z, y, mu, d, -) of each such candidate
    // G2 and G3 folded into the fused iteration: k_tc_xprox leaves B'X of the entries it pinned
    // (one partial set per asset tile, xp_sets x M x 64) and k_prox_roots adds the candidates and
    // solves for Q. An account whose P cannot be completed that way (its penalty
    // changed, or entries pinned by the fused pass were rewritten) has needP set and X rewritten in
    // full: the next iteration's G2 and G3 run for such accounts only (needP == null: for all)
    float* Pxp = nullptr;
    int xp_sets = 0;
    int fold = 0;                       // the fold is on (k_tc_xprox writes no X, forms its partial)
    // tile counter of the persistent fused x-update for this launch's chain: [0] next tile,
    // [1] CTAs done claiming (the last resets both); null = one CTA per tile
    unsigned* xq_ctr = nullptr;
    int xq_share = 1;                   // chains iterating side by side (each launches 2 x SMs / this CTAs)
    int* needP = nullptr;               // M, nonzero = P and Q from the product kernels
    unsigned long long* stats = nullptr;  // [0] prox calls, [1] sector-edge evaluations, [2] budget evaluations
    // factor-exposure bounds (the Eq. 1 rows B'w in [flo, fhi]) as a second splitting block
    // s = B'x with penalty rho and unscaled dual ys; null when the book has none. The small
    // solve updates s and ys and leaves the block's residuals in rps, rds for the convergence
    // test, and sflag (+1 at the upper bound, -1 at the lower, 0 inside) for the polish
    const float* flo = nullptr;         // M x K
    const float* fhi = nullptr;
    const float* G = nullptr;           // NRHO x K x K Gram matrices B' Delta_j^{-1} B
    float* s = nullptr;                 // M x K
    float* ys = nullptr;                // M x K
    float* rps = nullptr;               // M
    float* rds = nullptr;               // M
    int* sflag = nullptr;               // M x K
    // failure-path test only (environment PRISM_TEST_STALLED_WAIT_NS): the tensor-core G2 issues
    // no loads and its first bounded wait, on a barrier nothing completes, runs out after this
    // many ns; 0 in every normal call
    unsigned long long stall_ns = 0;
};

// launchers (admm.cu)
void launch_init_state(const Dev& D, cudaStream_t st);
void launch_gemm_P(const Dev& D, cudaStream_t st);       // G2: Ppart = X B (SIMT)
void launch_small_solve(const Dev& D, cudaStream_t st, bool pdl = false);  // G3: Q = Cinv * sum(Ppart)
void launch_gemm_x(const Dev& D, cudaStream_t st);       // G4: v from X - Delta^{-1} B Q (SIMT)
// G5/G6: projection, duals, control. cold: the staged form even for L1-only books (the first
// calls of a solve, before the multipliers have warm starts for the streaming form's margin)
void launch_prox(const Dev& D, cudaStream_t st, bool cold = false);
void launch_count_active(const Dev& D, cudaStream_t st);
void launch_mark_timeout(const Dev& D, cudaStream_t st);
int choose_nsplit(int M, int N);

// tensor-core products (tc_gemm.cu)
bool tc_available();                                     // tensor-map encoder reachable
int tc_nsplit(int M, int N, int* chunk, int sets = 0);   // partial sets of the tensor-core G2 (its asset chunk)
void launch_tc_gemm_P(const Dev& D, cudaStream_t st, bool pdl = false);    // G2 on tcgen05
void launch_tc_gemm_x(const Dev& D, cudaStream_t st);    // G4 on tcgen05 with fused epilogue
void launch_tc_xprox(const Dev& D, cudaStream_t st, bool pdl = false);     // G4 + the streaming pass of G5 (fused)
void launch_prox_roots(const Dev& D, cudaStream_t st, bool pdl = false);   // G5/G6 per account after k_tc_xprox
void launch_uniform(const Dev& D, float* lo_u, float* c_u, cudaStream_t st);   // per-account uniform l, c
constexpr int XP_NQMAX = 1024;                           // quarters the roots kernel holds (N <= 32768)
inline int xp_sets_for(int N) { return (N + 127) / 128; }   // partial sets of the fused x-update
void launch_refresh_X(const Dev& D, cudaStream_t st);    // X of every entry of the active accounts from z, y

}  // namespace prism
