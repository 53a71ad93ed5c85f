// polish.cu -- FP64 active-set polish (G7) and KKT / feasibility certification (G8).
//
// From the ADMM iterate z each weight is classified exactly as the projection
// left it: on a breakpoint of its transition cost (a box bound, w0 or a lot
// kink) -> FIXED there, otherwise FREE inside one linear segment. Bands the
// projection held at an edge and an active turnover cap become equality rows
// next to the budget. The equality-constrained QP on the free set F,
//
//   2 Sigma_FF w_F + E_F' lambda = mu_F - s_F - 2 Sigma_FA w_A,   E_F w_F = e,
//
// is solved in FP64 through a Cholesky factor of Sigma_FF itself when |F| <= K, else
// through the Woodbury identity
//   Sigma_FF^{-1} = D_F^{-1} - D_F^{-1} B_F (F^{-1} + B_F' D_F^{-1} B_F)^{-1} B_F' D_F^{-1}
// (K x K Cholesky), and a Schur complement over the working rows, so the
// budget row holds exactly in FP64. Then every KKT condition (Sec. 4.4) is
// checked from the recomputed FP64 gradient 2 (B F B' w + D w) - mu: free
// weights must stay inside their segment, fixed weights must satisfy
// -(g_i + nu + lambda_s(i)) in [left slope, right slope] of phi_i + theta |.-w0_i|,
// bands/cap outside the working set must hold and those inside need the right
// multiplier sign. Violators switch state (primal-dual active-set rounds); a
// round without violators certifies the account, and its residuals are the
// external diagnostics of Sec. 4.4 written to the result.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "polish.h"

namespace prism {

constexpr int PB = 256;             // threads per polish block
constexpr int ST_FREE = 32;         // state code: free in segment (code - ST_FREE)

// Breakpoints / slopes of phi_i restricted to [l_i, u_i] for one entry (FP64).
struct Pieces {
    double bp[MAXBP];
    double sl[MAXBP - 1];
    int nb;
    double w0;
    double c;          // plain L1 cost (pw < 0)
    double phi_lo;     // phi at bp[0] for piecewise-linear rows
    int pw;
};

__device__ __forceinline__ void entry_pieces(const PolDev& P, size_t e, Pieces& pc) {
    const double w0 = P.w0[e], lo = P.lo[e], up = P.up[e];
    pc.w0 = w0;
    const int pw = P.pw_idx ? P.pw_idx[e] : -1;
    pc.pw = pw;
    pc.c = P.c[e];
    pc.phi_lo = 0.0;
    if (pw >= 0) {
        pc.phi_lo = P.pw_phi_lo[pw];
        pc.nb = P.pw_nbp[pw];
        for (int j = 0; j < pc.nb; ++j) pc.bp[j] = P.pw_bp[(size_t)pw * MAXBP + j];
        for (int j = 0; j + 1 < pc.nb; ++j) pc.sl[j] = P.pw_sl[(size_t)pw * (MAXBP - 1) + j];
        return;
    }
    const double c = P.c[e];
    if (!(up > lo)) { pc.nb = 1; pc.bp[0] = lo; return; }
    if (w0 > lo && w0 < up) {
        pc.nb = 3; pc.bp[0] = lo; pc.bp[1] = w0; pc.bp[2] = up; pc.sl[0] = -c; pc.sl[1] = c;
    } else {
        pc.nb = 2; pc.bp[0] = lo; pc.bp[1] = up; pc.sl[0] = (w0 <= lo) ? c : -c;
    }
}

// The per-entry inputs of the checks, loaded together so that one thread has many
// independent loads in flight (the int8 state stores would otherwise order them).
struct EntryRaw {
    double w0, lo, up, c, W, d, mu, bn1;
    int code, sec, pw;
};

__device__ __forceinline__ void load_raw(const PolDev& P, size_t base, int p, EntryRaw& r) {
    const size_t e = base + p;
    r.w0 = P.w0[e]; r.lo = P.lo[e]; r.up = P.up[e]; r.c = P.c[e];
    r.W = P.W[e]; r.d = P.d64[p]; r.mu = P.mu64[p]; r.bn1 = P.Bn1[p];
    r.code = P.st[e];
    r.sec = P.sector[p];
    r.pw = P.pw_idx ? P.pw_idx[e] : -1;
}

__device__ __forceinline__ void pieces_from(const PolDev& P, const EntryRaw& r, Pieces& pc) {
    pc.w0 = r.w0;
    pc.pw = r.pw;
    pc.c = r.c;
    pc.phi_lo = 0.0;
    if (r.pw >= 0) {
        pc.phi_lo = P.pw_phi_lo[r.pw];
        pc.nb = P.pw_nbp[r.pw];
        for (int j = 0; j < pc.nb; ++j) pc.bp[j] = P.pw_bp[(size_t)r.pw * MAXBP + j];
        for (int j = 0; j + 1 < pc.nb; ++j) pc.sl[j] = P.pw_sl[(size_t)r.pw * (MAXBP - 1) + j];
        return;
    }
    if (!(r.up > r.lo)) { pc.nb = 1; pc.bp[0] = r.lo; return; }
    if (r.w0 > r.lo && r.w0 < r.up) {
        pc.nb = 3; pc.bp[0] = r.lo; pc.bp[1] = r.w0; pc.bp[2] = r.up; pc.sl[0] = -r.c; pc.sl[1] = r.c;
    } else {
        pc.nb = 2; pc.bp[0] = r.lo; pc.bp[1] = r.up; pc.sl[0] = (r.w0 <= r.lo) ? r.c : -r.c;
    }
}

__device__ __forceinline__ double seg_sign(const Pieces& pc, int j) {
    return (pc.bp[j] + pc.bp[j + 1] > 2.0 * pc.w0) ? 1.0 : -1.0;
}

// phi_i(w) in FP64: c|w - w0| for plain entries; for lot entries the value at the
// left breakpoint plus the integral of the segment slopes up to w.
__device__ __forceinline__ double phi_value(const Pieces& pc, double w) {
    if (pc.pw < 0) return pc.c * fabs(w - pc.w0);
    double acc = pc.phi_lo;
    for (int j = 0; j + 1 < pc.nb; ++j) {
        double s1 = fmin(w, pc.bp[j + 1]);
        if (s1 > pc.bp[j]) acc += pc.sl[j] * (s1 - pc.bp[j]);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// classification of the ADMM iterate: entry state codes and working rows
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PB) k_classify(PolDev P) {
    const int a = blockIdx.x;
    const size_t base = (size_t)a * P.Npad;
    if ((P.skip && P.skip[a]) || P.done[a] == 1 || (P.sel && P.sel[a] != P.gen)) return;
    for (int p = threadIdx.x; p < P.N; p += PB) {
        const size_t e = base + p;
        Pieces pc;
        entry_pieces(P, e, pc);
        const float z = P.z[e];
        int code = -1;
        for (int j = 0; j < pc.nb; ++j)
            if (z == float(pc.bp[j])) { code = j; break; }
        if (code < 0) {
            int j = 0;
            while (j + 2 < pc.nb && z > float(pc.bp[j + 1])) ++j;
            code = ST_FREE + j;
        }
        if (pc.nb == 1) code = 0;
        P.st[e] = (int8_t)code;
    }
    if (threadIdx.x < P.S) {
        const int s = threadIdx.x;
        const float nu = P.nu_f[a];
        int wb = 0;
        if (P.eta_hi_f[a * P.S + s] > nu) wb = 1;
        else if (P.eta_lo_f[a * P.S + s] < nu) wb = -1;
        P.wband[a * P.S + s] = wb;
    }
    if (threadIdx.x == 0) P.wcap[a] = (P.theta_f[a] > 0.f) ? 1 : 0;
    if (P.wfac)
        for (int k = threadIdx.x; k < P.K; k += PB) P.wfac[a * P.K + k] = P.sflag ? P.sflag[a * P.K + k] : 0;
}

// ---------------------------------------------------------------------------
// The polish: one block per account runs all of its active-set rounds.
//
// Each round (a) compacts the free set, (b) solves the equality-constrained QP on it,
// (c) checks every KKT condition and switches the violators. The solve factors the
// smaller of Sigma_FF (|F| x |F|) and the Woodbury capacitance (K x K), and the Schur
// complement, in FP32 and then applies FP64
// iterative refinement to the full reduced KKT system
//     [2 Sigma_FF  E_F'] [w_F]   [g0]
//     [E_F         0   ] [lam] = [e ]
// (FP64 residuals, FP32 corrections), which converges to FP64 accuracy because the
// system's condition number times the FP32 unit roundoff is far below one. GB300
// runs FP64 at 1/64 of its FP32 rate, so this keeps the O(min(|F|, K)^2 max(|F|, K))
// factorisation in FP32 and only O(|F| K) per refinement step in FP64.
// ---------------------------------------------------------------------------
constexpr int FS = 64;                    // free entries whose data live in shared memory
constexpr int COL_W = PMAXROWS - 1;       // column of Y holding w_F (FP64)
constexpr int COL_R = PMAXROWS;           // column of Y holding the refinement workspace
constexpr int MAXWROWS = PMAXROWS - 2;    // working rows this kernel accepts
constexpr int IR_STEPS = 6;
constexpr int YS = PMAXROWS + 1;          // row stride of Y
constexpr int AU = 4;                     // entries per lane whose loads are batched in the scans

struct PolishShared {
    float C[KMAX][KMAX + 1];              // FP32 capacitance, then its Cholesky factor
    float Bc[FS][KMAX + 1];               // FP32 rows of B of the first FS free entries
    double Bd[FS][KMAX + 1];              // FP64 rows of B of the first FS free entries
    double Ys[FS][YS];                    // Y rows of the first FS free entries
    double dinv_s[FS], sig_s[FS];
    double gF[FS];                        // B_p . (f .* h) of the free entries, for their checks
    float dinvf_s[FS];
    int Fl_s[FS];
    float Ldinv[KMAX];                    // reciprocal of the Cholesky diagonal
    float f32s[KMAX];                     // FP32 factor variances
    float T[KMAX][PMAXROWS + 1];          // FP32 Woodbury workspace
    double Sf[PMAXROWS][PMAXROWS + 1];    // Schur matrix after pivoted elimination
    double hA[KMAX], fhA[KMAX], fh[KMAX], t64[KMAX];
    alignas(16) float fh32[KMAX];
    double erhs[PMAXROWS], lam[PMAXROWS], rr2[PMAXROWS], dlam[PMAXROWS];
    int order[PMAXROWS], used[PMAXROWS];
    int rows[PMAXROWS];
    int nrows, nF, nNZ, fail, nc, go;
    double fhmax_s, quad_s;               // max_k |f_k h_k| and h' F h of the solved point
    int cntF[PB / 32], cntN[PB / 32];
    int qp[PB / 32][64];                  // per-warp queue of entries that need FP64 work
    float qg[PB / 32][64];
    double sumA[PB / 32], capA[PB / 32], turnA[PB / 32], objA[PB / 32];
    double lam_s[SMAX];
    double kap_s[KMAX];                   // multipliers of the factor rows (0 off the working set)
    float lam_s32[SMAX];
    double blo_s[SMAX], bhi_s[SMAX];      // the account's band edges
    int wb_s[SMAX];                       // working bands (mirrors P.wband of the account)
    int wf_s[KMAX];                       // working factor rows (mirrors P.wfac of the account)
    double flo_s[KMAX], fhi_s[KMAX];      // the account's factor-exposure bounds
    double fixS[SMAX];                    // per sector: sum of the fixed weights
    int secF[FS];                         // sector of each of the first FS free entries                  // its FP32 copy (the filter of the checks)
    double red[PB / 32][8];
    double secsum[SMAX];
    double mmin[PB / 32];
    int mwho[PB / 32];
};

// the free-set data of one account: shared memory when |F| <= FS, else global scratch
struct FreeSet {
    int* Fl;            // entry of each free index
    double* Y;          // rows of YS doubles
    double* dinv;
    double* sig;
    bool in_smem;
};

// Per-warp queue: entries whose checks need FP64 arithmetic are gathered so that the
// (slow on this part) FP64 pipe runs them 32 at a time instead of one lane per warp
struct WarpQueue {
    int* p;
    float* g;
    int n = 0;                            // queued entries (at most 63: one push onto at most 31)
    __device__ void push(bool need, int q, float gv, int lane) {
        const unsigned b = __ballot_sync(0xffffffffu, need);
        if (need) {
            const int pos = n + __popc(b & ((1u << lane) - 1u));
            p[pos] = q;
            g[pos] = gv;
        }
        n += __popc(b);
        __syncwarp();
    }
    // run body(q, g) on 32 queued entries at a time (on all that remain when ``all``)
    template <class Body>
    __device__ void drain(bool all, int lane, Body&& body) {
        while (n >= 32 || (all && n > 0)) {
            const int take = min(n, 32), rest = n - take;
            if (lane < take) body(p[lane], g[lane]);
            __syncwarp();
            int tq = 0;
            float tg = 0.f;
            if (lane < rest) { tq = p[32 + lane]; tg = g[32 + lane]; }
            __syncwarp();
            if (lane < rest) { p[lane] = tq; g[lane] = tg; }
            __syncwarp();
            n = rest;
        }
    }
};

__device__ __forceinline__ double brow64(const PolDev& P, const PolishShared& sh, const FreeSet& F, int q, int k);

// coefficient of free entry q in working row ``row``: the budget (row -1), the band of sector
// row (0 <= row < S), the cap (row S) or the exposure to factor row - S - 1 (sector from shared
// memory when q < FS)
__device__ __forceinline__ double coef_q(const PolDev& P, const PolishShared& sh, const FreeSet& F, int row, int q) {
    if (row < 0) return 1.0;
    if (row < P.S) return ((q < FS ? sh.secF[q] : P.sector[F.Fl[q]]) == row) ? 1.0 : 0.0;
    if (row == P.S) return F.sig[q];
    return brow64(P, sh, F, q, row - P.S - 1);          // factor-exposure row k = row - S - 1
}

// sum over the free set of coef(row, q) * Y[q][col]: one warp, lanes over q, combined in a
// fixed order (every lane returns the sum)
__device__ __forceinline__ double erow_dot(const PolDev& P, const PolishShared& sh, const FreeSet& F, int nF, int row,
                                           int col, int lane) {
    double acc = 0.0;
    for (int q = lane; q < nF; q += 32) acc += coef_q(P, sh, F, row, q) * F.Y[(size_t)q * YS + col];
    return warp_sum(acc);
}

__device__ __forceinline__ float brow32(const PolDev& P, const PolishShared& sh, const FreeSet& F, int q, int k) {
    return q < FS ? sh.Bc[q][k] : P.B32[(size_t)F.Fl[q] * P.K + k];
}
__device__ __forceinline__ double brow64(const PolDev& P, const PolishShared& sh, const FreeSet& F, int q, int k) {
    return q < FS ? sh.Bd[q][k] : P.B64[(size_t)F.Fl[q] * P.K + k];
}

// FP64 products with the free rows of B, spread over the whole block (the FP64 pipe
// runs a warp instruction at the same cost however few of its lanes are active, so the
// work goes to full warps): fin(q, sum_k B_F[q][k] x[k]) for each free row q, eight lanes per
// row, and fin(k, sum_q y(q) B_F[q][k]) for each factor k, four lanes per factor. The partial
// sums are combined in a fixed order. Block-collective (no barrier inside).
template <class Fin>
__device__ __forceinline__ void rows_dot64(const PolDev& P, const PolishShared& sh, const FreeSet& F, int nF,
                                           const double* x, Fin&& fin) {
    const int tid = threadIdx.x, g = tid >> 3, sub = tid & 7, K = P.K;
    for (int q0 = 0; q0 < nF; q0 += PB / 8) {
        const int q = q0 + g;
        double acc = 0.0;
        if (q < nF)
            for (int k = sub; k < K; k += 8) acc += brow64(P, sh, F, q, k) * x[k];
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (sub == 0 && q < nF) fin(q, acc);
    }
}

static_assert(PB / 4 >= KMAX, "four lanes per factor");
template <class Yf, class Fin>
__device__ __forceinline__ void cols_dot64(const PolDev& P, const PolishShared& sh, const FreeSet& F, int nF,
                                           Yf&& y, Fin&& fin) {
    const int tid = threadIdx.x, k = tid >> 2, sub = tid & 3, K = P.K;
    double acc = 0.0;
    if (k < K)
        for (int q = sub; q < nF; q += 4) acc += y(q) * brow64(P, sh, F, q, k);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (sub == 0 && k < K) fin(k, acc);
}

// FP32 Woodbury solve of Sigma_FF x = r for the columns c0..c1 of Y (in: D^{-1} r;
// out: x). Block-collective.
__device__ __noinline__ void woodbury32(const PolDev& P, PolishShared& sh, const FreeSet& F, int nF, int c0, int c1) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, nc = c1 - c0;
    for (int e2 = tid; e2 < K * nc; e2 += PB) {
        const int k = e2 / nc, c = c0 + e2 % nc;
        float acc = 0.f;
        for (int q = 0; q < nF; ++q) acc = fmaf(brow32(P, sh, F, q, k), float(F.Y[(size_t)q * YS + c]), acc);
        sh.T[k][c - c0] = acc;
    }
    __syncthreads();
    // L L' t = T column by column, one warp per column, rows lane and lane + 32 in registers
    for (int c = warp; c < nc; c += PB / 32) {
        float v0 = lane < K ? sh.T[lane][c] : 0.f, v1 = lane + 32 < K ? sh.T[lane + 32][c] : 0.f;
        for (int r = 0; r < K; ++r) {
            const float x = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) * sh.Ldinv[r];
            if (lane > r) v0 = fmaf(-sh.C[lane][r], x, v0);
            if (lane + 32 > r && lane + 32 < K) v1 = fmaf(-sh.C[lane + 32][r], x, v1);
            if (lane == (r & 31)) { if (r < 32) v0 = x; else v1 = x; }
        }
        for (int r = K - 1; r >= 0; --r) {
            const float x = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) * sh.Ldinv[r];
            if (lane < r) v0 = fmaf(-sh.C[r][lane], x, v0);
            if (lane + 32 < r) v1 = fmaf(-sh.C[r][lane + 32], x, v1);
            if (lane == (r & 31)) { if (r < 32) v0 = x; else v1 = x; }
        }
        if (lane < K) sh.T[lane][c] = v0;
        if (lane + 32 < K) sh.T[lane + 32][c] = v1;
    }
    __syncthreads();
    for (int e2 = tid; e2 < nF * nc; e2 += PB) {
        const int q = e2 / nc, c = c0 + e2 % nc;
        float acc = 0.f;
        for (int k = 0; k < K; ++k) acc = fmaf(brow32(P, sh, F, q, k), sh.T[k][c - c0], acc);
        F.Y[(size_t)q * YS + c] -= double(acc) * F.dinv[q];
    }
    __syncthreads();
}

// FP32 solve of Sigma_FF x = r for the columns c0..c1 of Y (in: D^{-1} r; out: x) with the
// Cholesky factor of Sigma_FF itself (|F| <= K, free set in shared memory): one warp per
// column, rows lane and lane + 32 in registers. Block-collective.
__device__ __noinline__ void direct32(PolishShared& sh, const FreeSet& F, int nF, int c0, int c1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = c0 + warp; c < c1; c += PB / 32) {
        float v0 = lane < nF ? float(F.Y[(size_t)lane * YS + c] / F.dinv[lane]) : 0.f;
        float v1 = lane + 32 < nF ? float(F.Y[(size_t)(lane + 32) * YS + c] / F.dinv[lane + 32]) : 0.f;
        for (int r = 0; r < nF; ++r) {
            const float x = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) * sh.Ldinv[r];
            if (lane > r && lane < nF) v0 = fmaf(-sh.C[lane][r], x, v0);
            if (lane + 32 > r && lane + 32 < nF) v1 = fmaf(-sh.C[lane + 32][r], x, v1);
            if (lane == (r & 31)) { if (r < 32) v0 = x; else v1 = x; }
        }
        for (int r = nF - 1; r >= 0; --r) {
            const float x = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) * sh.Ldinv[r];
            if (lane < r) v0 = fmaf(-sh.C[r][lane], x, v0);
            if (lane + 32 < r) v1 = fmaf(-sh.C[r][lane + 32], x, v1);
            if (lane == (r & 31)) { if (r < 32) v0 = x; else v1 = x; }
        }
        if (lane < nF) F.Y[(size_t)lane * YS + c] = v0;
        if (lane + 32 < nF) F.Y[(size_t)(lane + 32) * YS + c] = v1;
    }
    __syncthreads();
}

__device__ __forceinline__ void solve32(const PolDev& P, PolishShared& sh, const FreeSet& F, int nF, int c0,
                                        int c1, bool direct) {
    if (direct) direct32(sh, F, nF, c0, c1);
    else woodbury32(P, sh, F, nF, c0, c1);
}

// (b3) of a polish round: the FP32 matrix to factor (Sigma_FF = B_F F B_F' + D_F when
// ``direct``, else the Woodbury capacitance C = F^{-1} + B_F' D_F^{-1} B_F) and its Cholesky
// factor in sh.C (lower triangle, diagonal included) with the reciprocal diagonal in sh.Ldinv.
// Returns false when a pivot is not positive. Block-collective.
__device__ __noinline__ bool factor32(const PolDev& P, PolishShared& sh, const FreeSet& F, int nF, bool direct) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, nS = direct ? nF : K;
    if (direct) {
        for (int e2 = tid; e2 < nS * nS; e2 += PB) {
            const int r = e2 / nS, c = e2 % nS;
            if (c > r) continue;
            float acc = (r == c) ? float(P.d64[F.Fl[r]]) : 0.f;
            for (int k = 0; k < K; ++k) acc = fmaf(sh.Bc[r][k] * sh.f32s[k], sh.Bc[c][k], acc);
            sh.C[r][c] = acc;
        }
    } else {
        for (int e2 = tid; e2 < K * K; e2 += PB) {
            const int r = e2 / K, c = e2 % K;
            if (c > r) continue;
            float acc = (r == c) ? 1.f / sh.f32s[r] : 0.f;
            const int q1 = min(nF, FS);
            for (int q = 0; q < q1; ++q) acc = fmaf(sh.Bc[q][r] * sh.dinvf_s[q], sh.Bc[q][c], acc);
            for (int q = q1; q < nF; ++q)
                acc = fmaf(brow32(P, sh, F, q, r) * float(F.dinv[q]), brow32(P, sh, F, q, c), acc);
            sh.C[r][c] = acc;
        }
    }
    __syncthreads();
    // Cholesky in the L D L' form (column c of the trailing update reads only column c),
    // then L = L D^{1/2}
    bool chol_ok = true;
    for (int c = 0; c < nS; ++c) {
        const float piv = sh.C[c][c];
        if (!(piv > 0.f)) { chol_ok = false; break; }          // every thread reads the same pivot
        const float ip = 1.f / piv;
        for (int r = c + 1 + warp; r < nS; r += PB / 32) {
            const float lr = sh.C[r][c] * ip;
            for (int q = c + 1 + lane; q <= r; q += 32) sh.C[r][q] = fmaf(-lr, sh.C[q][c], sh.C[r][q]);
        }
        __syncthreads();
    }
    if (chol_ok) {
        for (int c = tid; c < nS; c += PB) sh.Ldinv[c] = sqrtf(sh.C[c][c]);
        __syncthreads();
        for (int e2 = tid; e2 < nS * nS; e2 += PB) {
            const int r = e2 / nS, c = e2 % nS;
            if (c < r) sh.C[r][c] /= sh.Ldinv[c];
        }
        __syncthreads();
        for (int c = tid; c < nS; c += PB) { sh.C[c][c] = sh.Ldinv[c]; sh.Ldinv[c] = 1.f / sh.Ldinv[c]; }
    }
    return chol_ok;
}

// A-posteriori bound on ||w - w*||_inf for the polished point w of one account.
// The risk term makes the objective strongly convex with modulus m = lambda_min(2 Sigma)
// >= 2 min_i d_i. Let r be the vector of per-entry stationarity residuals (the distances
// that r_stat takes the maximum of) and L the Lagrangian with the returned multipliers.
// Multipliers of the wrong sign are replaced by 0 for the argument, which moves every
// residual by at most their size (|lambda_s| on the entries of sector s, |theta| on all).
// With the signs right, L <= F on the feasible set, L is m-strongly convex and r is in
// its subdifferential at w, and F(w) >= F(w*) + m/2 ||w - w*||^2; together
//   m ||w - w*||^2 <= ||r||_2 ||w - w*|| + C,
//   C = sum_s |lambda_s| |slack_s| + |theta| |tau - ||w - w0||_1| + |nu| |1'w - 1|,
// so ||w - w*||_2 <= (||r||_2 + sqrt(||r||_2^2 + 4 m C)) / (2 m). This holds for a point
// that meets the constraints; the primal residuals reported beside it say by how much
// the returned point misses them (to FP64 rounding for a certified account).
__device__ __noinline__ double err_bound(const PolDev& P, const PolishShared& sh, double r2, double sw, double tu,
                                         double tau, double nu, double theta) {
    const double m = 2.0 * P.dmin;
    if (!(m > 0.0)) return INFINITY;
    double wrong = 0.0, C = fabs(nu) * fabs(sw - 1.0);
    for (int s = 0; s < P.S; ++s) {
        // lambda_s >= 0 prices the upper edge and lambda_s <= 0 the lower one; a multiplier
        // on an infinite edge has no such reading and counts as of the wrong sign
        // Either reading gives a valid bound, so each multiplier takes the one that adds less
        // (a tiny multiplier of a band held at its other edge is cheaper set to zero).
        const double ls = sh.lam_s[s], ssum = sh.secsum[s];
        const double edge = ls > 0.0 ? sh.bhi_s[s] : sh.blo_s[s];
        if (ls == 0.0) continue;
        const double as_comp = isfinite(edge) ? fabs(ls) * fabs(edge - ssum) : INFINITY;
        if (sqrt(as_comp / m) <= sqrt(double(P.N)) * fabs(ls) / m) C += as_comp;
        else wrong += fabs(ls);
    }
    for (int k = 0; k < P.K && P.flo; ++k) {
        // factor rows, read like the bands (kappa_k >= 0 prices the upper bound)
        const double kk = sh.kap_s[k], hk = sh.t64[k];
        if (kk == 0.0) continue;
        const double edge = kk > 0.0 ? sh.fhi_s[k] : sh.flo_s[k];
        // (a multiplier on an infinite bound has no such reading: C, and the bound, become +inf)
        C += isfinite(edge) ? fabs(kk) * fabs(edge - hk) : INFINITY;
    }
    if (theta != 0.0) {
        const double as_comp = (isfinite(tau) && theta > 0.0) ? theta * fabs(tau - tu) : INFINITY;
        if (sqrt(as_comp / m) <= sqrt(double(P.N)) * fabs(theta) / m) C += as_comp;
        else wrong += fabs(theta);
    }
    const double re = r2 + sqrt(double(P.N)) * wrong;
    return (re + sqrt(re * re + 4.0 * m * C)) / (2.0 * m);
}

// The factor-exposure rows' checks of one account (thread 0), like the bands': a row outside the
// working set joins it when violated; a working row leaves it when its multiplier has the wrong
// sign, or, found dependent on the free set, when it holds strictly inside its bounds.
__device__ __noinline__ void factor_row_checks(const PolDev& P, PolishShared& sh, int a, int m, double tol_p,
                                               double tol_d, double& r_exp, double& r_comp, int& bviol, int& dep_in,
                                               int& dep_out) {
    const int K = P.K, S = P.S;
    auto row_dependent = [&](int row) {
        for (int r = 1; r < m; ++r)
            if (sh.rows[r] == row) return sh.used[r] == 0;
        return false;
    };
    for (int k = 0; k < K; ++k) {
        const double hk = sh.t64[k], hi = sh.fhi_s[k], lo = sh.flo_s[k];
        r_exp = fmax(r_exp, fmax(lo - hk, hk - hi));
        const int wf = sh.wf_s[k];
        const double kk = sh.kap_s[k];
        const bool off = wf != 0 && fabs(hk - (wf > 0 ? hi : lo)) > tol_p;
        auto set_wf = [&](int v) { sh.wf_s[k] = v; P.wfac[a * K + k] = v; };
        if (off && row_dependent(S + 1 + k)) {
            ++bviol;
            if (wf > 0 ? hk < hi : hk > lo) { set_wf(0); ++dep_in; }
            else ++dep_out;
        } else if (wf == 0) {
            if (hk > hi + tol_p) { ++bviol; set_wf(1); }
            else if (hk < lo - tol_p) { ++bviol; set_wf(-1); }
        } else {
            if (off) ++bviol;
            if (wf > 0) {
                r_comp = fmax(r_comp, fabs(kk) * fabs(hi - hk));
                if (kk < -tol_d) { ++bviol; r_comp = fmax(r_comp, -kk); set_wf(0); }
            } else {
                r_comp = fmax(r_comp, fabs(kk) * fabs(hk - lo));
                if (kk > tol_d) { ++bviol; r_comp = fmax(r_comp, kk); set_wf(0); }
            }
        }
    }
}

__global__ void __launch_bounds__(PB, 2) k_polish(PolDev P, int rounds) {   // two blocks per SM
    const int a = blockIdx.x;
    if ((P.skip && P.skip[a]) || P.done[a] || (P.sel && P.sel[a] != P.gen)) return;
    extern __shared__ unsigned char smem_raw[];
    PolishShared& sh = *reinterpret_cast<PolishShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, S = P.S, N = P.N;
    const size_t base = (size_t)a * P.Npad;
    int* Flg = P.Flist + (size_t)a * P.FMAX;
    int* NZl = P.NZlist + (size_t)a * P.FMAX;
    double* W = P.W + base;
    const double tol_d = P.tol_dual, tol_p = P.tol_primal;
    for (int s2 = tid; s2 < S; s2 += PB) {
        sh.blo_s[s2] = P.band_lo[a * S + s2];
        sh.bhi_s[s2] = P.band_hi[a * S + s2];
        sh.wb_s[s2] = P.wband[a * S + s2];
    }
    for (int k = tid; k < K; k += PB) {
        sh.wf_s[k] = P.wfac ? P.wfac[a * K + k] : 0;
        sh.flo_s[k] = P.flo ? P.flo[a * K + k] : -INFINITY;
        sh.fhi_s[k] = P.fhi ? P.fhi[a * K + k] : INFINITY;
    }
    __syncthreads();
    for (int round = 0; round < rounds; ++round) {
        // ---- (a) ordered compaction in coalesced warp tiles; W of the fixed entries
        const int Lw = cdiv(cdiv(N, PB / 32), 32) * 32;
        const int w0r = min(N, warp * Lw), w1r = min(N, w0r + Lw);
        int nf = 0, nn = 0;
        double sa = 0.0, ca = 0.0, ta = 0.0, oa = 0.0;
        WarpQueue wq;
        wq.p = sh.qp[warp];
        wq.g = sh.qg[warp];
        auto fixed_or_free = [&](int p, float) {
            const int code = P.st[base + p];
            Pieces pc;
            entry_pieces(P, base + p, pc);
            if (code >= ST_FREE) {
                ++nf;
                ca -= seg_sign(pc, code - ST_FREE) * pc.w0;
            } else {
                // a fixed entry: its weight, and its parts of the budget, turnover and
                // objective sums of the checks (a fixed weight keeps its value all round)
                const double wv = pc.bp[code];
                W[p] = wv;
                sa += wv;
                const double tv = fabs(wv - pc.w0);
                ca += tv;
                ta += tv;
                oa += P.d64[p] * wv * wv - P.mu64[p] * wv + phi_value(pc, wv);
                nn += (wv != 0.0);
            }
        };
        for (int p0 = w0r; p0 < w1r; p0 += 32 * AU) {
            int code[AU], pwv[AU];
            float w0v[AU], lov[AU];
#pragma unroll
            for (int u = 0; u < AU; ++u) {              // all loads of the batch first
                const int p = p0 + 32 * u + lane;
                const size_t e = base + (p < w1r ? p : 0);
                code[u] = P.st[e];
                w0v[u] = P.w0f[e];
                lov[u] = P.lof[e];
                pwv[u] = P.pw_idx ? P.pw_idx[e] : -1;
            }
#pragma unroll
            for (int u = 0; u < AU; ++u) {
                const int p = p0 + 32 * u + lane;
                const bool zero_fixed = code[u] == 0 && w0v[u] == 0.f && lov[u] == 0.f && pwv[u] < 0;
                if (p < w1r && zero_fixed) W[p] = 0.0;
                wq.push(p < w1r && !zero_fixed, p, 0.f, lane);
                wq.drain(false, lane, fixed_or_free);     // keeps at most 31 queued before a push
            }
        }
        wq.drain(true, lane, fixed_or_free);
        nf = warp_sum(nf);
        nn = warp_sum(nn);
        sa = warp_sum(sa);
        ca = warp_sum(ca);
        ta = warp_sum(ta);
        oa = warp_sum(oa);
        if (lane == 0) {
            sh.cntF[warp] = nf; sh.cntN[warp] = nn;
            sh.sumA[warp] = sa; sh.capA[warp] = ca; sh.turnA[warp] = ta; sh.objA[warp] = oa;
        }
        __syncthreads();
        if (tid == 0) {
            int of = 0, on = 0;
            double ss = 0.0, cc = 0.0, tt = 0.0, oo = 0.0;
            for (int t = 0; t < PB / 32; ++t) {
                const int f = sh.cntF[t], n = sh.cntN[t];
                sh.cntF[t] = of; sh.cntN[t] = on;
                of += f; on += n;
                ss += sh.sumA[t]; cc += sh.capA[t]; tt += sh.turnA[t]; oo += sh.objA[t];
            }
            sh.nF = of; sh.nNZ = on;
            sh.sumA[0] = ss; sh.capA[0] = cc; sh.turnA[0] = tt; sh.objA[0] = oo;
            int r = 0;
            sh.rows[r++] = -1;
            for (int q = 0; q < S; ++q)
                if (sh.wb_s[q] != 0) { if (r < PMAXROWS) sh.rows[r] = q; ++r; }
            if (P.wcap[a]) { if (r < PMAXROWS) sh.rows[r] = S; ++r; }
            for (int k = 0; k < K; ++k)
                if (sh.wf_s[k] != 0) { if (r < PMAXROWS) sh.rows[r] = S + 1 + k; ++r; }
            sh.nrows = r;
            sh.fail = (of > P.FMAX || on > P.FMAX || of == 0 || r > MAXWROWS);
        }
        __syncthreads();
        if (sh.fail) {
            if (tid == 0) P.done[a] = 2;
            return;
        }
        {
            int of = sh.cntF[warp], on = sh.cntN[warp];
            const unsigned lt = (1u << lane) - 1u;
            for (int p0 = w0r; p0 < w1r; p0 += 32 * AU) {
                int code[AU];
                double wv[AU];
#pragma unroll
                for (int u = 0; u < AU; ++u) {
                    const int p = p0 + 32 * u + lane, pp = p < w1r ? p : 0;
                    code[u] = P.st[base + pp];
                    wv[u] = W[pp];
                }
#pragma unroll
                for (int u = 0; u < AU; ++u) {
                    const int p = p0 + 32 * u + lane;
                    const int isF = p < w1r && code[u] >= ST_FREE;
                    const int isNZ = p < w1r && !isF && wv[u] != 0.0;
                    const unsigned bF = __ballot_sync(0xffffffffu, isF), bN = __ballot_sync(0xffffffffu, isNZ);
                    if (isF) Flg[of + __popc(bF & lt)] = p;
                    if (isNZ) NZl[on + __popc(bN & lt)] = p;
                    of += __popc(bF);
                    on += __popc(bN);
                }
            }
        }
        __syncthreads();
        const int nF = sh.nF, nNZ = sh.nNZ, m = sh.nrows;
        const double sumA = sh.sumA[0], capA = sh.capA[0], turnA = sh.turnA[0], objA = sh.objA[0];
        // ---- (b1) h_A = B' w_A (FP64) over the nonzero fixed entries
        {
            const int k = tid >> 2, sub = tid & 3;
            double acc = 0.0;
            if (k < K)
                for (int q = sub; q < nNZ; q += 4) {
                    const int p = NZl[q];
                    acc += W[p] * P.B64[(size_t)p * K + k];
                }
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            if (sub == 0 && k < K) {
                sh.hA[k] = acc;
                sh.fhA[k] = P.f64[k] * acc;
            }
        }
        // per sector, the sum of the fixed weights (one warp per sector); the sectors of the
        // free entries whose data live in shared memory
        for (int s2 = warp; s2 < S; s2 += PB / 32) {
            double acc = 0.0;
            for (int q = lane; q < nNZ; q += 32) {
                const int p = NZl[q];
                if (P.sector[p] == s2) acc += W[p];
            }
            acc = warp_sum(acc);
            if (lane == 0) sh.fixS[s2] = acc;
        }
        for (int q = tid; q < min(nF, FS); q += PB) sh.secF[q] = P.sector[Flg[q]];
        __syncthreads();
        // ---- (b2) the free set: shared memory when small; rows of B in FP32 and FP64
        FreeSet F;
        F.in_smem = nF <= FS;
        if (F.in_smem) {
            F.Fl = sh.Fl_s; F.Y = &sh.Ys[0][0]; F.dinv = sh.dinv_s; F.sig = sh.sig_s;
            for (int q = tid; q < nF; q += PB) sh.Fl_s[q] = Flg[q];
        } else {
            F.Fl = Flg;
            F.Y = P.Y + (size_t)a * P.FMAX * YS;
            F.dinv = P.Fdinv + (size_t)a * P.FMAX;
            F.sig = P.Fsig + (size_t)a * P.FMAX;
        }
        for (int k = tid; k < K; k += PB) sh.f32s[k] = float(P.f64[k]);
        for (int e2 = tid; e2 < min(nF, FS) * K; e2 += PB) {
            const int q = e2 / K, k = e2 % K;
            const double b = P.B64[(size_t)Flg[q] * K + k];
            sh.Bd[q][k] = b;
            sh.Bc[q][k] = P.B32[(size_t)Flg[q] * K + k];
        }
        __syncthreads();
        // g0 (FP64), 1/d, cap signs
        rows_dot64(P, sh, F, nF, sh.fhA, [&](int q, double bf) {
            const int p = F.Fl[q];
            const size_t e = base + p;
            Pieces pc;
            entry_pieces(P, e, pc);
            const int seg = P.st[e] - ST_FREE;
            double* Yq = F.Y + (size_t)q * YS;
            Yq[0] = P.mu64[p] - pc.sl[seg] - 2.0 * bf;
            Yq[COL_W] = 0.0;
            F.dinv[q] = 1.0 / P.d64[p];
            if (q < FS) sh.dinvf_s[q] = float(F.dinv[q]);
            F.sig[q] = seg_sign(pc, seg);
        });
        __syncthreads();
        // ---- (b3) the FP32 matrix to factor: Sigma_FF = B_F F B_F' + D_F itself when the free
        // set is no larger than K (it then lives in shared memory), else the Woodbury
        // capacitance C = F^{-1} + B_F' D_F^{-1} B_F; then its Cholesky factor
        const bool direct = nF <= K && nF <= FS;
        const bool chol_ok = factor32(P, sh, F, nF, direct);
        __syncthreads();
        if (!chol_ok) {
            if (tid == 0) P.done[a] = 2;
            return;
        }
        // ---- (b4) Y_E = Sigma_FF^{-1} E_F' (FP32, stored in Y columns 1..m)
        for (int e2 = tid; e2 < nF * m; e2 += PB) {
            const int q = e2 / m, r = e2 % m;
            F.Y[(size_t)q * YS + 1 + r] = coef_q(P, sh, F, sh.rows[r], q) * F.dinv[q];
        }
        __syncthreads();
        solve32(P, sh, F, nF, 1, 1 + m, direct);
        // Schur matrix S = 1/2 E Y_E, and row edges e = edge - fixed part
        for (int e2 = warp; e2 < m * m; e2 += PB / 32) {
            const int r = e2 / m, c = e2 % m;
            const double acc = erow_dot(P, sh, F, nF, sh.rows[r], 1 + c, lane);
            if (lane == 0) sh.Sf[r][c] = 0.5 * acc;
        }
        for (int r = tid; r < m; r += PB) {
            const int row = sh.rows[r];
            double e_r;
            if (row < 0) {
                e_r = 1.0 - sumA;
            } else if (row < S) {
                const double edge = (sh.wb_s[row] > 0) ? sh.bhi_s[row] : sh.blo_s[row];
                e_r = edge - sh.fixS[row];
            } else if (row == S) {
                e_r = P.tau[a] - capA;
            } else {
                const int k = row - S - 1;
                e_r = ((sh.wf_s[k] > 0) ? sh.fhi_s[k] : sh.flo_s[k]) - sh.hA[k];
            }
            sh.erhs[r] = e_r;
            sh.lam[r] = 0.0;
        }
        __syncthreads();
        // pivoted symmetric elimination of S (budget row first); vanishing pivots mark
        // rows that depend on the free set: their multipliers stay 0
        if (tid == 0) {
            double scale = 0.0;
            for (int r = 0; r < m; ++r) { sh.used[r] = 0; scale = fmax(scale, fabs(sh.Sf[r][r])); }
            int nc = 0;
            for (int k = 0; k < m; ++k) {
                int p = -1;
                if (k == 0) p = 0;
                else {
                    double best = 0.0;
                    for (int j = 0; j < m; ++j)
                        if (!sh.used[j] && fabs(sh.Sf[j][j]) > best) { best = fabs(sh.Sf[j][j]); p = j; }
                }
                if (p < 0 || !(fabs(sh.Sf[p][p]) > 1e-9 * scale)) break;
                sh.used[p] = 1;
                sh.order[nc++] = p;
                for (int j = 0; j < m; ++j) {
                    if (sh.used[j]) continue;
                    const double f = sh.Sf[j][p] / sh.Sf[p][p];
                    // only columns not yet pivoted: pivoted ones of row j hold its multipliers
                    for (int q = 0; q < m; ++q) if (!sh.used[q]) sh.Sf[j][q] -= f * sh.Sf[p][q];
                    sh.Sf[j][p] = f;                       // multiplier of row j against pivot p
                }
            }
            sh.nc = nc;
            sh.fail = (nc == 0);
        }
        __syncthreads();
        if (sh.fail) {
            if (tid == 0) P.done[a] = 2;
            return;
        }
        const int ndep = m - sh.nc;
        // ---- (b5) iterative refinement: FP64 residuals, FP32 corrections
        for (int it = 0; it < IR_STEPS; ++it) {
            // t = B_F' w_F (FP64)
            cols_dot64(P, sh, F, nF, [&](int q) { return F.Y[(size_t)q * YS + COL_W]; },
                       [&](int k, double acc) { sh.t64[k] = P.f64[k] * acc; });
            __syncthreads();
            // r1 = g0 - 2 Sigma_FF w - E' lam ; stored scaled by D^{-1} in COL_R
            double rmax = 0.0;
            rows_dot64(P, sh, F, nF, sh.t64, [&](int q, double bt) {
                const int p = F.Fl[q];
                double* Yq = F.Y + (size_t)q * YS;
                double r1 = Yq[0] - 2.0 * (bt + P.d64[p] * Yq[COL_W]);
                for (int r = 0; r < m; ++r) r1 -= coef_q(P, sh, F, sh.rows[r], q) * sh.lam[r];
                rmax = fmax(rmax, fabs(r1));
                Yq[COL_R] = r1 * F.dinv[q];
            });
            // r2 = e - E w
            for (int r = warp; r < m; r += PB / 32) {
                const double acc = erow_dot(P, sh, F, nF, sh.rows[r], COL_W, lane);
                if (lane == 0) sh.rr2[r] = sh.erhs[r] - acc;
            }
            rmax = warp_max(rmax);
            if (lane == 0) sh.red[warp][0] = rmax;
            __syncthreads();
            // converged: every warp's residual maximum and every row residual within its limit,
            // tested lane-wise in each warp (the same answer in every warp; a NaN never passes)
            bool conv = lane >= PB / 32 || sh.red[lane][0] <= 1e-15;
            for (int r = lane; r < m; r += 32) conv = conv && fabs(sh.rr2[r]) <= 1e-16;
            conv = __all_sync(0xffffffffu, conv);
            if (it > 0 && conv) break;
            // Yr = Sigma_FF^{-1} r1 (FP32)
            solve32(P, sh, F, nF, COL_R, COL_R + 1, direct);
            // dlam = S^{-1} (1/2 E Yr - r2) with the eliminated S
            for (int r = warp; r < m; r += PB / 32) {
                const double acc = erow_dot(P, sh, F, nF, sh.rows[r], COL_R, lane);
                if (lane == 0) sh.dlam[r] = 0.5 * acc - sh.rr2[r];
            }
            __syncthreads();
            if (tid == 0) {
                // forward: apply the recorded eliminations in pivot order
                for (int k = 0; k < sh.nc; ++k) {
                    const int p = sh.order[k];
                    for (int j = 0; j < m; ++j) {
                        bool later = !sh.used[j];
                        for (int kk = k + 1; kk < sh.nc; ++kk) if (sh.order[kk] == j) later = true;
                        if (later && j != p) sh.dlam[j] -= sh.Sf[j][p] * sh.dlam[p];
                    }
                }
                double x[PMAXROWS];
                for (int r = 0; r < m; ++r) x[r] = 0.0;
                for (int k = sh.nc - 1; k >= 0; --k) {
                    const int p = sh.order[k];
                    double v = sh.dlam[p];
                    for (int kk = k + 1; kk < sh.nc; ++kk) { const int q = sh.order[kk]; v -= sh.Sf[p][q] * x[q]; }
                    x[p] = v / sh.Sf[p][p];
                }
                for (int r = 0; r < m; ++r) { sh.dlam[r] = x[r]; sh.lam[r] += x[r]; }
            }
            __syncthreads();
            // dw = 1/2 (Yr - Y_E dlam)
            for (int q = tid; q < nF; q += PB) {
                double* Yq = F.Y + (size_t)q * YS;
                double acc = Yq[COL_R];
                for (int r = 0; r < m; ++r) acc -= Yq[1 + r] * sh.dlam[r];
                Yq[COL_W] += 0.5 * acc;
            }
            __syncthreads();
        }
        // ---- (b6) the solved point: W_F, h = h_A + B_F' w_F, multipliers
        for (int q = tid; q < nF; q += PB) W[F.Fl[q]] = F.Y[(size_t)q * YS + COL_W];
        cols_dot64(P, sh, F, nF, [&](int q) { return F.Y[(size_t)q * YS + COL_W]; }, [&](int k, double bw) {
            const double acc = sh.hA[k] + bw;
            const double fhk = P.f64[k] * acc;
            sh.t64[k] = acc;
            sh.fh[k] = fhk;
            sh.fh32[k] = float(fhk);
        });
        for (int k = K + tid; k < KMAX; k += PB) sh.fh32[k] = 0.f;
        for (int s2 = tid; s2 < S; s2 += PB) sh.lam_s[s2] = 0.0;
        for (int k = tid; k < K; k += PB) sh.kap_s[k] = 0.0;
        __syncthreads();
        double theta = 0.0;
        for (int r = 1; r < m; ++r) if (sh.rows[r] == S) theta = sh.lam[r];
        if (tid == 0) {
            for (int r = 1; r < m; ++r) if (sh.rows[r] < S) sh.lam_s[sh.rows[r]] = sh.lam[r];
            // a factor row's multiplier kappa_k adds kappa_k B_ik to entry i's gradient: the
            // gradient's product B (F h) becomes B (F h + kappa / 2)
            for (int r = 1; r < m; ++r)
                if (sh.rows[r] > S) {
                    const int k = sh.rows[r] - S - 1;
                    sh.kap_s[k] = sh.lam[r];
                    sh.fh[k] += 0.5 * sh.lam[r];
                    sh.fh32[k] = float(sh.fh[k]);
                }
        }
        __syncthreads();
        if (warp == 1) {
            // once per block: lanes over the factors, combined in a fixed order (the quadratic
            // term h'F h from h itself, without the factor rows' multipliers)
            double fm = 0.0, qd = 0.0;
            for (int k = lane; k < K; k += 32) {
                fm = fmax(fm, fabs(sh.fh[k]));
                qd += sh.t64[k] * P.f64[k] * sh.t64[k];
            }
            fm = warp_max(fm);
            qd = warp_sum(qd);
            if (lane == 0) { sh.fhmax_s = fm; sh.quad_s = qd; }
        }
        __syncthreads();
        const double nu = sh.lam[0];
        const double fhmax = sh.fhmax_s, quad = sh.quad_s;
        // ---- (c) checks of every entry (Sec. 4.4): FP32 gradient as a filter, FP64 where it
        // cannot decide; violators switch state for the next round
        const float nu_f = float(nu), theta_f = float(theta), fhmax_f = float(fhmax);
        double r_stat = 0.0, r_box = 0.0, obj_lin = 0.0, sum_w = 0.0, turn = 0.0;
        double r_sq = 0.0;                 // squared 2-norm of the stationarity residuals
        int nviol = 0;
        double my_margin = INFINITY;
        int my_who = 0;
        // FP64 checks of one entry (run 32 entries at a time from the warp's queue); gx, when
        // given, is the entry's exact product B_p . fh computed beforehand
        auto check_entry3 = [&](int p, float g32, const double* gx) {
            const size_t e = base + p;
            const int code = P.st[e];
            const int sec = P.sector[p];
            EntryRaw rw;
            load_raw(P, base, p, rw);
            Pieces pc;
            pieces_from(P, rw, pc);
            const double wv = rw.W;
            const double dd = rw.d, mu = rw.mu;
            const double lam_s = sh.lam_s[sec];
            if (code >= ST_FREE) {
                // the fixed entries' parts of these sums come from the compaction; a fixed
                // weight sits on a breakpoint inside its box
                sum_w += wv;
                turn += fabs(wv - pc.w0);
                obj_lin += dd * wv * wv - mu * wv + phi_value(pc, wv);
                r_box = fmax(r_box, fmax(rw.lo - wv, wv - rw.up));
            }
            const double g_a = 2.0 * (double(g32) + dd * wv) - mu;
            const double delta = 1e-5 * (2.0 * rw.bn1 * fhmax + 2.0 * fabs(dd * wv) + fabs(mu) + fabs(nu) + fabs(lam_s));
            auto exact_rr = [&]() {
                const double* Bp = P.B64 + (size_t)p * K;
                double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
                int k = 0;
                for (; k + 4 <= K; k += 4) {
                    b0 += Bp[k] * sh.fh[k]; b1 += Bp[k + 1] * sh.fh[k + 1];
                    b2 += Bp[k + 2] * sh.fh[k + 2]; b3 += Bp[k + 3] * sh.fh[k + 3];
                }
                for (; k < K; ++k) b0 += Bp[k] * sh.fh[k];
                return 2.0 * (((b0 + b1) + (b2 + b3)) + dd * wv) - mu + nu + lam_s;
            };
            if (code >= ST_FREE) {
                const int seg = code - ST_FREE;
                const double rr = gx ? 2.0 * (*gx + dd * wv) - mu + nu + lam_s : exact_rr();
                const double res = fabs(rr + pc.sl[seg] + theta * seg_sign(pc, seg));
                r_stat = fmax(r_stat, res);
                r_sq += res * res;
                if (wv > pc.bp[seg + 1] + tol_p) { ++nviol; P.st[e] = (int8_t)(seg + 1); }
                else if (wv < pc.bp[seg] - tol_p) { ++nviol; P.st[e] = (int8_t)seg; }
            } else {
                const int j = code;
                const double left = (j > 0) ? pc.sl[j - 1] + theta * seg_sign(pc, j - 1) : -INFINITY;
                const double right = (j + 1 < pc.nb) ? pc.sl[j] + theta * seg_sign(pc, j) : INFINITY;
                double rr = g_a + nu + lam_s;
                double up = -rr - right, dn = left + rr;
                if (fmax(up, dn) > -delta) {            // too close to call in FP32
                    rr = exact_rr();
                    up = -rr - right;
                    dn = left + rr;
                }
                const double res = fmax(fmax(up, dn), 0.0);
                r_stat = fmax(r_stat, res);
                r_sq += res * res;
                if (pc.nb > 1) {
                    if (isfinite(right) && -up < my_margin) { my_margin = -up; my_who = p + 1; }
                    if (isfinite(left) && -dn < my_margin) { my_margin = -dn; my_who = -(p + 1); }
                }
                if (up > tol_d) { ++nviol; P.st[e] = (int8_t)(ST_FREE + j); }
                else if (dn > tol_d) { ++nviol; P.st[e] = (int8_t)(ST_FREE + j - 1); }
            }
        };
        auto check_entry = [&](int p, float g32) { check_entry3(p, g32, nullptr); };
        // the free entries of a free set in shared memory are checked in a pass of their own,
        // with their exact products computed here by the whole block
        const bool free_pass = F.in_smem;
        if (free_pass) rows_dot64(P, sh, F, nF, sh.fh, [&](int q, double v) { sh.gF[q] = v; });
        for (int s2 = tid; s2 < S; s2 += PB) sh.lam_s32[s2] = float(sh.lam_s[s2]);
        __syncthreads();
        float fmargin = INFINITY;
        int fwho = 0;
        // lane (4 r + j) holds columns 16 i + 4 j .. + 3 (i < 4) of fh in FP32
        float4 fr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) fr[i] = *reinterpret_cast<const float4*>(&sh.fh32[16 * i + 4 * (lane & 3)]);
        const int ntiles = cdiv(N, 32);
        // the per-entry inputs of a tile; the next tile's are loaded before the current one
        // is processed, so that their latency overlaps its product and checks
        struct TileIn { int code, pw, sec; float w0, lo, up, c, mu, bn1; };
        auto load_tile = [&](int ti, TileIn& t) {
            const int p = ti * 32 + lane;
            const size_t e = base + p;
            t.code = P.st[e];
            t.pw = P.pw_idx ? P.pw_idx[e] : -1;
            t.sec = P.sector[p];
            t.w0 = P.w0f[e]; t.lo = P.lof[e]; t.up = P.upf[e]; t.c = P.cf[e];
            t.mu = P.mu32[p]; t.bn1 = P.Bn1f[p];
        };
        TileIn cur{}, nxt{};
        if (warp < ntiles) load_tile(warp, cur);
        for (int ti = warp; ti < ntiles; ti += PB / 32) {
            if (ti + PB / 32 < ntiles) load_tile(ti + PB / 32, nxt);
            const int p = ti * 32 + lane;                 // entries of padding (p >= N) are skipped below
            const int code = cur.code, pwv = cur.pw, sec = cur.sec;
            const float w0v = cur.w0, lov = cur.lo, upv = cur.up, cv = cur.c;
            const float muf = cur.mu, bn1f = cur.bn1;
            // g32 = B_p . fh for the tile's 32 rows: four rows of 64 floats per group of 8 lanes x 4
            // float4, coalesced over the tile's contiguous 8 KB; lane p ends with its own row
            float g32 = 0.f;
            const float* Bt = P.B32p + (size_t)ti * 32 * KMAX;
#pragma unroll
            for (int grp = 0; grp < 4; ++grp) {
                const float4* Br = reinterpret_cast<const float4*>(Bt + (size_t)(grp * 8 + (lane >> 2)) * KMAX) + (lane & 3);
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 b = __ldg(Br + 4 * i);
                    acc = fmaf(b.x, fr[i].x, acc);
                    acc = fmaf(b.y, fr[i].y, acc);
                    acc = fmaf(b.z, fr[i].z, acc);
                    acc = fmaf(b.w, fr[i].w, acc);
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                const float v = __shfl_sync(0xffffffffu, acc, 4 * (lane & 7));
                if ((lane >> 3) == grp) g32 = v;
            }
            bool need = p < N;
            if (need && pwv < 0 && code == 0 && lov == 0.f && upv > 0.f) {
                // fixed at a lower bound of 0: the one condition is on the right slope of the
                // cost, c + theta when w0 <= 0 and -(c + theta) when w0 > 0 (a name sold out)
                const float lam_f = sh.lam_s32[sec];
                const float rr = 2.f * g32 - muf + nu_f + lam_f;
                const float right = (w0v > 0.f) ? -(cv + theta_f) : cv + theta_f;
                const float up = -rr - right;
                const float delta =
                    1e-5f * (2.f * bn1f * fhmax_f + fabsf(muf) + fabsf(nu_f) + fabsf(lam_f) + cv + theta_f) + 1e-9f;
                if (up < -delta) {
                    if (-up < fmargin) { fmargin = -up; fwho = p + 1; }
                    need = false;
                }
            } else if (need && pwv < 0 && code == 0 && lov == 0.f && upv == 0.f) {
                // an excluded name: its box is the point 0, so it has no stationarity
                // condition (its turnover and cost are summed in the compaction)
                need = false;
            }
            if (free_pass && code >= ST_FREE) need = false;
            wq.push(need, p, g32, lane);
            wq.drain(false, lane, check_entry);
            cur = nxt;
        }
        wq.drain(true, lane, check_entry);
        if (free_pass)
            for (int q = tid; q < nF; q += PB) check_entry3(F.Fl[q], 0.f, &sh.gF[q]);
        if (double(fmargin) < my_margin) { my_margin = double(fmargin); my_who = fwho; }
        r_stat = warp_max(r_stat); r_box = warp_max(r_box); r_sq = warp_sum(r_sq);
        obj_lin = warp_sum(obj_lin); sum_w = warp_sum(sum_w); turn = warp_sum(turn);
        nviol = warp_sum(nviol);
        for (int o = 16; o > 0; o >>= 1) {
            const double om = __shfl_xor_sync(0xffffffffu, my_margin, o);
            const int ow = __shfl_xor_sync(0xffffffffu, my_who, o);
            if (om < my_margin || (om == my_margin && abs(ow) < abs(my_who))) { my_margin = om; my_who = ow; }
        }
        if (lane == 0) {
            sh.red[warp][0] = r_stat; sh.red[warp][1] = r_box; sh.red[warp][2] = obj_lin;
            sh.red[warp][3] = sum_w; sh.red[warp][4] = turn; sh.red[warp][5] = double(nviol);
            sh.red[warp][6] = r_sq;
            sh.mmin[warp] = my_margin; sh.mwho[warp] = my_who;
        }
        // sector sums over the entries of nonzero weight: the nonzero fixed and the free ones
        for (int s2 = warp; s2 < S; s2 += PB / 32) {
            double acc = 0.0;
            for (int q = lane; q < nF; q += 32)
                if ((q < FS ? sh.secF[q] : P.sector[F.Fl[q]]) == s2) acc += F.Y[(size_t)q * YS + COL_W];
            acc = warp_sum(acc);
            if (lane == 0) sh.secsum[s2] = sh.fixS[s2] + acc;
        }
        __syncthreads();
        if (tid == 0) {
            double rs = 0, rb = 0, ol = 0, sw = 0, tu = 0, nv = 0, rq = 0;
            for (int w = 0; w < PB / 32; ++w) {
                rs = fmax(rs, sh.red[w][0]); rb = fmax(rb, sh.red[w][1]); ol += sh.red[w][2];
                sw += sh.red[w][3]; tu += sh.red[w][4]; nv += sh.red[w][5]; rq += sh.red[w][6];
            }
            sw += sumA;
            tu += turnA;
            ol += objA;
            double r_exp = 0.0, r_comp = 0.0;
            int bviol = 0, dep_in = 0, dep_out = 0;
            // a working row is dependent when the pivoted elimination left it unpivoted
            auto set_wb = [&](int s2, int v) { sh.wb_s[s2] = v; P.wband[a * S + s2] = v; };
            auto row_dependent = [&](int row) {
                for (int r = 1; r < m; ++r)
                    if (sh.rows[r] == row) return sh.used[r] == 0;
                return false;
            };
            for (int s2 = 0; s2 < S; ++s2) {
                const double ssum = sh.secsum[s2];
                const double hi = sh.bhi_s[s2], lo = sh.blo_s[s2];
                r_exp = fmax(r_exp, fmax(lo - ssum, ssum - hi));
                const int wb = sh.wb_s[s2];
                const double ls = sh.lam_s[s2];
                const bool off = wb != 0 && fabs(ssum - (wb > 0 ? hi : lo)) > tol_p;
                if (off && row_dependent(s2)) {
                    // dropped from the solve: inside the band it is inactive and leaves the
                    // working set; outside, a fixed entry is released
                    ++bviol;
                    if (wb > 0 ? ssum < hi : ssum > lo) { set_wb(s2, 0); ++dep_in; }
                    else ++dep_out;
                } else if (wb == 0) {
                    if (ssum > hi + tol_p) { ++bviol; set_wb(s2, 1); }
                    else if (ssum < lo - tol_p) { ++bviol; set_wb(s2, -1); }
                } else {
                    // an independent working row is off its bound only when free weights left
                    // their segments (counted in nviol): the next round solves again
                    if (off) ++bviol;
                    if (wb > 0) {
                        r_comp = fmax(r_comp, fabs(ls) * fabs(hi - ssum));
                        if (ls < -tol_d) { ++bviol; r_comp = fmax(r_comp, -ls); set_wb(s2, 0); }
                    } else {
                        r_comp = fmax(r_comp, fabs(ls) * fabs(ssum - lo));
                        if (ls > tol_d) { ++bviol; r_comp = fmax(r_comp, ls); set_wb(s2, 0); }
                    }
                }
            }
            double r_turn = 0.0;
            const double tau = P.tau[a];
            if (isfinite(tau)) {
                r_turn = fmax(tu - tau, 0.0);
                if (!P.wcap[a]) {
                    if (tu > tau + tol_p) { ++bviol; P.wcap[a] = 1; }
                } else {
                    const bool off = fabs(tu - tau) > tol_p;
                    if (off && row_dependent(S)) {
                        ++bviol;
                        if (tu < tau) { P.wcap[a] = 0; ++dep_in; }
                        else ++dep_out;
                    } else if (off) {
                        ++bviol;
                    }
                    r_comp = fmax(r_comp, fabs(theta) * fabs(tau - tu));
                    if (theta < -tol_d) { ++bviol; r_comp = fmax(r_comp, -theta); P.wcap[a] = 0; }
                }
            }
            // factor rows: exposures h = B'w against their bounds, like the bands
            if (P.flo) factor_row_checks(P, sh, a, m, tol_p, tol_d, r_exp, r_comp, bviol, dep_in, dep_out);
            const double r_budget = fabs(sw - 1.0);
            if (r_budget > tol_p) ++bviol;
            const int total = int(nv) + bviol;
            if (dep_out > 0 || (total > 0 && ndep > 0 && dep_in == 0)) {
                // a working row is dependent on the free set and cannot be met by it: free the
                // fixed entry closest to leaving its breakpoint, in the direction of least resistance
                double bm = INFINITY;
                int who = 0;
                for (int w = 0; w < PB / 32; ++w)
                    if (sh.mmin[w] < bm || (sh.mmin[w] == bm && abs(sh.mwho[w]) < abs(who))) { bm = sh.mmin[w]; who = sh.mwho[w]; }
                if (who != 0) {
                    const size_t e = base + (abs(who) - 1);
                    const int j = P.st[e];
                    if (j < ST_FREE) P.st[e] = (int8_t)(who > 0 ? ST_FREE + j : ST_FREE + j - 1);
                }
            }
            double* dg = P.diag + (size_t)a * PRISM_NDIAG;
            dg[PRISM_DIAG_BUDGET] = r_budget;
            dg[PRISM_DIAG_BOX] = fmax(rb, 0.0);
            dg[PRISM_DIAG_EXPOSURE] = fmax(r_exp, 0.0);
            dg[PRISM_DIAG_TURNOVER] = r_turn;
            dg[PRISM_DIAG_STAT] = rs;
            dg[PRISM_DIAG_COMP] = r_comp;
            dg[PRISM_DIAG_OBJ] = quad + ol;
            dg[PRISM_DIAG_ERR_EST] = err_bound(P, sh, sqrt(rq), sw, tu, tau, nu, theta);
            P.nu[a] = nu;
            P.theta[a] = theta;
            for (int s2 = 0; s2 < S; ++s2) P.lam[a * S + s2] = sh.lam_s[s2];
            if (P.kappa) for (int k = 0; k < K; ++k) P.kappa[a * K + k] = sh.kap_s[k];
            if (total == 0) P.done[a] = 1;
            sh.go = (total > 0);
        }
        __syncthreads();
        if (!sh.go) break;
    }
}

// Diagnostics of the fallback weights (no multipliers: stationarity is not certified).
__global__ void __launch_bounds__(PB) k_diag_only(PolDev P) {
    const int a = blockIdx.x;
    if ((P.skip && P.skip[a]) || P.done[a] == 1) return;
    __shared__ double red[PB / 32][4];
    __shared__ double secsum[SMAX];
    __shared__ double hk[KMAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, S = P.S, N = P.N;
    const size_t base = (size_t)a * P.Npad;
    const double* W = P.W + base;
    for (int k = tid; k < K; k += PB) {
        double acc = 0.0;
        for (int p = 0; p < N; ++p) {
            double wv = W[p];
            if (wv != 0.0) acc += wv * P.B64[(size_t)p * K + k];
        }
        hk[k] = acc;
    }
    double sw = 0.0, rb = 0.0, ol = 0.0, tu = 0.0;
    for (int p = tid; p < N; p += PB) {
        const size_t e = base + p;
        Pieces pc;
        entry_pieces(P, e, pc);
        const double wv = W[p];
        sw += wv;
        rb = fmax(rb, fmax(P.lo[e] - wv, wv - P.up[e]));
        tu += fabs(wv - pc.w0);
        ol += P.d64[p] * wv * wv - P.mu64[p] * wv + phi_value(pc, wv);
    }
    sw = warp_sum(sw); rb = warp_max(rb); ol = warp_sum(ol); tu = warp_sum(tu);
    if (lane == 0) { red[warp][0] = sw; red[warp][1] = rb; red[warp][2] = ol; red[warp][3] = tu; }
    for (int s = warp; s < S; s += PB / 32) {
        double acc = 0.0;
        for (int p = P.sec_start[s] + lane; p < P.sec_start[s + 1]; p += 32) acc += W[p];
        acc = warp_sum(acc);
        if (lane == 0) secsum[s] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int w = 0; w < PB / 32; ++w) { s0 += red[w][0]; s1 = fmax(s1, red[w][1]); s2 += red[w][2]; s3 += red[w][3]; }
        double r_exp = 0.0;
        for (int s = 0; s < S; ++s)
            r_exp = fmax(r_exp, fmax(P.band_lo[a * S + s] - secsum[s], secsum[s] - P.band_hi[a * S + s]));
        for (int k = 0; k < K && P.flo; ++k)
            r_exp = fmax(r_exp, fmax(P.flo[a * K + k] - hk[k], hk[k] - P.fhi[a * K + k]));
        double quad = 0.0;
        for (int k = 0; k < K; ++k) quad += hk[k] * P.f64[k] * hk[k];
        double* dg = P.diag + (size_t)a * PRISM_NDIAG;
        dg[PRISM_DIAG_BUDGET] = fabs(s0 - 1.0);
        dg[PRISM_DIAG_BOX] = fmax(s1, 0.0);
        dg[PRISM_DIAG_EXPOSURE] = fmax(r_exp, 0.0);
        const double tau = P.tau[a];
        dg[PRISM_DIAG_TURNOVER] = isfinite(tau) ? fmax(s3 - tau, 0.0) : 0.0;
        dg[PRISM_DIAG_STAT] = INFINITY;
        dg[PRISM_DIAG_COMP] = INFINITY;
        dg[PRISM_DIAG_OBJ] = quad + s2;
        dg[PRISM_DIAG_ERR_EST] = INFINITY;
    }
}

// Final status from the diagnostics and the polish outcome.
__global__ void k_finish_status(PolDev P, double eps) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= P.M) return;
    if (P.skip && P.skip[a]) return;
    const double* dg = P.diag + (size_t)a * PRISM_NDIAG;
    const double prim = fmax(fmax(dg[PRISM_DIAG_BUDGET], dg[PRISM_DIAG_BOX]),
                             fmax(dg[PRISM_DIAG_EXPOSURE], dg[PRISM_DIAG_TURNOVER]));
    const bool kkt = dg[PRISM_DIAG_STAT] <= eps && dg[PRISM_DIAG_COMP] <= eps;
    const int prior = P.status[a];
    bool finite = true;
    for (int q = 0; q < PRISM_NDIAG; ++q)
        if (q != PRISM_DIAG_STAT && q != PRISM_DIAG_COMP && q != PRISM_DIAG_ERR_EST && !isfinite(dg[q]))
            finite = false;
    int st;
    if (prior == PRISM_NUMERICAL_FAILURE || !finite) st = PRISM_NUMERICAL_FAILURE;
    else if (P.done[a] == 1 && prim <= eps && kkt) st = PRISM_CERTIFIED;
    else if (prior == PRISM_TIMEOUT) st = PRISM_TIMEOUT;
    else if (prim <= eps) st = PRISM_FEASIBLE_NONCERTIFIED;
    else st = PRISM_NO_FEASIBLE_RETURN;
    P.status[a] = st;
}

// Fallback weights for an account the polish could not settle: the ADMM iterate
// (feasible up to FP32 rounding), with diagnostics recomputed in FP64.
__global__ void k_fallback_weights(PolDev P) {
    const int a = blockIdx.x;
    if ((P.skip && P.skip[a]) || P.done[a] == 1) return;
    const size_t base = (size_t)a * P.Npad;
    for (int p = threadIdx.x; p < P.N; p += blockDim.x) P.W[base + p] = double(P.z[base + p]);
}

size_t polish_smem_bytes() { return sizeof(PolishShared); }

void launch_classify(const PolDev& P, cudaStream_t st) { k_classify<<<P.M, PB, 0, st>>>(P); }

// Up to `rounds` active-set rounds for every account not yet settled, in one launch.
void launch_polish(const PolDev& P, int rounds, cudaStream_t st) {
    cudaFuncSetAttribute(k_polish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PolishShared));
    k_polish<<<P.M, PB, sizeof(PolishShared), st>>>(P, rounds);
}

void launch_fallback(const PolDev& P, cudaStream_t st) {
    k_fallback_weights<<<P.M, 256, 0, st>>>(P);
    k_diag_only<<<P.M, PB, 0, st>>>(P);
}

void launch_finish_status(const PolDev& P, double eps, cudaStream_t st) {
    k_finish_status<<<cdiv(P.M, 128), 128, 0, st>>>(P, eps);
}

__global__ void k_adjoint_flags(PolDev P, uint8_t* flags) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)P.M * P.Npad) return;
    const int p = int(e % P.Npad);
    if (p >= P.N) { flags[e] = 0; return; }
    Pieces pc;
    entry_pieces(P, e, pc);
    const int code = P.st[e];
    int fl = 0;
    double sg;
    if (code >= ST_FREE) {
        fl = 1;
        sg = seg_sign(pc, code - ST_FREE);
    } else {
        if (code > 0 && code < pc.nb - 1) fl = 2;
        const double dw = P.W[e] - pc.w0;
        sg = dw > 0.0 ? 1.0 : (dw < 0.0 ? -1.0 : 0.0);
    }
    fl |= sg > 0.0 ? 4 : (sg < 0.0 ? 8 : 0);
    flags[e] = (uint8_t)fl;
}

void launch_adjoint_flags(const PolDev& P, uint8_t* flags, cudaStream_t st) {
    const size_t n = (size_t)P.M * P.Npad;
    k_adjoint_flags<<<(unsigned)cdiv64((int64_t)n, 256), 256, 0, st>>>(P, flags);
}

}  // namespace prism
