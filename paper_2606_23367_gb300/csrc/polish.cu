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
// is solved in FP64 through the Woodbury identity
//   Sigma_FF^{-1} = D_F^{-1} - D_F^{-1} B_F (F^{-1} + B_F' D_F^{-1} B_F)^{-1} B_F' D_F^{-1}
// (K x K Cholesky) and a Schur complement over the working rows, so the
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
    if ((P.skip && P.skip[a]) || P.done[a] == 1) return;
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
}

// ---------------------------------------------------------------------------
// one polish round (or the final certification when all states are settled)
// ---------------------------------------------------------------------------
struct PolShared {
    double C[KMAX][KMAX + 1];
    double h[KMAX];          // B' w (all entries)
    double hA[KMAX];         // B' w_A (fixed entries)
    double fh[KMAX];         // f .* h
    double T[KMAX][PMAXROWS + 1];
    double Sm[PMAXROWS][PMAXROWS + 1];
    double lam[PMAXROWS];
    double erhs[PMAXROWS];
    int rows[PMAXROWS];      // row id: -1 budget, s = band s, S = cap
    int nrows;
    int nF, nNZ;
    int wsum[PB / 32];
    double red[PB / 32][8];
    double secsum[SMAX];
    int viol;
    int fail;
    int ndep;                // working rows dependent on the free set this round
    double mmin[PB / 32];    // smallest dual margin of a fixed entry, per warp
    int mwho[PB / 32];       // its entry (signed: + release up, - release down) + 1
};

// coefficient of free entry p (cap sign sig) in working row ``row``
__device__ __forceinline__ double row_coef(const PolDev& P, int row, int p, double sig) {
    if (row < 0) return 1.0;                                  // budget
    if (row < P.S) return (P.sector[p] == row) ? 1.0 : 0.0;   // band
    return sig;                                               // cap
}

__global__ void __launch_bounds__(PB) k_polish_round(PolDev P) {
    const int final_round = 0;
    const int a = blockIdx.x;
    if ((P.skip && P.skip[a]) || P.done[a]) return;
    extern __shared__ unsigned char smem_raw[];
    PolShared& sh = *reinterpret_cast<PolShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, S = P.S, N = P.N;
    const size_t base = (size_t)a * P.Npad;
    int* Fl = P.Flist + (size_t)a * P.FMAX;
    int* NZl = P.NZlist + (size_t)a * P.FMAX;
    double* Y = P.Y + (size_t)a * P.FMAX * (PMAXROWS + 1);
    double* W = P.W + base;
    const double theta_prev = P.theta[a];
    // ---- 1. fixed values, compaction of free entries and nonzero fixed entries
    if (tid == 0) { sh.nF = 0; sh.nNZ = 0; sh.fail = 0; }
    __syncthreads();
    for (int p0 = 0; p0 < N; p0 += PB) {
        const int p = p0 + tid;
        int isF = 0, isNZ = 0;
        if (p < N) {
            const size_t e = base + p;
            const int code = P.st[e];
            if (code >= ST_FREE) {
                isF = 1;
            } else {
                Pieces pc;
                entry_pieces(P, e, pc);
                double wv = pc.bp[code];
                W[p] = wv;
                isNZ = (wv != 0.0);
            }
        }
        unsigned bF = __ballot_sync(0xffffffffu, isF), bN = __ballot_sync(0xffffffffu, isNZ);
        if (lane == 0) { sh.wsum[warp] = __popc(bF) | (__popc(bN) << 16); }
        __syncthreads();
        int offF = sh.nF, offN = sh.nNZ;
        for (int w = 0; w < warp; ++w) { offF += sh.wsum[w] & 0xffff; offN += sh.wsum[w] >> 16; }
        unsigned lt = (1u << lane) - 1u;
        if (isF) { int q = offF + __popc(bF & lt); if (q < P.FMAX) Fl[q] = p; }
        if (isNZ) { int q = offN + __popc(bN & lt); if (q < P.FMAX) NZl[q] = p; }
        __syncthreads();
        if (tid == 0) {
            int tF = 0, tN = 0;
            for (int w = 0; w < PB / 32; ++w) { tF += sh.wsum[w] & 0xffff; tN += sh.wsum[w] >> 16; }
            sh.nF += tF; sh.nNZ += tN;
        }
        __syncthreads();
    }
    const int nF = sh.nF, nNZ = sh.nNZ;
    if (nF > P.FMAX || nNZ > P.FMAX || nF == 0) {
        if (tid == 0) { P.done[a] = 2; }      // cannot polish this account
        return;
    }
    // ---- 2. working rows
    if (tid == 0) {
        int r = 0;
        sh.rows[r++] = -1;
        for (int s = 0; s < S; ++s)
            if (P.wband[a * S + s] != 0) { if (r < PMAXROWS) sh.rows[r] = s; ++r; }
        if (P.wcap[a]) { if (r < PMAXROWS) sh.rows[r] = S; ++r; }
        sh.nrows = r;
    }
    // ---- 3. hA = B' w_A over nonzero fixed entries
    __syncthreads();
    if (sh.nrows > PMAXROWS) {
        if (tid == 0) P.done[a] = 2;
        return;
    }
    const int m = sh.nrows;
    for (int k = tid; k < K; k += PB) {
        double acc = 0.0;
        for (int q = 0; q < nNZ; ++q) {
            int p = NZl[q];
            acc += W[p] * P.B64[(size_t)p * K + k];
        }
        sh.hA[k] = acc;
        sh.fh[k] = P.f64[k] * acc;
    }
    // ---- 4. capacitance C_F = F^{-1} + B_F' D_F^{-1} B_F (lower triangle)
    for (int e2 = tid; e2 < K * K; e2 += PB) {
        int r = e2 / K, c = e2 % K;
        if (c > r) continue;
        double acc = (r == c) ? 1.0 / P.f64[r] : 0.0;
        for (int q = 0; q < nF; ++q) {
            int p = Fl[q];
            const double* Bp = P.B64 + (size_t)p * K;
            acc += Bp[r] * Bp[c] / P.d64[p];
        }
        sh.C[r][c] = acc;
    }
    __syncthreads();
    // ---- 5. right-hand sides X = [g0, E_F'] scaled by D^{-1} into Y; rhs of rows
    for (int q = tid; q < nF; q += PB) {
        const int p = Fl[q];
        const size_t e = base + p;
        Pieces pc;
        entry_pieces(P, e, pc);
        const int seg = P.st[e] - ST_FREE;
        const double* Bp = P.B64 + (size_t)p * K;
        double bfh = 0.0;
        for (int k = 0; k < K; ++k) bfh += Bp[k] * sh.fh[k];
        const double g0 = P.mu64[p] - pc.sl[seg] - 2.0 * bfh;
        const double dinv = 1.0 / P.d64[p];
        const double sig = seg_sign(pc, seg);
        P.Fsig[(size_t)a * P.FMAX + q] = sig;
        Y[(size_t)q * (PMAXROWS + 1) + 0] = g0 * dinv;
        for (int r = 0; r < m; ++r)
            Y[(size_t)q * (PMAXROWS + 1) + 1 + r] = row_coef(P, sh.rows[r], p, sig) * dinv;
    }
    // Cholesky of C (in place, lower)
    for (int c = 0; c < K; ++c) {
        __syncthreads();
        if (tid == 0) sh.C[c][c] = sqrt(sh.C[c][c]);
        __syncthreads();
        for (int r = c + 1 + tid; r < K; r += PB) sh.C[r][c] /= sh.C[c][c];
        __syncthreads();
        for (int e2 = tid; e2 < (K - c - 1) * (K - c - 1); e2 += PB) {
            int r = c + 1 + e2 / (K - c - 1), q = c + 1 + e2 % (K - c - 1);
            if (q <= r) sh.C[r][q] -= sh.C[r][c] * sh.C[q][c];
        }
    }
    __syncthreads();
    // ---- 6. T = B_F' Y  (K x (m+1))
    for (int e2 = tid; e2 < K * (m + 1); e2 += PB) {
        int k = e2 / (m + 1), c = e2 % (m + 1);
        double acc = 0.0;
        for (int q = 0; q < nF; ++q) acc += P.B64[(size_t)Fl[q] * K + k] * Y[(size_t)q * (PMAXROWS + 1) + c];
        sh.T[k][c] = acc;
    }
    __syncthreads();
    // T <- C^{-1} T (one column per thread)
    for (int c = tid; c < m + 1; c += PB) {
        for (int r = 0; r < K; ++r) {
            double s = sh.T[r][c];
            for (int q = 0; q < r; ++q) s -= sh.C[r][q] * sh.T[q][c];
            sh.T[r][c] = s / sh.C[r][r];
        }
        for (int r = K - 1; r >= 0; --r) {
            double s = sh.T[r][c];
            for (int q = r + 1; q < K; ++q) s -= sh.C[q][r] * sh.T[q][c];
            sh.T[r][c] = s / sh.C[r][r];
        }
    }
    __syncthreads();
    // Y <- Y - D^{-1} B_F T   (now Y = Sigma_FF^{-1} [g0, E_F'])
    for (int e2 = tid; e2 < nF * (m + 1); e2 += PB) {
        int q = e2 / (m + 1), c = e2 % (m + 1);
        int p = Fl[q];
        const double* Bp = P.B64 + (size_t)p * K;
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += Bp[k] * sh.T[k][c];
        Y[(size_t)q * (PMAXROWS + 1) + c] -= acc / P.d64[p];
    }
    __syncthreads();
    // ---- 7. Schur system: (1/2) E Y_E lambda = (1/2) E Y_g - e
    for (int e2 = tid; e2 < m * (m + 1); e2 += PB) {
        int r = e2 / (m + 1), c = e2 % (m + 1);
        double acc = 0.0;
        const double* sig = P.Fsig + (size_t)a * P.FMAX;
        for (int q = 0; q < nF; ++q)
            acc += row_coef(P, sh.rows[r], Fl[q], sig[q]) * Y[(size_t)q * (PMAXROWS + 1) + c];
        if (c == 0) sh.erhs[r] = 0.5 * acc;
        else sh.Sm[r][c - 1] = 0.5 * acc;
    }
    // row right-hand sides e_r from the fixed entries
    if (warp == 0) {
        for (int r = 0; r < m; ++r) {
            const int row = sh.rows[r];
            double acc = 0.0;
            for (int p = lane; p < N; p += 32) {
                const size_t e = base + p;
                const int code = P.st[e];
                if (row < 0) { if (code < ST_FREE) acc += W[p]; }
                else if (row < S) { if (code < ST_FREE && P.sector[p] == row) acc += W[p]; }
                else {
                    if (code < ST_FREE) acc += fabs(W[p] - P.w0[e]);
                    else {
                        Pieces pc; entry_pieces(P, e, pc);
                        acc -= seg_sign(pc, code - ST_FREE) * P.w0[e];
                    }
                }
            }
            acc = warp_sum(acc);
            if (lane == 0) {
                double edge;
                if (row < 0) edge = 1.0;
                else if (row < S) edge = (P.wband[a * S + row] > 0) ? P.band_hi[a * S + row] : P.band_lo[a * S + row];
                else edge = P.tau[a];
                sh.erhs[r] -= (edge - acc);
            }
        }
    }
    __syncthreads();
    // solve the m x m PSD system by symmetric elimination with diagonal pivoting
    // (thread 0): the budget row first, then the largest remaining pivot; rows whose
    // pivot vanishes are linearly dependent on the free set and get multiplier 0
    // (their equations are checked after the solve).
    if (tid == 0) {
        double A[PMAXROWS][PMAXROWS + 1];
        int chosen[PMAXROWS], used[PMAXROWS];
        double scale = 0.0;
        for (int r = 0; r < m; ++r) {
            for (int c = 0; c < m; ++c) A[r][c] = sh.Sm[r][c];
            A[r][m] = sh.erhs[r];
            used[r] = 0;
            scale = fmax(scale, fabs(A[r][r]));
        }
        int nc = 0;
        for (int k = 0; k < m; ++k) {
            int p = -1;
            if (k == 0) p = 0;
            else {
                double best = 0.0;
                for (int j = 0; j < m; ++j)
                    if (!used[j] && fabs(A[j][j]) > best) { best = fabs(A[j][j]); p = j; }
            }
            if (p < 0 || !(fabs(A[p][p]) > 1e-11 * scale)) break;
            used[p] = 1;
            chosen[nc++] = p;
            for (int j = 0; j < m; ++j) {
                if (used[j]) continue;
                const double f = A[j][p] / A[p][p];
                for (int q = 0; q <= m; ++q) A[j][q] -= f * A[p][q];
            }
        }
        for (int r = 0; r < m; ++r) sh.lam[r] = 0.0;
        for (int k = nc - 1; k >= 0; --k) {
            const int p = chosen[k];
            double v = A[p][m];
            for (int q = 0; q < m; ++q) if (q != p && used[q]) v -= A[p][q] * sh.lam[q];
            sh.lam[p] = v / A[p][p];
        }
        sh.fail = (nc == 0);
        sh.ndep = m - nc;
    }
    __syncthreads();
    if (sh.fail) {
        if (tid == 0) P.done[a] = 2;
        return;
    }
    // ---- 8. w_F = 1/2 (Y_g - Y_E lambda)
    for (int q = tid; q < nF; q += PB) {
        double acc = Y[(size_t)q * (PMAXROWS + 1) + 0];
        for (int r = 0; r < m; ++r) acc -= Y[(size_t)q * (PMAXROWS + 1) + 1 + r] * sh.lam[r];
        W[Fl[q]] = 0.5 * acc;
    }
    __syncthreads();
    // multipliers in the result layout
    double nu = sh.lam[0];
    double theta = 0.0;
    // ---- 9. certification: h = B'w over all nonzero entries, gradient, checks
    for (int k = tid; k < K; k += PB) {
        double acc = sh.hA[k];
        for (int q = 0; q < nF; ++q) acc += W[Fl[q]] * P.B64[(size_t)Fl[q] * K + k];
        sh.h[k] = acc;
        sh.fh[k] = P.f64[k] * acc;
    }
    __syncthreads();
    for (int r = 1; r < m; ++r) if (sh.rows[r] == S) theta = sh.lam[r];
    // per-entry checks
    double r_stat = 0.0, r_box = 0.0, obj_lin = 0.0, sum_w = 0.0, turn = 0.0;
    int nviol = 0;
    double my_margin = INFINITY;
    int my_who = 0;
    const double tol_d = P.tol_dual, tol_p = P.tol_primal;
    for (int p = tid; p < N; p += PB) {
        const size_t e = base + p;
        Pieces pc;
        entry_pieces(P, e, pc);
        const int code = P.st[e];
        const double wv = W[p];
        const double* Bp = P.B64 + (size_t)p * K;
        double bfh = 0.0;
        for (int k = 0; k < K; ++k) bfh += Bp[k] * sh.fh[k];
        const double g = 2.0 * (bfh + P.d64[p] * wv) - P.mu64[p];
        const int s = P.sector[p];
        double lam_s = 0.0;
        for (int r = 1; r < m; ++r) if (sh.rows[r] == s) lam_s = sh.lam[r];
        const double rr = g + nu + lam_s;
        sum_w += wv;
        turn += fabs(wv - pc.w0);
        obj_lin += P.d64[p] * wv * wv - P.mu64[p] * wv + phi_value(pc, wv);
        r_box = fmax(r_box, fmax(P.lo[e] - wv, wv - P.up[e]));
        if (code >= ST_FREE) {
            const int seg = code - ST_FREE;
            const double stat = fabs(rr + pc.sl[seg] + theta * seg_sign(pc, seg));
            r_stat = fmax(r_stat, stat);
            if (wv > pc.bp[seg + 1] + tol_p) {
                ++nviol;
                if (!final_round) P.st[e] = (int8_t)(seg + 1);
            } else if (wv < pc.bp[seg] - tol_p) {
                ++nviol;
                if (!final_round) P.st[e] = (int8_t)seg;
            }
        } else {
            const int j = code;
            const double left = (j > 0) ? pc.sl[j - 1] + theta * seg_sign(pc, j - 1) : -INFINITY;
            const double right = (j + 1 < pc.nb) ? pc.sl[j] + theta * seg_sign(pc, j) : INFINITY;
            const double up = -rr - right, dn = left + rr;
            r_stat = fmax(r_stat, fmax(fmax(up, dn), 0.0));
            if (pc.nb > 1) {
                // slack of the release condition on each finite side
                if (isfinite(right) && -up < my_margin) { my_margin = -up; my_who = p + 1; }
                if (isfinite(left) && -dn < my_margin) { my_margin = -dn; my_who = -(p + 1); }
            }
            if (up > tol_d) {
                ++nviol;
                if (!final_round) P.st[e] = (int8_t)(ST_FREE + j);
            } else if (dn > tol_d) {
                ++nviol;
                if (!final_round) P.st[e] = (int8_t)(ST_FREE + j - 1);
            }
        }
    }
    // block reductions
    r_stat = warp_max(r_stat); r_box = warp_max(r_box);
    obj_lin = warp_sum(obj_lin); sum_w = warp_sum(sum_w); turn = warp_sum(turn);
    nviol = warp_sum(nviol);
    for (int o = 16; o > 0; o >>= 1) {
        double om = __shfl_xor_sync(0xffffffffu, my_margin, o);
        int ow = __shfl_xor_sync(0xffffffffu, my_who, o);
        if (om < my_margin || (om == my_margin && abs(ow) < abs(my_who))) { my_margin = om; my_who = ow; }
    }
    if (lane == 0) { sh.mmin[warp] = my_margin; sh.mwho[warp] = my_who; }
    if (lane == 0) {
        sh.red[warp][0] = r_stat; sh.red[warp][1] = r_box; sh.red[warp][2] = obj_lin;
        sh.red[warp][3] = sum_w; sh.red[warp][4] = turn; sh.red[warp][5] = double(nviol);
    }
    for (int s = warp; s < S; s += PB / 32) {
        double acc = 0.0;
        for (int p = P.sec_start[s] + lane; p < P.sec_start[s + 1]; p += 32) acc += W[p];
        acc = warp_sum(acc);
        if (lane == 0) sh.secsum[s] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        double rs = 0, rb = 0, ol = 0, sw = 0, tu = 0, nv = 0;
        for (int w = 0; w < PB / 32; ++w) {
            rs = fmax(rs, sh.red[w][0]); rb = fmax(rb, sh.red[w][1]); ol += sh.red[w][2];
            sw += sh.red[w][3]; tu += sh.red[w][4]; nv += sh.red[w][5];
        }
        // bands
        double r_exp = 0.0, r_comp = 0.0;
        int bviol = 0;
        double lam_out[SMAX];
        for (int s = 0; s < S; ++s) lam_out[s] = 0.0;
        for (int r = 1; r < m; ++r) if (sh.rows[r] < S) lam_out[sh.rows[r]] = sh.lam[r];
        for (int s = 0; s < S; ++s) {
            const double ssum = sh.secsum[s];
            const double hi = P.band_hi[a * S + s], lo = P.band_lo[a * S + s];
            r_exp = fmax(r_exp, fmax(lo - ssum, ssum - hi));
            const int wb = P.wband[a * S + s];
            if (wb != 0 && fabs(ssum - (wb > 0 ? hi : lo)) > tol_p) ++bviol;   // dropped dependent row
            if (wb == 0) {
                if (ssum > hi + tol_p) { ++bviol; if (!final_round) P.wband[a * S + s] = 1; }
                else if (ssum < lo - tol_p) { ++bviol; if (!final_round) P.wband[a * S + s] = -1; }
            } else if (wb > 0) {
                r_comp = fmax(r_comp, fabs(lam_out[s]) * fabs(hi - ssum));
                if (lam_out[s] < -tol_d) { ++bviol; r_comp = fmax(r_comp, -lam_out[s]); if (!final_round) P.wband[a * S + s] = 0; }
            } else {
                r_comp = fmax(r_comp, fabs(lam_out[s]) * fabs(ssum - lo));
                if (lam_out[s] > tol_d) { ++bviol; r_comp = fmax(r_comp, lam_out[s]); if (!final_round) P.wband[a * S + s] = 0; }
            }
        }
        double r_turn = 0.0;
        const double tau = P.tau[a];
        if (isfinite(tau)) {
            r_turn = fmax(tu - tau, 0.0);
            if (!P.wcap[a]) {
                if (tu > tau + tol_p) { ++bviol; if (!final_round) P.wcap[a] = 1; }
            } else {
                if (fabs(tu - tau) > tol_p) ++bviol;                            // dropped dependent row
                r_comp = fmax(r_comp, fabs(theta) * fabs(tau - tu));
                if (theta < -tol_d) { ++bviol; r_comp = fmax(r_comp, -theta); if (!final_round) P.wcap[a] = 0; }
            }
        }
        // objective: w'Sigma w - mu'w + sum phi = h' F h + sum(d w^2 - mu w + phi)
        double quad = 0.0;
        for (int k = 0; k < K; ++k) quad += sh.h[k] * sh.fh[k];
        const double obj = quad + ol;
        const double r_budget = fabs(sw - 1.0);
        const double r_box_v = fmax(rb, 0.0);
        if (r_budget > tol_p) ++bviol;
        int total = int(nv) + bviol;
        if (total > 0 && sh.ndep > 0 && !final_round) {
            // the working rows were dependent on the free set: free the fixed entry
            // closest to leaving its breakpoint, in the direction of least resistance
            double bm = INFINITY;
            int who = 0;
            for (int w = 0; w < PB / 32; ++w)
                if (sh.mmin[w] < bm || (sh.mmin[w] == bm && abs(sh.mwho[w]) < abs(who))) { bm = sh.mmin[w]; who = sh.mwho[w]; }
            if (who != 0) {
                const int p = abs(who) - 1;
                const size_t e = base + p;
                const int j = P.st[e];
                if (j < ST_FREE) P.st[e] = (int8_t)(who > 0 ? ST_FREE + j : ST_FREE + j - 1);
            }
        }
        double* dg = P.diag + (size_t)a * PRISM_NDIAG;
        dg[PRISM_DIAG_BUDGET] = r_budget;
        dg[PRISM_DIAG_BOX] = r_box_v;
        dg[PRISM_DIAG_EXPOSURE] = fmax(r_exp, 0.0);
        dg[PRISM_DIAG_TURNOVER] = r_turn;
        dg[PRISM_DIAG_STAT] = rs;
        dg[PRISM_DIAG_COMP] = r_comp;
        dg[PRISM_DIAG_OBJ] = obj;
        dg[PRISM_DIAG_ITERS] = dg[PRISM_DIAG_ITERS] + 1.0;
        P.nu[a] = nu;
        P.theta[a] = theta;
        for (int s = 0; s < S; ++s) P.lam[a * S + s] = lam_out[s];
        if (total == 0) P.done[a] = 1;
        (void)theta_prev;
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
        if (q != PRISM_DIAG_STAT && q != PRISM_DIAG_COMP && !isfinite(dg[q])) finite = false;
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

size_t polish_smem_bytes() { return sizeof(PolShared); }

void launch_classify(const PolDev& P, cudaStream_t st) { k_classify<<<P.M, PB, 0, st>>>(P); }

void launch_polish_round(const PolDev& P, cudaStream_t st) {
    cudaFuncSetAttribute(k_polish_round, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(PolShared));
    k_polish_round<<<P.M, PB, sizeof(PolShared), st>>>(P);
}

void launch_fallback(const PolDev& P, cudaStream_t st) {
    k_fallback_weights<<<P.M, 256, 0, st>>>(P);
    k_diag_only<<<P.M, PB, 0, st>>>(P);
}

void launch_finish_status(const PolDev& P, double eps, cudaStream_t st) {
    k_finish_status<<<cdiv(P.M, 128), 128, 0, st>>>(P, eps);
}

}  // namespace prism
