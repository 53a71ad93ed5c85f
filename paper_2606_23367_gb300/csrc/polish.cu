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

// The per-entry inputs of the checks, loaded together so that one thread has many
// independent loads in flight (the int8 state stores would otherwise order them).
struct EntryRaw {
    double w0, lo, up, c, W, d, mu, bn1;
    float g32;
    int code, sec, pw;
};

__device__ __forceinline__ void load_raw(const PolDev& P, size_t base, int p, EntryRaw& r) {
    const size_t e = base + p;
    r.w0 = P.w0[e]; r.lo = P.lo[e]; r.up = P.up[e]; r.c = P.c[e];
    r.W = P.W[e]; r.d = P.d64[p]; r.mu = P.mu64[p]; r.bn1 = P.Bn1[p];
    r.g32 = P.G32[e];
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
// P1: the FP64 equality-constrained solve on the current working set
// (one block per account still running)
// ---------------------------------------------------------------------------
constexpr int BCH = 64;   // rows of B_F staged in shared memory at a time

struct SolveShared {
    double C[KMAX][KMAX + 1];          // capacitance, then its Cholesky factor (lower)
    double Bc[BCH][KMAX + 1];          // staged rows of B_F
    double dinv[BCH];
    double T[KMAX][PMAXROWS + 1];
    double hA[KMAX], fhA[KMAX];
    double Sm[PMAXROWS][PMAXROWS + 1];
    double erhs[PMAXROWS], lam[PMAXROWS];
    int rows[PMAXROWS];
    int nrows, nF, nNZ, fail, ndep;
    int cntF[PB], cntN[PB];
    double sumA[PB], capA[PB];
};

// coefficient of free entry p (cap sign sig) in working row ``row``
__device__ __forceinline__ double row_coef(const PolDev& P, int row, int p, double sig) {
    if (row < 0) return 1.0;                                  // budget
    if (row < P.S) return (P.sector[p] == row) ? 1.0 : 0.0;   // band
    return sig;                                               // cap
}

__global__ void __launch_bounds__(PB) k_pol_solve(PolDev P) {
    const int a = blockIdx.x;
    if ((P.skip && P.skip[a]) || P.done[a]) return;
    extern __shared__ unsigned char smem_raw[];
    SolveShared& sh = *reinterpret_cast<SolveShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, S = P.S, N = P.N;
    const size_t base = (size_t)a * P.Npad;
    int* Fl = P.Flist + (size_t)a * P.FMAX;
    int* NZl = P.NZlist + (size_t)a * P.FMAX;
    double* Fsig = P.Fsig + (size_t)a * P.FMAX;
    double* Y = P.Y + (size_t)a * P.FMAX * (PMAXROWS + 1);
    double* W = P.W + base;
    // ---- 1. ordered compaction: warp w owns a contiguous range of entries, read in
    // coalesced tiles of 32; pass 1 counts (and fixes W of fixed entries), pass 2 writes
    const int Lw = cdiv(cdiv(N, PB / 32), 32) * 32;
    const int w0r = min(N, warp * Lw), w1r = min(N, w0r + Lw);
    int nf = 0, nn = 0;
    double sa = 0.0, ca = 0.0;
    for (int p = w0r + lane; p < w1r + lane; p += 32) {
        int isF = 0, isNZ = 0;
        if (p < w1r) {
            const size_t e = base + p;
            const int code = P.st[e];
            Pieces pc;
            entry_pieces(P, e, pc);
            if (code >= ST_FREE) {
                isF = 1;
                ca -= seg_sign(pc, code - ST_FREE) * pc.w0;
            } else {
                const double wv = pc.bp[code];
                W[p] = wv;
                sa += wv;
                ca += fabs(wv - pc.w0);
                isNZ = (wv != 0.0);
            }
        }
        nf += __popc(__ballot_sync(0xffffffffu, isF));
        nn += __popc(__ballot_sync(0xffffffffu, isNZ));
    }
    sa = warp_sum(sa);
    ca = warp_sum(ca);
    if (lane == 0) {
        sh.cntF[warp] = nf;
        sh.cntN[warp] = nn;
        sh.sumA[warp] = sa;
        sh.capA[warp] = ca;
    }
    __syncthreads();
    if (tid == 0) {
        int of = 0, on = 0;
        double ss = 0.0, cc = 0.0;
        for (int t = 0; t < PB / 32; ++t) {
            const int f = sh.cntF[t], n = sh.cntN[t];
            sh.cntF[t] = of; sh.cntN[t] = on;
            of += f; on += n;
            ss += sh.sumA[t]; cc += sh.capA[t];
        }
        sh.nF = of; sh.nNZ = on;
        sh.sumA[0] = ss; sh.capA[0] = cc;
        sh.fail = (of > P.FMAX || on > P.FMAX || of == 0);
        // working rows
        int r = 0;
        sh.rows[r++] = -1;
        for (int q = 0; q < S; ++q)
            if (P.wband[a * S + q] != 0) { if (r < PMAXROWS) sh.rows[r] = q; ++r; }
        if (P.wcap[a]) { if (r < PMAXROWS) sh.rows[r] = S; ++r; }
        sh.nrows = r;
        if (r > PMAXROWS) sh.fail = 1;
    }
    __syncthreads();
    if (sh.fail) {
        if (tid == 0) P.done[a] = 2;
        return;
    }
    {
        int of = sh.cntF[warp], on = sh.cntN[warp];
        const unsigned lt = (1u << lane) - 1u;
        for (int p = w0r + lane; p < w1r + lane; p += 32) {
            int isF = 0, isNZ = 0;
            if (p < w1r) {
                isF = P.st[base + p] >= ST_FREE;
                isNZ = !isF && W[p] != 0.0;
            }
            const unsigned bF = __ballot_sync(0xffffffffu, isF), bN = __ballot_sync(0xffffffffu, isNZ);
            if (isF) Fl[of + __popc(bF & lt)] = p;
            if (isNZ) NZl[on + __popc(bN & lt)] = p;
            of += __popc(bF);
            on += __popc(bN);
        }
    }
    __syncthreads();
    const int nF = sh.nF, nNZ = sh.nNZ, m = sh.nrows;
    const double sumA = sh.sumA[0], capA = sh.capA[0];
    // ---- 2. h_A = B' w_A over the nonzero fixed entries
    for (int k = tid; k < K; k += PB) {
        double acc = 0.0;
        for (int q = 0; q < nNZ; ++q) {
            const int p = NZl[q];
            acc += W[p] * P.B64[(size_t)p * K + k];
        }
        sh.hA[k] = acc;
        sh.fhA[k] = P.f64[k] * acc;
    }
    __syncthreads();
    // ---- 3. scaled right-hand sides D^{-1} [g0, E_F'] of the free entries
    for (int q = tid; q < nF; q += PB) {
        const int p = Fl[q];
        const size_t e = base + p;
        Pieces pc;
        entry_pieces(P, e, pc);
        const int seg = P.st[e] - ST_FREE;
        const double* Bp = P.B64 + (size_t)p * K;
        double bfh = 0.0;
        for (int k = 0; k < K; ++k) bfh += Bp[k] * sh.fhA[k];
        const double dinv = 1.0 / P.d64[p];
        const double sig = seg_sign(pc, seg);
        Fsig[q] = sig;
        double* Yq = Y + (size_t)q * (PMAXROWS + 1);
        Yq[0] = (P.mu64[p] - pc.sl[seg] - 2.0 * bfh) * dinv;
        for (int r = 0; r < m; ++r) Yq[1 + r] = row_coef(P, sh.rows[r], p, sig) * dinv;
    }
    // ---- 4. C = F^{-1} + B_F' D_F^{-1} B_F and T = B_F' Y, over staged chunks of B_F
    for (int e2 = tid; e2 < K * K; e2 += PB) {
        const int r = e2 / K, c = e2 % K;
        sh.C[r][c] = (r == c) ? 1.0 / P.f64[r] : 0.0;
    }
    for (int e2 = tid; e2 < K * (PMAXROWS + 1); e2 += PB) sh.T[e2 / (PMAXROWS + 1)][e2 % (PMAXROWS + 1)] = 0.0;
    for (int q0 = 0; q0 < nF; q0 += BCH) {
        const int nb = min(BCH, nF - q0);
        __syncthreads();
        for (int e2 = tid; e2 < nb * K; e2 += PB) {
            const int j = e2 / K, k = e2 % K;
            sh.Bc[j][k] = P.B64[(size_t)Fl[q0 + j] * K + k];
        }
        for (int j = tid; j < nb; j += PB) sh.dinv[j] = 1.0 / P.d64[Fl[q0 + j]];
        __syncthreads();
        for (int e2 = tid; e2 < K * K; e2 += PB) {
            const int r = e2 / K, c = e2 % K;
            if (c > r) continue;
            double acc = 0.0;
            for (int j = 0; j < nb; ++j) acc += sh.Bc[j][r] * sh.Bc[j][c] * sh.dinv[j];
            sh.C[r][c] += acc;
        }
        for (int e2 = tid; e2 < K * (m + 1); e2 += PB) {
            const int k = e2 / (m + 1), c = e2 % (m + 1);
            double acc = 0.0;
            for (int j = 0; j < nb; ++j) acc += sh.Bc[j][k] * Y[(size_t)(q0 + j) * (PMAXROWS + 1) + c];
            sh.T[k][c] += acc;
        }
    }
    __syncthreads();
    // ---- 5. Cholesky of C by warp 0 (lower triangle, in place)
    if (warp == 0) {
        for (int c = 0; c < K; ++c) {
            const double piv = sh.C[c][c];
            if (!(piv > 0.0)) { if (lane == 0) sh.fail = 1; break; }
            const double lc = sqrt(piv);
            __syncwarp();
            if (lane == 0) sh.C[c][c] = lc;
            for (int r = c + 1 + lane; r < K; r += 32) sh.C[r][c] /= lc;
            __syncwarp();
            const int w = K - c - 1;
            for (int idx = lane; idx < w * w; idx += 32) {
                const int r = c + 1 + idx / w, q = c + 1 + idx % w;
                if (q <= r) sh.C[r][q] -= sh.C[r][c] * sh.C[q][c];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    if (sh.fail) {
        if (tid == 0) P.done[a] = 2;
        return;
    }
    // ---- 6. T <- C^{-1} T, one column per warp at a time (substitution with lanes over rows)
    for (int c = warp; c < m + 1; c += PB / 32) {
        for (int r = 0; r < K; ++r) {
            const double x = sh.T[r][c] / sh.C[r][r];
            __syncwarp();
            for (int q = r + 1 + lane; q < K; q += 32) sh.T[q][c] -= sh.C[q][r] * x;
            if (lane == 0) sh.T[r][c] = x;
            __syncwarp();
        }
        for (int r = K - 1; r >= 0; --r) {
            const double x = sh.T[r][c] / sh.C[r][r];
            __syncwarp();
            for (int q = lane; q < r; q += 32) sh.T[q][c] -= sh.C[r][q] * x;
            if (lane == 0) sh.T[r][c] = x;
            __syncwarp();
        }
    }
    __syncthreads();
    // ---- 7. Y <- D^{-1} (X - B_F T): now Y = Sigma_FF^{-1} [g0, E_F']
    for (int q0 = 0; q0 < nF; q0 += BCH) {
        const int nb = min(BCH, nF - q0);
        __syncthreads();
        for (int e2 = tid; e2 < nb * K; e2 += PB) {
            const int j = e2 / K, k = e2 % K;
            sh.Bc[j][k] = P.B64[(size_t)Fl[q0 + j] * K + k];
        }
        for (int j = tid; j < nb; j += PB) sh.dinv[j] = 1.0 / P.d64[Fl[q0 + j]];
        __syncthreads();
        for (int e2 = tid; e2 < nb * (m + 1); e2 += PB) {
            const int j = e2 / (m + 1), c = e2 % (m + 1);
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += sh.Bc[j][k] * sh.T[k][c];
            Y[(size_t)(q0 + j) * (PMAXROWS + 1) + c] -= acc * sh.dinv[j];
        }
    }
    __syncthreads();
    // ---- 8. Schur system (1/2) E Y_E lambda = (1/2) E Y_g - e
    for (int e2 = tid; e2 < m * (m + 1); e2 += PB) {
        const int r = e2 / (m + 1), c = e2 % (m + 1);
        double acc = 0.0;
        for (int q = 0; q < nF; ++q)
            acc += row_coef(P, sh.rows[r], Fl[q], Fsig[q]) * Y[(size_t)q * (PMAXROWS + 1) + c];
        if (c == 0) sh.erhs[r] = 0.5 * acc;
        else sh.Sm[r][c - 1] = 0.5 * acc;
    }
    __syncthreads();
    // edges of the working rows minus what the fixed entries already contribute
    for (int r = tid; r < m; r += PB) {
        const int row = sh.rows[r];
        double e_r;
        if (row < 0) {
            e_r = 1.0 - sumA;
        } else if (row < S) {
            double fixed_s = 0.0;
            for (int q = 0; q < nNZ; ++q)
                if (P.sector[NZl[q]] == row) fixed_s += W[NZl[q]];
            const double edge = (P.wband[a * S + row] > 0) ? P.band_hi[a * S + row] : P.band_lo[a * S + row];
            e_r = edge - fixed_s;
        } else {
            e_r = P.tau[a] - capA;
        }
        sh.erhs[r] -= e_r;
    }
    __syncthreads();
    // symmetric elimination with diagonal pivoting (budget row first); rows whose pivot
    // vanishes are dependent on the free set and get multiplier 0
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
    // ---- 9. w_F = 1/2 (Y_g - Y_E lambda); h = h_A + B_F' w_F; multipliers
    for (int q = tid; q < nF; q += PB) {
        const double* Yq = Y + (size_t)q * (PMAXROWS + 1);
        double acc = Yq[0];
        for (int r = 0; r < m; ++r) acc -= Yq[1 + r] * sh.lam[r];
        W[Fl[q]] = 0.5 * acc;
    }
    __syncthreads();
    for (int k = tid; k < K; k += PB) {
        double acc = sh.hA[k];
        for (int q = 0; q < nF; ++q) acc += W[Fl[q]] * P.B64[(size_t)Fl[q] * K + k];
        const double fh = P.f64[k] * acc;
        P.fh64[(size_t)a * KMAX + k] = fh;
        P.fh32[(size_t)a * K + k] = float(fh);
        sh.hA[k] = acc;        // reuse: full h
        sh.fhA[k] = fh;
    }
    __syncthreads();
    if (tid == 0) {
        double quad = 0.0, fmax_ = 0.0;
        for (int k = 0; k < K; ++k) { quad += sh.hA[k] * sh.fhA[k]; fmax_ = fmax(fmax_, fabs(sh.fhA[k])); }
        P.quad[a] = quad;
        P.fhmax[a] = fmax_;
        P.nu[a] = sh.lam[0];
        double theta = 0.0;
        for (int s = 0; s < S; ++s) P.lam[a * S + s] = 0.0;
        for (int r = 1; r < m; ++r) {
            if (sh.rows[r] < S) P.lam[a * S + sh.rows[r]] = sh.lam[r];
            else theta = sh.lam[r];
        }
        P.theta[a] = theta;
        P.ndep[a] = sh.ndep;
    }
}

// ---------------------------------------------------------------------------
// P3: KKT / feasibility checks of the solved point (Sec. 4.4), state switches,
// diagnostics. The batched FP32 product G32 = B (F h) filters the entries: an
// entry whose FP32 margin exceeds a bound on the FP32 error is decided by it;
// every other entry, and every free entry, is recomputed in FP64.
// ---------------------------------------------------------------------------
struct CheckShared {
    double lam[SMAX];
    double fh[KMAX];
    double red[PB / 32][6];
    double secsum[SMAX];
    double mmin[PB / 32];
    int mwho[PB / 32];
};

__global__ void __launch_bounds__(PB) k_pol_check(PolDev P) {
    const int a = blockIdx.x;
    if ((P.skip && P.skip[a]) || P.done[a]) return;
    __shared__ CheckShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.K, S = P.S, N = P.N;
    const size_t base = (size_t)a * P.Npad;
    double* W = P.W + base;
    for (int s = tid; s < S; s += PB) sh.lam[s] = P.lam[a * S + s];
    for (int k = tid; k < K; k += PB) sh.fh[k] = P.fh64[(size_t)a * KMAX + k];
    __syncthreads();
    const double nu = P.nu[a], theta = P.theta[a], fhmax = P.fhmax[a];
    const double tol_d = P.tol_dual, tol_p = P.tol_primal;
    double r_stat = 0.0, r_box = 0.0, obj_lin = 0.0, sum_w = 0.0, turn = 0.0;
    int nviol = 0;
    double my_margin = INFINITY;
    int my_who = 0;
    constexpr int CH = 4;
    for (int p0 = tid; p0 < N; p0 += PB * CH) {
        EntryRaw raw[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int p = p0 + PB * c;
            if (p < N) load_raw(P, base, p, raw[c]);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
        const int p = p0 + PB * c;
        if (p >= N) break;
        const size_t e = base + p;
        const EntryRaw& rw = raw[c];
        Pieces pc;
        pieces_from(P, rw, pc);
        const int code = rw.code;
        const double wv = rw.W;
        const double dd = rw.d, mu = rw.mu;
        const double lam_s = sh.lam[rw.sec];
        sum_w += wv;
        turn += fabs(wv - pc.w0);
        obj_lin += dd * wv * wv - mu * wv + phi_value(pc, wv);
        r_box = fmax(r_box, fmax(rw.lo - wv, wv - rw.up));
        // FP32 gradient and its error bound
        const double g_a = 2.0 * (double(rw.g32) + dd * wv) - mu;
        const double delta = 1e-5 * (2.0 * rw.bn1 * fhmax + 2.0 * fabs(dd * wv) + fabs(mu) + fabs(nu) + fabs(lam_s));
        auto exact_rr = [&]() {
            const double* Bp = P.B64 + (size_t)p * K;
            double bfh = 0.0;
            for (int k = 0; k < K; ++k) bfh += Bp[k] * sh.fh[k];
            return 2.0 * (bfh + dd * wv) - mu + nu + lam_s;
        };
        if (code >= ST_FREE) {
            const int seg = code - ST_FREE;
            const double rr = exact_rr();
            r_stat = fmax(r_stat, fabs(rr + pc.sl[seg] + theta * seg_sign(pc, seg)));
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
            r_stat = fmax(r_stat, fmax(fmax(up, dn), 0.0));
            if (pc.nb > 1) {
                if (isfinite(right) && -up < my_margin) { my_margin = -up; my_who = p + 1; }
                if (isfinite(left) && -dn < my_margin) { my_margin = -dn; my_who = -(p + 1); }
            }
            if (up > tol_d) { ++nviol; P.st[e] = (int8_t)(ST_FREE + j); }
            else if (dn > tol_d) { ++nviol; P.st[e] = (int8_t)(ST_FREE + j - 1); }
        }
        }
    }
    r_stat = warp_max(r_stat); r_box = warp_max(r_box);
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
        sh.mmin[warp] = my_margin; sh.mwho[warp] = my_who;
    }
    for (int s = warp; s < S; s += PB / 32) {
        double acc = 0.0;
        for (int p = P.sec_start[s] + lane; p < P.sec_start[s + 1]; p += 32) acc += W[p];
        acc = warp_sum(acc);
        if (lane == 0) sh.secsum[s] = acc;
    }
    __syncthreads();
    if (tid != 0) return;
    double rs = 0, rb = 0, ol = 0, sw = 0, tu = 0, nv = 0;
    for (int w = 0; w < PB / 32; ++w) {
        rs = fmax(rs, sh.red[w][0]); rb = fmax(rb, sh.red[w][1]); ol += sh.red[w][2];
        sw += sh.red[w][3]; tu += sh.red[w][4]; nv += sh.red[w][5];
    }
    double r_exp = 0.0, r_comp = 0.0;
    int bviol = 0;
    for (int s = 0; s < S; ++s) {
        const double ssum = sh.secsum[s];
        const double hi = P.band_hi[a * S + s], lo = P.band_lo[a * S + s];
        r_exp = fmax(r_exp, fmax(lo - ssum, ssum - hi));
        const int wb = P.wband[a * S + s];
        const double ls = sh.lam[s];
        if (wb != 0 && fabs(ssum - (wb > 0 ? hi : lo)) > tol_p) ++bviol;   // dropped dependent row
        if (wb == 0) {
            if (ssum > hi + tol_p) { ++bviol; P.wband[a * S + s] = 1; }
            else if (ssum < lo - tol_p) { ++bviol; P.wband[a * S + s] = -1; }
        } else if (wb > 0) {
            r_comp = fmax(r_comp, fabs(ls) * fabs(hi - ssum));
            if (ls < -tol_d) { ++bviol; r_comp = fmax(r_comp, -ls); P.wband[a * S + s] = 0; }
        } else {
            r_comp = fmax(r_comp, fabs(ls) * fabs(ssum - lo));
            if (ls > tol_d) { ++bviol; r_comp = fmax(r_comp, ls); P.wband[a * S + s] = 0; }
        }
    }
    double r_turn = 0.0;
    const double tau = P.tau[a];
    if (isfinite(tau)) {
        r_turn = fmax(tu - tau, 0.0);
        if (!P.wcap[a]) {
            if (tu > tau + tol_p) { ++bviol; P.wcap[a] = 1; }
        } else {
            if (fabs(tu - tau) > tol_p) ++bviol;                            // dropped dependent row
            r_comp = fmax(r_comp, fabs(theta) * fabs(tau - tu));
            if (theta < -tol_d) { ++bviol; r_comp = fmax(r_comp, -theta); P.wcap[a] = 0; }
        }
    }
    const double r_budget = fabs(sw - 1.0);
    if (r_budget > tol_p) ++bviol;
    const int total = int(nv) + bviol;
    if (total > 0 && P.ndep[a] > 0) {
        // the working rows were dependent on the free set: free the fixed entry
        // closest to leaving its breakpoint, in the direction of least resistance
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
    dg[PRISM_DIAG_OBJ] = P.quad[a] + ol;
    dg[PRISM_DIAG_ITERS] = dg[PRISM_DIAG_ITERS] + 1.0;
    if (total == 0) P.done[a] = 1;
    else atomicAdd(P.pending, 1);
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

size_t polish_smem_bytes() { return sizeof(SolveShared); }

void launch_classify(const PolDev& P, cudaStream_t st) { k_classify<<<P.M, PB, 0, st>>>(P); }

// One polish round: FP64 solve, batched FP32 gradient product, checks. Accounts that
// still need work add themselves to *P.pending.
void launch_polish_round(const PolDev& P, cudaStream_t st) {
    cudaFuncSetAttribute(k_pol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SolveShared));
    cudaMemsetAsync(P.pending, 0, sizeof(int), st);
    k_pol_solve<<<P.M, PB, sizeof(SolveShared), st>>>(P);
    launch_gradient_product(P, st);
    k_pol_check<<<P.M, PB, 0, st>>>(P);
}

void launch_fallback(const PolDev& P, cudaStream_t st) {
    k_fallback_weights<<<P.M, 256, 0, st>>>(P);
    k_diag_only<<<P.M, PB, 0, st>>>(P);
}

void launch_finish_status(const PolDev& P, double eps, cudaStream_t st) {
    k_finish_status<<<cdiv(P.M, 128), 128, 0, st>>>(P, eps);
}

}  // namespace prism
