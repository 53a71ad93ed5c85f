// plain64.cu -- the PRISM_PLAIN_FP64 iterations: the same ADMM splitting as the batched
// kernels (x = z with f(x) = x' Sigma x - mu' x and g(z) = sum_i phi_i(z_i) + indicator of the
// Eq. 1 feasible set, Sec. 4.2), carried out in FP64 for one account per block, with all of
// the account's iterations in one launch.
//
// One iteration, penalty rho, relaxation alpha (Delta = diag(2 d + rho)):
//   X  = Delta^{-1} (mu + rho z - y)
//   Q  = C^{-1} B' X,            C = (2F)^{-1} + B' Delta^{-1} B      (Woodbury, K x K)
//   x  = X - Delta^{-1} B Q       = (2 Sigma + rho I)^{-1} (mu + rho z - y)
//   v  = alpha x + (1 - alpha) z + y / rho
//   z+ = argmin_{z in Z} sum_i phi_i(z_i) + rho/2 ||z - v||^2,   y+ = rho (v - z+)
// C is formed and Cholesky-factored in FP64 in shared memory whenever rho changes. The
// projection relaxes the budget (nu), the sector bands (lambda_s) and the turnover cap
// (theta): z_i = prox of (phi_i + theta |. - w0_i|)/rho on [l_i, u_i] at v_i - (nu +
// lambda_s(i))/rho; each sector sum S_s(eta) is nonincreasing and piecewise linear in eta,
// the budget reads sum_s clamp(S_s(nu), lo_s, hi_s) = 1, a sector held at an edge has its
// own eta_s = nu + lambda_s with S_s(eta_s) at that edge, and theta solves the turnover
// equation ||z(theta) - w0||_1 = tau when the cap binds. Every scalar root is bracketed and
// found by alternating secant and bisection steps (exact once the bracket lies on one linear
// piece). The result feeds the FP64 polish and certification like the other modes.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "plain64.h"

namespace prism {

constexpr int P64_THREADS = 256;
constexpr int P64_WARPS = P64_THREADS / 32;
constexpr int P64_ROOT_IT = 200;          // evaluations per scalar root (bisection alone needs ~110)

struct P64Shared {
    double L[KMAX][KMAX + 1];             // Cholesky factor of C (lower)
    double G[KMAX][KMAX + 1];             // B' Delta^{-1} B (factor-exposure block only)
    double P[KMAX], Q[KMAX];
    double s[KMAX], ys[KMAX], tv[KMAX], P0[KMAX];   // factor-exposure block: s = B'x, its dual
    double part[P64_THREADS / 64 > 0 ? P64_THREADS / 64 : 1][KMAX];
    double ssum[SMAX];                    // sector sums at the current evaluation point
    double eta_s[SMAX];                   // per-sector multiplier point (nu + lambda_s)
    double red[P64_WARPS][6];
    double nu, theta, rho, T, U;
    int go;
};

// Breakpoints and slopes of phi_i restricted to [l_i, u_i] (FP64).
struct P64Pieces {
    double bp[MAXBP];
    double sl[MAXBP - 1];
    int nb;
    double w0;
};

__device__ __forceinline__ void p64_pieces(const P64Args& A, size_t e, P64Pieces& pc) {
    const double w0 = A.w0[e], lo = A.lo[e], up = A.up[e], c = A.c[e];
    pc.w0 = w0;
    const int pw = A.pw_idx ? A.pw_idx[e] : -1;
    if (pw >= 0) {
        pc.nb = A.pw_nbp[pw];
        for (int j = 0; j < pc.nb; ++j) pc.bp[j] = A.pw_bp[(size_t)pw * MAXBP + j];
        for (int j = 0; j + 1 < pc.nb; ++j) pc.sl[j] = A.pw_sl[(size_t)pw * (MAXBP - 1) + j];
        return;
    }
    if (!(up > lo)) { pc.nb = 1; pc.bp[0] = lo; return; }
    if (w0 > lo && w0 < up) {
        pc.nb = 3; pc.bp[0] = lo; pc.bp[1] = w0; pc.bp[2] = up; pc.sl[0] = -c; pc.sl[1] = c;
    } else {
        pc.nb = 2; pc.bp[0] = lo; pc.bp[1] = up; pc.sl[0] = (w0 <= lo) ? c : -c;
    }
}

// Slope of phi_i + theta |. - w0| on segment j.
__device__ __forceinline__ double p64_slope(const P64Pieces& pc, int j, double theta) {
    const double mid = 0.5 * (pc.bp[j] + pc.bp[j + 1]);
    const double sg = mid > pc.w0 ? 1.0 : (mid < pc.w0 ? -1.0 : 0.0);
    return pc.sl[j] + theta * sg;
}

// argmin_z phi(z) + theta |z - w0| + rho/2 (z - t)^2 on [bp_0, bp_last]: the first segment j
// whose unconstrained minimiser t - s_j/rho falls left of its right end holds the answer,
// either inside it or at its left end (a kink or the lower bound).
__device__ __forceinline__ double p64_prox(const P64Pieces& pc, double t, double irho, double theta) {
    if (pc.nb == 1) return pc.bp[0];
    for (int j = 0; j + 1 < pc.nb; ++j) {
        const double zc = t - p64_slope(pc, j, theta) * irho;
        if (zc < pc.bp[j + 1]) return zc > pc.bp[j] ? zc : pc.bp[j];
    }
    return pc.bp[pc.nb - 1];
}

// Sum of z_i over sector s at eta (one warp; lane-strided over the sector's positions).
__device__ __forceinline__ double p64_sector_sum(const P64Args& A, const double* v, size_t base, int s, double eta,
                                                 double irho, double theta, int lane) {
    double acc = 0.0;
    for (int p = A.sec_start[s] + lane; p < A.sec_start[s + 1]; p += 32) {
        P64Pieces pc;
        p64_pieces(A, base + p, pc);
        acc += p64_prox(pc, v[base + p] - eta * irho, irho, theta);
    }
    return warp_sum(acc);
}

// Root of a nonincreasing function g on [a, b] with g(a) >= 0 >= g(b): alternate secant and
// bisection steps. Runs identically in every thread that calls it (eval is collective).
template <class Eval>
__device__ double p64_root(double a, double ga, double b, double gb, Eval&& eval) {
    for (int it = 0; it < P64_ROOT_IT; ++it) {
        if (ga == 0.0) return a;
        if (gb == 0.0) return b;
        const double w = b - a;
        if (!(w > 1e-15 * fmax(1.0, fmax(fabs(a), fabs(b))))) break;
        double m = (it & 1) ? 0.5 * (a + b) : a + w * ga / (ga - gb);
        if (!(m > a && m < b)) m = 0.5 * (a + b);
        const double gm = eval(m);
        if (gm > 0.0) { a = m; ga = gm; }
        else if (gm < 0.0) { b = m; gb = gm; }
        else return m;
    }
    return (ga < -gb) ? a : b;
}

// The projection of v (one account) onto Z for a given theta: the budget multiplier nu
// (in sh.nu) and each sector's eta_s (in sh.eta_s). Block-collective.
__device__ void p64_inner(const P64Args& A, P64Shared& sh, const double* v, size_t base, int a, double theta,
                          double eta_a, double eta_b, double irho) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = A.S;
    // T(eta) - 1 = sum_s clamp(S_s(eta), lo_s, hi_s) - 1, nonincreasing in eta
    auto T = [&](double eta) -> double {
        for (int s = warp; s < S; s += P64_WARPS) {
            const double sm = p64_sector_sum(A, v, base, s, eta, irho, theta, lane);
            if (lane == 0) sh.ssum[s] = fmin(fmax(sm, A.band_lo[a * S + s]), A.band_hi[a * S + s]);
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int s = 0; s < S; ++s) t += sh.ssum[s];
            sh.T = t - 1.0;
        }
        __syncthreads();
        const double r = sh.T;
        __syncthreads();
        return r;
    };
    const double ga = T(eta_a), gb = T(eta_b);
    const double nu = p64_root(eta_a, ga, eta_b, gb, T);
    // each sector held at an edge gets its own point (warp-local roots, no block barriers)
    for (int s = warp; s < S; s += P64_WARPS) {
        const double lo = A.band_lo[a * S + s], hi = A.band_hi[a * S + s];
        const double s0 = p64_sector_sum(A, v, base, s, nu, irho, theta, lane);
        double es = nu;
        auto G = [&](double target) {
            return [&, target](double eta) { return p64_sector_sum(A, v, base, s, eta, irho, theta, lane) - target; };
        };
        if (s0 > hi) {
            auto g = G(hi);
            es = p64_root(nu, s0 - hi, eta_b, g(eta_b), g);
        } else if (s0 < lo) {
            auto g = G(lo);
            es = p64_root(eta_a, g(eta_a), nu, s0 - lo, g);
        }
        if (lane == 0) sh.eta_s[s] = es;
    }
    if (tid == 0) sh.nu = nu;
    __syncthreads();
}

// ||z(theta) - w0||_1 of the projection just computed (block-collective).
__device__ double p64_turnover(const P64Args& A, P64Shared& sh, const double* v, size_t base, double theta,
                               double irho) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc = 0.0;
    for (int p = tid; p < A.N; p += P64_THREADS) {
        const int s = A.sector[p];
        if (s < 0) continue;
        P64Pieces pc;
        p64_pieces(A, base + p, pc);
        acc += fabs(p64_prox(pc, v[base + p] - sh.eta_s[s] * irho, irho, theta) - pc.w0);
    }
    acc = warp_sum(acc);
    if (lane == 0) sh.red[warp][0] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < P64_WARPS; ++w) t += sh.red[w][0];
        sh.U = t;
    }
    __syncthreads();
    const double r = sh.U;
    __syncthreads();
    return r;
}

// C = (2F)^{-1} + B' Delta^{-1} B and its Cholesky factor, in FP64 (block-collective). With the
// factor-exposure block (s = B'x split off with penalty rho) the diagonal term is (2F + rho I)^{-1}
// and G = B' Delta^{-1} B is kept beside the factor.
__device__ bool p64_factor(const P64Args& A, P64Shared& sh, double rho) {
    const bool fac = A.flo != nullptr;
    const int tid = threadIdx.x, K = A.K;
    const int npair = K * (K + 1) / 2;
    for (int q = tid; q < npair; q += P64_THREADS) {
        int r = 0, rem = q;
        while (rem > r) { rem -= r + 1; ++r; }
        const int c = rem;                                 // pair (r, c), c <= r
        double acc = 0.0;
        for (int p = 0; p < A.N; ++p)
            acc += A.B[(size_t)p * K + r] * A.B[(size_t)p * K + c] / (2.0 * A.d[p] + rho);
        if (fac) { sh.G[r][c] = acc; sh.G[c][r] = acc; }
        if (r == c) acc += fac ? 1.0 / (2.0 * A.f[r] + rho) : 1.0 / (2.0 * A.f[r]);
        sh.L[r][c] = acc;
    }
    __syncthreads();
    for (int c = 0; c < K; ++c) {
        if (tid == 0) sh.L[c][c] = sqrt(sh.L[c][c]);
        __syncthreads();
        for (int r = c + 1 + tid; r < K; r += P64_THREADS) sh.L[r][c] /= sh.L[c][c];
        __syncthreads();
        for (int r = c + 1 + tid; r < K; r += P64_THREADS)
            for (int q = c + 1; q <= r; ++q) sh.L[r][q] -= sh.L[r][c] * sh.L[q][c];
        __syncthreads();
    }
    bool ok = true;
    for (int c = 0; c < K; ++c) ok = ok && sh.L[c][c] > 0.0 && isfinite(sh.L[c][c]);
    return ok;
}

__global__ void __launch_bounds__(P64_THREADS) k_admm64(P64Args A) {
    extern __shared__ unsigned char smem_raw[];
    P64Shared& sh = *reinterpret_cast<P64Shared*>(smem_raw);
    const int a = blockIdx.x;
    if (A.skip && A.skip[a]) return;
    if (A.resume && !A.active[a]) return;         // a second pass runs the accounts sent back only
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = A.N, K = A.K, S = A.S;
    const size_t base = (size_t)a * A.Npad;
    double* z = A.z;
    double* y = A.y;
    double* X = A.X;          // X, then v, of this account
    if (!A.resume) {
        for (int p = tid; p < N; p += P64_THREADS) {
            const size_t e = base + p;
            z[e] = fmin(fmax(A.w0[e], A.lo[e]), A.up[e]);
            y[e] = 0.0;
        }
        if (tid == 0) { sh.rho = A.rho0; sh.nu = 0.0; sh.theta = 0.0; }
    } else if (tid == 0) {
        sh.rho = A.rho_state[a]; sh.nu = 0.0; sh.theta = A.theta_state[a];
    }
    const bool fac = A.flo != nullptr;
    if (fac && !A.resume)
        for (int k = tid; k < K; k += P64_THREADS) { sh.s[k] = 0.0; sh.ys[k] = 0.0; }
    if (fac && A.resume)
        for (int k = tid; k < K; k += P64_THREADS) { sh.s[k] = A.s_state[a * K + k]; sh.ys[k] = A.ys_state[a * K + k]; }
    __syncthreads();
    double rho = sh.rho;
    bool ok = p64_factor(A, sh, rho);
    const double alpha = A.alpha;
    int it = A.resume ? A.iters[a] : 0;
    int status = 0;
    double theta = sh.theta;
    const bool has_cap = isfinite(A.tau[a]);
    while (ok) {
        const double irho = 1.0 / rho;
        // ---- X and P = B' X (factor-group layout: thread (g, k) sums over entries p = g mod G)
        for (int p = tid; p < N; p += P64_THREADS) {
            const size_t e = base + p;
            X[e] = (A.mu[p] + rho * z[e] - y[e]) / (2.0 * A.d[p] + rho);
        }
        __syncthreads();
        {
            constexpr int G = P64_THREADS / 64;
            const int g = tid / 64, k = tid % 64;
            if (k < K) {
                double acc = 0.0;
                for (int p = g; p < N; p += G) acc += A.B[(size_t)p * K + k] * X[base + p];
                sh.part[g][k] = acc;
            }
            __syncthreads();
            if (tid < K) {
                double s = 0.0;
                for (int q = 0; q < G; ++q) s += sh.part[q][tid];
                sh.P[tid] = s;
            }
            __syncthreads();
        }
        // ---- Q = C^{-1} P (one thread: K^2 work). With the factor-exposure block the right side
        // gains B tv, tv = rho s - ys: Q' = C^{-1} (P0 + G tv) - tv, and B'x = P0 - G Q'
        if (fac) {
            for (int k = tid; k < K; k += P64_THREADS) { sh.tv[k] = rho * sh.s[k] - sh.ys[k]; sh.P0[k] = sh.P[k]; }
            __syncthreads();
            for (int k = tid; k < K; k += P64_THREADS) {
                double g = 0.0;
                for (int j = 0; j < K; ++j) g += sh.G[k][j] * sh.tv[j];
                sh.P[k] = sh.P0[k] + g;
            }
            __syncthreads();
        }
        if (tid == 0) {
            for (int r = 0; r < K; ++r) {
                double s = sh.P[r];
                for (int q = 0; q < r; ++q) s -= sh.L[r][q] * sh.Q[q];
                sh.Q[r] = s / sh.L[r][r];
            }
            for (int r = K - 1; r >= 0; --r) {
                double s = sh.Q[r];
                for (int q = r + 1; q < K; ++q) s -= sh.L[q][r] * sh.Q[q];
                sh.Q[r] = s / sh.L[r][r];
            }
            if (fac) for (int r = 0; r < K; ++r) sh.Q[r] -= sh.tv[r];
        }
        __syncthreads();
        double rps = 0.0, rds = 0.0;
        if (fac) {
            // the block's update: relaxed B'x, s = clip(., lo, hi), the dual step, residuals
            for (int k = tid; k < K; k += P64_THREADS) {
                double g = 0.0;
                for (int j = 0; j < K; ++j) g += sh.G[k][j] * sh.Q[j];
                const double bx = sh.P0[k] - g;
                const double xh = alpha * bx + (1.0 - alpha) * sh.s[k];
                const double sn = fmin(fmax(xh + sh.ys[k] * irho, A.flo[a * K + k]), A.fhi[a * K + k]);
                rps = fmax(rps, fabs(xh - sn));
                rds = fmax(rds, rho * fabs(sn - sh.s[k]));
                sh.ys[k] += rho * (xh - sn);
                sh.tv[k] = sn;                    // staged: s is read by other threads above
            }
            __syncthreads();
            for (int k = tid; k < K; k += P64_THREADS) sh.s[k] = sh.tv[k];
        }
        // ---- x, the relaxation and v (v overwrites X); bracket of the projection's multipliers
        double ea = INFINITY, eb = -INFINITY;
        for (int p = tid; p < N; p += P64_THREADS) {
            const size_t e = base + p;
            double bq = 0.0;
            for (int k = 0; k < K; ++k) bq += A.B[(size_t)p * K + k] * sh.Q[k];
            const double x = X[e] - bq / (2.0 * A.d[p] + rho);
            const double v = alpha * x + (1.0 - alpha) * z[e] + y[e] * irho;
            X[e] = v;
            P64Pieces pc;
            p64_pieces(A, e, pc);
            double smin = 0.0, smax = 0.0;
            for (int j = 0; j + 1 < pc.nb; ++j) {
                smin = fmin(smin, pc.sl[j]);
                smax = fmax(smax, pc.sl[j]);
            }
            // every z_i is at its upper end for eta <= ea and at its lower end for eta >= eb
            ea = fmin(ea, rho * (v - pc.bp[pc.nb - 1]) - smax);
            eb = fmax(eb, rho * (v - pc.bp[0]) - smin);
        }
        for (int o = 16; o > 0; o >>= 1) {
            ea = fmin(ea, __shfl_xor_sync(0xffffffffu, ea, o));
            eb = fmax(eb, __shfl_xor_sync(0xffffffffu, eb, o));
        }
        if (lane == 0) { sh.red[warp][0] = ea; sh.red[warp][1] = eb; }
        __syncthreads();
        if (tid == 0) {
            double a0 = INFINITY, b0 = -INFINITY;
            for (int w = 0; w < P64_WARPS; ++w) { a0 = fmin(a0, sh.red[w][0]); b0 = fmax(b0, sh.red[w][1]); }
            sh.red[0][2] = a0; sh.red[0][3] = b0;
        }
        __syncthreads();
        const double cap_pad = has_cap ? 1.0 : 0.0;
        double eta_a = sh.red[0][2] - 1.0, eta_b = sh.red[0][3] + 1.0;
        __syncthreads();
        // ---- projection: the cap multiplier theta by an outer root when the cap binds
        double th = 0.0;
        if (has_cap) {
            const double tau = A.tau[a];
            p64_inner(A, sh, X, base, a, 0.0, eta_a, eta_b, irho);
            const double u0 = p64_turnover(A, sh, X, base, 0.0, irho);
            if (u0 > tau) {
                // theta enlarges the slopes by at most theta: widen the eta bracket with it
                double hi = fmax(2.0 * theta, 1e-3);
                double uh = u0;
                for (int dbl = 0; dbl < 60; ++dbl) {
                    p64_inner(A, sh, X, base, a, hi, eta_a - hi - cap_pad, eta_b + hi + cap_pad, irho);
                    uh = p64_turnover(A, sh, X, base, hi, irho);
                    if (uh <= tau) break;
                    hi *= 2.0;
                }
                auto g = [&](double t) {
                    p64_inner(A, sh, X, base, a, t, eta_a - t - cap_pad, eta_b + t + cap_pad, irho);
                    return p64_turnover(A, sh, X, base, t, irho) - tau;
                };
                th = p64_root(0.0, u0 - tau, hi, uh - tau, g);
                th = fmax(th, 0.0);
            }
            theta = th;
        }
        p64_inner(A, sh, X, base, a, th, eta_a - th - cap_pad, eta_b + th + cap_pad, irho);
        // ---- z+, y+ and the residuals
        double rp = 0.0, rd = 0.0, nx = 0.0, nz = 0.0, ny = 0.0;
        int bad = 0;
        for (int p = tid; p < N; p += P64_THREADS) {
            const size_t e = base + p;
            const int s = A.sector[p];
            P64Pieces pc;
            p64_pieces(A, e, pc);
            const double v = X[e];
            const double zn = p64_prox(pc, v - sh.eta_s[s] * irho, irho, th);
            const double yn = rho * (v - zn);
            const double xh = v - y[e] * irho;
            rp = fmax(rp, fabs(xh - zn));
            rd = fmax(rd, rho * fabs(zn - z[e]));
            nx = fmax(nx, fabs(xh));
            nz = fmax(nz, fabs(zn));
            ny = fmax(ny, fabs(yn));
            bad |= !(isfinite(zn) && isfinite(yn));
            z[e] = zn;
            y[e] = yn;
        }
        rp = fmax(rp, rps);
        rd = fmax(rd, rds);
        rp = warp_max(rp); rd = warp_max(rd); nx = warp_max(nx); nz = warp_max(nz); ny = warp_max(ny);
        bad = warp_sum(bad);
        if (lane == 0) {
            sh.red[warp][0] = rp; sh.red[warp][1] = rd; sh.red[warp][2] = nx;
            sh.red[warp][3] = nz; sh.red[warp][4] = ny; sh.red[warp][5] = bad;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < P64_WARPS; ++w) {
                sh.red[0][0] = fmax(sh.red[0][0], sh.red[w][0]); sh.red[0][1] = fmax(sh.red[0][1], sh.red[w][1]);
                sh.red[0][2] = fmax(sh.red[0][2], sh.red[w][2]); sh.red[0][3] = fmax(sh.red[0][3], sh.red[w][3]);
                sh.red[0][4] = fmax(sh.red[0][4], sh.red[w][4]); sh.red[0][5] += sh.red[w][5];
            }
            ++it;
            const double rp_ = sh.red[0][0], rd_ = sh.red[0][1];
            int go = 1;
            double newrho = rho;
            if (sh.red[0][5] > 0.0 || !isfinite(rp_) || !isfinite(rd_)) { status = PRISM_NUMERICAL_FAILURE; go = 0; }
            else if (it >= A.min_iter && rp_ <= A.eps && rd_ <= A.eps) go = 0;
            else if (it >= A.max_iter) { status = PRISM_TIMEOUT; go = 0; }
            else if (it % A.adapt_every == 0) {
                const double pr = rp_ / fmax(fmax(sh.red[0][2], sh.red[0][3]), 1e-300);
                const double du = rd_ / fmax(sh.red[0][4], 1e-300);
                const double ratio = sqrt(pr / fmax(du, 1e-300));
                if (ratio > 2.0 || ratio < 0.5) newrho = rho * fmin(fmax(ratio, 0.1), 10.0);
                newrho = fmin(fmax(newrho, 1e-6), 1e6);
            }
            sh.go = go;
            sh.rho = newrho;
        }
        __syncthreads();
        if (!sh.go) break;
        if (sh.rho != rho) {
            rho = sh.rho;
            ok = p64_factor(A, sh, rho);
            if (!ok && tid == 0) status = PRISM_NUMERICAL_FAILURE;
        }
    }
    if (!ok) status = PRISM_NUMERICAL_FAILURE;
    // ---- what the polish reads: z (FP32 copy), the multipliers as FP32 signals
    for (int p = tid; p < A.Npad; p += P64_THREADS) A.zf[base + p] = p < N ? float(z[base + p]) : 0.f;
    for (int s = tid; s < S; s += P64_THREADS) {
        const double es = sh.eta_s[s], nu = sh.nu;
        // a sector held at its upper edge has eta_s > nu, at its lower edge eta_s < nu
        A.eta_hi_f[a * S + s] = es > nu ? float(es) : -FLT_MAX;
        A.eta_lo_f[a * S + s] = es < nu ? float(es) : FLT_MAX;
    }
    if (fac)
        for (int k = tid; k < K; k += P64_THREADS) {
            const double lo = A.flo[a * K + k], hi = A.fhi[a * K + k], sk = sh.s[k];
            A.sflag[a * K + k] = (sk >= hi) ? 1 : ((sk <= lo) ? -1 : 0);
            A.s_state[a * K + k] = sk;
            A.ys_state[a * K + k] = sh.ys[k];
        }
    if (tid == 0) {
        A.nu_f[a] = float(sh.nu);
        A.theta_f[a] = float(theta);
        A.theta_state[a] = theta;
        A.rho_state[a] = rho;
        A.iters[a] = it;
        A.active[a] = 0;
        if (status) A.status[a] = status;
    }
}

size_t p64_smem_bytes() { return sizeof(P64Shared); }

void launch_admm64(const P64Args& A, cudaStream_t st) {
    cudaFuncSetAttribute(k_admm64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(P64Shared));
    k_admm64<<<A.M, P64_THREADS, sizeof(P64Shared), st>>>(A);
}

}  // namespace prism
