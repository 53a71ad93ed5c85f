// block_admm.cu -- the ADMM iterations of one account in one thread block, all of them in one
// launch: the same splitting as the batched kernels (x = z with f(x) = x' Sigma x - mu' x and
// g(z) = sum_i phi_i(z_i) + indicator of the Eq. 1 feasible set, Sec. 4.2), for
//  - PRISM_PLAIN_FP64: FP64 over the dense layout (every position of the universe);
//  - ragged books in the batched modes: FP32 over a packed layout, the account's own names only,
//    staged in shared memory when they fit, with the Woodbury capacitance of the account's own
//    rows of B (C_a = (2F)^{-1} + B_a' Delta^{-1} B_a) instead of the universe's. Blocks are
//    persistent: each takes the next account from a work counter, largest accounts first.
//
// One iteration, penalty rho, relaxation alpha (Delta = diag(2 d + rho)):
//   X  = Delta^{-1} (mu + rho z - y)
//   Q  = C^{-1} B' X,            C = (2F)^{-1} + B' Delta^{-1} B      (Woodbury, K x K)
//   x  = X - Delta^{-1} B Q       = (2 Sigma + rho I)^{-1} (mu + rho z - y)
//   v  = alpha x + (1 - alpha) z + y / rho
//   z+ = argmin_{z in Z} sum_i phi_i(z_i) + rho/2 ||z - v||^2,   y+ = rho (v - z+)
// C is formed and Cholesky-factored in shared memory whenever rho changes. The projection relaxes
// the budget (nu), the sector bands (lambda_s) and the turnover cap (theta): z_i = prox of
// (phi_i + theta |. - w0_i|)/rho on [l_i, u_i] at v_i - (nu + lambda_s(i))/rho; each sector sum
// S_s(eta) is nonincreasing and piecewise linear in eta, the budget reads
// sum_s clamp(S_s(nu), lo_s, hi_s) = 1, a sector held at an edge has its own eta_s = nu + lambda_s
// with S_s(eta_s) at that edge, and theta solves ||z(theta) - w0||_1 = tau when the cap binds.
// Every scalar root is bracketed and found by alternating secant and bisection steps (exact
// once the bracket lies on one linear piece). Factor-exposure bounds (Eq. 1 rows B'w in
// [lo, hi]) are a second block s = B'x with the same penalty: the x-update's right side gains
// B (rho s - ys), so Q' = C^{-1} (P0 + G tv) - tv with tv = rho s - ys, G = B' Delta^{-1} B, and
// C's diagonal term becomes (2F + rho I)^{-1}. The result feeds the FP64 polish.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "block_admm.h"
#include "common.cuh"

namespace prism {

constexpr int BLK_ROOT_IT = 200;          // evaluations per scalar root (bisection alone needs ~110)

template <typename T> struct BlkCfg;
// EPS: relative width at which a root's bracket is closed; FTOL: a function value (a budget,
// band or turnover residual, all of order one) accepted as zero: the roots are solved to about the
// rounding of the sums themselves (the polish settles the final point in FP64)
template <> struct BlkCfg<double> {
    static constexpr int THREADS = 256;
    static constexpr double EPS = 1e-15, FTOL = 1e-13;
};
template <> struct BlkCfg<float> {
    static constexpr int THREADS = 512;
    static constexpr float EPS = 4e-7f, FTOL = 4e-6f;
};

template <typename T>
struct BlkShared {
    T L[KMAX][KMAX + 1];                  // Cholesky factor of C (lower)
    T G[KMAX][KMAX + 1];                  // B' Delta^{-1} B (factor-exposure block only)
    T P[KMAX], Q[KMAX];
    T part[BlkCfg<T>::THREADS / 32][KMAX];  // per-warp partial sums of B'X
    T Bc[32][KMAX + 1];                   // a chunk of the account's rows of B (capacitance build)
    T wdi[32];                            // their 1 / (2 d + rho)
    T s[KMAX], ys[KMAX], tv[KMAX], P0[KMAX];   // factor-exposure block: s = B'x and its dual
    T ssum[SMAX];                         // sector sums at the current evaluation point
    T eta_s[SMAX];                        // per-sector multiplier point (nu + lambda_s)
    T red[BlkCfg<T>::THREADS / 32][6];
    T nu, dnu, theta, rho, Tv, U;         // dnu: the last change of nu (first step of its search)
    int sec[SMAX + 1];                    // the account's sector ranges (entry indices)
    int go, acct;
};

__device__ __forceinline__ unsigned long long blk_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One account's entries: index q = 0 .. n-1 in increasing position order; pos[q] its position
// (null: q is the position), the per-entry arrays indexed by q.
template <typename T>
struct View {
    int n;
    const int* pos;
    const T *w0, *lo, *up, *c;
    const int* pw;
    T *z, *y, *X;
    __device__ int p(int q) const { return pos ? pos[q] : q; }
};

// B_p . Q for one row: the padded FP32 copy in 16-byte loads, all issued together (they are
// independent: the latency of the rows, which come from L2, overlaps), else element by element.
template <typename T>
__device__ __forceinline__ T brow_dot(const BlkArgs<T>& A, int p, const T* Q) {
    T acc = 0;
#pragma unroll 8
    for (int k = 0; k < A.K; ++k) acc += A.B[(size_t)p * A.K + k] * Q[k];
    return acc;
}
template <>
__device__ __forceinline__ float brow_dot<float>(const BlkArgs<float>& A, int p, const float* Q) {
    if (!A.Bp) {
        float acc = 0.f;
#pragma unroll 8
        for (int k = 0; k < A.K; ++k) acc += A.B[(size_t)p * A.K + k] * Q[k];
        return acc;
    }
    const float4* r = reinterpret_cast<const float4*>(A.Bp + (size_t)p * KMAX);
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int h = 0; h < KMAX / 32; ++h) {        // two halves of 32 factors: 8 loads in flight each
        if (32 * h >= A.K) break;
        float4 b[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (32 * h + 4 * c < A.K) b[c] = __ldg(r + 8 * h + c);
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (32 * h + 4 * c < A.K) {          // padding factors are zero in the copy and in Q
                const float* q = Q + 32 * h + 4 * c;
                a0 = fmaf(b[c].x, q[0], a0);
                a1 = fmaf(b[c].y, q[1], a1);
                a0 = fmaf(b[c].z, q[2], a0);
                a1 = fmaf(b[c].w, q[3], a1);
            }
    }
    return a0 + a1;
}

// Breakpoints and slopes of phi_i restricted to [l_i, u_i].
template <typename T>
struct Pcs {
    T bp[MAXBP];
    T sl[MAXBP - 1];
    int nb;
    T w0;
};

template <typename T>
__device__ __forceinline__ void pieces(const BlkArgs<T>& A, const View<T>& V, int q, Pcs<T>& pc) {
    const T w0 = V.w0[q], lo = V.lo[q], up = V.up[q], c = V.c[q];
    pc.w0 = w0;
    const int pw = V.pw ? V.pw[q] : -1;
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
template <typename T>
__device__ __forceinline__ T slope(const Pcs<T>& pc, int j, T theta) {
    const T mid = T(0.5) * (pc.bp[j] + pc.bp[j + 1]);
    const T sg = mid > pc.w0 ? T(1) : (mid < pc.w0 ? T(-1) : T(0));
    return pc.sl[j] + theta * sg;
}

// argmin_z phi(z) + theta |z - w0| + rho/2 (z - t)^2 on [bp_0, bp_last]: the first segment j
// whose unconstrained minimiser t - s_j/rho falls left of its right end holds the answer,
// either inside it or at its left end (a kink or the lower bound).
template <typename T>
__device__ __forceinline__ T prox1(const Pcs<T>& pc, T t, T irho, T theta) {
    if (pc.nb == 1) return pc.bp[0];
    for (int j = 0; j + 1 < pc.nb; ++j) {
        const T zc = t - slope(pc, j, theta) * irho;
        if (zc < pc.bp[j + 1]) return zc > pc.bp[j] ? zc : pc.bp[j];
    }
    return pc.bp[pc.nb - 1];
}

// Sum of z over the entries [q0, q1) at eta (one warp; lane-strided).
template <typename T>
__device__ __forceinline__ T range_sum(const BlkArgs<T>& A, const View<T>& V, int q0, int q1, T eta, T irho,
                                       T theta, int lane) {
    T acc = 0;
    for (int q = q0 + lane; q < q1; q += 32) {
        Pcs<T> pc;
        pieces(A, V, q, pc);
        acc += prox1(pc, V.X[q] - eta * irho, irho, theta);
    }
    return warp_sum(acc);
}

// Root of a nonincreasing function g on [a, b] with g(a) >= 0 >= g(b): alternate secant and
// bisection steps. Runs identically in every thread that calls it (eval may be collective).
template <typename T, class Eval>
__device__ T root(T a, T ga, T b, T gb, Eval&& eval) {
    for (int it = 0; it < BLK_ROOT_IT; ++it) {
        if (fabs(ga) <= BlkCfg<T>::FTOL) return a;
        if (fabs(gb) <= BlkCfg<T>::FTOL) return b;
        const T w = b - a;
        if (!(w > BlkCfg<T>::EPS * fmax(T(1), fmax(fabs(a), fabs(b))))) break;
        T m = (it & 1) ? T(0.5) * (a + b) : a + w * ga / (ga - gb);
        if (!(m > a && m < b)) m = T(0.5) * (a + b);
        const T gm = eval(m);
        if (fabs(gm) <= BlkCfg<T>::FTOL) return m;
        if (gm > T(0)) { a = m; ga = gm; }
        else { b = m; gb = gm; }
    }
    return (ga < -gb) ? a : b;
}

// The same root, searched from a warm start x0 in [lo, hi]: steps outward from x0 (growing four
// times per step) until the sign changes, then root() on that bracket. The function at lo and
// hi is evaluated only if the search reaches them.
template <typename T, class Eval>
__device__ T root_warm(T lo, T hi, T x0, T step, Eval&& eval) {
    x0 = fmin(fmax(x0, lo), hi);
    const T g0 = eval(x0);
    if (fabs(g0) <= BlkCfg<T>::FTOL) return x0;
    T a = x0, ga = g0;
    for (int k = 0; k < 80; ++k, step *= T(4)) {
        if (g0 > T(0)) {
            const T b = fmin(a + step, hi);
            const T gb = eval(b);
            if (gb <= T(0) || !(b < hi)) return root(a, ga, b, gb, eval);
            a = b; ga = gb;
        } else {
            const T b = fmax(a - step, lo);
            const T gb = eval(b);
            if (gb >= T(0) || !(b > lo)) return root(b, gb, a, ga, eval);
            a = b; ga = gb;
        }
    }
    return a;
}

// The projection of v (in V.X) onto Z for a given theta: the budget multiplier (sh.nu) and
// each sector's point eta_s (sh.eta_s). The budget's root is searched from the last call's nu,
// each sector's from its last point (warm starts: they move little between iterations), with a
// first step of four times the last move of nu. Block-collective.
template <typename T>
__device__ void inner(const BlkArgs<T>& A, BlkShared<T>& sh, const View<T>& V, int a, T theta, T eta_a, T eta_b,
                      T irho) {
    constexpr int NW = BlkCfg<T>::THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = A.S;
    auto Tf = [&](T eta) -> T {
        if (A.dbg && tid == 0) atomicAdd(A.dbg + 7, 1ull);
        for (int s = warp; s < S; s += NW) {
            const T sm = range_sum(A, V, sh.sec[s], sh.sec[s + 1], eta, irho, theta, lane);
            if (lane == 0) sh.ssum[s] = fmin(fmax(sm, A.band_lo[a * S + s]), A.band_hi[a * S + s]);
        }
        __syncthreads();
        if (tid == 0) {
            T t = 0;
            for (int s = 0; s < S; ++s) t += sh.ssum[s];
            sh.Tv = t - T(1);
        }
        __syncthreads();
        const T r = sh.Tv;
        __syncthreads();
        return r;
    };
    const T nu_prev = sh.nu;
    // (at least 1e-4 of the multiplier's scale: a step at the rounding level would take many
    // growth steps to reach a move of ordinary size)
    const T step = fmax(T(4) * sh.dnu, T(1e-4) * fmax(T(1), fabs(nu_prev)));
    const T nu = root_warm(eta_a, eta_b, nu_prev, step, Tf);
    // each sector held at an edge gets its own point (warp-local roots, no block barriers)
    for (int s = warp; s < S; s += NW) {
        const T lo = A.band_lo[a * S + s], hi = A.band_hi[a * S + s];
        const int q0 = sh.sec[s], q1 = sh.sec[s + 1];
        const T s0 = range_sum(A, V, q0, q1, nu, irho, theta, lane);
        const T prev = sh.eta_s[s];
        T es = nu;
        if (s0 > hi) {
            auto g = [&](T eta) { return range_sum(A, V, q0, q1, eta, irho, theta, lane) - hi; };
            es = root_warm(nu, eta_b, prev > nu ? prev : nu, step, g);
        } else if (s0 < lo) {
            auto g = [&](T eta) { return range_sum(A, V, q0, q1, eta, irho, theta, lane) - lo; };
            es = root_warm(eta_a, nu, prev < nu ? prev : nu, step, g);
        }
        __syncwarp();
        if (lane == 0) sh.eta_s[s] = es;
    }
    __syncthreads();
    if (tid == 0) { sh.dnu = fabs(nu - nu_prev); sh.nu = nu; }
    __syncthreads();
}

// ||z(theta) - w0||_1 of the projection just computed (block-collective).
template <typename T>
__device__ T turnover(const BlkArgs<T>& A, BlkShared<T>& sh, const View<T>& V, T theta, T irho) {
    constexpr int NW = BlkCfg<T>::THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T acc = 0;
    for (int s = warp; s < A.S; s += NW)
        for (int q = sh.sec[s] + lane; q < sh.sec[s + 1]; q += 32) {
            Pcs<T> pc;
            pieces(A, V, q, pc);
            acc += fabs(prox1(pc, V.X[q] - sh.eta_s[s] * irho, irho, theta) - pc.w0);
        }
    acc = warp_sum(acc);
    if (lane == 0) sh.red[warp][0] = acc;
    __syncthreads();
    if (tid == 0) {
        T t = 0;
        for (int w = 0; w < NW; ++w) t += sh.red[w][0];
        sh.U = t;
    }
    __syncthreads();
    const T r = sh.U;
    __syncthreads();
    return r;
}

// C = (2F)^{-1} + B_a' Delta^{-1} B_a over the account's entries, and its Cholesky factor
// (block-collective). With the factor-exposure block the diagonal term is (2F + rho I)^{-1}
// and G = B_a' Delta^{-1} B_a is kept beside the factor.
template <typename T>
__device__ bool factor(const BlkArgs<T>& A, BlkShared<T>& sh, const View<T>& V, T rho) {
    constexpr int NT = BlkCfg<T>::THREADS;
    constexpr int PPT = (KMAX * (KMAX + 1) / 2 + NT - 1) / NT;   // pairs per thread at most
    const bool fac = A.flo != nullptr;
    const int tid = threadIdx.x, K = A.K;
    const int npair = K * (K + 1) / 2;
    // this thread's pairs (r, c), c <= r, and their sums over the account's rows, which are staged
    // in shared memory 32 at a time
    int pr[PPT], pc[PPT];
    T acc[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int q = tid + j * NT;
        int r = 0, rem = q < npair ? q : 0;
        while (rem > r) { rem -= r + 1; ++r; }
        pr[j] = r; pc[j] = rem; acc[j] = 0;
    }
    for (int e0 = 0; e0 < V.n; e0 += 32) {
        const int ne = min(32, V.n - e0);
        for (int t = tid; t < ne * K; t += NT) {
            const int e = t / K, k = t % K, p = V.p(e0 + e);
            sh.Bc[e][k] = A.B[(size_t)p * K + k];
        }
        for (int e = tid; e < ne; e += NT) sh.wdi[e] = T(1) / (T(2) * A.d[V.p(e0 + e)] + rho);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PPT; ++j)
            if (tid + j * NT < npair)
                for (int e = 0; e < ne; ++e) acc[j] += sh.Bc[e][pr[j]] * sh.Bc[e][pc[j]] * sh.wdi[e];
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        if (tid + j * NT >= npair) continue;
        const int r = pr[j], c = pc[j];
        T v = acc[j];
        if (fac) { sh.G[r][c] = v; sh.G[c][r] = v; }
        if (r == c) v += fac ? T(1) / (T(2) * A.f[r] + rho) : T(1) / (T(2) * A.f[r]);
        sh.L[r][c] = v;
    }
    __syncthreads();
    for (int c = 0; c < K; ++c) {
        if (tid == 0) sh.L[c][c] = sqrt(sh.L[c][c]);
        __syncthreads();
        for (int r = c + 1 + tid; r < K; r += NT) sh.L[r][c] /= sh.L[c][c];
        __syncthreads();
        for (int r = c + 1 + tid; r < K; r += NT)
            for (int q = c + 1; q <= r; ++q) sh.L[r][q] -= sh.L[r][c] * sh.L[q][c];
        __syncthreads();
    }
    bool ok = true;
    for (int c = 0; c < K; ++c) ok = ok && sh.L[c][c] > T(0) && isfinite(sh.L[c][c]);
    return ok;
}

// All iterations of account a (block-collective).
template <typename T>
__device__ void solve_account(const BlkArgs<T>& A, BlkShared<T>& sh, const View<T>& V, int a) {
    constexpr int NT = BlkCfg<T>::THREADS, NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = A.K, S = A.S, n = V.n;
    const bool fac = A.flo != nullptr;
    if (!A.resume) {
        for (int q = tid; q < n; q += NT) {
            V.z[q] = fmin(fmax(V.w0[q], V.lo[q]), V.up[q]);
            V.y[q] = T(0);
        }
        if (tid == 0) { sh.rho = T(A.rho0); sh.nu = T(0); sh.dnu = T(1); sh.theta = T(0); }
        if (fac) for (int k = tid; k < K; k += NT) { sh.s[k] = T(0); sh.ys[k] = T(0); }
    } else {
        if (tid == 0) { sh.rho = A.rho_state[a]; sh.nu = T(0); sh.dnu = T(1); sh.theta = A.theta_state[a]; }
        if (fac)
            for (int k = tid; k < K; k += NT) { sh.s[k] = A.s_state[a * K + k]; sh.ys[k] = A.ys_state[a * K + k]; }
    }
    for (int s = tid; s < S; s += NT) sh.eta_s[s] = T(0);
    for (int k = tid; k < KMAX; k += NT) sh.Q[k] = T(0);   // factors beyond K stay zero (row dot products)
    __syncthreads();
    T rho = sh.rho;
    bool ok = factor(A, sh, V, rho);
    const T alpha = T(A.alpha);
    int it = A.resume ? A.iters[a] : 0;
    int status = 0;
    T theta = sh.theta;
    const bool has_cap = isfinite(A.tau[a]);
    unsigned long long tmark = 0;
    auto mark = [&](int slot) {
        if (A.dbg && tid == 0) {
            const unsigned long long t = blk_clock();
            if (slot >= 0) atomicAdd(A.dbg + slot, t - tmark);
            tmark = t;
        }
    };
    mark(-1);
    while (ok) {
        const T irho = T(1) / rho;
        // ---- X and P = B' X
#pragma unroll 4
        for (int q = tid; q < n; q += NT) {
            const int p = V.p(q);
            V.X[q] = (A.mu[p] + rho * V.z[q] - V.y[q]) / (T(2) * A.d[p] + rho);
        }
        __syncthreads();
        {
            // warp w takes entries w, w + NW, ...; lane l factors l and l + 32 of each row (the
            // row's loads coalesced), eight rows in flight per step
            constexpr int RU = 8;
            const T* Bb = A.Bp ? A.Bp : A.B;
            const int ld = A.Bp ? KMAX : K;
            T a0 = 0, a1 = 0;
            for (int q0 = warp; q0 < n; q0 += RU * NW) {
                T b0[RU], b1[RU], xv[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int q = q0 + u * NW;
                    const bool in = q < n;
                    const size_t row = in ? (size_t)V.p(q) * ld : 0;
                    b0[u] = (in && lane < K) ? Bb[row + lane] : T(0);
                    b1[u] = (in && lane + 32 < K) ? Bb[row + lane + 32] : T(0);
                    xv[u] = in ? V.X[q] : T(0);
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) { a0 += b0[u] * xv[u]; a1 += b1[u] * xv[u]; }
            }
            sh.part[warp][lane] = a0;
            sh.part[warp][lane + 32] = a1;
            __syncthreads();
            if (tid < K) {
                T s = 0;
                for (int w = 0; w < NW; ++w) s += sh.part[w][tid];
                sh.P[tid] = s;
            }
            __syncthreads();
        }
        mark(0);                                     // X and B'X
        // ---- Q = C^{-1} P (one thread: K^2 work); with the factor block Q' = C^{-1}(P0 + G tv) - tv
        if (fac) {
            for (int k = tid; k < K; k += NT) { sh.tv[k] = rho * sh.s[k] - sh.ys[k]; sh.P0[k] = sh.P[k]; }
            __syncthreads();
            for (int k = tid; k < K; k += NT) {
                T g = 0;
                for (int j = 0; j < K; ++j) g += sh.G[k][j] * sh.tv[j];
                sh.P[k] = sh.P0[k] + g;
            }
            __syncthreads();
        }
        if (warp == 0) {
            // L L' Q = P by one warp, lane r holding rows r and r + 32: column-oriented
            // substitutions (each solved value broadcast, the rows below updated in parallel)
            T v0 = lane < K ? sh.P[lane] : T(0), v1 = lane + 32 < K ? sh.P[lane + 32] : T(0);
            for (int r = 0; r < K; ++r) {
                const T xr = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) / sh.L[r][r];
                if (lane == (r & 31)) { if (r < 32) v0 = xr; else v1 = xr; }
                if (lane > r && lane < K) v0 -= sh.L[lane][r] * xr;
                if (lane + 32 > r && lane + 32 < K) v1 -= sh.L[lane + 32][r] * xr;
            }
            for (int r = K - 1; r >= 0; --r) {
                const T xr = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) / sh.L[r][r];
                if (lane == (r & 31)) { if (r < 32) v0 = xr; else v1 = xr; }
                if (lane < r) v0 -= sh.L[r][lane] * xr;
                if (lane + 32 < r) v1 -= sh.L[r][lane + 32] * xr;
            }
            if (lane < K) sh.Q[lane] = fac ? v0 - sh.tv[lane] : v0;
            if (lane + 32 < K) sh.Q[lane + 32] = fac ? v1 - sh.tv[lane + 32] : v1;
        }
        __syncthreads();
        T rps = 0, rds = 0;
        if (fac) {
            // the block's update: relaxed B'x = P0 - G Q', s = clip(., lo, hi), the dual step
            for (int k = tid; k < K; k += NT) {
                T g = 0;
                for (int j = 0; j < K; ++j) g += sh.G[k][j] * sh.Q[j];
                const T bx = sh.P0[k] - g;
                const T xh = alpha * bx + (T(1) - alpha) * sh.s[k];
                const T sn = fmin(fmax(xh + sh.ys[k] * irho, A.flo[a * K + k]), A.fhi[a * K + k]);
                rps = fmax(rps, fabs(xh - sn));
                rds = fmax(rds, rho * fabs(sn - sh.s[k]));
                sh.ys[k] += rho * (xh - sn);
                sh.tv[k] = sn;                    // staged: s is read by other threads above
            }
            __syncthreads();
            for (int k = tid; k < K; k += NT) sh.s[k] = sh.tv[k];
        }
        mark(1);                                     // the small solve
        // ---- x, the relaxation and v (v overwrites X); bracket of the projection's multipliers
        T ea = T(INFINITY), eb = T(-INFINITY);
#pragma unroll 2
        for (int q = tid; q < n; q += NT) {
            const int p = V.p(q);
            const T bq = brow_dot(A, p, sh.Q);
            const T x = V.X[q] - bq / (T(2) * A.d[p] + rho);
            const T v = alpha * x + (T(1) - alpha) * V.z[q] + V.y[q] * irho;
            V.X[q] = v;
            Pcs<T> pc;
            pieces(A, V, q, pc);
            T smin = 0, smax = 0;
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
            T a0 = T(INFINITY), b0 = T(-INFINITY);
            for (int w = 0; w < NW; ++w) { a0 = fmin(a0, sh.red[w][0]); b0 = fmax(b0, sh.red[w][1]); }
            sh.red[0][2] = a0; sh.red[0][3] = b0;
        }
        __syncthreads();
        const T pad = has_cap ? T(1) : T(0);
        const T eta_a = sh.red[0][2] - T(1), eta_b = sh.red[0][3] + T(1);
        __syncthreads();
        mark(2);                                     // x-update and bracket
        // ---- projection: the cap multiplier theta by an outer root when the cap binds
        T th = 0;
        if (has_cap) {
            const T tau = A.tau[a];
            inner(A, sh, V, a, T(0), eta_a, eta_b, irho);
            const T u0 = turnover(A, sh, V, T(0), irho);
            if (u0 > tau) {
                // theta enlarges the slopes by at most theta: widen the eta bracket with it
                T hi = fmax(T(2) * theta, T(1e-3));
                T uh = u0;
                for (int dbl = 0; dbl < 60; ++dbl) {
                    inner(A, sh, V, a, hi, eta_a - hi - pad, eta_b + hi + pad, irho);
                    uh = turnover(A, sh, V, hi, irho);
                    if (uh <= tau) break;
                    hi *= T(2);
                }
                auto g = [&](T t) {
                    inner(A, sh, V, a, t, eta_a - t - pad, eta_b + t + pad, irho);
                    return turnover(A, sh, V, t, irho) - tau;
                };
                th = root(T(0), u0 - tau, hi, uh - tau, g);
                th = fmax(th, T(0));
            }
            theta = th;
        }
        inner(A, sh, V, a, th, eta_a - th - pad, eta_b + th + pad, irho);
        mark(3);                                     // the projection's roots
        // ---- z+, y+ and the residuals
        T rp = 0, rd = 0, nx = 0, nz = 0, ny = 0;
        int bad = 0;
        for (int s = warp; s < S; s += NW)
            for (int q = sh.sec[s] + lane; q < sh.sec[s + 1]; q += 32) {
                Pcs<T> pc;
                pieces(A, V, q, pc);
                const T v = V.X[q];
                const T zn = prox1(pc, v - sh.eta_s[s] * irho, irho, th);
                const T yn = rho * (v - zn);
                const T xh = v - V.y[q] * irho;
                rp = fmax(rp, fabs(xh - zn));
                rd = fmax(rd, rho * fabs(zn - V.z[q]));
                nx = fmax(nx, fabs(xh));
                nz = fmax(nz, fabs(zn));
                ny = fmax(ny, fabs(yn));
                bad |= !(isfinite(zn) && isfinite(yn));
                V.z[q] = zn;
                V.y[q] = yn;
            }
        rp = fmax(rp, rps);
        rd = fmax(rd, rds);
        rp = warp_max(rp); rd = warp_max(rd); nx = warp_max(nx); nz = warp_max(nz); ny = warp_max(ny);
        bad = warp_sum(bad);
        if (lane == 0) {
            sh.red[warp][0] = rp; sh.red[warp][1] = rd; sh.red[warp][2] = nx;
            sh.red[warp][3] = nz; sh.red[warp][4] = ny; sh.red[warp][5] = T(bad);
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < NW; ++w) {
                sh.red[0][0] = fmax(sh.red[0][0], sh.red[w][0]); sh.red[0][1] = fmax(sh.red[0][1], sh.red[w][1]);
                sh.red[0][2] = fmax(sh.red[0][2], sh.red[w][2]); sh.red[0][3] = fmax(sh.red[0][3], sh.red[w][3]);
                sh.red[0][4] = fmax(sh.red[0][4], sh.red[w][4]); sh.red[0][5] += sh.red[w][5];
            }
            ++it;
            const T rp_ = sh.red[0][0], rd_ = sh.red[0][1];
            int go = 1;
            T newrho = rho;
            if (sh.red[0][5] > T(0) || !isfinite(rp_) || !isfinite(rd_)) { status = PRISM_NUMERICAL_FAILURE; go = 0; }
            else if (it >= A.min_iter && rp_ <= T(A.eps) && rd_ <= T(A.eps)) go = 0;
            else if (it >= A.max_iter) { status = PRISM_TIMEOUT; go = 0; }
            else if (it % A.adapt_every == 0) {
                const T tiny = BlkCfg<T>::EPS * T(1e-20);
                const T pr = rp_ / fmax(fmax(sh.red[0][2], sh.red[0][3]), tiny);
                const T du = rd_ / fmax(sh.red[0][4], tiny);
                const T ratio = sqrt(pr / fmax(du, tiny));
                if (ratio > T(2) || ratio < T(0.5)) newrho = rho * fmin(fmax(ratio, T(0.1)), T(10));
                newrho = fmin(fmax(newrho, T(1e-6)), T(1e6));
            }
            sh.go = go;
            sh.rho = newrho;
        }
        __syncthreads();
        mark(4);                                     // z, y, residuals and control
        if (A.dbg && tid == 0) atomicAdd(A.dbg + 6, 1ull);
        if (!sh.go) break;
        if (sh.rho != rho) {
            rho = sh.rho;
            ok = factor(A, sh, V, rho);
            if (!ok && tid == 0) status = PRISM_NUMERICAL_FAILURE;
            mark(5);                                 // capacitance at a new penalty
        }
    }
    if (!ok) status = PRISM_NUMERICAL_FAILURE;
    // ---- what the polish reads: z (FP32, dense layout), the multipliers as FP32 signals
    const size_t dbase = (size_t)a * A.Npad;
    for (int q = tid; q < n; q += NT) A.zf[dbase + V.p(q)] = float(V.z[q]);
    for (int s = tid; s < S; s += NT) {
        const T es = sh.eta_s[s], nu = sh.nu;
        // a sector held at its upper edge has eta_s > nu, at its lower edge eta_s < nu
        A.eta_hi_f[a * S + s] = es > nu ? float(es) : -FLT_MAX;
        A.eta_lo_f[a * S + s] = es < nu ? float(es) : FLT_MAX;
    }
    if (fac)
        for (int k = tid; k < K; k += NT) {
            const T lo = A.flo[a * K + k], hi = A.fhi[a * K + k], sk = sh.s[k];
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
    __syncthreads();
}

// Persistent blocks: each takes the next account from the work counter (in A.order when given).
template <typename T>
__global__ void __launch_bounds__(BlkCfg<T>::THREADS, 1) k_block_admm(BlkArgs<T> A) {
    constexpr int NT = BlkCfg<T>::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlkShared<T>& sh = *reinterpret_cast<BlkShared<T>*>(smem_raw);
    unsigned char* stage = smem_raw + ((sizeof(BlkShared<T>) + 15) / 16 * 16);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh.acct = atomicAdd(A.queue, 1);
        __syncthreads();
        const int idx = sh.acct;
        __syncthreads();
        if (idx >= A.M) break;
        const int a = A.order ? A.order[idx] : idx;
        if ((A.skip && A.skip[a]) || (A.resume && !A.active[a])) continue;
        View<T> V;
        const size_t dbase = (size_t)a * A.Npad;
        if (!A.plist) {
            // dense: every position of the universe; state in the dense arrays
            V.n = A.N; V.pos = nullptr;
            V.w0 = A.w0 + dbase; V.lo = A.lo + dbase; V.up = A.up + dbase; V.c = A.c + dbase;
            V.pw = A.pw_idx ? A.pw_idx + dbase : nullptr;
            V.z = A.z + dbase; V.y = A.y + dbase; V.X = A.X + dbase;
            for (int s = tid; s <= A.S; s += NT) sh.sec[s] = A.sec_start[s];
        } else {
            // packed: the account's own names, in shared memory when they fit
            const int64_t off = A.poff[a];
            const int n = int(A.poff[a + 1] - off);
            V.n = n;
            const bool staged = n <= A.stage_cap;
            T *w0, *lo, *up, *c, *z, *y, *X;
            int *pos, *pw;
            if (staged) {
                T* base = reinterpret_cast<T*>(stage);
                w0 = base; lo = w0 + n; up = lo + n; c = up + n; z = c + n; y = z + n; X = y + n;
                pos = reinterpret_cast<int*>(X + n);
                pw = pos + n;
            } else {
                w0 = A.w0p + off; lo = A.lop + off; up = A.upp + off; c = A.cp + off;
                z = A.z + off; y = A.y + off; X = A.X + off;
                pos = A.plist + off;
                pw = A.pwp + off;
            }
            for (int q = tid; q < n; q += NT) {
                const int p = A.plist[off + q];
                if (staged) pos[q] = p;
                w0[q] = A.w0[dbase + p]; lo[q] = A.lo[dbase + p]; up[q] = A.up[dbase + p]; c[q] = A.c[dbase + p];
                pw[q] = A.pw_idx ? A.pw_idx[dbase + p] : -1;
                if (staged && A.resume) { z[q] = A.z[off + q]; y[q] = A.y[off + q]; }
            }
            for (int s = tid; s <= A.S; s += NT) sh.sec[s] = A.psec[(size_t)a * (A.S + 1) + s];
            V.pos = pos; V.w0 = w0; V.lo = lo; V.up = up; V.c = c; V.pw = pw; V.z = z; V.y = y; V.X = X;
            __syncthreads();
            solve_account(A, sh, V, a);
            if (staged)                                  // the state for a second pass
                for (int q = tid; q < n; q += NT) { A.z[off + q] = z[q]; A.y[off + q] = y[q]; }
            __syncthreads();
            continue;
        }
        __syncthreads();
        solve_account(A, sh, V, a);
    }
}

template <typename T>
int blk_threads() { return BlkCfg<T>::THREADS; }

template <typename T>
size_t blk_smem_bytes(const BlkArgs<T>& A) {
    const size_t fixed = (sizeof(BlkShared<T>) + 15) / 16 * 16;
    return fixed + (size_t)A.stage_cap * (7 * sizeof(T) + 2 * sizeof(int));
}

template <typename T>
void launch_block_admm(const BlkArgs<T>& A, int grid, cudaStream_t st) {
    const size_t smem = blk_smem_bytes(A);
    cudaFuncSetAttribute(k_block_admm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaMemsetAsync(A.queue, 0, sizeof(int), st);
    k_block_admm<T><<<grid, BlkCfg<T>::THREADS, smem, st>>>(A);
}

template <typename T>
int blk_grid(const BlkArgs<T>& A) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = blk_smem_bytes(A);
    cudaFuncSetAttribute(k_block_admm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_block_admm<T>, BlkCfg<T>::THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        per = 1;
    }
    return std::max(1, std::min(A.M, std::max(1, sms) * std::max(1, per)));
}

template int blk_grid<float>(const BlkArgs<float>&);
template int blk_grid<double>(const BlkArgs<double>&);
template int blk_threads<float>();
template int blk_threads<double>();
template size_t blk_smem_bytes<float>(const BlkArgs<float>&);
template size_t blk_smem_bytes<double>(const BlkArgs<double>&);
template void launch_block_admm<float>(const BlkArgs<float>&, int, cudaStream_t);
template void launch_block_admm<double>(const BlkArgs<double>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// per-account position lists of a ragged book: the member positions of account a in increasing
// order (its range poff[a] .. poff[a+1] of plist) and its sector ranges within that list
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_member_lists(int Npad, int S, const int* member, const int* sec_start,
                                                       const int64_t* poff, int* plist, int* psec) {
    const int a = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ int wsum[32];
    __shared__ int carry;
    const int* mem = member + (size_t)a * Npad;
    int* out = plist + poff[a];
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int p0 = 0; p0 < Npad; p0 += 1024) {
        const int p = p0 + tid;
        const int m = (p < Npad) ? (mem[p] != 0) : 0;
        const unsigned b = __ballot_sync(0xffffffffu, m);
        if (lane == 0) wsum[warp] = __popc(b);
        __syncthreads();
        int before = carry;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (m) out[before + __popc(b & ((1u << lane) - 1u))] = p;
        __syncthreads();
        if (tid == 0) for (int w = 0; w < 32; ++w) carry += wsum[w];
        __syncthreads();
    }
    // sector s starts at the first listed position >= sec_start[s]
    const int n = int(poff[a + 1] - poff[a]);
    for (int s = tid; s <= S; s += 1024) {
        const int target = sec_start[s];
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (out[mid] < target) lo = mid + 1; else hi = mid;
        }
        psec[(size_t)a * (S + 1) + s] = lo;
    }
}

void launch_member_lists(int M, int Npad, int S, const int* member, const int* sec_start, const int64_t* poff,
                         int* plist, int* psec, cudaStream_t st) {
    if (M > 0) k_member_lists<<<M, 1024, 0, st>>>(Npad, S, member, sec_start, poff, plist, psec);
}

}  // namespace prism
