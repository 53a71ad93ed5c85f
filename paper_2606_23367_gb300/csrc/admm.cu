// admm.cu -- the batched ADMM iteration (SIMT products, prox/projection, control).
//
// Splitting (this library's method; the paper discloses none of its own, Sec. 3):
// x = z with f(x) = x' Sigma x - mu' x and g(z) = sum_i phi_i(z_i) + indicator of
// Z = {1'z = 1, l <= z <= u, lo_s <= sum_{i in s} z_i <= hi_s, ||z - w0||_1 <= tau}
// (Eq. 1 constraints, Sec. 4.2). One iteration, with penalty rho and relaxation alpha:
//
//   X  = Delta^{-1} (mu + rho z - y),     Delta = diag(2 d + rho)
//   P  = B' X                              (G2, shared-B product over assets)
//   Q  = C^{-1} P,  C = (2F)^{-1} + B' Delta^{-1} B      (G3, K x K)
//   x  = X - Delta^{-1} B Q                (G4, Woodbury: x = (2 Sigma + rho I)^{-1} (mu + rho z - y))
//   v  = alpha x + (1 - alpha) z + y / rho
//   z+ = argmin_{z in Z} sum phi_i(z_i) + rho/2 ||z - v||^2     (G5)
//   y+ = rho (v - z+)
//
// The projection in G5 relaxes the budget (nu), the bands (lambda_s) and the cap
// (theta): z_i = prox of (phi_i + theta |. - w0_i|)/rho on [l_i, u_i] at
// v_i - (nu + lambda_{s(i)})/rho. Each sector sum S_s(eta) is nonincreasing and
// piecewise linear in eta, so a sector held at its upper edge has eta_s solving
// S_s(eta_s) = hi_s, and the budget reads sum_s S_s(clamp(nu, eta_hi_s, eta_lo_s)) = 1.
// Each scalar root is found by Newton steps on the piecewise-linear sum (exact once
// on the right piece) safeguarded by a bracket; the cap multiplier theta is found
// by an outer bracketed secant on the turnover U(theta) = tau.
#include <cfloat>
#include <cmath>

#include <cstring>

#include "common.cuh"
#include "solver.h"

namespace prism {

constexpr int PROX_MAXIT = 80;

// ---------------------------------------------------------------------------
// initial state: z = clip(w0, l, u), y = 0, X = Delta^{-1}(mu + rho z)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rho_val(int j) {
    return float(RHO_MIN) * exp10f(float(j) / float(RHO_PER_DECADE));
}

__device__ __forceinline__ void store_X(const Dev& D, size_t e, float X) {
    if (D.bf16) {
        __nv_bfloat16 h = __float2bfloat16_rn(X);
        D.Xhi[e] = h;
        D.Xlo[e] = __float2bfloat16_rn(X - __bfloat162float(h));
    } else {
        D.X[e] = X;
    }
}

__global__ void k_init_state(Dev D) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)D.M * D.Npad) return;
    int a = int(e / D.Npad), p = int(e % D.Npad);
    float rho = rho_val(D.rho_idx[a]);
    float z = fminf(fmaxf(D.w0[e], D.lo[e]), D.up[e]);
    if (p >= D.N) z = 0.f;
    D.z[e] = z;
    D.y[e] = 0.f;
    float X = (p < D.N) ? (D.mu32[p] + rho * z) / (2.f * D.d32[p] + rho) : 0.f;
    store_X(D, e, X);
}

void launch_init_state(const Dev& D, cudaStream_t st) {
    size_t n = (size_t)D.M * D.Npad;
    k_init_state<<<(unsigned)cdiv64(n, 256), 256, 0, st>>>(D);
}

// ---------------------------------------------------------------------------
// G2 (SIMT): Ppart[s][m][k] = sum_{i in split s} X[m][i] B[i][k]
// block = 32 accounts x all K factors over one asset split; 256 threads,
// thread = one account x K/8 factors.
// ---------------------------------------------------------------------------
int choose_nsplit(int M, int N) {
    int tiles = cdiv(M, 32);
    int ns = std::max(1, 2 * 152 / tiles);
    ns = std::min(ns, cdiv(N, 32));
    return ns;
}

__device__ __forceinline__ bool tile_active(const Dev& D, int m0, int count) {
    int act = 0;
    if (threadIdx.x < count) {
        const int m = m0 + threadIdx.x;
        act = (D.active == nullptr) || (m < D.M && D.active[m]);
    }
    return __syncthreads_or(act) != 0;
}

__global__ void __launch_bounds__(256) k_gemm_P(Dev D) {
    const int m0 = blockIdx.x * 32;
    const int split = blockIdx.y;
    if (!tile_active(D, m0, 32)) return;
    const int chunk = cdiv(cdiv(D.N, D.nsplit), 32) * 32;
    const int i_begin = split * chunk, i_end = min(D.N, i_begin + chunk);
    __shared__ float sX[32][33];
    __shared__ float sB[32][KMAX + 1];
    const int t = threadIdx.x;
    const int am = t >> 3;            // account within tile
    const int kg = t & 7;             // factor group
    const int K = D.K;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    for (int i0 = i_begin; i0 < i_end; i0 += 32) {
        __syncthreads();
        for (int e = t; e < 32 * 32; e += 256) {
            int r = e >> 5, cc = e & 31;
            int m = m0 + r, i = i0 + cc;
            sX[r][cc] = (m < D.M && i < i_end) ? D.X[(size_t)m * D.Npad + i] : 0.f;
        }
        for (int e = t; e < 32 * K; e += 256) {
            int r = e / K, cc = e % K;
            int i = i0 + r;
            sB[r][cc] = (i < i_end) ? D.B32[(size_t)i * K + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
            float x = sX[am][r];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int k = kg + 8 * q;
                if (k < K) acc[q] = fmaf(x, sB[r][k], acc[q]);
            }
        }
    }
    int m = m0 + am;
    if (m < D.M) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int k = kg + 8 * q;
            if (k < K) D.Ppart[((size_t)split * D.M + m) * D.pstride + k] = acc[q];
        }
    }
}

void launch_gemm_P(const Dev& D, cudaStream_t st) {
    dim3 grid(cdiv(D.M, 32), D.nsplit);
    k_gemm_P<<<grid, 256, 0, st>>>(D);
}

// ---------------------------------------------------------------------------
// G3: Q[m] = Cinv[rho_idx[m]] * P[m]. solve_K is the per-account solve on a P in shared memory;
// k_small_solve runs it after G2 (P = sum_s Ppart[s][m]), k_prox_roots at the end of the fused
// iteration (P = the fused pass's partial sets plus its own candidates' share).
// ---------------------------------------------------------------------------
struct SolveScratch {
    float sT[KMAX], sP0[KMAX], sQ[KMAX];
    float red_p[KMAX / 32], red_d[KMAX / 32];
    float red[4][KMAX];                   // row-group partials of a block matrix-vector product
};

// y_t = sum_j A[j][t] x_j for t < K (A symmetric K x K, row-major: column t is contiguous over
// t) by GROUPS groups of KMAX threads, group g over rows g KMAX / GROUPS onwards, combined in
// shared memory in group order. Block-collective; the value is meaningful in threads t < K.
template <int GROUPS>
__device__ __forceinline__ float sym_matvec(const float* A, int K, const float* x, SolveScratch& w) {
    const int t = threadIdx.x, c = t % KMAX, g = t / KMAX;
    constexpr int RPG = KMAX / GROUPS;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (g < GROUPS && c < K) {
#pragma unroll
        for (int r = 0; r < RPG; r += 4) {
            const int j = g * RPG + r;
            if (j < K) a0 = fmaf(A[(size_t)j * K + c], x[j], a0);
            if (j + 1 < K) a1 = fmaf(A[(size_t)(j + 1) * K + c], x[j + 1], a1);
            if (j + 2 < K) a2 = fmaf(A[(size_t)(j + 2) * K + c], x[j + 2], a2);
            if (j + 3 < K) a3 = fmaf(A[(size_t)(j + 3) * K + c], x[j + 3], a3);
        }
    }
    const float part = (a0 + a1) + (a2 + a3);
    if (GROUPS == 1) return part;
    __syncthreads();
    if (g < GROUPS) w.red[g][c] = part;
    __syncthreads();
    float y = 0.f;
    if (t < KMAX)
#pragma unroll
        for (int h = 0; h < GROUPS; ++h) y += w.red[h][t];
    return y;
}

// Q = C^{-1} P for account m, P in shared memory (KMAX entries, zero past K), and the update of
// the factor-exposure block when the book has one. Block-collective: every thread of the block
// calls it; the block has at least GROUPS x KMAX threads, the products run over GROUPS row
// groups, and threads t < K write. cpre: column t of C^{-1} already in registers (GROUPS = 1),
// or null to read it here.
template <int GROUPS>
__device__ __forceinline__ void solve_K(const Dev& D, int m, float* sP, SolveScratch& w, const float* cpre) {
    const int K = D.K, t = threadIdx.x;
    const int jr = D.rho_idx[m];
    const float* C = D.Cinv + (size_t)jr * K * K;
    // Factor-exposure block (s = B'x, dual ys): the x-update's right side gains B (rho s - ys), so
    // with tv = rho s - ys the reduced right side is P0 + G tv and Q' = C^{-1} (P0 + G tv) - tv
    // (then x = X - Delta^{-1} B Q' as without the block, and B'x = P0 - G Q').
    const bool fac = D.s != nullptr;
    const float* Gj = fac ? D.G + (size_t)jr * K * K : nullptr;
    float rho = 0.f, s_old = 0.f, ys_old = 0.f;
    if (fac) {
        rho = rho_val(jr);
        if (t < K) { s_old = D.s[(size_t)m * K + t]; ys_old = D.ys[(size_t)m * K + t]; }
        if (t < KMAX) {
            w.sT[t] = t < K ? rho * s_old - ys_old : 0.f;
            w.sP0[t] = sP[t];
        }
        __syncthreads();
        const float g = sym_matvec<GROUPS>(Gj, K, w.sT, w);
        __syncthreads();
        if (t < KMAX) sP[t] = w.sP0[t] + g;
        __syncthreads();
    }
    float q = 0.f;
    if (cpre) {
        if (t < K) {
            float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
#pragma unroll
            for (int j = 0; j < KMAX; j += 4) {
                q0 = fmaf(cpre[j], sP[j], q0);
                q1 = fmaf(cpre[j + 1], sP[j + 1], q1);
                q2 = fmaf(cpre[j + 2], sP[j + 2], q2);
                q3 = fmaf(cpre[j + 3], sP[j + 3], q3);
            }
            q = (q0 + q1) + (q2 + q3);
        }
    } else {
        q = sym_matvec<GROUPS>(C, K, sP, w);
    }
    if (t < K) {
        if (fac) q -= w.sT[t];
        if (D.bf16) {
            __nv_bfloat16 h = __float2bfloat16_rn(q);
            D.Qhi[(size_t)m * KMAX + t] = h;     // row stride 64: the tensor-core operand layout
            D.Qlo[(size_t)m * KMAX + t] = __float2bfloat16_rn(q - __bfloat162float(h));
        }
        D.Q[(size_t)m * K + t] = q;
        if (fac) w.sQ[t] = q;
    }
    if (fac) {
        // the block's own update: relaxed B'x, s = clip(., lo, hi), dual step, residuals
        __syncthreads();
        const float g = sym_matvec<GROUPS>(Gj, K, w.sQ, w);
        float rp = 0.f, rd = 0.f;
        if (t < K) {
            const float bx = w.sP0[t] - g;
            const float xh = D.alpha * bx + (1.f - D.alpha) * s_old;
            const float lo = D.flo[(size_t)m * K + t], hi = D.fhi[(size_t)m * K + t];
            const float sn = fminf(fmaxf(xh + ys_old / rho, lo), hi);
            D.s[(size_t)m * K + t] = sn;
            D.ys[(size_t)m * K + t] = ys_old + rho * (xh - sn);
            D.sflag[(size_t)m * K + t] = (sn >= hi) ? 1 : ((sn <= lo) ? -1 : 0);
            rp = fabsf(xh - sn);
            rd = rho * fabsf(sn - s_old);
            if (!(isfinite(rp) && isfinite(rd))) rp = rd = INFINITY;
        }
        // (reduced through arrays of their own: a warp with no factors reaches this point while
        // another may still read sP0 above)
        rp = warp_max(rp);
        rd = warp_max(rd);
        if ((t & 31) == 0 && t < KMAX) { w.red_p[t >> 5] = rp; w.red_d[t >> 5] = rd; }
        __syncthreads();
        if (t == 0) {
            D.rps[m] = fmaxf(w.red_p[0], w.red_p[1]);
            D.rds[m] = fmaxf(w.red_d[0], w.red_d[1]);
        }
    }
}

__global__ void __launch_bounds__(KMAX) k_small_solve(Dev D) {
    const int m = D.m0 + blockIdx.x;
    if (D.active && !D.active[m]) return;
    if (D.needP && !D.needP[m]) return;    // its P and Q came from the fused iteration
    const int K = D.K;
    __shared__ float sP[KMAX];
    __shared__ SolveScratch w;
    const int t = threadIdx.x;
    // C^{-1} is symmetric: thread t reads column t (the block's loads are contiguous). The whole
    // column is loaded into registers first, so that it is in flight with the partial sums.
    float c[KMAX];
    const float* C = D.Cinv + (size_t)D.rho_idx[m] * K * K + t;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) c[j] = (t < K && j < K) ? C[(size_t)j * K] : 0.f;
    pdl_wait();                            // the partials of the product just before
    pdl_trigger();
    if (t < K) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float* pp = D.Ppart + (size_t)m * D.pstride + t;
        const size_t stride = (size_t)D.M * D.pstride;
        int sp = 0;
        for (; sp + 8 <= D.nsplit; sp += 8)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += pp[(size_t)(sp + u) * stride];
        for (; sp < D.nsplit; ++sp) acc[0] += pp[(size_t)sp * stride];
        sP[t] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    } else {
        sP[t] = 0.f;                       // factors beyond K (their column entries are zero too)
    }
    __syncthreads();
    solve_K<1>(D, m, sP, w, c);
}

void launch_small_solve(const Dev& D, cudaStream_t st, bool pdl) {
    launch_ex(k_small_solve, dim3((D.m1 ? D.m1 : D.M) - D.m0), dim3(KMAX), 0, st, pdl, D);
}

// ---------------------------------------------------------------------------
// G4 (SIMT): v = alpha x + (1-alpha) z + y/rho with x = X - Delta^{-1} (B Q)
// block = 32 accounts x 64 assets; thread = 4 accounts x 2 assets
// ---------------------------------------------------------------------------
// (x is recomputed from z and y in the epilogue, so the split copy of X feeds only the products)
__global__ void __launch_bounds__(256) k_gemm_x(Dev D) {
    const int m0 = blockIdx.y * 32;
    const int i0 = blockIdx.x * 64;
    const int K = D.K;
    if (!tile_active(D, m0, 32)) return;
    __shared__ float sQ[32][KMAX + 1];
    __shared__ float sB[64][KMAX + 1];
    const int t = threadIdx.x;
    for (int e = t; e < 32 * K; e += 256) {
        int r = e / K, cc = e % K;
        int m = m0 + r;
        sQ[r][cc] = (m < D.M) ? D.Q[(size_t)m * K + cc] : 0.f;
    }
    for (int e = t; e < 64 * K; e += 256) {
        int r = e / K, cc = e % K;
        int i = i0 + r;
        sB[r][cc] = (i < D.N) ? D.B32[(size_t)i * K + cc] : 0.f;
    }
    __syncthreads();
    const int lane = t & 31, grp = t >> 5;    // 8 groups of 4 accounts
    float acc[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = 0.f;
    for (int k = 0; k < K; ++k) {
        float b0 = sB[lane][k], b1 = sB[lane + 32][k];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float q = sQ[grp * 4 + u][k];
            acc[u][0] = fmaf(q, b0, acc[u][0]);
            acc[u][1] = fmaf(q, b1, acc[u][1]);
        }
    }
    if (D.raw_out) {          // the plain product (diagnostics, polish gradient)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = m0 + grp * 4 + u;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = i0 + lane + 32 * h;
                if (m < D.M && i < D.N) D.v[(size_t)m * D.Npad + i] = acc[u][h];
            }
        }
        return;
    }
    // epilogue: all loads of the thread's 8 outputs first, then the stores
    float zz[4][2], yy[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int m = m0 + grp * 4 + u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + lane + 32 * h;
            const bool ok = m < D.M && i < D.N;
            const size_t e = (size_t)m * D.Npad + i;
            zz[u][h] = ok ? __ldg(D.z + e) : 0.f;
            yy[u][h] = ok ? __ldg(D.y + e) : 0.f;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int m = m0 + grp * 4 + u;
        if (m >= D.M) continue;
        const float rho = rho_val(D.rho_idx[m]);
        const float irho = 1.f / rho;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + lane + 32 * h;
            if (i >= D.N) continue;
            const size_t e = (size_t)m * D.Npad + i;
            const float x = (D.mu32[i] + rho * zz[u][h] - yy[u][h] - acc[u][h]) / (2.f * D.d32[i] + rho);
            D.v[e] = D.alpha * x + (1.f - D.alpha) * zz[u][h] + yy[u][h] * irho;
        }
    }
}

void launch_gemm_x(const Dev& D, cudaStream_t st) {
    dim3 grid(cdiv(D.N, 64), cdiv(D.M, 32));
    k_gemm_x<<<grid, 256, 0, st>>>(D);
}



// ---------------------------------------------------------------------------
// G5/G6: projection onto Z with the transition prox, dual update, residuals,
// penalty adaptation, convergence. One block per account, warp w owns sectors
// w, w + nwarps, ... The account's per-entry data are read through a source:
// shared memory (staged once per launch) when the account fits, else global.
// ---------------------------------------------------------------------------
struct EntryEval {
    float z;
    int lin;   // 1 when dz/deta = -1/rho (z strictly inside a linear piece)
};

// per-entry data of one account, from global memory. After the fused streaming pass, which
// writes v only for its candidates, cm holds the account's candidate masks: an entry pinned at
// its lower bound has y = rho (v - l) just written, so v = l + y / rho.
struct GlobalSrc {
    const float *v, *w0, *lo, *up, *c;
    const int* pw;
    const unsigned* cm = nullptr;
    const float* yv = nullptr;
    float irho = 0.f;
    __device__ __forceinline__ GlobalSrc(const Dev& D, size_t base)
        : v(D.v + base), w0(D.w0 + base), lo(D.lo + base), up(D.up + base), c(D.c + base),
          pw(D.pw_idx ? D.pw_idx + base : nullptr) {}
    __device__ __forceinline__ float val(int p) const {
        if (cm && !((cm[p >> 5] >> (p & 31)) & 1u)) return lo[p] + yv[p] * irho;
        return v[p];
    }
};

// z_i(eta) for one entry: prox of (phi_i + theta|.-w0|)/rho on [l, u] at t = v - eta/rho.
template <class Src>
__device__ __forceinline__ EntryEval eval_entry(const Dev& D, const Src& S, int p, float eta, float theta,
                                                float irho) {
    EntryEval r;
    const float t = S.val(p) - eta * irho;
    const float w0 = S.w0[p], lo = S.lo[p], up = S.up[p];
    const int pw = S.pw ? S.pw[p] : -1;
    if (pw < 0) {
        const float k = (S.c[p] + theta) * irho;
        float z = (t > w0 + k) ? t - k : ((t < w0 - k) ? t + k : w0);
        z = fminf(fmaxf(z, lo), up);
        r.z = z;
        r.lin = (z > lo && z < up && z != w0) ? 1 : 0;
    } else {
        // segment search: the first segment j whose stationary point t - s_j/rho does
        // not lie above it decides; below its left end -> the breakpoint itself
        const float* bp = D.pw_bp + (size_t)pw * MAXBP;
        const float* sl = D.pw_sl + (size_t)pw * (MAXBP - 1);
        const int nb = D.pw_nbp[pw];
        float z = bp[nb - 1];
        int lin = 0;
        for (int j = 0; j + 1 < nb; ++j) {
            const float sj = sl[j] + theta * ((bp[j] + bp[j + 1] > 2.f * w0) ? 1.f : -1.f);
            const float cand = t - sj * irho;
            if (cand <= bp[j]) { z = bp[j]; break; }
            if (cand < bp[j + 1]) { z = cand; lin = 1; break; }
        }
        r.z = z;
        r.lin = lin;
    }
    return r;
}

// Warp-collective sum of z and count of linear entries over sorted positions [p0, p1).
template <class Src>
__device__ __forceinline__ void warp_sector_sum(const Dev& D, const Src& S, int p0, int p1, float eta,
                                                float theta, float irho, float& sum, int& cnt) {
    const int lane = threadIdx.x & 31;
    float s = 0.f;
    int n = 0;
    for (int p = p0 + lane; p < p1; p += 32) {
        const EntryEval r = eval_entry(D, S, p, eta, theta, irho);
        s += r.z;
        n += r.lin;
    }
    sum = warp_sum(s);
    cnt = warp_sum(n);
}

// Safeguarded Newton for g(x) = S(x) - target, S nonincreasing PWL with slope -cnt/rho.
struct Root {
    float x, a, b, step;
    int done;
};

__device__ __forceinline__ void root_init(Root& R, float x0, float step) {
    R.x = x0;
    R.a = -FLT_MAX;
    R.b = FLT_MAX;
    R.step = step;
    R.done = 0;
}

// One update from g = S(x) - target and the count of linear entries.
__device__ __forceinline__ void root_update(Root& R, float g, int cnt, float rho, float tol) {
    if (fabsf(g) <= tol) { R.done = 1; return; }
    if (g > 0.f) R.a = R.x; else R.b = R.x;
    float xn;
    bool ok = false;
    if (cnt > 0) {
        xn = R.x + g * rho / float(cnt);
        ok = (xn > R.a && xn < R.b);
    }
    if (!ok) {
        if (R.a > -FLT_MAX && R.b < FLT_MAX) {
            xn = 0.5f * (R.a + R.b);
        } else {
            xn = (g > 0.f) ? R.x + R.step : R.x - R.step;
            R.step *= 2.f;
        }
    }
    if (R.a > -FLT_MAX && R.b < FLT_MAX && (R.b - R.a) <= 4e-7f * fmaxf(1e-6f, fabsf(R.a) + fabsf(R.b))) {
        R.x = 0.5f * (R.a + R.b);
        R.done = 1;
        return;
    }
    R.x = xn;
}

struct ProxShared {
    int nflag;                          // sectors whose band edge was found binding in the latest check
    float eta_hi[SMAX], eta_lo[SMAX];
    float cap_hi[SMAX], floor_lo[SMAX];
    float red_f[32];
    int red_i[32];
    float red5[5][32];
    int red_bad[32];
    int newj;
};

// Inner projection at fixed theta: the budget root nu of sum_s S_s(clamp(nu, eta_hi_s, eta_lo_s)) = 1
// (S_s the sum of z over sector s, nonincreasing), with edge roots only for the sectors whose band
// binds. Every sector starts unclamped (eta_hi = -inf, eta_lo = +inf: S_s(nu) itself); after each
// budget root the sectors are checked at it, one whose sum leaves its band gets that edge's root
// (after which its clamp is exact at every nu), and the budget root is solved again, until no
// sector leaves its band. Returns nu; the edge multipliers in sh.eta_* (-inf / +inf for an edge
// that does not bind). Block-collective.
template <class Src>
__device__ float project_inner(const Dev& D, const Src& S, int a, float theta, float rho, float irho, float nu0,
                               ProxShared& sh) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const float step0 = 0.05f * rho + 1e-6f;
    for (int s = threadIdx.x; s < D.S; s += blockDim.x) {
        sh.eta_hi[s] = -FLT_MAX;
        sh.eta_lo[s] = FLT_MAX;
    }
    if (threadIdx.x == 0) sh.nflag = 0;
    __syncthreads();
    float nu = nu0;
    for (int round = 0; round <= 2 * D.S; ++round) {
        // budget root with the current clamps
        Root R;
        root_init(R, nu, step0);
        for (int it = 0; it < PROX_MAXIT; ++it) {
            float part = 0.f;
            int pc = 0;
            for (int s = warp; s < D.S; s += nwarps) {
                const int p0 = D.sec_start[s], p1 = D.sec_start[s + 1];
                const float arg = fminf(fmaxf(R.x, sh.eta_hi[s]), sh.eta_lo[s]);
                float sum; int cnt;
                warp_sector_sum(D, S, p0, p1, arg, theta, irho, sum, cnt);
                part += sum;
                if (arg == R.x) pc += cnt;
            }
            if (lane == 0) { sh.red_f[warp] = part; sh.red_i[warp] = pc; }
            __syncthreads();
            float T = 0.f;
            int C = 0;
            for (int w = 0; w < nwarps; ++w) { T += sh.red_f[w]; C += sh.red_i[w]; }
            __syncthreads();
            root_update(R, T - 1.f, C, rho, 1e-6f);
            if (D.stats && threadIdx.x == 0) atomicAdd(D.stats + 2, 1ull);
            if (R.done) break;
        }
        nu = R.x;
        // each sector at nu: an edge its sum leaves gets its root (one warp per sector)
        for (int s = warp; s < D.S; s += nwarps) {
            const int p0 = D.sec_start[s], p1 = D.sec_start[s + 1];
            if (p1 <= p0) continue;
            const float hi = D.band_hi[a * D.S + s], lo = D.band_lo[a * D.S + s];
            const bool free_hi = sh.eta_hi[s] == -FLT_MAX, free_lo = sh.eta_lo[s] == FLT_MAX;
            const float arg = fminf(fmaxf(nu, sh.eta_hi[s]), sh.eta_lo[s]);
            float Sv; int cv;
            warp_sector_sum(D, S, p0, p1, arg, theta, irho, Sv, cv);
            float eh = sh.eta_hi[s], el = sh.eta_lo[s];
            bool flag = false;
            if (free_hi && hi < sh.cap_hi[s] && Sv > hi + 1e-6f * fmaxf(hi, 1e-3f)) {
                Root E;
                const float w = D.eta_hi[a * D.S + s];
                root_init(E, (w > arg && w < FLT_MAX) ? w : arg, step0);
                E.a = arg;                                  // S_s(arg) > hi: the root lies above arg
                int it = 0;
                for (; it < PROX_MAXIT && !E.done; ++it) {
                    float sum; int cnt;
                    warp_sector_sum(D, S, p0, p1, E.x, theta, irho, sum, cnt);
                    root_update(E, sum - hi, cnt, rho, 1e-6f * fmaxf(hi, 1e-3f));
                }
                if (D.stats && lane == 0) atomicAdd(D.stats + 1, (unsigned long long)it);
                eh = E.x;
                flag = true;
            } else if (free_lo && lo > sh.floor_lo[s] && Sv < lo - 1e-6f * fmaxf(fabsf(lo), 1e-3f)) {
                Root E;
                const float w = D.eta_lo[a * D.S + s];
                root_init(E, (w < arg && w > -FLT_MAX) ? w : arg, step0);
                E.b = arg;                                  // S_s(arg) < lo: the root lies below arg
                for (int it = 0; it < PROX_MAXIT && !E.done; ++it) {
                    float sum; int cnt;
                    warp_sector_sum(D, S, p0, p1, E.x, theta, irho, sum, cnt);
                    root_update(E, sum - lo, cnt, rho, 1e-6f * fmaxf(fabsf(lo), 1e-3f));
                }
                el = E.x;
                flag = true;
            }
            if (lane == 0 && flag) {
                sh.eta_hi[s] = eh;
                sh.eta_lo[s] = el;
                atomicAdd(&sh.nflag, 1);
            }
        }
        __syncthreads();
        const int nf = sh.nflag;
        __syncthreads();
        if (threadIdx.x == 0) sh.nflag = 0;
        if (nf == 0) break;
    }
    __syncthreads();
    return nu;
}

// Turnover sum_i |z_i - w0_i| at the current (nu, eta, theta). Block-collective.
template <class Src>
__device__ float turnover_at(const Dev& D, const Src& S, float nu, float theta, float irho, ProxShared& sh) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    float part = 0.f;
    for (int s = warp; s < D.S; s += nwarps) {
        const int p0 = D.sec_start[s], p1 = D.sec_start[s + 1];
        const float arg = fminf(fmaxf(nu, sh.eta_hi[s]), sh.eta_lo[s]);
        float acc = 0.f;
        for (int p = p0 + lane; p < p1; p += 32) {
            const EntryEval r = eval_entry(D, S, p, arg, theta, irho);
            acc += fabsf(r.z - S.w0[p]);
        }
        part += warp_sum(acc);
    }
    if (lane == 0) sh.red_f[warp] = part;
    __syncthreads();
    float U = 0.f;
    for (int w = 0; w < nwarps; ++w) U += sh.red_f[w];
    __syncthreads();
    return U;
}

// The whole per-account step once the source is ready.
template <class Src>
__device__ void prox_account(const Dev& D, const Src& S, int a, ProxShared& sh) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    const size_t base = (size_t)a * D.Npad;
    const int j = D.rho_idx[a];
    const float rho = rho_val(j), irho = 1.f / rho;
    // sector capacities (largest / smallest attainable sums)
    for (int s = warp; s < D.S; s += nwarps) {
        const int p0 = D.sec_start[s], p1 = D.sec_start[s + 1];
        float cu = 0.f, cl = 0.f;
        for (int p = p0 + lane; p < p1; p += 32) {
            cu += S.up[p];
            cl += S.lo[p];
        }
        cu = warp_sum(cu);
        cl = warp_sum(cl);
        if (lane == 0) { sh.cap_hi[s] = cu; sh.floor_lo[s] = cl; }
    }
    __syncthreads();
    float theta = 0.f;
    const float nu_in = D.nu[a];
    float nu = project_inner(D, S, a, 0.f, rho, irho, nu_in, sh);
    const float tau = D.tau ? D.tau[a] : INFINITY;
    if (tau < INFINITY) {
        const float U = turnover_at(D, S, nu, 0.f, irho, sh);
        if (U > tau * (1.f + 1e-5f)) {
            // bracketed secant (Illinois) on U(theta) - tau, U nonincreasing in theta
            float t_lo = 0.f, u_lo = U - tau;
            float t_hi = fmaxf(D.theta[a], 1e-4f), u_hi = 0.f;
            for (int it = 0; it < 40; ++it) {
                nu = project_inner(D, S, a, t_hi, rho, irho, nu, sh);
                u_hi = turnover_at(D, S, nu, t_hi, irho, sh) - tau;
                if (u_hi <= 0.f) break;
                t_lo = t_hi; u_lo = u_hi;
                t_hi *= 4.f;
            }
            int side = 0;
            theta = t_hi;
            for (int it = 0; it < 60; ++it) {
                float tn = t_hi - u_hi * (t_hi - t_lo) / (u_hi - u_lo);
                if (!(tn > t_lo && tn < t_hi)) tn = 0.5f * (t_lo + t_hi);
                nu = project_inner(D, S, a, tn, rho, irho, nu, sh);
                const float un = turnover_at(D, S, nu, tn, irho, sh) - tau;
                theta = tn;
                // (the turnover is an FP32 sum of up to N terms: 1e-5 of tau is about its rounding,
                // and the polish settles the final point in FP64)
                if (fabsf(un) <= 1e-5f * tau || (t_hi - t_lo) <= 1e-7f * t_hi) break;
                if (un > 0.f) {
                    t_lo = tn; u_lo = un;
                    if (side == -1) u_hi *= 0.5f;
                    side = -1;
                } else {
                    t_hi = tn; u_hi = un;
                    if (side == 1) u_lo *= 0.5f;
                    side = 1;
                }
            }
        }
    }
    // final z, dual update, residuals, and X for the next iteration at the current
    // penalty; each lane's loads for a chunk of CH entries are issued before its stores
    constexpr int CH = 8;
    float rp = 0.f, rd = 0.f, nx = 0.f, nz = 0.f, ny = 0.f;
    int bad = 0;
    for (int s = warp; s < D.S; s += nwarps) {
        const int p0 = D.sec_start[s], p1 = D.sec_start[s + 1];
        const float arg = fminf(fmaxf(nu, sh.eta_hi[s]), sh.eta_lo[s]);
        for (int pb = p0 + lane; pb < p1; pb += 32 * CH) {
            float zo[CH], yo[CH], mu[CH], dd[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int p = pb + 32 * c;
                const bool in = p < p1;
                zo[c] = in ? D.z[base + p] : 0.f;
                yo[c] = in ? D.y[base + p] : 0.f;
                mu[c] = in ? D.mu32[p] : 0.f;
                dd[c] = in ? D.d32[p] : 1.f;
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int p = pb + 32 * c;
                if (p >= p1) break;
                const size_t e = base + p;
                const float vv = S.val(p);
                const EntryEval r = eval_entry(D, S, p, arg, theta, irho);
                const float yn = rho * (vv - r.z);
                rp = fmaxf(rp, fabsf(yn - yo[c]) * irho);
                rd = fmaxf(rd, rho * fabsf(r.z - zo[c]));
                nx = fmaxf(nx, fabsf(vv - yo[c] * irho));
                nz = fmaxf(nz, fabsf(r.z));
                ny = fmaxf(ny, fabsf(yn));
                bad |= !(isfinite(r.z) && isfinite(yn));
                D.z[e] = r.z;
                D.y[e] = yn;
                store_X(D, e, (mu[c] + rho * r.z - yn) / (2.f * dd[c] + rho));
            }
        }
    }
    rp = warp_max(rp); rd = warp_max(rd); nx = warp_max(nx); nz = warp_max(nz); ny = warp_max(ny);
    bad = warp_sum(bad);
    if (lane == 0) {
        sh.red5[0][warp] = rp; sh.red5[1][warp] = rd; sh.red5[2][warp] = nx; sh.red5[3][warp] = nz;
        sh.red5[4][warp] = ny; sh.red_bad[warp] = bad;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nwarps; ++w) {
            rp = fmaxf(rp, sh.red5[0][w]); rd = fmaxf(rd, sh.red5[1][w]); nx = fmaxf(nx, sh.red5[2][w]);
            nz = fmaxf(nz, sh.red5[3][w]); ny = fmaxf(ny, sh.red5[4][w]); bad += sh.red_bad[w];
        }
        const int it = D.iters[a] + 1;
        D.iters[a] = it;
        if (D.stats) atomicAdd(D.stats, 1ull);
        D.rp[a] = rp;
        D.rd[a] = rd;
        D.nu[a] = nu;
        if (D.dnu) D.dnu[a] = fabsf(nu - nu_in);          // the streaming form's margin
        D.theta[a] = theta;
        int newj = j;
        if (bad) {
            D.status[a] = PRISM_NUMERICAL_FAILURE;
            D.active[a] = 0;
        } else if (it >= D.min_iter && fmaxf(rp, D.rps ? D.rps[a] : 0.f) <= D.eps_admm &&
                   fmaxf(rd, D.rds ? D.rds[a] : 0.f) <= D.eps_admm) {
            D.active[a] = 0;
        } else if (it >= D.max_iter) {
            D.active[a] = 0;
            D.status[a] = PRISM_TIMEOUT;
        } else if (it % D.adapt_every == 0) {
            const float pr = rp / fmaxf(fmaxf(nx, nz), 1e-12f);
            const float du = rd / fmaxf(ny, 1e-12f);
            const float ratio = sqrtf(pr / fmaxf(du, 1e-20f));
            int dj = int(lrintf(float(RHO_PER_DECADE) * log10f(fmaxf(ratio, 1e-12f))));
            dj = max(-4, min(4, dj));
            newj = max(0, min(NRHO - 1, j + dj));
        }
        sh.newj = newj;
    }
    __syncthreads();
    const int newj = sh.newj;
    for (int s = warp; s < D.S; s += nwarps)
        if (lane == 0) {
            D.eta_hi[a * D.S + s] = sh.eta_hi[s];
            D.eta_lo[a * D.S + s] = sh.eta_lo[s];
        }
    if (newj != j) {
        // the penalty changed: X again at the new penalty (this block wrote z and y above)
        if (tid == 0) D.rho_idx[a] = newj;
        const float rn = rho_val(newj);
        for (int p = tid; p < D.N; p += blockDim.x) {
            const size_t e = base + p;
            store_X(D, e, (D.mu32[p] + rn * D.z[e] - D.y[e]) / (2.f * D.d32[p] + rn));
        }
    }
}

__global__ void __launch_bounds__(640, 1) k_prox(Dev D) {
    const int a = blockIdx.x;
    if (!D.active[a]) return;
    __shared__ ProxShared sh;
    const GlobalSrc S(D, (size_t)a * D.Npad);
    prox_account(D, S, a, sh);
}

// per-entry data of one account staged in shared memory
struct SmemSrc {
    const float *v, *w0, *lo, *up, *c;
    const int* pw;
    __device__ __forceinline__ float val(int p) const { return v[p]; }
};

__global__ void __launch_bounds__(640, 1) k_prox_smem(Dev D) {
    const int a = blockIdx.x;
    if (!D.active[a]) return;
    __shared__ ProxShared sh;
    extern __shared__ float4 dyn4[];
    float* dyn = reinterpret_cast<float*>(dyn4);
    const int NP = D.Npad;
    float* sv = dyn;
    float* sw0 = sv + NP;
    float* slo = sw0 + NP;
    float* sup = slo + NP;
    float* sc = sup + NP;
    int* spw = D.pw_idx ? reinterpret_cast<int*>(sc + NP) : nullptr;
    const size_t base = (size_t)a * NP;
    // one coalesced pass from global memory (Npad is a multiple of 64: float4-aligned)
    const float4* gv = reinterpret_cast<const float4*>(D.v + base);
    const float4* gw0 = reinterpret_cast<const float4*>(D.w0 + base);
    const float4* glo = reinterpret_cast<const float4*>(D.lo + base);
    const float4* gup = reinterpret_cast<const float4*>(D.up + base);
    const float4* gc = reinterpret_cast<const float4*>(D.c + base);
    for (int q0 = threadIdx.x; q0 < NP / 4; q0 += 2 * blockDim.x) {
        const int q1 = q0 + blockDim.x;
        const bool has1 = q1 < NP / 4;
        const float4 a0 = gv[q0], b0 = gw0[q0], c0 = glo[q0], d0 = gup[q0], e0 = gc[q0];
        float4 a1, b1, c1, d1, e1;
        if (has1) { a1 = gv[q1]; b1 = gw0[q1]; c1 = glo[q1]; d1 = gup[q1]; e1 = gc[q1]; }
        reinterpret_cast<float4*>(sv)[q0] = a0;
        reinterpret_cast<float4*>(sw0)[q0] = b0;
        reinterpret_cast<float4*>(slo)[q0] = c0;
        reinterpret_cast<float4*>(sup)[q0] = d0;
        reinterpret_cast<float4*>(sc)[q0] = e0;
        if (has1) {
            reinterpret_cast<float4*>(sv)[q1] = a1;
            reinterpret_cast<float4*>(sw0)[q1] = b1;
            reinterpret_cast<float4*>(slo)[q1] = c1;
            reinterpret_cast<float4*>(sup)[q1] = d1;
            reinterpret_cast<float4*>(sc)[q1] = e1;
        }
        if (spw) {
            reinterpret_cast<int4*>(spw)[q0] = reinterpret_cast<const int4*>(D.pw_idx + base)[q0];
            if (has1) reinterpret_cast<int4*>(spw)[q1] = reinterpret_cast<const int4*>(D.pw_idx + base)[q1];
        }
    }
    __syncthreads();
    const SmemSrc S{sv, sw0, slo, sup, sc, spw};
    prox_account(D, S, a, sh);
}

// ---------------------------------------------------------------------------
// G5/G6, streaming form (accounts with the L1 cost only and no turnover cap).
//
// z_i(eta) is nonincreasing in eta and equals l_i for every eta at or above the
// point where it first reaches l_i. With L = nu_prev - margin, an entry with
// z_i(L) == l_i takes z = l_i at every eta >= L: its new z, y and X are written
// during the single streaming pass. The other entries (held positions and names
// near activation, typically around 1% of the universe) are kept in shared
// memory for the root searches and written at the end. The budget equation is
// solved directly as
//     sum_s clamp(S_s(nu), lo_s, hi_s) = 1,
// which equals sum_s S_s(clamp(nu, eta_hi_s, eta_lo_s)) with the sector-edge
// roots (S_s nonincreasing); edge roots are found only for sectors that bind.
// A sector whose kept entries overflow their slots evaluates the rest of its
// range from global memory. If a root lies below L (the budget root when
// T(L) < 1, or a lower band edge), the sectors concerned are recomputed from
// global memory and this call reports infinite residuals (their old z and y
// are gone), so the account simply does not stop on this call.
// Global traffic per entry: one read of (v, w0, l, u, c, z, y) and one write of
// (z, y, X), the algorithmic minimum of the step.
// ---------------------------------------------------------------------------
constexpr int SP_WARPS = 8;             // warps per block; warp w owns sectors w, w + 8, ...
constexpr int SP_CW = 128;              // kept-entry slots per warp

struct StreamShared {
    int sec[SMAX + 1];                  // sector ranges (a copy of sec_start)
    float wh[SMAX], wl[SMAX];           // warm starts of the sector-edge multipliers
    int it0;                            // iterations before this call
    float blo[SMAX], bhi[SMAX];
    float SL[SMAX], sumlo[SMAX], Sx[SMAX];
    int CL[SMAX], Cx[SMAX];
    int cb[SMAX], ce[SMAX];             // slot range of each sector
    int gs[SMAX];                       // positions [gs, end) of the sector are read from global memory
    float eta_hi[SMAX], eta_lo[SMAX];
    float red5[5][SP_WARPS];
    int red_bad[SP_WARPS];
    int newj;
    int redo;                           // entries written before the tail were rewritten
    int cont;                           // the account iterates on
    float nu;
    // kept entries
    float v[SP_WARPS * SP_CW], w0[SP_WARPS * SP_CW], lo[SP_WARPS * SP_CW], up[SP_WARPS * SP_CW];
    float k[SP_WARPS * SP_CW], zo[SP_WARPS * SP_CW], yo[SP_WARPS * SP_CW];
    int pos[SP_WARPS * SP_CW];
};

// prox of c|.-w0|/rho on [l, u] at t = v - eta/rho with k = c/rho precomputed (the L1
// branch of eval_entry at theta = 0, bit for bit)
__device__ __forceinline__ EntryEval eval_l1(float v, float w0, float lo, float up, float k, float eta, float irho) {
    EntryEval r;
    const float t = v - eta * irho;
    float z = (t > w0 + k) ? t - k : ((t < w0 - k) ? t + k : w0);
    z = fminf(fmaxf(z, lo), up);
    r.z = z;
    r.lin = (z > lo && z < up && z != w0) ? 1 : 0;
    return r;
}

// Warp-collective S_s(eta) and the count of entries on a linear piece, for sector s.
__device__ __forceinline__ void stream_sector_eval(const Dev& D, const StreamShared& sh, const GlobalSrc& G, int s,
                                                   float eta, float irho, float& sum, int& cnt) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
    int n = 0;
    for (int q = sh.cb[s] + lane; q < sh.ce[s]; q += 32) {
        const EntryEval r = eval_l1(sh.v[q], sh.w0[q], sh.lo[q], sh.up[q], sh.k[q], eta, irho);
        acc += r.z;
        n += r.lin;
    }
    for (int p = sh.gs[s] + lane; p < sh.sec[s + 1]; p += 32) {
        const EntryEval r = eval_entry(D, G, p, eta, 0.f, irho);
        acc += r.z;
        n += r.lin;
    }
    sum = warp_sum(acc) + sh.sumlo[s];
    cnt = warp_sum(n);
}

// Residual maxima of one entry's update, then the writes of z, y, X.
struct StreamRes {
    float rp = 0.f, rd = 0.f, nx = 0.f, nz = 0.f, ny = 0.f;
    int bad = 0;
    // writes z and y = rho (v - z); returns X = Delta^{-1} (mu + rho z - y)
    __device__ __forceinline__ float put_zy(const Dev& D, size_t e, float z, float v, float zo, float yo, float mu,
                                            float dd, float rho, float irho) {
        const float yn = rho * (v - z);
        rp = fmaxf(rp, fabsf(yn - yo) * irho);
        rd = fmaxf(rd, rho * fabsf(z - zo));
        nx = fmaxf(nx, fabsf(v - yo * irho));
        nz = fmaxf(nz, fabsf(z));
        ny = fmaxf(ny, fabsf(yn));
        bad |= !(isfinite(z) && isfinite(yn));
        D.z[e] = z;
        D.y[e] = yn;
        return (mu + rho * z - yn) / (2.f * dd + rho);
    }
    __device__ __forceinline__ void put(const Dev& D, size_t e, float z, float v, float zo, float yo, float mu,
                                        float dd, float rho, float irho) {
        store_X(D, e, put_zy(D, e, z, v, zo, yo, mu, dd, rho, irho));
    }
};

// S_s(eta) and its linear count by one lane: the sector's kept entries, then its
// global-memory range (empty unless the sector was moved there)
__device__ __forceinline__ void lane_sector_eval(const Dev& D, const StreamShared& sh, const GlobalSrc& G, int s,
                                                 float eta, float irho, float& sum, int& cnt) {
    float acc = sh.sumlo[s];
    int n = 0;
    for (int q = sh.cb[s]; q < sh.ce[s]; ++q) {
        const EntryEval r = eval_l1(sh.v[q], sh.w0[q], sh.lo[q], sh.up[q], sh.k[q], eta, irho);
        acc += r.z;
        n += r.lin;
    }
    for (int p = sh.gs[s]; p < sh.sec[s + 1]; ++p) {
        const EntryEval r = eval_entry(D, G, p, eta, 0.f, irho);
        acc += r.z;
        n += r.lin;
    }
    sum = acc;
    cnt = n;
}

// Budget root and the edge roots of the binding sectors by warp 0 alone, lane s owning
// sectors s and s + 32. Writes sh.nu, sh.eta_hi, sh.eta_lo (and moves a sector whose lower
// edge lies below L to global memory).
__device__ void lane_solve(const Dev& D, StreamShared& sh, const GlobalSrc& G, int a, float L, float TL, float nu0,
                           float rho, float irho) {
    const int lane = threadIdx.x & 31, NS = D.S;
    const int s0 = lane, s1 = lane + 32;
    float S0 = s0 < NS ? sh.SL[s0] : 0.f, S1 = s1 < NS ? sh.SL[s1] : 0.f;
    Root R;
    root_init(R, nu0, 0.05f * rho + 1e-6f);
    R.a = L;
    if (L > -INFINITY && TL <= 1.f + 1e-6f) {
        R.x = L;                                         // L itself solves the budget equation
    } else {
        for (int it = 0; it < PROX_MAXIT; ++it) {
            float T = 0.f;
            int Cn = 0;
            if (s0 < NS) {
                int c;
                lane_sector_eval(D, sh, G, s0, R.x, irho, S0, c);
                T += fminf(fmaxf(S0, sh.blo[s0]), sh.bhi[s0]);
                if (S0 > sh.blo[s0] && S0 < sh.bhi[s0]) Cn += c;
            }
            if (s1 < NS) {
                int c;
                lane_sector_eval(D, sh, G, s1, R.x, irho, S1, c);
                T += fminf(fmaxf(S1, sh.blo[s1]), sh.bhi[s1]);
                if (S1 > sh.blo[s1] && S1 < sh.bhi[s1]) Cn += c;
            }
            T = warp_sum(T);
            Cn = warp_sum(Cn);
            const float x_eval = R.x;
            root_update(R, T - 1.f, Cn, rho, 1e-6f);
            if (D.stats && lane == 0) atomicAdd(D.stats + 2, 1ull);
            if (R.done && R.x == x_eval) break;
            if (R.done) {                                // bracket collapsed to a new point
                int c;
                if (s0 < NS) lane_sector_eval(D, sh, G, s0, R.x, irho, S0, c);
                if (s1 < NS) lane_sector_eval(D, sh, G, s1, R.x, irho, S1, c);
                break;
            }
        }
    }
    const float nu = R.x;
    for (int h = 0; h < 2; ++h) {
        const int s = h ? s1 : s0;
        if (s >= NS) continue;
        const float Sv = h ? S1 : S0;
        const float hi = sh.bhi[s], lo = sh.blo[s];
        float eh = -FLT_MAX, el = FLT_MAX;
        if (Sv > hi + 1e-6f * fmaxf(hi, 1e-3f)) {
            Root E;
            const float w = sh.wh[s];
            root_init(E, (w > nu && w < FLT_MAX) ? w : nu, 0.05f * rho + 1e-6f);
            E.a = nu;
            int it = 0;
            for (; it < PROX_MAXIT && !E.done; ++it) {
                float sum; int cnt;
                lane_sector_eval(D, sh, G, s, E.x, irho, sum, cnt);
                root_update(E, sum - hi, cnt, rho, 1e-6f * fmaxf(hi, 1e-3f));
            }
            if (D.stats) atomicAdd(D.stats + 1, (unsigned long long)it);
            eh = E.x;
        } else if (Sv < lo - 1e-6f * fmaxf(fabsf(lo), 1e-3f)) {
            if (sh.SL[s] < lo) {
                // the root lies below L: this sector from global memory
                sh.gs[s] = sh.sec[s];
                sh.ce[s] = sh.cb[s];
                sh.sumlo[s] = 0.f;
            }
            Root E;
            const float w = sh.wl[s];
            root_init(E, (w < nu && w > -FLT_MAX) ? w : nu, 0.05f * rho + 1e-6f);
            E.b = nu;
            for (int it = 0; it < PROX_MAXIT && !E.done; ++it) {
                float sum; int cnt;
                lane_sector_eval(D, sh, G, s, E.x, irho, sum, cnt);
                root_update(E, sum - lo, cnt, rho, 1e-6f * fmaxf(fabsf(lo), 1e-3f));
            }
            el = E.x;
        }
        sh.eta_hi[s] = eh;
        sh.eta_lo[s] = el;
    }
    if (lane == 0) sh.nu = nu;
}

// Everything after the streaming pass: the budget root, the edge roots of the sectors that
// bind, the writes of the kept and global-memory entries, the residuals and the control.
// Block-collective. sh holds the pass's sector sums at L (SL, CL, sumlo) and slot ranges.
// mask != null: the pass ran in the x-update's epilogue (k_tc_xprox), which already wrote
// every entry pinned at L (mask bit clear) and put its residuals into res; such an entry of a
// global-memory range is skipped here unless its sector is recomputed below L.
// In that case the slots also carry mu_i, d_i and their sector (smu, sdd, ssec; nslots of
// them, in sector order), and they are written by one block-wide pass.
__device__ void stream_tail(const Dev& D, StreamShared& sh, const GlobalSrc& G, int a, int j, float rho, float irho,
                            float nu0, float L, float margin, StreamRes& res, const unsigned* mask,
                            const float* smu = nullptr, const float* sdd = nullptr, const uint8_t* ssec = nullptr,
                            int nslots = 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int NS = D.S;
    const size_t base = (size_t)a * D.Npad;
    __syncthreads();
    // ---- budget multiplier
    float TL = 0.f;
    for (int s = 0; s < NS; ++s) TL += fminf(fmaxf(sh.SL[s], sh.blo[s]), sh.bhi[s]);
    const bool below = !(TL >= 1.f - 1e-6f);           // the root lies below L (or T is not finite)
    bool redo_all = below;
    if (below) {
        // every sector from global memory; the entries written above are redone
        __syncthreads();
        for (int s = tid; s < NS; s += blockDim.x) {
            sh.gs[s] = sh.sec[s];
            sh.ce[s] = sh.cb[s];
            sh.sumlo[s] = 0.f;
        }
        __syncthreads();
    }
    bool compact = !below;
    for (int s = 0; s < NS; ++s) compact &= (sh.gs[s] == sh.sec[s + 1]);
    if (compact) {
        // every sector's entries are in shared memory: warp 0 solves the budget and the
        // edge equations with lane s owning sector s (and s + 32), no block barriers
        if (warp == 0) lane_solve(D, sh, G, a, L, TL, nu0, rho, irho);
        __syncthreads();
    }
    Root R;
    root_init(R, nu0, 0.05f * rho + 1e-6f);
    if (!below) R.a = L;
    float x_eval = NAN;
    if (compact) {
        R.x = sh.nu;
    } else
    if (!below && L > -INFINITY && TL <= 1.f + 1e-6f) {
        R.x = L;                                         // L itself solves the budget equation
        x_eval = L;
        for (int s = tid; s < NS; s += blockDim.x) { sh.Sx[s] = sh.SL[s]; sh.Cx[s] = sh.CL[s]; }
        __syncthreads();
    } else {
        for (int it = 0; it < PROX_MAXIT; ++it) {
            for (int s = warp; s < NS; s += SP_WARPS) {
                float sum; int cnt;
                stream_sector_eval(D, sh, G, s, R.x, irho, sum, cnt);
                if (lane == 0) { sh.Sx[s] = sum; sh.Cx[s] = cnt; }
            }
            __syncthreads();
            float T = 0.f;
            int Cn = 0;
            for (int s = 0; s < NS; ++s) {
                const float v = sh.Sx[s];
                T += fminf(fmaxf(v, sh.blo[s]), sh.bhi[s]);
                if (v > sh.blo[s] && v < sh.bhi[s]) Cn += sh.Cx[s];
            }
            __syncthreads();
            x_eval = R.x;
            root_update(R, T - 1.f, Cn, rho, 1e-6f);
            if (D.stats && tid == 0) atomicAdd(D.stats + 2, 1ull);
            if (R.done) break;
        }
        if (R.x != x_eval) {
            for (int s = warp; s < NS; s += SP_WARPS) {
                float sum; int cnt;
                stream_sector_eval(D, sh, G, s, R.x, irho, sum, cnt);
                if (lane == 0) { sh.Sx[s] = sum; sh.Cx[s] = cnt; }
            }
            __syncthreads();
        }
    }
    const float nu = R.x;
    // ---- edge roots of the sectors that bind (warp per sector), then the kept and
    // global-memory entries of the sector
    int redo_mine = 0;
    for (int s = warp; s < NS; s += SP_WARPS) {
        float eh = -FLT_MAX, el = FLT_MAX;
        bool sec_redo = redo_all;           // every entry of the sector is recomputed below L
        const float Sv = compact ? 0.f : sh.Sx[s];
        const float hi = sh.bhi[s], lo = sh.blo[s];
        const int p0 = sh.sec[s], p1 = sh.sec[s + 1];
        if (compact) {
            eh = sh.eta_hi[s];
            el = sh.eta_lo[s];
            if (sh.gs[s] == p0 && p1 > p0) { redo_mine = 1; sec_redo = true; }   // a lower edge below L, redone in global memory
        } else if (Sv > hi + 1e-6f * fmaxf(hi, 1e-3f)) {
            Root E;
            const float w = sh.wh[s];
            root_init(E, (w > nu && w < FLT_MAX) ? w : nu, 0.05f * rho + 1e-6f);
            E.a = nu;
            int it = 0;
            for (; it < PROX_MAXIT && !E.done; ++it) {
                float sum; int cnt;
                stream_sector_eval(D, sh, G, s, E.x, irho, sum, cnt);
                root_update(E, sum - hi, cnt, rho, 1e-6f * fmaxf(hi, 1e-3f));
            }
            if (D.stats && lane == 0) atomicAdd(D.stats + 1, (unsigned long long)it);
            eh = E.x;
        } else if (Sv < lo - 1e-6f * fmaxf(fabsf(lo), 1e-3f)) {
            if (!redo_all && sh.SL[s] < lo) {
                // this sector's root lies below L: all of it from global memory
                __syncwarp();
                if (lane == 0) { sh.gs[s] = p0; sh.ce[s] = sh.cb[s]; sh.sumlo[s] = 0.f; }
                __syncwarp();
                redo_mine = 1;
                sec_redo = true;
            }
            Root E;
            const float w = sh.wl[s];
            root_init(E, (w < nu && w > -FLT_MAX) ? w : nu, 0.05f * rho + 1e-6f);
            E.b = nu;
            for (int it = 0; it < PROX_MAXIT && !E.done; ++it) {
                float sum; int cnt;
                stream_sector_eval(D, sh, G, s, E.x, irho, sum, cnt);
                root_update(E, sum - lo, cnt, rho, 1e-6f * fmaxf(fabsf(lo), 1e-3f));
            }
            el = E.x;
        }
        if (lane == 0) { sh.eta_hi[s] = eh; sh.eta_lo[s] = el; }
        if (D.stats && lane == 0 && sh.gs[s] < p1) atomicAdd(D.stats + 3, 1ull);
        const float arg = fminf(fmaxf(nu, eh), el);
        if (!mask) {
            for (int q = sh.cb[s] + lane; q < sh.ce[s]; q += 32) {
                const int p = sh.pos[q];
                const float z = eval_l1(sh.v[q], sh.w0[q], sh.lo[q], sh.up[q], sh.k[q], arg, irho).z;
                res.put(D, base + p, z, sh.v[q], sh.zo[q], sh.yo[q], D.mu32[p], D.d32[p], rho, irho);
            }
        }
        for (int p = sh.gs[s] + lane; p < p1; p += 32) {
            if (mask && !sec_redo && !((mask[p >> 5] >> (p & 31)) & 1u)) continue;   // written by the pass
            const float z = eval_entry(D, G, p, arg, 0.f, irho).z;
            const size_t e = base + p;
            res.put(D, e, z, G.val(p), D.z[e], D.y[e], D.mu32[p], D.d32[p], rho, irho);
        }
    }
    if (mask) {
        // the kept entries, every slot by its own thread (a slot of a sector that was moved
        // to global memory above lies outside its sector's range and was written there). With
        // the products folded the slot's X replaces its v in shared memory (the caller adds the
        // slots' share of B'X); otherwise it is stored
        __syncthreads();
        for (int q = tid; q < nslots; q += blockDim.x) {
            const int s = ssec[q];
            if (q >= sh.ce[s]) continue;
            const float arg = fminf(fmaxf(nu, sh.eta_hi[s]), sh.eta_lo[s]);
            const float z = eval_l1(sh.v[q], sh.w0[q], sh.lo[q], sh.up[q], sh.k[q], arg, irho).z;
            const float X = res.put_zy(D, base + sh.pos[q], z, sh.v[q], sh.zo[q], sh.yo[q], smu[q], sdd[q], rho, irho);
            if (D.fold) sh.v[q] = X;
            else store_X(D, base + sh.pos[q], X);
        }
    }
    float rp = warp_max(res.rp), rd = warp_max(res.rd), nx = warp_max(res.nx), nz = warp_max(res.nz),
          ny = warp_max(res.ny);
    int bad = warp_sum(res.bad) > 0 ? 1 : 0;
    redo_mine = warp_sum(redo_mine);
    if (lane == 0) {
        sh.red5[0][warp] = rp; sh.red5[1][warp] = rd; sh.red5[2][warp] = nx; sh.red5[3][warp] = nz;
        sh.red5[4][warp] = ny; sh.red_bad[warp] = bad | (redo_mine ? 2 : 0);
    }
    __syncthreads();
    if (tid == 0) {
        int redo = redo_all ? 1 : 0;
        bad = bad & 1;
        redo |= sh.red_bad[0] >> 1;
        for (int w = 1; w < SP_WARPS; ++w) {
            rp = fmaxf(rp, sh.red5[0][w]); rd = fmaxf(rd, sh.red5[1][w]); nx = fmaxf(nx, sh.red5[2][w]);
            nz = fmaxf(nz, sh.red5[3][w]); ny = fmaxf(ny, sh.red5[4][w]);
            bad |= sh.red_bad[w] & 1;
            redo |= sh.red_bad[w] >> 1;
        }
        if (redo) { rp = INFINITY; rd = INFINITY; }    // entries were rewritten: no residual this call
        sh.redo = redo;
        const int it = sh.it0 + 1;
        D.iters[a] = it;
        if (D.stats) atomicAdd(D.stats, 1ull);
        D.rp[a] = rp;
        D.rd[a] = rd;
        D.nu[a] = nu;
        D.theta[a] = 0.f;
        // the next call's margin: four times the last move of nu, or more after a miss
        D.dnu[a] = redo ? fmaxf(fabsf(nu - nu0), margin) : fabsf(nu - nu0);
        int newj = j;
        sh.cont = 0;
        if (bad) {
            D.status[a] = PRISM_NUMERICAL_FAILURE;
            D.active[a] = 0;
        } else if (it >= D.min_iter && fmaxf(rp, D.rps ? D.rps[a] : 0.f) <= D.eps_admm &&
                   fmaxf(rd, D.rds ? D.rds[a] : 0.f) <= D.eps_admm) {
            D.active[a] = 0;
        } else if (it >= D.max_iter) {
            D.active[a] = 0;
            D.status[a] = PRISM_TIMEOUT;
        } else {
            sh.cont = 1;
            if (!redo && it % D.adapt_every == 0) {
                const float pr = rp / fmaxf(fmaxf(nx, nz), 1e-12f);
                const float du = rd / fmaxf(ny, 1e-12f);
                const float ratio = sqrtf(pr / fmaxf(du, 1e-20f));
                int dj = int(lrintf(float(RHO_PER_DECADE) * log10f(fmaxf(ratio, 1e-12f))));
                dj = max(-4, min(4, dj));
                newj = max(0, min(NRHO - 1, j + dj));
            }
        }
        sh.newj = newj;
    }
    __syncthreads();
    const int newj = sh.newj;
    for (int s = tid; s < NS; s += blockDim.x) {
        D.eta_hi[a * NS + s] = sh.eta_hi[s];
        D.eta_lo[a * NS + s] = sh.eta_lo[s];
    }
    if (newj != j) {
        if (tid == 0) D.rho_idx[a] = newj;
        if (!(mask && D.fold)) {
            // (with the products folded the caller rewrites X itself: entries the pass pinned hold none)
            const float rn = rho_val(newj);
            for (int p = tid; p < D.N; p += blockDim.x) {
                const size_t e = base + p;
                store_X(D, e, (D.mu32[p] + rn * D.z[e] - D.y[e]) / (2.f * D.d32[p] + rn));
            }
        }
    }
}

__global__ void __launch_bounds__(32 * SP_WARPS, 4) k_prox_stream(Dev D) {
    const int a = blockIdx.x;
    if (!D.active[a]) return;
    extern __shared__ float4 dyn4[];
    StreamShared& sh = *reinterpret_cast<StreamShared*>(dyn4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int NS = D.S;
    const unsigned lt = (1u << lane) - 1u;
    for (int s = tid; s < NS; s += blockDim.x) {
        sh.blo[s] = D.band_lo[a * NS + s];
        sh.bhi[s] = D.band_hi[a * NS + s];
    }
    for (int s = tid; s <= NS; s += blockDim.x) sh.sec[s] = D.sec_start[s];
    for (int s = tid; s < NS; s += blockDim.x) { sh.wh[s] = D.eta_hi[a * NS + s]; sh.wl[s] = D.eta_lo[a * NS + s]; }
    if (tid == 0) sh.it0 = D.iters[a];
    __syncthreads();
    const size_t base = (size_t)a * D.Npad;
    const GlobalSrc G(D, base);
    const int j = D.rho_idx[a];
    const float rho = rho_val(j), irho = 1.f / rho;
    const float nu0 = D.nu[a];
    const float margin = fmaxf(4.f * D.dnu[a], 2e-3f);  // in units of nu (a price), not of weights
    const float L = nu0 - margin;
    StreamRes res;
    // ---- the streaming pass: every entry is evaluated at L; entries pinned at l are final
    constexpr int CH = 4;
    int wcnt = 0;                                   // slots used by this warp (uniform)
    for (int s = warp; s < NS; s += SP_WARPS) {
        const int p0 = sh.sec[s], p1 = sh.sec[s + 1];
        const int start = wcnt;
        int gs = p1;
        float sL = 0.f, slo = 0.f;
        int cL = 0;
        for (int pb = p0 + lane; pb - lane < p1; pb += 32 * CH) {
            float vv[CH], w0v[CH], lov[CH], upv[CH], cv[CH], zo[CH], yo[CH], mu[CH], dd[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int p = pb + 32 * c;
                const bool in = p < p1;
                vv[c] = in ? G.v[p] : 0.f;
                w0v[c] = in ? G.w0[p] : 0.f;
                lov[c] = in ? G.lo[p] : 0.f;
                upv[c] = in ? G.up[p] : 0.f;
                cv[c] = in ? G.c[p] : 0.f;
                zo[c] = in ? D.z[base + p] : 0.f;
                yo[c] = in ? D.y[base + p] : 0.f;
                mu[c] = in ? D.mu32[p] : 0.f;
                dd[c] = in ? D.d32[p] : 1.f;
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int p = pb + 32 * c;
                const bool in = p < p1;
                const float k = cv[c] * irho;
                const EntryEval r = eval_l1(vv[c], w0v[c], lov[c], upv[c], k, L, irho);
                const bool pinned = in && r.z == lov[c];
                if (in) { sL += r.z; cL += r.lin; }
                const int batch0 = pb - lane + 32 * c;   // first position of this row of the batch
                if (batch0 >= gs) continue;             // the rest of the sector reads global memory later
                const bool keep = in && !pinned;
                const unsigned b = __ballot_sync(0xffffffffu, keep);
                if (wcnt + __popc(b) > SP_CW) {
                    gs = batch0;                        // overflow: from here on, global memory
                    continue;
                }
                if (keep) {
                    const int q = warp * SP_CW + wcnt + __popc(b & lt);
                    sh.v[q] = vv[c]; sh.w0[q] = w0v[c]; sh.lo[q] = lov[c]; sh.up[q] = upv[c]; sh.k[q] = k;
                    sh.zo[q] = zo[c]; sh.yo[q] = yo[c]; sh.pos[q] = p;
                }
                wcnt += __popc(b);
                if (pinned) {
                    slo += lov[c];
                    res.put(D, base + p, lov[c], vv[c], zo[c], yo[c], mu[c], dd[c], rho, irho);
                }
            }
        }
        sL = warp_sum(sL);
        slo = warp_sum(slo);
        cL = warp_sum(cL);
        if (lane == 0) {
            sh.SL[s] = sL; sh.CL[s] = cL; sh.sumlo[s] = slo; sh.gs[s] = gs;
            sh.cb[s] = warp * SP_CW + start;
            sh.ce[s] = warp * SP_CW + wcnt;
        }
    }
    stream_tail(D, sh, G, a, j, rho, irho, nu0, L, margin, res, nullptr);
}

// ---------------------------------------------------------------------------
// G5/G6 after the fused pass (k_tc_xprox). That kernel evaluated every entry at L inside
// the x-update's epilogue, wrote v for all entries and z, y, X for the entries pinned at
// their lower bound, and left per-quarter candidate masks, per-tile residual maxima and (when
// l differs over the account) per-segment sums of l over the pinned entries. Here, one block
// per active account: the candidates (mask bits) are gathered into the shared-memory slots of
// their sectors in position order, the sector sums at L are formed from them in a fixed
// order, and the rest is the streaming form's tail.
// ---------------------------------------------------------------------------
struct RootsShared {
    StreamShared st;
    float mu[SP_WARPS * SP_CW], dd[SP_WARPS * SP_CW];   // mu_i, d_i of each slot
    uint8_t ssec[SP_WARPS * SP_CW];                     // sector of each slot
    int nslots;
    unsigned mask[XP_NQMAX];
    int qoff[XP_NQMAX];                 // candidates before quarter q
    int rank0[SMAX];                    // candidates before the first position of sector s
    int wsum[SP_WARPS];
    int total;
    int all_fit;                        // every sector's candidates are in slots (slot = rank)
};

__device__ __forceinline__ int cand_rank(const RootsShared& R, int nq, int p) {
    const int q = p >> 5;
    if (q >= nq) return R.total;
    return R.qoff[q] + __popc(R.mask[q] & ((1u << (p & 31)) - 1u));
}

// P = B'X of account a for the next iteration, then its Q (G2 and G3 folded into the fused
// iteration): the fused pass's partial sets hold the entries it pinned (tensor-core products,
// X split into two BF16 terms), and the slots, whose X the tail left in place of their v, add
// X_q B_q here (FP32, B in its BF16 rounding as in the products). Fixed summation order.
static_assert(sizeof(SolveScratch) <= sizeof(float) * SP_WARPS * SP_CW, "the solve's scratch fits in a slot array");

// X of every entry of account a at penalty index j, and the flag that sends the account through
// the product kernels of the next iteration
__device__ __noinline__ void rewrite_X(const Dev& D, int a, int j) {
    const size_t base = (size_t)a * D.Npad;
    const float rn = rho_val(j);
    for (int p = threadIdx.x; p < D.N; p += blockDim.x) {
        const size_t e = base + p;
        store_X(D, e, (D.mu32[p] + rn * D.z[e] - D.y[e]) / (2.f * D.d32[p] + rn));
    }
    if (threadIdx.x == 0) D.needP[a] = 1;
}

__device__ __noinline__ void fold_P_solve(const Dev& D, const RootsShared& R, StreamShared& sh, int a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    float* red = sh.w0;                          // [SP_WARPS][KMAX]; the slot arrays are free now
    const __nv_bfloat162* B2 = reinterpret_cast<const __nv_bfloat162*>(D.B16p);
    float a0 = 0.f, a1 = 0.f;
    const int n = R.nslots;
    int q = warp;
    for (; q + 3 * SP_WARPS < n; q += 4 * SP_WARPS) {
        float2 b[4];
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int qq = q + u * SP_WARPS;
            b[u] = __bfloat1622float2(B2[(size_t)sh.pos[qq] * (KMAX / 2) + lane]);
            x[u] = sh.v[qq];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) { a0 = fmaf(b[u].x, x[u], a0); a1 = fmaf(b[u].y, x[u], a1); }
    }
    for (; q < n; q += SP_WARPS) {
        const float2 b = __bfloat1622float2(B2[(size_t)sh.pos[q] * (KMAX / 2) + lane]);
        a0 = fmaf(b.x, sh.v[q], a0);
        a1 = fmaf(b.y, sh.v[q], a1);
    }
#pragma unroll 4
    for (int set = warp; set < D.xp_sets; set += SP_WARPS) {
        const float2 pp = reinterpret_cast<const float2*>(D.Pxp + ((size_t)set * D.M + a) * KMAX)[lane];
        a0 += pp.x;
        a1 += pp.y;
    }
    red[warp * KMAX + 2 * lane] = a0;
    red[warp * KMAX + 2 * lane + 1] = a1;
    __syncthreads();
    float* sP = sh.up;
    if (tid < KMAX) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < SP_WARPS; ++w) t += red[w * KMAX + tid];
        sP[tid] = t;
    }
    __syncthreads();
    solve_K<4>(D, a, sP, *reinterpret_cast<SolveScratch*>(sh.k), nullptr);
}

__global__ void __launch_bounds__(32 * SP_WARPS, 4) k_prox_roots(Dev D) {
    const int a = D.m0 + blockIdx.x;
    if (!D.active[a]) return;
    extern __shared__ float4 dyn4[];
    RootsShared& R = *reinterpret_cast<RootsShared*>(dyn4);
    StreamShared& sh = R.st;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int NS = D.S, M = D.M, nq = D.nq;
    for (int s = tid; s < NS; s += blockDim.x) {
        sh.blo[s] = D.band_lo[a * NS + s];
        sh.bhi[s] = D.band_hi[a * NS + s];
    }
    for (int s = tid; s <= NS; s += blockDim.x) sh.sec[s] = D.sec_start[s];
    for (int s = tid; s < NS; s += blockDim.x) { sh.wh[s] = D.eta_hi[a * NS + s]; sh.wl[s] = D.eta_lo[a * NS + s]; }
    if (tid == 0) sh.it0 = D.iters[a];
    const size_t base = (size_t)a * D.Npad;
    GlobalSrc G(D, base);
    const int j = D.rho_idx[a];
    const float rho = rho_val(j), irho = 1.f / rho;
    const float nu0 = D.nu[a];
    const float margin = fmaxf(4.f * D.dnu[a], 2e-3f);
    const float L = nu0 - margin;
    // the fused pass wrote v only for its candidates: a pinned entry's v comes from its new y
    G.cm = R.mask;
    G.yv = D.y + base;
    G.irho = irho;
    pdl_wait();                            // the masks, residuals and records of the fused pass
    pdl_trigger();
    // candidate masks and their exclusive prefix counts (four quarters per thread)
    unsigned w4[4];
    int c4 = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int q = 4 * tid + u;
        w4[u] = q < nq ? D.Cm[(size_t)a * nq + q] : 0u;
        c4 += __popc(w4[u]);
    }
    int incl = c4;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) R.wsum[warp] = incl;
    // residual maxima of the pinned entries, per asset tile
    StreamRes res;
    for (int t = tid; t < D.nt; t += blockDim.x) {
        float r5[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) r5[k] = D.Rt[((size_t)a * 5 + k) * D.nt + t];
        if (isnan(r5[0])) res.bad = 1;
        else res.rp = fmaxf(res.rp, r5[0]);
        res.rd = fmaxf(res.rd, r5[1]); res.nx = fmaxf(res.nx, r5[2]);
        res.nz = fmaxf(res.nz, r5[3]); res.ny = fmaxf(res.ny, r5[4]);
    }
    __syncthreads();
    // exclusive prefix counts per quarter; each candidate's position goes to the slot of its
    // rank, which is its final slot whenever every sector fits (the common case)
    constexpr int CAP = SP_WARPS * SP_CW;
    {
        int off = incl - c4;
        for (int w = 0; w < warp; ++w) off += R.wsum[w];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = 4 * tid + u;
            if (q < nq) { R.mask[q] = w4[u]; R.qoff[q] = off; }
            unsigned w = w4[u];
            int r = off;
            while (w) {
                const int b = __ffs(w) - 1;
                w &= w - 1u;
                if (r < CAP) sh.pos[r] = 32 * q + b;
                ++r;
            }
            off += __popc(w4[u]);
        }
        if (tid == blockDim.x - 1) R.total = off;
    }
    // the sum of l over each sector's pinned entries when l differs over the account: the
    // pass's segment sums (fixed order: lane g, then the warp sum)
    const float lo_u = D.lo_u[a], c_u = D.c_u[a];
    if (isnan(lo_u)) {
        for (int s = warp; s < NS; s += SP_WARPS) {
            float so = 0.f;
            for (int g = D.sseg[s] + lane; g < D.sseg[s + 1]; g += 32) so += D.SOp[(size_t)g * M + a];
            so = warp_sum(so);
            if (lane == 0) sh.sumlo[s] = so;
        }
    }
    __syncthreads();
    // gather the candidates' records into the rank slots (all loads issued first), and in the
    // meantime thread 0 lays out the slot ranges: sectors in order while the slots last; a
    // sector that does not fit is evaluated from global memory (v is there for every entry)
    const int nfit = min(R.total, CAP);
    if (D.pcount && tid == 0) {
        atomicAdd(D.pcount, (unsigned long long)R.total);
        atomicAdd(D.pcount + 1, (unsigned long long)D.N);
    }
    const float4* recs = reinterpret_cast<const float4*>(D.crec) + 2 * base;
    auto gather = [&](int slot, int p, int s) {
        const float4 r0 = recs[2 * (size_t)p], r1 = recs[2 * (size_t)p + 1];
        sh.v[slot] = r0.x; sh.w0[slot] = r0.y; sh.up[slot] = r0.z; sh.zo[slot] = r0.w; sh.yo[slot] = r1.x;
        R.mu[slot] = r1.y; R.dd[slot] = r1.z; R.ssec[slot] = (uint8_t)s;
        sh.lo[slot] = isnan(lo_u) ? G.lo[p] : lo_u;
        sh.k[slot] = (isnan(c_u) ? G.c[p] : c_u) * irho;
    };
    for (int r0 = tid; r0 < nfit; r0 += 4 * blockDim.x) {
        int pp[4];
        float4 ra[4], rb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * blockDim.x;
            pp[u] = r < nfit ? sh.pos[r] : -1;
            if (pp[u] >= 0) { ra[u] = recs[2 * (size_t)pp[u]]; rb[u] = recs[2 * (size_t)pp[u] + 1]; }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (pp[u] < 0) continue;
            const int r = r0 + u * blockDim.x, p = pp[u];
            // the sector of position p: the last s with sec[s] <= p
            int lo_s = 0, hi_s = NS - 1;
            while (lo_s < hi_s) {
                const int mid = (lo_s + hi_s + 1) >> 1;
                if (sh.sec[mid] <= p) lo_s = mid; else hi_s = mid - 1;
            }
            sh.v[r] = ra[u].x; sh.w0[r] = ra[u].y; sh.up[r] = ra[u].z; sh.zo[r] = ra[u].w; sh.yo[r] = rb[u].x;
            R.mu[r] = rb[u].y; R.dd[r] = rb[u].z; R.ssec[r] = (uint8_t)lo_s;
            sh.lo[r] = isnan(lo_u) ? G.lo[p] : lo_u;
            sh.k[r] = (isnan(c_u) ? G.c[p] : c_u) * irho;
        }
    }
    if (warp == 0) {
        // warp 0, lane s over sectors s and s + 32: the candidates of each sector (from the
        // ranks of its end positions), their prefix over the sectors in order, and the slot
        // ranges; when they all fit (the common case) every sector takes its own candidates'
        // slots, else lane 0 lays the sectors out in order while the slots last
        static_assert(SMAX <= 64, "two sectors per lane");
        int r0[2], n[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int sct = lane + 32 * h;
            r0[h] = 0; n[h] = 0;
            if (sct < NS) {
                r0[h] = cand_rank(R, nq, sh.sec[sct]);
                n[h] = cand_rank(R, nq, sh.sec[sct + 1]) - r0[h];
            }
        }
        int ex[2], tot = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int inc = n[h];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            ex[h] = tot + inc - n[h];
            tot += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (tot <= CAP) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int sct = lane + 32 * h;
                if (sct >= NS) continue;
                const int p0 = sh.sec[sct], p1 = sh.sec[sct + 1];
                R.rank0[sct] = r0[h];
                if (!isnan(lo_u)) sh.sumlo[sct] = lo_u * float(p1 - p0 - n[h]);
                sh.cb[sct] = ex[h];
                sh.ce[sct] = ex[h] + n[h];
                sh.gs[sct] = p1;
            }
            if (lane == 0) {
                R.all_fit = (tot == R.total);
                R.nslots = tot;
            }
        } else if (lane == 0) {
            int used = 0;
            for (int sct = 0; sct < NS; ++sct) {
                const int p0 = sh.sec[sct], p1 = sh.sec[sct + 1];
                const int q0 = cand_rank(R, nq, p0), nn = cand_rank(R, nq, p1) - q0;
                R.rank0[sct] = q0;
                if (!isnan(lo_u)) sh.sumlo[sct] = lo_u * float(p1 - p0 - nn);
                sh.cb[sct] = used;
                if (used + nn <= CAP) {
                    sh.ce[sct] = used + nn;
                    sh.gs[sct] = p1;
                    used += nn;
                } else {
                    sh.ce[sct] = used;
                    sh.gs[sct] = p0;
                    sh.sumlo[sct] = 0.f;
                }
            }
            R.all_fit = (used == R.total);
            R.nslots = used;
        }
    }
    __syncthreads();
    const bool all_fit = R.all_fit;
    if (!all_fit) {
        // a sector did not fit: the slots of the later sectors move down (rare)
        __syncthreads();
        for (int q = tid; q < nq; q += blockDim.x) {
            unsigned w = R.mask[q];
            const int qo = R.qoff[q];
            while (w) {
                const int b = __ffs(w) - 1;
                w &= w - 1u;
                const int p = 32 * q + b;
                const int s = D.sector[p];
                if (s < 0 || sh.gs[s] != sh.sec[s + 1]) continue;
                const int rank = qo + __popc(R.mask[q] & ((1u << b) - 1u));
                const int slot = sh.cb[s] + rank - R.rank0[s];
                if (slot < rank || rank >= CAP) {   // still unwritten or moved: rewrite it here
                    gather(slot, p, s);
                    sh.pos[slot] = p;
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0 && !isnan(lo_u) && R.total < D.N) res.nz = fmaxf(res.nz, fabsf(lo_u));   // pinned z = l
    // S_s(L) and the linear count at L, from the candidates (the pinned entries add sumlo):
    // a thread per sector over its slots; a sector in global memory by a warp
    if (tid < NS && sh.gs[tid] == sh.sec[tid + 1]) {
        float acc = sh.sumlo[tid];
        int n = 0;
        for (int q = sh.cb[tid]; q < sh.ce[tid]; ++q) {
            const EntryEval r = eval_l1(sh.v[q], sh.w0[q], sh.lo[q], sh.up[q], sh.k[q], L, irho);
            acc += r.z;
            n += r.lin;
        }
        sh.SL[tid] = acc;
        sh.CL[tid] = n;
    }
    if (!all_fit) {
        for (int s = warp; s < NS; s += SP_WARPS) {
            if (sh.gs[s] == sh.sec[s + 1]) continue;
            float sum;
            int cnt;
            stream_sector_eval(D, sh, G, s, L, irho, sum, cnt);
            if (lane == 0) { sh.SL[s] = sum; sh.CL[s] = cnt; }
        }
    }
    stream_tail(D, sh, G, a, j, rho, irho, nu0, L, margin, res, R.mask, R.mu, R.dd, R.ssec, R.nslots);
    // ---- the next iteration's P and Q of this account (products folded)
    if (!D.fold) return;
    __syncthreads();
    if (!sh.cont) return;
    const int newj = sh.newj;
    if (sh.redo || newj != j || !all_fit) {
        // P cannot be completed from the pass's partials (the penalty changed, entries the pass
        // pinned were rewritten, or a sector's candidates were read from global memory): X of
        // every entry at the penalty of the next iteration, for its product kernels
        rewrite_X(D, a, newj);
        return;
    }
    if (tid == 0) D.needP[a] = 0;
    fold_P_solve(D, R, sh, a);
}

size_t prox_roots_smem_bytes() { return sizeof(RootsShared); }

void launch_prox_roots(const Dev& D, cudaStream_t st, bool pdl) {
    const size_t smem = sizeof(RootsShared);
    cudaFuncSetAttribute(k_prox_roots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_ex(k_prox_roots, dim3((D.m1 ? D.m1 : D.M) - D.m0), dim3(32 * SP_WARPS), smem, st, pdl, D);
}

// Per account: l when it is the same at every position (else NaN), and c when it is the
// same at every position with u > l (else NaN; an entry with u = l is l whatever c is).
__global__ void k_uniform(Dev D, float* lo_u, float* c_u) {
    const int a = blockIdx.x;
    const size_t base = (size_t)a * D.Npad;
    float lmin = FLT_MAX, lmax = -FLT_MAX, cmin = FLT_MAX, cmax = -FLT_MAX;
    for (int p = threadIdx.x; p < D.N; p += blockDim.x) {
        const float l = D.lo[base + p], u = D.up[base + p];
        lmin = fminf(lmin, l); lmax = fmaxf(lmax, l);
        if (u > l) { const float c = D.c[base + p]; cmin = fminf(cmin, c); cmax = fmaxf(cmax, c); }
    }
    __shared__ float red[4][32];
    lmin = warp_min(lmin); lmax = warp_max(lmax); cmin = warp_min(cmin); cmax = warp_max(cmax);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = lmin; red[1][warp] = lmax; red[2][warp] = cmin; red[3][warp] = cmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lmin = fminf(lmin, red[0][w]); lmax = fmaxf(lmax, red[1][w]);
            cmin = fminf(cmin, red[2][w]); cmax = fmaxf(cmax, red[3][w]);
        }
        lo_u[a] = (lmin == lmax) ? lmin : NAN;
        c_u[a] = (cmin > cmax) ? 0.f : ((cmin == cmax) ? cmin : NAN);
    }
}

void launch_uniform(const Dev& D, float* lo_u, float* c_u, cudaStream_t st) {
    k_uniform<<<D.M, 256, 0, st>>>(D, lo_u, c_u);
}

size_t prox_stream_smem_bytes(const Dev&) { return sizeof(StreamShared); }

size_t prox_smem_bytes(const Dev& D) {
    return (size_t)D.Npad * 4 * (5 + (D.pw_idx ? 1 : 0));
}

void launch_prox(const Dev& D, cudaStream_t st, bool cold) {
    if (D.stream_prox && !cold) {
        const size_t smem = prox_stream_smem_bytes(D);
        cudaFuncSetAttribute(k_prox_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_prox_stream<<<D.M, 32 * SP_WARPS, smem, st>>>(D);
        return;
    }
    const int nw = std::min(20, std::max(4, D.S));      // at most 640 threads: warps loop over sectors
    const size_t smem = prox_smem_bytes(D);
    const size_t limit = 227 * 1024 - sizeof(ProxShared) - 1024;
    if (smem <= limit) {
        cudaFuncSetAttribute(k_prox_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_prox_smem<<<D.M, 32 * nw, smem, st>>>(D);
    } else {
        k_prox<<<D.M, 32 * nw, 0, st>>>(D);
    }
}

// X = Delta^{-1} (mu + rho z - y) of every entry of the accounts still iterating (the fused
// iteration keeps no X of the entries it pins: a return to the iterations rebuilds it)
__global__ void k_refresh_X(Dev D) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)D.M * D.Npad) return;
    const int a = int(e / D.Npad), p = int(e % D.Npad);
    if (!D.active[a] || p >= D.N) return;
    const float rho = rho_val(D.rho_idx[a]);
    store_X(D, e, (D.mu32[p] + rho * D.z[e] - D.y[e]) / (2.f * D.d32[p] + rho));
}

void launch_refresh_X(const Dev& D, cudaStream_t st) {
    k_refresh_X<<<(unsigned)cdiv64((int64_t)D.M * D.Npad, 256), 256, 0, st>>>(D);
}

__global__ void k_count_active(Dev D) {
    __shared__ int s[32];
    int n = 0;
    for (int a = threadIdx.x; a < D.M; a += blockDim.x) n += D.active[a];
    n = warp_sum(n);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        *D.n_active = t;
    }
}

void launch_count_active(const Dev& D, cudaStream_t st) { k_count_active<<<1, 1024, 0, st>>>(D); }

__global__ void k_mark_timeout(Dev D) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < D.M && D.active[a]) { D.active[a] = 0; D.status[a] = PRISM_TIMEOUT; }
}

void launch_mark_timeout(const Dev& D, cudaStream_t st) { k_mark_timeout<<<cdiv(D.M, 128), 128, 0, st>>>(D); }

}  // namespace prism
