// adjoint.cu -- implicit differentiation of the polished KKT system (the backward pass).
//
// At a certified solution the polish has identified, per account, the free weights F
// (strictly inside a linear piece of phi_i on [l_i, u_i]), the fixed ones and the
// working rows E (budget, bands held at an edge, the cap). The KKT conditions of
// Sec. 4.4 on that active set are linear in (w_F, lambda):
//
//     2 Sigma_FF w_F + E_F' lambda = mu_F - s_F - 2 Sigma_FA w_A,   E_F w_F = e - E_A w_A,
//
// with Sigma = B F B' + D (Eq. 1). For L = sum_a g_a' w_a, one adjoint solve per account
//
//     [2 Sigma_FF  E_F'] [u    ]   [g_F]
//     [E_F         0   ] [kappa] = [0  ]
//
// gives every gradient by the chain rule (u_i = 0 outside F, h = B'w, t = B_F' u):
//
//     dL/dmu_i = sum_a u_i,   dL/dd_i = -2 sum_a u_i w_i,
//     dL/dB_i  = -2 sum_a (u_i F h + w_i F t),
//     dL/dw0_i = g_i - 2 B_i . (F t) - kappa_budget - kappa_band(s(i))   (i fixed at a kink of phi,
//                                                                        which moves with w0_i)
//              = kappa_cap * sign(w_i - w0_i)                            (any other weight).
//
// The solve is the polish's Woodbury / Schur structure in FP64: C = F^{-1} + B_F' D_F^{-1} B_F
// (K x K Cholesky), Sigma_FF^{-1} X = D^{-1} X - D^{-1} B_F C^{-1} B_F' D^{-1} X for the columns
// [g_F, E_F'], the Schur complement E_F Sigma_FF^{-1} E_F' eliminated with diagonal pivoting
// (a dependent working row gets kappa = 0). Sums over accounts run in a fixed order.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "polish.h"

namespace prism {

namespace {

constexpr int AB = 256;                // threads per adjoint block (one block per account)
constexpr int AMAXROWS = PMAXROWS;     // working rows
constexpr int AYS = AMAXROWS + 1;      // row stride of Y: column 0 = g_F, columns 1..m = E_F'

struct AdjArgs {
    int M, N, Npad, K, S, fmax;
    const double *B64, *f64, *d64;
    const int* sector;
    const double* W;
    const uint8_t* flags;
    const int *wband, *wcap, *status;
    const double* G;                   // dL/dw in the sorted layout
    int *Flist, *NZlist;
    double* Y;
    double *U, *DW0, *Fh, *Ft;
    int* err;
};

struct AdjShared {
    double C[KMAX][KMAX + 1];
    double T[KMAX][AYS];
    double Ldinv[KMAX];
    double Sm[AMAXROWS][AMAXROWS + 1];
    double r[AMAXROWS], kappa[AMAXROWS];
    double ft[KMAX], fh[KMAX];
    int rows[AMAXROWS], used[AMAXROWS], order[AMAXROWS];
    int band_row[SMAX];
    int cntF[AB / 32], cntN[AB / 32];
    int nF, nNZ, m, nc, fail;
};

__device__ __forceinline__ double row_coef(const AdjArgs& A, const AdjShared& sh, int r, int p, uint8_t fl) {
    const int row = sh.rows[r];
    if (row < 0) return 1.0;                                    // budget
    if (row < A.S) return A.sector[p] == row ? 1.0 : 0.0;     // band
    return (fl & 4) ? 1.0 : ((fl & 8) ? -1.0 : 0.0);           // cap
}

__global__ void __launch_bounds__(AB) k_adjoint(AdjArgs A) {
    const int a = blockIdx.x;
    if (A.status[a] != PRISM_CERTIFIED) return;                // outputs stay zero
    extern __shared__ double adj_smem[];
    AdjShared& sh = *reinterpret_cast<AdjShared*>(adj_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = A.N, K = A.K, S = A.S;
    const size_t base = (size_t)a * A.Npad;
    const double* W = A.W + base;
    const uint8_t* FL = A.flags + base;
    int* Fl = A.Flist + (size_t)a * A.fmax;
    int* NZ = A.NZlist + base;
    double* Y = A.Y + (size_t)a * A.fmax * AYS;
    // ---- ordered lists of the free and the nonzero weights (warp tiles, ballots)
    const int Lw = cdiv(cdiv(N, AB / 32), 32) * 32;
    const int p0 = min(N, warp * Lw), p1 = min(N, p0 + Lw);
    {
        int nf = 0, nn = 0;
        for (int p = p0 + lane; p - lane < p1; p += 32) {
            const bool in = p < p1;
            nf += __popc(__ballot_sync(0xffffffffu, in && (FL[in ? p : 0] & 1)));
            nn += __popc(__ballot_sync(0xffffffffu, in && W[in ? p : 0] != 0.0));
        }
        if (lane == 0) { sh.cntF[warp] = nf; sh.cntN[warp] = nn; }
    }
    __syncthreads();
    if (tid == 0) {
        int of = 0, on = 0;
        for (int w = 0; w < AB / 32; ++w) {
            const int f = sh.cntF[w], n = sh.cntN[w];
            sh.cntF[w] = of; sh.cntN[w] = on;
            of += f; on += n;
        }
        sh.nF = of; sh.nNZ = on;
        int r = 0;
        sh.rows[r++] = -1;
        for (int s = 0; s < S; ++s) {
            sh.band_row[s] = -1;
            if (A.wband[a * S + s] != 0) { if (r < AMAXROWS) { sh.band_row[s] = r; sh.rows[r] = s; } ++r; }
        }
        if (A.wcap[a]) { if (r < AMAXROWS) sh.rows[r] = S; ++r; }
        sh.m = r;
        sh.fail = (of > A.fmax || r > AMAXROWS) ? 1 : 0;
    }
    __syncthreads();
    if (sh.fail) {
        if (tid == 0) atomicOr(A.err, 1);
        return;
    }
    {
        int of = sh.cntF[warp], on = sh.cntN[warp];
        const unsigned lt = (1u << lane) - 1u;
        for (int p = p0 + lane; p - lane < p1; p += 32) {
            const bool in = p < p1;
            const bool isF = in && (FL[in ? p : 0] & 1);
            const bool isN = in && W[in ? p : 0] != 0.0;
            const unsigned bF = __ballot_sync(0xffffffffu, isF), bN = __ballot_sync(0xffffffffu, isN);
            if (isF) Fl[of + __popc(bF & lt)] = p;
            if (isN) NZ[on + __popc(bN & lt)] = p;
            of += __popc(bF);
            on += __popc(bN);
        }
    }
    __syncthreads();
    const int nF = sh.nF, nNZ = sh.nNZ, m = sh.m, nc1 = 1 + m;
    // ---- right-hand sides scaled by D^{-1}: column 0 = g_F, columns 1..m = E_F'
    for (int q = tid; q < nF; q += AB) {
        const int p = Fl[q];
        const double di = 1.0 / A.d64[p];
        double* Yq = Y + (size_t)q * AYS;
        Yq[0] = A.G[base + p] * di;
        for (int r = 0; r < m; ++r) Yq[1 + r] = row_coef(A, sh, r, p, FL[p]) * di;
    }
    // ---- C = F^{-1} + B_F' D_F^{-1} B_F and its Cholesky factor (L D L', then L)
    for (int e2 = tid; e2 < K * K; e2 += AB) {
        const int r = e2 / K, c = e2 % K;
        if (c > r) continue;
        double acc = (r == c) ? 1.0 / A.f64[r] : 0.0;
        for (int q = 0; q < nF; ++q) {
            const int p = Fl[q];
            acc += A.B64[(size_t)p * K + r] * A.B64[(size_t)p * K + c] / A.d64[p];
        }
        sh.C[r][c] = acc;
    }
    __syncthreads();
    bool chol_ok = true;
    for (int c = 0; c < K; ++c) {
        const double piv = sh.C[c][c];
        if (!(piv > 0.0)) { chol_ok = false; break; }          // every thread reads the same pivot
        const double ip = 1.0 / piv;
        for (int r = c + 1 + warp; r < K; r += AB / 32) {
            const double lr = sh.C[r][c] * ip;
            for (int q = c + 1 + lane; q <= r; q += 32) sh.C[r][q] -= lr * sh.C[q][c];
        }
        __syncthreads();
    }
    if (!chol_ok) {
        if (tid == 0) atomicOr(A.err, 2);
        return;
    }
    for (int c = tid; c < K; c += AB) sh.Ldinv[c] = sqrt(sh.C[c][c]);
    __syncthreads();
    for (int e2 = tid; e2 < K * K; e2 += AB) {
        const int r = e2 / K, c = e2 % K;
        if (c < r) sh.C[r][c] /= sh.Ldinv[c];
    }
    __syncthreads();
    for (int c = tid; c < K; c += AB) { sh.C[c][c] = sh.Ldinv[c]; sh.Ldinv[c] = 1.0 / sh.Ldinv[c]; }
    // ---- Woodbury: Y <- Y - D^{-1} B_F C^{-1} B_F' Y
    for (int e2 = tid; e2 < K * nc1; e2 += AB) {
        const int k = e2 / nc1, c = e2 % nc1;
        double acc = 0.0;
        for (int q = 0; q < nF; ++q) acc += A.B64[(size_t)Fl[q] * K + k] * Y[(size_t)q * AYS + c];
        sh.T[k][c] = acc;
    }
    __syncthreads();
    for (int c = warp; c < nc1; c += AB / 32) {
        double v0 = lane < K ? sh.T[lane][c] : 0.0, v1 = lane + 32 < K ? sh.T[lane + 32][c] : 0.0;
        for (int r = 0; r < K; ++r) {
            const double x = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) * sh.Ldinv[r];
            if (lane > r) v0 -= sh.C[lane][r] * x;
            if (lane + 32 > r && lane + 32 < K) v1 -= sh.C[lane + 32][r] * x;
            if (lane == (r & 31)) { if (r < 32) v0 = x; else v1 = x; }
        }
        for (int r = K - 1; r >= 0; --r) {
            const double x = __shfl_sync(0xffffffffu, r < 32 ? v0 : v1, r & 31) * sh.Ldinv[r];
            if (lane < r) v0 -= sh.C[r][lane] * x;
            if (lane + 32 < r) v1 -= sh.C[r][lane + 32] * x;
            if (lane == (r & 31)) { if (r < 32) v0 = x; else v1 = x; }
        }
        if (lane < K) sh.T[lane][c] = v0;
        if (lane + 32 < K) sh.T[lane + 32][c] = v1;
    }
    __syncthreads();
    for (int e2 = tid; e2 < nF * nc1; e2 += AB) {
        const int q = e2 / nc1, c = e2 % nc1;
        const int p = Fl[q];
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += A.B64[(size_t)p * K + k] * sh.T[k][c];
        Y[(size_t)q * AYS + c] -= acc / A.d64[p];
    }
    __syncthreads();
    // ---- Schur complement S = E Y_E, r = E Y_g; pivoted elimination, kappa = S^+ r
    for (int e2 = tid; e2 < m * nc1; e2 += AB) {
        const int i = e2 / nc1, c = e2 % nc1;
        double acc = 0.0;
        for (int q = 0; q < nF; ++q) {
            const int p = Fl[q];
            acc += row_coef(A, sh, i, p, FL[p]) * Y[(size_t)q * AYS + c];
        }
        if (c == 0) sh.r[i] = acc; else sh.Sm[i][c - 1] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        double scale = 0.0;
        for (int i = 0; i < m; ++i) { sh.used[i] = 0; sh.kappa[i] = 0.0; scale = fmax(scale, fabs(sh.Sm[i][i])); }
        int nc = 0;
        for (int k = 0; k < m; ++k) {
            int pv = -1;
            double best = 1e-13 * scale;
            for (int j = 0; j < m; ++j)
                if (!sh.used[j] && fabs(sh.Sm[j][j]) > best) { best = fabs(sh.Sm[j][j]); pv = j; }
            if (pv < 0) break;                       // the remaining rows are dependent
            sh.used[pv] = 1;
            sh.order[nc++] = pv;
            for (int j = 0; j < m; ++j) {
                if (sh.used[j]) continue;
                const double fct = sh.Sm[j][pv] / sh.Sm[pv][pv];
                for (int l = 0; l < m; ++l)
                    if (!sh.used[l]) sh.Sm[j][l] -= fct * sh.Sm[pv][l];
                sh.r[j] -= fct * sh.r[pv];
            }
        }
        for (int k = nc - 1; k >= 0; --k) {
            const int pv = sh.order[k];
            double v = sh.r[pv];
            for (int kk = k + 1; kk < nc; ++kk) v -= sh.Sm[pv][sh.order[kk]] * sh.kappa[sh.order[kk]];
            sh.kappa[pv] = v / sh.Sm[pv][pv];
        }
        sh.nc = nc;
    }
    __syncthreads();
    // ---- u = 1/2 (Y_g - Y_E kappa), stored in U and (for t) in column 0 of Y
    for (int q = tid; q < nF; q += AB) {
        double* Yq = Y + (size_t)q * AYS;
        double acc = Yq[0];
        for (int j = 0; j < m; ++j) acc -= Yq[1 + j] * sh.kappa[j];
        const double u = 0.5 * acc;
        Yq[0] = u;
        A.U[base + Fl[q]] = u;
    }
    __syncthreads();
    // ---- F t = f o (B_F' u) and F h = f o (B' w)
    for (int k = tid; k < K; k += AB) {
        double t = 0.0, h = 0.0;
        for (int q = 0; q < nF; ++q) t += A.B64[(size_t)Fl[q] * K + k] * Y[(size_t)q * AYS];
        for (int q = 0; q < nNZ; ++q) h += A.B64[(size_t)NZ[q] * K + k] * W[NZ[q]];
        sh.ft[k] = A.f64[k] * t;
        sh.fh[k] = A.f64[k] * h;
        A.Ft[(size_t)a * K + k] = sh.ft[k];
        A.Fh[(size_t)a * K + k] = sh.fh[k];
    }
    __syncthreads();
    // ---- dL/dw0 of every entry of the account
    const int cap_row = A.wcap[a] ? m - 1 : -1;
    const double k_cap = cap_row >= 0 ? sh.kappa[cap_row] : 0.0;
    for (int p = tid; p < N; p += AB) {
        const uint8_t fl = FL[p];
        double v = 0.0;
        if (fl & 2) {
            double bt = 0.0;
            for (int k = 0; k < K; ++k) bt += A.B64[(size_t)p * K + k] * sh.ft[k];
            const int br = sh.band_row[A.sector[p]];
            v = A.G[base + p] - 2.0 * bt - sh.kappa[0] - (br >= 0 ? sh.kappa[br] : 0.0);
        } else if (cap_row >= 0) {
            v = k_cap * ((fl & 4) ? 1.0 : ((fl & 8) ? -1.0 : 0.0));
        }
        A.DW0[base + p] = v;
    }
}

// Sums over accounts (fixed order) and the return to the universe's asset order.
__global__ void k_adjoint_reduce(int M, int N, int Npad, int K, const int* perm, const double* U, const double* W,
                                 const double* Fh, const double* Ft, double* dmu, double* dd, double* dB) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * (K + 1)) return;
    const int p = int(e % N), k = int(e / N) - 1;     // k = -1: dmu and dd
    const int i = perm[p];
    if (k < 0) {
        double su = 0.0, sd = 0.0;
        for (int a = 0; a < M; ++a) {
            const double u = U[(size_t)a * Npad + p];
            su += u;
            sd += u * W[(size_t)a * Npad + p];
        }
        if (dmu) dmu[i] = su;
        if (dd) dd[i] = -2.0 * sd;
    } else if (dB) {
        double acc = 0.0;
        for (int a = 0; a < M; ++a)
            acc += U[(size_t)a * Npad + p] * Fh[(size_t)a * K + k] + W[(size_t)a * Npad + p] * Ft[(size_t)a * K + k];
        dB[(size_t)i * K + k] = -2.0 * acc;
    }
}

// ragged entry e -> (account, sorted position)
__device__ __forceinline__ size_t ragged_slot(const int64_t* offsets, const int32_t* asset_idx, const int* inv_perm,
                                              int M, int Npad, int64_t e) {
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offsets[mid] <= e) lo = mid; else hi = mid;
    }
    const int i = asset_idx ? asset_idx[e] : int(e - offsets[lo]);
    return (size_t)lo * Npad + inv_perm[i];
}

__global__ void k_adjoint_scatter(int M, int Npad, int64_t nnz, const int64_t* offsets, const int32_t* asset_idx,
                                  const int* inv_perm, const double* g, double* G) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    G[ragged_slot(offsets, asset_idx, inv_perm, M, Npad, e)] = g[e];
}

__global__ void k_adjoint_gather(int M, int Npad, int64_t nnz, const int64_t* offsets, const int32_t* asset_idx,
                                 const int* inv_perm, const double* DW0, double* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    out[e] = DW0[ragged_slot(offsets, asset_idx, inv_perm, M, Npad, e)];
}

template <class T>
bool dev_ptr(const T* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// Snapshot of a polished solve for the backward pass (called at the end of a solve with
// keep_for_backward). Copies the active set out of the solve's workspace.
int make_backward_state(const prism_universe* uh, const PolDev& P, const int* status_dev, const int64_t* offsets_dev,
                        const int32_t* asset_idx_dev, int64_t nnz, cudaStream_t st, prism_state** out) {
    const Universe& U = uh->u;
    auto* s = new prism_state();
    s->uh = uh; s->device = U.device; s->M = P.M; s->N = P.N; s->Npad = P.Npad; s->K = P.K; s->S = P.S; s->nnz = nnz;
    const size_t MN = (size_t)P.M * P.Npad;
    auto take = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        s->blocks.push_back(q);
        return q;
    };
    s->offsets = (int64_t*)take((P.M + 1) * 8);
    s->asset_idx = asset_idx_dev ? (int32_t*)take(nnz * 4) : nullptr;
    s->W = (double*)take(MN * 8);
    s->flags = (uint8_t*)take(MN);
    s->wband = (int*)take((size_t)P.M * P.S * 4);
    s->wcap = (int*)take(P.M * 4);
    s->status = (int*)take(P.M * 4);
    for (void* q : s->blocks)
        if (!q) { prism_free_state(s); set_error("cudaMalloc (backward state) failed"); return PRISM_ERR_ALLOCATION; }
    cudaMemcpyAsync(s->offsets, offsets_dev, (P.M + 1) * 8, cudaMemcpyDeviceToDevice, st);
    if (asset_idx_dev) cudaMemcpyAsync(s->asset_idx, asset_idx_dev, nnz * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s->W, P.W, MN * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s->wband, P.wband, (size_t)P.M * P.S * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s->wcap, P.wcap, P.M * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s->status, status_dev, P.M * 4, cudaMemcpyDeviceToDevice, st);
    launch_adjoint_flags(P, s->flags, st);
    *out = s;
    return PRISM_OK;
}

}  // namespace prism

extern "C" int prism_solve_batch_backward(prism_state* s, const double* dL_dw, double* dmu, double* dB, double* dd,
                                          double* dw0) {
    using namespace prism;
    if (!s || !dL_dw) { set_error("NULL argument"); return PRISM_ERR_ARGUMENT; }
    const Universe& U = s->uh->u;
    PRISM_CUDA_TRY(cudaSetDevice(s->device));
    const int M = s->M, N = s->N, Npad = s->Npad, K = s->K;
    const size_t MN = (size_t)M * Npad;
    if (!s->G) {
        s->fmax = std::min(Npad, 2048);
        auto take = [&](size_t bytes) -> void* {
            void* q = nullptr;
            if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
            s->blocks.push_back(q);
            return q;
        };
        s->G = (double*)take(MN * 8);
        s->U = (double*)take(MN * 8);
        s->DW0 = (double*)take(MN * 8);
        s->Fh = (double*)take((size_t)M * K * 8);
        s->Ft = (double*)take((size_t)M * K * 8);
        s->Y = (double*)take((size_t)M * s->fmax * AYS * 8);
        s->Flist = (int*)take((size_t)M * s->fmax * 4);
        s->NZlist = (int*)take(MN * 4);
        s->err = (int*)take(16);
        s->out_dmu = (double*)take((size_t)N * 8);
        s->out_dd = (double*)take((size_t)N * 8);
        s->out_dB = (double*)take((size_t)N * K * 8);
        s->out_dw0 = (double*)take(std::max<int64_t>(s->nnz, 1) * 8);
        s->in_g = (double*)take(std::max<int64_t>(s->nnz, 1) * 8);
        for (void* q : s->blocks)
            if (!q) { set_error("cudaMalloc (backward scratch) failed"); return PRISM_ERR_ALLOCATION; }
    }
    cudaStream_t st = 0;
    const double* g_dev = dL_dw;
    if (!dev_ptr(dL_dw)) {
        PRISM_CUDA_TRY(cudaMemcpy(s->in_g, dL_dw, s->nnz * 8, cudaMemcpyHostToDevice));
        g_dev = s->in_g;
    }
    cudaMemsetAsync(s->G, 0, MN * 8, st);
    cudaMemsetAsync(s->U, 0, MN * 8, st);
    cudaMemsetAsync(s->DW0, 0, MN * 8, st);
    cudaMemsetAsync(s->Fh, 0, (size_t)M * K * 8, st);
    cudaMemsetAsync(s->Ft, 0, (size_t)M * K * 8, st);
    cudaMemsetAsync(s->err, 0, 16, st);
    if (s->nnz > 0)
        k_adjoint_scatter<<<(unsigned)cdiv64(s->nnz, 256), 256, 0, st>>>(M, Npad, s->nnz, s->offsets, s->asset_idx,
                                                                          U.d_inv_perm, g_dev, s->G);
    AdjArgs A;
    A.M = M; A.N = N; A.Npad = Npad; A.K = K; A.S = s->S; A.fmax = s->fmax;
    A.B64 = U.d_B64; A.f64 = U.d_f64; A.d64 = U.d_d64; A.sector = U.d_sector;
    A.W = s->W; A.flags = s->flags; A.wband = s->wband; A.wcap = s->wcap; A.status = s->status; A.G = s->G;
    A.Flist = s->Flist; A.NZlist = s->NZlist; A.Y = s->Y;
    A.U = s->U; A.DW0 = s->DW0; A.Fh = s->Fh; A.Ft = s->Ft; A.err = s->err;
    const size_t smem = sizeof(AdjShared);
    cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_adjoint<<<M, AB, smem, st>>>(A);
    const int64_t nred = (int64_t)N * (K + 1);
    k_adjoint_reduce<<<(unsigned)cdiv64(nred, 256), 256, 0, st>>>(M, N, Npad, K, U.d_perm, s->U, s->W, s->Fh, s->Ft,
                                                                  s->out_dmu, s->out_dd, s->out_dB);
    if (dw0 && s->nnz > 0)
        k_adjoint_gather<<<(unsigned)cdiv64(s->nnz, 256), 256, 0, st>>>(M, Npad, s->nnz, s->offsets, s->asset_idx,
                                                                         U.d_inv_perm, s->DW0, s->out_dw0);
    PRISM_CUDA_TRY(cudaStreamSynchronize(st));
    PRISM_CUDA_TRY(cudaGetLastError());
    int err = 0;
    PRISM_CUDA_TRY(cudaMemcpy(&err, s->err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        set_error(err & 1 ? "backward: too many free weights or working rows in an account"
                          : "backward: capacitance matrix not positive definite");
        return PRISM_ERR_UNSUPPORTED;
    }
    auto out = [&](double* dst, const double* src, size_t n) -> cudaError_t {
        return dst ? cudaMemcpy(dst, src, n * 8, cudaMemcpyDefault) : cudaSuccess;
    };
    PRISM_CUDA_TRY(out(dmu, s->out_dmu, N));
    PRISM_CUDA_TRY(out(dd, s->out_dd, N));
    PRISM_CUDA_TRY(out(dB, s->out_dB, (size_t)N * K));
    if (s->nnz > 0) PRISM_CUDA_TRY(out(dw0, s->out_dw0, s->nnz));
    return PRISM_OK;
}

extern "C" void prism_free_state(prism_state* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    for (void* q : s->blocks) cudaFree(q);
    delete s;
}
