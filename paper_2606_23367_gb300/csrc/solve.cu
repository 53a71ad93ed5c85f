// solve.cu -- prism_solve_batch: packing, feasibility test, ADMM loop, polish, unpack.
//
// Call structure (one call = one book of accounts, Fig. 2 public solver call):
//   1. validate and pack the ragged FP64 inputs into a sector-sorted M x Npad
//      device layout (FP64 copies for the polish, FP32 copies for the iterations);
//      lot data become per-entry piecewise-linear cost tables;
//   2. closed-form capacity test per account (budget, box and bands admit a point);
//      accounts that fail get NO_FEASIBLE_RETURN;
//   3. ADMM iterations, check_every at a time, captured once in a CUDA graph and
//      replayed until every account has converged or hit its cap;
//   4. FP64 polish rounds and certification; accounts the polish cannot settle go
//      back to the iterations with a tighter target, then fall back to the
//      projected iterate (FEASIBLE_NONCERTIFIED when it passes the gates);
//   5. unpack weights, multipliers, status and diagnostics into the caller's layout.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "block_admm.h"
#include "polish.h"
#include "solver.h"

namespace prism {

// ---------------------------------------------------------------------------
// workspace: one device arena per universe handle, grown on demand
// ---------------------------------------------------------------------------
struct Arena {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    int alloc_fail = 0;
    template <typename T>
    T* take(size_t n) {
        size_t bytes = (n * sizeof(T) + 255) / 256 * 256;
        if (used + bytes > cap) { alloc_fail = 1; return nullptr; }
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

// Launch accounting and, in profile mode, CUDA events around every launch.
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Mark { int cls; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    int64_t launches[PRISM_NKCLASS] = {};
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void reset() {
        used = 0;
        marks.clear();
        for (auto& l : launches) l = 0;
    }
    template <class F>
    void run(int cls, int nkernels, cudaStream_t st, F f) {
        launches[cls] += nkernels;
        if (!on) { f(); return; }
        cudaEvent_t a = get(), b = get();
        cudaEventRecord(a, st);
        f();
        cudaEventRecord(b, st);
        marks.push_back({cls, a, b});
    }
};

struct SolveCache {
    Prof prof;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    int* pinned = nullptr;          // host-pinned counter readback
    cudaGraphExec_t gexec = nullptr;
    Dev gdev;                       // Dev the graph was captured with
    bool have_graph = false;
    int g_iters = 0;
    int64_t g_launches[PRISM_NKCLASS] = {};
    cudaEvent_t ev[6] = {};
    cudaStream_t pst = nullptr;                   // polish of the accounts that stopped iterating
    cudaEvent_t ev_pol = nullptr;
    int* hact = nullptr;                          // pinned: activity flags after each chunk (M)
    int* hsel = nullptr;                          // pinned: polish batch of each account (M)
    int hcap = 0;
    static constexpr int MAXCH = 4;               // independent chains of the fused iterations
    cudaStream_t chst[MAXCH - 1] = {};            // streams of chains 1 .. MAXCH-1 (chain 0: the solve stream)
    cudaEvent_t ev_fork = nullptr, ev_join[MAXCH - 1] = {};
    bool chains_ok = false;
};

static SolveCache& cache_of(prism_universe* uh) {
    static_assert(sizeof(void*) == 8, "64-bit only");
    // one cache per universe handle, stored alongside it
    struct Holder { prism_universe* u; SolveCache c; };
    static std::vector<Holder*> all;
    for (Holder* h : all) if (h->u == uh) return h->c;
    Holder* h = new Holder{uh, SolveCache()};
    all.push_back(h);
    return h->c;
}

void release_cache(prism_universe* uh);

// ---------------------------------------------------------------------------
// pack / validate
// ---------------------------------------------------------------------------
enum : int { ERR_INDEX = 1, ERR_NONFINITE = 2, ERR_BOUNDS = 4, ERR_DUP = 8, ERR_COST = 16, ERR_LEN = 32 };

struct PackArgs {
    int M, N, Npad;
    const int64_t* offsets;      // device
    const int32_t* asset_idx;    // device or null
    const double *w0, *lo, *up, *tc;   // device ragged
    const int* inv_perm;
    double *W0, *LO, *UP, *C;
    float *W0f, *LOf, *UPf, *Cf;
    int* member;
    int* err;
    int64_t nnz;
};

__global__ void k_pack(PackArgs A) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.nnz) return;
    // account of entry e: last a with offsets[a] <= e (every account spans the universe
    // when there is no asset_idx: then a = e / N)
    int a;
    if (A.asset_idx) {
        int lo = 0, hi = A.M;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (A.offsets[mid] <= e) lo = mid; else hi = mid;
        }
        a = lo;
    } else {
        a = int(e / A.N);
    }
    int i = A.asset_idx ? A.asset_idx[e] : int(e - (int64_t)a * A.N);
    if (i < 0 || i >= A.N) { atomicOr(A.err, ERR_INDEX); return; }
    const double w0 = A.w0[e], l = A.lo[e], u = A.up[e], c = A.tc[e];
    if (!(isfinite(w0) && isfinite(l) && isfinite(u) && isfinite(c))) { atomicOr(A.err, ERR_NONFINITE); return; }
    if (l > u) { atomicOr(A.err, ERR_BOUNDS); return; }
    if (c < 0) { atomicOr(A.err, ERR_COST); return; }
    const size_t d = (size_t)a * A.Npad + A.inv_perm[i];
    if (A.asset_idx) {
        if (atomicExch(&A.member[d], 1) != 0) { atomicOr(A.err, ERR_DUP); return; }
    } else {
        A.member[d] = 1;                   // position i of account a: no duplicate is possible
    }
    A.W0[d] = w0; A.LO[d] = l; A.UP[d] = u; A.C[d] = c;
    A.W0f[d] = float(w0); A.LOf[d] = float(l); A.UPf[d] = float(u); A.Cf[d] = float(c);
}

struct UnpackArgs {
    int M, Npad;
    const int64_t* offsets;
    const int32_t* asset_idx;
    const int* inv_perm;
    const double* W;
    double* out;
    int64_t nnz;
};

__global__ void k_unpack(UnpackArgs A) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.nnz) return;
    int lo = 0, hi = A.M;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (A.offsets[mid] <= e) lo = mid; else hi = mid;
    }
    const int a = lo;
    int i = A.asset_idx ? A.asset_idx[e] : int(e - A.offsets[a]);
    A.out[e] = A.W[(size_t)a * A.Npad + A.inv_perm[i]];
}

// Closed-form feasibility of budget + box + bands (+ the least-turnover test for a
// cap): sum_s max(lo_s, sum_{i in s} l_i) <= 1 <= sum_s min(hi_s, sum_{i in s} u_i).
// Closed-form feasibility of one account (budget, box, bands, and the cap when w0 sums to 1).
// The per-sector sums are taken first in FP32 from the iteration copies, one contiguous chunk
// of positions per thread (float4 loads, one pass); relative to their exact values they are
// off by less than 1e-5. The account is decided there when every comparison clears its
// threshold by 1e-4 relative; otherwise, and whenever a turnover cap is set, the sums are
// taken again in FP64 and decided as before.
__global__ void k_capacity(int S, int N, int Npad, const int* sec_start, const double* LO, const double* UP,
                           const double* W0, const float* LOf, const float* UPf, const float* W0f,
                           const double* band_lo, const double* band_hi, const double* tau, int* status, int* skip,
                           int* active) {
    const int a = blockIdx.x;
    __shared__ double s_up[SMAX], s_lo[SMAX], s_kept[SMAX], s_forced[SMAX], s_w0[SMAX];
    __shared__ float f_up[SMAX], f_lo[SMAX];
    __shared__ int sec[SMAX + 1];
    __shared__ int decided;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t base = (size_t)a * Npad;
    for (int s = threadIdx.x; s <= S; s += blockDim.x) sec[s] = sec_start[s];
    for (int s = threadIdx.x; s < S; s += blockDim.x) { f_up[s] = 0.f; f_lo[s] = 0.f; }
    __syncthreads();
    if (!isfinite(tau[a])) {
        // FP32 pass: Npad is a multiple of 64, so chunks of whole float4s cover it
        const int nq = Npad / 4, per = (nq + blockDim.x - 1) / blockDim.x;
        const int q0 = threadIdx.x * per, q1 = min(nq, q0 + per);
        int cs = 0;
        float su = 0.f, sl = 0.f;
        auto flush = [&](int s) {
            if (s < S) { atomicAdd(&f_up[s], su); atomicAdd(&f_lo[s], sl); }
            su = 0.f; sl = 0.f;
        };
        if (q0 < q1) {
            const int p0 = 4 * q0;
            while (cs < S && p0 >= sec[cs + 1]) ++cs;
            for (int q = q0; q < q1; ++q) {
                const float4 u4 = reinterpret_cast<const float4*>(UPf + base)[q];
                const float4 l4 = reinterpret_cast<const float4*>(LOf + base)[q];
                const float uu[4] = {u4.x, u4.y, u4.z, u4.w}, ll[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int p = 4 * q + k;
                    if (p >= N) break;
                    while (cs < S && p >= sec[cs + 1]) { flush(cs); ++cs; }
                    su += uu[k]; sl += ll[k];
                }
            }
            flush(cs);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // each comparison is decided only when it clears its threshold by 1e-4 relative
            bool ok = true, sure = true;
            double cap = 0, flo = 0, mag = 0;
            for (int s = 0; s < S; ++s) {
                const double hi = band_hi[a * S + s], lo = band_lo[a * S + s];
                const double u = f_up[s], l = f_lo[s];
                const double tol_u = 1e-4 * (u + fabs(lo)) + 1e-12, tol_l = 1e-4 * (l + fabs(hi)) + 1e-12;
                if (fabs(lo - u) <= tol_u && !(lo == 0.0 && u == 0.0)) sure = false;
                if (fabs(l - hi) <= tol_l && !(l == 0.0 && hi == 0.0)) sure = false;
                if (lo > u + 1e-12 || l > hi + 1e-12) ok = false;
                cap += fmin(hi, u);
                flo += fmax(lo, l);
                mag += fabs(fmin(hi, u)) + fabs(fmax(lo, l));
            }
            if (fabs(cap - 1.0) <= 1e-4 * fmax(mag, 1.0) || fabs(flo - 1.0) <= 1e-4 * fmax(mag, 1.0)) sure = false;
            if (!(cap >= 1.0 - 1e-12 && flo <= 1.0 + 1e-12)) ok = false;
            decided = sure;
            if (sure && !ok) {
                status[a] = PRISM_NO_FEASIBLE_RETURN;
                skip[a] = 1;
                active[a] = 0;
            }
        }
        __syncthreads();
        if (decided) return;
    }
    for (int s = warp; s < S; s += nw) {
        double su = 0, sl = 0, sk = 0, sf = 0, sw = 0;
        for (int p = sec[s] + lane; p < sec[s + 1]; p += 32) {
            double u = UP[base + p], l = LO[base + p], w = W0[base + p];
            su += u; sl += l; sk += fmin(w, u); sf += fmax(w - u, 0.0); sw += w;
        }
        su = warp_sum(su); sl = warp_sum(sl); sk = warp_sum(sk); sf = warp_sum(sf); sw = warp_sum(sw);
        if (lane == 0) { s_up[s] = su; s_lo[s] = sl; s_kept[s] = sk; s_forced[s] = sf; s_w0[s] = sw; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double cap = 0, flo = 0, forced = 0, w0s = 0;
        bool ok = true, lo_zero = true;
        for (int s = 0; s < S; ++s) {
            const double hi = band_hi[a * S + s], lo = band_lo[a * S + s];
            if (lo > s_up[s] + 1e-12 || s_lo[s] > hi + 1e-12) ok = false;
            cap += fmin(hi, s_up[s]);
            flo += fmax(lo, s_lo[s]);
            forced += s_forced[s] + fmax(s_kept[s] - hi, 0.0);
            w0s += s_w0[s];
            if (lo > 0 || s_lo[s] > 0) lo_zero = false;
        }
        if (!(cap >= 1.0 - 1e-12 && flo <= 1.0 + 1e-12)) ok = false;
        const double t = tau[a];
        if (ok && isfinite(t) && lo_zero && fabs(w0s - 1.0) < 1e-9 && 2.0 * forced > t * (1.0 + 1e-12)) ok = false;
        if (!ok) {
            status[a] = PRISM_NO_FEASIBLE_RETURN;
            skip[a] = 1;
            active[a] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// tax lots: convex piecewise-linear transition cost (lot-LP partial minimum)
// ---------------------------------------------------------------------------
struct PwlRow {
    double bp[MAXBP];
    double sl[MAXBP - 1];
    int nb;
    double phi_lo;
};

// phi(x) = c (x - w0) + G(max(S*, w0 - x)), G(S) = 2 c S + cheapest-first lot cost of S.
static double lot_phi(double x, double w0, double c, const std::vector<std::pair<double, double>>& lots) {
    double sstar = 0.0;
    for (auto& l : lots) if (2.0 * c + l.second < 0.0) sstar += l.first;
    double S = std::max(sstar, w0 - x);
    double g = 2.0 * c * S, rem = S;
    for (size_t j = 0; j < lots.size() && rem > 0; ++j) {
        double take = (j + 1 < lots.size()) ? std::min(rem, lots[j].first) : rem;
        g += lots[j].second * take;
        rem -= take;
    }
    return c * (x - w0) + g;
}

static bool build_pwl(double w0, double lo, double up, double c, std::vector<std::pair<double, double>> lots,
                      PwlRow& row) {
    std::stable_sort(lots.begin(), lots.end(),
                     [](const std::pair<double, double>& a, const std::pair<double, double>& b) { return a.second < b.second; });
    // kinks over the real line with the slope to their right
    std::vector<double> kinks;
    std::vector<double> right_slope;
    const int L = (int)lots.size();
    int js = 0;
    while (js < L && 2.0 * c + lots[js].second < 0.0) ++js;
    std::vector<double> slopes;   // left to right
    if (js < L) {
        double H = 0.0;
        for (int j = 0; j < js; ++j) H += lots[j].first;
        // slope right of w0 - S* is c; left of it the lots js, js+1, ... are sold in turn
        double x = w0 - H;
        kinks.push_back(x);
        double Hj = H;
        std::vector<double> xs{x};
        for (int j = js; j < L - 1; ++j) { Hj += lots[j].first; xs.push_back(w0 - Hj); }
        // xs decreasing; slopes left of xs[q] = -c - kappa[js + q]
        kinks.assign(xs.rbegin(), xs.rend());
        for (int j = L - 1; j >= js; --j) slopes.push_back(-c - lots[j].second);
        slopes.push_back(c);
    } else {
        slopes.push_back(c);
    }
    if (!(up > lo)) {
        row.nb = 1; row.bp[0] = lo; row.phi_lo = lot_phi(lo, w0, c, lots);
        return true;
    }
    std::vector<double> pts{lo};
    for (double x : kinks) if (x > lo && x < up) pts.push_back(x);
    if (w0 > lo && w0 < up) pts.push_back(w0);
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    pts.push_back(up);
    if ((int)pts.size() > MAXBP) return false;
    row.nb = (int)pts.size();
    for (int j = 0; j < row.nb; ++j) row.bp[j] = pts[j];
    for (int j = 0; j + 1 < row.nb; ++j) {
        double mid = 0.5 * (pts[j] + pts[j + 1]);
        int q = int(std::upper_bound(kinks.begin(), kinks.end(), mid) - kinks.begin());
        row.sl[j] = slopes[q];
    }
    row.phi_lo = lot_phi(lo, w0, c, lots);
    return true;
}

template <typename T>
static bool is_dev(const T* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

template <typename T>
static int to_host(const T* src, size_t n, std::vector<T>& dst) {
    dst.resize(n);
    if (!n) return PRISM_OK;
    PRISM_CUDA_TRY(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDefault));
    return PRISM_OK;
}

static double ms_between(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// ---------------------------------------------------------------------------
// one batched solve (all accounts share the launch sequence)
// ---------------------------------------------------------------------------
static int solve_core(prism_universe* uh, const prism_batch* b, const prism_solve_opts* o,
                      prism_result* res, bool batched_mode_bf16, bool plain, bool fp64 = false) {
    Universe& U = uh->u;
    SolveCache& SC = cache_of(uh);
    const auto t_call0 = std::chrono::steady_clock::now();
    PRISM_CUDA_TRY(cudaSetDevice(U.device));
    cudaStream_t st = o->cuda_stream ? (cudaStream_t)o->cuda_stream : U.stream;
    const int M = b->n_accounts, N = U.N, Npad = U.Npad, K = U.K, S = U.S;
    // ---- offsets
    std::vector<int64_t> offs;
    int rc = to_host(b->offsets, (size_t)M + 1, offs);
    if (rc) return rc;
    if (offs[0] != 0) { set_error("offsets[0] must be 0"); return PRISM_ERR_ARGUMENT; }
    for (int a = 0; a < M; ++a) {
        if (offs[a + 1] < offs[a]) { set_error("offsets must be nondecreasing"); return PRISM_ERR_ARGUMENT; }
        if (!b->asset_idx && offs[a + 1] - offs[a] != N) {
            set_error("without asset_idx every account must span the universe (N entries)");
            return PRISM_ERR_ARGUMENT;
        }
        if (offs[a + 1] - offs[a] > N) { set_error("account longer than the universe"); return PRISM_ERR_ARGUMENT; }
    }
    const int64_t nnz = offs[M];
    // ---- lots (host-side construction of the piecewise-linear tables)
    std::vector<PwlRow> pwl;
    std::vector<int> pw_of_entry;   // ragged entry -> pw row or -1
    const bool has_lots = b->lot_offsets != nullptr;
    if (has_lots) {
        std::vector<int64_t> lo_off;
        std::vector<double> lsz, lka, w0h, loh, uph, tch;
        if ((rc = to_host(b->lot_offsets, (size_t)nnz + 1, lo_off))) return rc;
        const int64_t nl = lo_off[nnz];
        if ((rc = to_host(b->lot_size, (size_t)nl, lsz)) || (rc = to_host(b->lot_kappa, (size_t)nl, lka)) ||
            (rc = to_host(b->w0, (size_t)nnz, w0h)) || (rc = to_host(b->lower, (size_t)nnz, loh)) ||
            (rc = to_host(b->upper, (size_t)nnz, uph)) || (rc = to_host(b->tc, (size_t)nnz, tch)))
            return rc;
        pw_of_entry.assign(nnz, -1);
        for (int64_t e = 0; e < nnz; ++e) {
            const int64_t l0 = lo_off[e], l1 = lo_off[e + 1];
            if (l1 < l0) { set_error("lot_offsets must be nondecreasing"); return PRISM_ERR_ARGUMENT; }
            if (l1 == l0) continue;
            if (l1 - l0 > MAXLOT) { set_error("more than 4 lots on one entry"); return PRISM_ERR_UNSUPPORTED; }
            if (loh[e] < 0) { set_error("lots need lower >= 0"); return PRISM_ERR_ARGUMENT; }
            std::vector<std::pair<double, double>> lots;
            double hs = 0;
            for (int64_t q = l0; q < l1; ++q) {
                if (!(lsz[q] >= 0) || !std::isfinite(lka[q])) { set_error("bad lot data"); return PRISM_ERR_ARGUMENT; }
                lots.push_back({lsz[q], lka[q]});
                hs += lsz[q];
            }
            if (std::fabs(hs - w0h[e]) > 1e-9 * std::max(1.0, std::fabs(w0h[e]))) {
                set_error("lot sizes of an entry must sum to its w0");
                return PRISM_ERR_ARGUMENT;
            }
            PwlRow row;
            if (!build_pwl(w0h[e], loh[e], uph[e], tch[e], lots, row)) {
                set_error("too many breakpoints in a lot cost");
                return PRISM_ERR_UNSUPPORTED;
            }
            pw_of_entry[e] = (int)pwl.size();
            pwl.push_back(row);
        }
    }
    // Tilts of the linear term (Eq. 1's per-account return tilt, and the benchmark's 2 Sigma w_b):
    // a term -t_i w_i is linear, so it shifts every slope of phi_i by -t_i; entries with a tilt
    // carry it in a piecewise-linear cost row (their lot row when they have lots)
    const bool has_tilt = b->mu_tilt || b->w_bench;
    if (has_tilt) {
        std::vector<double> tilt((size_t)nnz, 0.0), w0h, loh, uph, tch, tmp;
        std::vector<int32_t> aidx;
        if ((rc = to_host(b->w0, (size_t)nnz, w0h)) || (rc = to_host(b->lower, (size_t)nnz, loh)) ||
            (rc = to_host(b->upper, (size_t)nnz, uph)) || (rc = to_host(b->tc, (size_t)nnz, tch)))
            return rc;
        if (b->asset_idx && (rc = to_host(b->asset_idx, (size_t)nnz, aidx))) return rc;
        auto asset = [&](int a, int64_t e) { return b->asset_idx ? int(aidx[e]) : int(e - offs[a]); };
        if (b->mu_tilt) {
            if ((rc = to_host(b->mu_tilt, (size_t)nnz, tmp))) return rc;
            for (int64_t e = 0; e < nnz; ++e) tilt[e] = tmp[e];
        }
        if (b->w_bench) {
            // 2 Sigma_a w_b over the account's own names: 2 (B (F (B' w_b)) + D w_b), FP64
            std::vector<double> wb, Bh((size_t)U.Npad * K), fh, dh;
            if ((rc = to_host(b->w_bench, (size_t)nnz, wb)) || (rc = to_host(U.d_B64, (size_t)U.Npad * K, Bh)) ||
                (rc = to_host(U.d_f64, (size_t)K, fh)) || (rc = to_host(U.d_d64, (size_t)U.Npad, dh)))
                return rc;
            std::vector<double> h(K);
            for (int a = 0; a < M; ++a) {
                std::fill(h.begin(), h.end(), 0.0);
                for (int64_t e = offs[a]; e < offs[a + 1]; ++e) {
                    if (!std::isfinite(wb[e])) { set_error("w_bench must be finite"); return PRISM_ERR_ARGUMENT; }
                    const int i = asset(a, e);
                    if (i < 0 || i >= N) { set_error("asset index out of range"); return PRISM_ERR_ARGUMENT; }
                    const double* Bi = &Bh[(size_t)U.inv_perm[i] * K];
                    for (int k = 0; k < K; ++k) h[k] += Bi[k] * wb[e];
                }
                for (int k = 0; k < K; ++k) h[k] *= fh[k];
                for (int64_t e = offs[a]; e < offs[a + 1]; ++e) {
                    const int p = U.inv_perm[asset(a, e)];
                    const double* Bi = &Bh[(size_t)p * K];
                    double acc = dh[p] * wb[e];
                    for (int k = 0; k < K; ++k) acc += Bi[k] * h[k];
                    tilt[e] += 2.0 * acc;
                }
            }
        }
        if (pw_of_entry.empty()) pw_of_entry.assign(nnz, -1);
        for (int64_t e = 0; e < nnz; ++e) {
            const double t = tilt[e];
            if (!std::isfinite(t)) { set_error("mu_tilt must be finite"); return PRISM_ERR_ARGUMENT; }
            if (t == 0.0) continue;
            if (pw_of_entry[e] < 0) {
                // the plain L1 cost as a row: breakpoints l, w0 (inside the box), u
                PwlRow row;
                const double lo = loh[e], up = uph[e], w0 = w0h[e], c = tch[e];
                row.phi_lo = c * std::fabs(lo - w0);
                if (!(up > lo)) {
                    row.nb = 1; row.bp[0] = lo;
                } else if (w0 > lo && w0 < up) {
                    row.nb = 3; row.bp[0] = lo; row.bp[1] = w0; row.bp[2] = up; row.sl[0] = -c; row.sl[1] = c;
                } else {
                    row.nb = 2; row.bp[0] = lo; row.bp[1] = up; row.sl[0] = (w0 <= lo) ? c : -c;
                }
                pw_of_entry[e] = (int)pwl.size();
                pwl.push_back(row);
            }
            PwlRow& row = pwl[pw_of_entry[e]];
            for (int j = 0; j + 1 < row.nb; ++j) row.sl[j] -= t;
            row.phi_lo -= t * row.bp[0];
        }
    }
    const int n_pw = (int)pwl.size();
    const bool has_pw = has_lots || n_pw > 0;
    // factor-exposure bounds: validated on the host, any finite one turns the block on
    std::vector<double> flo_h, fhi_h;
    bool has_fac_in = false;
    if (b->factor_lo || b->factor_hi) {
        flo_h.assign((size_t)M * K, -INFINITY);
        fhi_h.assign((size_t)M * K, INFINITY);
        if (b->factor_lo && (rc = to_host(b->factor_lo, (size_t)M * K, flo_h))) return rc;
        if (b->factor_hi && (rc = to_host(b->factor_hi, (size_t)M * K, fhi_h))) return rc;
        for (size_t q = 0; q < flo_h.size(); ++q) {
            if (std::isnan(flo_h[q]) || std::isnan(fhi_h[q]) || flo_h[q] > fhi_h[q]) {
                set_error("factor_lo <= factor_hi required (no NaN)");
                return PRISM_ERR_ARGUMENT;
            }
            has_fac_in |= std::isfinite(flo_h[q]) || std::isfinite(fhi_h[q]);
        }
    }
    // ---- ragged books in the batched modes: dense-masked, or packed (each account's own names)
    bool packed = false;
    if (b->asset_idx && !plain) {
        packed = o->ragged_layout == 2;
    }
    // ---- workspace layout
    const size_t MN = (size_t)M * Npad;
    int tc_chunk = 0;
    const int nsplit = batched_mode_bf16 ? tc_nsplit(M, N, &tc_chunk, o->g2_sets) : choose_nsplit(M, N);
    const int FMAX = std::min(N, 2048);
    int* dsel = nullptr;               // device copy of SC.hsel (polish batches)
    BlkArgs<double> P64;               // PLAIN_FP64: the FP64 per-account kernel's arguments
    BlkArgs<float> PK;                 // ragged books, packed layout: the FP32 per-account kernel's
    auto layout = [&](Arena& A, Dev& D, PolDev& P, BatchDev& BD, void** stage, int** member, int** err,
                      int** pwidx_dev, double** ragged_out) {
        BD.w0 = A.take<double>(MN); BD.lo = A.take<double>(MN); BD.up = A.take<double>(MN); BD.c = A.take<double>(MN);
        BD.w0f = A.take<float>(MN); BD.lof = A.take<float>(MN); BD.upf = A.take<float>(MN); BD.cf = A.take<float>(MN);
        *member = A.take<int>(MN);
        *pwidx_dev = has_pw ? A.take<int>(MN) : nullptr;
        BD.band_lo = A.take<double>((size_t)M * S); BD.band_hi = A.take<double>((size_t)M * S);
        BD.band_lof = A.take<float>((size_t)M * S); BD.band_hif = A.take<float>((size_t)M * S);
        BD.tau = A.take<double>(M); BD.tauf = A.take<float>(M);
        {
            const size_t nf = has_fac_in ? (size_t)M * K : 0;
            BD.flo = A.take<double>(nf); BD.fhi = A.take<double>(nf);
            BD.flof = A.take<float>(nf); BD.fhif = A.take<float>(nf);
            D.s = A.take<float>(nf); D.ys = A.take<float>(nf); D.sflag = A.take<int>(nf);
            D.rps = A.take<float>(has_fac_in ? M : 0); D.rds = A.take<float>(has_fac_in ? M : 0);
            P.wfac = A.take<int>(nf);
        }
        P.kappa = A.take<double>((size_t)M * K);
        D.z = A.take<float>(MN); D.y = A.take<float>(MN); D.v = A.take<float>(MN);
        D.X = A.take<float>(MN);
        D.Xhi = A.take<__nv_bfloat16>(MN); D.Xlo = A.take<__nv_bfloat16>(MN);
        D.Ppart = A.take<float>((size_t)nsplit * M * KMAX);
        D.Q = A.take<float>((size_t)M * K);
        D.Qhi = A.take<__nv_bfloat16>((size_t)M * KMAX); D.Qlo = A.take<__nv_bfloat16>((size_t)M * KMAX);
        D.rho_idx = A.take<int>(M); D.iters = A.take<int>(M); D.active = A.take<int>(M); D.status = A.take<int>(M);
        D.nu = A.take<float>(M); D.dnu = A.take<float>(M); D.eta_hi = A.take<float>((size_t)M * S); D.eta_lo = A.take<float>((size_t)M * S);
        D.theta = A.take<float>(M); D.rp = A.take<float>(M); D.rd = A.take<float>(M); D.n_active = A.take<int>(2);
        D.stats = A.take<unsigned long long>(8);
        // partials of the fused pass (tensor-core mode)
        const int nt = cdiv(N, 128);
        D.SOp = A.take<float>((size_t)U.nseg * M);
        D.Rt = A.take<float>((size_t)5 * nt * M); D.Cm = A.take<unsigned>((size_t)U.nq * M);
        D.lo_u = A.take<float>(M); D.c_u = A.take<float>(M);
        D.crec = A.take<float>(MN * 8);
        D.Pxp = A.take<float>(batched_mode_bf16 ? (size_t)xp_sets_for(N) * M * KMAX : 0);
        D.needP = A.take<int>(M);
        D.pcount = A.take<unsigned long long>(2);
        D.xq_ctr = A.take<unsigned>(2 * SolveCache::MAXCH);
        P.st = A.take<int8_t>(MN); P.wband = A.take<int>((size_t)M * S); P.wcap = A.take<int>(M);
        P.done = A.take<int>(M); P.Flist = A.take<int>((size_t)M * FMAX); P.NZlist = A.take<int>((size_t)M * FMAX);
        P.Fsig = A.take<double>((size_t)M * FMAX);
        P.Y = A.take<double>((size_t)M * FMAX * (PMAXROWS + 1));
        P.Fdinv = A.take<double>((size_t)M * FMAX);
        P.fh64 = A.take<double>((size_t)M * KMAX); P.fh32 = A.take<float>((size_t)M * K);
        P.quad = A.take<double>(M); P.fhmax = A.take<double>(M);
        P.ndep = A.take<int>(M); P.pending = A.take<int>(1);
        P.W = A.take<double>(MN); P.nu = A.take<double>(M); P.lam = A.take<double>((size_t)M * S);
        P.theta = A.take<double>(M); P.diag = A.take<double>((size_t)M * PRISM_NDIAG);
        int* skip = A.take<int>(M);
        P.skip = skip;
        dsel = A.take<int>(M);
        *err = A.take<int>(4);
        // staging for host inputs / outputs (ragged FP64 x 4, offsets, asset_idx, out)
        stage[0] = A.take<double>((size_t)nnz); stage[1] = A.take<double>((size_t)nnz);
        stage[2] = A.take<double>((size_t)nnz); stage[3] = A.take<double>((size_t)nnz);
        stage[4] = A.take<int64_t>((size_t)M + 1);
        stage[5] = b->asset_idx ? (void*)A.take<int32_t>((size_t)nnz) : nullptr;
        *ragged_out = A.take<double>((size_t)nnz);
        BD.pw_bp = A.take<double>((size_t)std::max(n_pw, 1) * MAXBP);
        BD.pw_sl = A.take<double>((size_t)std::max(n_pw, 1) * (MAXBP - 1));
        BD.pw_bpf = A.take<float>((size_t)std::max(n_pw, 1) * MAXBP);
        BD.pw_slf = A.take<float>((size_t)std::max(n_pw, 1) * (MAXBP - 1));
        BD.pw_nbp = A.take<int>((size_t)std::max(n_pw, 1));
        stage[6] = A.take<double>((size_t)std::max(n_pw, 1));   // phi_lo
        // FP64 iteration state of PLAIN_FP64 (z, y, X/v per entry; penalty and cap multiplier)
        const size_t n64 = fp64 ? MN : 0;
        P64.z = A.take<double>(n64); P64.y = A.take<double>(n64); P64.X = A.take<double>(n64);
        P64.rho_state = A.take<double>(fp64 ? M : 0); P64.theta_state = A.take<double>(fp64 ? M : 0);
        P64.s_state = A.take<double>((fp64 && has_fac_in) ? (size_t)M * K : 0);
        P64.ys_state = A.take<double>((fp64 && has_fac_in) ? (size_t)M * K : 0);
        P64.queue = A.take<int>(4);
        // packed layout of a ragged book: position lists, sector ranges, processing order, FP32
        // state and input copies for accounts too large for shared memory
        const size_t np = packed ? (size_t)nnz : 0;
        PK.plist = A.take<int>(np); PK.psec = A.take<int>(packed ? (size_t)M * (S + 1) : 0);
        PK.order = A.take<int>(packed ? M : 0); PK.queue = A.take<int>(4);
        PK.z = A.take<float>(np); PK.y = A.take<float>(np); PK.X = A.take<float>(np);
        PK.w0p = A.take<float>(np); PK.lop = A.take<float>(np); PK.upp = A.take<float>(np); PK.cp = A.take<float>(np);
        PK.pwp = A.take<int>(np);
        PK.rho_state = A.take<float>(packed ? M : 0); PK.theta_state = A.take<float>(packed ? M : 0);
        PK.s_state = A.take<float>((packed && has_fac_in) ? (size_t)M * K : 0);
        PK.ys_state = A.take<float>((packed && has_fac_in) ? (size_t)M * K : 0);
    };
    Dev D;
    std::memset((void*)&D, 0, sizeof(Dev));   // padding bytes take part in the graph-reuse test
    PolDev P;
    BatchDev BD;
    void* stage[7];
    int *member, *err, *pwidx;
    double* ragged_out;
    {
        Arena probe;
        probe.base = nullptr; probe.cap = SIZE_MAX;
        layout(probe, D, P, BD, stage, &member, &err, &pwidx, &ragged_out);
        size_t need = probe.used + 4096;
        if (SC.arena_bytes < need) {
            if (SC.arena) { cudaFree(SC.arena); SC.arena = nullptr; SC.arena_bytes = 0; }
            if (SC.have_graph) { cudaGraphExecDestroy(SC.gexec); SC.have_graph = false; }
            if (SC.hact) { cudaFreeHost(SC.hact); cudaFreeHost(SC.hsel); SC.hact = SC.hsel = nullptr; SC.hcap = 0; }
            if (cudaMalloc(&SC.arena, need) != cudaSuccess) {
                cudaGetLastError();
                set_error("device workspace allocation failed");
                return PRISM_ERR_ALLOCATION;
            }
            SC.arena_bytes = need;
        }
        if (!SC.pinned) {
            if (cudaMallocHost(&SC.pinned, 64) != cudaSuccess) { set_error("pinned alloc failed"); return PRISM_ERR_ALLOCATION; }
            for (auto& e : SC.ev) cudaEventCreate(&e);
            if (cudaStreamCreateWithFlags(&SC.pst, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&SC.ev_pol, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                SC.pst = nullptr;                        // the polish waits for the iterations
            }
            SC.chains_ok = cudaEventCreateWithFlags(&SC.ev_fork, cudaEventDisableTiming) == cudaSuccess;
            for (int c = 0; c + 1 < SolveCache::MAXCH && SC.chains_ok; ++c)
                SC.chains_ok = cudaStreamCreateWithFlags(&SC.chst[c], cudaStreamNonBlocking) == cudaSuccess &&
                               cudaEventCreateWithFlags(&SC.ev_join[c], cudaEventDisableTiming) == cudaSuccess;
            if (!SC.chains_ok) cudaGetLastError();        // one chain only
        }
        if (SC.hcap < M) {
            if (SC.have_graph) { cudaGraphExecDestroy(SC.gexec); SC.have_graph = false; }
            if (SC.hact) { cudaFreeHost(SC.hact); cudaFreeHost(SC.hsel); SC.hact = SC.hsel = nullptr; SC.hcap = 0; }
            if (cudaMallocHost(&SC.hact, (size_t)M * 4) != cudaSuccess ||
                cudaMallocHost(&SC.hsel, (size_t)M * 4) != cudaSuccess) {
                cudaGetLastError();
                set_error("pinned alloc failed");
                return PRISM_ERR_ALLOCATION;
            }
            SC.hcap = M;
        }
        Arena A;
        A.base = SC.arena; A.cap = SC.arena_bytes;
        std::memset((void*)&D, 0, sizeof(Dev));
        P = PolDev(); BD = BatchDev(); P64 = BlkArgs<double>(); PK = BlkArgs<float>();
        layout(A, D, P, BD, stage, &member, &err, &pwidx, &ragged_out);
        if (A.alloc_fail) { set_error("workspace layout overflow"); return PRISM_ERR_ALLOCATION; }
    }
    SC.prof.reset();
    SC.prof.on = o->profile != 0;
    cudaEventRecord(SC.ev[0], st);
    // ---- stage inputs on the device
    auto stage_in = [&](const void* src, void* dst, size_t bytes) -> const void* {
        if (is_dev(src)) return src;
        cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        return dst;
    };
    PackArgs PA;
    PA.M = M; PA.N = N; PA.Npad = Npad; PA.nnz = nnz;
    PA.w0 = (const double*)stage_in(b->w0, stage[0], nnz * 8);
    PA.lo = (const double*)stage_in(b->lower, stage[1], nnz * 8);
    PA.up = (const double*)stage_in(b->upper, stage[2], nnz * 8);
    PA.tc = (const double*)stage_in(b->tc, stage[3], nnz * 8);
    cudaMemcpyAsync(stage[4], offs.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    PA.offsets = (const int64_t*)stage[4];
    PA.asset_idx = b->asset_idx ? (const int32_t*)stage_in(b->asset_idx, stage[5], nnz * 4) : nullptr;
    PA.inv_perm = U.d_inv_perm;
    PA.W0 = BD.w0; PA.LO = BD.lo; PA.UP = BD.up; PA.C = BD.c;
    PA.W0f = BD.w0f; PA.LOf = BD.lof; PA.UPf = BD.upf; PA.Cf = BD.cf;
    PA.member = member; PA.err = err;
    if (b->asset_idx) {
        // ragged accounts: every position the pack does not write is a non-member (zeros)
        cudaMemsetAsync(BD.w0, 0, MN * 8, st); cudaMemsetAsync(BD.lo, 0, MN * 8, st);
        cudaMemsetAsync(BD.up, 0, MN * 8, st); cudaMemsetAsync(BD.c, 0, MN * 8, st);
        cudaMemsetAsync(BD.w0f, 0, MN * 4, st); cudaMemsetAsync(BD.lof, 0, MN * 4, st);
        cudaMemsetAsync(BD.upf, 0, MN * 4, st); cudaMemsetAsync(BD.cf, 0, MN * 4, st);
        cudaMemsetAsync(member, 0, MN * 4, st);
    } else if (Npad > N) {
        // every account spans the universe, so the pack writes every position below N: only
        // the padding columns N .. Npad-1 are cleared
        auto pad = [&](void* p, size_t es) {
            cudaMemset2DAsync(static_cast<char*>(p) + (size_t)N * es, (size_t)Npad * es, 0, (size_t)(Npad - N) * es,
                              (size_t)M, st);
        };
        pad(BD.w0, 8); pad(BD.lo, 8); pad(BD.up, 8); pad(BD.c, 8);
        pad(BD.w0f, 4); pad(BD.lof, 4); pad(BD.upf, 4); pad(BD.cf, 4);
        pad(member, 4);
    }
    cudaMemsetAsync(err, 0, 16, st);
    if (nnz > 0) SC.prof.run(PRISM_K_PACK, 1, st, [&] { k_pack<<<(unsigned)cdiv64(nnz, 256), 256, 0, st>>>(PA); });
    // bands and caps
    {
        std::vector<double> blo, bhi, tau;
        if ((rc = to_host(b->band_lo, (size_t)M * S, blo)) || (rc = to_host(b->band_hi, (size_t)M * S, bhi))) return rc;
        if (b->turnover_cap) { if ((rc = to_host(b->turnover_cap, (size_t)M, tau))) return rc; }
        else tau.assign(M, INFINITY);
        for (size_t q = 0; q < blo.size(); ++q) {
            if (std::isnan(blo[q]) || std::isnan(bhi[q]) || blo[q] > bhi[q]) {
                set_error("band_lo <= band_hi required (no NaN)");
                return PRISM_ERR_ARGUMENT;
            }
        }
        bool cap_any = false;
        for (int a = 0; a < M; ++a) {
            if (std::isnan(tau[a]) || tau[a] < 0) { set_error("turnover_cap must be >= 0 or +inf"); return PRISM_ERR_ARGUMENT; }
            cap_any |= std::isfinite(tau[a]);
        }
        std::vector<float> blof(blo.begin(), blo.end()), bhif(bhi.begin(), bhi.end()), tauf(tau.begin(), tau.end());
        // the host vectors die at scope end: copy synchronously
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.band_lo, blo.data(), blo.size() * 8, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.band_hi, bhi.data(), bhi.size() * 8, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.band_lof, blof.data(), blof.size() * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.band_hif, bhif.data(), bhif.size() * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.tau, tau.data(), M * 8, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.tauf, tauf.data(), M * 4, cudaMemcpyHostToDevice, st));
        BD.has_cap = cap_any;
        std::vector<float> lf(flo_h.begin(), flo_h.end()), hf(fhi_h.begin(), fhi_h.end());
        if (has_fac_in) {
            PRISM_CUDA_TRY(cudaMemcpyAsync(BD.flo, flo_h.data(), flo_h.size() * 8, cudaMemcpyHostToDevice, st));
            PRISM_CUDA_TRY(cudaMemcpyAsync(BD.fhi, fhi_h.data(), fhi_h.size() * 8, cudaMemcpyHostToDevice, st));
            PRISM_CUDA_TRY(cudaMemcpyAsync(BD.flof, lf.data(), lf.size() * 4, cudaMemcpyHostToDevice, st));
            PRISM_CUDA_TRY(cudaMemcpyAsync(BD.fhif, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice, st));
            BD.has_fac = true;
        }
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // lot tables
    std::vector<double> h_phi;
    if (has_pw) {
        std::vector<double> bp((size_t)std::max(n_pw, 1) * MAXBP, 0.0), sl((size_t)std::max(n_pw, 1) * (MAXBP - 1), 0.0);
        std::vector<float> bpf(bp.size()), slf(sl.size());
        std::vector<int> nb(std::max(n_pw, 1), 1);
        h_phi.assign(std::max(n_pw, 1), 0.0);
        for (int r = 0; r < n_pw; ++r) {
            nb[r] = pwl[r].nb;
            h_phi[r] = pwl[r].phi_lo;
            for (int j = 0; j < pwl[r].nb; ++j) { bp[(size_t)r * MAXBP + j] = pwl[r].bp[j]; bpf[(size_t)r * MAXBP + j] = float(pwl[r].bp[j]); }
            for (int j = 0; j + 1 < pwl[r].nb; ++j) { sl[(size_t)r * (MAXBP - 1) + j] = pwl[r].sl[j]; slf[(size_t)r * (MAXBP - 1) + j] = float(pwl[r].sl[j]); }
        }
        // per sorted entry index of the table row
        std::vector<int> pwidx_h(MN, -1);
        std::vector<int32_t> aidx;
        if (b->asset_idx && (rc = to_host(b->asset_idx, (size_t)nnz, aidx))) return rc;
        for (int a = 0; a < M; ++a)
            for (int64_t e = offs[a]; e < offs[a + 1]; ++e) {
                int i = b->asset_idx ? aidx[e] : int(e - offs[a]);
                if (i < 0 || i >= N) { set_error("asset index out of range"); return PRISM_ERR_ARGUMENT; }
                pwidx_h[(size_t)a * Npad + U.inv_perm[i]] = pw_of_entry[e];
            }
        PRISM_CUDA_TRY(cudaMemcpyAsync(pwidx, pwidx_h.data(), MN * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.pw_bp, bp.data(), bp.size() * 8, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.pw_sl, sl.data(), sl.size() * 8, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.pw_bpf, bpf.data(), bpf.size() * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.pw_slf, slf.data(), slf.size() * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(BD.pw_nbp, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(stage[6], h_phi.data(), h_phi.size() * 8, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    {
        int herr = 0;
        PRISM_CUDA_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
        if (herr) {
            std::string m = "invalid batch input:";
            if (herr & ERR_INDEX) m += " asset index out of range;";
            if (herr & ERR_NONFINITE) m += " non-finite w0/lower/upper/tc;";
            if (herr & ERR_BOUNDS) m += " lower > upper;";
            if (herr & ERR_COST) m += " negative tc;";
            if (herr & ERR_DUP) m += " duplicate asset within an account;";
            set_error(m);
            return PRISM_ERR_ARGUMENT;
        }
    }
    // ---- device views
    D.M = M; D.N = N; D.Npad = Npad; D.K = K; D.S = S;
    D.B32 = U.d_B32; D.d32 = U.d_d32; D.mu32 = U.d_mu32; D.sec_start = U.d_sec_start; D.sector = U.d_sector;
    D.B16 = U.d_B16; D.Bt16 = U.d_Bt16; D.B16p = U.d_B16p; D.Bt16p = U.d_Bt16p;
    D.err = D.n_active + 1;
    if (!std::getenv("PRISM_DEBUG_STATS")) D.stats = nullptr;   // counters only when asked for
    if (const char* sw = std::getenv("PRISM_TEST_STALLED_WAIT_NS")) {
        // failure-path test: a bounded tensor-core wait on a barrier nothing completes (at most
        // 0.1 s, so that the test ends quickly and a stray setting cannot stall a real run long)
        const long long ns = std::atoll(sw);
        D.stall_ns = (unsigned long long)std::max(0LL, std::min(ns, 100000000LL));
    }
    if (!o->profile) D.pcount = nullptr;
    D.bf16 = batched_mode_bf16;
    D.Cinv = batched_mode_bf16 ? U.d_Cinv16 : U.d_Cinv32;
    D.w0 = BD.w0f; D.lo = BD.lof; D.up = BD.upf; D.c = BD.cf;
    D.pw_idx = pwidx; D.pw_bp = BD.pw_bpf; D.pw_sl = BD.pw_slf; D.pw_nbp = BD.pw_nbp;
    D.band_lo = BD.band_lof; D.band_hi = BD.band_hif; D.tau = BD.tauf;
    if (BD.has_fac) {
        // the factor-exposure block: its own capacitance inverses and the Gram matrices
        D.Cinv = batched_mode_bf16 ? U.d_CinvF16 : U.d_CinvF32;
        D.G = batched_mode_bf16 ? U.d_G16 : U.d_G32;
        D.flo = BD.flof; D.fhi = BD.fhif;
    } else {
        D.s = nullptr; D.ys = nullptr; D.sflag = nullptr; D.rps = nullptr; D.rds = nullptr;
    }
    D.stream_prox = (pwidx == nullptr && !BD.has_cap) ? 1 : 0;
    // the streaming pass runs inside the tensor-core x-update when the roots kernel can hold
    // the account's candidate masks
    D.fused = (D.stream_prox && batched_mode_bf16 && U.nq <= XP_NQMAX && o->fuse_prox) ? 1 : 0;
    D.nq = U.nq; D.nseg = U.nseg; D.nt = cdiv(N, 128); D.qseg = U.d_qseg; D.sseg = U.d_sseg;
    D.xp_sets = xp_sets_for(N);
    if (!D.fused || o->xupdate_form != 0) D.xq_ctr = nullptr;   // one CTA per tile
    int* const needP_buf = D.needP;            // set for the fused loop only (null: every account)
    D.needP = nullptr;
    D.nsplit = nsplit;
    D.g2_sets = batched_mode_bf16 ? o->g2_sets : 0;
    D.pstride = batched_mode_bf16 ? KMAX : K;
    D.alpha = (float)o->alpha; D.eps_admm = (float)o->eps_admm; D.min_iter = o->min_iter; D.max_iter = o->max_iter;
    D.adapt_every = o->adapt_every > 0 ? o->adapt_every : 25;
    P.M = M; P.N = N; P.Npad = Npad; P.K = K; P.S = S;
    P.B64 = U.d_B64; P.f64 = U.d_f64; P.d64 = U.d_d64; P.mu64 = U.d_mu64; P.sec_start = U.d_sec_start; P.sector = U.d_sector;
    P.B32 = U.d_B32; P.B32p = U.d_B32p; P.Bn1 = U.d_Bn1; P.Bn1f = U.d_Bn1f; P.mu32 = U.d_mu32;
    P.w0f = BD.w0f; P.lof = BD.lof; P.upf = BD.upf; P.cf = BD.cf;
    P.w0 = BD.w0; P.lo = BD.lo; P.up = BD.up; P.c = BD.c;
    P.pw_idx = pwidx; P.pw_bp = BD.pw_bp; P.pw_sl = BD.pw_sl; P.pw_phi_lo = (const double*)stage[6]; P.pw_nbp = BD.pw_nbp;
    P.band_lo = BD.band_lo; P.band_hi = BD.band_hi; P.tau = BD.tau;
    if (BD.has_fac) { P.flo = BD.flo; P.fhi = BD.fhi; P.sflag = D.sflag; }
    else P.wfac = nullptr;
    P.z = D.z; P.nu_f = D.nu; P.eta_hi_f = D.eta_hi; P.eta_lo_f = D.eta_lo; P.theta_f = D.theta;
    P.FMAX = FMAX;
    P.status = D.status;
    P.tol_dual = 1e-11; P.tol_primal = 1e-12;
    P.dmin = U.dmin;
    if (fp64) {
        P64.M = M; P64.N = N; P64.Npad = Npad; P64.K = K; P64.S = S;
        P64.B = U.d_B64; P64.f = U.d_f64; P64.d = U.d_d64; P64.mu = U.d_mu64;
        P64.sec_start = U.d_sec_start; P64.sector = U.d_sector;
        P64.w0 = BD.w0; P64.lo = BD.lo; P64.up = BD.up; P64.c = BD.c;
        P64.pw_idx = pwidx; P64.pw_bp = BD.pw_bp; P64.pw_sl = BD.pw_sl; P64.pw_nbp = BD.pw_nbp;
        P64.band_lo = BD.band_lo; P64.band_hi = BD.band_hi; P64.tau = BD.tau; P64.skip = P.skip;
        if (BD.has_fac) { P64.flo = BD.flo; P64.fhi = BD.fhi; P64.sflag = D.sflag; }
        P64.zf = D.z; P64.nu_f = D.nu; P64.eta_hi_f = D.eta_hi; P64.eta_lo_f = D.eta_lo; P64.theta_f = D.theta;
        P64.iters = D.iters; P64.active = D.active; P64.status = D.status;
        P64.alpha = o->alpha; P64.eps = o->eps_admm; P64.rho0 = o->rho0;
        P64.max_iter = o->max_iter; P64.min_iter = o->min_iter; P64.adapt_every = D.adapt_every;
    }
    std::vector<int> order_h;
    if (packed) {
        PK.M = M; PK.N = N; PK.Npad = Npad; PK.K = K; PK.S = S;
        PK.B = U.d_B32; PK.Bp = U.d_B32p; PK.f = U.d_f32; PK.d = U.d_d32; PK.mu = U.d_mu32;
        PK.sec_start = U.d_sec_start; PK.sector = U.d_sector;
        PK.w0 = BD.w0f; PK.lo = BD.lof; PK.up = BD.upf; PK.c = BD.cf;
        PK.pw_idx = pwidx; PK.pw_bp = BD.pw_bpf; PK.pw_sl = BD.pw_slf; PK.pw_nbp = BD.pw_nbp;
        PK.band_lo = BD.band_lof; PK.band_hi = BD.band_hif; PK.tau = BD.tauf; PK.skip = P.skip;
        if (BD.has_fac) { PK.flo = BD.flof; PK.fhi = BD.fhif; PK.sflag = D.sflag; }
        PK.poff = PA.offsets;
        PK.zf = D.z; PK.nu_f = D.nu; PK.eta_hi_f = D.eta_hi; PK.eta_lo_f = D.eta_lo; PK.theta_f = D.theta;
        PK.iters = D.iters; PK.active = D.active; PK.status = D.status;
        PK.alpha = o->alpha; PK.eps = o->eps_admm; PK.rho0 = o->rho0;
        PK.max_iter = o->max_iter; PK.min_iter = o->min_iter; PK.adapt_every = D.adapt_every;
        // accounts largest first (the persistent blocks take them in this order); accounts of at
        // most stage_cap names keep their entries in shared memory
        int64_t nmax = 0;
        order_h.resize(M);
        for (int a = 0; a < M; ++a) { order_h[a] = a; nmax = std::max(nmax, offs[a + 1] - offs[a]); }
        std::stable_sort(order_h.begin(), order_h.end(),
                         [&](int x, int y) { return offs[x + 1] - offs[x] > offs[y + 1] - offs[y]; });
        BlkArgs<float> probe = PK;
        probe.stage_cap = 0;
        const size_t fixed = blk_smem_bytes(probe), per = 7 * sizeof(float) + 2 * sizeof(int);
        const size_t room = 227 * 1024 - 1024 > fixed ? 227 * 1024 - 1024 - fixed : 0;
        PK.stage_cap = (int)std::min<int64_t>(nmax, (int64_t)(room / per));
        PRISM_CUDA_TRY(cudaMemcpyAsync(PK.order, order_h.data(), (size_t)M * 4, cudaMemcpyHostToDevice, st));
    }
    // ---- control init
    {
        int j0 = (int)std::lround(RHO_PER_DECADE * std::log10(std::max(o->rho0, 1e-12) / RHO_MIN));
        j0 = std::max(0, std::min(NRHO - 1, j0));
        std::vector<int> h(M, j0);
        PRISM_CUDA_TRY(cudaMemcpyAsync(D.rho_idx, h.data(), M * 4, cudaMemcpyHostToDevice, st));
        std::vector<int> one(M, 1);
        PRISM_CUDA_TRY(cudaMemcpyAsync(D.active, one.data(), M * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
        cudaMemsetAsync(D.iters, 0, M * 4, st);
        cudaMemsetAsync(D.status, 0, M * 4, st);
        cudaMemsetAsync(D.nu, 0, M * 4, st);
        cudaMemsetAsync(D.dnu, 0x7f, M * 4, st);                    // 3.4e38: no margin yet
        cudaMemsetAsync(D.theta, 0, M * 4, st);
        cudaMemsetAsync(D.eta_hi, 0xff, (size_t)M * S * 4, st);   // NaN: no warm start yet
        cudaMemsetAsync(D.eta_lo, 0xff, (size_t)M * S * 4, st);
        cudaMemsetAsync(P.skip, 0, M * 4, st);
        cudaMemsetAsync(P.done, 0, M * 4, st);
        cudaMemsetAsync(P.diag, 0, (size_t)M * PRISM_NDIAG * 8, st);
        cudaMemsetAsync(P.W, 0, MN * 8, st);
        cudaMemsetAsync(P.nu, 0, M * 8, st);
        cudaMemsetAsync(P.theta, 0, M * 8, st);
        cudaMemsetAsync(P.lam, 0, (size_t)M * S * 8, st);
        cudaMemsetAsync(P.kappa, 0, (size_t)M * K * 8, st);
        if (BD.has_fac) {
            cudaMemsetAsync(D.s, 0, (size_t)M * K * 4, st);     // s = 0 clipped on the first update
            cudaMemsetAsync(D.ys, 0, (size_t)M * K * 4, st);
            cudaMemsetAsync(D.sflag, 0, (size_t)M * K * 4, st);
            cudaMemsetAsync(D.rps, 0, M * 4, st);
            cudaMemsetAsync(D.rds, 0, M * 4, st);
        }
        cudaMemsetAsync(D.X, 0, MN * 4, st);
        cudaMemsetAsync(D.Xhi, 0, MN * 2, st);
        cudaMemsetAsync(D.Xlo, 0, MN * 2, st);
        cudaMemsetAsync(D.v, 0, MN * 4, st);
        cudaMemsetAsync(D.Qhi, 0, (size_t)M * KMAX * 2, st);
        cudaMemsetAsync(D.Qlo, 0, (size_t)M * KMAX * 2, st);
        cudaMemsetAsync(D.n_active, 0, 8, st);
        if (D.stats) cudaMemsetAsync(D.stats, 0, 32, st);
        if (D.pcount) cudaMemsetAsync(D.pcount, 0, 16, st);
        if (D.xq_ctr) cudaMemsetAsync(D.xq_ctr, 0, 2 * SolveCache::MAXCH * sizeof(unsigned), st);
    }
    SC.prof.run(PRISM_K_OTHER, 2, st, [&] {
        k_capacity<<<M, 256, 0, st>>>(S, N, Npad, U.d_sec_start, BD.lo, BD.up, BD.w0, BD.lof, BD.upf, BD.w0f,
                                      BD.band_lo, BD.band_hi, BD.tau, D.status, P.skip, D.active);
        launch_init_state(D, st);
    });
    if (D.fused) {
        SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_uniform(D, (float*)D.lo_u, (float*)D.c_u, st); });
        // the fused kernel's variant: per-account l and c throughout, or per-entry where they differ
        std::vector<float> lu(M), cu(M);
        PRISM_CUDA_TRY(cudaMemcpyAsync(lu.data(), D.lo_u, M * 4, cudaMemcpyDeviceToHost, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(cu.data(), D.c_u, M * 4, cudaMemcpyDeviceToHost, st));
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
        D.uniform = 1;
        for (int a = 0; a < M; ++a)
            if (std::isnan(lu[a]) || std::isnan(cu[a])) D.uniform = 0;
    }
    cudaEventRecord(SC.ev[1], st);
    // ---- ADMM iterations
    const int check_every = std::max(1, o->check_every);
    // Chains: the accounts are cut into up to MAXCH ranges that iterate independently on their
    // own streams, so that one range's latency-bound kernels (the roots, the small products)
    // run beside another range's streaming x-update. Every cut is a multiple of 128 (a product
    // tile never straddles two ranges); a range holds at least 128 accounts.
    int nch = 1;
    // automatic: as many chains as fit for the one-CTA-per-tile x-update; one for the persistent
    // form, whose CTAs take every SM (measured: several chains then lose more than they overlap)
    if (D.fused && SC.chains_ok && !D.xq_ctr) nch = std::min(SolveCache::MAXCH, std::max(1, M / 128));
    if (D.fused && SC.chains_ok && o->chains > 0) nch = std::min(std::min(SolveCache::MAXCH, std::max(1, M / 128)), o->chains);
    auto run_chunk = [&](int n) {
        if (nch > 1 && !SC.prof.on) {
            Dev DC[SolveCache::MAXCH];
            cudaStream_t cs[SolveCache::MAXCH];
            for (int c = 0; c < nch; ++c) {
                DC[c] = D;
                DC[c].m0 = ((M * c / nch) + 64) / 128 * 128;
                DC[c].m1 = (c + 1 == nch) ? M : ((M * (c + 1) / nch) + 64) / 128 * 128;
                if (D.xq_ctr) { DC[c].xq_ctr = D.xq_ctr + 2 * c; DC[c].xq_share = nch; }   // own tile counter
                cs[c] = c == 0 ? st : SC.chst[c - 1];
            }
            cudaEventRecord(SC.ev_fork, st);
            for (int c = 1; c < nch; ++c) cudaStreamWaitEvent(cs[c], SC.ev_fork, 0);
            for (int it = 0; it < n; ++it) {
                SC.prof.run(PRISM_K_GEMM_P, nch, st, [&] { for (int c = 0; c < nch; ++c) launch_tc_gemm_P(DC[c], cs[c], true); });
                SC.prof.run(PRISM_K_SOLVE_K, nch, st, [&] { for (int c = 0; c < nch; ++c) launch_small_solve(DC[c], cs[c], true); });
                SC.prof.run(PRISM_K_XPROX, nch, st, [&] { for (int c = 0; c < nch; ++c) launch_tc_xprox(DC[c], cs[c], true); });
                SC.prof.run(PRISM_K_ROOTS, nch, st, [&] { for (int c = 0; c < nch; ++c) launch_prox_roots(DC[c], cs[c], true); });
            }
            for (int c = 1; c < nch; ++c) {
                cudaEventRecord(SC.ev_join[c - 1], cs[c]);
                cudaStreamWaitEvent(st, SC.ev_join[c - 1], 0);
            }
            SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_count_active(D, st); });
            cudaMemcpyAsync(SC.pinned, D.n_active, 8, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(SC.hact, D.active, (size_t)M * 4, cudaMemcpyDeviceToHost, st);
            return;
        }
        for (int it = 0; it < n; ++it) {
            if (D.fused) {
                // the four kernels of an iteration overlap their prologues with the kernel
                // before (programmatic dependent launch; see pdl_wait)
                const bool pdl = !SC.prof.on;
                SC.prof.run(PRISM_K_GEMM_P, 1, st, [&] { launch_tc_gemm_P(D, st, pdl); });
                SC.prof.run(PRISM_K_SOLVE_K, 1, st, [&] { launch_small_solve(D, st, pdl); });
                SC.prof.run(PRISM_K_XPROX, 1, st, [&] { launch_tc_xprox(D, st, pdl); });
                SC.prof.run(PRISM_K_ROOTS, 1, st, [&] { launch_prox_roots(D, st, pdl); });
                continue;
            }
            SC.prof.run(PRISM_K_GEMM_P, 1, st, [&] { if (D.bf16) launch_tc_gemm_P(D, st); else launch_gemm_P(D, st); });
            SC.prof.run(PRISM_K_SOLVE_K, 1, st, [&] { launch_small_solve(D, st); });
            SC.prof.run(PRISM_K_GEMM_X, 1, st, [&] { if (D.bf16) launch_tc_gemm_x(D, st); else launch_gemm_x(D, st); });
            SC.prof.run(PRISM_K_PROX, 1, st, [&] { launch_prox(D, st); });
        }
        SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_count_active(D, st); });
        cudaMemcpyAsync(SC.pinned, D.n_active, 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(SC.hact, D.active, (size_t)M * 4, cudaMemcpyDeviceToHost, st);
    };
    int64_t chunk_launches[PRISM_NKCLASS] = {};
    // Accounts that stop iterating are polished on their own stream while the others iterate:
    // after each chunk, those that stopped since the last check form a batch (hsel[a] = its
    // number) and are classified and polished beside the next chunk. Only the accounts' own
    // rows are touched, which the iterations no longer read or write.
    const int rounds = std::max(1, o->polish_rounds);
    int pol_gen = 0;
    std::vector<char> was_active(M, 1);
    auto polish_batch = [&](int gen, cudaStream_t s) {
        PolDev PB2 = P;
        PB2.sel = dsel;
        PB2.gen = gen;
        SC.prof.run(PRISM_K_OTHER, 1, s, [&] { launch_classify(PB2, s); });
        SC.prof.run(PRISM_K_POLISH, 1, s, [&] { launch_polish(PB2, rounds, s); });
    };
    auto admm_loop = [&](int iter_budget, bool overlap) -> int {
        int done_iters = 0;
        if (D.needP) {
            // the folded iteration keeps no X of the entries it pins and leaves P, Q only for the
            // accounts that iterate on: on entry every active account gets X from its z, y, and
            // its first P and Q from the product kernels
            SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_refresh_X(D, st); });
            cudaMemsetAsync(D.needP, 0x01, (size_t)M * 4, st);
        }
        overlap = overlap && SC.pst && !SC.prof.on && o->polish_overlap > 0;
        bool use_graph = o->use_graph != 0 && !SC.prof.on;
        if (use_graph) {
            bool same = SC.have_graph && SC.g_iters == check_every && std::memcmp(&SC.gdev, &D, sizeof(Dev)) == 0;
            if (!same) {
                if (SC.have_graph) { cudaGraphExecDestroy(SC.gexec); SC.have_graph = false; }
                cudaGraph_t g;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { cudaGetLastError(); use_graph = false; }
                else {
                    int64_t before[PRISM_NKCLASS];
                    std::memcpy(before, SC.prof.launches, sizeof(before));
                    run_chunk(check_every);
                    for (int q = 0; q < PRISM_NKCLASS; ++q) {
                        chunk_launches[q] = SC.prof.launches[q] - before[q];
                        SC.prof.launches[q] = before[q];
                    }
                    if (cudaStreamEndCapture(st, &g) != cudaSuccess ||
                        cudaGraphInstantiate(&SC.gexec, g, 0) != cudaSuccess) {
                        cudaGetLastError();
                        use_graph = false;
                    } else {
                        SC.have_graph = true;
                        SC.gdev = D;
                        SC.g_iters = check_every;
                        std::memcpy(SC.g_launches, chunk_launches, sizeof(chunk_launches));
                    }
                    cudaGraphDestroy(g);
                }
            }
        }
        while (done_iters < iter_budget) {
            if (use_graph) {
                cudaGraphLaunch(SC.gexec, st);
                for (int q = 0; q < PRISM_NKCLASS; ++q) SC.prof.launches[q] += SC.g_launches[q];
            } else {
                run_chunk(check_every);
            }
            done_iters += check_every;
            if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
            if (SC.pinned[1] != 0) return -2;      // a bounded tensor-core wait expired
            if (overlap && SC.pinned[0] < o->polish_overlap * M) {
                int nnew = 0;
                for (int a = 0; a < M; ++a)
                    if (was_active[a] && !SC.hact[a]) { was_active[a] = 0; SC.hsel[a] = pol_gen + 1; ++nnew; }
                if (nnew) {
                    ++pol_gen;
                    cudaMemcpyAsync(dsel, SC.hsel, (size_t)M * 4, cudaMemcpyHostToDevice, SC.pst);
                    polish_batch(pol_gen, SC.pst);
                }
            }
            if (SC.pinned[0] == 0) break;
            if (o->time_budget_s > 0) {
                double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_call0).count();
                if (el > o->time_budget_s) break;
            }
        }
        return done_iters;
    };
    // the first iterations run the staged prox: the streaming form needs the budget multiplier
    // to have settled (its moves set the streaming form's margin) to keep its candidate lists short
    const bool blockwise = fp64 || packed;         // every iteration inside the per-account kernel
    const int cold = (D.stream_prox && !blockwise) ? std::min(std::max(0, o->stream_after), o->max_iter) : 0;
    if (fp64) {
        // PLAIN_FP64: every iteration of the account in one FP64 launch (block_admm.cu)
        P64.resume = 0;
        SC.prof.run(PRISM_K_BLOCK, 1, st, [&] { launch_block_admm(P64, blk_grid(P64), st); });
    }
    if (packed) {
        // ragged book, packed layout: the position lists, then one persistent FP32 launch
        SC.prof.run(PRISM_K_OTHER, 1, st, [&] {
            launch_member_lists(M, Npad, S, member, U.d_sec_start, PA.offsets, PK.plist, PK.psec, st);
        });
        PK.resume = 0;
        SC.prof.run(PRISM_K_BLOCK, 1, st, [&] { launch_block_admm(PK, blk_grid(PK), st); });
    }
    if ((fp64 || packed) && D.stats) {
        // diagnostics: ns per phase summed over accounts, iterations, projection evaluations
        unsigned long long h[8] = {};
        BlkArgs<float> DP = PK;
        BlkArgs<double> D64 = P64;
        cudaMemsetAsync(D.stats, 0, 64, st);
        if (packed) { DP.dbg = D.stats; launch_block_admm(DP, blk_grid(DP), st); }
        else { D64.dbg = D.stats; launch_block_admm(D64, blk_grid(D64), st); }
        cudaMemcpyAsync(h, D.stats, 64, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        std::fprintf(stderr, "prism block stats: iterations %llu, ns: X+B'X %llu, solve %llu, x-update %llu, roots %llu, "
                     "z/y %llu, factor %llu; evaluations per iteration %.1f\n", h[6], h[0], h[1], h[2], h[3], h[4], h[5],
                     h[6] ? double(h[7]) / h[6] : 0.0);
    }
    for (int it = 0; it < cold; ++it) {
        SC.prof.run(PRISM_K_GEMM_P, 1, st, [&] { if (D.bf16) launch_tc_gemm_P(D, st); else launch_gemm_P(D, st); });
        SC.prof.run(PRISM_K_SOLVE_K, 1, st, [&] { launch_small_solve(D, st); });
        SC.prof.run(PRISM_K_GEMM_X, 1, st, [&] { if (D.bf16) launch_tc_gemm_x(D, st); else launch_gemm_x(D, st); });
        SC.prof.run(PRISM_K_PROX, 1, st, [&] { launch_prox(D, st, true); });
    }
    std::memset(SC.hsel, 0, (size_t)M * 4);
    if (D.fused && o->fold_products) { D.needP = needP_buf; D.fold = 1; }
    int total_iters = blockwise ? 0 : admm_loop(o->max_iter + check_every - cold, true);
    if (total_iters >= 0) total_iters += cold;
    if (total_iters == -2) { set_error("tensor-core pipeline wait timed out (error flags " + std::to_string(SC.pinned[1]) + ")"); return PRISM_ERR_CUDA; }
    if (total_iters < 0) { set_error(std::string("ADMM loop failed: ") + cudaGetErrorString(cudaGetLastError())); return PRISM_ERR_CUDA; }
    SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_mark_timeout(D, st); });   // accounts still iterating
    cudaEventRecord(SC.ev[2], st);
    if (std::getenv("PRISM_DEBUG_STATS")) {
        unsigned long long h[4] = {0, 0, 0, 0};
        cudaMemcpyAsync(h, D.stats, 32, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        std::fprintf(stderr, "prism stats: ADMM iterations %d, prox account-calls %llu, sector-edge evals/call %.2f, "
                     "budget evals/call %.2f, sectors from global memory/call %.2f\n", total_iters, h[0],
                     h[0] ? double(h[1]) / h[0] : 0.0, h[0] ? double(h[2]) / h[0] : 0.0,
                     h[0] ? double(h[3]) / h[0] : 0.0);
    }
    // ---- polish, with up to two returns to the iterations at a tighter target
    // polish rounds until no account needs another (checked after each round)
    int n_rounds_run = 0, n_retried = 0;
    // all active-set rounds of every account in one launch; each block stops when settled (one
    // launch per round measured slower: each launch waits for its slowest block)
    auto polish_rounds = [&]() -> int {
        ++n_rounds_run;
        SC.prof.run(PRISM_K_POLISH, 1, st, [&] { launch_polish(P, rounds, st); });
        return 0;
    };
    if (pol_gen > 0) {
        // the batches polished beside the iterations, then every account not in one of them
        // (those that stopped in the last chunk, or were still iterating at the cap)
        cudaEventRecord(SC.ev_pol, SC.pst);
        cudaStreamWaitEvent(st, SC.ev_pol, 0);
        cudaMemcpyAsync(dsel, SC.hsel, (size_t)M * 4, cudaMemcpyHostToDevice, st);
        ++n_rounds_run;
        polish_batch(0, st);
    } else {
        SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_classify(P, st); });
        if (polish_rounds() < 0) { set_error("polish failed"); return PRISM_ERR_CUDA; }
    }
    for (int retry = 0; retry < 2; ++retry) {
        std::vector<int> done(M), skip(M), status(M);
        cudaMemcpyAsync(done.data(), P.done, M * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(skip.data(), P.skip, M * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(status.data(), D.status, M * 4, cudaMemcpyDeviceToHost, st);
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int> act(M, 0);
        int n_retry = 0;
        for (int a = 0; a < M; ++a) {
            if (skip[a] || done[a] == 1 || status[a] == PRISM_NUMERICAL_FAILURE) continue;
            act[a] = 1;
            done[a] = 0;
            status[a] = 0;
            ++n_retry;
        }
        if (!n_retry) break;
        n_retried += n_retry;
        if (o->time_budget_s > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t_call0).count() > o->time_budget_s) break;
        // iterate again, to a tighter target, only the accounts the polish could not settle
        PRISM_CUDA_TRY(cudaMemcpyAsync(D.active, act.data(), M * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(D.status, status.data(), M * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaMemcpyAsync(P.done, done.data(), M * 4, cudaMemcpyHostToDevice, st));
        PRISM_CUDA_TRY(cudaStreamSynchronize(st));
        int more = 0;
        if (fp64) {
            // continue the FP64 iterations of the accounts sent back, to a tighter target
            BlkArgs<double> R = P64;
            R.resume = 1;
            R.eps = P64.eps * (retry == 0 ? 0.1 : 0.01);
            R.max_iter = P64.max_iter * (retry + 2);
            SC.prof.run(PRISM_K_BLOCK, 1, st, [&] { launch_block_admm(R, blk_grid(R), st); });
        } else if (packed) {
            BlkArgs<float> R = PK;
            R.resume = 1;
            R.eps = PK.eps * (retry == 0 ? 0.1 : 0.01);
            R.max_iter = PK.max_iter * (retry + 2);
            SC.prof.run(PRISM_K_BLOCK, 1, st, [&] { launch_block_admm(R, blk_grid(R), st); });
        } else {
            Dev saved = D;
            D.eps_admm = saved.eps_admm * (retry == 0 ? 0.1f : 0.01f);
            D.max_iter = saved.max_iter * (retry + 2);
            more = admm_loop(D.max_iter, false);
            D = saved;
        }
        if (more == -2) { set_error("tensor-core pipeline wait timed out"); return PRISM_ERR_CUDA; }
        if (more < 0) { set_error("ADMM retry failed"); return PRISM_ERR_CUDA; }
        total_iters += more;
        SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_classify(P, st); });
        if (polish_rounds() < 0) { set_error("polish failed"); return PRISM_ERR_CUDA; }
    }
    if (std::getenv("PRISM_DEBUG_STATS"))
        std::fprintf(stderr, "prism stats: polish rounds %d, accounts sent back to the iterations %d\n", n_rounds_run,
                     n_retried);
    SC.prof.run(PRISM_K_OTHER, 2, st, [&] { launch_fallback(P, st); });
    cudaEventRecord(SC.ev[3], st);
    SC.prof.run(PRISM_K_OTHER, 1, st, [&] { launch_finish_status(P, o->eps_kkt, st); });
    cudaEventRecord(SC.ev[4], st);
    if (o->keep_for_backward) {
        if (int rc2 = make_backward_state(uh, P, D.status, PA.offsets, PA.asset_idx, nnz, st, res->state)) return rc2;
    }
    // ---- unpack
    UnpackArgs UA;
    UA.M = M; UA.Npad = Npad; UA.offsets = PA.offsets; UA.asset_idx = PA.asset_idx; UA.inv_perm = U.d_inv_perm;
    UA.W = P.W; UA.nnz = nnz;
    const bool w_dev = is_dev(res->w);
    UA.out = w_dev ? res->w : ragged_out;
    if (nnz > 0) SC.prof.run(PRISM_K_UNPACK, 1, st, [&] { k_unpack<<<(unsigned)cdiv64(nnz, 256), 256, 0, st>>>(UA); });
    if (!w_dev) cudaMemcpyAsync(res->w, ragged_out, nnz * 8, cudaMemcpyDeviceToHost, st);
    auto out = [&](void* dst, const void* src, size_t bytes) {
        if (dst) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
    };
    out(res->status, D.status, M * 4);
    out(res->iters, D.iters, M * 4);
    out(res->nu, P.nu, M * 8);
    out(res->lambda_band, P.lam, (size_t)M * S * 8);
    out(res->theta, P.theta, M * 8);
    out(res->diag, P.diag, (size_t)M * PRISM_NDIAG * 8);
    out(res->kappa, P.kappa, (size_t)M * K * 8);
    cudaEventRecord(SC.ev[5], st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_error(std::string("solve failed: ") + cudaGetErrorString(e)); return PRISM_ERR_CUDA; }
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("solve failed: ") + cudaGetErrorString(e)); return PRISM_ERR_CUDA; }
    res->t_phase_ms[0] = ms_between(SC.ev[0], SC.ev[1]);
    res->t_phase_ms[1] = ms_between(SC.ev[1], SC.ev[2]);
    res->t_phase_ms[2] = ms_between(SC.ev[2], SC.ev[3]);
    res->t_phase_ms[3] = ms_between(SC.ev[3], SC.ev[4]);
    res->t_device_ms = ms_between(SC.ev[0], SC.ev[5]);
    res->device_bytes = (int64_t)(SC.arena_bytes + U.bytes);
    int64_t nl = 0;
    for (int q = 0; q < PRISM_NKCLASS; ++q) {
        res->kernel_launches[q] = SC.prof.launches[q];
        res->kernel_ms[q] = 0.0;
        nl += SC.prof.launches[q];
    }
    for (auto& mk : SC.prof.marks) res->kernel_ms[mk.cls] += ms_between(mk.a, mk.b);
    res->stream_entries = res->stream_candidates = 0;
    if (D.pcount) {
        unsigned long long pc[2] = {0, 0};
        cudaMemcpy(pc, D.pcount, 16, cudaMemcpyDeviceToHost);
        res->stream_candidates = (int64_t)pc[0];
        res->stream_entries = (int64_t)pc[1];
    }
    res->n_launches = nl;
    res->t_call_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_call0).count();
    (void)plain;
    return PRISM_OK;
}

}  // namespace prism

extern "C" void prism_default_opts(prism_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps_kkt = 1e-6;
    o->eps_admm = 5e-4;
    o->rho0 = 3.0;
    o->alpha = 1.5;
    o->time_budget_s = 0.0;
    o->max_iter = 4000;
    o->check_every = 20;
    o->min_iter = 20;
    o->polish_rounds = 8;
    o->precision = PRISM_BATCHED_BF16;
    o->use_graph = 1;
    o->fuse_prox = 1;
    o->stream_after = 6;
    o->adapt_every = 25;
    o->chains = 0;
    o->polish_overlap = 0.0;
    o->keep_for_backward = 0;
    o->cuda_stream = nullptr;
}

extern "C" int prism_solve_batch(prism_universe* uh, const prism_batch* b, const prism_solve_opts* opts,
                                 prism_result* res) {
    using namespace prism;
    if (!uh || !b || !res) { set_error("NULL argument"); return PRISM_ERR_ARGUMENT; }
    prism_solve_opts o;
    if (opts) o = *opts; else prism_default_opts(&o);
    if (b->n_accounts < 1) { set_error("n_accounts must be >= 1"); return PRISM_ERR_ARGUMENT; }
    if (!b->offsets || !b->w0 || !b->lower || !b->upper || !b->tc || !b->band_lo || !b->band_hi) {
        set_error("required batch array is NULL");
        return PRISM_ERR_ARGUMENT;
    }
    if (!res->w || !res->status) { set_error("result w and status are required"); return PRISM_ERR_ARGUMENT; }
    if (b->lot_offsets && (!b->lot_size || !b->lot_kappa)) { set_error("lot arrays incomplete"); return PRISM_ERR_ARGUMENT; }
    if (!(o.eps_kkt > 0) || !(o.eps_admm > 0) || !(o.rho0 > 0) || !(o.alpha > 0 && o.alpha < 2) ||
        o.max_iter < 1 || o.check_every < 1 || o.g2_sets < 0 || o.g2_sets > 64 || o.ragged_layout < 0 ||
        o.ragged_layout > 2 || o.fold_products < 0 || o.fold_products > 1 || o.adapt_every < 0 ||
        o.xupdate_form < 0 || o.xupdate_form > 1) {
        set_error("invalid options");
        return PRISM_ERR_ARGUMENT;
    }
    if (o.keep_for_backward && !res->state) { set_error("keep_for_backward needs res->state"); return PRISM_ERR_ARGUMENT; }
    if (o.keep_for_backward && (o.precision == PRISM_PLAIN_FP32 || o.precision == PRISM_PLAIN_FP64)) {
        set_error("keep_for_backward is available in the batched modes");
        return PRISM_ERR_UNSUPPORTED;
    }
    if (o.keep_for_backward && (b->w_bench || b->factor_lo || b->factor_hi)) {
        set_error("keep_for_backward does not take a benchmark or factor-exposure bounds");
        return PRISM_ERR_UNSUPPORTED;
    }
    if (o.keep_for_backward) *res->state = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    if (o.precision == PRISM_BATCHED_FP32) return solve_core(uh, b, &o, res, false, false);
    if (o.precision == PRISM_BATCHED_BF16) {
        if (!tc_available()) {
            set_error("BATCHED_BF16 needs the tcgen05 product kernels, which this build does not provide");
            return PRISM_ERR_UNSUPPORTED;
        }
        return solve_core(uh, b, &o, res, true, false);
    }
    if (o.precision != PRISM_PLAIN_FP32 && o.precision != PRISM_PLAIN_FP64) {
        set_error("unknown precision mode");
        return PRISM_ERR_ARGUMENT;
    }
    const bool fp64 = o.precision == PRISM_PLAIN_FP64;
    // PLAIN_FP32 / PLAIN_FP64: one account per launch sequence (the single-account form)
    std::vector<int64_t> offs;
    if (int rc = to_host(b->offsets, (size_t)b->n_accounts + 1, offs)) return rc;
    const int S = uh->u.S;
    double tdev = 0, tph[4] = {0, 0, 0, 0}, kms[PRISM_NKCLASS] = {};
    int64_t dbytes = 0, nlaunch = 0, kl[PRISM_NKCLASS] = {};
    for (int a = 0; a < b->n_accounts; ++a) {
        int64_t sub_off[2] = {0, offs[a + 1] - offs[a]};
        prism_batch sb = *b;
        sb.n_accounts = 1;
        sb.offsets = sub_off;
        const int64_t e0 = offs[a];
        sb.asset_idx = b->asset_idx ? b->asset_idx + e0 : nullptr;
        sb.w0 = b->w0 + e0; sb.lower = b->lower + e0; sb.upper = b->upper + e0; sb.tc = b->tc + e0;
        sb.band_lo = b->band_lo + (size_t)a * S; sb.band_hi = b->band_hi + (size_t)a * S;
        sb.turnover_cap = b->turnover_cap ? b->turnover_cap + a : nullptr;
        sb.mu_tilt = b->mu_tilt ? b->mu_tilt + e0 : nullptr;
        sb.w_bench = b->w_bench ? b->w_bench + e0 : nullptr;
        sb.factor_lo = b->factor_lo ? b->factor_lo + (size_t)a * uh->u.K : nullptr;
        sb.factor_hi = b->factor_hi ? b->factor_hi + (size_t)a * uh->u.K : nullptr;
        std::vector<int64_t> lot_sub;
        if (b->lot_offsets) {
            std::vector<int64_t> lo_all;
            if (int rc = to_host(b->lot_offsets + e0, (size_t)(sub_off[1] + 1), lo_all)) return rc;
            lot_sub.resize(lo_all.size());
            for (size_t q = 0; q < lo_all.size(); ++q) lot_sub[q] = lo_all[q] - lo_all[0];
            sb.lot_offsets = lot_sub.data();
            sb.lot_size = b->lot_size + lo_all[0];
            sb.lot_kappa = b->lot_kappa + lo_all[0];
        }
        prism_result r1 = *res;
        r1.w = res->w + e0;
        r1.status = res->status + a;
        r1.iters = res->iters ? res->iters + a : nullptr;
        r1.nu = res->nu ? res->nu + a : nullptr;
        r1.lambda_band = res->lambda_band ? res->lambda_band + (size_t)a * S : nullptr;
        r1.theta = res->theta ? res->theta + a : nullptr;
        r1.diag = res->diag ? res->diag + (size_t)a * PRISM_NDIAG : nullptr;
        r1.kappa = res->kappa ? res->kappa + (size_t)a * uh->u.K : nullptr;
        int rc = solve_core(uh, &sb, &o, &r1, false, true, fp64);
        if (rc != PRISM_OK) return rc;
        tdev += r1.t_device_ms;
        for (int q = 0; q < 4; ++q) tph[q] += r1.t_phase_ms[q];
        nlaunch += r1.n_launches;
        for (int q = 0; q < PRISM_NKCLASS; ++q) { kms[q] += r1.kernel_ms[q]; kl[q] += r1.kernel_launches[q]; }
        dbytes = std::max(dbytes, r1.device_bytes);
    }
    res->t_device_ms = tdev;
    for (int q = 0; q < 4; ++q) res->t_phase_ms[q] = tph[q];
    res->device_bytes = dbytes;
    res->n_launches = nlaunch;
    for (int q = 0; q < PRISM_NKCLASS; ++q) { res->kernel_ms[q] = kms[q]; res->kernel_launches[q] = kl[q]; }
    res->stream_entries = res->stream_candidates = 0;
    res->t_call_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return PRISM_OK;
}


