// noalloc.cu -- prism_polish_noalloc: the FP64 polish / certification of caller-supplied
// weights, with every byte of device scratch taken from a fixed static array.
//
// Some callers cannot allocate device memory at the moment they need a result: a
// process that has reserved all of the GPU's memory up front for its own pool, or a
// host thread that must not block on the allocator inside a latency budget.
// For them this entry point runs the same polish / certification kernels as
// prism_solve_batch on weights they already hold (for example the result of an
// earlier solve, or a warm start), and takes its scratch from g_noalloc_scratch
// instead of allocating it.
//
// Limits (checked, PRISM_ERR_ARGUMENT beyond them): at most NA_MAX_ACCOUNTS
// accounts, at most NA_MAX_ENTRIES = accounts x padded universe width, at most
// NA_FMAX free weights per account (more make that account's polish fall back),
// no tax lots.
#include <cfloat>
#include <chrono>
#include <cstring>

#include "common.cuh"
#include "polish.h"

namespace prism {

constexpr int NA_MAX_ACCOUNTS = 32;
constexpr int64_t NA_MAX_ENTRIES = 131072;
constexpr int NA_FMAX = 512;
constexpr int NA_MAX_DEVICES = 64;

// Bytes the carve below needs at the limits, with 256-byte alignment slack per region.
constexpr size_t na_round(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t NA_BYTES =
    na_round(NA_MAX_ENTRIES * 8) * 5 +                       // w0, lo, up, c, W (FP64, sorted layout)
    na_round(NA_MAX_ENTRIES * 4) * 2 +                       // z (FP32), member flags
    na_round(NA_MAX_ENTRIES * 4) * 4 +                       // FP32 copies of w0, lo, up, c
    na_round(NA_MAX_ENTRIES) +                               // entry states
    na_round(NA_MAX_ENTRIES * 8) * 6 +                       // staged ragged w0, lo, up, tc, w_in, w_out
    na_round(NA_MAX_ENTRIES * 4) +                           // staged asset_idx
    na_round((NA_MAX_ACCOUNTS + 1) * 8) +                    // staged offsets
    na_round((size_t)NA_MAX_ACCOUNTS * SMAX * 8) * 3 +       // band_lo, band_hi, lambda
    na_round((size_t)NA_MAX_ACCOUNTS * SMAX * 4) * 3 +       // wband, synthetic eta_hi / eta_lo
    na_round(NA_MAX_ACCOUNTS * 8) * 3 +                      // tau, nu, theta
    na_round(NA_MAX_ACCOUNTS * 4) * 7 +                      // wcap, done, skip, status, nu_f, theta_f, iters
    na_round((size_t)NA_MAX_ACCOUNTS * PRISM_NDIAG * 8) +    // diag
    na_round((size_t)NA_MAX_ACCOUNTS * NA_FMAX * 4) * 2 +    // free / nonzero lists
    na_round((size_t)NA_MAX_ACCOUNTS * NA_FMAX * 8) +        // cap signs of free entries
    na_round((size_t)NA_MAX_ACCOUNTS * NA_FMAX * (PMAXROWS + 1) * 8) +   // Woodbury columns
    na_round((size_t)NA_MAX_ACCOUNTS * NA_FMAX * 8) +        // 1/d of free entries
    na_round((size_t)NA_MAX_ACCOUNTS * KMAX * 8) +           // f .* h (FP64)
    na_round((size_t)NA_MAX_ACCOUNTS * KMAX * 4) +           // f .* h (FP32)
    na_round(NA_MAX_ACCOUNTS * 8) * 2 +                      // quad, fhmax
    na_round(NA_MAX_ACCOUNTS * 4) +                          // ndep
    na_round(16) +                                           // pending counter
    na_round(16);                                            // error flags

// The scratch: resident on every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of g_noalloc_scratch per device ordinal (host-side stand-in is not usable).
static unsigned char* g_na_base[NA_MAX_DEVICES] = {};

struct NaPack {
    int M, N, Npad;
    int64_t nnz;
    const int64_t* offsets;
    const int32_t* asset_idx;
    const double *w0, *lo, *up, *tc, *w_in;
    const int* inv_perm;
    double *W0, *LO, *UP, *C;
    float *W0f, *LOf, *UPf, *Cf;
    float* Z;
    int* member;
    int* err;
};

__global__ void k_na_pack(NaPack A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.nnz) return;
    int lo = 0, hi = A.M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.offsets[mid] <= e) lo = mid; else hi = mid;
    }
    const int a = lo;
    const int i = A.asset_idx ? A.asset_idx[e] : int(e - A.offsets[a]);
    if (i < 0 || i >= A.N) { atomicOr(A.err, 1); return; }
    const double w0 = A.w0[e], l = A.lo[e], u = A.up[e], c = A.tc[e], w = A.w_in[e];
    if (!(isfinite(w0) && isfinite(l) && isfinite(u) && isfinite(c) && isfinite(w)) || l > u || c < 0) {
        atomicOr(A.err, 2);
        return;
    }
    const size_t d = (size_t)a * A.Npad + A.inv_perm[i];
    if (atomicExch(&A.member[d], 1) != 0) { atomicOr(A.err, 4); return; }
    A.W0[d] = w0; A.LO[d] = l; A.UP[d] = u; A.C[d] = c;
    A.W0f[d] = float(w0); A.LOf[d] = float(l); A.UPf[d] = float(u); A.Cf[d] = float(c);
    A.Z[d] = float(w);
}

// Working rows the given weights hold at an edge, written as the multiplier signals the
// classification kernel reads (band held at hi: eta_hi > nu; at lo: eta_lo < nu; cap: theta > 0).
// The given weights are a warm start, so a row within 1e-4 (relative) of its edge starts in the
// working set; the polish drops a row whose multiplier comes out with the wrong sign.
__global__ void k_na_rows(int M, int S, int Npad, const int* sec_start, const double* W0, const double* LO,
                          const float* Z, const double* band_lo, const double* band_hi, const double* tau,
                          float* nu_f, float* eta_hi_f, float* eta_lo_f, float* theta_f) {
    const int a = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t base = (size_t)a * Npad;
    __shared__ double turn_w[32];
    double turn = 0.0;
    for (int s = warp; s < S; s += nw) {
        double sw = 0.0, fl = 0.0;
        for (int p = sec_start[s] + lane; p < sec_start[s + 1]; p += 32) {
            const double w = double(Z[base + p]);
            sw += w;
            fl += LO[base + p];
            turn += fabs(w - W0[base + p]);
        }
        sw = warp_sum(sw);
        fl = warp_sum(fl);
        if (lane == 0) {
            const double hi = band_hi[a * S + s], lo = band_lo[a * S + s];
            const double tol = 1e-4 * fmax(1.0, fabs(hi));
            eta_hi_f[a * S + s] = (isfinite(hi) && fabs(sw - hi) <= tol) ? 1.f : -FLT_MAX;
            eta_lo_f[a * S + s] = (isfinite(lo) && lo > fl + 1e-12 && fabs(sw - lo) <= 1e-4 * fmax(1.0, fabs(lo)))
                                      ? -1.f : FLT_MAX;
        }
    }
    turn = warp_sum(turn);
    if (lane == 0) turn_w[warp] = turn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += turn_w[w];
        nu_f[a] = 0.f;
        theta_f[a] = (isfinite(tau[a]) && fabs(t - tau[a]) <= 1e-4 * fmax(1.0, tau[a])) ? 1.f : 0.f;
    }
}

__global__ void k_na_unpack(int M, int Npad, int64_t nnz, const int64_t* offsets, const int32_t* asset_idx,
                            const int* inv_perm, const double* W, double* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offsets[mid] <= e) lo = mid; else hi = mid;
    }
    const int i = asset_idx ? asset_idx[e] : int(e - offsets[lo]);
    out[e] = W[(size_t)lo * Npad + inv_perm[i]];
}

__global__ void k_na_fill(double* p, int n, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Where a caller pointer lives: 0 host memory (staged through the scratch), 1 memory the
// kernels on `device` can read in place (that device's memory, or managed memory), -1 device
// memory of another GPU (rejected: the kernels would read it across devices).
static int na_where(const void* p, int device) {
    if (!p) return 0;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) { cudaGetLastError(); return 0; }
    if (attr.type == cudaMemoryTypeManaged) return 1;
    if (attr.type == cudaMemoryTypeDevice) return attr.device == device ? 1 : -1;
    return 0;
}

// Bump carve over the static array; returns nullptr past the end.
struct NaCarve {
    unsigned char* base;
    size_t used = 0;
    bool overflow = false;
    template <typename T>
    T* take(size_t n) {
        const size_t bytes = na_round(n * sizeof(T));
        if (used + bytes > NA_BYTES) { overflow = true; return nullptr; }
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

static int na_fail(int code, const char* msg) {
    set_error(msg);
    return code;
}

}  // namespace prism

extern "C" int prism_polish_noalloc(prism_universe* uh, const prism_batch* b, const double* w_in,
                                    const prism_solve_opts* opts, prism_result* res) {
    using namespace prism;
    const auto t0 = std::chrono::steady_clock::now();
    if (!uh || !b || !w_in || !res || !res->w || !res->status) return na_fail(PRISM_ERR_ARGUMENT, "NULL argument");
    if (!b->offsets || !b->w0 || !b->lower || !b->upper || !b->tc || !b->band_lo || !b->band_hi)
        return na_fail(PRISM_ERR_ARGUMENT, "required batch array is NULL");
    if (b->lot_offsets) return na_fail(PRISM_ERR_UNSUPPORTED, "prism_polish_noalloc does not take tax lots");
    if (b->mu_tilt || b->w_bench || b->factor_lo || b->factor_hi)
        return na_fail(PRISM_ERR_UNSUPPORTED,
                       "prism_polish_noalloc does not take tilts, a benchmark or factor-exposure bounds");
    Universe& U = uh->u;
    const int M = b->n_accounts, N = U.N, Npad = U.Npad, K = U.K, S = U.S;
    if (M < 1 || M > NA_MAX_ACCOUNTS)
        return na_fail(PRISM_ERR_ARGUMENT, "prism_polish_noalloc: n_accounts must be in [1, 32]");
    if ((int64_t)M * Npad > NA_MAX_ENTRIES)
        return na_fail(PRISM_ERR_ARGUMENT,
                       "prism_polish_noalloc: n_accounts x padded universe width exceeds 131072 entries");
    if (cudaSetDevice(U.device) != cudaSuccess || U.device < 0 || U.device >= NA_MAX_DEVICES)
        return na_fail(PRISM_ERR_CUDA, "cudaSetDevice failed");
    // one-time set-up per device: the device address of the static scratch array
    if (!g_na_base[U.device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
            return PRISM_ERR_CUDA;
        }
        g_na_base[U.device] = static_cast<unsigned char*>(ptr);
    }
    prism_solve_opts o;
    if (opts) o = *opts; else prism_default_opts(&o);
    cudaStream_t st = o.cuda_stream ? (cudaStream_t)o.cuda_stream : U.stream;
    // offsets on the host (fixed-size buffer: no allocation)
    // every caller pointer is host memory or memory of this universe's device
    {
        const void* ptrs[] = {b->offsets, b->asset_idx, b->w0, b->lower, b->upper, b->tc, b->band_lo, b->band_hi,
                              b->turnover_cap, w_in, res->w, res->status, res->iters, res->nu, res->lambda_band,
                              res->theta, res->diag};
        for (const void* q : ptrs)
            if (na_where(q, U.device) < 0)
                return na_fail(PRISM_ERR_ARGUMENT, "prism_polish_noalloc: a buffer is on another GPU than the universe");
    }
    int64_t offs[NA_MAX_ACCOUNTS + 1];
    if (na_where(b->offsets, U.device) > 0) {
        if (cudaMemcpy(offs, b->offsets, (M + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return na_fail(PRISM_ERR_CUDA, "offsets copy failed");
    } else {
        std::memcpy(offs, b->offsets, (M + 1) * sizeof(int64_t));
    }
    if (offs[0] != 0) return na_fail(PRISM_ERR_ARGUMENT, "offsets[0] must be 0");
    for (int a = 0; a < M; ++a) {
        const int64_t len = offs[a + 1] - offs[a];
        if (len < 0 || len > N) return na_fail(PRISM_ERR_ARGUMENT, "bad offsets");
        if (!b->asset_idx && len != N)
            return na_fail(PRISM_ERR_ARGUMENT, "without asset_idx every account must span the universe");
    }
    const int64_t nnz = offs[M];
    const size_t MN = (size_t)M * Npad;
    // carve the static array
    NaCarve cv{g_na_base[U.device]};
    double* W0 = cv.take<double>(MN); double* LO = cv.take<double>(MN);
    double* UP = cv.take<double>(MN); double* Cc = cv.take<double>(MN);
    double* W = cv.take<double>(MN);
    float* Z = cv.take<float>(MN);
    float* W0f = cv.take<float>(MN); float* LOf = cv.take<float>(MN);
    float* UPf = cv.take<float>(MN); float* Cf = cv.take<float>(MN);
    int* member = cv.take<int>(MN);
    int8_t* stt = cv.take<int8_t>(MN);
    double* s_w0 = cv.take<double>(nnz); double* s_lo = cv.take<double>(nnz);
    double* s_up = cv.take<double>(nnz); double* s_tc = cv.take<double>(nnz);
    double* s_win = cv.take<double>(nnz); double* s_out = cv.take<double>(nnz);
    int32_t* s_idx = cv.take<int32_t>(nnz);
    int64_t* s_off = cv.take<int64_t>(M + 1);
    double* blo = cv.take<double>((size_t)M * S); double* bhi = cv.take<double>((size_t)M * S);
    double* lam = cv.take<double>((size_t)M * S);
    int* wband = cv.take<int>((size_t)M * S);
    float* eta_hi = cv.take<float>((size_t)M * S); float* eta_lo = cv.take<float>((size_t)M * S);
    double* tau = cv.take<double>(M); double* nu = cv.take<double>(M); double* theta = cv.take<double>(M);
    int* wcap = cv.take<int>(M); int* done = cv.take<int>(M); int* skip = cv.take<int>(M);
    int* status = cv.take<int>(M); float* nu_f = cv.take<float>(M); float* theta_f = cv.take<float>(M);
    int* iters = cv.take<int>(M);
    double* diag = cv.take<double>((size_t)M * PRISM_NDIAG);
    const int FMAX = std::min(N, NA_FMAX);
    int* Fl = cv.take<int>((size_t)M * FMAX); int* NZl = cv.take<int>((size_t)M * FMAX);
    double* Fsig = cv.take<double>((size_t)M * FMAX);
    double* Y = cv.take<double>((size_t)M * FMAX * (PMAXROWS + 1));
    double* Fdinv = cv.take<double>((size_t)M * FMAX);
    double* fh64 = cv.take<double>((size_t)M * KMAX);
    float* fh32 = cv.take<float>((size_t)M * K);
    double* quad = cv.take<double>(M);
    double* fhmax = cv.take<double>(M);
    int* ndep = cv.take<int>(M);
    int* pending = cv.take<int>(4);
    int* err = cv.take<int>(4);
    if (cv.overflow) return na_fail(PRISM_ERR_ARGUMENT, "prism_polish_noalloc: request exceeds the static scratch");
    // stage the inputs (host pointers are copied into the scratch, device pointers used in place)
    auto stage = [&](const void* src, void* dst, size_t bytes) -> const void* {
        if (na_where(src, U.device) > 0) return src;
        cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        return dst;
    };
    NaPack A;
    A.M = M; A.N = N; A.Npad = Npad; A.nnz = nnz;
    cudaMemcpyAsync(s_off, offs, (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    A.offsets = s_off;
    A.asset_idx = b->asset_idx ? (const int32_t*)stage(b->asset_idx, s_idx, nnz * 4) : nullptr;
    A.w0 = (const double*)stage(b->w0, s_w0, nnz * 8);
    A.lo = (const double*)stage(b->lower, s_lo, nnz * 8);
    A.up = (const double*)stage(b->upper, s_up, nnz * 8);
    A.tc = (const double*)stage(b->tc, s_tc, nnz * 8);
    A.w_in = (const double*)stage(w_in, s_win, nnz * 8);
    A.inv_perm = U.d_inv_perm;
    A.W0 = W0; A.LO = LO; A.UP = UP; A.C = Cc; A.Z = Z; A.member = member; A.err = err;
    A.W0f = W0f; A.LOf = LOf; A.UPf = UPf; A.Cf = Cf;
    // the array keeps the previous call's contents: clear everything read before written
    cudaMemsetAsync(W0, 0, MN * 8, st); cudaMemsetAsync(LO, 0, MN * 8, st);
    cudaMemsetAsync(UP, 0, MN * 8, st); cudaMemsetAsync(Cc, 0, MN * 8, st);
    cudaMemsetAsync(W, 0, MN * 8, st); cudaMemsetAsync(Z, 0, MN * 4, st);
    cudaMemsetAsync(W0f, 0, MN * 4, st); cudaMemsetAsync(LOf, 0, MN * 4, st);
    cudaMemsetAsync(UPf, 0, MN * 4, st); cudaMemsetAsync(Cf, 0, MN * 4, st);
    cudaMemsetAsync(member, 0, MN * 4, st); cudaMemsetAsync(err, 0, 16, st);
    cudaMemsetAsync(done, 0, M * 4, st); cudaMemsetAsync(skip, 0, M * 4, st);
    cudaMemsetAsync(status, 0, M * 4, st); cudaMemsetAsync(iters, 0, M * 4, st);
    cudaMemsetAsync(diag, 0, (size_t)M * PRISM_NDIAG * 8, st);
    cudaMemsetAsync(nu, 0, M * 8, st); cudaMemsetAsync(theta, 0, M * 8, st);
    cudaMemsetAsync(lam, 0, (size_t)M * S * 8, st);
    cudaMemcpyAsync(blo, b->band_lo, (size_t)M * S * 8, cudaMemcpyDefault, st);
    cudaMemcpyAsync(bhi, b->band_hi, (size_t)M * S * 8, cudaMemcpyDefault, st);
    if (b->turnover_cap) cudaMemcpyAsync(tau, b->turnover_cap, M * 8, cudaMemcpyDefault, st);
    else k_na_fill<<<1, 64, 0, st>>>(tau, M, INFINITY);
    if (nnz > 0) k_na_pack<<<(unsigned)cdiv64(nnz, 256), 256, 0, st>>>(A);
    int herr = 0;
    cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return na_fail(PRISM_ERR_CUDA, "staging failed");
    if (herr) return na_fail(PRISM_ERR_ARGUMENT, "invalid batch input or weights (index, non-finite, bounds or duplicate)");
    k_na_rows<<<M, 256, 0, st>>>(M, S, Npad, U.d_sec_start, W0, LO, Z, blo, bhi, tau, nu_f, eta_hi, eta_lo, theta_f);
    // the polish / certification kernels of prism_solve_batch, pointed at the static scratch
    PolDev P;
    P.M = M; P.N = N; P.Npad = Npad; P.K = K; P.S = S;
    P.B64 = U.d_B64; P.f64 = U.d_f64; P.d64 = U.d_d64; P.mu64 = U.d_mu64;
    P.B32 = U.d_B32; P.B32p = U.d_B32p; P.Bn1 = U.d_Bn1; P.Bn1f = U.d_Bn1f; P.mu32 = U.d_mu32;
    P.w0f = W0f; P.lof = LOf; P.upf = UPf; P.cf = Cf;
    P.Fdinv = Fdinv; P.fh64 = fh64; P.fh32 = fh32; P.quad = quad; P.fhmax = fhmax; P.ndep = ndep; P.pending = pending;
    P.sec_start = U.d_sec_start; P.sector = U.d_sector;
    P.w0 = W0; P.lo = LO; P.up = UP; P.c = Cc;
    P.band_lo = blo; P.band_hi = bhi; P.tau = tau;
    P.z = Z; P.nu_f = nu_f; P.eta_hi_f = eta_hi; P.eta_lo_f = eta_lo; P.theta_f = theta_f;
    P.skip = skip; P.st = stt; P.wband = wband; P.wcap = wcap; P.done = done;
    P.Flist = Fl; P.NZlist = NZl; P.Fsig = Fsig; P.Y = Y; P.FMAX = FMAX;
    P.dmin = U.dmin;
    P.kappa = nullptr;
    P.W = W; P.nu = nu; P.lam = lam; P.theta = theta; P.diag = diag; P.status = status;
    launch_classify(P, st);
    const int rounds = std::max(1, o.polish_rounds);
    launch_polish(P, rounds, st);
    launch_fallback(P, st);
    launch_finish_status(P, o.eps_kkt, st);
    const bool w_dev = na_where(res->w, U.device) > 0;
    if (nnz > 0)
        k_na_unpack<<<(unsigned)cdiv64(nnz, 256), 256, 0, st>>>(M, Npad, nnz, s_off, A.asset_idx, U.d_inv_perm, W,
                                                                 w_dev ? res->w : s_out);
    if (!w_dev) cudaMemcpyAsync(res->w, s_out, nnz * 8, cudaMemcpyDeviceToHost, st);
    auto out = [&](void* dst, const void* src, size_t bytes) {
        if (dst) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
    };
    out(res->status, status, M * 4);
    out(res->iters, iters, M * 4);
    out(res->nu, nu, M * 8);
    out(res->lambda_band, lam, (size_t)M * S * 8);
    out(res->theta, theta, M * 8);
    out(res->diag, diag, (size_t)M * PRISM_NDIAG * 8);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("prism_polish_noalloc: ") + cudaGetErrorString(e));
        return PRISM_ERR_CUDA;
    }
    res->t_device_ms = 0.0;
    for (double& x : res->t_phase_ms) x = 0.0;
    for (double& x : res->kernel_ms) x = 0.0;
    for (int64_t& x : res->kernel_launches) x = 0;
    // fill (no cap given), pack, rows, classify, polish, fallback (2), status, unpack
    res->n_launches = (b->turnover_cap ? 0 : 1) + (nnz > 0 ? 2 : 0) + 1 + 1 + 1 + 2 + 1;
    res->device_bytes = (int64_t)NA_BYTES;
    res->t_call_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    set_error("");
    return PRISM_OK;
}
