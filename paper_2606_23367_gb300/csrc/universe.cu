// universe.cu -- prism_create_universe / prism_destroy_universe.
//
// The risk model Sigma = B F B' + D (Eq. 1, factor-structured risk with O(N K)
// products, Sec. 4.2) is copied to the device once, in an asset order that
// makes each sector a contiguous range (the projection step reduces per
// sector). Alongside the FP64 copy the library keeps FP32 and BF16 copies of
// B (row-major and transposed for the tensor-core products) and, for each
// point of the penalty grid rho_j, the inverse of the Woodbury capacitance
//     C_j = (2F)^{-1} + B' Delta_j^{-1} B,   Delta_j = diag(2 d + rho_j),
// which turns the ADMM x-update (2 Sigma + rho I) x = r into K x K work.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>

#include "common.cuh"

namespace prism {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

// G_j[k1][k2] = sum_i B[i][k1] B[i][k2] / (2 d_i + rho_j), FP32 products summed
// in FP32 over chunks of 128 assets and in FP64 across chunks. One block per
// (j, 8-row stripe of k1); B rows staged through shared memory.
template <typename TB>
__global__ void k_gram(const TB* __restrict__ B, const float* __restrict__ d, int N, int K,
                       double* __restrict__ G) {
    const int j = blockIdx.x;
    const int k1_0 = blockIdx.y * 8;
    const float rho = float(RHO_MIN * pow(10.0, double(j) / RHO_PER_DECADE));
    __shared__ float sB[128][KMAX + 1];
    __shared__ float sw[128];
    const int t = threadIdx.x;            // 256 threads: pair (k1 = k1_0 + t/32 ... )
    // each thread owns up to 2 (k1, k2) pairs: k1 = k1_0 + (t >> 5), k2 = (t & 31) and +32
    const int k1 = k1_0 + (t >> 5);
    const int k2a = t & 31, k2b = (t & 31) + 32;
    double acc_a = 0.0, acc_b = 0.0;
    for (int i0 = 0; i0 < N; i0 += 128) {
        __syncthreads();
        for (int e = t; e < 128 * K; e += 256) {
            int r = e / K, c = e % K;
            int i = i0 + r;
            sB[r][c] = (i < N) ? float(B[(size_t)i * K + c]) : 0.f;
        }
        for (int r = t; r < 128; r += 256) {
            int i = i0 + r;
            sw[r] = (i < N) ? 1.0f / (2.0f * d[i] + rho) : 0.f;
        }
        __syncthreads();
        if (k1 < K) {
            float pa = 0.f, pb = 0.f;
            for (int r = 0; r < 128; ++r) {
                float bw = sB[r][k1] * sw[r];
                if (k2a < K) pa = fmaf(bw, sB[r][k2a], pa);
                if (k2b < K) pb = fmaf(bw, sB[r][k2b], pb);
            }
            acc_a += pa;
            acc_b += pb;
        }
    }
    if (k1 < K) {
        if (k2a < K) G[((size_t)j * K + k1) * K + k2a] = acc_a;
        if (k2b < K) G[((size_t)j * K + k1) * K + k2b] = acc_b;
    }
}

// Cinv_j = ((2F)^{-1} + G_j)^{-1} by an FP64 Cholesky factorisation in shared
// memory, then an explicit inverse (columns by forward/back substitution). With
// `split` the diagonal term is (2 f_k + rho_j)^{-1} instead: the capacitance of the
// x-update when the factor exposures are split off with the same penalty. Gout, when
// given, receives the FP32 copy of G_j.
__global__ void k_cinv(const double* __restrict__ G, const double* __restrict__ f, int K,
                       float* __restrict__ Cinv, int split, float* __restrict__ Gout) {
    const int j = blockIdx.x;
    __shared__ double L[KMAX][KMAX + 1];
    const int t = threadIdx.x;   // 64 threads
    const double rho = RHO_MIN * pow(10.0, double(j) / RHO_PER_DECADE);
    for (int e = t; e < K * K; e += blockDim.x) {
        int r = e / K, c = e % K;
        double v = G[((size_t)j * K + r) * K + c];
        if (Gout) Gout[((size_t)j * K + r) * K + c] = float(v);
        if (r == c) v += split ? 1.0 / (2.0 * f[r] + rho) : 1.0 / (2.0 * f[r]);
        L[r][c] = v;
    }
    __syncthreads();
    // right-looking Cholesky, lower triangle
    for (int c = 0; c < K; ++c) {
        if (t == 0) L[c][c] = sqrt(L[c][c]);
        __syncthreads();
        for (int r = c + 1 + t; r < K; r += blockDim.x) L[r][c] /= L[c][c];
        __syncthreads();
        for (int r = c + 1 + t; r < K; r += blockDim.x)
            for (int q = c + 1; q <= r; ++q) L[r][q] -= L[r][c] * L[q][c];
        __syncthreads();
    }
    // column t of the inverse: solve L L' x = e_t
    if (t < K) {
        double x[KMAX];
        for (int r = 0; r < K; ++r) {
            double s = (r == t) ? 1.0 : 0.0;
            for (int q = 0; q < r; ++q) s -= L[r][q] * x[q];
            x[r] = s / L[r][r];
        }
        for (int r = K - 1; r >= 0; --r) {
            double s = x[r];
            for (int q = r + 1; q < K; ++q) s -= L[q][r] * x[q];
            x[r] = s / L[r][r];
        }
        for (int r = 0; r < K; ++r) Cinv[((size_t)j * K + r) * K + t] = float(x[r]);
    }
}

__global__ void k_convert_B(const double* __restrict__ B64, int Npad, int K, float* __restrict__ B32,
                            float* __restrict__ B32p, __nv_bfloat16* __restrict__ B16, __nv_bfloat16* __restrict__ Bt16,
                            __nv_bfloat16* __restrict__ B16p, __nv_bfloat16* __restrict__ Bt16p) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)Npad * K) return;
    int i = int(e / K), k = int(e % K);
    double b = B64[e];
    B32[e] = float(b);
    B32p[(size_t)i * KMAX + k] = float(b);
    __nv_bfloat16 h = __float2bfloat16_rn(float(b));
    B16[e] = h;
    Bt16[(size_t)k * Npad + i] = h;
    B16p[(size_t)i * KMAX + k] = h;
    Bt16p[(size_t)k * Npad + i] = h;
}

__global__ void k_bf16_to_float(const __nv_bfloat16* __restrict__ a, float* __restrict__ b, size_t n) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = __bfloat162float(a[e]);
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Copy n elements of T from a host or device pointer to a host vector.
template <typename T>
static int fetch(const T* src, size_t n, std::vector<T>& dst) {
    dst.resize(n);
    if (n == 0) return PRISM_OK;
    if (is_device_ptr(src)) {
        PRISM_CUDA_TRY(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(dst.data(), src, n * sizeof(T));
    }
    return PRISM_OK;
}

static void free_universe(Universe& U) {
    void* ptrs[] = {U.d_inv_perm, U.d_perm, U.d_sec_start, U.d_sector, U.d_qseg, U.d_sseg, U.d_B64, U.d_f64, U.d_d64, U.d_Bn1, U.d_Bn1f,
                    U.d_mu64, U.d_B32, U.d_B32p, U.d_f32, U.d_d32, U.d_mu32, U.d_B16, U.d_Bt16, U.d_B16p, U.d_Bt16p,
                    U.d_Cinv32, U.d_Cinv16, U.d_G32, U.d_G16, U.d_CinvF32, U.d_CinvF16};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (U.stream) cudaStreamDestroy(U.stream);
    U = Universe();
}

template <typename T>
static int dalloc(Universe& U, T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return PRISM_ERR_ALLOCATION;
    }
    U.bytes += n * sizeof(T);
    return PRISM_OK;
}

#define TRY(x)                      \
    do {                            \
        int rc_ = (x);              \
        if (rc_ != PRISM_OK) {      \
            free_universe(U);       \
            return rc_;             \
        }                           \
    } while (0)

static int create(const prism_universe_desc* desc, Universe& U) {
    if (!desc) { set_error("desc is NULL"); return PRISM_ERR_ARGUMENT; }
    const int N = desc->n_assets, K = desc->n_factors, S = desc->n_sectors;
    if (N < 1 || K < 1 || K > KMAX || S < 1 || S > SMAX) {
        set_error("universe sizes out of range (N >= 1, 1 <= K <= 64, 1 <= S <= 64)");
        return PRISM_ERR_ARGUMENT;
    }
    if (!desc->B || !desc->f || !desc->d || !desc->mu || !desc->sector) {
        set_error("universe array is NULL");
        return PRISM_ERR_ARGUMENT;
    }
    int ndev = 0;
    PRISM_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (desc->device < 0 || desc->device >= ndev) {
        set_error("device ordinal out of range");
        return PRISM_ERR_ARGUMENT;
    }
    PRISM_CUDA_TRY(cudaSetDevice(desc->device));
    std::vector<double> B, f, d, mu;
    std::vector<int32_t> sec;
    int rc;
    if ((rc = fetch(desc->B, (size_t)N * K, B)) || (rc = fetch(desc->f, K, f)) ||
        (rc = fetch(desc->d, N, d)) || (rc = fetch(desc->mu, N, mu)) ||
        (rc = fetch(desc->sector, N, sec)))
        return rc;
    for (size_t e = 0; e < B.size(); ++e)
        if (!std::isfinite(B[e])) { set_error("B has a non-finite entry"); return PRISM_ERR_ARGUMENT; }
    for (int k = 0; k < K; ++k)
        if (!(f[k] > 0) || !std::isfinite(f[k])) { set_error("f must be positive and finite"); return PRISM_ERR_ARGUMENT; }
    for (int i = 0; i < N; ++i) {
        if (!(d[i] > 0) || !std::isfinite(d[i])) { set_error("d must be positive and finite"); return PRISM_ERR_ARGUMENT; }
        if (!std::isfinite(mu[i])) { set_error("mu has a non-finite entry"); return PRISM_ERR_ARGUMENT; }
        if (sec[i] < 0 || sec[i] >= S) { set_error("sector id out of range"); return PRISM_ERR_ARGUMENT; }
    }
    U.device = desc->device;
    U.N = N; U.K = K; U.S = S;
    U.dmin = *std::min_element(d.begin(), d.end());
    U.Npad = (N + 63) / 64 * 64;
    const int Npad = U.Npad;
    // stable sort of assets by sector
    U.perm.resize(N);
    std::iota(U.perm.begin(), U.perm.end(), 0);
    std::stable_sort(U.perm.begin(), U.perm.end(), [&](int a, int b) { return sec[a] < sec[b]; });
    U.inv_perm.resize(N);
    for (int p = 0; p < N; ++p) U.inv_perm[U.perm[p]] = p;
    U.sec_start.assign(S + 1, 0);
    for (int i = 0; i < N; ++i) U.sec_start[sec[i] + 1]++;
    for (int s = 0; s < S; ++s) U.sec_start[s + 1] += U.sec_start[s];
    std::vector<double> Bs((size_t)Npad * K, 0.0), ds(Npad, 1.0), mus(Npad, 0.0);
    std::vector<int> secs(Npad, -1);
    for (int p = 0; p < N; ++p) {
        int i = U.perm[p];
        std::memcpy(&Bs[(size_t)p * K], &B[(size_t)i * K], K * sizeof(double));
        ds[p] = d[i];
        mus[p] = mu[i];
        secs[p] = sec[i];
    }
    std::vector<float> f32(f.begin(), f.end()), d32(ds.begin(), ds.end()), mu32(mus.begin(), mus.end());
    // quarter / sector segments (sorted positions: sector ids are nondecreasing in p)
    U.nq = Npad / 32;
    std::vector<int> qseg(U.nq + 1, 0), sseg(S + 1, 0);
    for (int q = 0; q < U.nq; ++q) {
        int n = 0;
        for (int p = 32 * q; p < std::min(32 * q + 32, N); ++p)
            if (p == 32 * q || secs[p] != secs[p - 1]) { ++n; ++sseg[secs[p] + 1]; }
        qseg[q + 1] = qseg[q] + n;
    }
    for (int s = 0; s < S; ++s) sseg[s + 1] += sseg[s];
    U.nseg = qseg[U.nq];
    std::vector<double> bn1(Npad, 0.0);
    for (int p = 0; p < N; ++p)
        for (int k = 0; k < K; ++k) bn1[p] += std::fabs(Bs[(size_t)p * K + k]);
    std::vector<float> bn1f(bn1.begin(), bn1.end());
    cudaError_t se = cudaStreamCreateWithFlags(&U.stream, cudaStreamNonBlocking);
    if (se != cudaSuccess) { set_error(cudaGetErrorString(se)); return PRISM_ERR_CUDA; }
    TRY(dalloc(U, &U.d_inv_perm, N));
    TRY(dalloc(U, &U.d_perm, N));
    TRY(dalloc(U, &U.d_sec_start, S + 1));
    TRY(dalloc(U, &U.d_sector, Npad));
    TRY(dalloc(U, &U.d_qseg, U.nq + 1));
    TRY(dalloc(U, &U.d_sseg, S + 1));
    TRY(dalloc(U, &U.d_B64, (size_t)Npad * K));
    TRY(dalloc(U, &U.d_f64, K));
    TRY(dalloc(U, &U.d_d64, Npad));
    TRY(dalloc(U, &U.d_mu64, Npad));
    TRY(dalloc(U, &U.d_Bn1, Npad));
    TRY(dalloc(U, &U.d_Bn1f, Npad));
    TRY(dalloc(U, &U.d_B32, (size_t)Npad * K));
    TRY(dalloc(U, &U.d_B32p, (size_t)Npad * KMAX));
    TRY(dalloc(U, &U.d_f32, K));
    TRY(dalloc(U, &U.d_d32, Npad));
    TRY(dalloc(U, &U.d_mu32, Npad));
    TRY(dalloc(U, &U.d_B16, (size_t)Npad * K));
    TRY(dalloc(U, &U.d_Bt16, (size_t)K * Npad));
    TRY(dalloc(U, &U.d_B16p, (size_t)Npad * KMAX));
    TRY(dalloc(U, &U.d_Bt16p, (size_t)KMAX * Npad));
    TRY(dalloc(U, &U.d_Cinv32, (size_t)NRHO * K * K));
    TRY(dalloc(U, &U.d_Cinv16, (size_t)NRHO * K * K));
    TRY(dalloc(U, &U.d_G32, (size_t)NRHO * K * K));
    TRY(dalloc(U, &U.d_G16, (size_t)NRHO * K * K));
    TRY(dalloc(U, &U.d_CinvF32, (size_t)NRHO * K * K));
    TRY(dalloc(U, &U.d_CinvF16, (size_t)NRHO * K * K));
    auto H2D = [&](void* dst, const void* src, size_t n) {
        return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
    };
    if (H2D(U.d_inv_perm, U.inv_perm.data(), N * sizeof(int)) ||
        H2D(U.d_perm, U.perm.data(), N * sizeof(int)) ||
        H2D(U.d_sec_start, U.sec_start.data(), (S + 1) * sizeof(int)) ||
        H2D(U.d_sector, secs.data(), Npad * sizeof(int)) ||
        H2D(U.d_qseg, qseg.data(), (U.nq + 1) * sizeof(int)) ||
        H2D(U.d_sseg, sseg.data(), (S + 1) * sizeof(int)) ||
        H2D(U.d_B64, Bs.data(), Bs.size() * sizeof(double)) ||
        H2D(U.d_f64, f.data(), K * sizeof(double)) ||
        H2D(U.d_d64, ds.data(), Npad * sizeof(double)) ||
        H2D(U.d_mu64, mus.data(), Npad * sizeof(double)) ||
        H2D(U.d_Bn1, bn1.data(), Npad * sizeof(double)) ||
        H2D(U.d_Bn1f, bn1f.data(), Npad * sizeof(float)) ||
        H2D(U.d_f32, f32.data(), K * sizeof(float)) ||
        H2D(U.d_d32, d32.data(), Npad * sizeof(float)) ||
        H2D(U.d_mu32, mu32.data(), Npad * sizeof(float))) {
        set_error("universe upload failed");
        free_universe(U);
        return PRISM_ERR_CUDA;
    }
    {
        size_t n = (size_t)Npad * K;
        cudaMemsetAsync(U.d_B32p, 0, (size_t)Npad * KMAX * 4, U.stream);
        cudaMemsetAsync(U.d_B16p, 0, (size_t)Npad * KMAX * 2, U.stream);
        cudaMemsetAsync(U.d_Bt16p, 0, (size_t)KMAX * Npad * 2, U.stream);
        k_convert_B<<<(unsigned)cdiv64(n, 256), 256, 0, U.stream>>>(U.d_B64, Npad, K, U.d_B32, U.d_B32p, U.d_B16, U.d_Bt16,
                                                                      U.d_B16p, U.d_Bt16p);
        double* G = nullptr;
        if (cudaMalloc(&G, (size_t)NRHO * K * K * sizeof(double)) != cudaSuccess) {
            set_error("cudaMalloc (Gram scratch) failed");
            free_universe(U);
            return PRISM_ERR_ALLOCATION;
        }
        dim3 grid(NRHO, cdiv(K, 8));
        k_gram<float><<<grid, 256, 0, U.stream>>>(U.d_B32, U.d_d32, N, K, G);
        k_cinv<<<NRHO, 64, 0, U.stream>>>(G, U.d_f64, K, U.d_Cinv32, 0, U.d_G32);
        k_cinv<<<NRHO, 64, 0, U.stream>>>(G, U.d_f64, K, U.d_CinvF32, 1, nullptr);
        k_gram<__nv_bfloat16><<<grid, 256, 0, U.stream>>>(U.d_B16, U.d_d32, N, K, G);
        k_cinv<<<NRHO, 64, 0, U.stream>>>(G, U.d_f64, K, U.d_Cinv16, 0, U.d_G16);
        k_cinv<<<NRHO, 64, 0, U.stream>>>(G, U.d_f64, K, U.d_CinvF16, 1, nullptr);
        cudaError_t e = cudaStreamSynchronize(U.stream);
        cudaFree(G);
        if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            set_error(std::string("universe setup kernels failed: ") + cudaGetErrorString(e));
            free_universe(U);
            return PRISM_ERR_CUDA;
        }
    }
    return PRISM_OK;
}

}  // namespace prism

extern "C" int prism_create_universe(const prism_universe_desc* desc, prism_universe** out) {
    if (!out) { prism::set_error("out is NULL"); return PRISM_ERR_ARGUMENT; }
    *out = nullptr;
    prism_universe* h = new (std::nothrow) prism_universe();
    if (!h) { prism::set_error("host allocation failed"); return PRISM_ERR_ALLOCATION; }
    int rc = prism::create(desc, h->u);
    if (rc != PRISM_OK) { delete h; return rc; }
    *out = h;
    prism::set_error("");
    return PRISM_OK;
}

extern "C" void prism_destroy_universe(prism_universe* u) {
    if (!u) return;
    cudaSetDevice(u->u.device);
    prism::free_universe(u->u);
    delete u;
}

extern "C" const char* prism_last_error(void) { return prism::last_error(); }
extern "C" const char* prism_version(void) { return "prism-gb300 0.1 (sm_103a)"; }
