// diag.cu -- prism_shared_b_products: the x-update's two shared-B products on the
// solver's own kernels, for kernel-level checks and profiling.
//
//   P  = X B    (M x K)   the reduction over assets (G2)
//   BQ = Q B'   (M x N)   the broadcast back over assets (G4)
//
// Inputs are in universe asset order; the call permutes them into the solver's
// sector-sorted layout, runs exactly the kernels a solve of the given precision
// runs (SIMT FP32, or tcgen05 BF16 with the hi+lo operand split), and permutes
// the results back. It allocates its own temporaries (this is not a hot path).
#include <cstring>
#include <vector>

#include "common.cuh"
#include "solver.h"

namespace prism {

__global__ void k_diag_in(int M, int N, int Npad, const double* X, const double* Q, int K, const int* inv_perm,
                          float* Xs, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, float* Qf, __nv_bfloat16* Qhi,
                          __nv_bfloat16* Qlo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)M * N) {
        const int m = int(e / N), i = int(e % N);
        const float x = float(X[e]);
        const size_t d = (size_t)m * Npad + inv_perm[i];
        Xs[d] = x;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        Xhi[d] = h;
        Xlo[d] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
    if (e < (int64_t)M * K) {
        const int m = int(e / K), k = int(e % K);
        const float q = float(Q[e]);
        Qf[e] = q;
        const __nv_bfloat16 h = __float2bfloat16_rn(q);
        Qhi[(size_t)m * KMAX + k] = h;
        Qlo[(size_t)m * KMAX + k] = __float2bfloat16_rn(q - __bfloat162float(h));
    }
}

}  // namespace prism

extern "C" int prism_shared_b_products(prism_universe* uh, int32_t M, const double* X, const double* Q,
                                       int32_t precision, double* P, double* BQ) {
    using namespace prism;
    if (!uh || M < 1 || !X || !Q || !P || !BQ) { set_error("bad argument"); return PRISM_ERR_ARGUMENT; }
    const bool fused = (precision & PRISM_PRODUCTS_FUSED) != 0;
    precision &= ~PRISM_PRODUCTS_FUSED;
    if (precision != PRISM_BATCHED_FP32 && precision != PRISM_BATCHED_BF16 && precision != PRISM_PLAIN_FP32) {
        set_error("unknown precision"); return PRISM_ERR_ARGUMENT;
    }
    if (fused && precision != PRISM_BATCHED_BF16) {
        set_error("PRISM_PRODUCTS_FUSED needs PRISM_BATCHED_BF16"); return PRISM_ERR_ARGUMENT;
    }
    const bool bf16 = precision == PRISM_BATCHED_BF16;
    if (bf16 && !tc_available()) { set_error("tensor-core kernels unavailable"); return PRISM_ERR_UNSUPPORTED; }
    Universe& U = uh->u;
    PRISM_CUDA_TRY(cudaSetDevice(U.device));
    const int N = U.N, Npad = U.Npad, K = U.K;
    int chunk = 0;
    const int nsplit = bf16 ? tc_nsplit(M, N, &chunk) : choose_nsplit(M, N);
    const size_t MN = (size_t)M * Npad;
    std::vector<void*> allocs;
    auto take = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, bytes);
        allocs.push_back(p);
        return p;
    };
    auto cleanup = [&]() { for (void* p : allocs) cudaFree(p); };
    double* dX = (double*)take((size_t)M * N * 8);
    double* dQ = (double*)take((size_t)M * K * 8);
    Dev D;
    std::memset((void*)&D, 0, sizeof(Dev));
    D.M = M; D.N = N; D.Npad = Npad; D.K = K; D.S = U.S;
    D.B32 = U.d_B32; D.d32 = U.d_d32; D.mu32 = U.d_mu32; D.sec_start = U.d_sec_start; D.sector = U.d_sector;
    D.B16 = U.d_B16; D.Bt16 = U.d_Bt16; D.B16p = U.d_B16p; D.Bt16p = U.d_Bt16p;
    D.X = (float*)take(MN * 4);
    D.Xhi = (__nv_bfloat16*)take(MN * 2);
    D.Xlo = (__nv_bfloat16*)take(MN * 2);
    D.v = (float*)take(MN * 4);
    D.z = (float*)take(MN * 4);
    D.y = (float*)take(MN * 4);
    D.Ppart = (float*)take((size_t)nsplit * M * KMAX * 4);
    D.Q = (float*)take((size_t)M * K * 4);
    D.Qhi = (__nv_bfloat16*)take((size_t)M * KMAX * 2);
    D.Qlo = (__nv_bfloat16*)take((size_t)M * KMAX * 2);
    D.rho_idx = (int*)take((size_t)M * 4);
    D.n_active = (int*)take(8);
    D.err = D.n_active + 1;
    D.nsplit = nsplit;
    D.pstride = bf16 ? KMAX : K;
    D.bf16 = bf16;
    D.raw_out = 1;
    D.alpha = 1.f;
    size_t n_alloc = 14;
    if (fused) {
        // the fused x-update's own B'X (its second product over the X tile, summed over the
        // cluster's asset tiles): every account active, uniform l and c, the given X as the tile
        D.active = (int*)take((size_t)M * 4);
        D.iters = (int*)take((size_t)M * 4);
        D.nu = (float*)take((size_t)M * 4);
        D.dnu = (float*)take((size_t)M * 4);
        D.lo_u = (float*)take((size_t)M * 4);
        D.c_u = (float*)take((size_t)M * 4);
        D.xp_sets = xp_sets_for(N);
        D.Pxp = (float*)take((size_t)D.xp_sets * M * KMAX * 4);
        D.nt = cdiv(N, 128);
        D.nq = 0;
        D.uniform = 1;
        D.fold = 1;
        D.adapt_every = 1 << 30;
        D.w0 = D.z;
        D.up = D.y;
        n_alloc += 7;
    }
    for (void* p : allocs) if (!p) { cleanup(); set_error("allocation failed"); return PRISM_ERR_ALLOCATION; }
    if (allocs.size() != n_alloc) { cleanup(); set_error("allocation failed"); return PRISM_ERR_ALLOCATION; }
    if (fused) {
        std::vector<int> one(M, 1);
        cudaMemcpy((void*)D.active, one.data(), (size_t)M * 4, cudaMemcpyHostToDevice);
    }
    cudaMemcpy(dX, X, (size_t)M * N * 8, cudaMemcpyDefault);
    cudaMemcpy(dQ, Q, (size_t)M * K * 8, cudaMemcpyDefault);
    const int64_t work = std::max((int64_t)M * N, (int64_t)M * K);
    k_diag_in<<<(unsigned)cdiv64(work, 256), 256>>>(M, N, Npad, dX, dQ, K, U.d_inv_perm, D.X, D.Xhi, D.Xlo, D.Q,
                                                      D.Qhi, D.Qlo);
    if (fused) { launch_tc_xprox(D, 0); launch_tc_gemm_x(D, 0); }
    else if (bf16) { launch_tc_gemm_P(D, 0); launch_tc_gemm_x(D, 0); }
    else { launch_gemm_P(D, 0); launch_gemm_x(D, 0); }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { cleanup(); set_error(std::string("products failed: ") + cudaGetErrorString(e)); return PRISM_ERR_CUDA; }
    int err = 0;
    cudaMemcpy(&err, D.err, 4, cudaMemcpyDeviceToHost);
    if (err) { cleanup(); set_error("tensor-core pipeline wait timed out"); return PRISM_ERR_CUDA; }
    const int nsets = fused ? D.xp_sets : nsplit;
    std::vector<float> part((size_t)nsets * M * D.pstride), v(MN);
    cudaMemcpy(part.data(), fused ? D.Pxp : D.Ppart, part.size() * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(v.data(), D.v, MN * 4, cudaMemcpyDeviceToHost);
    std::vector<double> hP((size_t)M * K, 0.0), hBQ((size_t)M * N);
    for (int sp = 0; sp < nsets; ++sp)
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < K; ++k)
                hP[(size_t)m * K + k] += part[((size_t)sp * M + m) * D.pstride + k];
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < N; ++i) hBQ[(size_t)m * N + i] = v[(size_t)m * Npad + U.inv_perm[i]];
    cudaMemcpy(P, hP.data(), hP.size() * 8, cudaMemcpyDefault);
    cudaMemcpy(BQ, hBQ.data(), hBQ.size() * 8, cudaMemcpyDefault);
    cleanup();
    return PRISM_OK;
}
