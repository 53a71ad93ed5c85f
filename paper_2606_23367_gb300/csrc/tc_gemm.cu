// tc_gemm.cu -- the two shared-B products of the ADMM x-update on tcgen05 tensor cores.
//
//   G2:  P[m][k]  = sum_i X[m][i] B[i][k]          (B' X, contraction over assets)
//   G4:  BQ[i][m] = sum_k B[i][k] Q[m][k]          (B Q, contraction over factors)
//        + fused epilogue v = alpha x + (1 - alpha) z + y / rho,
//          x = (mu + rho z - y - BQ) / (2 d + rho)
//
// Both run BF16 operands with FP32 accumulation in tensor memory (kind::f16,
// cta_group::1). B is held in BF16 (the capacitance inverses of the BF16 mode
// are built from the same rounded B, so the x-update stays an exact solve of a
// consistent operator); the iterate-side operands are split into two BF16 terms
// (X = Xhi + Xlo, Q = Qhi + Qlo, 16 significant bits) and both are fed to the
// MMA, so the products keep near-FP32 accuracy while reading 4 bytes per X entry.
//
// Operands are staged by TMA (cp.async.bulk.tensor.2d) into 128-byte-swizzled
// shared memory, consumed by one elected thread issuing tcgen05.mma, and the
// accumulator is read back with tcgen05.ld (warp w reads TMEM lanes 32w..32w+31).
// Every mbarrier wait is bounded by a %globaltimer limit; on expiry the kernel
// records an error flag, skips the remaining work, releases its tensor memory
// and returns, and the host reports the failure.
#include <cuda.h>

#include "common.cuh"
#include "solver.h"

namespace prism {
namespace tc {

constexpr int TM = 128;            // MMA M (accounts in G2, assets in G4)
constexpr int TK = 64;             // BF16 elements per 128-byte swizzled row
constexpr int KP = 64;             // factors, zero-padded, in the BF16 copies of B and Q
#ifndef PRISM_G2_STAGES
#define PRISM_G2_STAGES 2
#endif
constexpr int G2_STAGES = PRISM_G2_STAGES;   // TMA stages of G2 (each 40 KB of shared memory)
constexpr int G2_CL = 8;           // CTAs per cluster along the asset splits (reduced over DSMEM)
constexpr int G2_PR = KP + 4;      // row stride (floats) of a CTA's partial in shared memory
constexpr uint32_t G2_A_BYTES = TM * TK * 2;      // 16 KB
constexpr uint32_t G2_B_BYTES = KP * TK * 2;      // 8 KB
constexpr int G4_TN = 128;                        // MMA N in G4 (accounts per tile)
constexpr uint32_t G4_TILE_BYTES = 128 * KP * 2;  // 16 KB
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull; // 1 s

// instruction descriptor, kind::f16: D = F32 (bit 4), A = B = BF16 (bits 7, 10),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete, for at most `limit` ns (WAIT_LIMIT_NS).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code,
                                          uint64_t limit = WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > limit) {
            atomicOr(err, code);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: 128-byte swizzle, 8-row groups 1024 B apart. K-major operands
// (rows of 64 BF16 along K) leave the leading byte offset unused. An MN-major operand whose MN
// extent is one 128-byte row (64 BF16) has a single swizzle atom along MN, so its leading offset
// (the stride between MN atoms) is never applied either, and its 8-row groups run along K; the
// offset is set to the 1024-byte group stride all the same.
__device__ __forceinline__ uint64_t sw128_desc(const void* smem, uint32_t lbo = 16) {
    const uint32_t a = smem_u32(smem);
    uint64_t d = 0;
    d |= uint64_t((a & 0x3FFFF) >> 4);       // start address (16-byte units)
    d |= uint64_t(lbo >> 4) << 16;           // leading byte offset
    d |= uint64_t(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
    d |= uint64_t(1) << 46;                  // descriptor version for tcgen05
    d |= uint64_t(2) << 61;                  // swizzle: 128 B
    return d;
}

// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// every thread of every CTA of the cluster; orders this CTA's shared-memory writes before
// the other CTAs' reads after the barrier
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16 bytes of CTA `rank`'s shared memory at the address this CTA uses for the same object
__device__ __forceinline__ float4 ld_dsmem_f4(uint32_t local_addr, uint32_t rank) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(local_addr), "r"(rank));
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(ra)
                 : "memory");
    return v;
}

__device__ __forceinline__ float rho_of_idx(int j) {
    return float(RHO_MIN) * exp10f(float(j) / float(RHO_PER_DECADE));
}

// ---------------------------------------------------------------------------
// G2: P[m][k] = sum_i (Xhi + Xlo)[m][i] B[i][k], split over assets.
// grid (account tiles, splits), clusters of G2_CL consecutive splits; 128 threads;
// thread 0 drives TMA and the MMAs. Each CTA stages its 128 x 64 FP32 partial in
// shared memory; CTA rank r of the cluster then sums rows 16r..16r+15 over the
// cluster's CTAs (fixed order, over DSMEM) and writes them as one partial set:
// Ppart[set][m][0..63], set = split / G2_CL.
// ---------------------------------------------------------------------------
struct __align__(1024) G2Smem {
    __nv_bfloat16 ahi[G2_STAGES][TM * TK];
    __nv_bfloat16 alo[G2_STAGES][TM * TK];
    __nv_bfloat16 b[G2_STAGES][KP * TK];
    uint64_t full[G2_STAGES];
    uint64_t empty[G2_STAGES];
    uint64_t done;
    uint32_t tmem;
    int fail;
};

__global__ void __launch_bounds__(128) k_tc_gemm_P(const __grid_constant__ CUtensorMap mXhi,
                                                    const __grid_constant__ CUtensorMap mXlo,
                                                    const __grid_constant__ CUtensorMap mBt, Dev D, int chunk) {
    extern __shared__ unsigned char raw[];
    G2Smem& s = *reinterpret_cast<G2Smem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, split = blockIdx.y;
    const int m_end = D.m1 ? D.m1 : D.M;
    const int mrow = D.m0 + mt * TM;                    // first account of this tile
    const int i0 = split * chunk, i1 = min(D.N, i0 + chunk);
    const int nk = (i1 > i0) ? (i1 - i0 + TK - 1) / TK : 0;
    constexpr uint32_t IDESC = idesc_bf16(TM, KP);
    pdl_wait();                            // X and the activity flags of the iteration before
    pdl_trigger();
    {
        // a tile whose accounts have all stopped iterating, or whose P all came from the fused
        // iteration, has nothing to compute
        const int m = mrow + tid;
        const int act = (D.active == nullptr) ||
                        (m < m_end && D.active[m] && (D.needP == nullptr || D.needP[m] != 0));
        if (!__syncthreads_or(act)) return;
    }
    if (warp == 0) tmem_alloc(&s.tmem, 64);
    if (tid == 0) {
        for (int q = 0; q < G2_STAGES; ++q) {
            mbar_init(&s.full[q], 1);
            mbar_init(&s.empty[q], 1);
        }
        mbar_init(&s.done, 1);
        s.fail = 0;
        fence_barrier_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s.tmem;
    if (tid == 0 && nk > 0) {
        auto load = [&](int kt) {
            const int q = kt % G2_STAGES;
            mbar_expect_tx(&s.full[q], 2 * G2_A_BYTES + G2_B_BYTES);
            tma_load_2d(s.ahi[q], &mXhi, &s.full[q], i0 + kt * TK, mrow);
            tma_load_2d(s.alo[q], &mXlo, &s.full[q], i0 + kt * TK, mrow);
            tma_load_2d(s.b[q], &mBt, &s.full[q], i0 + kt * TK, 0);
        };
        int issued = 0;
        // D.stall_ns (set only by the failure-path test): no load is issued, so the first wait
        // is on a barrier that nothing completes and runs out after stall_ns
        if (!D.stall_ns)
            for (; issued < G2_STAGES && issued < nk; ++issued) load(issued);
        bool ok = true;
        int consumed = 0;
        for (int kt = 0; kt < nk && ok; ++kt) {
            const int q = kt % G2_STAGES;
            const uint32_t par = (kt / G2_STAGES) & 1;
            if (!mbar_wait(&s.full[q], par, D.err, 1, D.stall_ns ? D.stall_ns : WAIT_LIMIT_NS)) { ok = false; break; }
            consumed = kt + 1;
            fence_after_sync();
            const uint64_t dhi = sw128_desc(s.ahi[q]), dlo = sw128_desc(s.alo[q]), db = sw128_desc(s.b[q]);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                // +32 bytes per 16-element K step inside the 128-byte swizzled row
                umma_bf16(tmem, dhi + 2 * kk, db + 2 * kk, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
                umma_bf16(tmem, dlo + 2 * kk, db + 2 * kk, IDESC, 1u);
            }
            umma_commit(&s.empty[q]);
            if (kt + G2_STAGES < nk) {
                if (!mbar_wait(&s.empty[q], par, D.err, 2)) { ok = false; break; }
                load(kt + G2_STAGES);
                ++issued;
            }
        }
        if (ok) {
            umma_commit(&s.done);
        } else {
            s.fail = 1;
            // drain the loads still in flight before the shared memory goes away
            for (int kt = consumed; kt < issued; ++kt)
                mbar_wait(&s.full[kt % G2_STAGES], (kt / G2_STAGES) & 1, D.err, 4);
        }
    }
    __syncthreads();
    bool have = (nk > 0) && !s.fail;
    if (have && !mbar_wait(&s.done, 0, D.err, 8)) have = false;
    have = __syncthreads_and(have);        // tcgen05.ld below is warp-collective: decide uniformly
    fence_after_sync();
    const uint32_t lane_addr = tmem + (uint32_t(warp * 32) << 16);
    // the stage buffers are free once the MMAs are done (or the loads drained on failure)
    float* part = reinterpret_cast<float*>(&s.ahi[0][0]);
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int c = 0; c < KP / 16; ++c) {
        float acc[16];
        if (have) tmem_ld16(lane_addr + c * 16, acc);
        else
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.f;
        float4* dst = reinterpret_cast<float4*>(part + row * G2_PR + c * 16);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
    }
    fence_before_sync();
    cluster_sync_all();
    {
        constexpr int ROWS = TM / G2_CL;           // rows this CTA reduces
        const uint32_t rank = cluster_ctarank();
        const int set = blockIdx.y / G2_CL;
        const uint32_t base_addr = smem_u32(part);
        for (int item = tid; item < ROWS * (KP / 4); item += blockDim.x) {
            const int r = int(rank) * ROWS + item / (KP / 4), c4 = item % (KP / 4);
            const uint32_t off = base_addr + uint32_t(r * G2_PR + c4 * 4) * 4u;
            float4 sum = ld_dsmem_f4(off, 0);
#pragma unroll
            for (int q = 1; q < G2_CL; ++q) {
                const float4 v = ld_dsmem_f4(off, uint32_t(q));
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            const int m = mrow + r;
            if (m < m_end) *reinterpret_cast<float4*>(D.Ppart + ((size_t)set * D.M + m) * KP + c4 * 4) = sum;
        }
    }
    cluster_sync_all();                          // no CTA leaves while another reads its partial
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------
// G4: one 128-asset x 128-account tile per block. TMEM lane = asset row, column =
// account, so the epilogue reads z, y and writes v coalesced along assets.
// ---------------------------------------------------------------------------
struct __align__(1024) G4Smem {
    __nv_bfloat16 a[TM * KP];        // B tile: 128 assets x 64 factors
    __nv_bfloat16 bhi[G4_TN * KP];   // Qhi tile: 128 accounts x 64 factors
    __nv_bfloat16 blo[G4_TN * KP];
    uint64_t full;
    uint64_t done;
    uint32_t tmem;
    int fail;
    float rho[G4_TN];
    float irho[G4_TN];
};

// 32 lanes x 8 consecutive FP32 columns of this warp's TMEM lane quarter
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

constexpr int G4_THREADS = 256;   // warp w: TMEM lane quarter w % 4 (32 assets), accounts 64 (w / 4) .. + 63
constexpr int G4_CC = 8;          // accounts per epilogue chunk

// z and y of one chunk of G4_CC accounts for this thread's asset (coalesced over the warp)
__device__ __forceinline__ void g4_load_chunk(const Dev& D, int i, int m0, float* zz, float* yy) {
#pragma unroll
    for (int j = 0; j < G4_CC; ++j) {
        const int m = m0 + j;
        const size_t e = (size_t)m * D.Npad + i;
        const bool ok = m < D.M;
        zz[j] = ok ? __ldg(D.z + e) : 0.f;
        yy[j] = ok ? __ldg(D.y + e) : 0.f;
    }
}

__global__ void __launch_bounds__(G4_THREADS, 3) k_tc_gemm_x(const __grid_constant__ CUtensorMap mB,
                                                            const __grid_constant__ CUtensorMap mQhi,
                                                            const __grid_constant__ CUtensorMap mQlo, Dev D) {
    extern __shared__ unsigned char raw[];
    G4Smem& s = *reinterpret_cast<G4Smem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int at = blockIdx.x, mt = blockIdx.y;
    constexpr uint32_t IDESC = idesc_bf16(TM, G4_TN);
    {
        const int m = mt * G4_TN + tid;
        const int act = tid < G4_TN && ((D.active == nullptr) || (m < D.M && D.active[m]));
        if (!__syncthreads_or(act)) return;
    }
    if (warp == 0) tmem_alloc(&s.tmem, G4_TN);
    if (tid == 0) {
        mbar_init(&s.full, 1);
        mbar_init(&s.done, 1);
        s.fail = 0;
        fence_barrier_init();
    }
    if (tid < G4_TN) {
        const int m = mt * G4_TN + tid;
        const float r = (m < D.M) ? rho_of_idx(D.rho_idx[m]) : 1.f;
        s.rho[tid] = r;
        s.irho[tid] = 1.f / r;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s.tmem;
    if (tid == 0) {
        mbar_expect_tx(&s.full, 3 * G4_TILE_BYTES);
        tma_load_2d(s.a, &mB, &s.full, 0, at * TM);
        tma_load_2d(s.bhi, &mQhi, &s.full, 0, mt * G4_TN);
        tma_load_2d(s.blo, &mQlo, &s.full, 0, mt * G4_TN);
    }
    // while the tile loads and multiplies: this thread's first two chunks of z and y
    const int q = warp & 3, half = warp >> 2;
    const int i = at * TM + q * 32 + lane;              // asset of this TMEM lane
    const int ii = i < D.N ? i : 0;
    const int col0 = half * (G4_TN / 2);                // first account column of this warp
    const int m_base = mt * G4_TN + col0;
    float za[G4_CC], ya[G4_CC], zb[G4_CC], yb[G4_CC];
    g4_load_chunk(D, ii, m_base, za, ya);
    g4_load_chunk(D, ii, m_base + G4_CC, zb, yb);
    const float mu = D.mu32[ii], dd = 2.f * D.d32[ii];
    if (tid == 0) {
        if (mbar_wait(&s.full, 0, D.err, 16)) {
            fence_after_sync();
            const uint64_t da = sw128_desc(s.a), dh = sw128_desc(s.bhi), dl = sw128_desc(s.blo);
#pragma unroll
            for (int kk = 0; kk < KP / 16; ++kk) {
                umma_bf16(tmem, da + 2 * kk, dh + 2 * kk, IDESC, kk > 0 ? 1u : 0u);
                umma_bf16(tmem, da + 2 * kk, dl + 2 * kk, IDESC, 1u);
            }
            umma_commit(&s.done);
        } else {
            s.fail = 1;
        }
    }
    __syncthreads();
    bool have = !s.fail && mbar_wait(&s.done, 0, D.err, 32);
    have = __syncthreads_and(have);
    fence_after_sync();
    const bool row_ok = have && i < D.N;
    const uint32_t lane_addr = tmem + (uint32_t(q * 32) << 16) + col0;
    // chunk c uses the buffer loaded two chunks earlier; the chunk after next is loaded
    // into it once it is consumed
    auto consume = [&](int c, float* zz, float* yy) {
        float bq[G4_CC];
        if (have) tmem_ld8(lane_addr + c * G4_CC, bq);
        const int m0 = m_base + c * G4_CC;
        if (row_ok) {
#pragma unroll
            for (int j = 0; j < G4_CC; ++j) {
                const int m = m0 + j;
                if (m >= D.M) break;
                const size_t e = (size_t)m * D.Npad + i;
                if (D.raw_out) { D.v[e] = bq[j]; continue; }
                const int col = col0 + c * G4_CC + j;
                const float rho = s.rho[col];
                const float x = (mu + rho * zz[j] - yy[j] - bq[j]) / (dd + rho);
                D.v[e] = D.alpha * x + (1.f - D.alpha) * zz[j] + yy[j] * s.irho[col];
            }
        }
        if (c + 2 < (G4_TN / 2) / G4_CC) g4_load_chunk(D, ii, m0 + 2 * G4_CC, zz, yy);
    };
#pragma unroll
    for (int c = 0; c < (G4_TN / 2) / G4_CC; c += 2) {
        consume(c, za, ya);
        consume(c + 1, zb, yb);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, G4_TN);
}

// ---------------------------------------------------------------------------
// G4 fused with the streaming pass of G5 (books with the L1 cost only, no cap).
// Tiles of 128 assets x 32 accounts (TMEM lane = asset, column = account), so that about six
// small CTAs share each SM and the loads of many of them are in flight together. For
// each entry the epilogue forms v, writes it, and evaluates the prox at L = nu_prev - margin:
//   z_i(L) = clip(soft(v_i - L/rho - w0_i, c_i/rho) + w0_i, l_i, u_i).
// z_i(eta) is nonincreasing in eta, so an entry with z_i(L) = l_i keeps z = l_i at every
// eta >= L: its z, y = rho (v - l) and X are final and written here. Per account and
// 32-position quarter the warp leaves the mask of the other entries (the candidates that
// k_prox_roots gathers) and the residual maxima of the pinned entries (combined over the
// tile's quarters); when l differs over the account, also the sum of l over the pinned
// entries of each sector segment.
// ---------------------------------------------------------------------------
constexpr int XP_TN = 16;         // accounts per tile (MMA N): small tiles, four CTAs per SM
#ifndef PRISM_XP_WARPS
#define PRISM_XP_WARPS 8
#endif
// warp w reads TMEM lane quarter w % 4 (32 assets) for the accounts of its half (w / 4) of the
// tile's columns: with eight warps each entry of a quarter has two warps over its accounts,
// so that more warps hide the epilogue's latencies
constexpr int XP_THREADS = 32 * PRISM_XP_WARPS;
constexpr int XP_SPLIT = XP_THREADS / 128;        // warps per lane quarter
constexpr int XP_JN = XP_TN / XP_SPLIT;           // accounts per warp
static_assert(XP_SPLIT == 1 || XP_SPLIT == 2, "four or eight warps");
constexpr uint32_t XP_Q_BYTES = XP_TN * KP * 2;

struct __align__(1024) XPSmem {
    __nv_bfloat16 a[TM * KP];         // B tile (operand A of both products); then the tile's P partial
    __nv_bfloat16 bhi[XP_TN * KP];    // Q split (operand B)
    __nv_bfloat16 blo[XP_TN * KP];
    float in[4][XP_TN][TM];           // z, y, w0, u of the tile: [array][account][asset]; then the X tile
    uint64_t full;                    // operands landed
    uint64_t full_in[XP_TN / 4];      // inputs of accounts 4g .. 4g + 3 landed
    uint64_t done;                    // MMA complete
    uint64_t done2;                   // the P product complete
    uint32_t tmem;
    int fail;
    float4 pa[XP_TN];                 // per account column: rho, 1/rho, L/rho, c/rho (NaN: c differs over positions)
    float4 pb[XP_TN];                 // l (NaN: differs), active, adaptation call, unused
    float r5[4][5][XP_TN];            // per lane quarter and account: residual maxima
    unsigned cm[4][XP_TN];            // per lane quarter and account: candidate masks
};

// 1/x to within 1 ulp (the hardware approximation; x > 0 and normal here)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// maximum over the warp of nonnegative floats (their bit patterns order as integers; a NaN
// with the sign bit clear orders above +inf, so it survives)
__device__ __forceinline__ float warp_max_nn(float v) {
    return __int_as_float(__reduce_max_sync(0xffffffffu, __float_as_int(v)));
}

struct XPMaps {
    CUtensorMap B, Qhi, Qlo, z, y, w0, up;   // inputs in boxes of 4 accounts
    CUtensorMap zr, yr, w0r, upr;            // the same arrays one account row at a time
    CUtensorMap mu, d;                       // mu and d of 128 positions (persistent form)
};

// The shared-memory views of one tile, for the per-tile epilogue of the fused x-update.
struct XPTileView {
    const float (*in)[XP_TN][TM];     // [4][XP_TN][TM]: z, y, w0, u
    const float4* pa;                 // [XP_TN]
    const float4* pb;                 // [XP_TN]
    uint64_t* full_in;                // [XP_TN / 4]: inputs of each group of four accounts
    uint32_t par;                     // parity of the phase of those barriers
    float (*r5)[5][XP_TN];            // [4][5][XP_TN]
    unsigned (*cm)[XP_TN];            // [4][XP_TN]
};

// A thread's asset of a tile: position, output offset, mu and 2 d, and the sector segments of
// its lane quarter (lanes with equal sectors are consecutive). Warp-collective.
struct XPAsset {
    int ia, i, obase, nsegq, segl, sbase;
    float mu, dd;
};

__device__ __forceinline__ XPAsset xp_asset(const Dev& D, int at, int q, int lane, int m_base) {
    XPAsset ax;
    ax.ia = q * 32 + lane;
    ax.i = at * TM + ax.ia;
    const int ii = ax.i < D.N ? ax.i : 0;
    ax.obase = m_base * D.Npad + ii;
    ax.mu = D.mu32[ii];
    ax.dd = 2.f * D.d32[ii];
    const int sec = ax.i < D.N ? D.sector[ax.i] : -1;
    const int prev = __shfl_up_sync(0xffffffffu, sec, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, ax.i < D.N && (lane == 0 || prev != sec));
    ax.nsegq = __popc(starts);
    ax.segl = __popc(starts & ((2u << lane) - 1u)) - 1;
    const int gq = at * 4 + q;
    ax.sbase = (gq < D.nq) ? D.qseg[gq] : 0;
    return ax;
}

// The per-entry arithmetic of the fused pass, written with explicitly rounded operations so that
// the compiler cannot fuse a product into a neighbouring add differently in the two forms of the
// fused x-update (which must give the same iterations bit for bit): the x-update
// x = (mu + rho z - y - (BQ)) / (2d + rho), the relaxation v = alpha x + (1 - alpha) z + y / rho,
// the prox at L, z = clip(soft(v - L/rho - w0, c/rho) + w0, l, u), and for an entry pinned at l its
// y = rho (v - l) and X = (mu + rho l - y) / (2d + rho).
struct XPEntry {
    float v, z, yn, X, yir;   // yir = y / rho (the adaptation's term v - y / rho)
};

__device__ __forceinline__ XPEntry xp_entry(float mu, float dd, float rho, float irho, float Lr, float k, float lo,
                                            float up, float z0, float y0, float w0, float bq, float alpha,
                                            float oma) {
    XPEntry e;
    const float inv = rcp_approx(__fadd_rn(dd, rho));
    const float x = __fmul_rn(__fsub_rn(__fsub_rn(__fmaf_rn(rho, z0, mu), y0), bq), inv);
    e.yir = __fmul_rn(y0, irho);
    e.v = __fmaf_rn(alpha, x, __fmaf_rn(oma, z0, e.yir));
    const float t = __fsub_rn(e.v, Lr);
    float z = (t > __fadd_rn(w0, k)) ? __fsub_rn(t, k) : ((t < __fsub_rn(w0, k)) ? __fadd_rn(t, k) : w0);
    e.z = fminf(fmaxf(z, lo), up);
    e.yn = __fmul_rn(rho, __fsub_rn(e.v, lo));
    e.X = __fmul_rn(__fsub_rn(__fmaf_rn(rho, lo, mu), e.yn), inv);
    return e;
}

// The epilogue of one tile for this warp's XP_JN accounts j0 .. j0 + XP_JN - 1: for each entry
// v, the prox at L, the final z, y, X of a pinned entry or the record of a candidate; per
// account and lane quarter the residual maxima and the candidate mask.
template <bool UNIFORM, bool FOLD>
__device__ __forceinline__ void xp_accounts(const Dev& D, const XPTileView& tv, const XPAsset& ax, const float* bq,
                                            int j0, int q, int lane, int m_base, bool have, uint32_t* xpk) {
    const bool row_ok = have && ax.i < D.N;
    const float alpha = D.alpha, oma = __fsub_rn(1.f, alpha);
    float4* crec = reinterpret_cast<float4*>(D.crec);
    // The accounts are processed without branches on the entry (an inactive account's values
    // are zero and nothing of it is stored), so their reductions interleave.
#pragma unroll
    for (int jj = 0; jj < XP_JN; ++jj) {
        const int j = j0 + jj;
        if (jj % 4 == 0) {
            // this group's inputs (an expired wait sets the error flag; the values are then
            // not used: the host fails the call)
            if (have) mbar_wait(&tv.full_in[j / 4], tv.par, D.err, 64);
        }
        const float4 pa = tv.pa[j], pb = tv.pb[j];
        const float rho = pa.x, irho = pa.y, Lr = pa.z;   // Lr = L / rho
        const bool ok = row_ok && pb.y != 0.f;
        const int off = ax.obase + j * D.Npad;
        if (FOLD && D.raw_out) {
            // diagnostic (uniform over the launch): the X tile is the given split X, nothing is stored
            xpk[jj] = ok ? (uint32_t(__bfloat16_as_ushort(D.Xhi[off])) |
                            (uint32_t(__bfloat16_as_ushort(D.Xlo[off])) << 16)) : 0u;
            continue;
        }
        float lo = pb.x, k = pa.w;                      // k = c / rho
        const bool lou = UNIFORM || !isnan(lo);         // warp-uniform
        if (!UNIFORM) {
            if (ok && !lou) lo = D.lo[off];
            if (ok && isnan(k)) k = __fmul_rn(D.c[off], irho);
        }
        const float z0 = tv.in[0][j][ax.ia], y0 = tv.in[1][j][ax.ia], w0 = tv.in[2][j][ax.ia], up = tv.in[3][j][ax.ia];
        const XPEntry en = xp_entry(ax.mu, ax.dd, rho, irho, Lr, k, lo, up, z0, y0, w0, bq[jj], alpha, oma);
        const float v = en.v, yn = en.yn;
        const bool pin = ok && (en.z == lo);
        const bool cand = ok && !pin;
        // the residual terms before their scale (1/rho, rho: applied to the warp's maxima, which
        // gives the same values); a non-finite update gives an infinite or NaN maximum
        const float e_rp = pin ? fabsf(__fsub_rn(yn, y0)) : 0.f;
        const float e_rd = pin ? fabsf(__fsub_rn(lo, z0)) : 0.f;
        // v of a pinned entry is not stored: it is l + y / rho from the y written below, which is
        // all a later recomputation of its sector needs; z is stored only when it changes. Its
        // X = Delta^{-1} (mu + rho l - y), split into two BF16 terms, is stored for the product
        // kernel, or with the products folded enters the tile's B'X partial through the X tile
        // (zero for every other entry)
        if (cand) D.v[off] = v;
        uint32_t xp = 0u;
        if (pin) {
            if (z0 != lo) D.z[off] = lo;
            D.y[off] = yn;
            const float X = en.X;
            const __nv_bfloat16 h = __float2bfloat16_rn(X);
            const __nv_bfloat16 l = __float2bfloat16_rn(__fsub_rn(X, __bfloat162float(h)));
            if constexpr (FOLD) {
                xp = uint32_t(__bfloat16_as_ushort(h)) | (uint32_t(__bfloat16_as_ushort(l)) << 16);
            } else {
                D.Xhi[off] = h;                     // for the separate product kernel
                D.Xlo[off] = l;
            }
        }
        if constexpr (FOLD) xpk[jj] = xp;
        if (cand) {
            // what the roots kernel needs of a candidate, in one 32-byte record: v, w0, u,
            // z, y, mu, d (l and c are read per entry there when they differ over the account)
            crec[2 * (size_t)off] = make_float4(v, w0, up, z0);
            crec[2 * (size_t)off + 1] = make_float4(y0, ax.mu, 0.5f * ax.dd, 0.f);
        }
        const unsigned cm = __ballot_sync(0xffffffffu, cand);
        float rp = warp_max_nn(e_rp), rd = __fmul_rn(warp_max_nn(e_rd), rho);
        rp = (rp == INFINITY) ? NAN : __fmul_rn(rp, irho);        // a non-finite pinned update: NaN (numerical failure)
        float nx = 0.f, nz = 0.f, ny = 0.f;
        if (pb.z != 0.f) {                              // penalty adaptation on this call (uniform)
            nx = warp_max_nn(pin ? fabsf(__fsub_rn(v, en.yir)) : 0.f);
            ny = warp_max_nn(pin ? fabsf(yn) : 0.f);
            if (!lou) nz = warp_max_nn(pin ? fabsf(lo) : 0.f);   // else |l| itself, added later
        }
        if (!UNIFORM && !lou) {
            // l differs over the account: the sums of l over the pinned entries, per segment
            for (int g = 0; g < ax.nsegq; ++g) {
                const bool mine = (ax.i < D.N) && ax.segl == g && pin;
                const float sg = warp_sum_f(mine ? lo : 0.f);
                if (lane == 0 && pb.y != 0.f) D.SOp[(size_t)(ax.sbase + g) * D.M + m_base + j] = sg;
            }
        }
        if (lane == 0) {
            tv.r5[q][0][j] = rp;
            tv.r5[q][1][j] = rd; tv.r5[q][2][j] = nx; tv.r5[q][3][j] = nz; tv.r5[q][4][j] = ny;
            tv.cm[q][j] = cm;
        }
    }
}

// Per-tile outputs: the residual maxima over the four quarters (NaN kept) and the masks, each
// row written coalesced over the tile's accounts. nthr threads, thread index t.
__device__ __forceinline__ void xp_tile_out(const Dev& D, const float (*r5)[5][XP_TN], const unsigned (*cm)[XP_TN],
                                            const float4* pb, int m_base, int m_end, int at, int t, int nthr) {
    for (int it = t; it < 5 * XP_TN; it += nthr) {
        const int kq = it / XP_TN, col = it % XP_TN, m = m_base + col;
        if (m >= m_end || pb[col].y == 0.f) continue;
        float r = 0.f;
        bool nan_ = false;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const float x = r5[qq][kq][col];
            nan_ |= isnan(x);
            r = fmaxf(r, x);
        }
        D.Rt[((size_t)m * 5 + kq) * D.nt + at] = nan_ ? NAN : r;
    }
    for (int it = t; it < 4 * XP_TN; it += nthr) {
        const int w = it / XP_TN, col = it % XP_TN, m = m_base + col;
        const int g = at * 4 + w;
        if (m >= m_end || pb[col].y == 0.f || g >= D.nq) continue;
        D.Cm[(size_t)m * D.nq + g] = cm[w][col];
    }
}

// The X tile of the B'X partial: [XP_TN accounts][128 positions] per BF16 term (4 KB), K-major
// with the 128-byte swizzle: two 64-position blocks of 2 KB, in each the 8-row groups 1024 B
// apart, and in each 128-byte row the 16-byte chunk (p % 64) / 8 stored at chunk XOR (row % 8).
constexpr uint32_t XT_BYTES = XP_TN * TM * 2;

static_assert(XP_TN == 16, "the P readback holds 16 accounts");
static_assert(2 * XT_BYTES <= sizeof(float) * 4 * XP_TN * TM, "the X tile fits in the inputs' buffer");

__device__ __forceinline__ uint32_t xtile_off(int j, int p) {
    const int c = p & 63;
    return uint32_t((p >> 6) * 2048 + (j >> 3) * 1024 + (j & 7) * 128 + (((c >> 3) ^ (j & 7)) << 4) + (c & 7) * 2);
}

// UNIFORM: every account has one l over its positions and one c over those with u > l (the
// values come from shared memory; no per-entry l, c and no segment sums of l).
//
// After the epilogue each CTA forms the B'X partial of its tile over the entries it pinned
// (the G2 product of those entries; the candidates' share is added per account by
// k_prox_roots): a second MMA, D2 (64 factors x XP_TN accounts) = B_tile' X_tile, reads the
// B tile already in shared memory as an MN-major operand (factors contiguous) and the X tile
// written by the epilogue, and the partial goes out as one set per asset tile,
// Pxp[tile][m][0..63] (k_prox_roots sums the sets in a fixed order).
template <bool UNIFORM, bool FOLD>
__global__ void __launch_bounds__(XP_THREADS, 4) k_tc_xprox(const __grid_constant__ XPMaps mp, Dev D) {
    extern __shared__ unsigned char raw[];
    XPSmem& s = *reinterpret_cast<XPSmem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int at = blockIdx.x;
    const int m_end = D.m1 ? D.m1 : D.M;
    const int m_base = D.m0 + blockIdx.y * XP_TN;       // first account of the tile
    constexpr uint32_t IDESC = idesc_bf16(TM, XP_TN);
    constexpr uint32_t IDESC_P = idesc_bf16(64, XP_TN) | (1u << 15);   // operand A transposed (MN-major)
    {
        const int m = m_base + tid;
        const int act = tid < XP_TN && (m < m_end && D.active[m]);
        if (!__syncthreads_or(act)) return;
    }
    {
        if (warp == 0) tmem_alloc(&s.tmem, 32);
        if (tid == 0) {
            mbar_init(&s.full, 1);
            for (int g = 0; g < XP_TN / 4; ++g) mbar_init(&s.full_in[g], 1);
            mbar_init(&s.done, 1);
            mbar_init(&s.done2, 1);
            s.fail = 0;
            fence_barrier_init();
        }
        if (tid < XP_TN) {
            const int m = m_base + tid;
            const bool ok = m < m_end;
            const float r = ok ? rho_of_idx(D.rho_idx[m]) : 1.f;
            const float L = ok ? D.nu[m] - fmaxf(4.f * D.dnu[m], 2e-3f) : 0.f;
            const float ir = 1.f / r;
            s.pa[tid] = make_float4(r, ir, L * ir, (ok ? D.c_u[m] : 0.f) * ir);
            const bool act = ok && D.active[m];
            const bool adapt = act && ((D.iters[m] + 1) % D.adapt_every == 0);
            s.pb[tid] = make_float4(ok ? D.lo_u[m] : 0.f, act ? 1.f : 0.f, adapt ? 1.f : 0.f, 0.f);
        }
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        const uint32_t tmem = s.tmem;
        if (tid == 0) {
            // B and the tile's inputs first (columns beyond Npad and rows beyond M arrive as
            // zeros): none of them comes from the small solve just before; Q after it. The inputs
            // come in four groups of four accounts, each with its own barrier, so that the epilogue
            // starts on the first group while the others are in flight. A group whose accounts all
            // iterate takes one box per array; otherwise one 128-position row per active account
            // and array, so that the traffic follows the accounts still iterating (the rows of
            // inactive accounts are left unread: their entries are skipped).
            mbar_expect_tx(&s.full, G4_TILE_BYTES + 2 * XP_Q_BYTES);
            tma_load_2d(s.a, &mp.B, &s.full, 0, at * TM);
            for (int g = 0; g < XP_TN / 4; ++g) {
                int nact = 0;
                for (int j = 4 * g; j < 4 * g + 4; ++j) nact += s.pb[j].y != 0.f;
                mbar_expect_tx(&s.full_in[g], (uint32_t)nact * 4u * (TM * 4u));
                if (nact == 4) {
                    tma_load_2d(s.in[0][4 * g], &mp.z, &s.full_in[g], at * TM, m_base + 4 * g);
                    tma_load_2d(s.in[1][4 * g], &mp.y, &s.full_in[g], at * TM, m_base + 4 * g);
                    tma_load_2d(s.in[2][4 * g], &mp.w0, &s.full_in[g], at * TM, m_base + 4 * g);
                    tma_load_2d(s.in[3][4 * g], &mp.up, &s.full_in[g], at * TM, m_base + 4 * g);
                } else {
                    for (int j = 4 * g; j < 4 * g + 4; ++j) {
                        if (s.pb[j].y == 0.f) continue;
                        const int m = m_base + j;
                        tma_load_2d(s.in[0][j], &mp.zr, &s.full_in[g], at * TM, m);
                        tma_load_2d(s.in[1][j], &mp.yr, &s.full_in[g], at * TM, m);
                        tma_load_2d(s.in[2][j], &mp.w0r, &s.full_in[g], at * TM, m);
                        tma_load_2d(s.in[3][j], &mp.upr, &s.full_in[g], at * TM, m);
                    }
                }
            }
        }
        pdl_wait();
        pdl_trigger();
        if (tid == 0) {
            tma_load_2d(s.bhi, &mp.Qhi, &s.full, 0, m_base);
            tma_load_2d(s.blo, &mp.Qlo, &s.full, 0, m_base);
        }
        const int q = warp & 3;                             // TMEM lane quarter
        const int j0 = (warp >> 2) * XP_JN;                 // first account (column) of this warp
        const XPAsset ax = xp_asset(D, at, q, lane, m_base);
        if (tid == 0) {
            if (mbar_wait(&s.full, 0, D.err, 16)) {
                fence_after_sync();
                const uint64_t da = sw128_desc(s.a), dh = sw128_desc(s.bhi), dl = sw128_desc(s.blo);
#pragma unroll
                for (int kk = 0; kk < KP / 16; ++kk) {
                    umma_bf16(tmem, da + 2 * kk, dh + 2 * kk, IDESC, kk > 0 ? 1u : 0u);
                    umma_bf16(tmem, da + 2 * kk, dl + 2 * kk, IDESC, 1u);
                }
                umma_commit(&s.done);
            } else {
                s.fail = 1;
            }
        }
        __syncthreads();
        bool have = !s.fail && mbar_wait(&s.done, 0, D.err, 32);
        have = __syncthreads_and(have);
        fence_after_sync();
        float bq[XP_JN];
        if (have) {
            if constexpr (XP_JN == 16) tmem_ld16(tmem + (uint32_t(q * 32) << 16), bq);
            else tmem_ld8(tmem + (uint32_t(q * 32) << 16) + uint32_t(j0), bq);
        }
        const XPTileView tv{s.in, s.pa, s.pb, s.full_in, 0u, s.r5, s.cm};
        uint32_t xpk[XP_JN];
        xp_accounts<UNIFORM, FOLD>(D, tv, ax, bq, j0, q, lane, m_base, have, xpk);
        fence_before_sync();
        __syncthreads();
        if constexpr (!FOLD) {
            if (warp == 0) tmem_dealloc(tmem, 32);
            if (have) xp_tile_out(D, s.r5, s.cm, s.pb, m_base, m_end, at, tid, XP_THREADS);
            return;
        }
        // the staged inputs are consumed: their buffer takes the X tile (hi term, then lo)
        uint8_t* xt = reinterpret_cast<uint8_t*>(&s.in[0][0][0]);
#pragma unroll
        for (int jj = 0; jj < XP_JN; ++jj) {
            const uint32_t o = xtile_off(j0 + jj, ax.ia);
            *reinterpret_cast<uint16_t*>(xt + o) = uint16_t(xpk[jj] & 0xffffu);
            *reinterpret_cast<uint16_t*>(xt + XT_BYTES + o) = uint16_t(xpk[jj] >> 16);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && have) {
            fence_after_sync();
            const uint64_t da = sw128_desc(s.a, 1024), dh = sw128_desc(xt), dl = sw128_desc(xt + XT_BYTES);
#pragma unroll
            for (int kk = 0; kk < TM / 16; ++kk) {
                // 16 positions per MMA: 16 rows of 128 B further in the B tile; +32 B in the X
                // tile's swizzled rows, and its next 64-position block 2 KB on
                const uint64_t oa = uint64_t(kk * 16 * 128) >> 4;
                const uint64_t ob = uint64_t((kk >> 2) * 2048 + (kk & 3) * 32) >> 4;
                umma_bf16(tmem + 16u, da + oa, dh + ob, IDESC_P, kk > 0 ? 1u : 0u);
                umma_bf16(tmem + 16u, da + oa, dl + ob, IDESC_P, 1u);
            }
            umma_commit(&s.done2);
        }
        __syncthreads();
        bool have2 = have && mbar_wait(&s.done2, 0, D.err, 128);
        have2 = __syncthreads_and(have2);
        fence_after_sync();
        // D2 with M = 64: factor 16 w + l in lane l < 16 of TMEM lane quarter w, accounts in columns;
        // the partial set of this tile, 16 consecutive factors per warp and account
        if (warp < 4) {
            float pv[16];
            if (have2) tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + 16u, pv);
            if (have2 && lane < 16)
#pragma unroll
                for (int j = 0; j < XP_TN; ++j) {
                    const int m = m_base + j;
                    if (m < m_end) D.Pxp[((size_t)at * D.M + m) * KP + warp * 16 + lane] = pv[j];
                }
        }
        fence_before_sync();
        __syncthreads();
        if (warp == 0) tmem_dealloc(tmem, 32);
        if (have && !D.raw_out) xp_tile_out(D, s.r5, s.cm, s.pb, m_base, m_end, at, tid, XP_THREADS);
    }
}

// ---------------------------------------------------------------------------
// The same fused x-update as a persistent, warp-specialised kernel over the accounts that still
// iterate. Two CTAs per SM (a share of that when several chains iterate side by side), each
// taking tiles of 128 positions x 16 accounts from its chain's tile counter until none is left.
// A tile's accounts are 16 consecutive ones of the chain's active accounts (the list is formed
// by each CTA at its start), so an account that has stopped iterating costs no work:
//   warp 8 (producer): claims a tile, writes its accounts and their constants into a stage of a
//     two-stage ring, loads the B tile, mu, d and the accounts' input rows by TMA (one box of four
//     rows where four accounts are consecutive), and the Q split rows (a box when all 16 accounts
//     are consecutive, else copied by the warp into the product's 128-byte-swizzled layout);
//   warp 9 (MMA): one thread issues the B Q product of each stage into that stage's 16 TMEM
//     columns once its operands are in place;
//   warps 0-7 (epilogue): for each entry the pass of k_tc_xprox (the same arithmetic), then the
//     tile's residual maxima and candidate masks; the stage goes back to the producer.
// Every mbarrier wait is bounded; after an expired wait each role leaves its loop, waits
// (bounded) for its own copies and products still in flight, and the CTA frees its tensor
// memory and returns (the error flag fails the call). The last CTA to finish claiming resets
// the counter for the next launch.
// Measured on the 500 x 10,000 book against this shape (two CTAs per SM, two stages, eight
// epilogue warps meeting at two named barriers per tile): sixteen epilogue warps per CTA, one
// CTA per SM with four stages, and epilogue warps that never wait for one another (the producer
// writing each tile's outputs) were all slower.
// ---------------------------------------------------------------------------
constexpr int XQ_STAGES = 2;
constexpr int XQ_EPI = 256;                       // epilogue threads (warps 0-7)
constexpr int XQ_THREADS = XQ_EPI + 64;           // + producer warp + MMA warp
constexpr int XQ_WMAX = 256;                      // 32-account words of the active list (8,192 accounts)
static_assert(XP_THREADS == XQ_EPI, "the epilogue assumes eight warps");

struct __align__(1024) XQStage {
    __nv_bfloat16 a[TM * KP];         // B tile (operand A)
    __nv_bfloat16 bhi[XP_TN * KP];    // Q split rows of the tile's accounts (operand B)
    __nv_bfloat16 blo[XP_TN * KP];
    float in[4][XP_TN][TM];           // z, y, w0, u: [array][account column][position]
    float md[2][TM];                  // mu, d of the tile's positions
};
static_assert(sizeof(XQStage) % 1024 == 0, "stages keep the operands' 1024-byte alignment");

struct __align__(1024) XQSmem {
    XQStage st[XQ_STAGES];
    uint64_t full_bq[XQ_STAGES];              // B, mu, d landed (TMA) and the Q rows written: 2 arrivals
    uint64_t full_in[XQ_STAGES][XP_TN / 4];   // input rows of columns 4g .. 4g + 3 landed
    uint64_t done[XQ_STAGES];                 // the stage's product is in its TMEM columns
    uint64_t tfree[XQ_STAGES];                // the epilogue has read those columns
    uint64_t empty[XQ_STAGES];                // the epilogue is done with the stage
    int at[XQ_STAGES];                        // position tile; -1: no more tiles
    int tad[XQ_STAGES];                       // some column adapts its penalty on this call
    int acc[XQ_STAGES][XP_TN];                // account of each column (-1: padding)
    float4 pa[XQ_STAGES][XP_TN];              // rho, 1/rho, L/rho, c/rho (NaN: c differs over positions)
    float4 pb[XQ_STAGES][XP_TN];              // l (NaN: differs), active, adaptation call, unused
    float r5[XQ_STAGES][4][5][XP_TN];         // per lane quarter and column: residual maxima
    unsigned cm[XQ_STAGES][4][XP_TN];         // per lane quarter and column: candidate masks
    unsigned amask[XQ_WMAX];                  // bit b of word w: account m0 + 32 w + b iterates
    uint16_t apre[XQ_WMAX];                   // active accounts in the words before w
    int nact;
    uint32_t tmem;
};
// two CTAs per SM: 2 x (this + its alignment slack + 1 KB reserved per CTA) <= 228 KB
static_assert(2 * (sizeof(XQSmem) + 1024 + 1024) <= 228 * 1024, "two persistent CTAs fit one SM");
constexpr uint32_t XQ_BMD_BYTES = G4_TILE_BYTES + 2 * TM * 4;   // B tile, mu, d (by TMA)

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// the epilogue warps only (named barrier 1)
__device__ __forceinline__ void xq_epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(XQ_EPI) : "memory"); }

// the same barrier, returning to every epilogue thread whether v was true for any of them
__device__ __forceinline__ bool xq_epi_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(uint32_t(v)), "n"(XQ_EPI)
        : "memory");
    return r != 0;
}

// bit index of the n-th (from 0) set bit of w (w has more than n set bits)
__device__ __forceinline__ int nth_set_bit(unsigned w, int n) {
    for (int i = 0; i < n; ++i) w &= w - 1u;
    return __ffs(w) - 1;
}

// The epilogue of one stage's tile for this warp's columns j0 .. j0 + XP_JN - 1: the arithmetic of
// xp_accounts (products not folded) with each column's account taken from the stage. A padding
// column is evaluated like the others and nothing of it is stored (no branch on the column, so
// that the columns' reductions interleave). ax.obase is the position alone.
// ADAPT: some column of the tile adapts its penalty on this call (the terms of the adaptation's
// residual ratio are formed for the columns that do); chosen per tile, so that the loop over the
// columns has no branch on a column's flag. The inputs of all the warp's columns are waited for
// before the loop, for the same reason.
template <bool UNIFORM, bool ADAPT>
__device__ __forceinline__ void xq_accounts(const Dev& D, XQSmem& s, int sti, const XPAsset& ax, const float* bq,
                                            int j0, int q, int lane, uint32_t par, bool have) {
    const bool row_ok = have && ax.i < D.N;
    const float alpha = D.alpha, oma = __fsub_rn(1.f, alpha);
    float4* crec = reinterpret_cast<float4*>(D.crec);
    const XQStage& S = s.st[sti];
    if (have)
        for (int g = j0 / 4; g < (j0 + XP_JN) / 4; ++g) mbar_wait(&s.full_in[sti][g], par, D.err, 64);
#pragma unroll
    for (int jj = 0; jj < XP_JN; ++jj) {
        const int j = j0 + jj;
        const int m = s.acc[sti][j];
        const float4 pa = s.pa[sti][j], pb = s.pb[sti][j];
        const float rho = pa.x, irho = pa.y, Lr = pa.z;   // Lr = L / rho
        const bool ok = row_ok && m >= 0;
        // element offset in 32 bits (as in k_tc_xprox): a book of 2^32 entries could not hold its
        // workspace in device memory
        const uint32_t off = uint32_t(m >= 0 ? m : 0) * uint32_t(D.Npad) + uint32_t(ax.obase);
        float lo = pb.x, k = pa.w;                      // k = c / rho
        const bool lou = UNIFORM || !isnan(lo);         // warp-uniform
        if (!UNIFORM) {
            if (ok && !lou) lo = D.lo[off];
            if (ok && isnan(k)) k = __fmul_rn(D.c[off], irho);
        }
        const float z0 = S.in[0][j][ax.ia], y0 = S.in[1][j][ax.ia], w0 = S.in[2][j][ax.ia], up = S.in[3][j][ax.ia];
        const XPEntry en = xp_entry(ax.mu, ax.dd, rho, irho, Lr, k, lo, up, z0, y0, w0, bq[jj], alpha, oma);
        const float v = en.v, yn = en.yn;
        const bool pin = ok && (en.z == lo);
        const bool cand = ok && !pin;
        const float e_rp = pin ? fabsf(__fsub_rn(yn, y0)) : 0.f;
        const float e_rd = pin ? fabsf(__fsub_rn(lo, z0)) : 0.f;
        if (cand) D.v[off] = v;
        if (pin) {
            if (z0 != lo) D.z[off] = lo;
            D.y[off] = yn;
            const float X = en.X;
            const __nv_bfloat16 h = __float2bfloat16_rn(X);
            D.Xhi[off] = h;
            D.Xlo[off] = __float2bfloat16_rn(__fsub_rn(X, __bfloat162float(h)));
        }
        if (cand) {
            crec[2 * (size_t)off] = make_float4(v, w0, up, z0);
            crec[2 * (size_t)off + 1] = make_float4(y0, ax.mu, 0.5f * ax.dd, 0.f);
        }
        const unsigned cm = __ballot_sync(0xffffffffu, cand);
        float rp = warp_max_nn(e_rp), rd = __fmul_rn(warp_max_nn(e_rd), rho);
        rp = (rp == INFINITY) ? NAN : __fmul_rn(rp, irho);        // a non-finite pinned update: NaN (numerical failure)
        float nx = 0.f, nz = 0.f, ny = 0.f;
        if constexpr (ADAPT) {                          // penalty adaptation on this call (per column)
            const bool ad = pin && pb.z != 0.f;
            nx = warp_max_nn(ad ? fabsf(__fsub_rn(v, en.yir)) : 0.f);
            ny = warp_max_nn(ad ? fabsf(yn) : 0.f);
            if (!lou) nz = warp_max_nn(ad ? fabsf(lo) : 0.f);
        }
        if (!UNIFORM && !lou) {
            for (int g = 0; g < ax.nsegq; ++g) {
                const bool mine = (ax.i < D.N) && ax.segl == g && pin;
                const float sg = warp_sum_f(mine ? lo : 0.f);
                if (lane == 0 && m >= 0) D.SOp[(size_t)(ax.sbase + g) * D.M + m] = sg;
            }
        }
        if (lane == 0) {
            s.r5[sti][q][0][j] = rp;
            s.r5[sti][q][1][j] = rd; s.r5[sti][q][2][j] = nx; s.r5[sti][q][3][j] = nz; s.r5[sti][q][4][j] = ny;
            s.cm[sti][q][j] = cm;
        }
    }
}

// Per-tile outputs of a stage: the residual maxima over the four quarters (NaN kept) and the
// masks, by account. Epilogue thread t.
__device__ __forceinline__ void xq_tile_out(const Dev& D, const XQSmem& s, int sti, int at, int t) {
    if (t < 5 * XP_TN) {
        const int kq = t / XP_TN, col = t % XP_TN, m = s.acc[sti][col];
        if (m >= 0) {
            float r = 0.f;
            bool nan_ = false;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const float x = s.r5[sti][qq][kq][col];
                nan_ |= isnan(x);
                r = fmaxf(r, x);
            }
            D.Rt[((size_t)m * 5 + kq) * D.nt + at] = nan_ ? NAN : r;
        }
    } else if (t >= 128 && t < 128 + 4 * XP_TN) {
        const int w = (t - 128) / XP_TN, col = (t - 128) % XP_TN, m = s.acc[sti][col];
        const int g = at * 4 + w;
        if (m >= 0 && g < D.nq) D.Cm[(size_t)m * D.nq + g] = s.cm[sti][w][col];
    }
}

template <bool UNIFORM>
__global__ void __launch_bounds__(XQ_THREADS, 2) k_tc_xprox_pers(const __grid_constant__ XPMaps mp, Dev D) {
    extern __shared__ unsigned char raw[];
    XQSmem& s = *reinterpret_cast<XQSmem*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m_end = D.m1 ? D.m1 : D.M;
    const int nat = D.nt;
    const int nw = cdiv(m_end - D.m0, 32);              // <= XQ_WMAX (checked by the host)
    constexpr int PROD = XQ_EPI / 32, MMAW = PROD + 1;
    constexpr uint32_t IDESC = idesc_bf16(TM, XP_TN);
    if (warp == 0) tmem_alloc(&s.tmem, 32);
    int t_first = 0;                                    // the producer's first claim
    if (warp == PROD) {
        // the first tile is claimed now, so that the atomic's round trip overlaps the list below
        if (lane == 0) t_first = (int)atomicAdd(D.xq_ctr, 1u);
        // the chain's accounts that iterate (the flags were written by kernels two or more
        // launches back, so they are readable before the dependency wait): a bit mask per 32
        // accounts and the count before each word; the loads of up to 16 words in flight at once
        for (int w0 = 0; w0 < nw; w0 += 16) {
            bool a[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int m = D.m0 + 32 * (w0 + u) + lane;
                a[u] = (w0 + u < nw) && m < m_end && D.active[m] != 0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const unsigned b = __ballot_sync(0xffffffffu, a[u]);
                if (lane == 0 && w0 + u < nw) s.amask[w0 + u] = b;
            }
        }
        __syncwarp();
        int c = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int w = lane * 8 + u;
            if (w < nw) c += __popc(s.amask[w]);
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - c;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int w = lane * 8 + u;
            if (w < nw) {
                s.apre[w] = (uint16_t)run;
                run += __popc(s.amask[w]);
            }
        }
        if (lane == 31) s.nact = incl;
        if (lane == 0) {
            for (int i = 0; i < XQ_STAGES; ++i) {
                mbar_init(&s.full_bq[i], 2);
                for (int g = 0; g < XP_TN / 4; ++g) mbar_init(&s.full_in[i][g], 1);
                mbar_init(&s.done[i], 1);
                mbar_init(&s.tfree[i], XQ_EPI / 32);
                mbar_init(&s.empty[i], XQ_EPI / 32);
            }
            fence_barrier_init();
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s.tmem;
    if (warp == PROD) {
        // ---- producer. The claim of the next tile and the constants of its accounts are fetched
        // before the wait for a free stage, so that their latency overlaps it.
        unsigned* ctr = D.xq_ctr;
        const int nact = s.nact;
        const int total = cdiv(nact, XP_TN) * nat;
        static_assert(XQ_STAGES == 2, "the last use of each stage is kept in two registers");
        int last0 = -1, last1 = -1;      // last use of each stage that issued loads
        bool waited = false;
        int t = __shfl_sync(0xffffffffu, t_first, 0);
        for (int k = 0;; ++k) {
            const int sti = k % XQ_STAGES, use = k / XQ_STAGES;
            XQStage& S = s.st[sti];
            const bool more = t < total;
            const int grp = more ? t / nat : 0, at = more ? t % nat : 0;
            // lane j < 16: the (16 grp + j)-th active account of the chain, and its constants
            int m = -1, ridx = 0, itr = 0;
            float nu = 0.f, dnu = 0.f, cu = 0.f, lu = 0.f;
            if (more && lane < XP_TN) {
                const int r = grp * XP_TN + lane;
                if (r < nact) {
                    int lo = 0, hi = nw - 1;                 // the last word with apre <= r
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((int)s.apre[mid] <= r) lo = mid; else hi = mid - 1;
                    }
                    m = D.m0 + 32 * lo + nth_set_bit(s.amask[lo], r - (int)s.apre[lo]);
                    ridx = D.rho_idx[m]; nu = D.nu[m]; dnu = D.dnu[m]; cu = D.c_u[m]; lu = D.lo_u[m];
                    itr = D.iters[m];
                }
            }
            int tn = 0;
            if (more && lane == 0) tn = (int)atomicAdd(ctr, 1u);
            if (use > 0 && !mbar_wait(&s.empty[sti], (use - 1) & 1, D.err, 256)) break;
            if (!more) {
                if (lane == 0) {
                    s.at[sti] = -1;
                    mbar_arrive(&s.full_in[sti][0]);
                    mbar_arrive(&s.full_bq[sti]);
                    mbar_arrive(&s.full_bq[sti]);
                    if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
                        ctr[0] = 0;
                        ctr[1] = 0;
                    }
                }
                if (sti == 0) last0 = -1; else last1 = -1;   // released by the epilogue, no loads since
                break;
            }
            if (lane < XP_TN) {
                const bool ok = m >= 0;
                const float r = ok ? rho_of_idx(ridx) : 1.f;
                const float L = ok ? nu - fmaxf(4.f * dnu, 2e-3f) : 0.f;
                const float ir = 1.f / r;
                const bool adapt = ok && ((itr + 1) % D.adapt_every == 0);
                s.acc[sti][lane] = m;
                s.pa[sti][lane] = make_float4(r, ir, L * ir, (ok ? cu : 0.f) * ir);
                s.pb[sti][lane] = make_float4(ok ? lu : 0.f, ok ? 1.f : 0.f, adapt ? 1.f : 0.f, 0.f);
            }
            // columns with an account; groups of four whose accounts are consecutive take one
            // box of four rows per array, the others a row per account; a tile of 16 consecutive
            // accounts takes its Q split as a box too
            const int m0c = __shfl_sync(0xffffffffu, m, 0);
            const unsigned have_col = __ballot_sync(0xffffffffu, lane < XP_TN && m >= 0);
            const unsigned adapt_col =
                __ballot_sync(0xffffffffu, lane < XP_TN && m >= 0 && (itr + 1) % D.adapt_every == 0);
            const unsigned cons = __ballot_sync(0xffffffffu, lane < XP_TN && m >= 0 && m == m0c + lane);
            const bool qbox = (cons & 0xffffu) == 0xffffu;
            unsigned gbox = 0u;                              // bit g: group g as one box
#pragma unroll
            for (int g = 0; g < XP_TN / 4; ++g) {
                const unsigned gm = 0xfu << (4 * g);
                const int mg = __shfl_sync(0xffffffffu, m, 4 * g);
                const unsigned gc = __ballot_sync(0xffffffffu, lane >= 4 * g && lane < 4 * g + 4 && m >= 0 &&
                                                                   m == mg + (lane - 4 * g));
                if ((gc & gm) == gm) gbox |= 1u << g;
            }
            if (lane == 0) {
                s.at[sti] = at;
                s.tad[sti] = adapt_col != 0u;
                mbar_expect_tx(&s.full_bq[sti], XQ_BMD_BYTES + (qbox ? 2 * XP_Q_BYTES : 0u));
                tma_load_2d(S.a, &mp.B, &s.full_bq[sti], 0, at * TM);
                tma_load_2d(S.md[0], &mp.mu, &s.full_bq[sti], at * TM, 0);
                tma_load_2d(S.md[1], &mp.d, &s.full_bq[sti], at * TM, 0);
                for (int g = 0; g < XP_TN / 4; ++g)
                    mbar_expect_tx(&s.full_in[sti][g], (uint32_t)__popc((have_col >> (4 * g)) & 0xfu) * 4u * (TM * 4u));
            }
            __syncwarp();
            if (lane < XP_TN && m >= 0) {
                uint64_t* bar = &s.full_in[sti][lane / 4];
                if (gbox & (1u << (lane / 4))) {
                    if ((lane & 3) == 0) {
                        tma_load_2d(S.in[0][lane], &mp.z, bar, at * TM, m);
                        tma_load_2d(S.in[1][lane], &mp.y, bar, at * TM, m);
                        tma_load_2d(S.in[2][lane], &mp.w0, bar, at * TM, m);
                        tma_load_2d(S.in[3][lane], &mp.up, bar, at * TM, m);
                    }
                } else {
                    tma_load_2d(S.in[0][lane], &mp.zr, bar, at * TM, m);
                    tma_load_2d(S.in[1][lane], &mp.yr, bar, at * TM, m);
                    tma_load_2d(S.in[2][lane], &mp.w0r, bar, at * TM, m);
                    tma_load_2d(S.in[3][lane], &mp.upr, bar, at * TM, m);
                }
            }
            // Q comes from the small solve just before: the first tile's other operands go out
            // before the dependency wait, its Q after. Without the box, lane l copies 64 bytes of
            // row l / 2 of each split term into the K-major 128-byte-swizzled layout (16-byte
            // chunk c of row r at chunk c ^ (r % 8)); a padding row is zero.
            if (!waited) {
                pdl_wait();
                pdl_trigger();
                waited = true;
            }
            if (qbox) {
                if (lane == 0) {
                    tma_load_2d(S.bhi, &mp.Qhi, &s.full_bq[sti], 0, m0c);
                    tma_load_2d(S.blo, &mp.Qlo, &s.full_bq[sti], 0, m0c);
                }
            } else {
                const int r = lane >> 1, h = lane & 1;
                const int mr = __shfl_sync(0xffffffffu, m, r);
                uint4 vh[4], vl[4];
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int ch = h * 4 + c4;
                    if (mr >= 0) {
                        vh[c4] = reinterpret_cast<const uint4*>(D.Qhi + (size_t)mr * KP)[ch];
                        vl[c4] = reinterpret_cast<const uint4*>(D.Qlo + (size_t)mr * KP)[ch];
                    } else {
                        vh[c4] = make_uint4(0u, 0u, 0u, 0u);
                        vl[c4] = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
                uint8_t* bh = reinterpret_cast<uint8_t*>(S.bhi);
                uint8_t* bl = reinterpret_cast<uint8_t*>(S.blo);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int ch = h * 4 + c4;
                    const uint32_t o = uint32_t(r * 128 + ((ch ^ (r & 7)) << 4));
                    *reinterpret_cast<uint4*>(bh + o) = vh[c4];
                    *reinterpret_cast<uint4*>(bl + o) = vl[c4];
                }
                fence_proxy_async_smem();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.full_bq[sti]);
            if (sti == 0) last0 = use; else last1 = use;
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
        if (!waited) {
            pdl_wait();
            pdl_trigger();
        }
        // copies of this CTA still in flight (none unless a wait expired)
        if (lane == 0)
            for (int i = 0; i < XQ_STAGES; ++i) {
                const int lu = i == 0 ? last0 : last1;
                if (lu < 0) continue;
                const uint32_t par = lu & 1;
                mbar_wait(&s.full_bq[i], par, D.err, 256);
                for (int g = 0; g < XP_TN / 4; ++g) mbar_wait(&s.full_in[i][g], par, D.err, 256);
            }
        __syncwarp();
    } else if (warp == MMAW) {
        // ---- MMA issue
        pdl_wait();
        pdl_trigger();
        if (lane == 0) {
            int last0 = -1, last1 = -1;  // last use of each stage that issued a product
            for (int k = 0;; ++k) {
                const int sti = k % XQ_STAGES, use = k / XQ_STAGES;
                if (!mbar_wait(&s.full_bq[sti], use & 1, D.err, 16)) break;
                if (*reinterpret_cast<volatile int*>(&s.at[sti]) < 0) break;
                if (use > 0 && !mbar_wait(&s.tfree[sti], (use - 1) & 1, D.err, 16)) break;
                fence_after_sync();
                const XQStage& S = s.st[sti];
                const uint64_t da = sw128_desc(S.a), dh = sw128_desc(S.bhi), dl = sw128_desc(S.blo);
                const uint32_t dt = tmem + uint32_t(sti * XP_TN);
#pragma unroll
                for (int kk = 0; kk < KP / 16; ++kk) {
                    umma_bf16(dt, da + 2 * kk, dh + 2 * kk, IDESC, kk > 0 ? 1u : 0u);
                    umma_bf16(dt, da + 2 * kk, dl + 2 * kk, IDESC, 1u);
                }
                umma_commit(&s.done[sti]);
                if (sti == 0) last0 = use; else last1 = use;
            }
            // products of this CTA still running (none unless a wait expired)
            if (last0 >= 0) mbar_wait(&s.done[0], last0 & 1, D.err, 16);
            if (last1 >= 0) mbar_wait(&s.done[1], last1 & 1, D.err, 16);
        }
        __syncwarp();
    } else {
        // ---- epilogue
        pdl_wait();
        pdl_trigger();
        const int q = warp & 3;                              // TMEM lane quarter
        const int j0 = (warp >> 2) * XP_JN;                  // first account column of this warp
        bool bad = false;                                    // a wait of this warp expired
        for (int k = 0;; ++k) {
            const int sti = k % XQ_STAGES, use = k / XQ_STAGES;
            const uint32_t par = use & 1;
            const bool got = mbar_wait(&s.full_in[sti][0], par, D.err, 64);
            const int at = got ? *reinterpret_cast<volatile int*>(&s.at[sti]) : -1;
            // every epilogue warp takes the same branch: the tile word is the same for all, and
            // an expired wait of any warp stops all of them
            if (xq_epi_sync_or(bad || !got || at < 0)) break;
            // the product, and the stage's operands it followed (mu and d among them)
            const bool have = mbar_wait(&s.done[sti], par, D.err, 32) && mbar_wait(&s.full_bq[sti], par, D.err, 32);
            float bq[XP_JN];
            if (have) {
                fence_after_sync();
                tmem_ld8(tmem + (uint32_t(q * 32) << 16) + uint32_t(sti * XP_TN + j0), bq);
            } else {
                bad = true;
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.tfree[sti]);
            XPAsset ax;
            if constexpr (UNIFORM) {
                // no sector segments in this form: the position, and mu, d from the stage
                ax.ia = q * 32 + lane;
                ax.i = at * TM + ax.ia;
                ax.obase = ax.i < D.N ? ax.i : 0;
                ax.mu = s.st[sti].md[0][ax.ia];
                ax.dd = 2.f * s.st[sti].md[1][ax.ia];
                ax.nsegq = 0; ax.segl = 0; ax.sbase = 0;
            } else {
                ax = xp_asset(D, at, q, lane, 0);
            }
            if (s.tad[sti]) xq_accounts<UNIFORM, true>(D, s, sti, ax, bq, j0, q, lane, par, have);
            else xq_accounts<UNIFORM, false>(D, s, sti, ax, bq, j0, q, lane, par, have);
            xq_epi_sync();
            if (have) xq_tile_out(D, s, sti, at, tid);
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.empty[sti]);
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------------------------------
// host side: tensor maps and launches
// ---------------------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D BF16 map: inner dimension dim0 (contiguous), rows dim1 with the given byte stride.
static bool map2d(CUtensorMap* m, const void* base, uint64_t dim0, uint64_t dim1, uint64_t row_bytes, uint32_t box0,
                  uint32_t box1) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {dim0, dim1};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D FP32 map of an M x Npad account-major array: boxes of box0 positions x box1 accounts,
// no swizzle (the epilogue reads a row of positions per account), zero fill out of range.
static bool map2d_f32(CUtensorMap* m, const void* base, uint64_t npad, uint64_t rows, uint32_t box0, uint32_t box1) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {npad, rows};
    cuuint64_t strides[1] = {npad * 4};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

bool tc_available() { return tc::encoder() != nullptr; }

int tc_nsplit(int M, int N, int* chunk_out, int sets) {
    // about one CTA per SM: G2_CL splits per cluster, nsets clusters per account tile (or the
    // caller's tile shape)
    const int mtiles = cdiv(M, tc::TM);
    int nsets = sets > 0 ? sets : std::max(1, int(std::lround(152.0 / double(mtiles * tc::G2_CL))));
    nsets = std::min(nsets, std::max(1, cdiv(cdiv(N, tc::TK), tc::G2_CL)));
    const int ns = nsets * tc::G2_CL;
    *chunk_out = std::max(tc::TK, cdiv(cdiv(N, ns), tc::TK) * tc::TK);
    return nsets;
}

void launch_tc_gemm_P(const Dev& D, cudaStream_t st, bool pdl) {
    CUtensorMap mXhi, mXlo, mBt;
    bool ok = tc::map2d(&mXhi, D.Xhi, D.Npad, D.M, (uint64_t)D.Npad * 2, tc::TK, tc::TM) &&
              tc::map2d(&mXlo, D.Xlo, D.Npad, D.M, (uint64_t)D.Npad * 2, tc::TK, tc::TM) &&
              tc::map2d(&mBt, D.Bt16p, D.Npad, tc::KP, (uint64_t)D.Npad * 2, tc::TK, tc::KP);
    if (!ok) { set_error("tensor map encoding failed (G2)"); return; }
    int chunk = 0;
    const int nsets = tc_nsplit(D.M, D.N, &chunk, D.g2_sets);
    const size_t smem = sizeof(tc::G2Smem) + 1024;
    cudaFuncSetAttribute(tc::k_tc_gemm_P, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cdiv((D.m1 ? D.m1 : D.M) - D.m0, tc::TM), nsets * tc::G2_CL);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = tc::G2_CL;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, tc::k_tc_gemm_P, mXhi, mXlo, mBt, D, chunk);
}

void launch_tc_gemm_x(const Dev& D, cudaStream_t st) {
    CUtensorMap mB, mQhi, mQlo;
    bool ok = tc::map2d(&mB, D.B16p, tc::KP, D.Npad, tc::KP * 2, tc::KP, tc::TM) &&
              tc::map2d(&mQhi, D.Qhi, tc::KP, D.M, tc::KP * 2, tc::KP, tc::G4_TN) &&
              tc::map2d(&mQlo, D.Qlo, tc::KP, D.M, tc::KP * 2, tc::KP, tc::G4_TN);
    if (!ok) { set_error("tensor map encoding failed (G4)"); return; }
    const size_t smem = sizeof(tc::G4Smem) + 1024;
    cudaFuncSetAttribute(tc::k_tc_gemm_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(cdiv(D.N, tc::TM), cdiv(D.M, tc::G4_TN));
    tc::k_tc_gemm_x<<<grid, tc::G4_THREADS, smem, st>>>(mB, mQhi, mQlo, D);
}

void launch_tc_xprox(const Dev& D, cudaStream_t st, bool pdl) {
    tc::XPMaps mp;
    bool ok = tc::map2d(&mp.B, D.B16p, tc::KP, D.Npad, tc::KP * 2, tc::KP, tc::TM) &&
              tc::map2d(&mp.Qhi, D.Qhi, tc::KP, D.M, tc::KP * 2, tc::KP, tc::XP_TN) &&
              tc::map2d(&mp.Qlo, D.Qlo, tc::KP, D.M, tc::KP * 2, tc::KP, tc::XP_TN) &&
              tc::map2d_f32(&mp.z, D.z, D.Npad, D.M, tc::TM, 4) &&
              tc::map2d_f32(&mp.y, D.y, D.Npad, D.M, tc::TM, 4) &&
              tc::map2d_f32(&mp.w0, D.w0, D.Npad, D.M, tc::TM, 4) &&
              tc::map2d_f32(&mp.up, D.up, D.Npad, D.M, tc::TM, 4) &&
              tc::map2d_f32(&mp.zr, D.z, D.Npad, D.M, tc::TM, 1) &&
              tc::map2d_f32(&mp.yr, D.y, D.Npad, D.M, tc::TM, 1) &&
              tc::map2d_f32(&mp.w0r, D.w0, D.Npad, D.M, tc::TM, 1) &&
              tc::map2d_f32(&mp.upr, D.up, D.Npad, D.M, tc::TM, 1) &&
              tc::map2d_f32(&mp.mu, D.mu32, D.Npad, 1, tc::TM, 1) &&
              tc::map2d_f32(&mp.d, D.d32, D.Npad, 1, tc::TM, 1);
    if (!ok) { set_error("tensor map encoding failed (G4 fused)"); return; }
    const size_t smem = sizeof(tc::XPSmem) + 1024;
    dim3 grid(cdiv(D.N, tc::TM), cdiv((D.m1 ? D.m1 : D.M) - D.m0, tc::XP_TN));
    const int mspan = (D.m1 ? D.m1 : D.M) - D.m0;
    if (!D.fold && D.xq_ctr && cdiv(mspan, 32) <= tc::XQ_WMAX) {
        // persistent CTAs, two per SM (no more than there are tiles)
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            cudaGetLastError();
            nsm = 1;
        }
        const size_t psmem = sizeof(tc::XQSmem) + 1024;
        const int tiles = cdiv(D.N, tc::TM) * cdiv(mspan, tc::XP_TN);
        auto pk = D.uniform ? tc::k_tc_xprox_pers<true> : tc::k_tc_xprox_pers<false>;
        cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
        // a chain of several takes its share of the SMs, so that the other chains' kernels
        // keep room beside it
        const int ctas = std::max(1, 2 * nsm / std::max(1, D.xq_share));
        launch_ex(pk, dim3(std::min(tiles, ctas)), dim3(tc::XQ_THREADS), psmem, st, pdl, mp, D);
        return;
    }
    auto kern = D.fold ? (D.uniform ? tc::k_tc_xprox<true, true> : tc::k_tc_xprox<false, true>)
                       : (D.uniform ? tc::k_tc_xprox<true, false> : tc::k_tc_xprox<false, false>);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_ex(kern, grid, dim3(tc::XP_THREADS), smem, st, pdl, mp, D);
}

}  // namespace prism
