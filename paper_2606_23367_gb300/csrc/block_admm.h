// block_admm.h -- the per-account ADMM kernel (block_admm.cu): every iteration of an account in
// one thread block, either in FP64 over the dense layout (PRISM_PLAIN_FP64) or in FP32 over a
// packed ragged layout (only the account's own names, the layout of ragged books).
#pragma once

#include "internal.h"

namespace prism {

template <typename T>
struct BlkArgs {
    int M = 0, N = 0, Npad = 0, K = 0, S = 0;
    // universe, sorted positions
    const T* B = nullptr;               // Npad x K
    const T* Bp = nullptr;              // Npad x 64 (factors zero-padded, 16-byte aligned rows), or null
    const T* f = nullptr;               // K
    const T* d = nullptr;               // Npad
    const T* mu = nullptr;              // Npad
    const int* sec_start = nullptr;     // S + 1
    const int* sector = nullptr;        // Npad (-1 = padding)
    // per entry, dense M x Npad (sorted positions)
    const T *w0 = nullptr, *lo = nullptr, *up = nullptr, *c = nullptr;
    const int* pw_idx = nullptr;        // -1 = plain L1 entry
    const T* pw_bp = nullptr;           // n_pw x MAXBP
    const T* pw_sl = nullptr;           // n_pw x (MAXBP - 1)
    const int* pw_nbp = nullptr;
    const T *band_lo = nullptr, *band_hi = nullptr;   // M x S
    const T* tau = nullptr;             // M (+inf = no cap)
    const T *flo = nullptr, *fhi = nullptr;           // M x K factor-exposure bounds, or null
    const int* skip = nullptr;          // M: accounts the capacity test rejected
    // packed layout (null plist: every position of the universe, dense indexing)
    int* plist = nullptr;               // per account, its positions in increasing order (nnz)
    const int64_t* poff = nullptr;      // M + 1: the account's range in plist and in the packed state
    int* psec = nullptr;                // M x (S + 1): sector ranges within the account's list
    int* order = nullptr;               // processing order of the accounts (largest first), or null
    int* queue = nullptr;               // work counter of the persistent blocks
    // state, kept between calls of one solve: dense (M x Npad) or packed (nnz) when plist is set
    T *z = nullptr, *y = nullptr, *X = nullptr;
    T *w0p = nullptr, *lop = nullptr, *upp = nullptr, *cp = nullptr;   // packed copies of the inputs
    int* pwp = nullptr;
    T *rho_state = nullptr, *theta_state = nullptr;   // M
    T *s_state = nullptr, *ys_state = nullptr;        // M x K (factor-exposure block)
    // what the polish reads
    float* zf = nullptr;                // M x Npad
    float *nu_f = nullptr, *eta_hi_f = nullptr, *eta_lo_f = nullptr, *theta_f = nullptr;
    int *iters = nullptr, *active = nullptr, *status = nullptr, *sflag = nullptr;
    double alpha = 1.5, eps = 5e-4, rho0 = 3.0;
    int max_iter = 4000, min_iter = 20, adapt_every = 25;
    int resume = 0;                     // 1: continue from the state (a tighter second pass)
    int stage_cap = 0;                  // packed accounts of at most this many names live in shared memory
    unsigned long long* dbg = nullptr;  // diagnostics (PRISM_DEBUG_STATS): ns per phase, evaluations
};

template <typename T>
int blk_threads();                      // threads per block of the kernel for T
template <typename T>
size_t blk_smem_bytes(const BlkArgs<T>& A);
template <typename T>
void launch_block_admm(const BlkArgs<T>& A, int grid, cudaStream_t st);
template <typename T>
int blk_grid(const BlkArgs<T>& A);      // persistent blocks: SMs x resident blocks, at most M
// per-account position lists and sector ranges of a ragged book (member flags of the dense layout)
void launch_member_lists(int M, int Npad, int S, const int* member, const int* sec_start, const int64_t* poff,
                         int* plist, int* psec, cudaStream_t st);

}  // namespace prism
