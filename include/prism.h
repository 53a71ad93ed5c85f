/*
 * prism.h -- C-ABI of the GB300 batched rebalancing solver.
 *
 * The library solves a book of account rebalancing problems in one call. Each
 * account a is the convex program of Eq. 1 (Sec. 4.2) as the workloads use it,
 * with the objective scaled as in the Sec. 9 display (Q = 2 Sigma, eta = 1):
 *
 *   minimise   w' Sigma w - mu' w + sum_i phi_i(w_i)
 *   subject to 1'w = 1,  l <= w <= u,  lo_s <= sum_{i in s} w_i <= hi_s,
 *              ||w - w0||_1 <= tau,          Sigma = B diag(f) B' + diag(d),
 *
 * where phi_i is the transition cost against the current holdings w0: an L1
 * cost c_i |w_i - w0_i|, or, when tax lots are given, the convex lot model
 * phi(w) = c (w - w0) + G(max(S*, w0 - w)), G(S) = 2 c S + (cheapest-first tax
 * cost of selling S), S* = total size of lots with 2c + kappa < 0.
 *
 * The boundary follows the paper's public solver call (Fig. 2, Sec. 4.3):
 * problem data in; weights, per-account status codes (Table "Status
 * vocabulary", Sec. 10.2), timings, memory class and the feasibility / KKT
 * diagnostics of Sec. 4.4 out.
 *
 * Conventions for every entry point
 *  - Pointers may be host or device memory; the library tells them apart with
 *    cudaPointerGetAttributes. The caller owns every input and output buffer;
 *    the library copies what it needs and never keeps a caller pointer.
 *  - Return value: 0 on success, a negative PRISM_ERR_* code on a call-level
 *    error (bad argument, CUDA error, allocation failure). The message is
 *    available from prism_last_error() (thread-local). Per-account outcomes
 *    are reported through prism_result.status, not the return value.
 *  - Nothing here throws or aborts; no entry point may be called concurrently
 *    on the same handle from two threads.
 */
#ifndef PRISM_H
#define PRISM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- call-level return codes ---------------------------------------- */
#define PRISM_OK                 0
#define PRISM_ERR_ARGUMENT     (-1)   /* bad size, NULL pointer, non-finite data, infeasible layout */
#define PRISM_ERR_CUDA         (-2)   /* a CUDA runtime call failed */
#define PRISM_ERR_ALLOCATION   (-3)   /* device or host allocation failed */
#define PRISM_ERR_UNSUPPORTED  (-4)   /* option combination not implemented */

/* ---- per-account status codes (Table "Status vocabulary", Sec. 10.2) ----- */
#define PRISM_CERTIFIED              0  /* weights returned, all external checks pass */
#define PRISM_FEASIBLE_NONCERTIFIED  1  /* feasibility passes, KKT certification does not */
#define PRISM_TIMEOUT                2  /* iteration cap or time budget reached first */
#define PRISM_DEADLINE_EXCEEDED      3  /* completed after the window (queue runs only) */
#define PRISM_NO_FEASIBLE_RETURN     4  /* no output passed the gates (incl. capacity test) */
#define PRISM_ALLOCATION_FAILURE     5  /* problem object could not be allocated */
#define PRISM_NUMERICAL_FAILURE      6  /* NaN/Inf met in the iterates */

/* ---- precision modes ---------------------------------------------------- */
#define PRISM_PLAIN_FP32    0  /* one account per launch sequence, FP32 B, SIMT products */
#define PRISM_BATCHED_FP32  1  /* all accounts batched, FP32 B, SIMT products */
#define PRISM_BATCHED_BF16  2  /* all accounts batched, tcgen05 BF16 products (split hi+lo
                                  operands), FP32 accumulate */
#define PRISM_PLAIN_FP64    3  /* one account per launch sequence, FP64 iterations: all of an
                                  account's ADMM iterations in one FP64 launch (capacitance
                                  formed and factored in FP64 per penalty); the time budget is
                                  checked between accounts */

/* ---- universe ----------------------------------------------------------- */
/* Universe-level data shared by every account (Eq. 1 risk model, Sec. 4.2
 * "structural facts": factor-structured risk, O(N K) objective and gradient).
 * All arrays are FP64 (sector: int32), host or device; the library copies them. */
typedef struct {
    int32_t n_assets;       /* N >= 1 */
    int32_t n_factors;      /* K in [1, 64] */
    int32_t n_sectors;      /* S in [1, 64] */
    const double* B;        /* N x K factor loadings, row-major */
    const double* f;        /* K factor variances (> 0), F = diag(f) */
    const double* d;        /* N idiosyncratic variances (> 0), D = diag(d) */
    const double* mu;       /* N return input */
    const int32_t* sector;  /* N sector ids in [0, S) */
    int32_t device;         /* CUDA device ordinal */
} prism_universe_desc;

typedef struct prism_universe prism_universe;
typedef struct prism_state prism_state;

/* Validate and copy a universe to the device; precompute the FP32/BF16 copies
 * of B and the Woodbury capacitance inverses (2F)^{-1} + B' Delta^{-1} B for the
 * solver's penalty grid. *out receives an opaque handle owned by the caller
 * (release with prism_destroy_universe). */
int prism_create_universe(const prism_universe_desc* desc, prism_universe** out);
void prism_destroy_universe(prism_universe* u);

/* ---- a book of accounts ------------------------------------------------- */
/* Per-account data, ragged: account a owns entries offsets[a] .. offsets[a+1]-1.
 * Entry e refers to universe asset asset_idx[e], or, when asset_idx is NULL,
 * entry offsets[a] + i refers to asset i (every account spans the universe in
 * universe order, offsets[a+1] - offsets[a] == N). All FP64 unless noted. */
typedef struct {
    int32_t n_accounts;             /* M >= 1 */
    const int64_t* offsets;         /* M + 1, offsets[0] == 0, nondecreasing */
    const int32_t* asset_idx;       /* ragged universe rows, or NULL */
    const double* w0;               /* current holdings, ragged */
    const double* lower;            /* box lower bounds l, ragged (>= 0 when lots are given) */
    const double* upper;            /* box upper bounds u, ragged (u == l excludes the name) */
    const double* tc;               /* L1 transition cost c_i >= 0 per unit traded, ragged */
    const double* band_lo;          /* M x S sector band lower edges (may be -inf) */
    const double* band_hi;          /* M x S sector band upper edges (may be +inf) */
    const double* turnover_cap;     /* M turnover caps tau (+inf = none), or NULL = none */
    const int64_t* lot_offsets;     /* ragged+1 lot ranges per entry, or NULL = no lots */
    const double* lot_size;         /* lot sizes (weight units), sum per entry == w0 */
    const double* lot_kappa;        /* marginal tax per unit sold (negative = harvest) */
    /* Further families of Eq. 1 (Sec. 4.2); each NULL = absent. */
    const double* mu_tilt;          /* ragged per-account tilt t of the return input: the linear
                                       term is (mu + t)'w for that account */
    const double* w_bench;          /* ragged benchmark weights w_b: the risk term is
                                       (w - w_b)' Sigma (w - w_b), i.e. a tilt of 2 Sigma w_b
                                       (the objective in diag column 6 omits the constant
                                       w_b' Sigma w_b) */
    const double* factor_lo;        /* M x K lower bounds on the factor exposures B'w (the
                                       general rows a_lo <= A w <= a_hi of Eq. 1 with A = B' of
                                       the account's names; -inf = none) */
    const double* factor_hi;        /* M x K upper bounds (+inf = none); NULL both = no bounds */
} prism_batch;

/* ---- options -------------------------------------------------------------- */
typedef struct {
    double  eps_kkt;          /* certification gate on every residual (default 1e-6) */
    double  eps_admm;         /* ADMM residual target before the polish (default 5e-4) */
    double  rho0;             /* initial ADMM penalty (default 3.0) */
    double  alpha;            /* over-relaxation (default 1.5) */
    double  time_budget_s;    /* wall-clock ceiling for the call (<= 0: none) */
    int32_t max_iter;         /* ADMM iteration cap per account (default 4000) */
    int32_t check_every;      /* iterations per captured graph launch (default 20) */
    int32_t min_iter;         /* iterations before a convergence test may stop an account */
    int32_t polish_rounds;    /* active-set correction rounds per polish (default 8) */
    int32_t precision;        /* PRISM_PLAIN_FP32 | PRISM_BATCHED_FP32 | PRISM_BATCHED_BF16 | PRISM_PLAIN_FP64 */
    int32_t use_graph;        /* capture the iteration loop in a CUDA graph (default 1) */
    int32_t keep_for_backward;/* 1: *res->state receives the polished active set for
                                 prism_solve_batch_backward (batched modes only) */
    int32_t profile;          /* 1: no graph; CUDA events around every launch, per kernel class */
    double  polish_overlap;   /* accounts that stop iterating are polished beside the iterations once
                                 fewer than this fraction of the book still iterates (0 = never:
                                 the whole book is polished after the iterations; default 0) */
    int32_t chains;           /* fused iterations: the book is cut into this many account ranges
                                 (multiples of 128) that iterate independently on their own
                                 streams; 0 = one with the persistent x-update (xupdate_form 0),
                                 else as many as fit, up to 4 (default 0) */
    int32_t stream_after;     /* iterations of the staged prox before the streaming form, which
                                 needs settled multipliers for its margin (default 6) */
    int32_t fuse_prox;        /* 1: for books with the L1 cost only (no lots, no cap) in BATCHED_BF16,
                                 the prox's streaming pass runs inside the tensor-core x-update
                                 (default 1); 0: separate x-update and prox kernels (same method) */
    void*   cuda_stream;      /* cudaStream_t to run on (NULL = the library's own stream) */
    int32_t ragged_layout;    /* books with asset_idx in the batched modes: 1 = dense-masked over the
                                 universe (every product over all N positions, non-members pinned
                                 at 0); 2 = packed (each account's own names only, one persistent
                                 launch of per-account blocks with the account's own capacitance);
                                 0 = dense-masked (the faster of the two on the workloads measured;
                                 prism_autotune times both for a book) (default 0) */
    int32_t g2_sets;          /* tile shape of the tensor-core product B'X: clusters of 8 CTAs per
                                 128-account tile along the assets, each CTA summing an asset chunk
                                 of N / (8 g2_sets) (rounded up to 64); 0 = about one CTA per SM
                                 (default 0; searched by prism_autotune) */
    int32_t fold_products;    /* fused iterations (fuse_prox): 1 = the product B'X of the entries the
                                 fused x-update pins is formed inside that kernel (a second tensor-core
                                 product over its tile) and the roots kernel adds the other entries and
                                 solves for the next Q, so that the separate product and small-solve
                                 kernels work only for accounts whose penalty changed or whose pinned
                                 entries were rewritten; 0 = those kernels every iteration (default 0:
                                 faster on the workloads measured; searched by prism_autotune) */
    int32_t adapt_every;      /* iterations between penalty adaptations of an account (residual
                                 balancing on the rho grid; 0 = 25) (default 25; searched by
                                 prism_autotune) */
    int32_t xupdate_form;     /* fused iterations without folded products: 0 = the fused x-update as
                                 persistent CTAs (two per SM) that take 128-position x 16-account
                                 tiles from a counter, loading the next tiles while the current one
                                 is evaluated; 1 = one CTA per tile (same arithmetic, bit for bit)
                                 (default 0; searched by prism_autotune) */
} prism_solve_opts;

/* Fill *o with the defaults documented above. */
void prism_default_opts(prism_solve_opts* o);

/* ---- results ------------------------------------------------------------- */
/* Diagnostic columns of prism_result.diag (FP64, Sec. 4.4, computed on the
 * device in FP64 from the returned weights and multipliers). */
#define PRISM_DIAG_BUDGET    0  /* |1'w - 1| */
#define PRISM_DIAG_BOX       1  /* largest bound violation */
#define PRISM_DIAG_EXPOSURE  2  /* largest band violation */
#define PRISM_DIAG_TURNOVER  3  /* (||w - w0||_1 - tau)_+ */
#define PRISM_DIAG_STAT      4  /* subgradient stationarity distance */
#define PRISM_DIAG_COMP      5  /* complementarity of bands and cap */
#define PRISM_DIAG_OBJ       6  /* objective w'Sigma w - mu'w + sum phi_i(w_i) */
#define PRISM_DIAG_ERR_EST   7  /* a-posteriori bound on max_i |w_i - w*_i| against the exact
                                     minimiser w*: (|r|_2 + sqrt(|r|_2^2 + 4 m C)) / (2 m) with r
                                     the per-entry stationarity residuals, m = 2 min_i d_i the
                                     strong-convexity modulus of the risk and C the multipliers
                                     times their constraints' slacks; valid for a point that
                                     meets the constraints (columns 0-3 give how far the returned
                                     point misses them); +inf for an uncertified account */
#define PRISM_NDIAG          8

/* Kernel classes of prism_result.kernel_ms / kernel_launches (profile mode). */
#define PRISM_K_GEMM_P   0  /* shared-B reduction P = B' X over assets */
#define PRISM_K_SOLVE_K  1  /* K x K capacitance solves */
#define PRISM_K_GEMM_X   2  /* x-update B Q with the relaxation epilogue */
#define PRISM_K_PROX     3  /* prox / projection / dual update / control */
#define PRISM_K_POLISH   4  /* FP64 polish round (includes the certification checks) */
#define PRISM_K_PACK     5  /* input packing and validation */
#define PRISM_K_OTHER    6  /* capacity test, init, counters, classification, status */
#define PRISM_K_UNPACK   7  /* output unpacking */
#define PRISM_K_XPROX    8  /* x-update B Q fused with the streaming pass of the prox (L1-only books) */
#define PRISM_K_ROOTS    9  /* per-account multipliers, candidates and control after PRISM_K_XPROX */
#define PRISM_K_BLOCK   10  /* every iteration of an account in one block (PLAIN_FP64; packed ragged books) */
#define PRISM_NKCLASS   11

typedef struct {
    double*  w;             /* ragged weights, same layout as prism_batch (required) */
    double*  nu;            /* M budget multipliers, or NULL */
    double*  lambda_band;   /* M x S band multipliers, or NULL */
    double*  theta;         /* M cap multipliers, or NULL */
    int32_t* status;        /* M per-account status (required) */
    int32_t* iters;         /* M ADMM iterations used, or NULL */
    double*  diag;          /* M x PRISM_NDIAG diagnostics, or NULL */
    /* host scalars written by the call */
    double   t_device_ms;   /* device time of the solve (CUDA events on the solve stream) */
    double   t_call_ms;     /* host wall clock of the whole call (full-call lane, Sec. 5.4) */
    double   t_phase_ms[4]; /* device time of: setup, ADMM iterations, polish, certification */
    int64_t  device_bytes;  /* device memory held by the solve (memory class, Sec. 6) */
    int64_t  n_launches;    /* kernels this call launched (graph replays included) */
    double   kernel_ms[PRISM_NKCLASS];        /* profile mode: summed event time per class */
    int64_t  kernel_launches[PRISM_NKCLASS];  /* profile mode: launches per class */
    int64_t  stream_entries;     /* profile mode: account-entries the fused streaming pass evaluated */
    int64_t  stream_candidates;  /* profile mode: of those, entries not pinned at their lower bound */
    prism_state** state;    /* receives the state for the backward pass, if requested */
    double*  kappa;         /* M x K multipliers of the factor-exposure bounds (>= 0 at the
                               upper bound, <= 0 at the lower), or NULL */
} prism_result;

/* Solve every account of *batch against universe u. All accounts' inputs are
 * validated first (a bad input fails the whole call with PRISM_ERR_ARGUMENT);
 * per-account outcomes are reported in res->status. Output buffers may be host
 * or device memory and must be sized as documented above. */
int prism_solve_batch(prism_universe* u, const prism_batch* batch,
                      const prism_solve_opts* opts, prism_result* res);

/* Implicit differentiation of the polished KKT system (Sec. 4.4 conditions on the
 * active set the polish identified; the variables are those of Eq. 1).
 *
 * For L = sum_a g_a' w_a with g = dL/dw given ragged in the solve's layout (nnz
 * doubles), writes dL/dmu (N), dL/dB (N x K row-major, universe asset order) and
 * dL/dd (N), each summed over the book's accounts, and dL/dw0 (nnz, ragged). Every
 * pointer may be host or device memory; an output pointer may be NULL. Per account
 * one FP64 solve of [2 Sigma_FF, E_F'; E_F, 0] [u; kappa] = [g_F; 0] on the free
 * weights F and working rows E gives all four gradients; the sums over accounts run
 * in a fixed order, so repeated calls return identical numbers. Accounts whose status
 * is not CERTIFIED contribute nothing (their active set is not identified). A weight
 * held at a kink of phi_i (w0_i itself or a tax-lot kink) moves with w0_i; the
 * derivative is that of the locally constant active set (one-sided at degenerate points).
 *
 * state: from prism_solve_batch with keep_for_backward = 1; owned by the caller, who
 * frees it with prism_free_state; the universe it came from must outlive it. It may be
 * used for any number of backward calls (not concurrently). Scratch device memory is
 * allocated on the first call and kept by the state.
 * Returns PRISM_OK; PRISM_ERR_ARGUMENT for NULL state or dL_dw; PRISM_ERR_UNSUPPORTED
 * when an account has more than min(Npad, 2048) free weights or more than 24 working
 * rows; PRISM_ERR_CUDA / PRISM_ERR_ALLOCATION on device failures. */
int prism_solve_batch_backward(prism_state* state, const double* dL_dw,
                               double* dmu, double* dB, double* dd, double* dw0);
/* Release a backward state and its device memory (NULL is a no-op). */
void prism_free_state(prism_state* state);

/* Diagnostic: the two shared-B products of one ADMM x-update, run on the solver's
 * own kernels for the given precision (this library's method; the paper discloses no
 * solver internals, Sec. 3):
 *   P  = X B   (M x K, FP64 out)   and   BQ = Q B'  (M x N, FP64 out),
 * with X (M x N) and Q (M x K) row-major FP64 in universe asset order, host or
 * device. In BATCHED_BF16 mode B is used rounded to BF16 and X, Q are split into
 * two BF16 terms each, exactly as in the solve. PRISM_BATCHED_BF16 | PRISM_PRODUCTS_FUSED
 * takes P from the fused x-update kernel's own product (the one it forms over the entries
 * it pins during a solve; here over every entry of X) instead of the separate G2 kernel.
 * Allocates its own temporaries. */
#define PRISM_PRODUCTS_FUSED 0x100
int prism_shared_b_products(prism_universe* u, int32_t n_accounts, const double* X, const double* Q,
                            int32_t precision, double* P, double* BQ);

/* Allocation-free polish and certification of weights the caller already holds.
 *
 * The paper has no counterpart to this entry point. It exists for callers that
 * cannot allocate device memory when they need an answer: a process that has
 * reserved the whole GPU for its own memory pool, or a latency-bound thread that
 * must not wait on the allocator. Given weights w_in (ragged, the prism_batch
 * layout; for example an earlier solve's result or a warm start) it runs the
 * same FP64 active-set polish and certification kernels as prism_solve_batch
 * and fills res (w, status, nu, lambda_band, theta, diag; iters is set to 0;
 * timings other than t_call_ms are 0).
 *
 * It calls no cudaMalloc / cudaFree and no allocating library routine: all
 * device scratch comes from one static __device__ array that every GPU loading
 * the library holds until the process exits (about 17 MB). Limits
 * (PRISM_ERR_ARGUMENT beyond them): n_accounts <= 32, n_accounts x (universe
 * width rounded up to 64) <= 131072, no tax lots (PRISM_ERR_UNSUPPORTED); an
 * account with more than 512 free weights falls back to the given weights
 * (status FEASIBLE_NONCERTIFIED at best). Buffers are host memory or memory of
 * the universe's device (PRISM_ERR_ARGUMENT for another GPU's memory).
 *
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress. Every call reuses the same array and clears what it
 * reads, so calls that overlap on
 * the GPU (two streams, two threads) race and must be serialised by the caller.
 * Only opts->eps_kkt, opts->polish_rounds and opts->cuda_stream are used. */
int prism_polish_noalloc(prism_universe* u, const prism_batch* batch, const double* w_in,
                         const prism_solve_opts* opts, prism_result* res);

/* Autotuner (no counterpart in the paper, which discloses no solver internals, Sec. 3):
 * picks the iteration schedule for a book by timing trial solves of that book on this GPU.
 * Coordinate-wise search over the initial penalty rho0 (0.5 .. 8), the over-relaxation alpha
 * (1.4 .. 1.8), the iterations per captured graph (5, 10, 20), the staged prox iterations
 * before the streaming form (2 .. 10), the account chains (1, 2, 4) and the ADMM target
 * eps_admm (1e-4 .. 7e-4), the tile shape of the tensor-core product B'X (g2_sets 1 .. 8, BATCHED_BF16),
 * the folded products (fold_products 0, 1; BATCHED_BF16), the form of the fused x-update
 * (xupdate_form 0, 1; BATCHED_BF16 without folded products), the penalty adaptation period
 * (adapt_every 10 .. 50) and, for books of ragged accounts,
 * the layout (dense-masked or packed), starting
 * from *base (or the defaults when base is NULL); a candidate's score is certified accounts
 * per second of device time; one that certifies fewer accounts never wins, and one that
 * certifies as many must be faster than the best so far by more than 1%. Writes the
 * chosen options to *tuned (the other fields copied from base). Runs about 100 full solves,
 * each allocated and timed like a normal call; the book's buffers may be host or device memory and are
 * only read. PLAIN_FP32 is returned unchanged. Returns PRISM_OK or the first failing
 * solve's error code. */
int prism_autotune(prism_universe* u, const prism_batch* batch, const prism_solve_opts* base,
                   prism_solve_opts* tuned);

/* Message of the last failed call on this thread ("" when none). */
const char* prism_last_error(void);

/* Library version string. */
const char* prism_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PRISM_H */
