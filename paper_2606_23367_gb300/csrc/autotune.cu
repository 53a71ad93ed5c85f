// autotune.cu -- prism_autotune: pick the solver schedule (initial penalty, over-relaxation,
// iterations per captured graph, staged iterations before the streaming prox, account
// chains, ADMM target)
// for a book by timing trial solves of that very book.
//
// The search is coordinate-wise over small grids: first the initial penalty rho0 (the
// schedule's largest effect: it sets how many iterations the accounts need), then the
// over-relaxation alpha, then the graph chunk length, then the number of staged prox
// iterations (fewer are cheaper, but the streaming form then misses its margin more often),
// then the number of independent account chains, then the ADMM target before the polish
// (a looser one saves iterations and costs polish rounds), then the tile shape of the
// tensor-core product B'X (its asset chunk per CTA) and, for ragged books, the layout. A candidate's score is certified
// accounts per second of device time; a candidate that certifies fewer accounts than the
// best so far never wins, and one that certifies as many must be faster by more than 1% (the
// run-to-run spread of a trial). Each trial is a full prism_solve_batch with the caller's book, so
// the result is specific to that book's shape and data (and to this GPU).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace prism {
namespace {

struct Trial {
    double score = -1.0;
    int certified = -1;
    double device_ms = 0.0;
};

Trial run_trial(prism_universe* u, const prism_batch* b, const prism_solve_opts& o, int64_t nnz, int M, int S,
                int reps, int* rc) {
    std::vector<double> w(std::max<int64_t>(nnz, 1)), nu(M), lam((size_t)M * S), theta(M), diag((size_t)M * PRISM_NDIAG);
    std::vector<int32_t> status(M), iters(M);
    Trial t;
    std::vector<double> times;
    for (int r = 0; r < reps; ++r) {
        prism_result res;
        std::memset(&res, 0, sizeof(res));
        res.w = w.data(); res.nu = nu.data(); res.lambda_band = lam.data(); res.theta = theta.data();
        res.status = status.data(); res.iters = iters.data(); res.diag = diag.data();
        *rc = prism_solve_batch(u, b, &o, &res);
        if (*rc != PRISM_OK) return t;
        times.push_back(res.t_device_ms);
    }
    std::sort(times.begin(), times.end());
    t.device_ms = times[times.size() / 2];
    t.certified = (int)std::count(status.begin(), status.end(), PRISM_CERTIFIED);
    t.score = t.device_ms > 0 ? t.certified / (t.device_ms * 1e-3) : 0.0;
    return t;
}

// a candidate replaces the best schedule only if it certifies more accounts, or as many and
// is faster by more than the run-to-run spread of a trial's time (1%)
bool better(const Trial& a, const Trial& b) {
    if (a.certified != b.certified) return a.certified > b.certified;
    return a.score > b.score * 1.01;
}

}  // namespace
}  // namespace prism

extern "C" int prism_autotune(prism_universe* u, const prism_batch* b, const prism_solve_opts* base,
                              prism_solve_opts* tuned) {
    using namespace prism;
    if (!u || !b || !tuned) { set_error("NULL argument"); return PRISM_ERR_ARGUMENT; }
    prism_solve_opts o;
    if (base) o = *base; else prism_default_opts(&o);
    o.keep_for_backward = 0;
    o.profile = 0;
    if (o.precision == PRISM_PLAIN_FP32) { *tuned = o; return PRISM_OK; }   // nothing batched to tune
    const int M = b->n_accounts;
    if (M < 1 || !b->offsets) { set_error("empty book"); return PRISM_ERR_ARGUMENT; }
    int64_t nnz = 0;
    {
        cudaPointerAttributes at;
        const bool dev = cudaPointerGetAttributes(&at, b->offsets) == cudaSuccess &&
                         (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (dev) {
            if (cudaMemcpy(&nnz, b->offsets + M, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
                set_error("reading offsets failed");
                return PRISM_ERR_CUDA;
            }
        } else {
            nnz = b->offsets[M];
        }
    }
    const int S = u->u.S;
    int rc = PRISM_OK;
    constexpr int REPS = 3;
    // warm the caches and graphs of the universe handle once
    run_trial(u, b, o, nnz, M, S, 1, &rc);
    if (rc != PRISM_OK) return rc;
    prism_solve_opts best = o;
    Trial tb = run_trial(u, b, best, nnz, M, S, REPS, &rc);
    if (rc != PRISM_OK) return rc;
    auto consider = [&](prism_solve_opts cand) -> int {
        int r2 = PRISM_OK;
        const Trial tc = run_trial(u, b, cand, nnz, M, S, REPS, &r2);
        if (r2 != PRISM_OK) return r2;
        if (better(tc, tb)) { tb = tc; best = cand; }
        return PRISM_OK;
    };
    for (double rho0 : {0.5, 1.0, 2.0, 3.0, 5.0, 8.0}) {
        if (rho0 == o.rho0) continue;
        prism_solve_opts c = best;
        c.rho0 = rho0;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    for (double alpha : {1.4, 1.5, 1.6, 1.7, 1.8}) {
        if (alpha == best.alpha) continue;
        prism_solve_opts c = best;
        c.alpha = alpha;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    for (int ce : {5, 10, 20}) {
        if (ce == best.check_every) continue;
        prism_solve_opts c = best;
        c.check_every = ce;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    for (int sa : {2, 4, 6, 8, 10}) {
        if (sa == best.stream_after) continue;
        prism_solve_opts c = best;
        c.stream_after = sa;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    for (int ch : {1, 2, 4}) {
        if (ch == best.chains) continue;
        prism_solve_opts c = best;
        c.chains = ch;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    for (double eps : {1e-4, 2e-4, 3e-4, 5e-4, 7e-4}) {
        if (eps == best.eps_admm) continue;
        prism_solve_opts c = best;
        c.eps_admm = eps;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    for (int ae : {10, 15, 25, 50}) {
        if (ae == best.adapt_every || (ae == 25 && best.adapt_every == 0)) continue;
        prism_solve_opts c = best;
        c.adapt_every = ae;
        if ((rc = consider(c)) != PRISM_OK) return rc;
    }
    if (o.precision == PRISM_BATCHED_BF16) {
        // the tile shape of the tensor-core B'X: clusters of 8 CTAs per account tile (asset chunk)
        for (int gs : {1, 2, 3, 4, 6, 8}) {
            if (gs == best.g2_sets) continue;
            prism_solve_opts c = best;
            c.g2_sets = gs;
            if ((rc = consider(c)) != PRISM_OK) return rc;
        }
        // B'X of the pinned entries inside the fused x-update, the rest and Q in the roots kernel
        prism_solve_opts c = best;
        c.fold_products = 1 - best.fold_products;
        if ((rc = consider(c)) != PRISM_OK) return rc;
        // the fused x-update as persistent CTAs or one CTA per tile (unfolded products only)
        if (best.fold_products == 0) {
            prism_solve_opts c2 = best;
            c2.xupdate_form = 1 - best.xupdate_form;
            if ((rc = consider(c2)) != PRISM_OK) return rc;
        }
    }
    if (b->asset_idx) {
        // ragged accounts: dense-masked over the universe against packed per-account blocks
        for (int lay : {1, 2}) {
            if (lay == best.ragged_layout || (lay == 1 && best.ragged_layout == 0)) continue;
            prism_solve_opts c = best;
            c.ragged_layout = lay;
            if ((rc = consider(c)) != PRISM_OK) return rc;
        }
    }
    *tuned = best;
    tuned->keep_for_backward = base ? base->keep_for_backward : 0;
    tuned->profile = base ? base->profile : 0;
    return PRISM_OK;
}
