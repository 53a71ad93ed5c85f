"""GPU adjoint (prism_solve_batch_backward): gradients of L = sum_a g_a'w_a with respect to
(mu, B, d, w0) against the oracle-side adjoint (FP64 CPU, its own KKT solve on the oracle's
active set), against central differences of the GPU solve itself, and the torch.autograd
wrapper against the C-ABI call.

Tolerance: 1e-6 relative to the largest magnitude of each gradient (both sides solve the same
FP64 linear system on the same active set; the weights they start from agree to 1e-6 or better).
"""
import numpy as np
import pytest

from oracle import adjoint
from oracle.active_set import account_problem
from paper_2606_23367_gb300 import build, prism
from paper_2606_23367_gb300.workloads import make_workload
from tests.oracle_pool import adjoint_all

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6

SMALL = {
    "bands": dict(N=300, K=8, M=6, S=4, band_hi=0.3, upper=(0.05, 0.1), held=(40, 80)),
    "cap": dict(N=300, K=8, M=6, S=4, band_hi=0.35, upper=(0.05, 0.1), held=(40, 80), tau=0.8),
    "lots_cap": dict(N=300, K=8, M=6, S=4, band_hi=0.35, upper=(0.05, 0.1), held=(40, 80), tau=0.9,
                     lots=True, restrict=0.05),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    prism.load_library()


def oracle_grads(uni, batch, accounts, g):
    N, K = uni.B.shape
    dmu, dB, dd = np.zeros(N), np.zeros((N, K)), np.zeros(N)
    dw0 = np.zeros(int(batch.offsets[-1]))
    for a in accounts:
        prob = account_problem(uni, batch, a)
        res = prob.solve()
        sl = batch.account_slice(a)
        idx = batch.account_assets(a, N)
        m, b, d_, w0g = adjoint.account_gradients(prob, res, g[sl])
        dmu[idx] += m
        dB[idx] += b
        dd[idx] += d_
        dw0[sl] = w0g
    return dict(dmu=dmu, dB=dB, dd=dd, dw0=dw0)


def assert_close(got, ref, what):
    scale = max(float(np.max(np.abs(ref))), 1e-12)
    err = float(np.max(np.abs(got - ref))) / scale
    assert err <= GRAD_TOL, (what, err, scale)


@pytest.mark.parametrize("mode", [prism.PRISM_BATCHED_FP32, prism.PRISM_BATCHED_BF16])
@pytest.mark.parametrize("family", sorted(SMALL))
def test_backward_matches_oracle_adjoint(family, mode):
    uni, batch = make_workload(4, **SMALL[family])
    h = prism.create_universe(uni)
    res = prism.solve(h, batch, precision=mode, keep_for_backward=1)
    assert np.all(res["status"] == prism.PRISM_CERTIFIED), res["status"]
    g = np.random.default_rng(5).normal(size=int(batch.offsets[-1]))
    got = prism.prism_solve_batch_backward(res["state"], g)
    ref = oracle_grads(uni, batch, range(batch.n_accounts), g)
    for k in ("dmu", "dB", "dd", "dw0"):
        assert_close(got[k], ref[k], k)
    # a second backward on the same state gives the same numbers (scratch reuse)
    again = prism.prism_solve_batch_backward(res["state"], g)
    for k in ("dmu", "dB", "dd", "dw0"):
        assert np.array_equal(again[k], got[k]), k


def test_backward_full_size_every_account():
    # the differentiation workload at its full size (128 accounts x 2,000 assets, K = 32), the
    # loss weighting every account; the oracle adjoint of each account runs in a host pool
    uni, batch = make_workload(4)
    h = prism.create_universe(uni)
    res = prism.solve(h, batch, precision=prism.PRISM_BATCHED_BF16, keep_for_backward=1)
    assert np.all(res["status"] == prism.PRISM_CERTIFIED), res["status"]
    g = np.random.default_rng(11).normal(size=int(batch.offsets[-1]))
    got = prism.prism_solve_batch_backward(res["state"], g)
    ref = adjoint_all(4, g)
    for k in ("dmu", "dB", "dd", "dw0"):
        assert_close(got[k], ref[k], k)


def _classes(w, batch):
    """Which bound or kink each weight sits on (0 lower, 1 upper, 2 at w0, 3 elsewhere)."""
    c = np.full(w.shape, 3)
    c[np.abs(w - batch.w0) <= 1e-13] = 2
    c[np.abs(w - batch.upper) <= 1e-13] = 1
    c[np.abs(w - batch.lower) <= 1e-13] = 0
    return c


N_DIRECTIONS = 20


@pytest.mark.parametrize("family", ["bands", "cap"])
def test_backward_matches_central_differences_of_the_gpu_solve(family):
    # FP64 central differences (h = 1e-6) of L = g'w along 20 seeded directions that move mu, B, d
    # and the held names' w0 together, each through a full GPU solve of the perturbed problem;
    # a direction whose perturbed solves leave the base active set is not comparable and skipped
    import dataclasses
    uni, batch = make_workload(4, **SMALL[family])
    h = prism.create_universe(uni)
    res = prism.solve(h, batch, precision=prism.PRISM_BATCHED_FP32, keep_for_backward=1)
    g = np.random.default_rng(9).normal(size=int(batch.offsets[-1]))
    got = prism.prism_solve_batch_backward(res["state"], g)
    base_cls = _classes(res["w"], batch)
    rng = np.random.default_rng(21)
    step = 1e-6
    kept, errs = 0, []
    for _ in range(N_DIRECTIONS):
        vmu = rng.normal(size=uni.mu.shape) * 0.02
        vd = rng.normal(size=uni.d.shape) * 0.01
        vB = rng.normal(size=uni.B.shape) * 0.3
        vw0 = rng.normal(size=batch.w0.shape) * 0.01 * (batch.w0 > 0)
        ad = float(got["dmu"] @ vmu + got["dd"] @ vd + np.sum(got["dB"] * vB) + got["dw0"] @ vw0)
        # the size of the directional derivative's terms: the GPU's polished weights carry
        # ~1e-14 of rounding, which h = 1e-6 turns into ~1e-8 of noise in the difference
        # quotient, so a derivative that cancels to far below its terms is compared at their scale
        terms = float(np.abs(got["dmu"] * vmu).sum() + np.abs(got["dd"] * vd).sum() +
                      np.abs(got["dB"] * vB).sum() + np.abs(got["dw0"] * vw0).sum())
        ws = []
        for sgn in (1.0, -1.0):
            u2 = type(uni)(B=uni.B + sgn * step * vB, f=uni.f, d=uni.d + sgn * step * vd,
                           mu=uni.mu + sgn * step * vmu, sector=uni.sector, n_sectors=uni.n_sectors)
            b2 = dataclasses.replace(batch, w0=batch.w0 + sgn * step * vw0)
            h2 = prism.create_universe(u2)
            r2 = prism.solve(h2, b2, precision=prism.PRISM_BATCHED_FP32)
            h2.close()
            ws.append((r2, b2))
        if not all(np.all(r["status"] == prism.PRISM_CERTIFIED) for r, _ in ws):
            continue
        if not all(np.array_equal(_classes(r["w"], b2), base_cls) for r, b2 in ws):
            continue
        fd = float(g @ (ws[0][0]["w"] - ws[1][0]["w"])) / (2 * step)
        scale = max(abs(ad), terms, 1e-3)
        errs.append(abs(fd - ad) / scale)
        assert abs(fd - ad) <= 1e-6 * scale, (fd, ad, terms)
        kept += 1
    print(f"{family}: {kept} of {N_DIRECTIONS} directions compared, worst relative gap {max(errs):.1e}")
    assert kept >= 15


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_function_matches_the_c_abi(device):
    # the torch.autograd wrapper against the C-ABI calls: host tensors, or CUDA tensors that stay
    # on the device (the solve on the current stream, weights and gradients in device tensors);
    # a second forward with the same tensors reuses the wrapper's universe handle
    torch = pytest.importorskip("torch")
    from paper_2606_23367_gb300 import autograd as pag
    uni, batch = make_workload(4, **SMALL["bands"])
    g = np.random.default_rng(3).normal(size=int(batch.offsets[-1]))
    t = lambda x: torch.tensor(x, dtype=torch.float64, device=device, requires_grad=True)
    mu, B, d, w0 = t(uni.mu), t(uni.B), t(uni.d), t(batch.w0)
    spec = dict(f=uni.f, sector=uni.sector, n_sectors=uni.n_sectors, offsets=batch.offsets, lower=batch.lower,
                upper=batch.upper, tc=batch.tc, band_lo=batch.band_lo, band_hi=batch.band_hi,
                precision=prism.PRISM_BATCHED_FP32)
    w = pag.solve(mu, B, d, w0, **spec)
    assert w.device.type == device
    (w * torch.tensor(g, dtype=torch.float64, device=device)).sum().backward()
    n_cached = len(pag._UNIVERSES)
    w_again = pag.solve(mu, B, d, w0, **spec)
    assert len(pag._UNIVERSES) == n_cached
    h = prism.create_universe(uni)
    res = prism.solve(h, batch, precision=prism.PRISM_BATCHED_FP32, keep_for_backward=1)
    ref = prism.prism_solve_batch_backward(res["state"], g)
    c = lambda x: x.detach().cpu().numpy()
    assert np.allclose(c(w), res["w"], rtol=0, atol=1e-14)
    assert np.allclose(c(w_again), res["w"], rtol=0, atol=1e-14)
    assert mu.grad.device.type == device
    assert np.allclose(c(mu.grad), ref["dmu"], rtol=1e-12, atol=1e-12)
    assert np.allclose(c(B.grad), ref["dB"], rtol=1e-12, atol=1e-12)
    assert np.allclose(c(d.grad), ref["dd"], rtol=1e-12, atol=1e-12)
    assert np.allclose(c(w0.grad), ref["dw0"], rtol=1e-12, atol=1e-12)
