"""GPU checks of the solver's non-fatal outcomes, with the failures made on the host: a
source holding NaN or Inf is reported as DL_BREAKDOWN for its column (NaN residual) while
the other columns of the batch converge; an iteration limit below what the tolerance needs
returns DL_NOT_CONVERGED with the last iterate and its residual."""
import numpy as np
import pytest

import synth
from oracle import noise
from oracle import operator as op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as m
    m.lib()
    return m


DIMS = (4, 4, 4, 4)
KAPPA, AMU = 0.16, 0.01


def _ctx(dl, links):
    ctx = dl.dl_create(DIMS, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
    dl.dl_set_params(ctx, KAPPA, AMU)
    return ctx


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_source_is_a_breakdown(dl, bad):
    links = synth.gauge_links(DIMS, 0.3, 1000)
    eta = np.stack([noise.z4_noise(DIMS, 2200, r) for r in range(3)])
    eta[1, 2, 1, 0, 3, 2, 1] = bad
    ctx = _ctx(dl, links)
    try:
        src = torch.from_numpy(eta).cuda()
        sol = torch.empty_like(src)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=50000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.1,
                                 flavour=1, chunk=8)
        st, stats = dl.dl_solve(ctx, src, sol, 3, dl.DL_C128, prm)
        got = sol.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    assert st == dl.DL_BREAKDOWN
    assert np.isnan(stats.resid[1])
    for r in (0, 2):
        assert stats.resid[r] < 1e-10
        res = op.apply_m(links, got[r], KAPPA, AMU) - eta[r]
        assert np.linalg.norm(res) / np.linalg.norm(eta[r]) < 1e-7


def test_iteration_limit_returns_last_iterate(dl):
    links = synth.gauge_links(DIMS, 0.3, 1000)
    eta = np.stack([noise.z4_noise(DIMS, 2201, r) for r in range(2)])
    ctx = _ctx(dl, links)
    try:
        src = torch.from_numpy(eta).cuda()
        sol = torch.empty_like(src)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=5, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.1,
                                 flavour=1, chunk=8)
        st, stats = dl.dl_solve(ctx, src, sol, 2, dl.DL_C128, prm)
        got = sol.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    assert st == dl.DL_NOT_CONVERGED
    for r in range(2):
        assert 1 <= stats.iters[r] <= 5
        assert np.isfinite(stats.resid[r]) and stats.resid[r] > 1e-10
        assert np.isfinite(got[r]).all() and np.abs(got[r]).max() > 0
        # the last iterate is returned: its true residual is the one the stats report
        res = op.apply_m(links, got[r], KAPPA, AMU) - eta[r]
        assert abs(np.linalg.norm(res) / np.linalg.norm(eta[r]) - stats.true_resid[r]) < 1e-6


def test_repeated_solve_and_contraction_are_bitwise_equal(dl):
    """No floating-point atomics: the same solve (16-bit Krylov vectors, reliable updates) and
    contraction on the same inputs give the same bits, the second time from the cached graph
    (4^3 x 8, kappa 0.161, a*mu 0.0055, five noise vectors to 1e-10)."""
    dims = (4, 4, 4, 8)
    links = synth.gauge_links(dims, 0.4, 41)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
        dl.dl_set_params(ctx, 0.161, 0.0055)
        eta = torch.empty((5,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4(ctx, 7, 0, 5, eta, dl.DL_C128)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=100000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F16, delta=0.1,
                                 flavour=1, chunk=16)
        runs = []
        for _ in range(2):
            sol = torch.empty_like(eta)
            st, stats = dl.dl_solve(ctx, eta, sol, 5, dl.DL_C128, prm)
            assert st == 0
            out = torch.zeros((5, dims[3], 1, 1, 4, 4), dtype=torch.complex128, device="cuda")
            dl.dl_contract(ctx, dl.DL_EST_ONE_END, eta, sol, 5, dl.DL_C128, 0, 0, out)
            runs.append((sol.cpu().numpy(), out.cpu().numpy(), list(stats.iters[:5])))
    finally:
        dl.dl_destroy(ctx)
    assert runs[0][2] == runs[1][2]
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
