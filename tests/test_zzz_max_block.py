"""The largest block of right-hand sides (DL_MAX_RHS = 32 columns in one launch) through
noise, solve and contraction against the oracle, and the first size beyond it rejected."""
import numpy as np
import pytest

import synth
from oracle import loops, noise
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


def test_thirty_two_columns(dl):
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n = dl.DL_MAX_RHS
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
        dl.dl_set_params(ctx, kappa, amu)
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4(ctx, 2300, 0, n, eta, dl.DL_C128)
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=50000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F64, delta=0.0,
                                 flavour=1, chunk=8)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
        assert st == 0
        out = torch.zeros((n, dims[3], 1, 1, 4, 4), dtype=torch.complex128, device="cuda")
        dl.dl_contract(ctx, dl.DL_EST_STANDARD, eta, sol, n, dl.DL_C128, 0, 0, out)
        got_eta, got_sol, got = eta.cpu().numpy(), sol.cpu().numpy(), out.cpu().numpy()
        big = torch.empty((n + 1,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(dl.DLError):
            dl.dl_noise_z4(ctx, 2300, 0, n + 1, big, dl.DL_C128)
        with pytest.raises(dl.DLError):
            dl.dl_solve(ctx, big, big, n + 1, dl.DL_C128, prm)
    finally:
        dl.dl_destroy(ctx)
    for r in range(n):
        assert np.array_equal(got_eta[r], noise.z4_noise(dims, 2300, r)), r
        assert stats.resid[r] < 1e-10, r
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    for r in (0, 1, 13, 30, 31):
        s = (minv @ got_eta[r].ravel()).reshape(got_eta[r].shape)
        assert np.linalg.norm(got_sol[r] - s) / np.linalg.norm(s) < 1e-7, r
        ref = loops.project_momenta(loops.bilinear(got_eta[r], s), dims, 0)[:, 0]
        assert np.abs(got[r, :, 0, 0] - ref).max() < 1e-8 * np.abs(ref).max(), r
