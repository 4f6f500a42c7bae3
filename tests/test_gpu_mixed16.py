"""The mixed-precision batched workload on 16^3 x 32 (eps 0.4, kappa 0.161, a*mu 0.0055):
12 Z4 noise vectors solved as one block to 1e-10 with 16-bit or FP32 Krylov vectors and
FP64 reliable updates, then one-end loops for the 16 local Gamma and the four
covariant-derivative directions at |n|^2 <= 4 (33 momenta).  The oracle checks M psi = eta
at sampled sites and recomputes every loop of two columns from the GPU's solution."""
import numpy as np
import pytest

import synth
from oracle import lattice, loops
from oracle import operator as op

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (16, 16, 16, 32)
KAPPA, AMU = 0.161, 0.0055
V = 16 * 16 * 16 * 32
SHAPE = (32, 16, 16, 16, 4, 3)


@pytest.fixture(scope="module")
def lat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as dl
    links = synth.gauge_links(DIMS, 0.4, 1001)
    ctx = dl.dl_create(DIMS, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
    dl.dl_set_params(ctx, KAPPA, AMU)
    yield dl, ctx, links
    dl.dl_destroy(ctx)


@pytest.mark.parametrize("lo", ["f16", "f32"])
def test_block_of_12_solves_and_derivative_loops(lat, lo):
    dl, ctx, links = lat
    n = 12
    eta = torch.empty((n,) + SHAPE, dtype=torch.complex128, device="cuda")
    dl.dl_noise_z4(ctx, 2001, 0, n, eta, dl.DL_C128)
    sol = torch.empty_like(eta)
    prm = dl.dl_solve_params(tol=1e-10, max_iter=20000, prec_hi=dl.DL_F64,
                             prec_lo=dl.DL_F16 if lo == "f16" else dl.DL_F32, delta=0.01, flavour=1, chunk=0)
    st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
    assert st == 0, dl.dl_last_error(ctx)
    assert all(stats.resid[i] < 1e-10 for i in range(n))
    assert all(stats.true_resid[i] < 1e-8 for i in range(n))
    npm = len(dl.dl_momenta(4))
    assert npm == 33
    out = torch.zeros((n, DIMS[3], npm, 5, 4, 4), dtype=torch.complex128, device="cuda")
    dl.dl_contract(ctx, dl.DL_EST_ONE_END, eta, sol, n, dl.DL_C128, 1, 4, out)
    got = out.cpu().numpy()
    rng = np.random.default_rng(3)
    pre = loops.prefactor("one_end", KAPPA, AMU)
    for r in (0, n - 1):
        s = sol[r].cpu().numpy()
        e = eta[r].cpu().numpy()
        for _ in range(8):
            site = tuple(int(rng.integers(0, k)) for k in SHAPE[:4])
            res = op.apply_m_at(links, s, site, KAPPA, AMU, 1) - e[site]
            assert np.abs(res).max() < 1e-8, (r, site)
        xi, phi = loops.pair("one_end", links, e, s, KAPPA, AMU)
        ref = [pre * loops.project_momenta(loops.bilinear(xi, phi), DIMS, 4)]
        for mu in range(4):
            ref.append(pre * loops.project_momenta(loops.derivative_bilinear(links, xi, phi, mu), DIMS, 4))
        for d in range(5):
            a = got[r, :, :, d]
            b = ref[d]
            assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), (r, d)
    assert [tuple(p) for p in dl.dl_momenta(4)] == [tuple(p) for p in lattice.momenta(4)]
