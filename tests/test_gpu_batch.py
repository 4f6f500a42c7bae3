"""Several lattices in one batched solve (dl_batch_loops) against the oracle."""
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


def _loops_p0(est, links, eta, s, kappa, amu):
    xi, phi = loops.pair(est, links, eta, s, kappa, amu)
    return loops.prefactor(est, kappa, amu) * loops.bilinear(xi, phi).sum(axis=(1, 2, 3))  # [t][4][4]


@pytest.mark.parametrize("tile", [4, 0])
def test_batch_small_lattices_against_dense(dl, tile):
    """Three lattices (different sizes, links, kappa, a*mu), 5 noise vectors each
    (instances of 4 + 1 columns, or an autotuned tile), loops and solutions vs dense LU."""
    lat = [((4, 4, 4, 4), 0.3, 0.16, 0.01), ((4, 2, 4, 6), 0.4, 0.161, 0.0055), ((6, 4, 2, 4), 0.35, 0.158, 0.02)]
    n, seed = 5, 777
    links = [synth.gauge_links(d, eps, 300 + i) for i, (d, eps, _, _) in enumerate(lat)]
    ctx = dl.dl_create_multi([d for d, *_ in lat], 0, torch.cuda.current_stream())
    try:
        for i, (d, eps, kappa, amu) in enumerate(lat):
            dl.dl_load_gauge_lat(ctx, i, links[i], -1.0, 12, 12)
            dl.dl_set_params_lat(ctx, i, kappa, amu)
        sizes = [n * int(np.prod(d)) * 12 for d, *_ in lat]
        sol = torch.zeros(sum(sizes), dtype=torch.complex128, device="cuda")
        T = [d[3] for d, *_ in lat]
        out = np.zeros(sum(2 * n * t * 16 for t in T), dtype=np.complex128)
        prm = dl.dl_batch_params(n=n, tol=1e-11, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.1, seed=seed,
                                 max_iter=20000, tile=tile)
        st, info = dl.dl_batch_loops(ctx, prm, out, sol)
        assert st == 0
        assert info.tile in ((4,) if tile == 4 else (8, 16, 32))
        s_all = sol.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    lo = so = 0
    for i, (d, eps, kappa, amu) in enumerate(lat):
        Vd = int(np.prod(d))
        minv = np.linalg.inv(op.dense_matrix(links[i], kappa, amu, 1))
        got = out[lo:lo + 2 * n * d[3] * 16].reshape(2, n, d[3], 4, 4)
        sg = s_all[so:so + n * Vd * 12].reshape((n,) + d[::-1] + (4, 3))
        for r in range(n):
            eta = noise.z4_noise(d, seed, i * n + r)
            s = (minv @ eta.ravel()).reshape(eta.shape)
            assert np.linalg.norm(sg[r] - s) / np.linalg.norm(s) < 1e-8, (i, r)
            for k, est in enumerate(("one_end", "gen_one_end")):
                ref = _loops_p0(est, links[i], eta, s, kappa, amu)
                assert np.abs(got[k, r] - ref).max() < 1e-8 * np.abs(ref).max(), (i, r, est)
        lo += 2 * n * d[3] * 16
        so += n * Vd * 12


def test_batch_six_lattices_full_configuration(dl):
    """Two each of 12^3x24, 16^3x32, 24^3x48 (eps 0.4, kappa 0.161, a*mu 0.0055), 32 noise
    vectors per lattice, one batched solve to 1e-8 with an autotuned tile; residuals of sampled
    columns at sampled sites and loops at sampled t from the oracle."""
    dims = [(12, 12, 12, 24)] * 2 + [(16, 16, 16, 32)] * 2 + [(24, 24, 24, 48)] * 2
    kappa, amu, n, seed = 0.161, 0.0055, 32, 2004
    links = [synth.gauge_links(d, 0.4, 1004 + 10 * i) for i, d in enumerate(dims)]
    ctx = dl.dl_create_multi(dims, 0, torch.cuda.current_stream())
    try:
        for i in range(6):
            dl.dl_load_gauge_lat(ctx, i, links[i], -1.0, 12, 12)
        dl.dl_set_params(ctx, kappa, amu)
        sizes = [n * int(np.prod(d)) * 12 for d in dims]
        sol = torch.zeros(sum(sizes), dtype=torch.complex128, device="cuda")
        out = np.zeros(sum(2 * n * d[3] * 16 for d in dims), dtype=np.complex128)
        prm = dl.dl_batch_params(n=n, tol=1e-8, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.1, seed=seed,
                                 max_iter=20000, tile=0)
        st, info = dl.dl_batch_loops(ctx, prm, out, sol)
        assert st == 0 and info.not_converged == 0
        assert all(info.resid_max[i] < 1e-8 for i in range(6))
        offs = np.cumsum([0] + sizes)
        picks = {}
        for i in (0, 5):
            for r in (0, 31):
                picks[(i, r)] = sol[offs[i] + r * sizes[i] // n: offs[i] + (r + 1) * sizes[i] // n].cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    lo = np.cumsum([0] + [2 * n * d[3] * 16 for d in dims])
    rng = np.random.default_rng(5)
    for (i, r), flat in picks.items():
        d = dims[i]
        s = flat.reshape(d[::-1] + (4, 3))
        eta = noise.z4_noise(d, seed, i * n + r)
        for _ in range(12):
            site = tuple(int(rng.integers(0, k)) for k in d[::-1])
            res = op.apply_m_at(links[i], s, site, kappa, amu, 1) - eta[site]
            assert np.abs(res).max() < 1e-5, (i, r, site)
        got = out[lo[i]:lo[i + 1]].reshape(2, n, d[3], 4, 4)
        for t in (0, d[3] - 1):
            c1 = loops.bilinear(loops.g5(s[t]), s[t]).sum(axis=(0, 1, 2)) * loops.prefactor("one_end", kappa, amu)
            assert np.abs(got[0, r, t] - c1).max() < 1e-10 * np.abs(c1).max(), (i, r, t)
