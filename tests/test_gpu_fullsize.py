"""Full-size parity at 32^3 x 64 in the launch configuration bench.py times
(16-column blocks, 16-bit LP / FP32 + FP64 HP Krylov, recon-12 links), checked on
outputs the oracle computes one by one: whole noise fields for sampled columns,
the operator at sampled sites, solve residuals at sampled sites, and projected
loops for sampled (t, p)."""
import numpy as np
import pytest

import synth
from oracle import lattice, loops, noise
from oracle import operator as op

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (32, 32, 32, 64)
KAPPA, AMU = 0.1612, 0.0055
V = 32 * 32 * 32 * 64
SHAPE = (64, 32, 32, 32, 4, 3)


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as dl
    links = synth.gauge_links(DIMS, 0.4, 1002)
    ctx = dl.dl_create(DIMS, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
    dl.dl_set_params(ctx, KAPPA, AMU)
    state = {}
    yield dl, ctx, links, state
    dl.dl_destroy(ctx)


def _sites(k, seed):
    rng = np.random.default_rng(seed)
    out = [(0, 0, 0, 0), (63, 31, 31, 31), (63, 0, 5, 31), (0, 17, 31, 0)]
    while len(out) < k:
        out.append(tuple(int(rng.integers(0, n)) for n in (64, 32, 32, 32)))
    return out


def test_fullsize_noise_bit_exact(big):
    dl, ctx, links, state = big
    n = 16
    eta = torch.empty((n,) + SHAPE, dtype=torch.complex128, device="cuda")
    dl.dl_noise_z4(ctx, 2002, 0, n, eta, dl.DL_C128)
    for r in (0, 9, 15):
        assert np.array_equal(eta[r].cpu().numpy(), noise.z4_noise(DIMS, 2002, r))
    state["eta"] = eta


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6), (2, 3e-4)])
def test_fullsize_operator_sampled(big, prec, tol):
    dl, ctx, links, state = big
    n = 2
    x = synth.gaussian_spinors(DIMS, n, 404)
    xin = torch.from_numpy(x).cuda()
    out = torch.empty_like(xin)
    dl.dl_apply(ctx, dl.DL_OP_M, prec, 1, n, xin, None, out, dl.DL_C128)
    got = out.cpu().numpy()
    for r in range(n):
        for site in _sites(24, 7 + r):
            ref = op.apply_m_at(links, x[r], site, KAPPA, AMU, 1)
            assert np.abs(got[r][site] - ref).max() <= tol * max(np.abs(ref).max(), 1.0), (prec, r, site)


def test_fullsize_lp_and_hp_solves(big):
    """One 16-column block as the TSM runs it: LP (16-bit Krylov, 1e-2) and HP (FP32 Krylov,
    FP64 reliable updates, 1e-10); M psi = eta checked by the oracle at sampled sites."""
    dl, ctx, links, state = big
    eta = state.get("eta")
    if eta is None:
        pytest.skip("noise test did not run")
    n = 16
    sol = torch.empty_like(eta)
    lp = dl.dl_solve_params(tol=1e-2, max_iter=1000, prec_hi=dl.DL_F32, prec_lo=dl.DL_F16, delta=0.0, flavour=1,
                            chunk=0)
    st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, lp)
    assert st == 0
    assert all(stats.resid[i] < 1e-2 for i in range(n))
    assert all(stats.true_resid[i] < 5e-2 for i in range(n))
    hp = dl.dl_solve_params(tol=1e-10, max_iter=5000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.1, flavour=1,
                            chunk=0)
    st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, hp)
    assert st == 0
    assert all(stats.resid[i] < 1e-10 for i in range(n))
    assert all(stats.true_resid[i] < 1e-8 for i in range(n))
    s_np = sol[:2].cpu().numpy()
    e_np = eta[:2].cpu().numpy()
    for r in range(2):
        for site in _sites(16, 31 + r):
            res = op.apply_m_at(links, s_np[r], site, KAPPA, AMU, 1) - e_np[r][site]
            assert np.abs(res).max() < 1e-8, (r, site)
    state["sol"] = sol


def test_fullsize_contraction_sampled(big):
    """One-end and generalised loops at |p|^2 <= 9 for sampled (t, p) against the oracle's
    direct sum over the time slice."""
    dl, ctx, links, state = big
    sol, eta = state.get("sol"), state.get("eta")
    if sol is None:
        pytest.skip("solve test did not run")
    n = 2
    npm = len(dl.dl_momenta(9))
    plist = lattice.momenta(9)
    for est, code in (("one_end", dl.DL_EST_ONE_END), ("gen_one_end", dl.DL_EST_GEN)):
        out = torch.zeros((n, 64, npm, 1, 4, 4), dtype=torch.complex128, device="cuda")
        dl.dl_contract(ctx, code, eta[:n].contiguous(), sol[:n].contiguous(), n, dl.DL_C128, 0, 9, out)
        got = out.cpu().numpy()
        s_np = sol[:n].cpu().numpy()
        e_np = eta[:n].cpu().numpy()
        pre = loops.prefactor(est, KAPPA, AMU)
        z, y, x = np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij")
        for r in range(n):
            for t in (0, 31, 63):
                xi = loops.g5(s_np[r][t])
                if est == "one_end":
                    phi = s_np[r][t]
                else:  # g5 D_W s with D_W = M at amu = 0, site by site (Eq. loopStD)
                    dw = np.empty((32, 32, 32, 4, 3), dtype=np.complex128)
                    for zz in range(32):
                        for yy in range(32):
                            for xx in range(32):
                                dw[zz, yy, xx] = op.apply_m_at(links, s_np[r], (t, zz, yy, xx), KAPPA, 0.0, 1)
                    phi = loops.g5(dw)
                c = loops.bilinear(xi, phi)  # [z][y][x][4][4]
                for ip in (0, 7, 61, 122):
                    nx, ny, nz = plist[ip]
                    ph = np.exp(-2j * np.pi * (nx * x + ny * y + nz * z) / 32)
                    ref = pre * np.einsum("zyx,zyxab->ab", ph, c)
                    tol = 1e-10 if est == "one_end" else 1e-8  # the GPU uses D_W s = eta - 2i k amu g5 s
                    assert np.abs(got[r, t, ip, 0] - ref).max() < tol * max(np.abs(ref).max(), 1.0), (est, r, t, ip)
