"""GPU parity of time dilution (Sec. 2.3): time-diluted and coherent Z4 sources through
the C ABI against the oracle (bit-exact), and the loops of their solutions (standard and HPE
estimators) against dense-inverse loops within 1e-8."""
import numpy as np
import pytest

import synth
from oracle import lattice, loops, noise
from oracle import operator as op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("dims,n,cases", [((4, 4, 4, 4), 3, [(0, 4), (3, 4), (1, 2), (0, 1)]),
                                          ((6, 2, 4, 8), 5, [(5, 8), (1, 4), (0, 2), (2, 3)])])
def test_time_diluted_noise_bit_exact(dl, dims, n, cases):
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        out = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        out64 = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex64, device="cuda")
        full64 = torch.empty_like(out64)
        for t0, dt in cases:
            dl.dl_noise_z4_tdil(ctx, 2024, 7, n, out, t0, dt)
            got = out.cpu().numpy()
            for r in range(n):
                ref = noise.time_diluted(noise.z4_noise(dims, 2024, 7 + r), t0, dt)
                assert np.array_equal(got[r], ref), (t0, dt, r)
            # complex64 fields: the kept slices equal the undiluted complex64 noise, the rest is zero
            dl.dl_noise_z4_tdil(ctx, 2024, 7, n, out64, t0, dt, dl.DL_C64)
            dl.dl_noise_z4(ctx, 2024, 7, n, full64, dl.DL_C64)
            g64, f64 = out64.cpu().numpy(), full64.cpu().numpy()
            keep = (np.arange(dims[3]) % dt) == t0
            assert np.array_equal(g64[:, keep], f64[:, keep]) and not g64[:, ~keep].any(), (t0, dt)
        with pytest.raises(dl.DLError):
            dl.dl_noise_z4_tdil(ctx, 1, 0, n, out, 2, 2)
        with pytest.raises(dl.DLError):
            dl.dl_noise_z4_tdil(ctx, 1, 0, n, out, 0, dims[3] + 1)
    finally:
        dl.dl_destroy(ctx)


def test_time_diluted_loops_standard_and_hpe(dl):
    """4^4, kappa 0.16, amu 0.01: coherent sources on t = 1, 3 solved to CG residual 1e-10;
    standard loops (|n|^2 <= 1) and the HPE estimate (remainder + exact part on the kept
    slices, p = 0) against the dense inverse; loops of the other slices are exactly zero."""
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n, t0, dt, p2 = 4, 1, 2, 1
    npm = len(dl.dl_momenta(p2))
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
        dl.dl_set_params(ctx, kappa, amu)
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4_tdil(ctx, 2100, 0, n, eta, t0, dt)
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=50000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F64, delta=0.0,
                                 flavour=1, chunk=8)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
        assert st == 0
        std = torch.zeros((n, dims[3], npm, 1, 4, 4), dtype=torch.complex128, device="cuda")
        dl.dl_contract(ctx, dl.DL_EST_STANDARD, eta, sol, n, dl.DL_C128, 0, p2, std)
        hpe = torch.zeros((n, dims[3], 1, 1, 4, 4), dtype=torch.complex128, device="cuda")
        dl.dl_contract(ctx, dl.DL_EST_HPE, eta, sol, n, dl.DL_C128, 0, 0, hpe)
        exact_c = dl.dl_hpe_exact(ctx, 1)
        got_std, got_hpe = std.cpu().numpy(), hpe.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    keep = (np.arange(dims[3]) % dt) == t0
    assert not got_std[:, ~keep].any() and not got_hpe[:, ~keep].any()
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    n_space = dims[0] * dims[1] * dims[2]
    ex_ref = loops.hpe_exact_c(links, kappa, amu, (0, 0, 0, 0))
    assert np.abs(exact_c - ex_ref).max() < 1e-13
    for r in range(n):
        e = noise.time_diluted(noise.z4_noise(dims, 2100, r), t0, dt)
        s = (minv @ e.ravel()).reshape(e.shape)
        assert stats.resid[r] < 1e-10
        ref = loops.project_momenta(loops.bilinear(e, s), dims, p2)
        assert _rel(got_std[r, :, :, 0], ref) < 1e-8, (r, _rel(got_std[r, :, :, 0], ref))
        xi, phi = loops.pair("hpe", links, e, s, kappa, amu)
        ref_h = loops.project_momenta(loops.bilinear(xi, phi), dims, 0)[:, 0]
        ref_h[keep] += n_space * ex_ref
        est_h = got_hpe[r, :, 0, 0].copy()
        est_h[keep] += n_space * exact_c
        assert _rel(est_h, ref_h) < 1e-8, (r, _rel(est_h, ref_h))


@pytest.mark.parametrize("dtype_name,p2", [("c128", 1), ("c64", 9)])
@pytest.mark.parametrize("t0,dt", [(3, 8), (1, 2), (2, 3)])
def test_contract_slices_against_full_contraction(dl, dtype_name, p2, t0, dt):
    """dl_contract_slices on 8 x 4 x 4 x 8: the standard and HPE local loops of a
    time-diluted source equal dl_contract's on the kept slices t = t0 (mod dt) (the same
    arithmetic on fewer rows) and are zero on the others; dl_contract's own loops vanish
    there because the source does."""
    dims = (8, 4, 4, 8)
    links = synth.gauge_links(dims, 0.4, 2201)
    n = 5
    c128 = dtype_name == "c128"
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, 0.161, 0.0055)
        tdt = torch.complex128 if c128 else torch.complex64
        code = dl.DL_C128 if c128 else dl.DL_C64
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=tdt, device="cuda")
        dl.dl_noise_z4_tdil(ctx, 2202, 0, n, eta, t0, dt, code)
        sol = torch.from_numpy(synth.gaussian_spinors(dims, n, 2203)).to(tdt).cuda()
        npm = len(dl.dl_momenta(p2))
        for est in (dl.DL_EST_STANDARD, dl.DL_EST_HPE):
            full = torch.zeros((n, dims[3], npm, 1, 4, 4), dtype=torch.complex128, device="cuda")
            part = torch.full_like(full, float("nan"))
            dl.dl_contract(ctx, est, eta, sol, n, code, 0, p2, full)
            dl.dl_contract_slices(ctx, est, eta, sol, n, code, p2, t0, dt, part)
            f, g = full.cpu().numpy(), part.cpu().numpy()
            keep = (np.arange(dims[3]) % dt) == t0
            assert not g[:, ~keep].any() and not f[:, ~keep].any(), est
            assert np.abs(g[:, keep] - f[:, keep]).max() <= 1e-13 * np.abs(f).max(), est
        with pytest.raises(dl.DLError):
            dl.dl_contract_slices(ctx, dl.DL_EST_STANDARD, eta, sol, n, code, p2, dt, dt, part)
    finally:
        dl.dl_destroy(ctx)


@pytest.mark.parametrize("t0,dt", [(1, 2), (3, 4)])
def test_tsm_with_time_diluted_sources(dl, t0, dt):
    """dl_tsm_run with tdil_dt (Sec. 2.3 with the TSM, Eq. estiTSM) on 4^4, kappa 0.16,
    amu 0.01: HP solves to 1e-11 (FP32 Krylov, double-float reliable updates, started from
    the LP solution, HPE correction from the HP-LP difference), LP solves to 1e-5.  The
    standard and HPE loops equal the mean of the exact per-noise loops of the diluted
    sources (dense inverse, exact HPE part on the kept slices) up to the LP error, vanish
    exactly off the kept slices, and the HP per-noise observables are exact."""
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n_hp, n_lp, p2 = 3, 5, 1
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, kappa, amu)
        prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-11, tol_lp=1e-5, prec_hp_lo=dl.DL_F32,
                               prec_lp_lo=dl.DL_F32, delta_hp=1e-4, block=4, seed=2300, p2max=p2, with_deriv=0, hpe=1,
                               max_iter=50000, chunk=8, hp_guess=1, hpe_diff=1, tdil_dt=dt, tdil_t0=t0)
        npm = len(dl.dl_momenta(p2))
        out = np.zeros((2, dims[3], npm, 1, 4, 4), dtype=np.complex128)
        ohp = np.zeros((n_hp, 4))
        st, info = dl.dl_tsm_run(ctx, prm, out, ohp)
        assert st == 0 and info.n_est == 2
        bad = dl.dl_tsm_params(n_hp=1, n_lp=1, tol_hp=1e-10, tol_lp=1e-2, prec_hp_lo=dl.DL_F32, prec_lp_lo=dl.DL_F32,
                               delta_hp=1e-4, block=4, seed=1, p2max=0, with_deriv=1, hpe=0, max_iter=100, chunk=8,
                               tdil_dt=2, tdil_t0=0)
        with pytest.raises(dl.DLError):
            dl.dl_tsm_run(ctx, bad)
    finally:
        dl.dl_destroy(ctx)
    keep = (np.arange(dims[3]) % dt) == t0
    assert not out[:, ~keep].any()
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    ex = loops.hpe_exact_c(links, kappa, amu, (0, 0, 0, 0))
    ip0 = [tuple(p) for p in dl.dl_momenta(p2)].index((0, 0, 0))
    per = {"standard": [], "hpe": []}
    obs = []
    for r in range(n_hp + n_lp):
        e = noise.time_diluted(noise.z4_noise(dims, 2300, r), t0, dt)
        s = (minv @ e.ravel()).reshape(e.shape)
        for est in per:
            xi, phi = loops.pair(est, links, e, s, kappa, amu)
            f = loops.project_momenta(loops.bilinear(xi, phi), dims, p2)
            if est == "hpe":
                f[keep, ip0] += dims[0] * dims[1] * dims[2] * ex
            per[est].append(f)
        c = loops.project_momenta(loops.bilinear(e, s), dims, 0)[:, 0]  # [t][4][4] at p = 0
        obs.append((loops.loop_from_c(c, 1j * lattice.GAMMA5).sum(), loops.loop_from_c(c, lattice.GAMMAS16[11]).sum()))
    for k, est in enumerate(per):
        f = np.array(per[est])
        ref = loops.tsm_estimate(f[:n_hp], f[:n_hp], f[n_hp:])
        assert _rel(out[k, :, :, 0], ref) < 1e-4, est
    obs = np.array(obs)
    scale = np.abs(obs).max()
    assert np.abs(ohp[:, 0] + 1j * ohp[:, 1] - obs[:n_hp, 0]).max() < 1e-7 * scale
    assert np.abs(ohp[:, 2] + 1j * ohp[:, 3] - obs[:n_hp, 1]).max() < 1e-7 * scale
