"""GPU parity of the exact configuration the benchmark runs, on a small lattice.

The full-size TSM sweep (32^3 x 64) uses: 16-bit Krylov vectors for the LP solves
(tol 1e-2, FP32 accumulation), FP32 Krylov vectors with double-float reliable
updates every four decades for the HP solves (tol 1e-10), HP solves started from the
LP solution of the same noise, the HPE correction formed from s_HP - s_LP, blocks of
16 right-hand sides, momenta |n|^2 <= 9 and recon-12 links in both low precisions.
Its LP contractions run the FP32 fused bilinear + x-DFT kernel with the compile-time
x-momentum extent 3 (|n|^2 <= 9, no derivative).  These tests run exactly those
kernels and settings on lattices whose x extent (8) keeps the seven x momenta apart.

Tolerances: HP quantities within 1e-8 of loops from exact solutions (Sec. 2.2: HP
solves to 1e-10); LP loops (FP32 contraction of FP32/16-bit fields) within 1e-6 of
the FP64 oracle applied to the same low-precision solution, relative to the largest
element; Eq. estiTSM assembled from those within 2e-6.
"""
import numpy as np
import pytest

import synth
from oracle import lattice, loops, noise
from oracle import operator as op

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KAPPA, AMU = 0.1612, 0.0055  # the full-size workload's parameters
P2 = 9
BLOCK = 16


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as m
    m.lib()
    return m


def _ctx(dl, dims, links):
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
    dl.dl_set_params(ctx, KAPPA, AMU)
    return ctx


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _functional(est, links, e, s, hpe_ex):
    """The per-noise loop functional the library applies to any (possibly inexact)
    solution s of noise e: the estimator pairs of Eqs. loopSt, loopVv, loopStD and
    loopHPE1 with their factors; for the generalised estimator D_W s is evaluated as
    e - 2i kappa amu g5 s (equal to D_W s for the exact solution).  The HPE value
    includes the exact orders 0 and 2 (Eq. HPE, hpe_ex = loops.hpe_exact_c) at zero
    momentum on every time slice."""
    if est == "gen_one_end":
        xi, phi = loops.g5(s), loops.g5(e - 2j * KAPPA * AMU * loops.g5(s))
    else:
        xi, phi = loops.pair(est, links, e, s, KAPPA, AMU)
    dims = (links.shape[3], links.shape[2], links.shape[1], links.shape[0])
    f = loops.prefactor(est, KAPPA, AMU) * loops.project_momenta(loops.bilinear(xi, phi), dims, P2)
    if est == "hpe":
        ip0 = [tuple(p) for p in lattice.momenta(P2)].index((0, 0, 0))
        f[:, ip0] += dims[0] * dims[1] * dims[2] * hpe_ex
    return f


def _observables(links, e, s):
    """sigma loop (one-end, X = i g5) and isoscalar axial loop (generalised one-end,
    X = g_z g_5 = Gamma_11), zero momentum, summed over t: the per-noise observables
    dl_tsm_run returns as (Re, Im) pairs."""
    c1 = loops.bilinear(loops.g5(s), s)
    sig = loops.prefactor("one_end", KAPPA, AMU) * loops.loop_from_c(c1, 1j * lattice.GAMMA5).sum()
    c2 = loops.bilinear(loops.g5(s), loops.g5(e - 2j * KAPPA * AMU * loops.g5(s)))
    ax = loops.prefactor("gen_one_end", KAPPA, AMU) * loops.loop_from_c(c2, lattice.GAMMAS16[11]).sum()
    return np.array([sig.real, sig.imag, ax.real, ax.imag])


@pytest.mark.parametrize("est", ["standard", "one_end", "gen_one_end", "hpe"])
def test_fp32_contraction_p2max9_no_derivative(dl, est):
    """complex64 fields, no derivative, |n|^2 <= 9, recon-12 links, 16 columns: the
    FP32 fused contraction with x-momentum extent 3 (the kernel that produces every LP
    loop of the benchmark), element by element over [t][p][4][4]."""
    dims = (8, 8, 8, 4)
    links = synth.gauge_links(dims, 0.4, 301)
    n = 16
    eta = np.stack([noise.z4_noise(dims, 302, r) for r in range(n)]).astype(np.complex64)
    s = synth.gaussian_spinors(dims, n, 303).astype(np.complex64)
    ctx = _ctx(dl, dims, links)
    try:
        npm = len(dl.dl_momenta(P2))
        assert npm == 123
        out = torch.zeros((n, dims[3], npm, 1, 4, 4), dtype=torch.complex128, device="cuda")
        code = {"standard": 0, "one_end": 1, "gen_one_end": 2, "hpe": 3}[est]
        dl.dl_contract(ctx, code, torch.from_numpy(eta).cuda(), torch.from_numpy(s).cuda(), n, dl.DL_C64, 0, P2, out)
        got = out.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    tol = 2e-6 if est == "hpe" else 1e-6  # HPE: four FP32 stencil applications before the contraction
    for r in range(n):
        e, x = eta[r].astype(np.complex128), s[r].astype(np.complex128)
        if est == "gen_one_end":
            xi, phi = loops.g5(x), loops.g5(e - 2j * KAPPA * AMU * loops.g5(x))
        else:
            xi, phi = loops.pair(est, links, e, x, KAPPA, AMU)
        ref = loops.prefactor(est, KAPPA, AMU) * loops.project_momenta(loops.bilinear(xi, phi), dims, P2)
        assert _rel(got[r, :, :, 0], ref) < tol, (est, r, _rel(got[r, :, :, 0], ref))


def _lp_solutions(dl, ctx, dims, seed, first, n):
    """The LP map of the TSM for noise indices first .. first+n-1, in blocks of 16 as
    the TSM forms them: 16-bit Krylov vectors, FP32 accumulation, CG to 1e-2, no
    reliable updates.  Returns (eta, s) as complex128 arrays."""
    shape = (n,) + dims[::-1] + (4, 3)
    eta = torch.empty(shape, dtype=torch.complex64, device="cuda")
    dl.dl_noise_z4(ctx, seed, first, n, eta, dl.DL_C64)
    sol = torch.empty_like(eta)
    prm = dl.dl_solve_params(tol=1e-2, max_iter=200000, prec_hi=dl.DL_F32, prec_lo=dl.DL_F16, delta=0.0, flavour=1,
                             chunk=32)
    for b0 in range(0, n, BLOCK):
        m = min(BLOCK, n - b0)
        st, _ = dl.dl_solve(ctx, eta[b0:b0 + m], sol[b0:b0 + m], m, dl.DL_C64, prm)
        assert st == 0
    return eta.cpu().numpy().astype(np.complex128), sol.cpu().numpy().astype(np.complex128)


def test_tsm_benchmark_configuration(dl):
    """dl_tsm_run with the benchmark's parameters (17 HP pairs: a full block of 16 and
    a ragged block of 1; 21 fresh LP solves: 16 + 5) on 8 x 4 x 4 x 4.  HP per-noise
    observables against exact solutions (dense LU) within 1e-8; LP per-noise observables
    against the oracle functional of the GPU's own LP solutions (the same map, rerun
    through dl_solve) within 1e-6; the Eq. estiTSM loops of all three estimators
    element by element over [t][p][4][4] within 2e-6."""
    dims = (8, 4, 4, 4)  # every extent >= 4: the exact HPE orders hold in closed form
    links = synth.gauge_links(dims, 0.4, 311)
    n_hp, n_lp, seed = 17, 21, 2311
    ctx = _ctx(dl, dims, links)
    try:
        prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-10, tol_lp=1e-2, prec_hp_lo=dl.DL_F32,
                               prec_lp_lo=dl.DL_F16, delta_hp=1e-4, block=BLOCK, seed=seed, p2max=P2, with_deriv=0,
                               hpe=1, max_iter=200000, chunk=32, hp_guess=1, hpe_diff=1)
        npm = len(dl.dl_momenta(P2))
        out = np.zeros((3, dims[3], npm, 1, 4, 4), dtype=np.complex128)
        ohp, olpp, olp = np.zeros((n_hp, 4)), np.zeros((n_hp, 4)), np.zeros((n_lp, 4))
        st, info = dl.dl_tsm_run(ctx, prm, out, ohp, olpp, olp)
        assert st == 0 and info.not_converged == 0
        eta_p, s_lp_p = _lp_solutions(dl, ctx, dims, seed, 0, n_hp)
        eta_f, s_lp_f = _lp_solutions(dl, ctx, dims, seed, n_hp, n_lp)
    finally:
        dl.dl_destroy(ctx)
    for r in range(n_hp):
        assert np.array_equal(eta_p[r], noise.z4_noise(dims, seed, r).astype(np.complex64))
    # exact HP solutions of the same noise (dense LU of M_u)
    m = op.dense_matrix(links, KAPPA, AMU, 1)
    e_exact = np.stack([noise.z4_noise(dims, seed, r) for r in range(n_hp)])
    s_hp = np.linalg.solve(m, e_exact.reshape(n_hp, -1).T).T.reshape(e_exact.shape)
    # per-noise observables
    ref_hp = np.stack([_observables(links, e_exact[r], s_hp[r]) for r in range(n_hp)])
    ref_lpp = np.stack([_observables(links, e_exact[r], s_lp_p[r]) for r in range(n_hp)])
    ref_lp = np.stack([_observables(links, eta_f[r], s_lp_f[r]) for r in range(n_lp)])
    for k in (0, 2):  # sigma (real), axial (real); scale: the largest |value| of that observable
        scale = np.abs(ref_hp[:, k]).max()
        assert np.abs(ohp[:, k] - ref_hp[:, k]).max() < 1e-8 * scale, (k, np.abs(ohp[:, k] - ref_hp[:, k]).max() / scale)
        assert np.abs(olpp[:, k] - ref_lpp[:, k]).max() < 1e-6 * scale, k
        assert np.abs(olp[:, k] - ref_lp[:, k]).max() < 1e-6 * np.abs(ref_lp[:, k]).max(), k
    # the LP map really is truncated: its observables differ from the HP ones by far more than the tolerance
    assert np.abs(ref_lpp[:, 2] - ref_hp[:, 2]).max() > 1e-4 * np.abs(ref_hp[:, 2]).max()
    # Eq. estiTSM element by element for the three estimators of the sweep
    ex = loops.hpe_exact_c(links, KAPPA, AMU, (0, 0, 0, 0))
    for k, est in enumerate(("one_end", "gen_one_end", "hpe")):
        fh = [_functional(est, links, e_exact[r], s_hp[r], ex) for r in range(n_hp)]
        fp = [_functional(est, links, e_exact[r], s_lp_p[r], ex) for r in range(n_hp)]
        ff = [_functional(est, links, eta_f[r], s_lp_f[r], ex) for r in range(n_lp)]
        ref = loops.tsm_estimate(fh, fp, ff)
        assert _rel(out[k, :, :, 0], ref) < 2e-6, (est, _rel(out[k, :, :, 0], ref))
        # the HP-LP correction is far above that tolerance, so an error in the HP part would show
        corr_ref = (np.asarray(fh) - np.asarray(fp)).mean(axis=0)
        assert np.abs(corr_ref).max() > 1e-4 * np.abs(ref).max()


def test_tsm_hp_solve_from_lp_guess_after_drift(dl):
    """HP solves started from the LP solution with FP32 Krylov vectors on a gauge field where,
    before search directions were restarted on drift, one column's iterated residual ran far
    below the FP32 floor while it waited for a batched reliable update, the kept direction lost
    conjugacy and the solve diverged (reported as a breakdown the TSM ignored).  Now: status 0
    and HP observables within 1e-8 of exact solutions (dense LU) of the same noise."""
    dims = (8, 4, 4, 4)
    links = synth.gauge_links(dims, 0.4, 313)
    n_hp, n_lp, seed = 5, 1, 2313
    npm = len(dl.dl_momenta(P2))
    ctx = _ctx(dl, dims, links)
    try:
        prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-10, tol_lp=1e-2, prec_hp_lo=dl.DL_F32,
                               prec_lp_lo=dl.DL_F16, delta_hp=1e-4, block=BLOCK, seed=seed, p2max=P2, with_deriv=0,
                               hpe=1, max_iter=200000, chunk=8, hp_guess=1, hpe_diff=1)
        out = np.zeros((3, dims[3], npm, 1, 4, 4), dtype=np.complex128)
        ohp = np.zeros((n_hp, 4))
        st, info = dl.dl_tsm_run(ctx, prm, out, ohp, None, None)
    finally:
        dl.dl_destroy(ctx)
    assert st == 0 and info.not_converged == 0
    assert np.all(np.isfinite(out))
    m = op.dense_matrix(links, KAPPA, AMU, 1)
    e_exact = np.stack([noise.z4_noise(dims, seed, r) for r in range(n_hp)])
    s_hp = np.linalg.solve(m, e_exact.reshape(n_hp, -1).T).T.reshape(e_exact.shape)
    ref = np.stack([_observables(links, e_exact[r], s_hp[r]) for r in range(n_hp)])
    for k in (0, 2):
        scale = np.abs(ref[:, k]).max()
        assert np.abs(ohp[:, k] - ref[:, k]).max() < 1e-8 * scale, k


def test_tsm_autotuned_block(dl):
    """block = 0: the first call times LP blocks of 8, 16 and 32 right-hand sides and keeps
    the fastest per right-hand side; a second call reuses the choice without timing; both
    give bit for bit the loops and observables of a call with that block given explicitly."""
    dims = (8, 4, 4, 4)
    links = synth.gauge_links(dims, 0.4, 313)
    n_hp, n_lp, seed = 5, 9, 2313
    npm = len(dl.dl_momenta(P2))
    ctx = _ctx(dl, dims, links)
    res = []
    try:
        for blk in (0, 0, None):
            prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-10, tol_lp=1e-2, prec_hp_lo=dl.DL_F32,
                                   prec_lp_lo=dl.DL_F16, delta_hp=1e-4, block=res[0][1].block if blk is None else blk,
                                   seed=seed, p2max=P2, with_deriv=0, hpe=1, max_iter=200000, chunk=32, hp_guess=1,
                                   hpe_diff=1)
            out = np.zeros((3, dims[3], npm, 1, 4, 4), dtype=np.complex128)
            ohp, olp = np.zeros((n_hp, 4)), np.zeros((n_lp, 4))
            st, info = dl.dl_tsm_run(ctx, prm, out, ohp, None, olp)
            assert st == 0 and info.not_converged == 0
            res.append(((out, ohp, olp), info))
    finally:
        dl.dl_destroy(ctx)
    (a, ia), (b, ib), (c, ic) = res
    assert ia.block in (8, 16, 32) and ia.seconds_tune > 0.0
    assert ib.block == ia.block and ib.seconds_tune == 0.0
    assert ic.block == ia.block and ic.seconds_tune == 0.0
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, z) and np.array_equal(y, z)


def test_hp_loop_errors_per_gamma(dl):
    """The benchmark's HP map (FP32 Krylov vectors, double-float reliable updates every
    four decades, CG to 1e-10) for 12 noise vectors as one block on 4 x 4 x 4 x 8: the
    one-end and generalised one-end loops of all 16 Gamma, local and one-derivative,
    |n|^2 <= 4, each within 1e-8 of the loops of the exact solutions (dense LU) relative
    to the largest loop of the same Gamma and slot."""
    dims = (4, 4, 4, 8)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 321)
    n, p2 = 12, 4
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, kappa, amu)
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4(ctx, 322, 0, n, eta, dl.DL_C128)
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=200000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=1e-4,
                                 flavour=1, chunk=32)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
        assert st == 0
        npm = len(dl.dl_momenta(p2))
        got = {}
        for est, code in (("one_end", dl.DL_EST_ONE_END), ("gen_one_end", dl.DL_EST_GEN)):
            out = torch.zeros((n, dims[3], npm, 5, 4, 4), dtype=torch.complex128, device="cuda")
            dl.dl_contract(ctx, code, eta, sol, n, dl.DL_C128, 1, p2, out)
            got[est] = out.cpu().numpy()
        e_all = eta.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    m = op.dense_matrix(links, kappa, amu, 1)
    s_ex = np.linalg.solve(m, e_all.reshape(n, -1).T).T.reshape(e_all.shape)
    g16 = np.stack(lattice.GAMMAS16)
    for est in got:
        ref = np.empty_like(got[est])
        for r in range(n):
            xi, phi = loops.pair(est, links, e_all[r], s_ex[r], kappa, amu)
            pre = loops.prefactor(est, kappa, amu)
            ref[r, :, :, 0] = pre * loops.project_momenta(loops.bilinear(xi, phi), dims, p2)
            for mu in range(4):
                ref[r, :, :, 1 + mu] = pre * loops.project_momenta(loops.derivative_bilinear(links, xi, phi, mu), dims, p2)
        lg = np.einsum("gab,...ab->...g", g16, got[est])
        lr = np.einsum("gab,...ab->...g", g16, ref)
        err = np.abs(lg - lr).max(axis=(0, 1, 2))  # [slot][Gamma]
        scale = np.abs(lr).max(axis=(0, 1, 2))
        rel = err / np.maximum(scale, 1e-4 * scale.max())  # loops below 1e-4 of the largest: absolute
        assert rel.max() < 1e-8, (est, float(rel.max()), np.unravel_index(np.argmax(rel), rel.shape))
