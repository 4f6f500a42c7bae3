"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: FP64 operators <= 1e-13 relative, FP32 <= 2e-6 (the target bounds of
this path), 16-bit storage <= 3e-4 (int16 fixed point with a
per-site scale); noise and indexing bit-exact; loops from solves converged to CG residual
1e-10 within 1e-8 of the dense-inverse loops.
"""
import numpy as np
import pytest

import synth
from oracle import loops, noise, solver
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


def _ctx(dl, dims, links, kappa, amu, r32=12, r16=8):
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, r32, r16)
    dl.dl_set_params(ctx, kappa, amu)
    return ctx


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 4), 3), ((6, 2, 4, 8), 5), ((8, 8, 8, 8), 16)])
def test_noise_bit_exact(dl, dims, n):
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        out = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4(ctx, 2024, 7, n, out, dl.DL_C128)
        got = out.cpu().numpy()
        for r in range(n):
            assert np.array_equal(got[r], noise.z4_noise(dims, 2024, 7 + r)), r
        dl.dl_noise_z4(ctx, 99, 0, n, out, dl.DL_C128, 1)
        got = out.cpu().numpy()
        for r in range(n):
            assert np.array_equal(got[r], noise.z4_noise(dims, 99, r, quadrant=True))
    finally:
        dl.dl_destroy(ctx)


OPS = ["M", "MDAG", "HOP", "MHAT", "MHAT_DAG", "PREP", "RECON", "BH"]


def _oracle_op(name, links, x, aux, kappa, amu, f, dims):
    if name == "M":
        return op.apply_m(links, x, kappa, amu, f)
    if name == "MDAG":
        return op.apply_m_dag(links, x, kappa, amu, f)
    if name == "HOP":
        return op.hop(links, x)
    if name == "MHAT":
        return op.mhat(links, op.project(x, dims, 0), kappa, amu, f, -1.0, dims)
    if name == "MHAT_DAG":
        return op.mhat_dag(links, op.project(x, dims, 0), kappa, amu, f, -1.0, dims)
    if name == "PREP":
        return op.prep_source(links, x, kappa, amu, f, -1.0, dims)
    if name == "RECON":
        xe = op.project(x, dims, 0)
        return xe + op.reconstruct_odd(links, xe, aux, kappa, amu, f, -1.0, dims)
    if name == "BH":
        return loops.bh_apply(links, x, kappa, amu, -1.0, f)
    raise ValueError(name)


@pytest.fixture(scope="module")
def opcase():
    dims = (4, 6, 4, 8)
    links = synth.gauge_links(dims, 0.4, 31)
    x = synth.gaussian_spinors(dims, 3, 32)
    aux = synth.gaussian_spinors(dims, 3, 33)
    return dims, links, x, aux


@pytest.mark.parametrize("name", OPS)
@pytest.mark.parametrize("f", [1, -1])
def test_operator_f64(dl, opcase, name, f):
    dims, links, x, aux = opcase
    kappa, amu = 0.161, 0.0055
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        xin, ain = _dev(x), _dev(aux)
        out = torch.empty_like(xin)
        dl.dl_apply(ctx, getattr(dl, "DL_OP_" + name), dl.DL_F64, f, 3, xin, ain, out, dl.DL_C128)
        got = out.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    for r in range(3):
        ref = _oracle_op(name, links, x[r], aux[r], kappa, amu, f, dims)
        assert _rel(got[r], ref) < 1e-13, (name, r, _rel(got[r], ref))


@pytest.mark.parametrize("name", ["M", "MHAT", "MHAT_DAG", "RECON", "BH"])
@pytest.mark.parametrize("prec,recon,tol", [(1, 12, 2e-6), (1, 8, 2e-6), (2, 12, 3e-4), (2, 8, 3e-4)])
def test_operator_low_precision(dl, opcase, name, prec, recon, tol):
    dims, links, x, aux = opcase
    kappa, amu = 0.161, 0.0055
    ctx = _ctx(dl, dims, links, kappa, amu, r32=recon if prec == 1 else 12, r16=recon if prec == 2 else 8)
    try:
        xin, ain = _dev(x), _dev(aux)
        out = torch.empty_like(xin)
        dl.dl_apply(ctx, getattr(dl, "DL_OP_" + name), prec, 1, 3, xin, ain, out, dl.DL_C128)
        got = out.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    for r in range(3):
        ref = _oracle_op(name, links, x[r], aux[r], kappa, amu, 1, dims)
        err = np.linalg.norm(got[r] - ref) / np.linalg.norm(ref)
        assert err < tol, (name, prec, recon, err)


def test_solve_and_loops_tiny_config(dl):
    """4^4, eps 0.3, kappa 0.16, amu 0.01, 8 Z4 noise vectors, CG to 1e-10:
    the 16 local Gamma loops per time slice at p = 0 against dense exact inversion."""
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n = 8
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4(ctx, 2000, 0, n, eta, dl.DL_C128)
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=50000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F64, delta=0.0,
                                 flavour=1, chunk=8)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
        assert st == 0
        out = torch.zeros((n, dims[3], 1, 1, 4, 4), dtype=torch.complex128, device="cuda")
        dl.dl_contract(ctx, dl.DL_EST_STANDARD, eta, sol, n, dl.DL_C128, 0, 0, out)
        got = out.cpu().numpy()
        s_got = sol.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    for r in range(n):
        e = noise.z4_noise(dims, 2000, r)
        s = (minv @ e.ravel()).reshape(e.shape)
        assert stats.resid[r] < 1e-10
        ref = loops.project_momenta(loops.bilinear(e, s), dims, 0)[:, 0]
        assert _rel(got[r, :, 0, 0], ref) < 1e-8, (r, _rel(got[r, :, 0, 0], ref))
        # the 16 Gamma loops per t (sum_ab Gamma_ab C_ab)
        from oracle import lattice
        for b in range(16):
            lg = np.einsum("ab,tab->t", lattice.GAMMAS16[b], got[r, :, 0, 0])
            lr = np.einsum("ab,tab->t", lattice.GAMMAS16[b], ref)
            assert np.abs(lg - lr).max() < 1e-8 * np.abs(ref).max()
        assert stats.true_resid[r] < 1e-7
        assert np.linalg.norm(s_got[r] - s) / np.linalg.norm(s) < 1e-7


@pytest.mark.parametrize("lo,delta", [(1, 0.1), (2, 0.1)])
def test_mixed_precision_solve(dl, lo, delta):
    """FP32 / 16-bit Krylov vectors with FP64 reliable updates reach 1e-10."""
    dims = (4, 4, 4, 8)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 41)
    n = 5
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex128, device="cuda")
        dl.dl_noise_z4(ctx, 7, 0, n, eta, dl.DL_C128)
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=1e-10, max_iter=100000, prec_hi=dl.DL_F64, prec_lo=lo, delta=delta, flavour=1,
                                 chunk=16)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
        assert st == 0
        s_got = sol.cpu().numpy()
        e_all = eta.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    for r in range(n):
        assert stats.resid[r] < 1e-10
        x = solver.solve_dense(links, e_all[r], kappa, amu)
        assert np.linalg.norm(s_got[r] - x) / np.linalg.norm(x) < 1e-6
    assert stats.reliable_updates > 0


@pytest.mark.parametrize("est", ["standard", "one_end", "gen_one_end", "hpe"])
def test_contractions_with_momenta(dl, est):
    """Bilinears, derivative bilinears and momentum projection against the oracle,
    for s = M_u^-1 eta exactly (the generalised estimator uses D_W s = eta - 2 i k amu g5 s)."""
    dims = (4, 6, 2, 4)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 51)
    n = 3
    eta = np.stack([noise.z4_noise(dims, 52, r) for r in range(n)])
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    s = np.stack([(minv @ e.ravel()).reshape(e.shape) for e in eta])
    with_deriv = 0 if est == "hpe" else 1
    p2 = 4
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        nd = 5 if with_deriv else 1
        npm = len(dl.dl_momenta(p2))
        out = torch.zeros((n, dims[3], npm, nd, 4, 4), dtype=torch.complex128, device="cuda")
        code = {"standard": 0, "one_end": 1, "gen_one_end": 2, "hpe": 3}[est]
        dl.dl_contract(ctx, code, _dev(eta), _dev(s), n, dl.DL_C128, with_deriv, p2, out)
        got = out.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    pre = loops.prefactor(est, kappa, amu)
    for r in range(n):
        xi, phi = loops.pair(est, links, eta[r], s[r], kappa, amu)
        ref = pre * loops.project_momenta(loops.bilinear(xi, phi), dims, p2)
        assert _rel(got[r, :, :, 0], ref) < 1e-11, (est, r, _rel(got[r, :, :, 0], ref))
        if with_deriv:
            for mu in range(4):
                refd = pre * loops.project_momenta(loops.derivative_bilinear(links, xi, phi, mu), dims, p2)
                assert _rel(got[r, :, :, 1 + mu], refd) < 1e-11, (est, r, mu)


def test_contraction_fp32_inputs(dl):
    """complex64 inputs (the low-precision pipeline): FP32 products and DFT, within 1e-6."""
    dims = (4, 6, 4, 8)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 54)
    n = 5
    eta = np.stack([noise.z4_noise(dims, 55, r) for r in range(n)]).astype(np.complex64)
    s = synth.gaussian_spinors(dims, n, 56).astype(np.complex64)
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        npm = len(dl.dl_momenta(4))
        out = torch.zeros((n, dims[3], npm, 5, 4, 4), dtype=torch.complex128, device="cuda")
        dl.dl_contract(ctx, dl.DL_EST_ONE_END, _dev(eta), _dev(s), n, dl.DL_C64, 1, 4, out)
        got = out.cpu().numpy()
    finally:
        dl.dl_destroy(ctx)
    pre = loops.prefactor("one_end", kappa, amu)
    for r in range(n):
        xi, phi = loops.pair("one_end", links, eta[r].astype(np.complex128), s[r].astype(np.complex128), kappa, amu)
        ref = pre * loops.project_momenta(loops.bilinear(xi, phi), dims, 4)
        assert _rel(got[r, :, :, 0], ref) < 1e-6
        for mu in range(4):
            refd = pre * loops.project_momenta(loops.derivative_bilinear(links, xi, phi, mu), dims, 4)
            assert _rel(got[r, :, :, 1 + mu], refd) < 1e-6


def test_hpe_exact_matches_oracle(dl):
    dims = (4, 4, 4, 4)
    kappa, amu = 0.1612, 0.0055
    links = synth.gauge_links(dims, 0.4, 61)
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        got = dl.dl_hpe_exact(ctx, 1)
    finally:
        dl.dl_destroy(ctx)
    ref = loops.hpe_exact_c(links, kappa, amu, (1, 2, 3, 0))
    assert np.abs(got - ref).max() < 1e-14


@pytest.mark.parametrize("hp_guess,hpe_diff", [(0, 0), (1, 0), (1, 1)])
def test_tsm_against_exact_loops(dl, hp_guess, hpe_diff):
    """Eq. estiTSM with an HP map converged to 1e-11 and an LP map converged to 1e-5:
    the estimate is the mean of the exact per-noise loops (dense inverse) over the HP
    and LP sets up to the LP error; the HP per-noise observables are exact (also when
    every HP solve starts from its LP solution)."""
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n_hp, n_lp = 3, 5
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-11, tol_lp=1e-5, prec_hp_lo=dl.DL_F64,
                               prec_lp_lo=dl.DL_F32, delta_hp=0.1, block=4, seed=2000, p2max=1, with_deriv=0, hpe=1,
                               max_iter=50000, chunk=8, hp_guess=hp_guess, hpe_diff=hpe_diff)
        np_ = len(dl.dl_momenta(1))
        out = np.zeros((3, dims[3], np_, 1, 4, 4), dtype=np.complex128)
        ohp = np.zeros((n_hp, 4))
        olpp = np.zeros((n_hp, 4))
        olp = np.zeros((n_lp, 4))
        st, info = dl.dl_tsm_run(ctx, prm, out, ohp, olpp, olp)
        assert st == 0
    finally:
        dl.dl_destroy(ctx)
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    per = {"one_end": [], "gen_one_end": [], "hpe": []}
    sig = []
    for r in range(n_hp + n_lp):
        e = noise.z4_noise(dims, 2000, r)
        s = (minv @ e.ravel()).reshape(e.shape)
        for est in per:
            xi, phi = loops.pair(est, links, e, s, kappa, amu)
            per[est].append(loops.prefactor(est, kappa, amu) * loops.project_momenta(loops.bilinear(xi, phi), dims, 1))
        xi, phi = loops.pair("one_end", links, e, s, kappa, amu)
        sig.append(loops.prefactor("one_end", kappa, amu) * loops.loop_from_c(loops.bilinear(xi, phi), 1j * np.diag([1, 1, -1, -1])).sum())
    ex = loops.hpe_exact_c(links, kappa, amu, (0, 0, 0, 0))
    ip0 = [tuple(p) for p in dl.dl_momenta(1)].index((0, 0, 0))
    for k, est in enumerate(per):
        f = np.array(per[est])
        if est == "hpe":
            f[:, :, ip0] += dims[0] * dims[1] * dims[2] * ex
        ref = loops.tsm_estimate(f[:n_hp], f[:n_hp], f[n_hp:])
        assert _rel(out[k, :, :, 0], ref) < 1e-4, est
    assert np.abs(ohp[:, 0] - np.real(sig[:n_hp])).max() < 1e-7 * np.abs(sig).max()
