"""Host logic of bench.py (no GPU): the equal-error metric (the paper's cost x error^2
figure of merit, Sec. 4) and the roofline arithmetic of the dominant stencil launch."""
import types

import numpy as np
import pytest

import bench


def _obs(re, im=None):
    """Per-noise observables [n][4]: sigma (re, im), axial (re, im), here equal."""
    im = np.zeros_like(re) if im is None else im
    return np.stack([re, im, re, im], axis=1)


def test_equal_error_exact_lp_map():
    """LP solutions equal to the HP ones: the HP-LP term has no variance, and the error
    of a sweep is var(f_LP) / N_LP, i.e. N_LP plain estimates when var(f_LP) = var(f_HP)."""
    rng = np.random.default_rng(0)
    f_hp = rng.normal(size=24)
    f_lp = rng.permutation(np.tile(f_hp, 20))[:480]  # same distribution, 480 fresh
    out = bench._equal_error(_obs(f_hp), _obs(f_hp), _obs(f_lp), 24, 480, 2.0)
    for name in ("sigma", "axial"):
        e = out[name]
        assert e["v_diff"] == 0.0
        assert e["err2_step"] == pytest.approx(np.var(f_lp, ddof=1) / 480)
        assert e["plain_equiv_per_step"] == pytest.approx(np.var(f_hp, ddof=1) / (np.var(f_lp, ddof=1) / 480))
        assert e["per_s"] == pytest.approx(e["plain_equiv_per_step"] / 2.0)


def test_equal_error_useless_lp_map():
    """LP estimates independent of the HP ones: the correction carries var(f_HP) + var(f_LP),
    so the sweep is worth fewer plain estimates than its N_HP HP solves."""
    rng = np.random.default_rng(1)
    n_hp, n_lp = 4000, 4000
    f_hp, f_pr, f_lp = rng.normal(size=n_hp), rng.normal(size=n_hp), rng.normal(size=n_lp)
    e = bench._equal_error(_obs(f_hp), _obs(f_pr), _obs(f_lp), n_hp, n_lp, 1.0)["axial"]
    # err^2 = 2/N_HP + 1/N_LP for unit variances: N_eq = 1 / (3 / 4000)
    assert e["plain_equiv_per_step"] == pytest.approx(4000 / 3, rel=0.08)
    assert abs(e["r_c"]) < 0.05


def test_roofline_bytes_of_the_16bit_stage3_launch():
    """Algorithmic bytes of one 16-bit stage-3 launch on 32^3 x 64 with 16 columns:
    all 4V links once (24 B, 16-bit recon-12) plus 7 spinor streams of Vh x 16 x 52 B."""
    V = 32 ** 3 * 64
    Vh = V // 2
    prof = np.zeros((4, 3, 3))
    prof[3, 2] = (10, 10 * 1.6, 10 * Vh * 16)  # 10 launches of 1.6 ms, 16 columns each
    prof[0, 1] = (10, 10 * 0.5, 10 * Vh * 16)
    infos = [types.SimpleNamespace(iters_hp=24 * 44, iters_lp=524 * 40)]
    r = bench.roofline(prof, infos)
    expect = 4 * V * 24 + 7 * Vh * 16 * 52
    assert r["bytes_per_launch"] == expect
    assert r["avg_launch_ms"] == pytest.approx(1.6)
    assert r["achieved"] == pytest.approx(expect / 1.6e-3 / 1e9, rel=1e-3)
    peaks, _ = bench._peaks()
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"], rel=1e-3)
    # the ncu traffic of the 24^3 x 24 capture, scaled by site-columns
    assert r["traffic"] == int(1002.4e6 / (24 ** 4 // 2 * 16) * Vh * 16)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
