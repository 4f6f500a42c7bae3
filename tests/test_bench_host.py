"""Host logic of bench.py (no GPU): the equal-error metric (the paper's cost x error^2
figure of merit, Sec. 4) and the roofline arithmetic of the dominant stencil launch."""
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


def test_roofline_picks_the_class_with_the_most_time_per_sweep():
    """Stencil statistics of two steps: a 16-bit CG-update class (7 spinor streams) with
    many short launches and a double-float class with few long ones.  The roofline
    kernel is the class with the larger launches x average duration; its algorithmic
    bytes are all 4V links once plus every spinor stream of Vh x columns once."""
    V = 32 ** 3 * 64
    Vh = V // 2
    st = np.zeros((4, 4, 2, 4))
    # 16-bit (storage 2), cg-update (epilogue 3), dagger: 600 launches, 20 timed at 1.6 ms, 16 columns
    st[2, 3, 1] = (600, 20, 20 * 1.6, 20 * Vh * 16)
    # double-float (storage 0), plain, not dagger: 40 launches, 10 timed at 5 ms, 16 columns
    st[0, 0, 0] = (40, 10, 10 * 5.0, 10 * Vh * 16)
    r, rows = bench.roofline(st, steps=2)
    assert [x["kernel"] for x in rows] == ["stencil 16-bit cg-update dagger", "stencil double-float plain"]
    assert rows[0]["ms_per_step"] == pytest.approx(600 * 1.6 / 2)
    assert rows[1]["ms_per_step"] == pytest.approx(40 * 5.0 / 2)
    expect = 4 * V * 24 + 7 * Vh * 16 * 52
    assert r["kernel"] == "stencil 16-bit cg-update dagger"
    assert r["bytes_per_launch"] == expect
    assert r["avg_launch_ms"] == pytest.approx(1.6)
    assert r["achieved"] == pytest.approx(expect / 1.6e-3 / 1e9, rel=1e-3)
    peaks, _ = bench._peaks()
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"], rel=1e-3)
    assert rows[1]["bytes_per_launch"] == 4 * V * 144 + 2 * Vh * 16 * 192
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # traffic: the ncu bytes per site-column of the class, times the launch's site-columns
    per_item = bench.NCU_DRAM_BYTES_PER_ITEM[("16-bit", "cg-update")]
    assert r["traffic"] == int(per_item * Vh * 16)
    assert 0.9 < r["traffic"] / expect < 1.1


def test_gamma_matrices_of_the_error_report():
    """The error report forms loops with its own 16 Gamma_b; they are the oracle's."""
    from oracle import lattice
    g = bench._gammas16()
    for b in range(16):
        assert np.abs(g[b] - lattice.GAMMAS16[b]).max() == 0.0
