"""Pins of the oracle's conventions: gammas, indexing, momenta, noise, storage (CPU only)."""
import json
import os

import numpy as np

from oracle import lattice, loops, noise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_gamma_algebra():
    g = lattice.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(lattice.GAMMA5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(g[mu] @ lattice.GAMMA5 + lattice.GAMMA5 @ g[mu], 0)


def test_gamma16_basis():
    G = lattice.GAMMAS16
    assert np.allclose(G[0], np.eye(4))
    assert np.allclose(G[15], lattice.GAMMA5)
    # gamma_mu gamma_5 in the bitmask basis (closed forms of the ordering)
    g5 = lattice.GAMMA5
    assert np.allclose(lattice.GAMMA[0] @ g5, G[14])
    assert np.allclose(lattice.GAMMA[1] @ g5, -G[13])
    assert np.allclose(lattice.GAMMA[2] @ g5, G[11])
    assert np.allclose(lattice.GAMMA[3] @ g5, -G[7])
    # the 16 are orthogonal under the trace: a basis of 4x4 matrices
    gram = np.array([[np.trace(a.conj().T @ b) for b in G] for a in G])
    assert np.allclose(gram, 4 * np.eye(16))


def test_indexing():
    dims = (4, 2, 6, 4)
    X, Y, Z, T = dims
    lex = lattice.lex_index(dims)
    assert lex[1, 2, 1, 3] == 3 + X * (1 + Y * (2 + Z * 1))
    par = lattice.parity(dims)
    cb = lattice.cb_index(dims)
    V = X * Y * Z * T
    for p in (0, 1):
        idx = np.sort(cb[par == p])
        assert np.array_equal(idx, np.arange(V // 2))
    assert par[0, 0, 0, 0] == 0 and par[0, 0, 0, 1] == 1


def test_momenta_counts():
    assert len(lattice.momenta(0)) == 1
    assert len(lattice.momenta(4)) == 33
    assert len(lattice.momenta(9)) == 123
    pl = lattice.momenta(4)
    assert pl[0] == (0, 0, -2) and pl[-1] == (0, 0, 2)
    assert pl.index((0, 0, 0)) == 16


def test_insertion_count_golden():
    g = _golden("insertion_count.json")
    n = g["n_gamma"] * (1 + g["n_derivative_directions"]) * g["n_flavour_structures"]
    assert n == g["total_insertions"] == 160
    assert len(lattice.GAMMAS16) == g["n_gamma"]


def test_splitmix64_golden():
    g = _golden("splitmix64_reference.json")
    out = noise.splitmix64(1234567, np.arange(5, dtype=np.uint64))
    assert [int(v) for v in out] == g["seed_1234567_first5"]
    out0 = noise.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out0] == [int(h, 16) for h in g["seed_0_first3_hex"]]


def test_noise_values_and_moments():
    dims = (4, 4, 4, 4)
    eta = np.stack([noise.z4_noise(dims, 77, r) for r in range(64)])
    assert np.allclose(np.abs(eta), 1.0)
    vals = np.unique(np.round(eta.ravel() * np.sqrt(2), 12))
    assert len(vals) == 4
    v = eta.reshape(64, -1)
    # E[eta] = 0 and E[eta eta^dagger] = 1 (Eqs. eq1, eq2) within sampling error
    assert np.abs(v.mean()) < 5.0 / np.sqrt(v.size)
    cov = v.conj().T @ v / 64.0
    assert np.allclose(np.diag(cov), 1.0)
    off = cov - np.diag(np.diag(cov))
    assert np.abs(off).mean() < 3.0 / np.sqrt(64)
    # the counter fixes every entry: noise r is independent of how many others are drawn
    assert np.array_equal(noise.z4_noise(dims, 77, 5), eta[5])
    q = noise.z4_noise(dims, 77, 3, quadrant=True)
    assert set(np.round(q.ravel(), 12).tolist()) <= {1, 1j, -1, -1j}


def test_binary_storage_golden():
    g = _golden("binary_storage_example.json")
    rng = np.random.default_rng(0)
    per = rng.normal(size=(15, 3))
    files = loops.binary_storage_files(per)
    assert sorted(files) == g["weights"]
    n = sum(w * m for w, m in zip(g["weights"], g["mask"]))
    assert n == g["total"]
    rebuilt = loops.binary_storage_reconstruct(files, n)
    # File.1 = noise 0, File.4 = noise 3..6, File.8 = noise 7..14
    expect = per[0] + per[3:7].sum(0) + per[7:15].sum(0)
    assert np.allclose(rebuilt, expect)
    assert np.allclose(loops.binary_storage_reconstruct(files, 15), per.sum(0))
