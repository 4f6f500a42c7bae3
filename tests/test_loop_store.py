"""Base-2 storage of per-noise loops (App. A, "Binary storage system", Fig. St):
the library's host writer and reader against the oracle's restatement of the scheme,
an independent reader of the file format, and the paper's worked example.  No GPU."""
import ctypes as C
import json
import os
import struct

import numpy as np
import pytest

import synth
from oracle import lattice, loops, noise, solver

HERE = os.path.dirname(os.path.abspath(__file__))


def _dl():
    import paper_1309_2256_gb300 as dl
    return dl


def _fnv1a64(data: bytes) -> int:
    """FNV-1a, 64-bit, from its published definition (offset basis, prime)."""
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def _read_file(path):
    """Independent reader of the documented format: (header dict, float64 payload)."""
    raw = open(path, "rb").read()
    magic, version, zero, weight, count, first, n_values, checksum = struct.unpack("<8sIIQQQQQ", raw[:56])
    payload = raw[56:]
    assert magic == b"DLLOOPB2" and version == 1 and zero == 0
    assert len(payload) == 8 * n_values
    assert _fnv1a64(payload) == checksum
    return dict(weight=weight, count=count, first=first, n_values=n_values), np.frombuffer(payload, "<f8")


def _write_sources(prefix, per_noise, chunks=None):
    dl = _dl()
    flat = np.ascontiguousarray(per_noise).reshape(len(per_noise), -1)
    if flat.dtype == np.complex128:
        flat = flat.view(np.float64)
    st = dl.dl_store_open(prefix, flat.shape[1])
    chunks = chunks or [len(flat)]
    at = 0
    for c in chunks:
        dl.dl_store_add(st, flat[at:at + c])
        at += c
    assert dl.dl_store_count(st) == len(flat)
    dl.dl_store_close(st)
    return flat


def test_fnv1a64_published_vectors():
    # the offset basis is the hash of the empty string; values of the FNV authors' test suite
    assert _fnv1a64(b"") == 0xCBF29CE484222325
    assert _fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert _fnv1a64(b"foobar") == 0x85944171F73967E8


def test_files_match_oracle(tmp_path):
    """23 sources: complete files 1, 2, 4, 8 (sources 0-14) and a .partial with 15-22."""
    rng = np.random.default_rng(11)
    per = rng.normal(size=(23, 4, 16)) + 1j * rng.normal(size=(23, 4, 16))
    prefix = str(tmp_path / "loops")
    flat = _write_sources(prefix, per, chunks=[3, 1, 9, 10])
    files = loops.binary_storage_files(flat)
    assert sorted(files) == [1, 2, 4, 8]
    assert sorted(os.listdir(tmp_path)) == ["loops.1", "loops.2", "loops.4", "loops.8", "loops.partial"]
    for w, ref in files.items():
        head, got = _read_file(f"{prefix}.{w}")
        assert head == dict(weight=w, count=w, first=w - 1, n_values=flat.shape[1])
        # both sides add the sources of a group in index order
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15 * w * np.abs(flat).max())
    head, got = _read_file(prefix + ".partial")
    assert head == dict(weight=16, count=8, first=15, n_values=flat.shape[1])
    np.testing.assert_allclose(got, flat[15:23].sum(0), rtol=0, atol=1e-14 * np.abs(flat).max())


def test_dyadic_sources_are_exact(tmp_path):
    """Small-integer sources add without rounding: files equal the oracle's bit for bit."""
    rng = np.random.default_rng(12)
    flat = rng.integers(-1000, 1000, size=(31, 50)).astype(np.float64) / 8.0
    prefix = str(tmp_path / "d")
    _write_sources(prefix, flat)
    files = loops.binary_storage_files(flat)
    for w, ref in files.items():
        assert np.array_equal(_read_file(f"{prefix}.{w}")[1], ref)
    for n in range(32):
        got = _dl().dl_store_load(prefix, 50, n)
        ref = loops.binary_storage_reconstruct(files, n) if n else np.zeros(50)
        assert np.array_equal(got, ref), n


def test_reconstruction_of_every_size(tmp_path):
    """load(n) is the sum over the n sources dl_store_sources(n) names, for every n < 16."""
    dl = _dl()
    rng = np.random.default_rng(13)
    flat = rng.normal(size=(15, 7))
    prefix = str(tmp_path / "r")
    _write_sources(prefix, flat)
    files = loops.binary_storage_files(flat)
    for n in range(16):
        idx = dl.dl_store_sources(n)
        assert len(idx) == n and len(set(idx.tolist())) == n and (idx < 15).all()
        got = dl.dl_store_load(prefix, 7, n)
        np.testing.assert_allclose(got, flat[idx].sum(0) if n else 0.0, rtol=0, atol=1e-13)
        if n:
            np.testing.assert_allclose(got, loops.binary_storage_reconstruct(files, n), rtol=0, atol=1e-13)


def test_paper_example_thirteen_sources(tmp_path):
    """Fig. St: 13 = 1 + 4 + 8 sources, from the files of weights 1, 4 and 8 (mask 1 0 1 1)."""
    dl = _dl()
    g = json.load(open(os.path.join(HERE, "golden", "binary_storage_example.json")))
    total = sum(w * m for w, m in zip(g["weights"], g["mask"]))
    assert total == g["total"] == 13
    idx = dl.dl_store_sources(total).tolist()
    used = [w for w, m in zip(g["weights"], g["mask"]) if m]
    assert idx == [i for w in used for i in range(w - 1, 2 * w - 1)]
    assert idx == [0] + list(range(3, 15))
    rng = np.random.default_rng(14)
    flat = rng.normal(size=(15, 5))
    prefix = str(tmp_path / "fig")
    _write_sources(prefix, flat)
    os.remove(prefix + ".2")  # the unused file is not read
    np.testing.assert_allclose(dl.dl_store_load(prefix, 5, total), flat[idx].sum(0), rtol=0, atol=1e-13)


def test_resume_equals_one_pass(tmp_path):
    dl = _dl()
    rng = np.random.default_rng(15)
    flat = rng.normal(size=(27, 12))
    one = str(tmp_path / "one")
    _write_sources(one, flat)
    parts = str(tmp_path / "parts")
    at = 0
    for c in (2, 5, 1, 0, 9, 10):
        st = dl.dl_store_open(parts, 12, resume=1 if at else 0)
        assert dl.dl_store_count(st) == at
        dl.dl_store_add(st, flat[at:at + c])
        at += c
        dl.dl_store_close(st)
    assert at == 27
    names = sorted(os.listdir(tmp_path))
    assert [n for n in names if n.startswith("one")] == ["one.1", "one.2", "one.4", "one.8", "one.partial"]
    for suffix in ("1", "2", "4", "8", "partial"):
        assert open(f"{one}.{suffix}", "rb").read() == open(f"{parts}.{suffix}", "rb").read(), suffix


def test_partial_removed_when_group_completes(tmp_path):
    dl = _dl()
    flat = np.arange(14.0).reshape(7, 2)
    p = str(tmp_path / "c")
    st = dl.dl_store_open(p, 2)
    dl.dl_store_add(st, flat[:5])
    dl.dl_store_close(st)
    assert os.path.exists(p + ".partial")
    st = dl.dl_store_open(p, 2, resume=1)
    dl.dl_store_add(st, flat[5:])
    assert not os.path.exists(p + ".partial")  # sources 3-6 now form the file of weight 4
    dl.dl_store_close(st)
    assert sorted(os.listdir(tmp_path)) == ["c.1", "c.2", "c.4"]
    np.testing.assert_array_equal(dl.dl_store_load(p, 2, 7), flat.sum(0))


def test_guards(tmp_path):
    dl = _dl()
    h = dl.lib()
    flat = np.random.default_rng(16).normal(size=(9, 4))
    p = str(tmp_path / "g")
    _write_sources(p, flat)
    # an existing store is not overwritten by a new writer
    with pytest.raises(dl.DLError) as e:
        dl.dl_store_open(p, 4)
    assert e.value.status == dl.DL_ERR_STATE
    # resume with another array size
    with pytest.raises(dl.DLError) as e:
        dl.dl_store_open(p, 5, resume=1)
    assert e.value.status == dl.DL_ERR_IO and "values" in str(e.value)
    # nine sources: files 1, 2, 4 and two in .partial; n = 8 needs the missing file of weight 8
    with pytest.raises(dl.DLError) as e:
        dl.dl_store_load(p, 4, 8)
    assert e.value.status == dl.DL_ERR_IO and "missing" in str(e.value)
    # a damaged payload fails its checksum
    raw = bytearray(open(p + ".4", "rb").read())
    raw[60] ^= 1
    open(p + ".4", "wb").write(bytes(raw))
    with pytest.raises(dl.DLError) as e:
        dl.dl_store_load(p, 4, 4)
    assert e.value.status == dl.DL_ERR_IO and "checksum" in str(e.value)
    # a truncated file
    open(p + ".4", "wb").write(bytes(raw[:70]))
    with pytest.raises(dl.DLError):
        dl.dl_store_load(p, 4, 4)
    # a gap in the complete files stops a resume
    os.remove(p + ".2")
    with pytest.raises(dl.DLError) as e:
        dl.dl_store_open(p, 4, resume=1)
    assert e.value.status == dl.DL_ERR_IO
    # argument checks
    out = C.c_void_p()
    assert h.dl_store_open(None, b"x", 4, 0) == dl.DL_ERR_ARG
    assert h.dl_store_open(C.byref(out), b"", 4, 0) == dl.DL_ERR_ARG
    assert h.dl_store_open(C.byref(out), os.fsencode(str(tmp_path / "z")), 0, 0) == dl.DL_ERR_ARG
    assert h.dl_store_open(C.byref(out), os.fsencode(str(tmp_path / "z")), 4, 2) == dl.DL_ERR_ARG
    assert out.value is None
    assert h.dl_store_add(None, None, 1) == dl.DL_ERR_ARG
    assert h.dl_store_load(os.fsencode(p), 4, -1, None) == dl.DL_ERR_ARG
    assert h.dl_store_sources(-1, None) == dl.DL_ERR_ARG
    assert h.dl_store_close(None) == dl.DL_OK
    # a directory that does not exist: the first complete group cannot be written
    st = dl.dl_store_open(str(tmp_path / "nodir" / "x"), 4)
    with pytest.raises(dl.DLError) as e:
        dl.dl_store_add(st, flat[:1])
    assert e.value.status == dl.DL_ERR_IO
    assert dl.dl_store_count(st) == 1  # the source is kept; the write is retried
    os.mkdir(tmp_path / "nodir")
    dl.dl_store_add(st, flat[1:3])
    dl.dl_store_close(st)
    np.testing.assert_allclose(dl.dl_store_load(str(tmp_path / "nodir" / "x"), 4, 3), flat[:3].sum(0), atol=1e-15)


def test_tsm_estimate_from_stores(tmp_path):
    """The paper's use: per-noise one-end loops of the 4^4 lattice (HP to 1e-9, LP to 1e-2)
    stored as HP-LP corrections and fresh LP loops; Eq. estiTSM over the base-2 source sets
    equals the oracle's estimate over the same sources."""
    dl = _dl()
    dims, kappa, amu = (4, 4, 4, 4), 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n_hp, n_lp = 7, 11

    def one_end(eta, s):
        xi, phi = loops.pair("one_end", links, eta, s, kappa, amu)
        return loops.project_momenta(loops.bilinear(xi, phi), dims, 1)

    f_hp, f_lp_pair, f_lp = [], [], []
    for r in range(n_hp + n_lp):
        eta = noise.z4_noise(dims, 2000, r)
        s_lp = solver.solve_eo(links, eta, kappa, amu, tol=1e-2)[0]
        if r < n_hp:
            f_hp.append(one_end(eta, solver.solve_eo(links, eta, kappa, amu, tol=1e-9)[0]))
            f_lp_pair.append(one_end(eta, s_lp))
        else:
            f_lp.append(one_end(eta, s_lp))
    f_hp, f_lp_pair, f_lp = map(np.array, (f_hp, f_lp_pair, f_lp))
    assert f_hp.shape[1:] == (dims[3], len(lattice.momenta(1)), 4, 4)
    corr, fresh = str(tmp_path / "corr"), str(tmp_path / "lp")
    _write_sources(corr, f_hp - f_lp_pair)
    _write_sources(fresh, f_lp)
    nv = 2 * f_hp[0].size
    for nh, nl in ((7, 7), (3, 5), (1, 6)):
        ih, il = dl.dl_store_sources(nh), dl.dl_store_sources(nl)
        est = (dl.dl_store_load(corr, nv, nh) / nh + dl.dl_store_load(fresh, nv, nl) / nl).view(np.complex128)
        ref = loops.tsm_estimate(f_hp[ih], f_lp_pair[ih], f_lp[il]).ravel()
        np.testing.assert_allclose(est, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
