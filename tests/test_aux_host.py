"""Host-side auxiliary subsystems, checked without a GPU: the phase-range trace
hook (the library's NVTX ranges), the tile-shape JSON file and the autotuner's
cache, the L-BFGS state image (its header and checksum, against an FNV-1a
written here from its published definition), and the registration state file.
None of these calls touches a CUDA device."""
import ctypes
import json
import os
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def meta():
    from paper_2106_08817_gb300 import _build
    _build.build()
    import paper_2106_08817_gb300 as m
    return m


# ------------------------------------------------------------------ tracing

def test_trace_hook_sees_nested_pushes_and_pops_in_order(meta):
    lib = meta._load()
    with meta.trace() as ev:
        assert lib.meta_trace_selftest() == 0
        assert lib.meta_trace_selftest() == 0
    one = [("meta.selftest", 1), ("meta.selftest.inner", 1), ("meta.selftest.inner", 0),
           ("meta.selftest", 0)]
    assert ev == one + one
    n = len(ev)
    assert lib.meta_trace_selftest() == 0  # hook removed: nothing more is seen
    assert len(ev) == n


# ------------------------------------------------------- tile-shape file

SHAPES = [  # (dims, batch, sigma, tuning)
    ((160, 192, 160), 1, 6.0, dict(zc_transport=8, zc_advect=16, ly=64, lz=32, txw=160,
                                   split=1)),
    ((256, 256), 16, 3.0, dict(zc_transport=0, zc_advect=0, ly=64, lz=0, txw=128, split=4)),
    ((40, 56), 2, 0.1, dict(zc_transport=0, zc_advect=0, ly=16, lz=0, txw=24, split=2)),
]


def _forget(meta):
    for dims, B, sg, _ in SHAPES:
        meta.set_tuning(dims, B, sg, None)


def test_tuning_file_round_trip_is_exact(meta, tmp_path):
    _forget(meta)
    for dims, B, sg, t in SHAPES:
        meta.set_tuning(dims, B, sg, t)
    f = tmp_path / "tiles.json"
    meta.tuning_save(f)
    doc = json.loads(f.read_text())  # a plain JSON document
    assert doc["format"] == "meta-tuning" and doc["version"] == 1
    got = {(tuple(e["dims"]), e["batch"]): e for e in doc["entries"]}
    for dims, B, sg, t in SHAPES:
        e = got[(dims, B)]
        assert struct.unpack("<I", struct.pack("<f", sg))[0] == e["sigma_bits"]
        assert {k: e[k] for k in t} == t
    _forget(meta)
    assert meta.tuning((40, 56), 2, 0.1)["txw"] != 24  # back to the built-in choice
    assert meta.tuning_load(f) >= len(SHAPES)
    for dims, B, sg, t in SHAPES:
        assert meta.tuning(dims, B, sg) == t
    _forget(meta)


def _doc(entries):
    return {"format": "meta-tuning", "version": 1, "entries": entries}


GOOD = {"ndim": 2, "dims": [40, 56], "batch": 2, "sigma": 0.1, "zc_transport": 0,
        "zc_advect": 0, "ly": 16, "lz": 0, "txw": 24, "split": 2}


@pytest.mark.parametrize("text", [
    "",                                                    # empty
    "{",                                                   # truncated
    json.dumps(_doc([GOOD])) + " x",                       # trailing garbage
    json.dumps({"format": "other", "version": 1, "entries": []}),
    json.dumps({"format": "meta-tuning", "version": 2, "entries": []}),
    json.dumps({"format": "meta-tuning", "version": 1}),   # no entries
    json.dumps(_doc([GOOD, dict(GOOD, txw=20)])),          # not a multiple of 8
    json.dumps(_doc([GOOD, dict(GOOD, txw=264)])),         # wider than the TMA box
    json.dumps(_doc([GOOD, dict(GOOD, dims=[40, 56, 8])])),  # dims do not match ndim
    json.dumps(_doc([GOOD, dict(GOOD, split=3)])),         # split beyond the batch
    json.dumps(_doc([GOOD, dict(GOOD, ly=16.5)])),         # not an integer
    json.dumps(_doc([GOOD, dict(GOOD, lz=16)])),           # lz in 2-D
    json.dumps(_doc([GOOD, dict(GOOD, sigma=40.0)])),      # sigma out of range
    json.dumps(_doc([{k: v for k, v in GOOD.items() if k != "ly"}])),
    '{"format": "meta-tuning", "version": 1, "entries": [1e999]}',
    '{"format": "meta-tuning", "version": 1, "entries": ["\\ud800"]}',
])
def test_malformed_tuning_files_are_refused_whole(meta, tmp_path, text):
    _forget(meta)
    f = tmp_path / "bad.json"
    f.write_text(text)
    with pytest.raises(meta.MetaError) as e:
        meta.tuning_load(f)
    assert e.value.code == 8  # META_ERR_FORMAT
    assert meta.tuning((40, 56), 2, 0.1)["txw"] != 24  # nothing recorded, not even GOOD


def test_missing_tuning_file_is_an_io_error(meta, tmp_path):
    with pytest.raises(meta.MetaError) as e:
        meta.tuning_load(tmp_path / "absent.json")
    assert e.value.code == 9  # META_ERR_IO


def test_tuning_file_extra_keys_and_sigma_without_bits(meta, tmp_path):
    _forget(meta)
    f = tmp_path / "t.json"
    f.write_text(json.dumps(dict(_doc([dict(GOOD, note="hand-written")]), device="any")))
    assert meta.tuning_load(f) == 1
    assert meta.tuning((40, 56), 2, 0.1)["txw"] == 24
    _forget(meta)


# ------------------------------------------------------ autotuner cache

def _autotune_raw(meta, dims, B, sigma):
    """meta_autotune with placeholder pointers, called only where the cache holds
    the shape: a hit returns before any argument but the problem is used (a miss
    would time kernels on these pointers, so no test calls it that way)."""
    lib = meta._load()
    pr = meta._problem(len(dims), dims, B, 4, sigma)
    t = meta._Tuning()
    fake = ctypes.c_void_p(256)
    rc = lib.meta_autotune(ctypes.byref(pr), fake, fake, fake, fake, fake, fake, fake, fake,
                           fake, 1 << 20, None, ctypes.byref(t))
    return rc, {f: getattr(t, f) for f in meta.TUNING_FIELDS}


def test_autotuner_cache_hit_records_the_entry_without_timing(meta, tmp_path):
    _forget(meta)
    f = tmp_path / "cache.json"
    try:
        assert meta.tuning_cache(f) == 0  # no file yet: an empty cache
        assert not f.exists()
        f.write_text(json.dumps(_doc([GOOD])))
        assert meta.tuning_cache(f) == 1  # read now, and recorded
        assert meta.tuning((40, 56), 2, 0.1)["txw"] == 24
        _forget(meta)
        rc, t = _autotune_raw(meta, (40, 56), 2, 0.1)
        assert rc == 0 and t["txw"] == 24 and t["ly"] == 16 and t["split"] == 2
        assert meta.tuning((40, 56), 2, 0.1)["txw"] == 24
    finally:
        meta.tuning_cache(None)
        _forget(meta)


def test_malformed_cache_file_is_refused_and_the_cache_stays_off(meta, tmp_path):
    f = tmp_path / "cache.json"
    f.write_text("not json")
    with pytest.raises(meta.MetaError) as e:
        meta.tuning_cache(f)
    assert e.value.code == 8
    assert meta.tuning((40, 56), 2, 0.1)["txw"] != 24  # nothing recorded


# ------------------------------------------------ L-BFGS state image

def fnv1a64(data: bytes) -> int:
    """FNV-1a, 64-bit: offset basis 0xcbf29ce484222325, prime 0x100000001b3."""
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def state_image(dims, B, m, k=7, h=2, head=1, seed=0, **over):
    """An image in the documented layout: 80-byte header, then g, S, Y (f32),
    rho, gamma, L (f64), stopped, done (i32)."""
    N = int(np.prod(dims))
    r = np.random.default_rng(seed)
    parts = [r.normal(size=B * N).astype("<f4"), r.normal(size=m * B * N).astype("<f4"),
             r.normal(size=m * B * N).astype("<f4"), r.normal(size=m * B).astype("<f8"),
             r.normal(size=B).astype("<f8"), r.normal(size=B).astype("<f8"),
             r.integers(0, 2, size=B).astype("<i4"), r.integers(0, max(k, 0) + 1, size=B).astype("<i4")]
    payload = b"".join(p.tobytes() for p in parts)
    d3 = list(dims) + [0] * (3 - len(dims))
    f = dict(tag=b"METALBFS", version=1, ndim=len(dims), dims=d3, batch=B, m=m, k=k, h=h,
             head=head, pad=(0, 0), n=N, payload=len(payload), checksum=fnv1a64(payload))
    f.update(over)
    hdr = struct.pack("<8sIi3iiiiii2iQQQ", f["tag"], f["version"], f["ndim"], *f["dims"],
                      f["batch"], f["m"], f["k"], f["h"], f["head"], *f["pad"], f["n"],
                      f["payload"], f["checksum"])
    assert len(hdr) == 80
    return hdr + payload


def _check(meta, dims, B, m, blob):
    pr = meta._problem(len(dims), dims, B, 4, 2.0)
    buf = (ctypes.c_ubyte * len(blob)).from_buffer_copy(blob)
    return meta._load().meta_lbfgs_state_check(ctypes.byref(pr), m, buf, len(blob))


@pytest.mark.parametrize("dims,B,m", [((4, 6), 2, 3), ((3, 4, 5), 1, 1), ((5, 7), 3, 5)])
def test_state_image_layout_and_checks(meta, dims, B, m):
    blob = state_image(dims, B, m, h=min(2, m), head=m - 1)
    pr = meta._problem(len(dims), dims, B, 4, 2.0)
    n = ctypes.c_size_t(0)
    assert meta._load().meta_lbfgs_state_size(ctypes.byref(pr), m, ctypes.byref(n)) == 0
    assert n.value == len(blob)
    assert _check(meta, dims, B, m, blob) == 0
    bad = bytearray(blob)
    bad[80 + len(blob[80:]) // 2] ^= 1  # one bit of the payload
    assert _check(meta, dims, B, m, bytes(bad)) == 8
    assert _check(meta, dims, B, m, blob[:-1]) == 8  # truncated
    assert _check(meta, dims, B, m + 1, blob) == 8   # another m
    other = tuple(x + 1 for x in dims)
    assert _check(meta, other, B, m, blob) == 8      # another shape
    for over in (dict(tag=b"METALBFX"), dict(version=2), dict(head=m), dict(h=m + 1),
                 dict(k=-1), dict(pad=(1, 0)), dict(pad=(0, 1)),
                 dict(batch=B + 1)):
        kw = dict(h=min(2, m))
        kw.update(over)
        assert _check(meta, dims, B, m, state_image(dims, B, m, **kw)) == 8, over


def test_state_save_refuses_a_workspace_without_a_run(meta):
    # argument checks come before any device access
    pr = meta._problem(2, (4, 6), 1, 4, 2.0)
    lib = meta._load()
    buf = (ctypes.c_ubyte * 16)()
    assert lib.meta_lbfgs_state_save(ctypes.byref(pr), 2, None, 0, buf, 16, None) == 1
    assert lib.meta_lbfgs_state_load(ctypes.byref(pr), 2, buf, 16, None, 0, None) == 8


# ------------------------------------------------ registration state file

def _settings(**over):
    s = dict(optimizer="lbfgs", ndim=2, dims=[4, 6], batch=2, T=5, sigma=2.0, mu=[0.1, 0.0],
             rho=[1.0, 1.3], lam=[1e-3, 1e-2], m=3, h0=0.05, ckpt=0, p_update=0, scheme="sl",
             iterations=4)
    s.update(over)
    return s


def test_registration_file_round_trip_and_refusals(tmp_path):
    from paper_2106_08817_gb300 import checkpoint as ck
    r = np.random.default_rng(3)
    p = r.normal(size=(2, 4, 6)).astype(np.float32)
    costs = r.normal(size=(5, 2))
    I0, J = r.normal(size=(2, 4, 6)), r.normal(size=(2, 4, 6))
    dg = ck.images_digest(I0, J)
    assert dg != ck.images_digest(J, I0) and dg == ck.images_digest(I0.astype(np.float32), J)
    blob = bytes(r.integers(0, 256, size=333, dtype=np.uint8))
    f = tmp_path / "reg.npz"
    ck.write(f, _settings(), p, costs, dg, blob)
    got = ck.read(f)
    assert np.array_equal(got["p"], p) and got["p"].dtype == np.float32
    assert np.array_equal(got["costs"], costs)
    assert got["lbfgs_state"] == blob and got["images_sha256"] == dg
    assert {k: got[k] for k in ck.SETTINGS} == _settings()
    assert [x.name for x in tmp_path.iterdir()] == ["reg.npz"]  # no temporary left
    # gradient descent carries no optimiser image
    ck.write(f, _settings(optimizer="gd"), p, costs, dg, None)
    assert ck.read(f)["lbfgs_state"] is None
    with pytest.raises(ValueError):
        ck.write(f, _settings(optimizer="gd"), p, costs, dg, blob)
    with pytest.raises(ValueError):
        ck.write(f, _settings(), p, costs[:3], dg, blob)  # history / iteration mismatch
    with pytest.raises(ValueError):
        ck.write(f, {k: v for k, v in _settings().items() if k != "T"}, p, costs, dg, blob)
    # files that are not registration states, or that disagree with themselves
    np.savez(tmp_path / "other.npz", x=np.zeros(3))
    with pytest.raises(ValueError):
        ck.read(tmp_path / "other.npz")
    import json as _json
    for over in (dict(version=np.array(2)), dict(format=np.array("something")),
                 dict(meta=np.array(_json.dumps(_settings(dims=[4, 7]))))):
        arrays = dict(format=np.array(ck.FORMAT), version=np.array(1),
                      meta=np.array(_json.dumps(_settings())), p=p, costs=costs,
                      images_sha256=np.array(dg), lbfgs_state=np.frombuffer(blob, np.uint8))
        arrays.update(over)
        np.savez(tmp_path / "bad.npz", **arrays)
        with pytest.raises(ValueError):
            ck.read(tmp_path / "bad.npz")
