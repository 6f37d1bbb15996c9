"""Checkpoint files of the learned-start network (rh_surrogate_save / _load /
_file_info).  The format is written here independently of the library, from
its documented layout: "RH15DMLP", uint32 version 1, int32 nin, hidden,
nhidden, nout, int64 nparam, nparam float32, and the 64-bit FNV-1a hash of
the state bytes (little-endian).  rh_surrogate_file_info reads such files
without a context or GPU and must reject every damaged one."""
import struct

import numpy as np
import pytest


def _nparam(nin, hidden, nhidden, nout):
    n = nin * hidden + hidden + (nhidden - 1) * (hidden * hidden + hidden) + hidden * nout + nout
    return n + 2 * nin


def _fnv1a(b: bytes) -> int:
    h = 0xcbf29ce484222325
    for x in b:
        h = ((h ^ x) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _write(path, sizes, state, version=1, magic=b"RH15DMLP", nparam=None, tail=b""):
    body = np.asarray(state, dtype="<f4").tobytes()
    n = len(state) if nparam is None else nparam
    with open(path, "wb") as f:
        f.write(magic + struct.pack("<I4iq", version, *sizes, n) + body + struct.pack("<Q", _fnv1a(body)) + tail)


@pytest.fixture(scope="module")
def rh():
    import paper_1411_1079_gb300 as m
    m.build()
    return m


SIZES = (48, 16, 2, 72)       # 12 depths, 6 levels x 12 depths


def _state(seed=0):
    return np.random.default_rng(seed).standard_normal(_nparam(*SIZES)).astype(np.float32)


def test_file_info_reads_a_valid_file(rh, tmp_path):
    p = tmp_path / "net.rhmlp"
    _write(p, SIZES, _state())
    info = rh.surrogate_file_info(p)
    assert (info["nin"], info["hidden"], info["nhidden"], info["nout"]) == SIZES
    assert info["nparam"] == _nparam(*SIZES)


@pytest.mark.parametrize("damage", ["magic", "version", "nparam", "byte", "truncated", "trailing", "missing"])
def test_file_info_rejects_damaged_files(rh, tmp_path, damage):
    p = tmp_path / "net.rhmlp"
    st = _state(1)
    if damage == "magic":
        _write(p, SIZES, st, magic=b"RH15DXXX")
    elif damage == "version":
        _write(p, SIZES, st, version=2)
    elif damage == "nparam":
        _write(p, SIZES, st[:-1], nparam=len(st) - 1)
    elif damage == "trailing":
        _write(p, SIZES, st, tail=b"\0")
    elif damage != "missing":
        _write(p, SIZES, st)
        raw = bytearray(p.read_bytes())
        if damage == "byte":
            raw[36 + 4 * 100] ^= 0x01
        else:
            raw = raw[:-20]
        p.write_bytes(bytes(raw))
    with pytest.raises(rh.RhError) as e:
        rh.surrogate_file_info(p)
    assert e.value.code == rh.RH_EINVAL


@pytest.mark.gpu
def test_save_load_round_trip(rh, orc, tmp_path):
    import rh_synth
    from oracle import mlp
    atom = rh_synth.hydrogen_like_atom()
    cols = rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, seed=5), slice(0, 64))
    o = orc.Oracle()
    o.setup_atom(atom)
    o.load_columns(cols)
    X = mlp.features(cols["T"], o.lte()[1], cols["nH"], cols["vz"])
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(cols)
    ctx.surrogate_init(hidden=32, nhidden=2, seed=3)
    rng = np.random.default_rng(3)
    parts = []
    for di, do in mlp.layer_dims(X.shape[1], 32, 2, atom["nlev"] * X.shape[1] // 4):
        parts += [rng.standard_normal(do * di) * np.sqrt(2.0 / di), np.zeros(do)]
    parts += [X.mean(axis=0), 1.0 / np.maximum(X.std(axis=0), 1e-6)]
    state = np.concatenate(parts).astype(np.float32)
    ctx.surrogate_set_state(state)
    p = tmp_path / "net.rhmlp"
    ctx.surrogate_save(p)
    info = rh.surrogate_file_info(p)
    assert (info["nin"], info["hidden"], info["nhidden"], info["nout"]) == (X.shape[1], 32, 2,
                                                                           atom["nlev"] * X.shape[1] // 4)
    ctx2 = rh.Context(0)
    ctx2.setup_atom(atom)
    ctx2.load_columns(cols)
    ctx2.surrogate_load(p)
    assert np.array_equal(ctx2.surrogate_state(), state)
    np.testing.assert_array_equal(ctx2.surrogate_predict(), ctx.surrogate_predict())
    # a network for another depth count is refused
    ctx3 = rh.Context(0)
    ctx3.setup_atom(atom)
    ctx3.load_columns(rh_synth.subset(rh_synth.chromosphere_cube(nx=8, ny=8, ndep=40, seed=5), slice(0, 4)))
    with pytest.raises(rh.RhError) as e:
        ctx3.surrogate_load(p)
    assert e.value.code == rh.RH_EINVAL
