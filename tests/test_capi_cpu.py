"""C-ABI library checks that need no GPU: it builds, loads, exports every
function include/rh15d.h declares, and fails loudly (no CPU fallback) when no
GPU is present."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|void|int64_t|const char \*)\s*\*?\s*(rh_\w+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_1411_1079_gb300._build import build
    return build()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rh_\w+)", out))
    declared = _declared()
    assert len(declared) >= 12
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(built):
    import paper_1411_1079_gb300 as rh
    assert sorted(rh.EXPORTS) == _declared()
    L = rh.lib()
    for n in _declared():
        assert hasattr(L, n)


def test_no_silent_cpu_fallback_without_gpu(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1411_1079_gb300 as rh
    with pytest.raises(rh.RhError) as e:
        rh.Context(0)
    assert e.value.code == rh.RH_ECUDA


def test_library_missing_raises(tmp_path):
    import importlib

    import paper_1411_1079_gb300 as rh
    saved = rh._lib
    try:
        rh._lib = None
        with pytest.raises(RuntimeError):
            rh.lib(str(tmp_path / "nope.so"))
    finally:
        rh._lib = saved
        importlib.reload  # keep flake quiet


def test_header_is_plain_c(tmp_path):
    """include/rh15d.h compiles as C99 on its own (no C++ or CUDA types)."""
    src = tmp_path / "use_header.c"
    src.write_text('#include "rh15d.h"\nint main(void) { rh_ctx *c = 0; (void)c; return 0; }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_column_kernel_shared_memory_layout():
    """The column kernel's shared memory is sized and carved by one layout
    (host computation, no GPU): regions follow each other without overlap,
    the FP64 regions are 8-byte and the background block, the Voigt
    table and the profile rings 16-byte aligned, the rings take 2304 bytes per
    warp, the carve ends exactly at the allocated size, and the H atom's FP32
    block with the rings of 8 warps fits two per SM (228 KB) at 82 depths and
    one at 128 depths.  A carve
    that reserved more than the allocation -- a region dropped from the size
    but not from the carve -- would write past the block's shared memory."""
    import paper_1411_1079_gb300 as rh
    sizes = {"double": 8, "float": 4}
    for prec in (0, 1):
        R = 4 if prec == 1 else 8
        for (L, N, ntr, ncont, nline, macc), rw in zip([(2, 2, 1, 0, 1, 2), (4, 13, 5, 3, 2, 20),
                                                        (6, 82, 15, 5, 10, 117), (6, 128, 15, 5, 10, 180),
                                                        (8, 4096, 32, 7, 25, 300)], [0, 3, 8, 8, 0]):
            off, nbytes = rh.column_smem_layout(prec, L, N, ntr, ncont, nline, macc, rw)
            # n, nn, Cr, red, slot, dz, ivth, vz, (pad) bg[N][4], Gc, ad, nr, (pad) vtab, ibuf, (pad) ring, end
            want = [8 * L * N, 8 * L * N, 8 * N * 2 * ntr, 8 * (5 * 64 + 8), R * macc * N, R * N, R * N]
            for i, w in enumerate(want):
                assert off[i + 1] - off[i] == w, (prec, i)
            assert off[7] + R * N <= off[8] < off[7] + R * N + 16 and off[8] % 16 == 0
            assert off[9] - off[8] == 4 * R * N
            assert off[10] - off[9] == R * ncont * N and off[11] - off[10] == R * nline * N
            assert all(o % 8 == 0 for o in off[:5]) and off[12] % 16 == 0
            assert off[11] + R * L * N <= off[12] < off[11] + R * L * N + 16
            assert off[13] == off[12] + 16 * 1025
            assert off[13] + 32 <= off[14] < off[13] + 48 and off[14] % 16 == 0
            assert off[15] == off[14] + 2304 * rw and off[15] == nbytes
    h82 = rh.column_smem_layout(1, 6, 82, 15, 5, 10, 117, 8)[1]
    assert 2 * (h82 + 1024) <= 228 * 1024        # 1 KB per block reserved by the driver
    assert rh.column_smem_layout(1, 6, 128, 15, 5, 10, 180, 8)[1] <= 227 * 1024
