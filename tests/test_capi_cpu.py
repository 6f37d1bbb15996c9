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
