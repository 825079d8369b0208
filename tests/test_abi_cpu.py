"""C ABI checks that need no GPU: the library loads and exports every entry
point that include/burgers.h declares, and the binding covers each of them."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(burgers_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("burgers_explicit_advance", "burgers_btcs_advance", "burgers_rel_l2",
                 "burgers_cfl_dt", "burgers_ctx_create", "burgers_ctx_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2601_12204_b300 import _lib as L
    lib = L.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2601_12204_b300 import _lib as L
    assert declared_functions() == set(L.SIGNATURES)


def test_library_is_built_for_sm_103a():
    from paper_2601_12204_b300 import build as B
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert os.path.exists(B.LIB)


def test_no_gpu_means_clean_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2601_12204_b300 import api
    with pytest.raises(Exception):
        api.Context(0)
