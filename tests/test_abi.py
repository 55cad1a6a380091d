"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; host-only calls validate their arguments."""
import ctypes as C
import os
import re

import pytest

from paper_2212_08836_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    import paper_2212_08836_gb300 as P
    return P.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_and_workspace_size(lib):
    import paper_2212_08836_gb300 as P
    assert lib.pic_strerror(P.PIC_E_NOCONV).decode().startswith("Picard")
    cfg = P.Config(**P.small_reactor())
    nb = C.c_size_t(0)
    assert lib.pic_workspace_size(C.byref(cfg), C.byref(nb)) == 0
    cap = int(40000 * 1.5)
    assert nb.value > 2 * 2 * cap * 56  # double-buffered SoA of both species
    bad = P.Config(**P.small_reactor(nr=1))
    assert lib.pic_workspace_size(C.byref(bad), C.byref(nb)) == P.PIC_E_CONFIG
    h = C.c_void_p()
    assert lib.pic_init(C.byref(bad), None, 0, None, C.byref(h)) == P.PIC_E_CONFIG
    good = P.Config(**P.small_reactor())
    assert lib.pic_init(C.byref(good), None, 0, None, C.byref(h)) == P.PIC_E_WORKSPACE
    assert lib.pic_init(C.byref(good), 16, 1 << 30, None, C.byref(h)) == P.PIC_E_WORKSPACE


def test_cnn_workspace_size_validates_config(lib):
    import paper_2212_08836_gb300 as P
    lib.pic_cnn_workspace_size.restype = C.c_size_t
    good = P.CnnConfig(nr=8, nz=12, width=64, depth=5, batch=2, seed=0)
    n = lib.pic_cnn_workspace_size(C.byref(good))
    H, W = 9, 13
    assert n > 2 * H * W * 64 * 2 * 4  # activations of the hidden layers
    for bad in (dict(width=32), dict(depth=1), dict(depth=9), dict(batch=0), dict(nr=0)):
        c = dict(nr=8, nz=12, width=64, depth=5, batch=2, seed=0)
        c.update(bad)
        assert lib.pic_cnn_workspace_size(C.byref(P.CnnConfig(**c))) == 0
    h = C.c_void_p()
    assert lib.pic_cnn_init(C.byref(good), None, 0, None, C.byref(h)) == P.PIC_E_WORKSPACE
    assert lib.pic_set_guess(None, 0, None) == P.PIC_E_CONFIG
