"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import glob
import os
import re

import pytest

from paper_2103_06737_gb300 import build as B


def _declared():
    names = set()
    for h in glob.glob(os.path.join(B.ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fem_pic_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def so():
    return B.build()


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("fem_pic_create", "fem_pic_push_deposit", "fem_pic_destroy", "fem_pic_status",
                 "fem_pic_sort", "fem_pic_residuals", "fem_pic_deposit_charge"):
        assert need in names


def test_library_exports_every_symbol(so):
    lib = ctypes.CDLL(so)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_without_gpu(so):
    lib = ctypes.CDLL(so)
    lib.fem_pic_last_error.restype = ctypes.c_char_p
    lib.fem_pic_last_error.argtypes = [ctypes.c_void_p]
    assert lib.fem_pic_last_error(None) is not None


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2103_06737_gb300 import fem_pic as F
    monkeypatch.setattr(F, "_lib", None)
    monkeypatch.setattr(F._build, "SO", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        F.lib()
