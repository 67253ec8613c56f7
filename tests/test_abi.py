"""The C-ABI library loads and exports every entry point that include/*.h declares;
host-side checks that need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2002_04889_gb300 import build as B
from paper_2002_04889_gb300 import volna

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vg_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    assert _declared() <= set(volna._SIGNATURES), _declared() - set(volna._SIGNATURES)


def test_host_only_calls():
    assert volna.vg_version() >= 10000
    assert volna.vg_strerror(volna.VG_EINVAL) == "invalid argument"
    p = volna.vg_default_params()
    assert p.g == 9.81 and p.cfl == 0.9 and p.order == 2 and p.gauge_every == 1


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(volna.VolnaError) as e:
        volna.vg_create(64, 0)
    assert e.value.code == volna.VG_ECUDA
    with pytest.raises(volna.VolnaError):
        volna.vg_create(16, 0)
