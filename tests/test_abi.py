"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/ttice.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttice.h")
LIB = os.path.join(ROOT, "paper_2211_12487_gb300", "libttice.so")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttice_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_12487_gb300 import build

    build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ttice_create", "ttice_update", "ttice_project", "ttice_ranks", "ttice_reconstruct",
              "ttice_stats", "ttice_destroy", "ttice_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_same_names(lib):
    from paper_2211_12487_gb300 import ttice

    for n in _declared():
        assert hasattr(ttice, n), n


def test_defaults_and_strerror(lib):
    from paper_2211_12487_gb300 import ttice

    h = ttice.ttice_default_heuristics()
    assert h.skip_mode == ttice.TTICE_SKIP_EXACT and h.subselect == 1 and h.occupancy_tau == 1.0
    c = ttice.ttice_default_capacity()
    assert c.max_batch >= 1 and c.max_rank >= 1
    assert ttice.ttice_strerror(ttice.TTICE_ECAPACITY).startswith("rank capacity")
    # invalid arguments are rejected on the host before any device work
    with pytest.raises(ttice.TTICEError) as ei:
        ttice.ttice_create([4, 4], 1.5)
    assert ei.value.code == ttice.TTICE_EINVAL
    with pytest.raises(ttice.TTICEError):
        ttice.ttice_create([], 0.1)


def test_stats_struct_layout(lib):
    from paper_2211_12487_gb300 import ttice

    # int32,int32,double*3,int64[18],int32[16],int64,int64,int32 x4 with natural alignment
    assert ctypes.sizeof(ttice.ttice_update_stats) == 8 + 24 + 144 + 64 + 16 + 8 + 8
