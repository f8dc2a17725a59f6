"""The C-ABI library loads and exports every function include/*.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(rope_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so():
    from paper_2603_22245_gb300 import build, rotormap

    if not os.path.exists(rotormap.LIB_PATH):
        build.build()
    return ctypes.CDLL(rotormap.LIB_PATH)


def test_header_declares_the_path():
    names = declared_functions()
    for fn in ("rope_encode_reads", "rope_encode_reference", "rope_score_topk", "rope_map", "rope_index_free",
               "rope_status_string", "rope_last_error"):
        assert fn in names


def test_every_declared_symbol_is_exported(so):
    for name in declared_functions():
        assert hasattr(so, name), name


def test_binding_covers_every_symbol():
    from paper_2603_22245_gb300 import rotormap

    for name in declared_functions():
        assert name in rotormap.EXPORTS, name


def test_host_only_calls(so):
    from paper_2603_22245_gb300 import rotormap

    lib = rotormap.load()
    assert lib.rope_status_string(2) == b"ROPE_ERR_INVALID_BASE"
    assert rotormap.rope_dim(rotormap.Params()) == 32
    assert rotormap.rope_dim(rotormap.Params(m=4, t=2)) == 64
    assert rotormap.rope_dim(rotormap.Params(s=8, m=4, t=4, window_len=20000)) == 1024
    assert rotormap.rope_dim(rotormap.Params(s=9)) == -1
    assert rotormap.rope_dim(rotormap.Params(t=5)) == -1
    assert rotormap.rope_dim(rotormap.Params(window_len=2)) == -1
    assert rotormap.rope_dim(rotormap.Params(stride=0)) == -1
