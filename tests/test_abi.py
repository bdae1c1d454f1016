"""The C-ABI library builds, loads and exports every declared symbol (no GPU).

Only calls that need no device are made: parameter sizes and argument
validation that fails before any CUDA call.
"""
import ctypes
import os
import re

import pytest

import oracle
from conftest import ROOT, read_golden

HEADER = os.path.join(ROOT, "include", "sntrup_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2106_08759_gb300 import build as b
    b.build()
    import paper_2106_08759_gb300 as snt
    return snt.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(snt_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "snt_batch_keygen" in names and len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("P", [653, 761, 857])
def test_param_sizes_match_oracle_and_paper(lib, P):
    import paper_2106_08759_gb300 as snt
    pkb, skb, ctb, ssb = snt.snt_param_sizes(P)
    opk, osk, _ = oracle.sizes(P)
    assert (pkb, skb, ssb) == (opk, osk, 32)
    storage = {int(r[0]): int(r[1]) for r in read_golden("table4_keypair_storage.txt")}
    assert pkb + skb == storage[P]
    if P == 761:  # Table 1: key + ciphertext = 2197 bytes
        row = read_golden("table1_sizes.txt")[0]
        assert pkb + ctb == int(row[1])


def test_invalid_arguments_fail_before_the_device(lib):
    import paper_2106_08759_gb300 as snt
    with pytest.raises(snt.SntError) as e:
        snt.snt_param_sizes(760)
    assert e.value.status == -1
    assert lib.snt_batch_keygen(None, 761, 0, 0, 4, None, None, None) == -1
    assert b"null context" in lib.snt_last_error_string()
    out = ctypes.c_void_p()
    assert lib.snt_ctx_create(0, 0, None) == -1
