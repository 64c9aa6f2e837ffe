"""The C-ABI library builds, loads and exports every symbol its header declares
(no GPU needed: nothing here launches device work)."""
import os
import re
import subprocess

import pytest

import paper_2409_17299_gb300 as q
from paper_2409_17299_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"\b(qed_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_builds_and_exports_header_symbols():
    lib = b.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (qed_[a-z_0-9]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, declared - exported
    assert set(q.EXPORTED) == declared


def test_library_loads_and_strerror():
    b.build()
    L = q.lib()
    for name in q.EXPORTED:
        assert hasattr(L, name)
    assert q.qed_strerror(q.QED_ERR_CAPACITY) == "particle buffer capacity exceeded"
    assert q.qed_strerror(0) == "ok"


def test_sm103a_only_build_flags():
    assert "arch=compute_103a,code=sm_103a" in b.ARCH
