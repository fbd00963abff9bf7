"""The C-ABI library builds, loads and exports every symbol that
include/npsolve.h declares (no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

from paper_2310_00177_b300 import binding
from paper_2310_00177_b300 import build as nbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            syms |= set(re.findall(r"\b(npsolve_\w+)\s*\(", text))
    return syms


def test_library_builds_and_exports_every_declared_symbol():
    path = nbuild.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (npsolve_\w+)", out))
    declared = declared_symbols()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_the_header_and_loads():
    lib = binding.load_library()
    declared = declared_symbols()
    assert declared == set(binding.SIGNATURES), set(binding.SIGNATURES) ^ declared
    for name in declared:
        assert getattr(lib, name) is not None
