"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every symbol the
headers declare (no compute call: there is no GPU here)."""

import ctypes
import os
import re

import pytest

from paper_2604_00037_gb300 import binding, buildlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in ("aci.h", "aci_kernels.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(aci_[a-z_0-9]+)\s*\(", src))
    return names - {"aci_alloc_fn", "aci_free_fn"}


def test_library_builds_and_exports_every_declared_symbol():
    path = buildlib.build()
    lib = ctypes.CDLL(path)
    decl = declared_symbols()
    assert decl == set(binding.EXPORTS), decl ^ set(binding.EXPORTS)
    for name in decl:
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # sizes implied by include/aci.h on LP64
    assert ctypes.sizeof(binding.AciOp) == 8 + 64
    assert ctypes.sizeof(binding.AciTT) == 16 + 24
    assert ctypes.sizeof(binding.AciOpts) == 16 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(binding.AciStats) == 16 + 32 + 8 + 32 + 32 + 32 + 32 + 32


def test_product_path_has_no_cpu_fallback():
    # the package never imports the oracle, and the context refuses to start without CUDA
    import paper_2604_00037_gb300 as pkg
    src = "".join(open(os.path.join(os.path.dirname(pkg.__file__), f)).read()
                  for f in os.listdir(os.path.dirname(pkg.__file__)) if f.endswith(".py"))
    assert "oracle" not in src.replace("oracle/", "")
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            pkg.Context(0)
