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
    assert ctypes.sizeof(binding.AciOpts) == 16 + 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(binding.AciStats) == 16 + 32 + 8 + 32 + 32 + 32 + 32 + 32 + 24


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


def _header():
    return re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "aci.h")).read(), flags=re.S)


def _enum_values(src, prefix):
    return {m.group(1): int(m.group(2)) for m in re.finditer(rf"\b({prefix}[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_binding_enums_match_header():
    src = _header()
    piv = _enum_values(src, "ACI_PIVOT_")
    assert {k: piv["ACI_PIVOT_" + k.upper()] for k in binding.PIVOT_MODES} == binding.PIVOT_MODES
    ovl = _enum_values(src, "ACI_OVERLAP_")
    assert {k: ovl["ACI_OVERLAP_" + k.upper()] for k in binding.OVERLAP_MODES} == binding.OVERLAP_MODES
    prec = _enum_values(src, "ACI_PREC_")
    assert {k: prec["ACI_PREC_" + k.upper()] for k in binding.PRECISIONS} == binding.PRECISIONS


def test_opts_fields_match_header_order():
    src = _header()
    body = re.search(r"typedef struct \{([^{}]*?)\} aci_opts;", src, flags=re.S).group(1)
    fields = [m.group(1) for m in re.finditer(r"\b(?:int32_t|uint64_t|double)\s+(\w+)\s*;", body)]
    fields += [m.group(1) for m in re.finditer(r"const aci_tt \*(\w+)\s*;", body)]
    names = [f[0] for f in binding.AciOpts._fields_]
    assert sorted(names) == sorted(fields), (names, fields)
    # declaration order (pointers included) is the struct's memory order
    order = [m.group(1) for m in re.finditer(r"(?:int32_t|uint64_t|double|const aci_tt \*)\s*(\w+)\s*;", body)]
    assert names == order, (names, order)
