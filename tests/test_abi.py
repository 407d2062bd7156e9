"""The C-ABI library: every symbol declared in include/*.h is exported (no GPU calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(fp_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("fp_init", "fp_modes", "fp_set_modes", "fp_rates4", "fp_rates4_device", "fp_free", "fp_last_error"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2104_04895_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in sorted(declared_symbols()):
        assert hasattr(lib, n), n
    from paper_2104_04895_gb300 import binding
    L = binding.load()
    assert L.fp_version() >= 10000
    for n in binding.EXPORTS:
        assert n in declared_symbols()


def test_init_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2104_04895_gb300 import binding, synth
    with pytest.raises(binding.FourPhononError) as ei:
        binding.Context.from_crystal(synth.simple_cubic((2, 2, 2)))
    assert ei.value.code in (binding.FP_ECUDA, binding.FP_EINVAL)
