"""The C-ABI library loads on a machine without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2606_25569_b300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_declares_every_symbol():
    from paper_2606_25569_b300 import binding
    assert set(_declared()) == set(binding.FUNCTIONS)


def test_invalid_arguments_rejected_without_gpu():
    import numpy as np
    from paper_2606_25569_b300 import binding
    with pytest.raises(binding.VsError) as e:
        binding.Suspension(np.zeros(2 * 7), [0, 7])
    assert e.value.status == 1  # odd N is rejected before any CUDA call
