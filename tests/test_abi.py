"""The C ABI library loads on the CPU and exports every declared symbol."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(vqe_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(lib_built):
    from paper_2402_11878_gb300 import binding
    lib = ctypes.CDLL(binding.library_path())
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTED) == names


def test_version_and_layouts(lib_built):
    import paper_2402_11878_gb300 as pkg
    from paper_2402_11878_gb300 import plans
    assert "sm_103a" in pkg.version()
    plans.plan(8, 2, "c64")     # checks record sizes against the library


def test_create_fails_loudly_without_gpu(lib_built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2402_11878_gb300 as pkg
    with pytest.raises(pkg.VQEError) as ei:
        pkg.Engine(8, 2, "c64")
    assert ei.value.status == 4


def test_create_argument_checks(lib_built):
    from paper_2402_11878_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    for n, d, p in [(0, 1, 0), (33, 1, 0), (8, 0, 0), (8, 1, 7)]:
        assert lib.vqe_create(n, d, p, None, ctypes.byref(h)) == 1
    assert lib.vqe_create(8, 1, 0, None, None) == 1
