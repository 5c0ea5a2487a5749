"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sesw.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(sesw_\w+)\s*\(", txt, re.M)))


def test_header_declarations_are_the_binding_exports():
    from paper_2311_08241_gb300 import sesw

    assert _declared() == sorted(sesw.EXPORTS)


def test_library_loads_and_exports_every_symbol():
    from paper_2311_08241_gb300 import build

    path = build.build()
    L = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sesw_\w+)", out))
    assert set(_declared()) <= exported


def test_library_is_built_for_sm_103a():
    from paper_2311_08241_gb300 import build

    path = build.build()
    out = subprocess.run(["cuobjdump", "--list-elf", path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_create_without_gpu_fails_cleanly():
    """Without a usable device the library returns an error code instead of crashing."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2311_08241_gb300 import sesw

    L = sesw.load()
    h = ctypes.c_void_p()
    rc = L.sesw_create(ctypes.byref(h), 0, None, sesw.ALLOC_FN(0), sesw.FREE_FN(0), None)
    assert rc == sesw.SESW_ECUDA and not h.value
