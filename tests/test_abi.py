"""The C-ABI library builds, loads and exports every symbol include/ocsc.h
declares (CPU only: no compute calls)."""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ocsc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ocsc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1706_06972_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["ocsc_init", "ocsc_code", "ocsc_update_dict", "ocsc_get_dict", "ocsc_set_dict",
                 "ocsc_destroy", "ocsc_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ocsc_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol(libpath):
    import paper_1706_06972_gb300 as pkg

    L = pkg.lib()
    for n in declared_functions():
        assert hasattr(L, n)
        assert n in pkg.EXPORTED


def test_no_cpu_fallback_in_binding():
    """The product package never imports the oracle."""
    pkgdir = os.path.join(ROOT, "paper_1706_06972_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src


def test_init_without_gpu_fails_cleanly(libpath):
    """Without a GPU, ocsc_init returns an error status instead of aborting."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1706_06972_gb300 as pkg

    with pytest.raises(pkg.OCSCError):
        pkg.ocsc_init(4, 3, 3, 1.0, 1.0)
