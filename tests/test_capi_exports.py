"""The C-ABI library builds for sm_103a and exports every function that
include/*.h declares (no compute call: this runs without a GPU)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|int64_t|void|const char\*)\s+(caps_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("caps_build", "caps_search_batch", "caps_free", "caps_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2308_15014_gb300 import build as B
    path = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared() - exported
    assert not missing, f"not exported: {missing}"
    import paper_2308_15014_gb300 as caps
    assert set(caps.EXPORTS) == _declared()


def test_library_loads_and_reports_errors_without_gpu():
    import ctypes as ct
    import paper_2308_15014_gb300 as caps
    L = caps.lib()
    # argument checks run before any CUDA call
    rc = L.caps_search_batch(None, None, 0, None, 10, 4, None, None, None)
    assert rc == caps.CAPS_EINVAL
    assert b"null index" in L.caps_last_error()
    h = ct.c_void_p()
    assert L.caps_build(None, None, 0, 0, None, None, ct.byref(h)) == caps.CAPS_EINVAL
