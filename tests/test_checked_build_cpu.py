"""The bounds-checked build (SDEB_CHECKED) without a GPU: it compiles from
the same sources into libsdeb_checked.so, exports every declared entry
point, reports the status word's absence of a device as a CUDA error (no
GPU here), and the unchecked library answers the check calls with
SDEB_EUNSUPPORTED without a CUDA call."""
import ctypes
import os
import subprocess
import sys

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_unchecked_library_answers_unsupported():
    st, word = sdeb.sdeb_check_status()
    assert st == sdeb.SDEB_EUNSUPPORTED and word == 0
    assert sdeb.lib().sdeb_check_selftest(None) == sdeb.SDEB_EUNSUPPORTED
    assert "not a checked build" in sdeb.sdeb_last_error()


def test_checked_library_builds_and_exports_every_symbol():
    path = sdeb_build.build(checked=True)
    assert path.endswith("libsdeb_checked.so") and os.path.exists(path)
    L = ctypes.CDLL(path)
    for name in sdeb.EXPORTED_SYMBOLS:
        assert hasattr(L, name), name
    # the binding loads it under SDEB_LIBRARY=checked; without a GPU the
    # status read fails as a CUDA error, not a crash
    code = ("import sys; sys.path.insert(0, %r); import paper_1908_03869_gb300 as s; "
            "print(s.library_path()); st, w = s.sdeb_check_status(); print(st, w)") % ROOT
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, SDEB_LIBRARY="checked"),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    assert lines[0].endswith("libsdeb_checked.so")
    if not os.path.exists("/dev/nvidia0"):
        assert lines[1].split()[0] == str(sdeb.SDEB_ECUDA)
