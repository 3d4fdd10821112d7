"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

from paper_1302_5010_gb300 import build as libbuild
from paper_1302_5010_gb300 import mpl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_header():
    lib = libbuild.build()
    assert os.path.exists(lib)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    declared = _declared()
    assert {"mpl_create", "bmpl_solve", "mpl_destroy"} <= declared
    missing = declared - exported
    assert not missing, f"declared but not exported: {missing}"
    assert set(mpl.EXPORTED) <= exported


def test_binding_loads_and_status_strings():
    lib = mpl.load()
    assert isinstance(lib, ctypes.CDLL)
    assert mpl.mpl_status_string(0) == "ok"
    assert "not certified" in mpl.mpl_status_string(5)


def test_null_handle_is_rejected():
    lib = mpl.load()
    # argument validation happens before any device work
    assert lib.bmpl_solve(None, None, 0, None, None, 1e-6, None) == mpl.MPL_ERR_ARG
    assert lib.mpl_set_option(None, 0, 1.0) == mpl.MPL_ERR_ARG
    lib.mpl_destroy(None)
