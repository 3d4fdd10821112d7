"""The Python binding restates the C ABI of include/mpl.h (enum values, struct
layouts, limits); this checks the restatement against the header text itself, so
that a key added on one side only fails here rather than as a wrong option on a
GPU."""
import ctypes
import os
import re

import pytest

from paper_1302_5010_gb300 import mpl

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mpl.h")


def _header():
    with open(HEADER) as f:
        text = f.read()
    # comments out (enum values and struct fields stay)
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def _enum_values(text):
    return {k: int(v) for k, v in re.findall(r"\b(MPL_[A-Z0-9_]+)\s*=\s*(-?\d+)\s*[,}\n]", text)}


def _struct_fields(text, name):
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if decl:
            ctype, field = decl.rsplit(None, 1)
            fields.append((field, ctype))
    return fields


def test_enum_values_match():
    vals = _enum_values(_header())
    assert len(vals) >= 30
    for k, v in vals.items():
        if hasattr(mpl, k):
            assert getattr(mpl, k) == v, k
    # every option, status and per-signal outcome of the header is bound
    for prefix in ("MPL_OPT_", "MPL_SIG_", "MPL_ERR_"):
        missing = [k for k in vals if k.startswith(prefix) and not hasattr(mpl, k)]
        assert not missing, missing


_CTYPES = {"int": ctypes.c_int32, "int32_t": ctypes.c_int32, "double": ctypes.c_double}


@pytest.mark.parametrize("cname,pyname", [("mpl_signal_stats_t", "SignalStats"), ("mpl_tune_result_t", "TuneResult")])
def test_struct_layouts_match(cname, pyname):
    fields = _struct_fields(_header(), cname)
    py = getattr(mpl, pyname)._fields_
    assert [f for f, _ in fields] == [f for f, _ in py]
    for (f, ctype), (_, pytype) in zip(fields, py):
        assert _CTYPES[ctype] == pytype, f
