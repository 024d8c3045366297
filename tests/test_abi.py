"""The C ABI library builds, loads, and exports every symbol include/sgn.h declares.

No GPU needed: only symbol lookup and the pure-host entry point sgn_kenney_laub."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"SGN_API\s+[\w\s\*]+?\b(sgn_\w+)\s*\(", txt)
    return names


@pytest.fixture(scope="module")
def libsgn():
    from paper_0910_2927_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libsgn):
    names = _declared()
    assert len(names) >= 19
    for name in names:
        assert hasattr(libsgn, name), f"{name} missing from libsgn.so"


def test_binding_covers_every_symbol():
    from paper_0910_2927_gb300 import _abi
    assert set(_declared()) == set(_abi.SIGNATURES)


def test_kenney_laub_matches_oracle_formula():
    """The library's eq. (6.2) against the oracle's (both written from the paper)."""
    import oracle as O
    import paper_0910_2927_gb300 as pkg
    for s, c in [(1, 1.0), (16, 0.43), (20, 0.21)]:
        sg, om = pkg.kenney_laub(s, c)
        so, oo = O.kenney_laub(s, c)
        np.testing.assert_allclose(sg, so, rtol=1e-15)
        np.testing.assert_allclose(om, oo, rtol=1e-15)


def test_kenney_laub_rejects_bad_arguments():
    import paper_0910_2927_gb300 as pkg
    with pytest.raises(pkg.SignError):
        pkg.kenney_laub(0, 1.0)
    with pytest.raises(pkg.SignError):
        pkg.kenney_laub(4, -1.0)


def test_version_string():
    import paper_0910_2927_gb300 as pkg
    assert b"sm_103a" in pkg.lib().sgn_version()


def test_enum_constants_match_header():
    """The binding's enum values are the ones include/sgn.h declares."""
    from paper_0910_2927_gb300 import _abi
    txt = open(os.path.join(ROOT, "include", "sgn.h")).read()
    vals = dict((k, int(v)) for k, v in re.findall(r"\b(SGN_LINKS_\w+|SGN_PREC_\w+)\s*=\s*(\d+)", txt))
    vals.update((k, int(v)) for k, v in re.findall(r"#define\s+(SGN_HW_\w+)\s+(\d+)", txt))
    for name in ("LINKS_FP32", "LINKS_BF16", "LINKS_FP16", "PREC_FP64", "PREC_MIXED", "HW_ADJOINT", "HW_PACKED",
                 "HW_FLOAT_FLOAT"):
        assert vals["SGN_" + name] == getattr(_abi, name), name
