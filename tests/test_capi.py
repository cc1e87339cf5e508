"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/otassign.h declares (CPU only: no compute calls)."""
import ctypes

import pytest


def test_library_exports_every_declared_symbol(lib_path):
    from paper_2005_01182_gb300 import otassign as ot
    names = ot.declared_symbols()
    for must in ("ot_assign_solve", "ot_assign_solve_batched", "ot_assign_submit", "ot_assign_poll",
                 "ot_ctx_create", "ot_ctx_destroy"):
        assert must in names
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    ot.load(lib_path)
    assert ot.ot_version().startswith("otassign")


def test_binding_covers_header():
    from paper_2005_01182_gb300 import otassign as ot
    for n in ot.declared_symbols():
        assert hasattr(ot, n), f"binding lacks {n}"


def test_no_cpu_fallback_in_product():
    # the product package never imports the oracle
    import pathlib
    import re
    pkg = pathlib.Path(__file__).resolve().parent.parent / "paper_2005_01182_gb300"
    for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")):
        txt = f.read_text()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
        assert "ot_oracle" not in txt and "liboracle" not in txt, f


def test_serving_client_library_builds_and_exports_replay(lib_path):
    """The host-only serving client that the served benchmark drives is built
    beside the library, links against it and exports its replay entry."""
    from paper_2005_01182_gb300 import build
    lib = ctypes.CDLL(build.CLIENT_LIB)
    assert hasattr(lib, "otc_replay")
    # argument checks return before any serving call
    lib.otc_replay.restype = ctypes.c_int
    total = ctypes.c_double()
    assert lib.otc_replay(None, 0, None, None, None, 0, None, 1, 0, None, None, ctypes.byref(total)) == -1
