"""The C-ABI library loads on a machine without a GPU and exports every entry point
declared in include/lsamg.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lsamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsamg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_07485_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "lsamg_setup" in names and "lsamg_solve" in names and "lsamg_apply" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in lsamg.h but not exported"


def test_binding_lists_match_header():
    from paper_2607_07485_b300 import EXPORTS
    assert set(EXPORTS) <= set(_declared())


def test_options_default_matches_paper(lib):
    from paper_2607_07485_b300 import options
    o = options()
    assert o.tau_c == 0.75 and o.agg_passes == 2 and o.max_levels == 3
    assert o.min_coarse == 10 and o.max_density == 0.25 and o.rtol == 1e-8
