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


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program compiled against lsamg.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lsamg.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("name,struct", [("Options", "lsamg_options"), ("Problem", "lsamg_problem"),
                                         ("Stats", "lsamg_stats")])
def test_binding_structs_match_header_layout(name, struct, tmp_path):
    from paper_2607_07485_b300 import lsamg as LB
    cls = getattr(LB, name)
    fields = [f for f, _ in cls._fields_]
    size, offs = _c_layout(struct, fields, tmp_path)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_new_option_defaults(lib):
    from paper_2607_07485_b300 import options
    o = options()
    assert o.smoother == 0 and o.sweep_block == 0 and o.split_sweep == 0 and o.use_graph == 0


def test_closure_option(lib):
    # 0 = G-row closure (the paper's method, the default), 1 = algebraic A-closure (Def. 5.2)
    from paper_2607_07485_b300 import options
    assert options().closure == 0
    assert options(closure="A").closure == 1 and options(closure="G").closure == 0
    with pytest.raises(ValueError):
        options(closure="B")
