"""The C-ABI library builds, loads, and exports every symbol that
include/pamo.h declares; the ctypes structures match the C layouts.
No GPU needed (nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "pamo.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pamo_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_05595_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pamo_simplify", "pamo_ctx_create", "pamo_round_cost", "pamo_round_select",
              "pamo_round_collapse", "pamo_round_check_undo", "pamo_round_commit",
              "pamo_ctx_export", "pamo_ctx_destroy", "pamo_check_self_intersections",
              "pamo_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(pamo_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_resolves(libpath):
    import paper_2509_05595_gb300 as pamo
    L = pamo.lib()
    for n in _declared():
        assert hasattr(L, n)
    o = pamo._Options()
    L.pamo_default_options(ctypes.byref(o))
    assert (o.w_e, o.w_s, o.tolerance) == (0.001, 0.005, 4)
    assert (o.exact_target, o.max_cost) == (0, float("inf"))
    assert pamo.Options().c().tolerance == o.tolerance


def test_struct_layouts_match_c(tmp_path):
    import paper_2509_05595_gb300 as pamo
    prog = tmp_path / "sz.c"
    prog.write_text('#include "pamo.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(){printf("%zu %zu %zu %zu\\n", sizeof(pamo_options), '
                    'sizeof(pamo_stats), offsetof(pamo_stats, committed), '
                    'offsetof(pamo_options, device_loop));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    a, b, c, d = map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                         check=True).stdout.split())
    assert a == ctypes.sizeof(pamo._Options)
    assert b == ctypes.sizeof(pamo._Stats)
    assert c == pamo._Stats.committed.offset
    assert d == pamo._Options.device_loop.offset


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2509_05595_gb300 as pamo
    monkeypatch.setattr(pamo, "_lib", None)
    monkeypatch.setattr(pamo, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pamo.lib()
