"""The C-ABI library builds, loads and exports every entry point that
include/rt.h declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1206_3710_gb300 import build
    return build.build()


def test_library_exports_all_declared_symbols(built_lib):
    names = declared_functions()
    assert "rt_trace" in names and "rt_peel" in names and "rt_build_grid" in names
    assert "rt_dust_temperature" in names
    L = ctypes.CDLL(built_lib)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rt_[a-z_0-9]+)", out))
    assert set(names) <= exported


def test_binding_covers_header(built_lib):
    from paper_1206_3710_gb300 import rt
    assert set(declared_functions()) <= set(rt.EXPORTED)
    rt.lib()
    assert b"sm_103a" in rt.lib().rt_version()


def test_binding_struct_sizes_match_header(built_lib):
    """The ctypes mirrors have the C layout (checked against a tiny C probe
    compiled from the header with gcc)."""
    import tempfile

    from paper_1206_3710_gb300 import rt
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "rt.h"
int main(void){
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(rt_tree_desc), sizeof(rt_grid_info),
         sizeof(rt_optics), sizeof(rt_dust), sizeof(rt_source), sizeof(rt_trace_params), sizeof(rt_ledger),
         sizeof(rt_observers), offsetof(rt_trace_params, packet_log_dev), offsetof(rt_trace_params, hits_dev),
         sizeof(rt_lambda_params), sizeof(rt_lambda_result), sizeof(rt_job), sizeof(rt_tune_result),
         sizeof(rt_server_config), sizeof(rt_serve_job));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    mine = [ctypes.sizeof(rt.rt_tree_desc), ctypes.sizeof(rt.rt_grid_info), ctypes.sizeof(rt.rt_optics),
            ctypes.sizeof(rt.rt_dust), ctypes.sizeof(rt.rt_source), ctypes.sizeof(rt.rt_trace_params),
            ctypes.sizeof(rt.rt_ledger), ctypes.sizeof(rt.rt_observers), rt.rt_trace_params.packet_log_dev.offset,
            rt.rt_trace_params.hits_dev.offset, ctypes.sizeof(rt.rt_lambda_params), ctypes.sizeof(rt.rt_lambda_result),
            ctypes.sizeof(rt.rt_job), ctypes.sizeof(rt.rt_tune_result), ctypes.sizeof(rt.rt_server_config),
            ctypes.sizeof(rt.rt_serve_job)]
    assert vals == mine


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1206_3710_gb300 import rt
    monkeypatch.setattr(rt, "_lib", None)
    monkeypatch.setattr(rt, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        rt.lib()


STRUCTS = ["rt_tree_desc", "rt_grid_info", "rt_optics", "rt_dust", "rt_source", "rt_trace_params", "rt_ledger",
           "rt_observers", "rt_job", "rt_tune_result", "rt_server_config", "rt_serve_job", "rt_lambda_params",
           "rt_lambda_result", "rt_subiter_params", "rt_subiter_result"]


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors in the binding have the sizes and field offsets of
    the C structs in include/rt.h (compiled with the host C compiler)."""
    from paper_1206_3710_gb300 import rt
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rt.h"', 'int main(void) {']
    checks = []
    for s in STRUCTS:
        cls = getattr(rt, s)
        lines.append(f'  printf("%zu\\n", sizeof({s}));')
        checks.append((s, None, ctypes.sizeof(cls)))
        for name, _ in cls._fields_:
            cname = "lambda" if (s == "rt_subiter_result" and name == "lambda_") else name
            lines.append(f'  printf("%zu\\n", offsetof({s}, {cname}));')
            checks.append((s, name, getattr(cls, name).offset))
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert len(out) == len(checks)
    bad = [(s, f, int(v), want) for (s, f, want), v in zip(checks, out) if int(v) != want]
    assert not bad, bad


def test_binding_declares_every_argument_list(built_lib):
    """Every entry point the binding calls has its argument types declared:
    without them ctypes passes Python ints (device pointers, streams) as
    32-bit C ints, and the library would see truncated addresses."""
    from paper_1206_3710_gb300 import rt
    L = rt.lib()
    missing = [n for n in rt.EXPORTED if getattr(L, n).argtypes is None]
    assert not missing, missing
