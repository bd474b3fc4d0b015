"""CPU checks of the boundary: the C-ABI library builds, loads and exports
every entry point declared in include/gbp.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2308_08410_gb300 import build, gbp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "gbp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(gbp_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(gbp.exported_symbols()) == set(names)


def test_status_strings_without_gpu():
    lib = gbp.load()
    for s in range(10):
        assert lib.gbp_status_string(s)


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        gbp.Context(0)


PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "gbp.h"
#define F(T, m) printf("%s.%s %zu %zu\n", #T, #m, offsetof(T, m), sizeof(((T *)0)->m))
int main(void)
{
    printf("sizeof gbp_solve_opts %zu\n", sizeof(gbp_solve_opts));
    printf("sizeof gbp_solve_stats %zu\n", sizeof(gbp_solve_stats));
    printf("sizeof gbp_template %zu\n", sizeof(gbp_template));
    F(gbp_solve_opts, local_solver); F(gbp_solve_opts, n_f); F(gbp_solve_opts, eps); F(gbp_solve_opts, max_iters);
    F(gbp_solve_stats, iterations); F(gbp_solve_stats, candidates); F(gbp_solve_stats, face_updates);
    F(gbp_solve_stats, fp64_fallbacks); F(gbp_solve_stats, unreached); F(gbp_solve_stats, adj_levels);
    F(gbp_solve_stats, adj_cycle_nodes); F(gbp_solve_stats, adj_cycle_iters); F(gbp_solve_stats, status);
    F(gbp_solve_stats, reserved); F(gbp_solve_stats, adj_dataflow_ms); F(gbp_solve_stats, adj_cycle_ms);
    F(gbp_solve_stats, fim_deferred); F(gbp_solve_stats, fim_repaired);
    F(gbp_template, K0); F(gbp_template, K1); F(gbp_template, tau); F(gbp_template, t0); F(gbp_template, dt);
    F(gbp_template, T);
    printf("const LOCAL_EXACT %d\nconst LOCAL_FISTA %d\n", GBP_LOCAL_EXACT, GBP_LOCAL_FISTA);
    printf("const ONSET_NODAL %d\nconst ONSET_ELEMENT %d\n", GBP_ONSET_NODAL, GBP_ONSET_ELEMENT);
    printf("const PREC_FP32 %d\nconst PREC_BF16 %d\n", GBP_PREC_FP32, GBP_PREC_BF16);
    printf("const STATUS_LAST %d\n", (int)GBP_ERR_NO_MEMORY);
    return 0;
}
"""


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes structures and constants of gbp.py have the header's field
    offsets, sizes and enum values (a C probe compiled with gcc prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "probe.c"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    structs = {"gbp_solve_opts": gbp.SolveOpts, "gbp_solve_stats": gbp.SolveStats, "gbp_template": gbp.Template}
    seen = 0
    for line in filter(None, out):
        a, *vals = line.split()
        if a == "sizeof":
            assert ctypes.sizeof(structs[vals[0]]) == int(vals[1]), line
        elif a == "const":
            if vals[0] == "STATUS_LAST":
                assert max(gbp._STATUS) == int(vals[1])
            else:
                assert getattr(gbp, vals[0]) == int(vals[1]), line
        else:
            sname, field = a.split(".")
            desc = getattr(structs[sname], field)
            assert (desc.offset, desc.size) == (int(vals[0]), int(vals[1])), line
        seen += 1
    assert seen == 3 + 24 + 7


def _c_kind(decl):
    decl = decl.strip()
    if "*" in decl:
        return "ptr"
    toks = decl.replace("const ", "").split()
    t = toks[0] if toks else "void"
    return {"int64_t": "i64", "int32_t": "i32", "int": "i32", "float": "f32", "double": "f64",
            "gbp_status": "i32", "void": None}[t]


def _ctypes_kind(t):
    if t is None:
        return None
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    if t is ctypes.c_float:
        return "f32"
    if t is ctypes.c_double:
        return "f64"
    return "i%d" % (8 * ctypes.sizeof(t))


def test_binding_signatures_match_the_header():
    """Every prototype of include/gbp.h has the arity, argument widths
    (pointer / 32- / 64-bit integer / float) and return kind that the
    binding's argtypes and restype give it."""
    hdr = open(os.path.join(ROOT, "include", "gbp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    hdr = re.sub(r"//[^\n]*", "", hdr)
    protos = re.findall(r"([A-Za-z_][\w \t\*]*?)\b(gbp_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", hdr)
    lib = gbp.load()
    checked = 0
    for ret, name, params in protos:
        params = " ".join(params.split())
        cargs = [] if params in ("", "void") else [_c_kind(p) for p in params.split(",")]
        fn = getattr(lib, name)
        assert [_ctypes_kind(a) for a in fn.argtypes] == cargs, name
        assert _ctypes_kind(fn.restype) == _c_kind(ret.replace("static", "")), name
        checked += 1
    assert checked == len(gbp.exported_symbols())
