"""The Python binding agrees with include/fourphonon.h (no GPU calls).

A small C program compiled against the header prints the size and the field offsets of every struct of the
boundary and the value of every FP_* constant; the binding's ctypes structures and constants must match them, so
a field added to the header but not to the binding (or the reverse) fails here rather than corrupting a call.
The host-only entry points that fill defaults are called and checked against their documented values.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fourphonon.h")

STRUCTS = ["fp_fc2", "fp_fc4", "fp_fc3", "fp_rates_opts", "fp_stats", "fp_surrogate_opts", "fp_surrogate_report"]


def header_text():
    with open(HEADER) as f:
        return f.read()


def struct_fields(text, name):
    """Field names of `typedef struct { ... } name;` in declaration order (comments removed)."""
    code = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", code)
    assert body, name
    decl = body.group(1)
    fields = []
    for stmt in decl.split(";"):
        if not stmt.strip():
            continue
        parts = [re.sub(r"\[.*?\]", "", p).replace("*", " ").split() for p in stmt.split(",")]
        fields.append(parts[0][-1])                 # the first declarator follows the type
        fields += [p[0] for p in parts[1:]]
    return fields


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    text = header_text()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fourphonon.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("size {s} %zu\\n", sizeof({s}));')
        for fld in struct_fields(text, s):
            lines.append(f'  printf("off {s} {fld} %zu\\n", offsetof({s}, {fld}));')
    consts = re.findall(r"#define (FP_[A-Z0-9_]+) ", text)
    for c in consts:
        lines.append(f'  printf("const {c} %d\\n", (int){c});')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", exe, src])
    out = {"size": {}, "off": {}, "const": {}}
    for ln in subprocess.check_output([exe], text=True).splitlines():
        kind, *rest = ln.split()
        if kind == "size":
            out["size"][rest[0]] = int(rest[1])
        elif kind == "off":
            out["off"][(rest[0], rest[1])] = int(rest[2])
        else:
            out["const"][rest[0]] = int(rest[1])
    return out


def test_struct_layouts_match_the_header(layout):
    from paper_2104_04895_gb300 import binding
    text = header_text()
    for s in STRUCTS:
        cls = getattr(binding, s)
        names = [f[0] for f in cls._fields_]
        assert names == struct_fields(text, s), s
        assert ctypes.sizeof(cls) == layout["size"][s], s
        for n in names:
            assert getattr(cls, n).offset == layout["off"][(s, n)], (s, n)


def test_constants_match_the_header(layout):
    from paper_2104_04895_gb300 import binding
    for name, value in layout["const"].items():
        assert getattr(binding, name) == value, name


def test_host_defaults():
    from paper_2104_04895_gb300 import binding
    L = binding.load()
    o = binding.fp_rates_opts()
    L.fp_default_opts(ctypes.byref(o))
    assert (o.precision, o.window, o.sigma_min, o.dq_mode, bool(o.mode_mask)) == (binding.FP_PREC_FP64, 2.0, 1e-10,
                                                                                    0, False)
    assert (o.q_begin, o.q_end, o.no_graph, o.process_mask, o.nu_select, o.no_time_reversal, o.tensor_cores) == \
        (0, 0, 0, 0, 0, 0, 0)
    s = binding.fp_surrogate_opts()
    L.fp_surrogate_default_opts.argtypes = [ctypes.POINTER(binding.fp_surrogate_opts)]
    L.fp_surrogate_default_opts(ctypes.byref(s))
    assert (s.train_frac, s.holdout_frac, s.tol, s.epochs, s.batch, s.lr, s.precision) == \
        (0.10, 0.05, 0.05, 400, 1024, 2e-3, binding.FP_PREC_MIXED)
    import oracle.mlp as om
    L.fp_mlp_params_size.argtypes = [ctypes.c_int]
    for F in (1, 7, 19):
        assert L.fp_mlp_params_size(F) == om.n_params(F)
