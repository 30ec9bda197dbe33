"""The Python binding against include/cosma.h, without a GPU: every prototype's
parameters and result have the kind and width of the binding's ctypes
signature, and the binding's structures have the header's field offsets and
sizes as gcc lays them out, and the enumerators carry the values the binding
uses (a mismatch would pass garbage through the ABI)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cosma.h")

# width and kind of the scalar C types the header uses
C_SCALARS = {"int": ("i", 4), "unsigned": ("i", 4), "unsigned int": ("i", 4),
             "int64_t": ("i", 8), "long long": ("i", 8), "size_t": ("i", 8),
             "double": ("f", 8), "float": ("f", 4), "void": ("v", 0)}


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def prototypes():
    text = _strip_comments(open(HEADER).read())
    out = {}
    for ret, name, params in re.findall(
            r"^\s*((?:const\s+)?[A-Za-z_][\w ]*?\**)\s*\b(cosma_\w+)\s*\(([^)]*)\)\s*;", text,
            flags=re.M | re.S):
        params = " ".join(params.split())
        out[name] = (ret.strip(), [] if params in ("", "void") else
                     [p.strip() for p in params.split(",")])
    return out


def c_kind(decl, has_name=True):
    """(kind, bytes) of a C declaration: 'p' pointer, 'i' integer, 'f' float, 'v' void."""
    if "*" in decl or "[" in decl:
        return ("p", 8)
    words = [w for w in decl.replace("const", " ").split() if w]
    if has_name and len(words) > 1:
        words = words[:-1]   # drop the parameter name
    return C_SCALARS[" ".join(words)]


def ctypes_kind(t):
    if t is None:
        return ("v", 0)
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return ("p", 8)
    if t in (ctypes.c_float, ctypes.c_double):
        return ("f", ctypes.sizeof(t))
    return ("i", ctypes.sizeof(t))


@pytest.fixture(scope="module")
def binding():
    from paper_1908_09606_gb300 import cosma
    return cosma


def test_every_prototype_matches_the_binding(binding):
    protos = prototypes()
    sigs = {name: (res, args) for name, res, args in binding.SIGNATURES}
    assert len(protos) >= 30
    assert set(protos) == set(sigs), set(protos) ^ set(sigs)
    for name, (ret, params) in protos.items():
        res, args = sigs[name]
        assert c_kind(ret, has_name=False) == ctypes_kind(res), name
        assert len(params) == len(args), name
        for i, (p, a) in enumerate(zip(params, args)):
            assert c_kind(p) == ctypes_kind(a), (name, i, p, a)


def test_struct_layouts_match_gcc(binding, tmp_path):
    structs = [binding.cosma_config, binding.cosma_plan, binding.cosma_problem]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cosma.h"', "int main(void) {"]
    for s in structs:
        name = s.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in s._fields_:
            lines.append(f'  printf("{name} {field} %zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name}*)0)->{field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER),
                    str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    table = {}
    for line in got:
        w = line.split()
        if len(w) == 3:
            table[(w[0], "size")] = int(w[2])
        elif len(w) == 4:
            table[(w[0], w[1])] = (int(w[2]), int(w[3]))
    for s in structs:
        name = s.__name__
        assert ctypes.sizeof(s) == table[(name, "size")], name
        for field, t in s._fields_:
            assert (getattr(s, field).offset, ctypes.sizeof(t)) == table[(name, field)], \
                (name, field)


def _enums():
    text = _strip_comments(open(HEADER).read())
    out = {}
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}\s*\w+\s*;", text, flags=re.S):
        for name, value in re.findall(r"(COSMA_\w+)\s*=\s*(-?\d+)", body):
            out[name] = int(value)
    return out


def test_enum_values_match_the_binding(binding):
    enums = _enums()
    assert len(enums) >= 20
    # the binding's dtype names map to the header's enumerators
    assert binding.DTYPES == {name.lower(): enums["COSMA_" + name.upper()] for name in
                              binding.DTYPES}
    for name, value in enums.items():
        if hasattr(binding, name):
            assert getattr(binding, name) == value, name
    kernels = {v: k[len("COSMA_KERNEL_"):].lower() for k, v in enums.items()
               if k.startswith("COSMA_KERNEL_")}
    assert kernels == binding.KERNELS
    for s in ("OK", "ERR_INVALID_ARG", "ERR_UNSUPPORTED", "ERR_CUDA", "ERR_TIMEOUT",
              "ERR_NONFINITE", "ERR_NO_WORKSPACE"):
        assert getattr(binding, "COSMA_" + s) == enums["COSMA_" + s]
