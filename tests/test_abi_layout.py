"""The Python binding and include/gsync.h describe the same ABI: every struct the binding
passes has the C compiler's size and field offsets, and every function the binding declares
takes as many arguments as its C prototype (CPU only: gcc compiles a layout printer)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsync.h")


def _structs():
    from paper_1110_4623_gb300 import gsync as G
    return {name: obj for name, obj in vars(G).items()
            if isinstance(obj, type) and issubclass(obj, ctypes.Structure) and name.startswith("gsync_")}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """{struct: (sizeof, {field: offsetof})} as gcc lays them out."""
    structs = _structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gsync.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("%s size %zu\\n", "{name}", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("%s %s %zu\\n", "{name}", "{field}", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        size, offsets = layout.setdefault(name, [0, {}])
        if field == "size":
            layout[name][0] = int(value)
        else:
            offsets[field] = int(value)
    return layout


def test_every_struct_matches_the_c_layout(c_layout):
    structs = _structs()
    assert set(structs) == set(c_layout)
    for name, cls in structs.items():
        size, offsets = c_layout[name]
        assert ctypes.sizeof(cls) == size, name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == offsets[field], (name, field)


def test_binding_covers_every_c_struct_it_passes():
    # each typedef'd struct of the header that a function takes by pointer has a binding
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    c_structs = set(re.findall(r"typedef struct (gsync_\w+)", src))
    assert c_structs <= set(_structs()), c_structs - set(_structs())


def _prototypes():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    protos = {}
    for m in re.finditer(r"^\s*(?:int|size_t|void|uint32_t|uint64_t)\s+\**\s*(gsync_\w+)\s*\(([^)]*)\)\s*;", src,
                         flags=re.M):
        args = " ".join(m.group(2).split())
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return protos


def test_binding_argument_counts_match_the_prototypes():
    from paper_1110_4623_gb300 import gsync as G
    protos = _prototypes()
    from test_capi_symbols import declared_functions
    assert set(protos) == set(declared_functions())  # the parser saw every prototype
    for name, nargs in protos.items():
        assert name in G._SIG, name
        assert len(G._SIG[name][1]) == nargs, (name, len(G._SIG[name][1]), nargs)
