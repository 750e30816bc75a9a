"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(CPU only; no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2512_00233_gb300 as K
from paper_2512_00233_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions() -> set[str]:
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(kcore_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_for_sm103a():
    path = _build.build()
    assert os.path.exists(path)
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 20
    handle = ctypes.CDLL(_build.build())
    missing = [n for n in sorted(names) if not hasattr(handle, n)]
    assert not missing, missing


def test_python_binding_covers_every_symbol():
    assert declared_functions() <= set(_lib.SIGNATURES)


def test_defaults_and_version():
    o = K.default_options()
    assert o.struct_size == ctypes.sizeof(K.Options)
    assert (o.t_lo, o.t_hi, o.block) == (16, 2048, 512)
    assert o.timeout_s > 0
    assert o.build_sort == 0
    assert "sm_103a" in K.version()
    s = K.default_serve_options()
    assert s.struct_size == ctypes.sizeof(K.ServeOptions)
    assert s.host_staging == 1 << 30


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's size and offsets."""
    import subprocess
    structs = {"kcore_options": K.Options, "kcore_run_stats": K.RunStats,
               "kcore_serve_options": K.ServeOptions, "kcore_batch_stats": K.BatchStats,
               "kcore_ticket_info": K.TicketInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kcore.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_no_oracle_import_in_library():
    pkg = os.path.join(ROOT, "paper_2512_00233_gb300")
    for p in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if p.endswith((".py", ".cu", ".cuh", ".h")):
            assert "oracle" not in open(p).read().lower().replace("oracles", ""), p
