"""The binding's ctypes structures against the C header: a small C program,
compiled with the host compiler against include/dgh.h, prints sizeof and
offsetof of every field the binding declares (a field the header lacks
fails to compile), and each must equal ctypes' own layout.  CPU only."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1610_05023_b300 as dgh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"dgh_desc": dgh._Desc, "dgh_info": dgh._Info, "dgh_launch": dgh._Launch, "dgh_train_cfg": dgh._TrainCfg}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_binding_structures_match_the_header(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dgh.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append('    printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in py._fields_:
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            *key, val = line.split()
            got[tuple(key)] = int(val)
    for cname, py in STRUCTS.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
