"""The ctypes structures of the Python binding have the C header's layout: a small C
program compiled against include/phia.h prints every field's offset and each struct's
size, and the binding's ctypes.Structure must agree field by field (CPU only)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2407_10205_gb300 import phia

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("phia_opts", phia.Opts), ("phia_schedule", phia.Schedule), ("phia_stats", phia.Stats),
         ("phia_tune_result", phia.TuneResult), ("phia_instance_desc", phia.InstanceDesc),
         ("phia_server_opts", phia.ServerOpts), ("phia_request_status", phia.RequestStatus),
         ("phia_server_stats", phia.ServerStats), ("phia_gahmc_schedule", phia.GahmcSchedule)]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "phia.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in PAIRS:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
