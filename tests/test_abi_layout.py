"""The binding's record and option layouts against the C header (CPU):
a small C program compiled with the system compiler against include/epi.h
prints each struct's size and field offsets, which must equal those of the
ctypes structures and of the numpy record type in the binding."""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELDS = {
    "epi_result": ["snp", "mi", "mi_f32", "order", "rank"],
    "epi_proposer_opts": ["top_triples", "budget", "top_n", "chunk", "quad_features"],
    "epi_proposer_stats": ["candidates", "kept", "proposals", "ms_lower", "ms_rank", "ms_rescore",
                           "exact_in_proposals"],
    "epi_train_opts": ["top_triples", "epochs", "batch", "lr", "wd", "tail_fraction", "seed", "target"],
}


def _c_layouts(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "epi.h"', "int main(void) {"]
    for name, fields in FIELDS.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'    printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, key, val = line.split()
        got[(name, key)] = int(val)
    return got


def test_struct_layouts_match_the_header(tmp_path):
    from paper_2201_02460_gb300 import epi
    c = _c_layouts(tmp_path)
    py = {"epi_proposer_opts": epi.ProposerOpts, "epi_proposer_stats": epi.ProposerStats,
          "epi_train_opts": epi.TrainOpts}
    for name, cls in py.items():
        assert C.sizeof(cls) == c[(name, "size")], name
        for f in FIELDS[name]:
            assert getattr(cls, f).offset == c[(name, f)], (name, f)
    rd = epi.RESULT_DTYPE
    assert rd.itemsize == c[("epi_result", "size")]
    for f in FIELDS["epi_result"]:
        assert rd.fields[f][1] == c[("epi_result", f)], f
