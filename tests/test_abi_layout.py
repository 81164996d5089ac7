"""The binding's ctypes structures have the layout of include/cpt.h: a small C
program compiled against the header prints each structure's size and each
member's offset, and the ctypes side must agree member by member (a mismatch
would hand the library shifted arguments without any error).  A plain C client
links the library and calls its host-only entry points."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2510_25143_gb300 import cpt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "cpt_dims": cpt.Dims,
    "cpt_params": cpt.Params,
    "cpt_stats": cpt.Stats,
    "cpt_debug": cpt.Debug,
    "cpt_batch_stats": cpt.BatchStats,
    "cpt_trajs": cpt.Trajs,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cpt.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_ctypes_structures_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert C.sizeof(cls) == layout[(name, "sizeof")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)


def test_every_header_member_is_bound():
    """Each structure of the header has exactly the members the binding lists,
    in the same order."""
    import re
    src = open(os.path.join(ROOT, "include", "cpt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for name, cls in STRUCTS.items():
        m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", src)
        assert m, name
        members = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            decl = re.sub(r"\[[^\]]*\]", "", decl)         # array extents
            typ_and_first, *rest = decl.split(",")
            members.append(re.findall(r"[A-Za-z_]\w*", typ_and_first)[-1])
            members += [re.findall(r"[A-Za-z_]\w*", r)[-1] for r in rest]
        assert members == [f for f, _ in cls._fields_], name


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "cpt.h"

int main(void) {
    uint64_t freq[5] = {10, 0, 3, 3, 1};
    uint8_t len[5];
    if (cpt_huffman_lengths(freq, 5, 24, len) != CPT_OK) return 1;
    int32_t field[4] = {3, 40, 0, 0}; /* T = 3, H = 40: two strips, no prediction units */
    uint64_t n = 0;
    if (cpt_pipeline_order(1, field, NULL, NULL, &n) != CPT_OK || n != 6) return 2;
    int32_t items[18];
    if (cpt_pipeline_order(1, field, NULL, items, &n) != CPT_OK) return 3;
    if (cpt_compress(NULL, NULL, NULL, NULL, NULL, NULL) != CPT_ERR_ARG) return 4;
    printf("%u %s %u %u %u %u %u %d %d %d\n", (unsigned)(cpt_version() & 0xFFu), cpt_error_string(CPT_ERR_CORRUPT),
           len[0], len[1], len[2], len[3], len[4], items[0], items[1], items[2]);
    return 0;
}
"""


def test_plain_c_client_links_and_runs(tmp_path):
    """The boundary is a C ABI: a C11 program includes the header, links the
    built library and calls its host-only entry points (no GPU needed)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2510_25143_gb300 import build
    so = build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), so,
                    "-Wl,-rpath," + os.path.dirname(so), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == "1" and out[1:3] == ["corrupt", "stream"]
    assert [int(x) for x in out[3:8]] == list(cpt.huffman_lengths(np.array([10, 0, 3, 3, 1], np.uint64)))
    assert [int(x) for x in out[8:11]] == [0, 0, 0]  # the first item: field 0, slice 0, strip 0

