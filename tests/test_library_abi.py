"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/cd.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1304_4453_gb300 import build, cd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(cd_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cd_graph_create", "cd_plp", "cd_plm", "cd_epp", "cd_modularity"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header():
    for n in declared_functions():
        if n in ("cd_opts_default", "cd_status_str", "cd_last_error"):
            continue
        assert hasattr(cd, n), n


def test_status_strings_without_gpu():
    L = cd.lib()
    assert L.cd_status_str(0) == b"CD_OK"
    assert L.cd_status_str(4) == b"CD_ENOTCONV"
    o = cd.default_opts()
    assert (o.seed, o.max_sweeps, o.max_levels, o.max_iters) == (1, 256, 64, 1000)


def test_option_defaults_and_struct_layout(tmp_path):
    """cd_opts_default fills the resolution 1 / 1 and the colour-class
    schedule, and the binding's structs have the header's layout (a C
    program compiled against include/cd.h reports sizes and offsets)."""
    o = cd.default_opts()
    assert (o.res_num, o.res_den, o.schedule, o.scratch_budget, o.int_path) == (1, 1, 0, 0, 0)
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "cd.h"\n'
        'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cd_opts), offsetof(cd_opts, bin_max),'
        ' offsetof(cd_opts, res_num), offsetof(cd_opts, res_den), offsetof(cd_opts, schedule),'
        ' sizeof(cd_stats), offsetof(cd_opts, scratch_budget)); return 0; }\n')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(cd.cd_opts), cd.cd_opts.bin_max.offset, cd.cd_opts.res_num.offset,
            cd.cd_opts.res_den.offset, cd.cd_opts.schedule.offset, ctypes.sizeof(cd.cd_stats),
            cd.cd_opts.scratch_budget.offset]
    assert got == want
