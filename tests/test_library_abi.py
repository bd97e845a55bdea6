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
